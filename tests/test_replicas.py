"""The replica (multi-process) path on CPU: two gloo ranks, each running the
reconstruction of its own batch with no data exchange, then the host-side
max-over-ranks timing and the whole-job rate.  The per-rank work here is the
oracle, so the test needs no GPU; with GPUs each rank runs its own st_ctx in
exactly the same structure (bench.py)."""

import json
import os
import socket
import time

import pytest

from paper_2606_14480_gb300 import replicas

WS = 2


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _seed_lists(batch, cfg):
    import oracle
    out = []
    for e in range(batch.n_events):
        x, zone = batch.hits_of(e)
        s = oracle.seeding_event(cfg, x, zone)["seeds"]
        out.append(sorted(tuple(int(v) for v in h) for h in s["hits"]))
    return out


def _worker(rank, ws, port, out_dir, job_events):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import oracle
    from synth import make_workload
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, local = replicas.dist_env()
        assert (w, r, local) == (ws, rank, rank)
        batch = make_workload("tiny", n_events=4, seed=replicas.replica_seed(1001, r))
        cfg = oracle.default_config()
        replicas.barrier()
        t0 = time.perf_counter()
        seeds = _seed_lists(batch, cfg)
        if r == 1:
            time.sleep(0.3)  # the slower rank sets the job time
        dt = time.perf_counter() - t0
        tmax = replicas.max_over_ranks(dt)
        rate = replicas.job_rate(batch.n_events, w, tmax)
        lo, hi = replicas.shard(job_events, w, r)
        n_total = replicas.max_over_ranks(hi)  # the last shard ends at the job size
        replicas.barrier()
        with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
            json.dump({"dt": dt, "tmax": tmax, "rate": rate, "n": batch.n_events, "seeds": seeds,
                       "shard": [lo, hi], "n_total": n_total}, f)
    finally:
        dist.destroy_process_group()


def test_shard_covers_the_job_once():
    for n in (0, 1, 7, 1000, 1001):
        for ws in (1, 2, 3, 8):
            got = [replicas.shard(n, ws, r) for r in range(ws)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            sizes = [h - l for l, h in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.shard(10, 2, 2)


def test_no_process_group_is_identity():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_rate(1000, 1, 0.5) == 2000.0
    replicas.barrier()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    from synth import make_workload

    import oracle
    port = _free_port()
    mp.start_processes(_worker, args=(WS, port, str(tmp_path), 1001), nprocs=WS, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(WS)]
    # host-side reduction: both ranks see the slowest rank's time
    tmax = max(r["dt"] for r in res)
    for r in res:
        assert r["tmax"] == pytest.approx(tmax, rel=1e-12)
        assert r["rate"] == pytest.approx(WS * r["n"] / tmax, rel=1e-12)
        assert r["n_total"] == 1001
    assert res[1]["dt"] > 0.3
    assert [tuple(r["shard"]) for r in res] == [(0, 501), (501, 1001)]
    # each replica computed its own events, exactly as a lone process does
    cfg = oracle.default_config()
    for rank, r in enumerate(res):
        b = make_workload("tiny", n_events=4, seed=replicas.replica_seed(1001, rank))
        want = _seed_lists(b, cfg)
        assert [[list(h) for h in ev] for ev in want] == r["seeds"]
    assert res[0]["seeds"] != res[1]["seeds"]
    assert sum(len(ev) for ev in res[0]["seeds"]) > 0
