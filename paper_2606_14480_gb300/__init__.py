"""GB300 (sm_103a) SciFi Seeding + VELO-SciFi Matching.

The compute path is the CUDA library libst.so (sources in csrc/, C ABI in
include/st.h); `st` is its ctypes binding.
"""

from . import build  # noqa: F401
