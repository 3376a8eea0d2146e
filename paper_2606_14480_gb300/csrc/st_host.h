// st_host.h -- host-side helpers shared by the library's translation units.
#pragma once

#include <string>

#include "st.h"
#include "st_device.cuh"

namespace st {
}

// Derive the device constants from a configuration (validates it; false and a
// message on an invalid configuration).
bool derive_params(const st_config& c, st::DevParams& P, std::string& err);
