// Internal interface of the tile-width table (tune.cu).
#pragma once

#include <string>

#include "css_common.cuh"

namespace css {

// Name of the current CUDA device (cached per device).
std::string current_device_name();
// Tuned tile width for the current device and this shape, or 0 if none.
int tuned_tile(int dt, int64_t m, int64_t n);
// Tuned value of a knob (0 tile width, 1 split share, 2 pivot cost), or -1.
int tuned_knob(int dt, int64_t m, int64_t n, int knob);

}  // namespace css
