// Host-side table builders shared by the translation units of the library.
#pragma once
#include <cuda_runtime.h>

#include <vector>

namespace pwf {
// Twiddles of the length-n transform in direction D (FWD or INV) in the layout
// read by fft_stages; false if the schedule does not fit the table.
bool host_twiddles(int n, int D, std::vector<float2>& tab);
}  // namespace pwf
