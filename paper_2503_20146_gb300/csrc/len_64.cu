// Row/column pass kernels for transform length 64.
#include "persist.cuh"

namespace pwf {
const LengthKernels* length_kernels_64() {
  static const LengthKernels k = with_persist<64>(make_length_kernels<64>());
  return &k;
}
}  // namespace pwf
