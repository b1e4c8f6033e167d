// Row/column pass kernels for transform length 64.
#include "passes.cuh"

namespace pwf {
const LengthKernels* length_kernels_64() {
  static const LengthKernels k = make_length_kernels<64>();
  return &k;
}
}  // namespace pwf
