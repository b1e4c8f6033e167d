// Row/column pass kernels for transform length 2048.
#include "passes.cuh"

namespace pwf {
const LengthKernels* length_kernels_2048() {
  static const LengthKernels k = make_length_kernels<2048>();
  return &k;
}
}  // namespace pwf
