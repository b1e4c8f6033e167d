// Row/column pass kernels for transform length 256.
#include "passes.cuh"

namespace pwf {
const LengthKernels* length_kernels_256() {
  static const LengthKernels k = make_length_kernels<256>();
  return &k;
}
}  // namespace pwf
