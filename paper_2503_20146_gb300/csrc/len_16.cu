// Row/column pass kernels for transform length 16.
#include "passes.cuh"

namespace pwf {
const LengthKernels* length_kernels_16() {
  static const LengthKernels k = make_length_kernels<16>();
  return &k;
}
}  // namespace pwf
