// Row/column pass kernels for transform length 32.
#include "passes.cuh"

namespace pwf {
const LengthKernels* length_kernels_32() {
  static const LengthKernels k = make_length_kernels<32>();
  return &k;
}
}  // namespace pwf
