// Row/column pass kernels for transform length 768.
#include "passes.cuh"

namespace pwf {
const LengthKernels* length_kernels_768() {
  static const LengthKernels k = make_length_kernels<768>();
  return &k;
}
}  // namespace pwf
