// Row/column pass kernels for transform length 1536.
#include "passes.cuh"

namespace pwf {
const LengthKernels* length_kernels_1536() {
  static const LengthKernels k = make_length_kernels<1536>();
  return &k;
}
}  // namespace pwf
