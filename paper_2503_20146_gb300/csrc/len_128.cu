// Row/column pass kernels for transform length 128.
#include "passes.cuh"

namespace pwf {
const LengthKernels* length_kernels_128() {
  static const LengthKernels k = make_length_kernels<128>();
  return &k;
}
}  // namespace pwf
