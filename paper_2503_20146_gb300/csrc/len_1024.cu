// Row/column pass kernels for transform length 1024.
#include "passes.cuh"

namespace pwf {
const LengthKernels* length_kernels_1024() {
  static const LengthKernels k = make_length_kernels<1024>();
  return &k;
}
}  // namespace pwf
