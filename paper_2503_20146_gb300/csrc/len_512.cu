// Row/column pass kernels for transform length 512.
#include "passes.cuh"

namespace pwf {
const LengthKernels* length_kernels_512() {
  static const LengthKernels k = make_length_kernels<512>();
  return &k;
}
}  // namespace pwf
