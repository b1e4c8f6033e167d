// Row/column pass kernels for transform length 96.
#include "passes.cuh"

namespace pwf {
const LengthKernels* length_kernels_96() {
  static const LengthKernels k = make_length_kernels<96>();
  return &k;
}
}  // namespace pwf
