// Row/column pass kernels for transform length 512.
#include "persist.cuh"

namespace pwf {
const LengthKernels* length_kernels_512() {
  static const LengthKernels k = with_persist<512>(make_length_kernels<512>());
  return &k;
}
}  // namespace pwf
