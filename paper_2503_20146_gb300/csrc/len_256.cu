// Row/column pass kernels for transform length 256.
#include "persist.cuh"

namespace pwf {
const LengthKernels* length_kernels_256() {
  static const LengthKernels k = with_persist<256>(make_length_kernels<256>());
  return &k;
}
}  // namespace pwf
