// Row/column pass kernels for transform length 128.
#include "persist.cuh"

namespace pwf {
const LengthKernels* length_kernels_128() {
  static const LengthKernels k = with_persist<128>(make_length_kernels<128>());
  return &k;
}
}  // namespace pwf
