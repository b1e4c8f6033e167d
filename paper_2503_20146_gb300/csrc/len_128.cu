// Row/column pass kernels for transform length 128.
#include "persist.cuh"

namespace pwf {
void add_alt_column_shapes_128(LengthKernels& k);

const LengthKernels* length_kernels_128() {
  static const LengthKernels k = [] {
    LengthKernels t = with_persist<128>(make_length_kernels<128>());
    add_alt_column_shapes_128(t);  // len_128_alt.cu
    return t;
  }();
  return &k;
}
}  // namespace pwf
