// Row/column pass kernels for transform length 256.
#include "persist.cuh"

namespace pwf {
void add_alt_column_shapes_256(LengthKernels& k);

const LengthKernels* length_kernels_256() {
  static const LengthKernels k = [] {
    LengthKernels t = with_persist<256>(make_length_kernels<256>());
    add_alt_column_shapes_256(t);  // len_256_alt.cu
    return t;
  }();
  return &k;
}
}  // namespace pwf
