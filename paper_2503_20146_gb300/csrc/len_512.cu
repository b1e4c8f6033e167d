// Row/column pass kernels for transform length 512.
#include "persist.cuh"

namespace pwf {
void add_alt_column_shapes_512(LengthKernels& k);

const LengthKernels* length_kernels_512() {
  static const LengthKernels k = [] {
    LengthKernels t = with_persist<512>(make_length_kernels<512>());
    add_alt_column_shapes_512(t);  // len_512_alt.cu
    return t;
  }();
  return &k;
}
}  // namespace pwf
