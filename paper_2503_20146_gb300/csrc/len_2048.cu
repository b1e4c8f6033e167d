// Row/column pass kernels for transform length 2048.
#include "passes.cuh"

namespace pwf {
void add_alt_column_shapes_2048(LengthKernels& k);

const LengthKernels* length_kernels_2048() {
  static const LengthKernels k = [] {
    LengthKernels t = make_length_kernels<2048>();
    add_alt_column_shapes_2048(t);  // len_2048_alt.cu
    return t;
  }();
  return &k;
}
}  // namespace pwf
