// Row/column pass kernels for transform length 1024.
#include "passes.cuh"

namespace pwf {
void add_alt_column_shapes_1024(LengthKernels& k);

const LengthKernels* length_kernels_1024() {
  static const LengthKernels k = [] {
    LengthKernels t = make_length_kernels<1024>();
    add_alt_column_shapes_1024(t);  // len_1024_alt.cu
    return t;
  }();
  return &k;
}
}  // namespace pwf
