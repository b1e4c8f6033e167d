// Row/column pass kernels for transform length 768.
#include "passes.cuh"

namespace pwf {
void add_alt_column_shapes_768(LengthKernels& k);

const LengthKernels* length_kernels_768() {
  static const LengthKernels k = [] {
    LengthKernels t = make_length_kernels<768>();
    add_alt_column_shapes_768(t);  // len_768_alt.cu
    return t;
  }();
  return &k;
}
}  // namespace pwf
