// Row/column pass kernels for transform length 1536.
#include "passes.cuh"

namespace pwf {
void add_alt_column_shapes_1536(LengthKernels& k);

const LengthKernels* length_kernels_1536() {
  static const LengthKernels k = [] {
    LengthKernels t = make_length_kernels<1536>();
    add_alt_column_shapes_1536(t);  // len_1536_alt.cu
    return t;
  }();
  return &k;
}
}  // namespace pwf
