// Column-pass shapes of transform length 1536 built with the alternative radix
// schedule (sched_alt in fft.cuh), for the plan-time tuner to time beside the
// default schedule's.
#define PWF_SCHED_VARIANT 1
#include "passes.cuh"

namespace pwf {
void add_alt_column_shapes_1536(LengthKernels& k) { sched1::add_schedule_shapes<1536>(k); }
}  // namespace pwf
