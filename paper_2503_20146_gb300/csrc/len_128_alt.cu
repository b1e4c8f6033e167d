// Column-pass shapes of transform length 128 built with the alternative radix
// schedule (sched_alt in fft.cuh), for the plan-time tuner to time beside the
// default schedule's, and the cluster-resident solver with that schedule.
#define PWF_SCHED_VARIANT 1
#include "persist.cuh"

namespace pwf {
void add_alt_column_shapes_128(LengthKernels& k) {
  sched1::add_schedule_shapes<128>(k);
  sched1::add_schedule_cluster<128>(k);  // and the cluster-resident solver
}
}  // namespace pwf
