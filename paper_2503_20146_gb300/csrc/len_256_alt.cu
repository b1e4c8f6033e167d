// Column-pass shapes of transform length 256 built with the alternative radix
// schedule (sched_alt in fft.cuh), for the plan-time tuner to time beside the
// default schedule's, and the cluster-resident solver with that schedule.
#define PWF_SCHED_VARIANT 1
#include "persist.cuh"

namespace pwf {
void add_alt_column_shapes_256(LengthKernels& k) {
  sched1::add_schedule_shapes<256>(k);
  sched1::add_schedule_cluster<256>(k);  // and the cluster-resident solver
}
}  // namespace pwf
