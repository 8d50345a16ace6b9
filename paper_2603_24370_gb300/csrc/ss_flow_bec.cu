// ss_flow_bec.cu -- the flow pass kernels of the rotating BEC, instantiated in a
// translation unit of their own (see ss_flow_kernel.cuh).
//
// Launch shape of the single-problem FP32 kernels: without a bound they hold 99 / 96 /
// 90 registers (passes 1 / 2 / 3), one or two blocks per SM; bounds of 3 blocks per SM
// for all three passes were the best of a sweep on the rotating BEC workload of the
// benchmark: 0.111 + 0.099 -> 0.094 + 0.087 ms at 2048^2.
#define SS_MINB_THEORY 4  // TH_BEC
#define SS_MINB1 3
#define SS_MINB2 3
#define SS_MINB3 3
#include "ss_flow_kernel.cuh"

namespace ss {
static_assert(SS_MINB_THEORY == TH_BEC, "the launch bounds above are this theory's kernels'");
template cudaError_t launch_pass_theory<TH_BEC>(const BatchLaunch& b, int pass, cudaStream_t s);
template void occupancy_theory<TH_BEC>(int prec, int ts, bool one, int occ[3]);
}  // namespace ss
