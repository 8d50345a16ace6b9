// ss_flow_bs.cu -- the flow pass kernels of the Baby Skyrme, instantiated in a
// translation unit of their own (see ss_flow_kernel.cuh).
//
// Launch shape of the single-problem FP32 kernels: without a bound they hold 137 / 128
// / 125 registers (passes 1 / 2 / 3), one or two blocks per SM; bounds of 3 blocks per
// SM for all three passes with one staged site in flight for passes 1 and 2 were the
// best of a sweep on the Baby Skyrme workload of the benchmark: 0.190 + 0.186 -> 0.154
// + 0.168 ms at 2048^2. With the packed stage pairs passes 1 and 2 spilled 644 / 292 B
// at 3 blocks per SM (0.180 + 0.148 ms); at 2 they spill 32 / 0 B: 0.137 + 0.145 ms
// (one GPU, both builds).
#define SS_MINB_THEORY 3  // TH_BS
#define SS_MINB1 2
#define SS_MINB2 2
#define SS_MINB3 3
#define SS_LU1 1
#define SS_LU2 1
// Pass 1 stages the tiles at the grid's edge through the scalar path: with the masked
// vector loop beside the plain one it ran 0.139 -> 0.143 ms at 2048^2 (pass 2 gained
// 0.141 -> 0.139 ms from it).
#define SS_VEDGE1 0
#include "ss_flow_kernel.cuh"

namespace ss {
static_assert(SS_MINB_THEORY == TH_BS, "the launch bounds above are this theory's kernels'");
template cudaError_t launch_pass_theory<TH_BS>(const BatchLaunch& b, int pass, cudaStream_t s);
template void occupancy_theory<TH_BS>(int prec, int ts, bool one, int occ[3]);
}  // namespace ss
