// ss_flow_ah.cu -- the flow pass kernels of the Abelian Higgs, instantiated in a
// translation unit of their own (see ss_flow_kernel.cuh).
//
// Launch shape of the FP32 kernels: without a bound they hold 146 / 128 / 114
// registers (passes 1 / 2 / 3), one or two blocks per SM. Bounds of 2 / 3 / 3 blocks
// per SM with one staged site in flight for pass 2 were the best of a sweep on a
// 64-problem batch of the batched set: 0.515 -> 0.404 ms per step. Batched pass 2,
// whose tile search and per-tile descriptor hold more registers, spilled 600 B at 3
// blocks per SM; at 2 it spills 52 B and the 256-problem set relaxes in 8.5 s instead
// of 9.8 s. The single-problem pass 2, packed stage pairs and all, spilled 148 B at 3;
// at 2 blocks per SM it takes 0.155 ms instead of 0.169 ms at 2048^2 (one GPU).
#define SS_MINB_THEORY 1  // TH_AH
#define SS_MINB_BATCH 1
#define SS_MINB1 2
#define SS_MINB2 2
#define SS_MINB3 3
#define SS_LU2 1
#include "ss_flow_kernel.cuh"

namespace ss {
static_assert(SS_MINB_THEORY == TH_AH, "the launch bounds above are the Abelian Higgs kernels'");
template cudaError_t launch_pass_theory<TH_AH>(const BatchLaunch& b, int pass, cudaStream_t s);
template void occupancy_theory<TH_AH>(int prec, int ts, bool one, int occ[3]);
}  // namespace ss
