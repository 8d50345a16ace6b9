// ss_flow_sid.cu -- the flow pass kernels of the s+id superconductor, instantiated in a
// translation unit of their own (see ss_flow_kernel.cuh).
//
// Launch shape of the single-problem FP32 kernels: without a bound they hold 177 / 176
// / 160 registers (passes 1 / 2 / 3), one or two blocks per SM; bounds of 2 blocks per
// SM for all three passes with one staged site in flight for passes 1 and 2 were the
// best of a sweep on the s+id superconductor workload of the benchmark: 0.350 + 0.381
// -> 0.273 + 0.227 ms at 2048^2.
#define SS_MINB_THEORY 5  // TH_SID
#define SS_MINB1 2
#define SS_MINB2 2
#define SS_MINB3 2
#define SS_LU1 1
#define SS_LU2 1
// Tiles at the grid's edge take the scalar staging: with the masked vector loop beside
// the plain one passes 1 and 2 ran 0.280 + 0.221 -> 0.297 + 0.226 ms at 2048^2.
#define SS_VEDGE 0
#include "ss_flow_kernel.cuh"

namespace ss {
static_assert(SS_MINB_THEORY == TH_SID, "the launch bounds above are this theory's kernels'");
template cudaError_t launch_pass_theory<TH_SID>(const BatchLaunch& b, int pass, cudaStream_t s);
template void occupancy_theory<TH_SID>(int prec, int ts, bool one, int occ[3]);
}  // namespace ss
