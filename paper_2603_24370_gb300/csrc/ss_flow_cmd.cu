// ss_flow_cmd.cu -- the flow pass kernels of the chiral magnet with demagnetisation,
// instantiated in a translation unit of their own (see ss_flow_kernel.cuh).
//
// Launch shape of the single-problem FP32 kernels: without a bound they hold 124 / 123
// / 108 registers (passes 1 / 2 / 3), one or two blocks per SM; bounds of 3 blocks per
// SM for all three passes with two staged sites in flight for pass 2 were the best of a
// sweep on the chiral magnet with demagnetisation workload of the benchmark: 0.622 +
// 0.596 -> 0.547 + 0.552 ms at 4096^2. With the packed stage pairs pass 1 spilled at 3
// blocks per SM; at 2, staging only the units its stencils read, it measured 0.522 ms
// against 0.556 ms (one GPU, both builds).
#define SS_MINB_THEORY 6  // TH_CMD
#define SS_MINB1 2
#define SS_VSKIP1 1
#define SS_MINB2 3
#define SS_MINB3 3
#define SS_LU2 2
// Pass 2 stages the tiles at the grid's edge through the scalar path: with the masked
// vector loop it ran 0.420 -> 0.424 ms at 4096^2, while pass 1 gained 0.520 -> 0.489 ms.
#define SS_VEDGE2 0
#include "ss_flow_kernel.cuh"

namespace ss {
static_assert(SS_MINB_THEORY == TH_CMD, "the launch bounds above are this theory's kernels'");
template cudaError_t launch_pass_theory<TH_CMD>(const BatchLaunch& b, int pass, cudaStream_t s);
template void occupancy_theory<TH_CMD>(int prec, int ts, bool one, int occ[3]);
}  // namespace ss
