// ss_flow_cm.cu -- the flow pass kernels of the chiral magnet, instantiated in a
// translation unit of their own (see ss_flow_kernel.cuh).
//
// Launch shape: the header's defaults (3 / 4 / 5 blocks per SM for passes 1 / 2 / 3)
// except pass 2, which loads each site's stored values for the RK4 combination
// before its stage forces and runs at 3 blocks per SM for the registers that takes:
// on the 4096^2 workload, in one call, pass 2 0.454 -> 0.442 ms (the step 0.894 ->
// 0.869 ms); at 4 blocks per SM the early loads spill.
//
// The descent pass unrolls its vector staging loop by three (0.264 -> 0.253 ms at
// 4096^2; passes 1 and 2 measured no gain from it).
//
// Pass 2 stages the tiles at the grid's edge through the scalar path: beside the
// masked vector loop its single-problem kernel spills (0 -> 56 bytes), and with
// that loop it ran 1.7% slower at 4096^2 (0.4286 -> 0.4360 ms).
#define SS_VEDGE2 0
#define SS_PF2 1
#define SS_MINB2 3
#define SS_VUNR3 3
#include "ss_flow_kernel.cuh"

namespace ss {
template cudaError_t launch_pass_theory<TH_CM>(const BatchLaunch& b, int pass, cudaStream_t s);
template void occupancy_theory<TH_CM>(int prec, int ts, bool one, int occ[3]);
}  // namespace ss
