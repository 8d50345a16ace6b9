// ss_flow_cm.cu -- the flow pass kernels of the chiral magnet, instantiated in a
// translation unit of their own (see ss_flow_kernel.cuh).
#include "ss_flow_kernel.cuh"

namespace ss {
template cudaError_t launch_pass_theory<TH_CM>(const BatchLaunch& b, int pass, cudaStream_t s);
template void occupancy_theory<TH_CM>(int prec, int ts, bool one, int occ[3]);
}  // namespace ss
