// ss_flow_bs.cu -- the flow pass kernels of the Baby Skyrme, instantiated in a
// translation unit of their own (see ss_flow_kernel.cuh).
#include "ss_flow_kernel.cuh"

namespace ss {
template cudaError_t launch_pass_theory<TH_BS>(const BatchLaunch& b, int pass, cudaStream_t s);
template void occupancy_theory<TH_BS>(int prec, int ts, bool one, int occ[3]);
}  // namespace ss
