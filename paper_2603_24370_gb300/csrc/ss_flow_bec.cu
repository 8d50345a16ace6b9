// ss_flow_bec.cu -- the flow pass kernels of the rotating BEC, instantiated in a
// translation unit of their own (see ss_flow_kernel.cuh).
#include "ss_flow_kernel.cuh"

namespace ss {
template cudaError_t launch_pass_theory<TH_BEC>(const BatchLaunch& b, int pass, cudaStream_t s);
template void occupancy_theory<TH_BEC>(int prec, int ts, bool one, int occ[3]);
}  // namespace ss
