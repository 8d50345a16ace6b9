// ss_flow_cmd.cu -- the flow pass kernels of the chiral magnet with demagnetisation,
// instantiated in a translation unit of their own (see ss_flow_kernel.cuh).
#include "ss_flow_kernel.cuh"

namespace ss {
template cudaError_t launch_pass_theory<TH_CMD>(const BatchLaunch& b, int pass, cudaStream_t s);
template void occupancy_theory<TH_CMD>(int prec, int ts, bool one, int occ[3]);
}  // namespace ss
