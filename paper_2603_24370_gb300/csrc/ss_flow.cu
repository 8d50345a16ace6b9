// ss_flow.cu -- host side of the flow passes (arxiv 2603.24370, Sec. 3.2): the
// per-theory dispatch of the pass launches and occupancy queries, the pass grids,
// and the control kernels over the per-problem flow records. The pass kernels
// themselves are in ss_flow_kernel.cuh, instantiated per theory in ss_flow_ah.cu,
// ss_flow_cm.cu, ss_flow_bs.cu, ss_flow_bec.cu, ss_flow_sid.cu and ss_flow_cmd.cu.
#include "ss_internal.h"

namespace ss {

void flow_tile_dims(int prec, int ts, int* tx, int* ty) {
  *tx = 32;
  *ty = BY * ((prec == PREC_F64 ? 1 : 2) << (ts ? 1 : 0));
}

// ------------------------------------------------------------------ control kernels
__global__ void k_reset_states(DevState* st, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    DevState* s = st + i;
    s->E_last = __longlong_as_double(0x7ff0000000000000LL);  // +inf: no arrest on the first step
    s->E_cur = 0.0;
    s->dE = 0.0;
    s->gmax = 0.0;
    s->tol = -1.0;
    s->steps = 0;
    s->arrests = 0;
    s->head_step = -1;
    s->step_limit = 0;
    s->arrest = 0;
    s->converged = 0;
    s->nonfinite = 0;
    s->ticket = 0;
    s->obs_ticket = 0;
    s->mu_held = 0.0;
    s->fn_scale = 1.0;
    s->fn_alpha = 0.0;
    s->fn_step = -1;
    s->fn_pending = 0;
    s->fn_ticket = 0;
  }
}

// Start of a run: threshold, step budget, and the convergence verdict of an
// already-evaluated head under the new threshold.
__global__ void k_set_run_all(DevState* st, int n, double tol, long long max_steps) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    DevState* s = st + i;
    s->tol = tol;
    s->step_limit = s->steps + max_steps;
    s->converged = (s->head_step == s->steps && s->gmax < tol) ? 1 : 0;
  }
}

__global__ void k_count_active(const DevState* st, int n, int* out) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int mine = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const DevState* s = st + i;
    // running: not stopped, and either budget left or the last field not yet
    // evaluated (a descent pass evaluates the field its last step produced)
    mine += !(s->converged || s->nonfinite || (s->steps >= s->step_limit && s->head_step == s->steps));
  }
  atomicAdd(&cnt, mine);
  __syncthreads();
  if (threadIdx.x == 0) *out = cnt;
}

template <typename R>
__global__ void k_scaled_copy(R* __restrict__ out, const R* __restrict__ in, size_t n, R scale) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = scale * in[i];
}

cudaError_t launch_pass(const BatchLaunch& b, int pass, cudaStream_t s) {
  if (b.theory == TH_AH) return launch_pass_theory<TH_AH>(b, pass, s);
  if (b.theory == TH_CM) return launch_pass_theory<TH_CM>(b, pass, s);
  if (b.theory == TH_BS) return launch_pass_theory<TH_BS>(b, pass, s);
  if (b.theory == TH_SID) return launch_pass_theory<TH_SID>(b, pass, s);
  if (b.theory == TH_CMD) return launch_pass_theory<TH_CMD>(b, pass, s);
  return launch_pass_theory<TH_BEC>(b, pass, s);
}

cudaError_t launch_reset_states(DevState* st, int n, cudaStream_t s) {
  k_reset_states<<<(n + 255) / 256, 256, 0, s>>>(st, n);
  return cudaGetLastError();
}

cudaError_t launch_set_run_all(DevState* st, int n, double tol, long long max_steps, cudaStream_t s) {
  k_set_run_all<<<(n + 255) / 256, 256, 0, s>>>(st, n, tol, max_steps);
  return cudaGetLastError();
}

cudaError_t launch_count_active(const DevState* st, int n, int* out, cudaStream_t s) {
  k_count_active<<<1, 256, 0, s>>>(st, n, out);
  return cudaGetLastError();
}

cudaError_t launch_scaled_copy(const LaunchCtx& c, void* out, const void* in, double scale, cudaStream_t s) {
  const int C = c.theory == TH_AH ? 4 : (c.theory == TH_BEC ? 2 : (c.theory == TH_SID ? 6 : 3));
  const size_t n = (size_t)C * c.plane;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = (int)((n + 255) / 256 < (size_t)nsm * 8 ? (n + 255) / 256 : (size_t)nsm * 8);
  if (c.prec != PREC_F64) k_scaled_copy<float><<<blocks, 256, 0, s>>>((float*)out, (const float*)in, n, (float)scale);
  else k_scaled_copy<double><<<blocks, 256, 0, s>>>((double*)out, (const double*)in, n, scale);
  return cudaGetLastError();
}

void flow_occupancy(int theory, int prec, int ts, bool one, int occ[3]) {
  occ[0] = occ[1] = occ[2] = 1;
  if (theory == TH_AH) occupancy_theory<TH_AH>(prec, ts, one, occ);
  else if (theory == TH_CM) occupancy_theory<TH_CM>(prec, ts, one, occ);
  else if (theory == TH_BS) occupancy_theory<TH_BS>(prec, ts, one, occ);
  else if (theory == TH_SID) occupancy_theory<TH_SID>(prec, ts, one, occ);
  else if (theory == TH_CMD) occupancy_theory<TH_CMD>(prec, ts, one, occ);
  else occupancy_theory<TH_BEC>(prec, ts, one, occ);
  for (int i = 0; i < 3; ++i)
    if (occ[i] < 1) occ[i] = 1;
}

// Default grid of each pass: its occupancy x SMs, capped by the tile count.
void flow_grid(int theory, int prec, int ts, int total_tiles, bool one, int blocks[3]) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int occ[3];
  flow_occupancy(theory, prec, ts, one, occ);
  for (int i = 0; i < 3; ++i) {
    const int g = nsm * occ[i];
    blocks[i] = total_tiles < g ? total_tiles : g;
  }
}

}  // namespace ss
