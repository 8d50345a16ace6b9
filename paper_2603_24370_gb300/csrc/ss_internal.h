// ss_internal.h -- host-side interface between the C-ABI runtime (ss_api.cu) and
// the kernel translation units (ss_flow.cu, ss_observe.cu). Not installed.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <string>

#include "ss_device.cuh"

namespace ss {

// Precision codes (the SS_FP* values of soliton.h): compensated FP32 fields (hi + lo
// planes), all-FP64, single-plane FP32.
enum { PREC_F32C = 1, PREC_F64 = 2, PREC_F32 = 3 };

// Everything a launch needs about one context, prepared by the runtime.
struct LaunchCtx {
  int theory;      // TH_AH / TH_CM
  int prec;        // 1 = FP32, 2 = FP64
  int nx, ny;
  size_t plane;    // nx * ny
  double dx, dy, dt;
  double coup[10]; // Couplings layout of ss_device.cuh, in FP64
  void* phi[2];    // ping-pong field buffers [C][ny][nx] (hi part when compensated)
  void* lo[2];     // compensated FP32: lo parts of phi[2] (else unused)
  void* v[2];      // ping-pong velocity buffers
  void* kv[2];     // RK stage accelerations k_v1, k_v2 (k_v3, k_v4 never leave registers)
  DevState* st;
  FlowPartial* fpart;
  ObsPartial* opart;
  int flow_blocks; // grid of the flow kernels (grid-stride over tiles)
  int obs_blocks;
  int ntiles_x, ntiles_y;
};

// Pass 1 (RK stages 1-2 + reductions + arrest decision) or pass 2 (stages 3-4 +
// combination) of the RK4 step whose current field is phi[cur] (Sec. 3.2).
cudaError_t launch_pass(const LaunchCtx& c, int pass, int cur, cudaStream_t s);
// Control kernels: reset the flow record for new fields; start a run with a
// convergence threshold (tol < 0: none) and a budget of max_steps further steps.
cudaError_t launch_reset_state(const LaunchCtx& c, cudaStream_t s);
cudaError_t launch_set_run(const LaunchCtx& c, double tol, long long max_steps, cudaStream_t s);
// out = scale * in over the C planes of a context.
cudaError_t launch_scaled_copy(const LaunchCtx& c, void* out, const void* in, double scale, cudaStream_t s);
// Observables of phi[cur] in FP64 (energy, charge, flux, residual, |n|-1).
cudaError_t launch_observables(const LaunchCtx& c, int cur, cudaStream_t s);
// Ansatz of n solitons (device array of 5 doubles each) into both field buffers.
cudaError_t launch_ansatz(const LaunchCtx& c, const double* d_sol, int n, cudaStream_t s);

// Record the calling thread's error message for ss_last_error().
void set_last_error(const std::string& msg);

// Flow-kernel grid size for a context (occupancy x SMs, capped by the tile count).
int flow_grid(int theory, int prec, int nx, int ny);
int obs_grid(int theory, int prec, int ntiles);

}  // namespace ss
