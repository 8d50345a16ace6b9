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
  double coup[NCOUP]; // Couplings layout of ss_device.cuh, in FP64
  void* phi[2];    // ping-pong field buffers [C][ny][nx] (hi part when compensated)
  void* lo[2];     // compensated FP32: lo parts of phi[2] (else unused)
  void* v[2];      // ping-pong velocity buffers
  void* kv[2];     // RK stage accelerations k_v1, k_v2 (k_v3, k_v4 never leave registers)
  void* psi[2];    // chiral magnet with demagnetisation: magnetostatic potential planes
  DevState* st;
  FlowPartial* fpart;
  ObsPartial* opart;
  int flow_blocks; // grid of the flow kernels (grid-stride over tiles)
  int obs_blocks;
  int ntiles_x, ntiles_y;
};

// One relaxation problem as the flow kernels see it (device array, one entry per
// problem of a batch; a single-grid context is a batch of one). R is the working
// type of the batch.
template <typename R>
struct ProbDesc {
  int nx, ny;
  int ntx, ntiles;  // tiles along x, tiles in total
  int tile0;        // index of the problem's first tile in the batch
  int vec;          // FP32 rows start on 16-byte boundaries (nx % 4 == 0; every plane is 256-byte aligned)
  long long plane;  // nx * ny
  R* phi[2];        // ping-pong field buffers [C][ny][nx] (value part when compensated)
  R* lo[2];         // compensated FP32: remainder planes (else null)
  R* v[2];          // ping-pong velocities
  R* kv[2];         // k_v1, k_v2
  R* psi[2];        // chiral magnet with demagnetisation: magnetostatic potential of phi[0], phi[1]
  R dt;
  R tau;            // gradient descent: the step dtau of phi <- phi - dtau G
  R hx, hy;         // dx, dy (site positions of the BEC's trap and rotation terms)
  Spacing<R> h;
  Couplings<R> k;
  double area;      // dx dy
  DevState* st;     // the problem's flow record
  FlowPartial* part;  // ntiles reduction partials
};

// Minimisers (the SS_METHOD_* values of soliton.h).
enum { METHOD_ANF = 0, METHOD_GD = 1 };

// Pass numbers of launch_pass: the arrested flow's two passes and the descent pass.
enum { PASS_ANF1 = 1, PASS_ANF2 = 2, PASS_GD = 3 };

// A batch launch: the problem table, the tile -> problem map, the grid.
struct BatchLaunch {
  int theory;        // TH_AH / TH_CM (one theory per batch)
  int prec;          // PREC_*
  const void* probs; // ProbDesc<R>[n] on the device
  const int* tile_prob;  // [total_tiles] problem index of every tile
  int total_tiles;
  int flow_blocks[3];  // grid of pass 1 / pass 2 / the descent pass
  const void* one;     // host copy of the ProbDesc<R> of a single-problem batch, else NULL
  int ts;              // tile shape: 0 small, 1 large (flow_tile_dims)
  int nprob;           // problems of the batch
};

// One theory's flow-pass launcher and occupancy query (ss_flow_kernel.cuh), each
// instantiated in that theory's translation unit.
template <int TH>
cudaError_t launch_pass_theory(const BatchLaunch& b, int pass, cudaStream_t s);
template <int TH>
void occupancy_theory(int prec, int ts, bool one, int occ[3]);

// Tile shape of the flow kernels for a precision (sites per tile along x, y).
void flow_tile_dims(int prec, int ts, int* tx, int* ty);

// Pass 1 (RK stages 1-2, reductions, arrest and convergence decisions) or pass 2
// (RK stages 3-4, combination) of one flow step of every problem of a batch that
// is still running (Sec. 3.2), or pass 3: one gradient-descent step (force,
// reductions, decision and the new field in one launch). Each problem uses its own
// ping-pong parity.
cudaError_t launch_pass(const BatchLaunch& b, int pass, cudaStream_t s);
// Control kernels over the n flow records of a batch.
cudaError_t launch_reset_states(DevState* st, int n, cudaStream_t s);
cudaError_t launch_set_run_all(DevState* st, int n, double tol, long long max_steps, cudaStream_t s);
// Number of problems still running (not converged, finite, and under the step
// limit or with the field of its last step not yet evaluated).
cudaError_t launch_count_active(const DevState* st, int n, int* out, cudaStream_t s);

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

// Magnetostatic potential of one chiral-magnet problem (Eq. 6; ss_demag.cu): the sine
// transform solver of the 5-point Poisson problem with its transform plans and buffers.
struct DemagSolver;
// Returns 0, or -1 (device allocation failed) / -2 (transform plan failed).
int demag_create(DemagSolver** out, int nx, int ny, double dx, double dy, int prec);
void demag_destroy(DemagSolver* d);
// psi[cur] = L^{-1} rho(phi[cur] (+ lo[cur])), cur = st->steps & 1 read on the device.
cudaError_t demag_solve(DemagSolver* d, const DevState* st, void* const phi[2], void* const lo[2], void* const psi[2],
                        cudaStream_t s);

// The rotating BEC at a fixed atom number (ss_fixedn.cu): the refresh of a new field
// (scale to the atom number, velocity tangent to the constraint, the multiplier
// st->mu_held), three launches that skip unless the current field is new.
struct FixedNLaunch {
  int prec;                          // PREC_*
  void* phi[2]; void* lo[2]; void* v[2];
  int nx, ny;
  double dx, dy, g, omega, atoms;
  DevState* st;
  ObsPartial* part;                  // >= blocks entries
  int blocks;                        // grid cap
};
cudaError_t launch_fixed_n_refresh(const FixedNLaunch& L, cudaStream_t s);

// Record the calling thread's error message for ss_last_error().
void set_last_error(const std::string& msg);

// Validate the parameters of an SS_* theory (ss_set_theory's rules) and pack them as
// the kernels' couplings; *C = components per site. Returns SS_OK or SS_ERR_ARG
// (message set). ss_api.cu.
int pack_couplings(int theory, const double* params, int n_params, double k[NCOUP], int* C);

// Grid of each flow pass 1, 2, 3 (its occupancy x SMs, capped by the tile count).
void flow_grid(int theory, int prec, int ts, int total_tiles, bool one, int blocks[3]);
// Blocks of each pass 1, 2, 3 that fit on one SM.
void flow_occupancy(int theory, int prec, int ts, bool one, int occ[3]);
int obs_grid(int theory, int prec, int ntiles);

}  // namespace ss
