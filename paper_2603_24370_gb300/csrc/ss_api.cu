// ss_api.cu -- host runtime and C-ABI of the soliton relaxation library
// (declarations and argument contracts in include/soliton.h).
//
// The runtime follows the paper's workflow (Sec. 4.1): select a theory and its
// parameters, allocate the device buffer set, initialise the field from an ansatz,
// then minimise. The buffer set is reduced to what the fused stage kernels need
// (Sec. 3.1 lists fields, velocity, gradient, derivative work arrays and RK stages):
//   phi[2], v[2]   ping-pong field and velocity (RK4 reads phi^n around each site
//                  while writing phi^{n+1}; phi^{n-1} feeds the arrest test),
//   kv[2]          stage accelerations k_v1, k_v2 (k_v3, k_v4 stay in registers),
//   lo[2]          compensated FP32 only: the lo parts of phi[2],
// plus one device status record and per-block reduction partials. Derivatives never
// touch memory. Steps are enqueued as CUDA graphs of K_CHUNK steps; convergence,
// arrest and the step budget are decided on the device, so the host only polls a
// small status record once per chunk (one chunk ahead).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "soliton.h"
#include "ss_internal.h"

using namespace ss;

namespace {

constexpr int K_CHUNK = 32;  // steps per captured graph (even: parity returns)
constexpr int NBUF = 6;      // phi[2], v[2], kv[2] (+ lo[2] when compensated)

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

}  // namespace

void ss::set_last_error(const std::string& msg) { g_err = msg; }

#define SS_CK(call)                                                                            \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail(SS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct ss_ctx {
  int nx = 0, ny = 0;
  double dx = 0, dy = 0, dt = 0;
  int prec = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int theory = 0;
  int C = 0;
  size_t elem = 0;
  bool fields_set = false;
  int cur = 0;                    // phi[cur] holds the current field
  void* base = nullptr;           // one device allocation for every plane
  DevState* h_st[2] = {nullptr, nullptr};  // pinned copies of the status record
  cudaEvent_t ev[2] = {nullptr, nullptr};
  double* d_sol = nullptr;
  int sol_cap = 0;
  cudaGraphExec_t chunk[2] = {nullptr, nullptr};  // K_CHUNK steps from parity 0 / 1
  LaunchCtx L{};
};

namespace {

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

void free_buffers(ss_ctx* c) {
  for (int p = 0; p < 2; ++p)
    if (c->chunk[p]) { cudaGraphExecDestroy(c->chunk[p]); c->chunk[p] = nullptr; }
  if (c->base) { cudaFree(c->base); c->base = nullptr; }
  c->fields_set = false;
}

// Parity bookkeeping: the device counts steps; the field sits in phi[steps & 1]
// relative to the parity the fields were set at (always 0).
int refresh(ss_ctx* c, DevState* h) {
  c->cur = (int)(h->steps & 1);
  return SS_OK;
}

int read_state(ss_ctx* c, DevState* out) {
  SS_CK(cudaMemcpyAsync(c->h_st[0], c->L.st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
  SS_CK(cudaStreamSynchronize(c->stream));
  *out = *c->h_st[0];
  refresh(c, out);
  return SS_OK;
}

// One step from parity p: pass 2 (stages 3-4, new field), then pass 1 (stages 1-2,
// reductions, arrest decision) of the new field, which is the next step's head.
int enqueue_step(ss_ctx* c, int p) {
  SS_CK(launch_pass(c->L, 2, p, c->stream));
  SS_CK(launch_pass(c->L, 1, p ^ 1, c->stream));
  return SS_OK;
}

int ensure_chunk(ss_ctx* c, int p) {
  if (c->chunk[p]) return SS_OK;
  cudaGraph_t g = nullptr;
  SS_CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  int rc = SS_OK;
  for (int k = 0; k < K_CHUNK && rc == SS_OK; ++k) rc = enqueue_step(c, p ^ (k & 1));
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (rc != SS_OK) { if (g) cudaGraphDestroy(g); return rc; }
  if (e != cudaSuccess) return fail(SS_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&c->chunk[p], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(SS_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  return SS_OK;
}

int check_ready(ss_ctx* c) {
  if (!c) return fail(SS_ERR_ARG, "null context");
  if (!c->theory) return fail(SS_ERR_STATE, "ss_set_theory has not been called");
  if (!c->fields_set) return fail(SS_ERR_STATE, "fields not set (ss_init_ansatz / ss_set_fields)");
  return SS_OK;
}

int new_fields(ss_ctx* c) {
  const size_t bytes = (size_t)c->C * c->L.plane * c->elem;
  SS_CK(cudaMemsetAsync(c->L.v[0], 0, bytes, c->stream));
  SS_CK(cudaMemsetAsync(c->L.v[1], 0, bytes, c->stream));
  if (c->prec == SS_FP32) {  // compensated: the given field is exact, lo = 0
    SS_CK(cudaMemsetAsync(c->L.lo[0], 0, bytes, c->stream));
    SS_CK(cudaMemsetAsync(c->L.lo[1], 0, bytes, c->stream));
  }
  SS_CK(launch_reset_state(c->L, c->stream));
  c->cur = 0;
  c->fields_set = true;
  return SS_OK;
}

void fill_status(const DevState& h, ss_status* out) {
  if (!out) return;
  out->energy = h.E_cur;
  out->grad_max = h.gmax;
  out->steps = h.steps;
  out->arrests = h.arrests;
  out->converged = h.converged;
  out->arrested = h.arrest;
  out->energy_change = h.dE;
}

// Run up to max_steps steps with threshold tol (< 0: none). Chunk i is enqueued
// before the status of chunk i-1 is checked, so the GPU never waits for the host;
// once the device has stopped (converged, non-finite, step budget spent) the rest
// of an enqueued chunk is a row of no-op launches.
int run(ss_ctx* c, double tol, long long max_steps, DevState* fin) {
  const int p0 = c->cur;
  SS_CK(launch_set_run(c->L, tol, max_steps, c->stream));
  SS_CK(launch_pass(c->L, 1, p0, c->stream));  // head of the current field (no-op if done)
  const long long nchunks = (max_steps + K_CHUNK - 1) / K_CHUNK;
  if (nchunks > 0) {
    int rc = ensure_chunk(c, p0);
    if (rc != SS_OK) return rc;
  }
  int prev = -1;
  for (long long i = 0; i < nchunks; ++i) {
    const int slot = (int)(i & 1);
    SS_CK(cudaGraphLaunch(c->chunk[p0], c->stream));
    SS_CK(cudaMemcpyAsync(c->h_st[slot], c->L.st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    SS_CK(cudaEventRecord(c->ev[slot], c->stream));
    if (prev >= 0) {
      SS_CK(cudaEventSynchronize(c->ev[prev]));
      const DevState* h = c->h_st[prev];
      if (h->converged || h->nonfinite || h->steps >= h->step_limit) break;
    }
    prev = slot;
  }
  return read_state(c, fin);
}

}  // namespace

extern "C" {

const char* ss_last_error(void) { return g_err.c_str(); }

int ss_version(void) { return 3; }

int ss_create_grid(ss_ctx** out, int nx, int ny, double dx, double dy, int precision, void* cuda_stream) {
  if (!out) return fail(SS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (nx < 5 || ny < 5) return fail(SS_ERR_ARG, "nx and ny must be >= 5 (halo of width 2 on each side)");
  if ((long long)nx * ny > (1LL << 31)) return fail(SS_ERR_ARG, "grid too large (nx * ny > 2^31)");
  if (!(dx > 0.0) || !(dy > 0.0) || !std::isfinite(dx) || !std::isfinite(dy))
    return fail(SS_ERR_ARG, "dx and dy must be positive and finite");
  if (precision != SS_FP32 && precision != SS_FP64 && precision != SS_FP32_PLAIN)
    return fail(SS_ERR_ARG, "precision must be SS_FP32, SS_FP64 or SS_FP32_PLAIN");
  int dev = 0;
  SS_CK(cudaGetDevice(&dev));
  ss_ctx* c = new (std::nothrow) ss_ctx();
  if (!c) return fail(SS_ERR_NOMEM, "host allocation failed");
  c->nx = nx;
  c->ny = ny;
  c->dx = dx;
  c->dy = dy;
  c->dt = 0.5 * (dx < dy ? dx : dy);  // Sec. 3.1: C = dt / dx = 0.5
  c->prec = precision;
  c->elem = precision == SS_FP64 ? 8 : 4;
  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    c->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {  // graphs cannot be captured on the legacy stream: own a blocking stream
    e = cudaStreamCreate(&c->stream);
    c->own_stream = true;
  }
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaMallocHost(&c->h_st[i], sizeof(DevState));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    ss_destroy(c);
    return fail(SS_ERR_CUDA, std::string("ss_create_grid: ") + cudaGetErrorString(e));
  }
  c->L.nx = nx;
  c->L.ny = ny;
  c->L.plane = (size_t)nx * ny;
  c->L.dx = dx;
  c->L.dy = dy;
  c->L.dt = c->dt;
  c->L.prec = precision;
  c->L.ntiles_x = (nx + TX - 1) / TX;
  c->L.ntiles_y = (ny + TY - 1) / TY;
  *out = c;
  return SS_OK;
}

int ss_set_theory(ss_ctx* c, int theory, const double* params, int n_params) {
  if (!c) return fail(SS_ERR_ARG, "null context");
  if (!params && n_params > 0) return fail(SS_ERR_ARG, "params is NULL");
  double k[10] = {0};
  int C = 0;
  if (theory == SS_ABELIAN_HIGGS) {
    if (n_params < 1 || n_params > 2) return fail(SS_ERR_ARG, "Abelian Higgs takes {lambda[, u]}");
    const double lam = params[0], u = n_params > 1 ? params[1] : 1.0;
    if (!std::isfinite(lam) || !std::isfinite(u) || lam < 0.0) return fail(SS_ERR_ARG, "lambda must be finite and >= 0");
    k[0] = lam;
    k[1] = u * u;
    C = 4;
  } else if (theory == SS_CHIRAL_MAGNET) {
    if (n_params < 4 || n_params > 5) return fail(SS_ERR_ARG, "chiral magnet takes {J, D, K, h[, dmi_type]}");
    for (int i = 0; i < n_params; ++i)
      if (!std::isfinite(params[i])) return fail(SS_ERR_ARG, "chiral-magnet parameters must be finite");
    if (!(params[0] > 0.0)) return fail(SS_ERR_ARG, "J must be > 0");
    const int type = n_params > 4 ? (int)params[4] : 0;
    if (type < 0 || type > 2 || (n_params > 4 && params[4] != (double)type))
      return fail(SS_ERR_ARG, "dmi_type must be 0 (interfacial), 1 (bulk) or 2 (D_2d)");
    k[0] = params[0];
    k[1] = params[1];
    k[2] = params[2];
    k[3] = params[3];
    // DMI vectors d_1 (k[4..6]) and d_2 (k[7..9]) of Eq. 5
    if (type == 0) { k[5] = 1.0; k[7] = -1.0; }      // d_i = e_3 x e_i
    else if (type == 1) { k[4] = 1.0; k[8] = 1.0; }  // d_i = e_i
    else { k[4] = 1.0; k[8] = -1.0; }                // d_1 = e_1, d_2 = -e_2
    C = 3;
  } else {
    return fail(SS_ERR_ARG, "unknown theory");
  }
  if (c->theory != theory || c->C != C || !c->base) {
    free_buffers(c);
    const size_t pb = align256((size_t)C * c->L.plane * c->elem);
    const int ntiles = c->L.ntiles_x * c->L.ntiles_y;
    const int fb = flow_grid(theory == SS_ABELIAN_HIGGS ? TH_AH : TH_CM, c->prec, c->nx, c->ny);
    const int ob = obs_grid(theory == SS_ABELIAN_HIGGS ? TH_AH : TH_CM, c->prec, ntiles);
    const size_t stb = align256(sizeof(DevState));
    const size_t fpb = align256(sizeof(FlowPartial) * (size_t)fb);
    const size_t opb = align256(sizeof(ObsPartial) * (size_t)ob);
    const bool comp = c->prec == SS_FP32;
    const int nbuf = NBUF + (comp ? 2 : 0);
    const size_t total = nbuf * pb + stb + fpb + opb;
    cudaError_t e = cudaMalloc(&c->base, total);
    if (e != cudaSuccess) {
      c->base = nullptr;
      return fail(SS_ERR_NOMEM, std::string("cudaMalloc of the buffer set failed: ") + cudaGetErrorString(e));
    }
    // zero everything once: k_v and v stay zero on the halo for ever
    SS_CK(cudaMemsetAsync(c->base, 0, total, c->stream));
    char* p = static_cast<char*>(c->base);
    c->L.phi[0] = p; p += pb;
    c->L.phi[1] = p; p += pb;
    c->L.v[0] = p; p += pb;
    c->L.v[1] = p; p += pb;
    for (int i = 0; i < 2; ++i) { c->L.kv[i] = p; p += pb; }
    c->L.lo[0] = c->L.lo[1] = nullptr;
    if (comp) {
      c->L.lo[0] = p; p += pb;
      c->L.lo[1] = p; p += pb;
    }
    c->L.st = reinterpret_cast<DevState*>(p); p += stb;
    c->L.fpart = reinterpret_cast<FlowPartial*>(p); p += fpb;
    c->L.opart = reinterpret_cast<ObsPartial*>(p);
    c->L.flow_blocks = fb;
    c->L.obs_blocks = ob;
  }
  c->theory = theory;
  c->C = C;
  c->L.theory = theory == SS_ABELIAN_HIGGS ? TH_AH : TH_CM;
  std::memcpy(c->L.coup, k, sizeof(k));
  // couplings are baked into captured graphs: drop them
  for (int q = 0; q < 2; ++q)
    if (c->chunk[q]) { cudaGraphExecDestroy(c->chunk[q]); c->chunk[q] = nullptr; }
  c->fields_set = false;
  SS_CK(launch_reset_state(c->L, c->stream));
  SS_CK(cudaStreamSynchronize(c->stream));
  return SS_OK;
}

int ss_init_ansatz(ss_ctx* c, const ss_soliton* s, int n) {
  if (!c) return fail(SS_ERR_ARG, "null context");
  if (!c->theory) return fail(SS_ERR_STATE, "ss_set_theory has not been called");
  if (!s || n < 1) return fail(SS_ERR_ARG, "need at least one soliton");
  for (int i = 0; i < n; ++i)
    if (!(s[i].size > 0.0) || !std::isfinite(s[i].x) || !std::isfinite(s[i].y) || !std::isfinite(s[i].phase))
      return fail(SS_ERR_ARG, "soliton entries must be finite with size > 0");
  if (n > c->sol_cap) {
    if (c->d_sol) cudaFree(c->d_sol);
    c->d_sol = nullptr;
    c->sol_cap = 0;
    SS_CK(cudaMalloc(&c->d_sol, sizeof(double) * 5 * (size_t)n));
    c->sol_cap = n;
  }
  double* h = nullptr;
  SS_CK(cudaMallocHost(&h, sizeof(double) * 5 * (size_t)n));
  for (int i = 0; i < n; ++i) {
    h[5 * i] = s[i].x;
    h[5 * i + 1] = s[i].y;
    h[5 * i + 2] = (double)s[i].charge;
    h[5 * i + 3] = s[i].size;
    h[5 * i + 4] = s[i].phase;
  }
  cudaError_t e = cudaMemcpyAsync(c->d_sol, h, sizeof(double) * 5 * (size_t)n, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = launch_ansatz(c->L, c->d_sol, n, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFreeHost(h);
  if (e != cudaSuccess) return fail(SS_ERR_CUDA, std::string("ss_init_ansatz: ") + cudaGetErrorString(e));
  int rc = new_fields(c);
  if (rc != SS_OK) return rc;
  SS_CK(cudaStreamSynchronize(c->stream));
  return SS_OK;
}

int ss_set_fields(ss_ctx* c, const void* f, int is_device) {
  if (!c) return fail(SS_ERR_ARG, "null context");
  if (!c->theory) return fail(SS_ERR_STATE, "ss_set_theory has not been called");
  if (!f) return fail(SS_ERR_ARG, "fields is NULL");
  const size_t bytes = (size_t)c->C * c->L.plane * c->elem;
  const cudaMemcpyKind kind = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  SS_CK(cudaMemcpyAsync(c->L.phi[0], f, bytes, kind, c->stream));
  SS_CK(cudaMemcpyAsync(c->L.phi[1], c->L.phi[0], bytes, cudaMemcpyDeviceToDevice, c->stream));
  int rc = new_fields(c);
  if (rc != SS_OK) return rc;
  SS_CK(cudaStreamSynchronize(c->stream));
  return SS_OK;
}

int ss_get_fields(ss_ctx* c, void* f, int is_device) {
  int rc = check_ready(c);
  if (rc != SS_OK) return rc;
  if (!f) return fail(SS_ERR_ARG, "fields is NULL");
  const size_t bytes = (size_t)c->C * c->L.plane * c->elem;
  SS_CK(cudaMemcpyAsync(f, c->L.phi[c->cur], bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        c->stream));
  SS_CK(cudaStreamSynchronize(c->stream));
  return SS_OK;
}

int ss_get_remainder(ss_ctx* c, void* lo, int is_device) {
  int rc = check_ready(c);
  if (rc != SS_OK) return rc;
  if (!lo) return fail(SS_ERR_ARG, "remainder is NULL");
  const size_t bytes = (size_t)c->C * c->L.plane * c->elem;
  if (c->prec == SS_FP32) {
    SS_CK(cudaMemcpyAsync(lo, c->L.lo[c->cur], bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          c->stream));
  } else if (is_device) {
    SS_CK(cudaMemsetAsync(lo, 0, bytes, c->stream));
  } else {
    std::memset(lo, 0, bytes);
  }
  SS_CK(cudaStreamSynchronize(c->stream));
  return SS_OK;
}

int ss_get_velocity(ss_ctx* c, void* out, int is_device) {
  int rc = check_ready(c);
  if (rc != SS_OK) return rc;
  if (!out) return fail(SS_ERR_ARG, "velocity is NULL");
  SS_CK(launch_pass(c->L, 1, c->cur, c->stream));  // resolves a pending arrest (no-op if known)
  DevState h;
  rc = read_state(c, &h);
  if (rc != SS_OK) return rc;
  const size_t bytes = (size_t)c->C * c->L.plane * c->elem;
  if (h.arrest) {
    if (is_device) SS_CK(cudaMemsetAsync(out, 0, bytes, c->stream));
    else std::memset(out, 0, bytes);
  } else {
    SS_CK(cudaMemcpyAsync(out, c->L.v[c->cur], bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          c->stream));
  }
  SS_CK(cudaStreamSynchronize(c->stream));
  return SS_OK;
}

int ss_force(ss_ctx* c, void* out, int is_device, double* energy, double* grad_max) {
  int rc = check_ready(c);
  if (rc != SS_OK) return rc;
  if (!out) return fail(SS_ERR_ARG, "force is NULL");
  SS_CK(launch_pass(c->L, 1, c->cur, c->stream));  // k_v1 = -G of the current field
  const size_t bytes = (size_t)c->C * c->L.plane * c->elem;
  if (is_device) {
    SS_CK(launch_scaled_copy(c->L, out, c->L.kv[0], -1.0, c->stream));
  } else {
    // v[cur ^ 1] is the next step's output buffer: free scratch, and -G keeps its halo zero
    void* scratch = c->L.v[c->cur ^ 1];
    SS_CK(launch_scaled_copy(c->L, scratch, c->L.kv[0], -1.0, c->stream));
    SS_CK(cudaMemcpyAsync(out, scratch, bytes, cudaMemcpyDeviceToHost, c->stream));
  }
  DevState h;
  rc = read_state(c, &h);
  if (rc != SS_OK) return rc;
  if (energy) *energy = h.E_cur;
  if (grad_max) *grad_max = h.gmax;
  return SS_OK;
}

int ss_step(ss_ctx* c, int n_steps, ss_status* out) {
  int rc = check_ready(c);
  if (rc != SS_OK) return rc;
  if (n_steps < 0) return fail(SS_ERR_ARG, "n_steps must be >= 0");
  DevState h;
  rc = run(c, -1.0, n_steps, &h);
  if (rc != SS_OK) return rc;
  fill_status(h, out);
  if (h.nonfinite) return fail(SS_ERR_NONFINITE, "energy or force became non-finite; the flow stopped");
  return SS_OK;
}

int ss_minimise(ss_ctx* c, double tol, long long max_steps, ss_status* out) {
  int rc = check_ready(c);
  if (rc != SS_OK) return rc;
  if (max_steps < 0) return fail(SS_ERR_ARG, "max_steps must be >= 0");
  if (!(tol >= 0.0)) return fail(SS_ERR_ARG, "tol must be >= 0");
  DevState h;
  rc = run(c, tol, max_steps, &h);
  if (rc != SS_OK) return rc;
  fill_status(h, out);
  if (h.nonfinite) return fail(SS_ERR_NONFINITE, "energy or force became non-finite; the flow stopped");
  if (!h.converged) return fail(SS_ERR_NOT_CONVERGED, "max_steps reached before the tolerance");
  return SS_OK;
}

int ss_observables(ss_ctx* c, ss_obs* out) {
  int rc = check_ready(c);
  if (rc != SS_OK) return rc;
  if (!out) return fail(SS_ERR_ARG, "out is NULL");
  SS_CK(launch_observables(c->L, c->cur, c->stream));
  DevState h;
  rc = read_state(c, &h);
  if (rc != SS_OK) return rc;
  out->energy = h.obs_energy;
  out->charge = h.obs_charge;
  out->flux = h.obs_flux;
  out->grad_max = h.obs_gmax_raw * c->dx * c->dy;
  out->grad_max_raw = h.obs_gmax_raw;
  out->norm_dev = h.obs_normdev;
  out->steps = h.steps;
  return SS_OK;
}

int ss_profile_stages(ss_ctx* c, int n_steps, float* ms_out) {
  int rc = check_ready(c);
  if (rc != SS_OK) return rc;
  if (n_steps < 1 || n_steps > 4096 || !ms_out) return fail(SS_ERR_ARG, "n_steps must be in 1..4096 and ms_out non-NULL");
  SS_CK(launch_set_run(c->L, -1.0, n_steps, c->stream));
  SS_CK(launch_pass(c->L, 1, c->cur, c->stream));  // head of the current field, untimed
  cudaEvent_t ev[3];
  for (int i = 0; i < 3; ++i) SS_CK(cudaEventCreate(&ev[i]));
  double acc[2] = {0, 0};
  int p = c->cur;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < n_steps && e == cudaSuccess; ++k) {
    e = cudaEventRecord(ev[0], c->stream);
    if (e == cudaSuccess) e = launch_pass(c->L, 2, p, c->stream);      // stages 3-4 -> new field
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], c->stream);
    if (e == cudaSuccess) e = launch_pass(c->L, 1, p ^ 1, c->stream);  // stages 1-2 of the new field
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[2]);
    float m1 = 0.f, m2 = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&m2, ev[0], ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&m1, ev[1], ev[2]);
    acc[0] += m1;
    acc[1] += m2;
    p ^= 1;
  }
  for (int i = 0; i < 3; ++i) cudaEventDestroy(ev[i]);
  if (e != cudaSuccess) return fail(SS_ERR_CUDA, std::string("ss_profile_stages: ") + cudaGetErrorString(e));
  DevState h;
  rc = read_state(c, &h);
  if (rc != SS_OK) return rc;
  ms_out[0] = (float)(acc[0] / n_steps);
  ms_out[1] = (float)(acc[1] / n_steps);
  if (h.nonfinite) return fail(SS_ERR_NONFINITE, "energy or force became non-finite; the flow stopped");
  return SS_OK;
}

int ss_destroy(ss_ctx* c) {
  if (!c) return SS_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_buffers(c);
  if (c->d_sol) cudaFree(c->d_sol);
  for (int i = 0; i < 2; ++i) {
    if (c->h_st[i]) cudaFreeHost(c->h_st[i]);
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  }
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return SS_OK;
}

}  // extern "C"
