// ss_api.cu -- host runtime and C-ABI of the soliton relaxation library
// (declarations and argument contracts in include/soliton.h).
//
// The runtime follows the paper's workflow (Sec. 4.1): select a theory and its
// parameters, allocate the device buffer set, initialise the field from an ansatz,
// then minimise. Everything runs on batches: a batch is any number of independent
// problems (grid, spacing, couplings, initial solitons) of one theory and one
// precision, and a single-grid context (ss_ctx) is a batch of one.
//
// Per problem the buffer set is reduced to what the fused pass kernels need
// (Sec. 3.1 lists fields, velocity, gradient, derivative work arrays and RK stages):
//   phi[2], v[2]   ping-pong field and velocity (RK4 reads phi^n around each site
//                  while writing phi^{n+1}; phi^{n-1} feeds the arrest test),
//   kv[2]          stage accelerations k_v1, k_v2 (k_v3, k_v4 stay in registers),
//   lo[2]          compensated FP32 only: the remainder planes of phi[2],
// plus one device flow record and one reduction partial per tile. Derivatives never
// touch memory. Steps are enqueued as CUDA graphs of K_CHUNK steps; convergence,
// arrest and the step budget are decided on the device per problem, so the host
// only polls one counter of still-running problems once per graph, one graph ahead.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "soliton.h"
#include "ss_internal.h"

using namespace ss;

namespace {

constexpr int K_CHUNK = 32;  // steps per captured graph

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

void ss::set_last_error(const std::string& msg) { g_err = msg; }

#define SS_CK(call)                                                                                       \
  do {                                                                                                    \
    cudaError_t e_ = (call);                                                                              \
    if (e_ != cudaSuccess) return fail(SS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Couplings of Table 1 / Eq. 5 packed as the kernels read them (Couplings in
// ss_device.cuh). Returns SS_OK or an error code (message set).
int ss::pack_couplings(int theory, const double* params, int n_params, double k[NCOUP], int* C) {
  if (!params && n_params > 0) return fail(SS_ERR_ARG, "params is NULL");
  for (int i = 0; i < NCOUP; ++i) k[i] = 0.0;
  if (theory == SS_ABELIAN_HIGGS) {
    if (n_params < 1 || n_params > 2) return fail(SS_ERR_ARG, "Abelian Higgs takes {lambda[, u]}");
    const double lam = params[0], u = n_params > 1 ? params[1] : 1.0;
    if (!std::isfinite(lam) || !std::isfinite(u) || lam < 0.0) return fail(SS_ERR_ARG, "lambda must be finite and >= 0");
    k[0] = lam;
    k[1] = u * u;
    *C = 4;
  } else if (theory == SS_CHIRAL_MAGNET) {
    if (n_params < 4 || n_params > 6)
      return fail(SS_ERR_ARG, "chiral magnet takes {J, D, K, h[, dmi_type[, mu_d]]}");
    for (int i = 0; i < n_params; ++i)
      if (!std::isfinite(params[i])) return fail(SS_ERR_ARG, "chiral-magnet parameters must be finite");
    if (!(params[0] > 0.0)) return fail(SS_ERR_ARG, "J must be > 0");
    const int type = n_params > 4 ? (int)params[4] : 0;
    if (type < 0 || type > 2 || (n_params > 4 && params[4] != (double)type))
      return fail(SS_ERR_ARG, "dmi_type must be 0 (interfacial), 1 (bulk) or 2 (D_2d)");
    for (int i = 0; i < 4; ++i) k[i] = params[i];
    // DMI vectors d_1 (k[4..6]) and d_2 (k[7..9]) of Eq. 5
    if (type == 0) { k[5] = 1.0; k[7] = -1.0; }      // d_i = e_3 x e_i
    else if (type == 1) { k[4] = 1.0; k[8] = 1.0; }  // d_i = e_i
    else { k[4] = 1.0; k[8] = -1.0; }                // d_1 = e_1, d_2 = -e_2
    if (n_params > 5) {  // demagnetisation (Eq. 6), mu_d = mu_0 M_s^2 in the energy's units
      if (!(params[5] >= 0.0)) return fail(SS_ERR_ARG, "mu_d must be >= 0");
      k[10] = params[5];
    }
    *C = 3;
  } else if (theory == SS_SID) {
    if (n_params != 7) return fail(SS_ERR_ARG, "s+id takes {a1, a2, b1, b2, b3, b4, nu}");
    for (int i = 0; i < 7; ++i)
      if (!std::isfinite(params[i])) return fail(SS_ERR_ARG, "s+id parameters must be finite");
    const double b1 = params[2], b2 = params[3], b3e = params[4] - 2.0 * std::fabs(params[5]);
    if (!(b1 > 0.0) || !(b2 > 0.0) || !(4.0 * b1 * b2 > b3e * b3e))
      return fail(SS_ERR_ARG, "s+id quartic potential must be bounded below (b1, b2 > 0, 4 b1 b2 > (b3 - 2|b4|)^2)");
    if (!(std::fabs(params[6]) < 1.0)) return fail(SS_ERR_ARG, "|nu| must be < 1 (positive gradient energy)");
    for (int i = 0; i < 7; ++i) k[i] = params[i];
    *C = 6;
  } else if (theory == SS_BEC) {
    if (n_params < 3 || n_params > 4) return fail(SS_ERR_ARG, "BEC takes {g, Omega, mu[, N]}");
    for (int i = 0; i < n_params; ++i)
      if (!std::isfinite(params[i])) return fail(SS_ERR_ARG, "BEC parameters must be finite");
    if (!(params[0] > 0.0)) return fail(SS_ERR_ARG, "g must be > 0 (the functional is unbounded below otherwise)");
    const double atoms = n_params > 3 ? params[3] : 0.0;
    if (atoms < 0.0) return fail(SS_ERR_ARG, "the atom number N must be >= 0 (0: grand-canonical form)");
    k[0] = params[0];  // g
    k[1] = params[1];  // Omega
    k[2] = atoms > 0.0 ? 0.0 : params[2];  // mu (fixed N: the energy at mu = 0; the multiplier is held per step)
    k[4] = atoms;      // fixed atom number N0 (0: none); host-side only
    *C = 2;
  } else if (theory == SS_BABY_SKYRME) {
    if (n_params < 2 || n_params > 3) return fail(SS_ERR_ARG, "Baby Skyrme takes {kappa, mu[, nu]}");
    for (int i = 0; i < n_params; ++i)
      if (!std::isfinite(params[i])) return fail(SS_ERR_ARG, "Baby Skyrme parameters must be finite");
    const double nu = n_params > 2 ? params[2] : 0.0;
    k[0] = params[0] * params[0];  // kappa^2 (Skyrme term)
    k[1] = params[1] * params[1];  // mu^2 (1 - m_3)
    k[2] = nu * nu;                // nu^2 / 2 m_1^2
    *C = 3;
  } else {
    return fail(SS_ERR_ARG, "unknown theory");
  }
  return SS_OK;
}

namespace {

// Kernel theory tag of an SS_* theory code (the chiral magnet with mu_d > 0 runs the
// demagnetisation kernels: th_of_coup).
int th_of(int theory) {
  switch (theory) {
    case SS_ABELIAN_HIGGS: return TH_AH;
    case SS_CHIRAL_MAGNET: return TH_CM;
    case SS_BABY_SKYRME: return TH_BS;
    case SS_SID: return TH_SID;
    default: return TH_BEC;
  }
}
int th_of_coup(int theory, const double* k) { return theory == SS_CHIRAL_MAGNET && k[10] > 0.0 ? TH_CMD : th_of(theory); }

int check_grid(int nx, int ny, double dx, double dy) {
  if (nx < 5 || ny < 5) return fail(SS_ERR_ARG, "nx and ny must be >= 5 (halo of width 2 on each side)");
  if ((long long)nx * ny > (1LL << 31)) return fail(SS_ERR_ARG, "grid too large (nx * ny > 2^31)");
  if (!(dx > 0.0) || !(dy > 0.0) || !std::isfinite(dx) || !std::isfinite(dy))
    return fail(SS_ERR_ARG, "dx and dy must be positive and finite");
  return SS_OK;
}

// Gradient descent: dtau = factor x the Euler stability limit 2 / lambda_max. For the
// Eq. 2 Laplacian lambda_max = (16/3)(1/dx^2 + 1/dy^2) (the stencil's largest
// eigenvalue, at the checkerboard mode). The BEC adds bounds on its position-dependent
// terms over the grid: the trap r_max^2, the interaction at the Thomas-Fermi density
// 4 |mu|, and the rotation 2 |Omega| r_max s1 with s1 = 1.3722 / min(dx, dy), the
// largest magnitude of the Eq. 1 symbol. The s+id mixed gradient scales the Laplacian
// bound by 1 + |nu|.
double descent_step(double dx, double dy, double factor, int theory = 0, int nx = 0, int ny = 0,
                    const double* coup = nullptr) {
  double lam = (16.0 / 3.0) * (1.0 / (dx * dx) + 1.0 / (dy * dy));
  if (theory == SS_SID && coup) lam *= 1.0 + std::fabs(coup[6]);  // the mixed gradient's band coupling
  if (theory == SS_BEC && coup) {
    const double hx = 0.5 * (nx - 1) * dx, hy = 0.5 * (ny - 1) * dy;
    const double r2 = hx * hx + hy * hy;
    // at a fixed atom number the chemical potential is not known in advance: its
    // Thomas-Fermi value sqrt(g N / pi) (harmonic trap, 2D) stands in for |mu|
    const double mu = coup[4] > 0.0 ? std::sqrt(coup[0] * coup[4] / 3.14159265358979323846) : std::fabs(coup[2]);
    lam += r2 + 4.0 * mu + 2.0 * std::fabs(coup[1]) * std::sqrt(r2) * 1.3722 / (dx < dy ? dx : dy);
  }
  return factor * 2.0 / lam;
}
constexpr double DEFAULT_STEP_FACTOR = 0.8;

// One problem of a batch, host view.
struct Problem {
  int nx = 0, ny = 0;
  double dx = 0, dy = 0, dt = 0;
  double tau = 0;  // gradient-descent step
  double coup[NCOUP] = {0};
  size_t plane = 0;
  int ntx = 0, ntiles = 0, tile0 = 0;
  void* phi[2] = {nullptr, nullptr};
  void* lo[2] = {nullptr, nullptr};
  void* v[2] = {nullptr, nullptr};
  void* kv[2] = {nullptr, nullptr};
  void* psi[2] = {nullptr, nullptr};  // demagnetisation: the potential of phi[0], phi[1]
};

template <typename R>
ProbDesc<R> make_desc(const Problem& p, DevState* st, FlowPartial* part) {
  ProbDesc<R> d{};
  d.nx = p.nx;
  d.ny = p.ny;
  d.ntx = p.ntx;
  d.ntiles = p.ntiles;
  d.tile0 = p.tile0;
  d.vec = (sizeof(R) == 4 && p.nx % 4 == 0) ? 1 : 0;
  d.plane = (long long)p.plane;
  for (int i = 0; i < 2; ++i) {
    d.phi[i] = static_cast<R*>(p.phi[i]);
    d.lo[i] = static_cast<R*>(p.lo[i]);
    d.v[i] = static_cast<R*>(p.v[i]);
    d.kv[i] = static_cast<R*>(p.kv[i]);
    d.psi[i] = static_cast<R*>(p.psi[i]);
  }
  d.dt = (R)p.dt;
  d.tau = (R)p.tau;
  d.hx = (R)p.dx;
  d.hy = (R)p.dy;
  d.h.i12dx = (R)(1.0 / (12.0 * p.dx));
  d.h.i12dy = (R)(1.0 / (12.0 * p.dy));
  d.h.i12dx2 = (R)(1.0 / (12.0 * p.dx * p.dx));
  d.h.i12dy2 = (R)(1.0 / (12.0 * p.dy * p.dy));
  d.h.i144dxdy = (R)(1.0 / (144.0 * p.dx * p.dy));
  for (int i = 0; i < NCOUP; ++i) d.k.c[i] = (R)p.coup[i];
  d.area = p.dx * p.dy;
  d.st = st;
  d.part = part;
  return d;
}

}  // namespace

// A batch of independent problems of one theory and precision.
struct ss_batch {
  int theory = 0;  // SS_ABELIAN_HIGGS / SS_CHIRAL_MAGNET / SS_BABY_SKYRME
  int prec = 0;    // SS_FP32 / SS_FP64 / SS_FP32_PLAIN
  int C = 0;
  size_t elem = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<Problem> probs;
  void* base = nullptr;         // every device buffer of the batch
  void* desc = nullptr;         // ProbDesc<R>[n]
  int* tile_prob = nullptr;     // [total_tiles]
  DevState* st = nullptr;       // [n]
  FlowPartial* part = nullptr;  // [total_tiles]
  ObsPartial* opart = nullptr;  // observables scratch, one problem at a time
  int obs_cap = 0;
  double* d_sol = nullptr;
  int sol_cap = 0;
  int* d_active = nullptr;
  BatchLaunch BL{};
  int method = METHOD_ANF;      // SS_METHOD_ANF / SS_METHOD_GRADIENT
  bool demag = false;           // chiral magnet with demagnetisation (single problem)
  bool fixed_n = false;         // BEC at a fixed atom number (single problem)
  DemagSolver* ds = nullptr;
  cudaGraphExec_t chunk = nullptr;  // K_CHUNK steps of the current method
  DevState* h_st = nullptr;  // pinned [n]
  int* h_active = nullptr;   // pinned [2]
  cudaEvent_t ev[2] = {nullptr, nullptr};
  std::vector<int> fields_set;
  std::vector<unsigned char> one_desc;  // host copy of problem 0's descriptor

  int n() const { return (int)probs.size(); }
};

namespace {

void batch_free(ss_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->chunk) cudaGraphExecDestroy(b->chunk);
  if (b->ds) demag_destroy(b->ds);
  if (b->base) cudaFree(b->base);
  if (b->d_sol) cudaFree(b->d_sol);
  if (b->h_st) cudaFreeHost(b->h_st);
  if (b->h_active) cudaFreeHost(b->h_active);
  for (int i = 0; i < 2; ++i)
    if (b->ev[i]) cudaEventDestroy(b->ev[i]);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

template <typename R>
int upload_descs(ss_batch* b) {
  const int n = b->n();
  std::vector<ProbDesc<R>> d(n);
  for (int i = 0; i < n; ++i) d[i] = make_desc<R>(b->probs[i], b->st + i, b->part + b->probs[i].tile0);
  SS_CK(cudaMemcpy(b->desc, d.data(), sizeof(ProbDesc<R>) * n, cudaMemcpyHostToDevice));
  b->one_desc.assign(reinterpret_cast<const unsigned char*>(d.data()),
                     reinterpret_cast<const unsigned char*>(d.data()) + sizeof(ProbDesc<R>));
  return SS_OK;
}

// Tile the batch with tile shape ts (0 small, 1 large): every problem's tiles, the
// tile -> problem map, the descriptors and the pass grids (`blocks`: passes 1 and 2
// of the arrested flow, or blocks[0] for the descent pass under gradient descent;
// each pass's occupancy x SMs when NULL). The captured step graph is dropped and
// re-captured. Call only while no launch of the batch is in flight.
int batch_layout(ss_batch* b, int ts, const int* blocks) {
  const int n = b->n();
  int tx, ty;
  flow_tile_dims(b->prec, ts, &tx, &ty);
  int total = 0;
  for (Problem& p : b->probs) {
    p.ntx = (p.nx + tx - 1) / tx;
    p.ntiles = p.ntx * ((p.ny + ty - 1) / ty);
    p.tile0 = total;
    total += p.ntiles;
  }
  std::vector<int> tp((size_t)total);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < b->probs[i].ntiles; ++k) tp[(size_t)b->probs[i].tile0 + k] = i;
  SS_CK(cudaStreamSynchronize(b->stream));
  int rc = b->prec == SS_FP64 ? upload_descs<double>(b) : upload_descs<float>(b);
  if (rc != SS_OK) return rc;
  SS_CK(cudaMemcpy(b->tile_prob, tp.data(), sizeof(int) * tp.size(), cudaMemcpyHostToDevice));
  b->BL.total_tiles = total;
  b->BL.ts = ts;
  b->BL.nprob = n;
  // a batch of one passes its descriptor to the pass kernels by value
  b->BL.one = n == 1 ? static_cast<const void*>(b->one_desc.data()) : nullptr;
  const int th = (b->demag ? TH_CMD : th_of(b->theory));
  flow_grid(th, b->prec, ts, total, n == 1, b->BL.flow_blocks);
  if (blocks) {
    if (b->method == METHOD_GD) b->BL.flow_blocks[2] = blocks[0] < total ? blocks[0] : total;
    else
      for (int i = 0; i < 2; ++i) b->BL.flow_blocks[i] = blocks[i] < total ? blocks[i] : total;
  }
  if (b->chunk) {
    cudaGraphExecDestroy(b->chunk);
    b->chunk = nullptr;
  }
  return SS_OK;
}

// Allocate and lay out every buffer of a batch whose problems are filled in.
int batch_alloc(ss_batch* b) {
  const int n = b->n();
  int tx, ty;
  flow_tile_dims(b->prec, 0, &tx, &ty);  // the small tile shape has the most tiles
  const int nbuf = 6 + (b->prec == SS_FP32 ? 2 : 0);
  size_t bytes = 0;
  int total_tiles = 0, obs_need = 1;
  const int th = (b->demag ? TH_CMD : th_of(b->theory));
  for (Problem& p : b->probs) {
    p.plane = (size_t)p.nx * p.ny;
    total_tiles += ((p.nx + tx - 1) / tx) * ((p.ny + ty - 1) / ty);
    bytes += nbuf * align256((size_t)b->C * p.plane * b->elem);
    if (b->demag) bytes += 2 * align256(p.plane * b->elem);
    const int otiles = ((p.nx + TX - 1) / TX) * ((p.ny + TY - 1) / TY);
    const int og = obs_grid(th, b->prec, otiles);
    if (og > obs_need) obs_need = og;
  }
  const size_t desc_b = align256((b->prec == SS_FP64 ? sizeof(ProbDesc<double>) : sizeof(ProbDesc<float>)) * n);
  const size_t tile_b = align256(sizeof(int) * (size_t)total_tiles);
  const size_t st_b = align256(sizeof(DevState) * (size_t)n);
  const size_t part_b = align256(sizeof(FlowPartial) * (size_t)total_tiles);
  const size_t opart_b = align256(sizeof(ObsPartial) * (size_t)obs_need);
  const size_t act_b = 256;
  const size_t total = bytes + desc_b + tile_b + st_b + part_b + opart_b + act_b;
  cudaError_t e = cudaMalloc(&b->base, total);
  if (e != cudaSuccess) {
    b->base = nullptr;
    return fail(SS_ERR_NOMEM, std::string("cudaMalloc of the buffer set failed: ") + cudaGetErrorString(e));
  }
  // zero everything once: k_v and v stay zero on the halo for ever
  SS_CK(cudaMemsetAsync(b->base, 0, total, b->stream));
  char* q = static_cast<char*>(b->base);
  for (Problem& p : b->probs) {
    const size_t pb = align256((size_t)b->C * p.plane * b->elem);
    void** slots[8] = {&p.phi[0], &p.phi[1], &p.v[0], &p.v[1], &p.kv[0], &p.kv[1], &p.lo[0], &p.lo[1]};
    for (int i = 0; i < nbuf; ++i) {
      *slots[i] = q;
      q += pb;
    }
    if (b->demag)
      for (int k = 0; k < 2; ++k) {
        p.psi[k] = q;
        q += align256(p.plane * b->elem);
      }
  }
  b->desc = q;
  q += desc_b;
  b->tile_prob = reinterpret_cast<int*>(q);
  q += tile_b;
  b->st = reinterpret_cast<DevState*>(q);
  q += st_b;
  b->part = reinterpret_cast<FlowPartial*>(q);
  q += part_b;
  b->opart = reinterpret_cast<ObsPartial*>(q);
  q += opart_b;
  b->d_active = reinterpret_cast<int*>(q);
  b->obs_cap = obs_need;

  SS_CK(cudaStreamSynchronize(b->stream));  // the memset above precedes the copies
  b->BL.theory = th;
  b->BL.prec = b->prec;
  b->BL.probs = b->desc;
  b->BL.tile_prob = b->tile_prob;
  int rc = batch_layout(b, 1, nullptr);  // large tiles by default
  if (rc != SS_OK) return rc;
  SS_CK(cudaMallocHost(&b->h_st, sizeof(DevState) * n));
  SS_CK(cudaMallocHost(&b->h_active, sizeof(int) * 2));
  for (int i = 0; i < 2; ++i) SS_CK(cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming));
  if (b->demag) {
    const Problem& p = b->probs[0];
    const int dr = demag_create(&b->ds, p.nx, p.ny, p.dx, p.dy, b->prec == SS_FP64 ? PREC_F64 : PREC_F32);
    if (dr != 0)
      return fail(dr == -1 ? SS_ERR_NOMEM : SS_ERR_CUDA, "demagnetisation solver: allocation or transform plan failed");
  }
  SS_CK(launch_reset_states(b->st, n, b->stream));
  SS_CK(cudaStreamSynchronize(b->stream));
  b->fields_set.assign(n, 0);
  return SS_OK;
}

// What a new field needs before its step: the demagnetising potential, or the BEC's
// fixed-atom-number refresh (a no-op for every other problem).
cudaError_t field_refresh(ss_batch* b) {
  const Problem& p = b->probs[0];
  if (b->demag) return demag_solve(b->ds, b->st, p.phi, p.lo, p.psi, b->stream);
  if (!b->fixed_n) return cudaSuccess;
  FixedNLaunch L{};
  L.prec = b->prec;
  for (int k = 0; k < 2; ++k) {
    L.phi[k] = p.phi[k];
    L.lo[k] = p.lo[k];
    L.v[k] = p.v[k];
  }
  L.nx = p.nx;
  L.ny = p.ny;
  L.dx = p.dx;
  L.dy = p.dy;
  L.g = p.coup[0];
  L.omega = p.coup[1];
  L.atoms = p.coup[4];
  L.st = b->st;
  L.part = b->opart;
  L.blocks = b->obs_cap;
  return launch_fixed_n_refresh(L, b->stream);
}
bool has_refresh(const ss_batch* b) { return b->demag || b->fixed_n; }

// Launch view of one problem for the per-problem kernels (ansatz, observables);
// phi[0] of the view is the problem's current field (parity cur).
LaunchCtx problem_ctx(const ss_batch* b, int i, int cur) {
  const Problem& p = b->probs[i];
  LaunchCtx L{};
  L.theory = (b->demag ? TH_CMD : th_of(b->theory));
  L.prec = b->prec;
  L.nx = p.nx;
  L.ny = p.ny;
  L.plane = p.plane;
  L.dx = p.dx;
  L.dy = p.dy;
  L.dt = p.dt;
  std::memcpy(L.coup, p.coup, sizeof(L.coup));
  for (int k = 0; k < 2; ++k) {
    L.phi[k] = p.phi[k ^ cur];
    L.lo[k] = p.lo[k ^ cur];
    L.v[k] = p.v[k ^ cur];
    L.kv[k] = p.kv[k];
    L.psi[k] = p.psi[k ^ cur];
  }
  L.st = b->st + i;
  L.opart = b->opart;
  L.ntiles_x = (p.nx + TX - 1) / TX;
  L.ntiles_y = (p.ny + TY - 1) / TY;
  const int og = obs_grid(L.theory, b->prec, L.ntiles_x * L.ntiles_y);
  L.obs_blocks = og < b->obs_cap ? og : b->obs_cap;
  return L;
}

int read_states(ss_batch* b) {
  SS_CK(cudaMemcpyAsync(b->h_st, b->st, sizeof(DevState) * b->n(), cudaMemcpyDeviceToHost, b->stream));
  SS_CK(cudaStreamSynchronize(b->stream));
  return SS_OK;
}

int cur_of(const ss_batch* b, int i) { return (int)(b->h_st[i].steps & 1); }

// New fields for problem i (already in phi[0], phi[1]): zero v and lo, reset its record,
// and (refresh) the potential or atom-number refresh of the new field.
int problem_new_fields(ss_batch* b, int i, bool refresh = true) {
  const Problem& p = b->probs[i];
  const size_t bytes = (size_t)b->C * p.plane * b->elem;
  for (int k = 0; k < 2; ++k) {
    SS_CK(cudaMemsetAsync(p.v[k], 0, bytes, b->stream));
    if (p.lo[k]) SS_CK(cudaMemsetAsync(p.lo[k], 0, bytes, b->stream));
  }
  SS_CK(launch_reset_states(b->st + i, 1, b->stream));
  if (refresh) SS_CK(field_refresh(b));  // the new field's potential or atom-number refresh (step count 0: buffer 0)
  b->fields_set[i] = 1;
  return SS_OK;
}

int problem_ansatz(ss_batch* b, int i, const ss_soliton* s, int n) {
  if (!s || n < 1) return fail(SS_ERR_ARG, "need at least one soliton");
  for (int k = 0; k < n; ++k)
    if (!(s[k].size > 0.0) || !std::isfinite(s[k].x) || !std::isfinite(s[k].y) || !std::isfinite(s[k].phase))
      return fail(SS_ERR_ARG, "soliton entries must be finite with size > 0");
  SS_CK(cudaStreamSynchronize(b->stream));  // the staging buffer may still be in use
  if (n > b->sol_cap) {
    if (b->d_sol) cudaFree(b->d_sol);
    b->d_sol = nullptr;
    b->sol_cap = 0;
    SS_CK(cudaMalloc(&b->d_sol, sizeof(double) * 5 * (size_t)n));
    b->sol_cap = n;
  }
  std::vector<double> h(5 * (size_t)n);
  for (int k = 0; k < n; ++k) {
    h[5 * k] = s[k].x;
    h[5 * k + 1] = s[k].y;
    h[5 * k + 2] = (double)s[k].charge;
    h[5 * k + 3] = s[k].size;
    h[5 * k + 4] = s[k].phase;
  }
  SS_CK(cudaMemcpyAsync(b->d_sol, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, b->stream));
  SS_CK(launch_ansatz(problem_ctx(b, i, 0), b->d_sol, n, b->stream));
  SS_CK(cudaStreamSynchronize(b->stream));  // h is a host temporary
  return problem_new_fields(b, i);
}

int ensure_chunk(ss_batch* b) {
  if (b->chunk) return SS_OK;
  cudaGraph_t g = nullptr;
  SS_CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < K_CHUNK && e == cudaSuccess; ++k) {
    if (b->method == METHOD_GD) {
      e = launch_pass(b->BL, PASS_GD, b->stream);  // evaluate, then step
      if (e == cudaSuccess) e = field_refresh(b);  // refresh of the new field
      continue;
    }
    e = launch_pass(b->BL, 2, b->stream);                        // stages 3-4: new fields
    if (e == cudaSuccess) e = field_refresh(b);                  // their refresh (potential, atom number)
    if (e == cudaSuccess) e = launch_pass(b->BL, 1, b->stream);  // stages 1-2 of the new fields
  }
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(SS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&b->chunk, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(SS_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  return SS_OK;
}

// Run every problem up to max_steps more steps with threshold tol (< 0: none).
// Chunk i is enqueued before the running count of chunk i-1 is checked, so the GPU
// never waits for the host; once every problem has stopped the rest of an enqueued
// chunk is a row of launches whose tiles all skip.
// Under gradient descent each pass evaluates a field and then steps, so a run takes
// max_steps + 1 passes, the last one evaluating the final field.
int batch_steps(ss_batch* b, long long max_steps);

int batch_run(ss_batch* b, double tol, long long max_steps) {
  SS_CK(launch_set_run_all(b->st, b->n(), tol, max_steps, b->stream));
  return batch_steps(b, max_steps);
}

// The run loop of batch_run, for run parameters already set in the flow records.
int batch_steps(ss_batch* b, long long max_steps) {
  const int n = b->n();
  long long passes = max_steps;
  if (b->method == METHOD_GD) passes += 1;
  else SS_CK(launch_pass(b->BL, 1, b->stream));  // heads of the current fields (skipped where done)
  // whole chunks as graphs, the remainder (< K_CHUNK steps) as direct launches
  const long long nchunks = passes / K_CHUNK;
  const int rem = (int)(passes % K_CHUNK);
  if (nchunks > 0) {
    int rc = ensure_chunk(b);
    if (rc != SS_OK) return rc;
  }
  int prev = -1;
  bool stopped = false;
  for (long long i = 0; i < nchunks; ++i) {
    const int slot = (int)(i & 1);
    SS_CK(cudaGraphLaunch(b->chunk, b->stream));
    SS_CK(launch_count_active(b->st, n, b->d_active, b->stream));
    SS_CK(cudaMemcpyAsync(b->h_active + slot, b->d_active, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    SS_CK(cudaEventRecord(b->ev[slot], b->stream));
    if (prev >= 0) {
      SS_CK(cudaEventSynchronize(b->ev[prev]));
      if (b->h_active[prev] == 0) {
        stopped = true;
        break;
      }
    }
    prev = slot;
  }
  for (int k = 0; k < rem && !stopped; ++k) {
    if (b->method == METHOD_GD) {
      SS_CK(launch_pass(b->BL, PASS_GD, b->stream));
      SS_CK(field_refresh(b));
    } else {
      SS_CK(launch_pass(b->BL, 2, b->stream));
      SS_CK(field_refresh(b));
      SS_CK(launch_pass(b->BL, 1, b->stream));
    }
  }
  return read_states(b);
}

int problem_observables(ss_batch* b, int i, ss_obs* out);

// The convergence verdict after a run under threshold tol that started at step
// start[i] of problem i and may take max_steps steps. FP64: the flow's own test. FP32
// fields: the flow judged its residual in FP32 arithmetic, whose rounding noise near
// 1e-6 is a sizeable fraction of it, so the verdict is the FP64 evaluation of the
// stored field (value + remainder, as the observables): a problem the flow stopped as
// converged whose FP64 residual is not below tol takes further rounds of steps (1/64
// of the steps it took so far, 8 to 512) within its budget, and is judged again.
// conv[i] receives the verdict; the flow records are read back (h_st) on return.
int batch_verify(ss_batch* b, double tol, long long max_steps, const std::vector<long long>& start,
                 std::vector<char>& conv) {
  const int n = b->n();
  conv.assign(n, 0);
  int rc = read_states(b);
  if (rc != SS_OK) return rc;
  std::vector<char> pending(n, 0);
  for (int i = 0; i < n; ++i) {
    conv[i] = b->h_st[i].converged && !b->h_st[i].nonfinite;
    pending[i] = b->prec != SS_FP64 && conv[i];
  }
  if (b->prec == SS_FP64) return SS_OK;
  std::vector<double> g64(n, 0.0);
  for (;;) {
    for (int i = 0; i < n; ++i) {  // (each evaluation re-reads the flow records)
      if (!pending[i]) continue;
      ss_obs o{};
      rc = problem_observables(b, i, &o);
      if (rc != SS_OK) return rc;
      g64[i] = o.grad_max;
    }
    bool more = false;
    long long kmax = 0;
    for (int i = 0; i < n; ++i) {
      DevState& h = b->h_st[i];
      if (!pending[i]) {
        if (!conv[i] && !h.nonfinite) h.step_limit = h.steps;  // stays stopped
        continue;
      }
      if (g64[i] < tol) {
        conv[i] = 1;
        pending[i] = 0;
        h.converged = 1;
        continue;
      }
      conv[i] = 0;
      h.converged = 0;
      const long long used = h.steps - start[i];
      if (h.nonfinite || used >= max_steps) {
        pending[i] = 0;
        h.step_limit = h.steps;  // stopped: budget spent
        continue;
      }
      long long k = used / 64;
      k = k < 8 ? 8 : (k > 512 ? 512 : k);
      if (k > max_steps - used) k = max_steps - used;
      h.tol = -1.0;
      h.step_limit = h.steps + k;
      if (k > kmax) kmax = k;
      more = true;
    }
    SS_CK(cudaMemcpyAsync(b->st, b->h_st, sizeof(DevState) * n, cudaMemcpyHostToDevice, b->stream));
    if (!more) break;
    rc = batch_steps(b, kmax);
    if (rc != SS_OK) return rc;
    rc = read_states(b);
    if (rc != SS_OK) return rc;
  }
  return read_states(b);
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

int copy_planes(ss_batch* b, int i, void* dst, const void* src, int is_device) {
  const size_t bytes = (size_t)b->C * b->probs[i].plane * b->elem;
  SS_CK(cudaMemcpyAsync(dst, src, bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
  SS_CK(cudaStreamSynchronize(b->stream));
  return SS_OK;
}

int problem_observables(ss_batch* b, int i, ss_obs* out) {
  int rc = read_states(b);
  if (rc != SS_OK) return rc;
  LaunchCtx L = problem_ctx(b, i, cur_of(b, i));
  if (b->fixed_n) L.coup[3] = b->h_st[i].mu_held;  // the residual of the constrained problem
  SS_CK(launch_observables(L, 0, b->stream));
  rc = read_states(b);
  if (rc != SS_OK) return rc;
  const DevState& h = b->h_st[i];
  out->energy = h.obs_energy;
  out->charge = h.obs_charge;
  out->flux = h.obs_flux;
  out->grad_max = h.obs_gmax_raw * b->probs[i].dx * b->probs[i].dy;
  out->grad_max_raw = h.obs_gmax_raw;
  out->norm_dev = h.obs_normdev;
  out->steps = h.steps;
  out->atoms = h.obs_atoms;
  out->angular_momentum = h.obs_lz;
  out->chemical_potential = b->theory != SS_BEC ? 0.0 : (b->fixed_n ? h.mu_held : b->probs[i].coup[2]);
  return SS_OK;
}

int make_stream(ss_batch* b, void* cuda_stream) {
  if (cuda_stream) {
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    return SS_OK;
  }
  // graphs cannot be captured on the legacy stream: own a blocking stream
  SS_CK(cudaStreamCreate(&b->stream));
  b->own_stream = true;
  return SS_OK;
}

int batch_finish(ss_batch* b, ss_status* per_item, bool need_converged) {
  int nonfinite = 0, unconverged = 0;
  for (int i = 0; i < b->n(); ++i) {
    const DevState& h = b->h_st[i];
    if (per_item) fill_status(h, per_item + i);
    nonfinite += h.nonfinite != 0;
    unconverged += !h.converged;
  }
  if (nonfinite) return fail(SS_ERR_NONFINITE, std::to_string(nonfinite) + " problem(s) became non-finite");
  if (need_converged && unconverged)
    return fail(SS_ERR_NOT_CONVERGED, std::to_string(unconverged) + " problem(s) reached max_steps first");
  return SS_OK;
}

}  // namespace

// ================================================================== single grid
struct ss_ctx {
  int nx = 0, ny = 0;
  double dx = 0, dy = 0;
  int prec = 0;
  void* user_stream = nullptr;
  ss_batch* b = nullptr;  // a batch of one, created by ss_set_theory
};

namespace {

int check_ready(ss_ctx* c) {
  if (!c) return fail(SS_ERR_ARG, "null context");
  if (!c->b) return fail(SS_ERR_STATE, "ss_set_theory has not been called");
  if (!c->b->fields_set[0]) return fail(SS_ERR_STATE, "fields not set (ss_init_ansatz / ss_set_fields)");
  return SS_OK;
}

}  // namespace

extern "C" {

const char* ss_last_error(void) { return g_err.c_str(); }

int ss_version(void) { return 5; }

int ss_create_grid(ss_ctx** out, int nx, int ny, double dx, double dy, int precision, void* cuda_stream) {
  if (!out) return fail(SS_ERR_ARG, "out is NULL");
  *out = nullptr;
  int rc = check_grid(nx, ny, dx, dy);
  if (rc != SS_OK) return rc;
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
  c->prec = precision;
  c->user_stream = cuda_stream;
  *out = c;
  return SS_OK;
}

int ss_set_theory(ss_ctx* c, int theory, const double* params, int n_params) {
  if (!c) return fail(SS_ERR_ARG, "null context");
  double k[NCOUP];
  int C = 0;
  int rc = pack_couplings(theory, params, n_params, k, &C);
  if (rc != SS_OK) return rc;
  if (c->b) {
    batch_free(c->b);
    c->b = nullptr;
  }
  ss_batch* b = new (std::nothrow) ss_batch();
  if (!b) return fail(SS_ERR_NOMEM, "host allocation failed");
  b->theory = theory;
  b->prec = c->prec;
  b->C = C;
  b->elem = c->prec == SS_FP64 ? 8 : 4;
  b->demag = th_of_coup(theory, k) == TH_CMD;
  b->fixed_n = theory == SS_BEC && k[4] > 0.0;
  rc = make_stream(b, c->user_stream);
  if (rc != SS_OK) {
    batch_free(b);
    return rc;
  }
  Problem p;
  p.nx = c->nx;
  p.ny = c->ny;
  p.dx = c->dx;
  p.dy = c->dy;
  p.dt = 0.5 * (c->dx < c->dy ? c->dx : c->dy);  // Sec. 3.1: C = dt / dx = 0.5
  p.tau = descent_step(p.dx, p.dy, DEFAULT_STEP_FACTOR, theory, p.nx, p.ny, k);
  std::memcpy(p.coup, k, sizeof(k));
  b->probs.push_back(p);
  rc = batch_alloc(b);
  if (rc != SS_OK) {
    batch_free(b);
    return rc;
  }
  c->b = b;
  return SS_OK;
}

int ss_init_ansatz(ss_ctx* c, const ss_soliton* s, int n) {
  if (!c) return fail(SS_ERR_ARG, "null context");
  if (!c->b) return fail(SS_ERR_STATE, "ss_set_theory has not been called");
  int rc = problem_ansatz(c->b, 0, s, n);
  if (rc != SS_OK) return rc;
  return read_states(c->b);
}

int ss_set_fields(ss_ctx* c, const void* f, int is_device) {
  if (!c) return fail(SS_ERR_ARG, "null context");
  if (!c->b) return fail(SS_ERR_STATE, "ss_set_theory has not been called");
  if (!f) return fail(SS_ERR_ARG, "fields is NULL");
  ss_batch* b = c->b;
  const Problem& p = b->probs[0];
  const size_t bytes = (size_t)b->C * p.plane * b->elem;
  SS_CK(cudaMemcpyAsync(p.phi[0], f, bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->stream));
  SS_CK(cudaMemcpyAsync(p.phi[1], p.phi[0], bytes, cudaMemcpyDeviceToDevice, b->stream));
  int rc = problem_new_fields(b, 0);
  if (rc != SS_OK) return rc;
  return read_states(b);
}

int ss_get_fields(ss_ctx* c, void* f, int is_device) {
  int rc = check_ready(c);
  if (rc != SS_OK) return rc;
  if (!f) return fail(SS_ERR_ARG, "fields is NULL");
  rc = read_states(c->b);
  if (rc != SS_OK) return rc;
  return copy_planes(c->b, 0, f, c->b->probs[0].phi[cur_of(c->b, 0)], is_device);
}

int ss_get_remainder(ss_ctx* c, void* lo, int is_device) {
  int rc = check_ready(c);
  if (rc != SS_OK) return rc;
  if (!lo) return fail(SS_ERR_ARG, "remainder is NULL");
  ss_batch* b = c->b;
  rc = read_states(b);
  if (rc != SS_OK) return rc;
  if (b->prec == SS_FP32) return copy_planes(b, 0, lo, b->probs[0].lo[cur_of(b, 0)], is_device);
  const size_t bytes = (size_t)b->C * b->probs[0].plane * b->elem;
  if (is_device) SS_CK(cudaMemsetAsync(lo, 0, bytes, b->stream));
  else std::memset(lo, 0, bytes);
  SS_CK(cudaStreamSynchronize(b->stream));
  return SS_OK;
}

int ss_get_velocity(ss_ctx* c, void* out, int is_device) {
  int rc = check_ready(c);
  if (rc != SS_OK) return rc;
  if (!out) return fail(SS_ERR_ARG, "velocity is NULL");
  ss_batch* b = c->b;
  if (b->method != METHOD_GD) SS_CK(launch_pass(b->BL, 1, b->stream));  // resolves a pending arrest
  rc = read_states(b);
  if (rc != SS_OK) return rc;
  const size_t bytes = (size_t)b->C * b->probs[0].plane * b->elem;
  if (b->method == METHOD_GD || b->h_st[0].arrest) {  // gradient descent has no velocity
    if (is_device) SS_CK(cudaMemsetAsync(out, 0, bytes, b->stream));
    else std::memset(out, 0, bytes);
    SS_CK(cudaStreamSynchronize(b->stream));
    return SS_OK;
  }
  return copy_planes(b, 0, out, b->probs[0].v[cur_of(b, 0)], is_device);
}

int ss_force(ss_ctx* c, void* out, int is_device, double* energy, double* grad_max) {
  int rc = check_ready(c);
  if (rc != SS_OK) return rc;
  if (!out) return fail(SS_ERR_ARG, "force is NULL");
  ss_batch* b = c->b;
  SS_CK(launch_pass(b->BL, 1, b->stream));  // k_v1 = -G of the current field
  rc = read_states(b);
  if (rc != SS_OK) return rc;
  const int cur = cur_of(b, 0);
  const Problem& p = b->probs[0];
  const LaunchCtx L = problem_ctx(b, 0, cur);
  const size_t bytes = (size_t)b->C * p.plane * b->elem;
  if (is_device) {
    SS_CK(launch_scaled_copy(L, out, p.kv[0], -1.0, b->stream));
  } else {
    // v of the other parity is the next step's output buffer: free scratch, and -G
    // keeps its halo zero
    void* scratch = p.v[cur ^ 1];
    SS_CK(launch_scaled_copy(L, scratch, p.kv[0], -1.0, b->stream));
    SS_CK(cudaMemcpyAsync(out, scratch, bytes, cudaMemcpyDeviceToHost, b->stream));
  }
  SS_CK(cudaStreamSynchronize(b->stream));
  if (energy) *energy = b->h_st[0].E_cur;
  if (grad_max) *grad_max = b->h_st[0].gmax;
  return SS_OK;
}

int ss_step(ss_ctx* c, int n_steps, ss_status* out) {
  int rc = check_ready(c);
  if (rc != SS_OK) return rc;
  if (n_steps < 0) return fail(SS_ERR_ARG, "n_steps must be >= 0");
  rc = batch_run(c->b, -1.0, n_steps);
  if (rc != SS_OK) return rc;
  const DevState& h = c->b->h_st[0];
  fill_status(h, out);
  if (h.nonfinite) return fail(SS_ERR_NONFINITE, "energy or force became non-finite; the flow stopped");
  return SS_OK;
}

int ss_minimise(ss_ctx* c, double tol, long long max_steps, ss_status* out) {
  int rc = check_ready(c);
  if (rc != SS_OK) return rc;
  if (max_steps < 0) return fail(SS_ERR_ARG, "max_steps must be >= 0");
  if (!(tol >= 0.0)) return fail(SS_ERR_ARG, "tol must be >= 0");
  ss_batch* b = c->b;
  rc = read_states(b);
  if (rc != SS_OK) return rc;
  const long long start = b->h_st[0].steps;
  rc = batch_run(b, tol, max_steps);
  if (rc != SS_OK) return rc;
  const DevState& h = b->h_st[0];
  std::vector<long long> first(1, start);
  std::vector<char> conv;
  rc = batch_verify(b, tol, max_steps, first, conv);
  if (rc != SS_OK) return rc;
  fill_status(h, out);
  if (out) out->converged = conv[0];
  if (h.nonfinite) return fail(SS_ERR_NONFINITE, "energy or force became non-finite; the flow stopped");
  if (!conv[0]) return fail(SS_ERR_NOT_CONVERGED, "max_steps reached before the tolerance");
  return SS_OK;
}

int ss_observables(ss_ctx* c, ss_obs* out) {
  int rc = check_ready(c);
  if (rc != SS_OK) return rc;
  if (!out) return fail(SS_ERR_ARG, "out is NULL");
  return problem_observables(c->b, 0, out);
}

int ss_profile_stages(ss_ctx* c, int n_steps, float* ms_out) {
  int rc = check_ready(c);
  if (rc != SS_OK) return rc;
  if (n_steps < 1 || n_steps > 4096 || !ms_out) return fail(SS_ERR_ARG, "n_steps must be in 1..4096 and ms_out non-NULL");
  ss_batch* b = c->b;
  const bool gd = b->method == METHOD_GD;
  SS_CK(launch_set_run_all(b->st, b->n(), -1.0, n_steps, b->stream));
  if (!gd) SS_CK(launch_pass(b->BL, 1, b->stream));  // head of the current field, untimed
  cudaEvent_t ev[3];
  for (int i = 0; i < 3; ++i) SS_CK(cudaEventCreate(&ev[i]));
  double acc[2] = {0, 0};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < n_steps && e == cudaSuccess && gd; ++k) {  // gradient descent: one pass per step
    e = cudaEventRecord(ev[0], b->stream);
    if (e == cudaSuccess) e = launch_pass(b->BL, PASS_GD, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float m = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&m, ev[0], ev[1]);
    if (e == cudaSuccess) e = field_refresh(b);
    acc[0] += m;
  }
  if (gd && e == cudaSuccess) e = launch_pass(b->BL, PASS_GD, b->stream);  // evaluates the last field
  for (int k = 0; k < n_steps && e == cudaSuccess && !gd; ++k) {
    e = cudaEventRecord(ev[0], b->stream);
    if (e == cudaSuccess) e = launch_pass(b->BL, 2, b->stream);  // stages 3-4 -> new field
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], b->stream);
    float m1 = 0.f, m2 = 0.f;
    if (e == cudaSuccess && has_refresh(b)) {  // the new field's refresh, outside both intervals
      e = cudaEventSynchronize(ev[1]);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&m2, ev[0], ev[1]);
      if (e == cudaSuccess) e = field_refresh(b);
      if (e == cudaSuccess) e = cudaEventRecord(ev[1], b->stream);  // pass 1 starts after the solve
    }
    if (e == cudaSuccess) e = launch_pass(b->BL, 1, b->stream);  // stages 1-2 of the new field
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[2]);
    if (e == cudaSuccess && !has_refresh(b)) e = cudaEventElapsedTime(&m2, ev[0], ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&m1, ev[1], ev[2]);
    acc[0] += m1;
    acc[1] += m2;
  }
  for (int i = 0; i < 3; ++i) cudaEventDestroy(ev[i]);
  if (e != cudaSuccess) return fail(SS_ERR_CUDA, std::string("ss_profile_stages: ") + cudaGetErrorString(e));
  rc = read_states(b);
  if (rc != SS_OK) return rc;
  ms_out[0] = (float)(acc[0] / n_steps);
  ms_out[1] = (float)(acc[1] / n_steps);
  if (b->h_st[0].nonfinite) return fail(SS_ERR_NONFINITE, "energy or force became non-finite; the flow stopped");
  return SS_OK;
}

int ss_destroy(ss_ctx* c) {
  if (!c) return SS_OK;
  batch_free(c->b);
  delete c;
  return SS_OK;
}

// ================================================================== batches
int ss_batch_create(ss_batch** out, int theory, int precision, const ss_batch_item* items, int n, void* cuda_stream) {
  if (!out) return fail(SS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!items || n < 1) return fail(SS_ERR_ARG, "need at least one batch item");
  if (precision != SS_FP32 && precision != SS_FP64 && precision != SS_FP32_PLAIN)
    return fail(SS_ERR_ARG, "precision must be SS_FP32, SS_FP64 or SS_FP32_PLAIN");
  ss_batch* b = new (std::nothrow) ss_batch();
  if (!b) return fail(SS_ERR_NOMEM, "host allocation failed");
  b->theory = theory;
  b->prec = precision;
  b->elem = precision == SS_FP64 ? 8 : 4;
  for (int i = 0; i < n; ++i) {
    const ss_batch_item& it = items[i];
    int rc = check_grid(it.nx, it.ny, it.dx, it.dy);
    double k[NCOUP];
    int C = 0;
    if (rc == SS_OK) rc = pack_couplings(theory, it.params, it.n_params, k, &C);
    if (rc == SS_OK && th_of_coup(theory, k) == TH_CMD)
      rc = fail(SS_ERR_ARG, "demagnetisation (mu_d > 0) needs a single-grid context (ss_create_grid)");
    if (rc == SS_OK && theory == SS_BEC && k[4] > 0.0)
      rc = fail(SS_ERR_ARG, "a fixed atom number (N > 0) needs a single-grid context (ss_create_grid)");
    if (rc == SS_OK && (!it.solitons || it.n_solitons < 1)) rc = fail(SS_ERR_ARG, "every item needs at least one soliton");
    if (rc != SS_OK) {
      g_err = "item " + std::to_string(i) + ": " + g_err;
      batch_free(b);
      return rc;
    }
    b->C = C;
    Problem p;
    p.nx = it.nx;
    p.ny = it.ny;
    p.dx = it.dx;
    p.dy = it.dy;
    p.dt = 0.5 * (it.dx < it.dy ? it.dx : it.dy);  // Sec. 3.1
    p.tau = descent_step(p.dx, p.dy, DEFAULT_STEP_FACTOR, theory, p.nx, p.ny, k);
    std::memcpy(p.coup, k, sizeof(k));
    b->probs.push_back(p);
  }
  int rc = make_stream(b, cuda_stream);
  if (rc == SS_OK) rc = batch_alloc(b);
  for (int i = 0; i < n && rc == SS_OK; ++i) rc = problem_ansatz(b, i, items[i].solitons, items[i].n_solitons);
  if (rc == SS_OK) rc = read_states(b);
  if (rc != SS_OK) {
    batch_free(b);
    return rc;
  }
  *out = b;
  return SS_OK;
}

int ss_batch_size(ss_batch* b) { return b ? b->n() : 0; }

int ss_batch_step(ss_batch* b, int n_steps, ss_status* per_item) {
  if (!b) return fail(SS_ERR_ARG, "null batch");
  if (n_steps < 0) return fail(SS_ERR_ARG, "n_steps must be >= 0");
  int rc = batch_run(b, -1.0, n_steps);
  if (rc != SS_OK) return rc;
  return batch_finish(b, per_item, false);
}

int ss_batch_minimise(ss_batch* b, double tol, long long max_steps, ss_status* per_item) {
  if (!b) return fail(SS_ERR_ARG, "null batch");
  if (max_steps < 0) return fail(SS_ERR_ARG, "max_steps must be >= 0");
  if (!(tol >= 0.0)) return fail(SS_ERR_ARG, "tol must be >= 0");
  int rc = read_states(b);
  if (rc != SS_OK) return rc;
  std::vector<long long> start(b->n());
  for (int i = 0; i < b->n(); ++i) start[i] = b->h_st[i].steps;
  rc = batch_run(b, tol, max_steps);
  if (rc != SS_OK) return rc;
  std::vector<char> conv;
  rc = batch_verify(b, tol, max_steps, start, conv);
  if (rc != SS_OK) return rc;
  return batch_finish(b, per_item, true);
}

int ss_batch_get_fields(ss_batch* b, int item, void* fields, int is_device) {
  if (!b) return fail(SS_ERR_ARG, "null batch");
  if (item < 0 || item >= b->n()) return fail(SS_ERR_ARG, "item out of range");
  if (!fields) return fail(SS_ERR_ARG, "fields is NULL");
  int rc = read_states(b);
  if (rc != SS_OK) return rc;
  return copy_planes(b, item, fields, b->probs[item].phi[cur_of(b, item)], is_device);
}

int ss_batch_set_fields(ss_batch* b, int item, const void* fields, int is_device) {
  if (!b) return fail(SS_ERR_ARG, "null batch");
  if (item < 0 || item >= b->n()) return fail(SS_ERR_ARG, "item out of range");
  if (!fields) return fail(SS_ERR_ARG, "fields is NULL");
  const Problem& p = b->probs[item];
  const size_t bytes = (size_t)b->C * p.plane * b->elem;
  SS_CK(cudaMemcpyAsync(p.phi[0], fields, bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        b->stream));
  SS_CK(cudaMemcpyAsync(p.phi[1], p.phi[0], bytes, cudaMemcpyDeviceToDevice, b->stream));
  int rc = problem_new_fields(b, item);
  if (rc != SS_OK) return rc;
  return read_states(b);
}

// Autotuner of the flow launch: tile shape (32 x 16 or 32 x 32 sites in FP32) and the
// grid of each pass (1 .. occupancy blocks per SM), each candidate timed with CUDA
// events over trial_steps flow steps of the batch's own problems, starting from
// their current fields. The fastest combination is kept; every problem is then
// reset to its field at the call, at rest, with a fresh step count.
int batch_autotune(ss_batch* b, int trial_steps, int* choice) {
  if (trial_steps < 1 || trial_steps > 1000) return fail(SS_ERR_ARG, "trial_steps must be in 1..1000");
  int rc = read_states(b);
  if (rc != SS_OK) return rc;
  const int n = b->n();
  const bool lo = b->prec == SS_FP32;
  std::vector<size_t> off(n + 1, 0);
  for (int i = 0; i < n; ++i) off[i + 1] = off[i] + (size_t)b->C * b->probs[i].plane * b->elem * (lo ? 2 : 1);
  char* snap = nullptr;
  SS_CK(cudaMalloc(&snap, off[n]));
  auto release = [&](int code) {
    cudaStreamSynchronize(b->stream);
    cudaFree(snap);
    return code;
  };
  for (int i = 0; i < n; ++i) {
    const Problem& p = b->probs[i];
    const size_t bytes = (size_t)b->C * p.plane * b->elem;
    const int cur = cur_of(b, i);
    if (cudaMemcpyAsync(snap + off[i], p.phi[cur], bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess ||
        (lo && cudaMemcpyAsync(snap + off[i] + bytes, p.lo[cur], bytes, cudaMemcpyDeviceToDevice, b->stream) !=
                   cudaSuccess))
      return release(fail(SS_ERR_CUDA, "autotune: snapshot copy failed"));
  }
  auto restore = [&]() -> int {
    for (int i = 0; i < n; ++i) {
      const Problem& p = b->probs[i];
      const size_t bytes = (size_t)b->C * p.plane * b->elem;
      int r = problem_new_fields(b, i, false);  // the refresh must see the restored field
      if (r != SS_OK) return r;
      for (int k = 0; k < 2; ++k) {
        SS_CK(cudaMemcpyAsync(p.phi[k], snap + off[i], bytes, cudaMemcpyDeviceToDevice, b->stream));
        if (lo) SS_CK(cudaMemcpyAsync(p.lo[k], snap + off[i] + bytes, bytes, cudaMemcpyDeviceToDevice, b->stream));
      }
    }
    SS_CK(field_refresh(b));
    return SS_OK;
  };
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int th = (b->demag ? TH_CMD : th_of(b->theory));
  cudaEvent_t ev[3];
  for (int i = 0; i < 3; ++i)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) return release(fail(SS_ERR_CUDA, "autotune: event creation failed"));
  auto destroy_events = [&]() {
    for (int i = 0; i < 3; ++i) cudaEventDestroy(ev[i]);
  };
  // gradient descent: the descent pass alone, its grid in blocks[0] / occ[0]
  const bool gd = b->method == METHOD_GD;
  double best = 1e300;
  int best_ts = 1, best_blocks[2] = {0, 0};
  for (int ts = 0; ts < 2; ++ts) {
    int occ[3];
    flow_occupancy(th, b->prec, ts, n == 1, occ);
    if (gd) occ[0] = occ[1] = occ[2];
    const int kmax = occ[0] > occ[1] ? occ[0] : occ[1];
    double tbest[2] = {1e300, gd ? 0.0 : 1e300};
    int kbest[2] = {1, 1};
    for (int k = 1; k <= kmax; ++k) {
      const int blocks[2] = {(k < occ[0] ? k : occ[0]) * nsm, (k < occ[1] ? k : occ[1]) * nsm};
      if ((rc = batch_layout(b, ts, blocks)) != SS_OK || (rc = restore()) != SS_OK) {
        destroy_events();
        return release(rc);
      }
      cudaError_t e = launch_set_run_all(b->st, n, -1.0, trial_steps + 1, b->stream);
      double acc[2] = {0.0, 0.0};
      if (gd) {
        if (e == cudaSuccess) e = launch_pass(b->BL, PASS_GD, b->stream);  // one untimed step
        for (int step = 0; step < trial_steps && e == cudaSuccess; ++step) {
          e = cudaEventRecord(ev[0], b->stream);
          if (e == cudaSuccess) e = launch_pass(b->BL, PASS_GD, b->stream);
          if (e == cudaSuccess) e = cudaEventRecord(ev[1], b->stream);
          if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
          float m = 0.f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&m, ev[0], ev[1]);
          acc[0] += m;
        }
      } else {
        if (e == cudaSuccess) e = launch_pass(b->BL, 1, b->stream);  // head, untimed
        if (e == cudaSuccess) e = launch_pass(b->BL, 2, b->stream);  // one untimed step
        if (e == cudaSuccess) e = launch_pass(b->BL, 1, b->stream);
      }
      for (int step = 0; step < trial_steps && e == cudaSuccess && !gd; ++step) {
        e = cudaEventRecord(ev[0], b->stream);
        if (e == cudaSuccess) e = launch_pass(b->BL, 2, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], b->stream);
        if (e == cudaSuccess) e = launch_pass(b->BL, 1, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2], b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[2]);
        float m1 = 0.f, m2 = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&m2, ev[0], ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&m1, ev[1], ev[2]);
        acc[0] += m1;
        acc[1] += m2;
      }
      if (e != cudaSuccess) {
        destroy_events();
        return release(fail(SS_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e)));
      }
      for (int q = 0; q < (gd ? 1 : 2); ++q)
        if (k <= occ[q] && acc[q] < tbest[q]) {
          tbest[q] = acc[q];
          kbest[q] = k;
        }
    }
    if (tbest[0] + tbest[1] < best) {
      best = tbest[0] + tbest[1];
      best_ts = ts;
      best_blocks[0] = kbest[0] * nsm;
      best_blocks[1] = kbest[1] * nsm;
    }
  }
  destroy_events();
  if ((rc = batch_layout(b, best_ts, best_blocks)) != SS_OK || (rc = restore()) != SS_OK) return release(rc);
  rc = release(read_states(b));
  if (rc != SS_OK) return rc;
  if (choice) {
    choice[0] = best_ts;
    choice[1] = gd ? b->BL.flow_blocks[2] : b->BL.flow_blocks[0];
    choice[2] = gd ? 0 : b->BL.flow_blocks[1];
  }
  return SS_OK;
}

int batch_set_launch(ss_batch* b, int tile_shape, const int* blocks) {
  if (tile_shape != 0 && tile_shape != 1) return fail(SS_ERR_ARG, "tile_shape must be 0 or 1");
  if (blocks && (blocks[0] < 1 || (b->method != METHOD_GD && blocks[1] < 1)))
    return fail(SS_ERR_ARG, "block counts must be >= 1");
  return batch_layout(b, tile_shape, blocks);
}

// Switch the minimiser. Every problem whose fields are set restarts from its
// current field at rest: the field goes into both ping-pong buffers, velocity and
// step count are cleared, and the flow record is reset (the two methods keep
// different state: velocity and previous field for the arrested flow, none for
// descent).
int batch_set_method(ss_batch* b, int method, double step_factor) {
  if (method != SS_METHOD_ANF && method != SS_METHOD_GRADIENT)
    return fail(SS_ERR_ARG, "method must be SS_METHOD_ANF or SS_METHOD_GRADIENT");
  if (step_factor <= 0.0) step_factor = DEFAULT_STEP_FACTOR;
  if (!std::isfinite(step_factor) || step_factor > 1.0)
    return fail(SS_ERR_ARG, "step_factor must be in (0, 1] (<= 0 selects the default)");
  int rc = read_states(b);
  if (rc != SS_OK) return rc;
  for (int i = 0; i < b->n(); ++i) {
    Problem& p = b->probs[i];
    p.tau = descent_step(p.dx, p.dy, step_factor, b->theory, p.nx, p.ny, p.coup);
    if (!b->fields_set[i]) continue;
    const int cur = cur_of(b, i);
    const size_t bytes = (size_t)b->C * p.plane * b->elem;
    SS_CK(cudaMemcpyAsync(p.phi[cur ^ 1], p.phi[cur], bytes, cudaMemcpyDeviceToDevice, b->stream));
    if (p.lo[0]) SS_CK(cudaMemcpyAsync(p.lo[cur ^ 1], p.lo[cur], bytes, cudaMemcpyDeviceToDevice, b->stream));
    for (int k = 0; k < 2; ++k) SS_CK(cudaMemsetAsync(p.v[k], 0, bytes, b->stream));
    SS_CK(launch_reset_states(b->st + i, 1, b->stream));
  }
  if (b->fields_set[0]) SS_CK(field_refresh(b));  // step count 0: refresh of buffer 0
  b->method = method;
  const int blocks_keep[2] = {b->BL.flow_blocks[0], b->BL.flow_blocks[1]};
  b->BL.flow_blocks[2] = 0;
  rc = batch_layout(b, b->BL.ts, nullptr);  // new descriptors (dtau), default grids, graph dropped
  if (rc != SS_OK) return rc;
  b->BL.flow_blocks[0] = blocks_keep[0];  // an arrested-flow grid set before stays in force
  b->BL.flow_blocks[1] = blocks_keep[1];
  return read_states(b);
}

int ss_batch_set_launch(ss_batch* b, int tile_shape, const int* blocks) {
  if (!b) return fail(SS_ERR_ARG, "null batch");
  return batch_set_launch(b, tile_shape, blocks);
}

int ss_set_launch(ss_ctx* c, int tile_shape, const int* blocks) {
  int rc = check_ready(c);
  if (rc != SS_OK) return rc;
  return batch_set_launch(c->b, tile_shape, blocks);
}

int ss_batch_set_method(ss_batch* b, int method, double step_factor) {
  if (!b) return fail(SS_ERR_ARG, "null batch");
  return batch_set_method(b, method, step_factor);
}

int ss_set_method(ss_ctx* c, int method, double step_factor) {
  if (!c) return fail(SS_ERR_ARG, "null context");
  if (!c->b) return fail(SS_ERR_STATE, "ss_set_theory has not been called");
  return batch_set_method(c->b, method, step_factor);
}

int ss_batch_autotune(ss_batch* b, int trial_steps, int* choice) {
  if (!b) return fail(SS_ERR_ARG, "null batch");
  return batch_autotune(b, trial_steps, choice);
}

int ss_autotune(ss_ctx* c, int trial_steps, int* choice) {
  int rc = check_ready(c);
  if (rc != SS_OK) return rc;
  return batch_autotune(c->b, trial_steps, choice);
}

int ss_batch_observables(ss_batch* b, int item, ss_obs* out) {
  if (!b) return fail(SS_ERR_ARG, "null batch");
  if (item < 0 || item >= b->n()) return fail(SS_ERR_ARG, "item out of range");
  if (!out) return fail(SS_ERR_ARG, "out is NULL");
  return problem_observables(b, item, out);
}

int ss_batch_destroy(ss_batch* b) {
  batch_free(b);
  return SS_OK;
}

}  // extern "C"
