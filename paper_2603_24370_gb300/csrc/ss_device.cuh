// ss_device.cuh -- device-side building blocks of the soliton relaxation kernels:
// the flow's device status record, compensated FP64 reductions, the 4th-order
// stencils and the Euler-Lagrange forces / energy densities of the two theories.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

// The per-site physics (densities, forces, energy differences, stencil arithmetic)
// is plain arithmetic, compiled for host and device so that host-only checks can
// exercise exactly the code the kernels run.
#define SS_HD __host__ __device__ __forceinline__

namespace ss {

// ------------------------------------------------------------------ tiling
// A tile is TX x TY output sites; a block of BX x BY threads covers it with each
// thread owning TY/BY sites of one column. The shared tile carries the width-2
// halo of the 5-point stencils (Sec. 3.1).
constexpr int TX = 32, TY = 16, BX = 32, BY = 8, NT = BX * BY;
constexpr int HALO = 2;
constexpr int SX = TX + 2 * HALO, SY = TY + 2 * HALO;
constexpr int ROWS_PER_THREAD = TY / BY;

enum { TH_AH = 1, TH_CM = 2, TH_BS = 3, TH_BEC = 4, TH_SID = 5, TH_CMD = 6 };

template <int TH> struct NComp;
template <> struct NComp<TH_AH> { static constexpr int C = 4; };
template <> struct NComp<TH_CM> { static constexpr int C = 3; };
template <> struct NComp<TH_BS> { static constexpr int C = 3; };
template <> struct NComp<TH_BEC> { static constexpr int C = 2; };
template <> struct NComp<TH_SID> { static constexpr int C = 6; };
template <> struct NComp<TH_CMD> { static constexpr int C = 3; };  // chiral magnet with demagnetisation

// Theories whose field is a unit 3-vector (projected onto the sphere).
template <int TH> struct UnitVector { static constexpr bool value = TH == TH_CM || TH == TH_BS || TH == TH_CMD; };

// ------------------------------------------------------------------ flow state
// One per context, in device memory. Written only by the single last-arriving
// block of a reduction kernel (or by 1-thread control kernels), read by the
// following launches in stream order.
struct DevState {
  double E_last;   // E_h of the previous head field (Eq. 4 compares against it)
  double E_cur;    // E_h of the current head field
  double dE;       // E_h(current) - E_h(previous field), cancellation-free (0 if none)
  double gmax;     // dx dy max_I |G| of the current head field
  double tol;      // convergence threshold on gmax (< 0 disables)
  long long steps;       // steps taken since the fields were set
  long long arrests;     // arrests since the fields were set
  long long head_step;   // value of `steps` when stage 1 last evaluated the field (-1: never)
  long long step_limit;  // stages 2-4 do nothing once steps >= step_limit
  int arrest;      // 1: the current velocity counts as zero (pending arrest)
  int converged;   // 1: gmax < tol; stage kernels become no-ops
  int nonfinite;   // 1: E or G not finite; stage kernels become no-ops
  int pad0;
  unsigned int ticket;      // arrival counter of the flow reduction
  unsigned int obs_ticket;  // arrival counter of the observables reduction
  // observables (FP64 evaluation)
  double obs_energy, obs_charge, obs_flux, obs_gmax_raw, obs_normdev;
  double obs_atoms, obs_lz;  // BEC: dx dy sum_I |psi|^2 and dx dy sum_I Re(psi* L_z psi)
  // BEC at a fixed atom number (ss_fixedn.cu)
  double mu_held;             // multiplier of the current field, held through its step's stages
  double fn_scale, fn_alpha;  // refresh in progress: psi <- s psi, v <- v - alpha psi
  long long fn_step;          // `steps` of the last refreshed field (-1: none)
  int fn_pending;             // 1 from the refresh's first kernel to its last
  unsigned int fn_ticket;     // arrival counter of the refresh kernels
};

struct FlowPartial {  // per-block part of the flow reduction (64 B)
  double es, ec;  // sum of e
  double ds, dc;  // sum of e(new) - e(previous)
  double m;       // max |G|
  double pad[3];
};
struct ObsPartial {  // per-block part of the observables reduction (64 B)
  double es, ec, fs, fc, qs, qc, gm, nd;
};

// ------------------------------------------------------------------ compensated sums
struct DD {
  double s, c;
};
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}
__device__ __forceinline__ DD dd_add(DD x, DD y) {
  double s, e;
  two_sum(x.s, y.s, s, e);
  return DD{s, x.c + y.c + e};
}
// Neumaier's compensated addition of one term.
__device__ __forceinline__ void neumaier(DD& a, double x) {
  const double t = a.s + x;
  if (fabs(a.s) >= fabs(x)) a.c += (a.s - t) + x; else a.c += (x - t) + a.s;
  a.s = t;
}
__device__ __forceinline__ DD shfl_down_dd(DD v, int off) {
  return DD{__shfl_down_sync(0xffffffffu, v.s, off), __shfl_down_sync(0xffffffffu, v.c, off)};
}
// Fixed-shape warp tree: lane 0 ends with the warp's value; the order never depends
// on timing, so results are bitwise reproducible.
__device__ __forceinline__ DD warp_sum(DD v) {
  for (int off = 16; off > 0; off >>= 1) v = dd_add(v, shfl_down_dd(v, off));
  return v;
}
// Maximum that propagates NaN (fmax would drop it and hide a blown-up force).
__device__ __forceinline__ double nanmax(double a, double b) { return (b > a || b != b) ? b : a; }
__device__ __forceinline__ double warp_max(double m) {
  for (int off = 16; off > 0; off >>= 1) m = nanmax(m, __shfl_down_sync(0xffffffffu, m, off));
  return m;
}

// Shared doubles that block_reduce<K, L> needs; every caller sizes its buffer
// with this so the two can never disagree.
template <int K, int L>
struct RedSmem {
  static constexpr int n = (NT / 32) * (2 * K + L);
};

// Block reduction of K compensated sums and L maxima over NT threads; thread 0
// returns the block result. sm must hold RedSmem<K, L>::n doubles.
template <int K, int L>
__device__ __forceinline__ void block_reduce(DD (&s)[K], double (&m)[L], double* sm) {
  constexpr int W = NT / 32;
  const int lane = threadIdx.x & 31, wid = (threadIdx.y * BX + threadIdx.x) >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) s[k] = warp_sum(s[k]);
#pragma unroll
  for (int l = 0; l < L; ++l) m[l] = warp_max(m[l]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) { sm[(2 * k) * W + wid] = s[k].s; sm[(2 * k + 1) * W + wid] = s[k].c; }
#pragma unroll
    for (int l = 0; l < L; ++l) sm[(2 * K + l) * W + wid] = m[l];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k)
      s[k] = lane < W ? DD{sm[(2 * k) * W + lane], sm[(2 * k + 1) * W + lane]} : DD{0.0, 0.0};
#pragma unroll
    for (int l = 0; l < L; ++l) m[l] = lane < W ? sm[(2 * K + l) * W + lane] : 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) s[k] = warp_sum(s[k]);
#pragma unroll
    for (int l = 0; l < L; ++l) m[l] = warp_max(m[l]);
  }
  __syncthreads();
}

// ------------------------------------------------------------------ FP32 compensated sums
// FP32 pairs keep reductions of FP32 kernels on the FP32 units: this GPU's FP64 rate
// is a small fraction of its FP32 rate, and an FP64 block reduction would stall the
// SM for microseconds.
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

// Block reduction in the working type: two compensated sums, one max.
template <typename R>
struct RPair {
  R s, c;
};
__device__ __forceinline__ RPair<float> pair_add(RPair<float> x, RPair<float> y) {
  float s, e;
  two_sum_f(x.s, y.s, s, e);
  return RPair<float>{s, x.c + y.c + e};
}
__device__ __forceinline__ RPair<double> pair_add(RPair<double> x, RPair<double> y) {
  double s, e;
  two_sum(x.s, y.s, s, e);
  return RPair<double>{s, x.c + y.c + e};
}
template <typename R>
__device__ __forceinline__ R rmax(R a, R b) {
  return (b > a || b != b) ? b : a;  // propagates NaN
}
// Block-wide: thread 0 ends with the block's two pairs and maximum. sm holds
// (NT / 32) * 5 values of R. Fixed shape: bitwise reproducible.
template <typename R>
__device__ __forceinline__ void tile_reduce(RPair<R>& a, RPair<R>& b, R& m, R* sm) {
  constexpr int W = NT / 32;
  const int lane = threadIdx.x & 31, wid = (threadIdx.y * BX + threadIdx.x) >> 5;
  for (int off = 16; off > 0; off >>= 1) {
    a = pair_add(a, RPair<R>{__shfl_down_sync(0xffffffffu, a.s, off), __shfl_down_sync(0xffffffffu, a.c, off)});
    b = pair_add(b, RPair<R>{__shfl_down_sync(0xffffffffu, b.s, off), __shfl_down_sync(0xffffffffu, b.c, off)});
    m = rmax(m, __shfl_down_sync(0xffffffffu, m, off));
  }
  if (lane == 0) {
    sm[wid] = a.s; sm[W + wid] = a.c; sm[2 * W + wid] = b.s; sm[3 * W + wid] = b.c; sm[4 * W + wid] = m;
  }
  __syncthreads();
  if (wid == 0) {
    a = lane < W ? RPair<R>{sm[lane], sm[W + lane]} : RPair<R>{R(0), R(0)};
    b = lane < W ? RPair<R>{sm[2 * W + lane], sm[3 * W + lane]} : RPair<R>{R(0), R(0)};
    m = lane < W ? sm[4 * W + lane] : R(0);
    for (int off = 16; off > 0; off >>= 1) {
      a = pair_add(a, RPair<R>{__shfl_down_sync(0xffffffffu, a.s, off), __shfl_down_sync(0xffffffffu, a.c, off)});
      b = pair_add(b, RPair<R>{__shfl_down_sync(0xffffffffu, b.s, off), __shfl_down_sync(0xffffffffu, b.c, off)});
      m = rmax(m, __shfl_down_sync(0xffffffffu, m, off));
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------ stencils
// Spacing factors of Eq. 1 / Eq. 2, precomputed per context in the working type.
template <typename R>
struct Spacing {
  R i12dx, i12dy;      // 1 / (12 dx), 1 / (12 dy)
  R i12dx2, i12dy2;    // 1 / (12 dx^2), 1 / (12 dy^2)
  R i144dxdy;          // 1 / (144 dx dy)
};

// Derivatives of one component at shared-tile position (sx, sy). Differences are
// formed first so that FP32 keeps the small differences of neighbouring values.
template <typename R>
struct Deriv {
  R v, fx, fy, fxx, fyy, fxy;
};

// Eq. 1 / Eq. 2 in x and y at tile position (sx, sy) of plane P (row stride SX).
template <typename R, bool SECOND, bool MIXED>
SS_HD Deriv<R> stencil(const R* P, int sx, int sy, const Spacing<R>& h) {
  Deriv<R> d;
  const R* r = P + sy * SX + sx;
  const R c = r[0];
  const R xm2 = r[-2], xm1 = r[-1], xp1 = r[1], xp2 = r[2];
  const R ym2 = r[-2 * SX], ym1 = r[-SX], yp1 = r[SX], yp2 = r[2 * SX];
  d.v = c;
  // Eq. 1: (-f_{+2} + 8 f_{+1} - 8 f_{-1} + f_{-2}) / (12 h) = (8 (f_{+1} - f_{-1}) - (f_{+2} - f_{-2})) / (12 h)
  d.fx = (R(8) * (xp1 - xm1) - (xp2 - xm2)) * h.i12dx;
  d.fy = (R(8) * (yp1 - ym1) - (yp2 - ym2)) * h.i12dy;
  if (SECOND) {
    // Eq. 2: (16 ((f_{+1} - f_0) + (f_{-1} - f_0)) - ((f_{+2} - f_0) + (f_{-2} - f_0))) / (12 h^2)
    d.fxx = (R(16) * ((xp1 - c) + (xm1 - c)) - ((xp2 - c) + (xm2 - c))) * h.i12dx2;
    d.fyy = (R(16) * ((yp1 - c) + (ym1 - c)) - ((yp2 - c) + (ym2 - c))) * h.i12dy2;
  } else {
    d.fxx = d.fyy = R(0);
  }
  if (MIXED) {
    // d_x d_y: Eq. 1 along y of the (unscaled) Eq. 1 along x.
    auto gx = [&](int dy) {
      const R* q = r + dy * SX;
      return R(8) * (q[1] - q[-1]) - (q[2] - q[-2]);
    };
    d.fxy = (R(8) * (gx(1) - gx(-1)) - (gx(2) - gx(-2))) * h.i144dxdy;
  } else {
    d.fxy = R(0);
  }
  return d;
}

// ------------------------------------------------------------------ theories
// Couplings in the working type. Abelian Higgs: c[0] = lambda, c[1] = u^2.
// Chiral magnet: c[0] = J, c[1] = D, c[2] = K, c[3] = h, c[4..6] = d_1, c[7..9] = d_2.
// Baby Skyrme: c[0] = kappa^2, c[1] = mu^2, c[2] = nu^2.
// BEC: c[0] = g, c[1] = Omega, c[2] = mu (chemical potential), c[3] = the held
// multiplier of the fixed-atom-number form (force only; set per tile from the flow
// record, 0 in the grand-canonical form).
// s+id: c[0..6] = a1, a2, b1, b2, b3, b4, nu.
// Chiral magnet with demagnetisation: the chiral magnet's c[0..9], c[10] = mu_d.
constexpr int NCOUP = 12;  // couplings per problem
template <typename R>
struct Couplings {
  R c[NCOUP];
};

// Abelian Higgs (Table 1): e = 1/2 |D psi|^2 + 1/2 B^2 + lambda/8 (u^2 - |psi|^2)^2,
// D_i = d_i - i A_i, B = d_1 A_2 - d_2 A_1. Components: 0 Re psi, 1 Im psi, 2 A_1, 3 A_2.
template <typename R>
SS_HD R density_ah(const Couplings<R>& k, const R* v, const R* fx, const R* fy) {
  const R p1 = v[0], p2 = v[1], A1 = v[2], A2 = v[3];
  const R re1 = fx[0] + A1 * p2, im1 = fx[1] - A1 * p1;
  const R re2 = fy[0] + A2 * p2, im2 = fy[1] - A2 * p1;
  const R B = fx[3] - fy[2];
  const R w = k.c[1] - (p1 * p1 + p2 * p2);
  return R(0.5) * (re1 * re1 + im1 * im1 + re2 * re2 + im2 * im2) + R(0.5) * B * B + k.c[0] * R(0.125) * w * w;
}

// Euler-Lagrange force of the Abelian Higgs energy:
//   G_psi = -lap psi + i (div A) psi + 2 i A_i d_i psi + |A|^2 psi - lambda/2 (u^2 - |psi|^2) psi
//   G_A1 = d_2 B + psi_2 d_1 psi_1 - psi_1 d_1 psi_2 + A_1 |psi|^2
//   G_A2 = -d_1 B + psi_2 d_2 psi_1 - psi_1 d_2 psi_2 + A_2 |psi|^2
template <typename R>
SS_HD void force_ah(const Couplings<R>& k, const R* v, const R* fx, const R* fy, const R* fxx,
                                         const R* fyy, const R* fxy, R* G) {
  const R p1 = v[0], p2 = v[1], A1 = v[2], A2 = v[3];
  const R divA = fx[2] + fy[3];
  const R AA = A1 * A1 + A2 * A2, mod2 = p1 * p1 + p2 * p2;
  const R pot = R(0.5) * k.c[0] * (k.c[1] - mod2);
  G[0] = -(fxx[0] + fyy[0]) - R(2) * (A1 * fx[1] + A2 * fy[1]) - divA * p2 + (AA - pot) * p1;
  G[1] = -(fxx[1] + fyy[1]) + R(2) * (A1 * fx[0] + A2 * fy[0]) + divA * p1 + (AA - pot) * p2;
  G[2] = (fxy[3] - fyy[2]) + (p2 * fx[0] - p1 * fx[1]) + A1 * mod2;
  G[3] = (fxy[2] - fxx[3]) + (p2 * fy[0] - p1 * fy[1]) + A2 * mod2;
}

template <typename R>
SS_HD void cross3(const R* a, const R* b, R* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// Chiral magnet (Eq. 5, no demag): e = J/2 |d n|^2 + D sum_i d_i . (n x d_i n)
//   + K (1 - n_3^2) + h (1 - n_3).
template <typename R>
SS_HD R density_cm(const Couplings<R>& k, const R* n, const R* fx, const R* fy) {
  R c1[3], c2[3];
  cross3(n, fx, c1);
  cross3(n, fy, c2);
  const R ex = R(0.5) * k.c[0] * (fx[0] * fx[0] + fx[1] * fx[1] + fx[2] * fx[2] + fy[0] * fy[0] + fy[1] * fy[1] +
                                  fy[2] * fy[2]);
  const R dmi = k.c[1] * (k.c[4] * c1[0] + k.c[5] * c1[1] + k.c[6] * c1[2] + k.c[7] * c2[0] + k.c[8] * c2[1] +
                          k.c[9] * c2[2]);
  const R one_m = R(1) - n[2];
  return ex + dmi + k.c[2] * one_m * (R(1) + n[2]) + k.c[3] * one_m;
}

// G = -J lap n - 2 D sum_i d_i x d_i n - 2 K n_3 e_3 - h e_3, then G <- G - (G.n) n.
template <typename R>
SS_HD void force_cm_raw(const Couplings<R>& k, const R* n, const R* fx, const R* fy, const R* fxx, const R* fyy,
                        R* G) {
  R c1[3], c2[3];
  const R d1[3] = {k.c[4], k.c[5], k.c[6]}, d2[3] = {k.c[7], k.c[8], k.c[9]};
  cross3(d1, fx, c1);
  cross3(d2, fy, c2);
  const R twoD = R(2) * k.c[1];
#pragma unroll
  for (int a = 0; a < 3; ++a) G[a] = -k.c[0] * (fxx[a] + fyy[a]) - twoD * (c1[a] + c2[a]);
  G[2] += -R(2) * k.c[2] * n[2] - k.c[3];
}
template <typename R>
SS_HD void project_tangent(const R* n, R* G) {
  const R gn = G[0] * n[0] + G[1] * n[1] + G[2] * n[2];
#pragma unroll
  for (int a = 0; a < 3; ++a) G[a] -= gn * n[a];
}
template <typename R>
SS_HD void force_cm(const Couplings<R>& k, const R* n, const R* fx, const R* fy, const R* fxx,
                                         const R* fyy, R* G) {
  force_cm_raw<R>(k, n, fx, fy, fxx, fyy, G);
  project_tangent<R>(n, G);
}

// Demagnetisation (Eq. 6) with psi = phi / (mu_0 M_s), lap psi = div n: the energy
// -mu_d/2 int psi rho (rho = d_1 n_1 + d_2 n_2) has the force mu_d (d_1 psi, d_2 psi, 0),
// added before the projection; psi is computed for the whole lattice (ss_demag.cu).
template <typename R>
SS_HD void force_cmd(const Couplings<R>& k, const R* n, const R* fx, const R* fy, const R* fxx, const R* fyy, R psx,
                     R psy, R* G) {
  force_cm_raw<R>(k, n, fx, fy, fxx, fyy, G);
  G[0] += k.c[10] * psx;
  G[1] += k.c[10] * psy;
  project_tangent<R>(n, G);
}

// Baby Skyrme (Table 1): e = 1/2 |d m|^2 + kappa^2/4 sum_{i,j} |d_i m x d_j m|^2 + V(m)
//   = 1/2 (|a|^2 + |b|^2) + kappa^2/2 |a x b|^2 + mu^2 (1 - m_3) + nu^2/2 m_1^2,
// with a = d_1 m, b = d_2 m (the double sum counts a x b twice).
template <typename R>
SS_HD R density_bs(const Couplings<R>& k, const R* m, const R* a, const R* b) {
  R X[3];
  cross3(a, b, X);
  const R sig = a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  return R(0.5) * sig + R(0.5) * k.c[0] * (X[0] * X[0] + X[1] * X[1] + X[2] * X[2]) + k.c[1] * (R(1) - m[2]) +
         R(0.5) * k.c[2] * m[0] * m[0];
}

// Euler-Lagrange force of the Baby Skyrme energy. The Skyrme term S = kappa^2/2
// (|a|^2 |b|^2 - (a.b)^2) contributes -d_1 dS/da - d_2 dS/db =
//   -kappa^2 [ |b|^2 m_11 + |a|^2 m_22 - 2 (a.b) m_12 + (b.m_12 - a.m_22) a + (a.m_12 - b.m_11) b ],
// the potential (nu^2 m_1, 0, -mu^2); then G <- G - (G.m) m.
template <typename R>
SS_HD void force_bs(const Couplings<R>& k, const R* m, const R* a, const R* b, const R* m11, const R* m22,
                    const R* m12, R* G) {
  const R aa = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
  const R bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  const R ab = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
  const R ca = (b[0] * m12[0] + b[1] * m12[1] + b[2] * m12[2]) - (a[0] * m22[0] + a[1] * m22[1] + a[2] * m22[2]);
  const R cb = (a[0] * m12[0] + a[1] * m12[1] + a[2] * m12[2]) - (b[0] * m11[0] + b[1] * m11[1] + b[2] * m11[2]);
#pragma unroll
  for (int c = 0; c < 3; ++c)
    G[c] = -(m11[c] + m22[c]) - k.c[0] * (bb * m11[c] + aa * m22[c] - R(2) * ab * m12[c] + ca * a[c] + cb * b[c]);
  G[0] += k.c[2] * m[0];
  G[2] -= k.c[1];
  const R gn = G[0] * m[0] + G[1] * m[1] + G[2] * m[2];
#pragma unroll
  for (int c = 0; c < 3; ++c) G[c] -= gn * m[c];
}

// Rotating trapped BEC (Table 1), dimensionless (hbar = m = omega = 1), in the
// grand-canonical form at chemical potential mu, psi = u + i v, D = x d_y - y d_x:
//   e = 1/2 |grad psi|^2 + (r^2/2 + g/2 |psi|^2 - mu) |psi|^2 - Omega (u D v - v D u)
// (u D v - v D u is the real part of psi* L_z psi; the imaginary part is a total
// derivative). (x, y) is the site's position, origin at the grid centre.
template <typename R>
SS_HD R density_bec(const Couplings<R>& k, const R* v, const R* fx, const R* fy, R x, R y) {
  const R n = v[0] * v[0] + v[1] * v[1];
  const R Du = x * fy[0] - y * fx[0], Dv = x * fy[1] - y * fx[1];
  const R kin = R(0.5) * (fx[0] * fx[0] + fy[0] * fy[0] + fx[1] * fx[1] + fy[1] * fy[1]);
  return kin + (R(0.5) * (x * x + y * y) + R(0.5) * k.c[0] * n - k.c[2]) * n - k.c[1] * (v[0] * Dv - v[1] * Du);
}

// G_u = -lap u + (r^2 + 2 g |psi|^2 - 2 mu) u - 2 Omega D v,
// G_v = -lap v + (r^2 + 2 g |psi|^2 - 2 mu) v + 2 Omega D u,
// with mu = c[2] + c[3] (the held multiplier at a fixed atom number).
template <typename R>
SS_HD void force_bec(const Couplings<R>& k, const R* v, const R* fx, const R* fy, const R* fxx, const R* fyy, R x,
                     R y, R* G) {
  const R w = (x * x + y * y) + R(2) * k.c[0] * (v[0] * v[0] + v[1] * v[1]) - R(2) * (k.c[2] + k.c[3]);
  const R Du = x * fy[0] - y * fx[0], Dv = x * fy[1] - y * fx[1];
  G[0] = -(fxx[0] + fyy[0]) + w * v[0] - R(2) * k.c[1] * Dv;
  G[1] = -(fxx[1] + fyy[1]) + w * v[1] + R(2) * k.c[1] * Du;
}

// s+id two-band superconductor (Table 1), components (Re, Im Delta_s, Re, Im Delta_d,
// A_1, A_2), D = d - i A. Gradient tensor: identity within each band, nu diag(1, -1)
// between the bands (d_{x^2-y^2}). With X_aj = d_j u_a + A_j w_a, Y_aj = d_j w_a - A_j u_a
// (real and imaginary parts of D_j Delta_a), S = |Delta_s|^2, D = |Delta_d|^2 and
// p + i q = Delta_s conj(Delta_d):
//   e = 1/2 sum (X^2 + Y^2) + nu sum_j eta_j (X_sj X_dj + Y_sj Y_dj) + B^2 / 2
//       + a1 S + a2 D + b1 S^2 + b2 D^2 + b3 S D + 2 b4 (p^2 - q^2),   eta = (1, -1).
template <typename R>
SS_HD R density_sid(const Couplings<R>& k, const R* v, const R* fx, const R* fy) {
  const R A1 = v[4], A2 = v[5];
  const R Xs1 = fx[0] + A1 * v[1], Ys1 = fx[1] - A1 * v[0], Xs2 = fy[0] + A2 * v[1], Ys2 = fy[1] - A2 * v[0];
  const R Xd1 = fx[2] + A1 * v[3], Yd1 = fx[3] - A1 * v[2], Xd2 = fy[2] + A2 * v[3], Yd2 = fy[3] - A2 * v[2];
  const R grad = R(0.5) * (Xs1 * Xs1 + Ys1 * Ys1 + Xs2 * Xs2 + Ys2 * Ys2 + Xd1 * Xd1 + Yd1 * Yd1 + Xd2 * Xd2 +
                           Yd2 * Yd2);
  const R mix = (Xs1 * Xd1 + Ys1 * Yd1) - (Xs2 * Xd2 + Ys2 * Yd2);
  const R B = fx[5] - fy[4];
  const R S = v[0] * v[0] + v[1] * v[1], D = v[2] * v[2] + v[3] * v[3];
  const R p = v[0] * v[2] + v[1] * v[3], q = v[1] * v[2] - v[0] * v[3];
  return grad + k.c[6] * mix + R(0.5) * B * B + k.c[0] * S + k.c[1] * D + k.c[2] * S * S + k.c[3] * D * D +
         k.c[4] * S * D + R(2) * k.c[5] * (p * p - q * q);
}

// s+id force: with the conjugates P_aj = X_aj + nu eta_j X_bj, Q_aj = Y_aj + nu eta_j Y_bj
// (b the other band) and d_j X_aj = d_j^2 u_a + (d_j A_j) w_a + A_j d_j w_a,
// d_j Y_aj = d_j^2 w_a - (d_j A_j) u_a - A_j d_j u_a:
//   G_{u_a} = dV/du_a - sum_j (A_j Q_aj + d_j P_aj),  G_{w_a} = dV/dw_a + sum_j (A_j P_aj - d_j Q_aj),
//   G_{A_1} = d_2 B + sum_a (P_a1 w_a - Q_a1 u_a),   G_{A_2} = -d_1 B + sum_a (P_a2 w_a - Q_a2 u_a).
template <typename R>
SS_HD void force_sid(const Couplings<R>& k, const R* v, const R* fx, const R* fy, const R* fxx, const R* fyy,
                     const R* fxy, R* G) {
  const R A[2] = {v[4], v[5]}, dA[2] = {fx[4], fy[5]};
  const R nu = k.c[6];
  R X[2][2], Y[2][2], dX[2][2], dY[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const R u = v[2 * a], w = v[2 * a + 1];
    const R du[2] = {fx[2 * a], fy[2 * a]}, dw[2] = {fx[2 * a + 1], fy[2 * a + 1]};
    const R uu[2] = {fxx[2 * a], fyy[2 * a]}, ww[2] = {fxx[2 * a + 1], fyy[2 * a + 1]};
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      X[a][j] = du[j] + A[j] * w;
      Y[a][j] = dw[j] - A[j] * u;
      dX[a][j] = uu[j] + dA[j] * w + A[j] * dw[j];
      dY[a][j] = ww[j] - dA[j] * u - A[j] * du[j];
    }
  }
  const R s1 = v[0], s2 = v[1], d1 = v[2], d2 = v[3];
  const R S = s1 * s1 + s2 * s2, D = d1 * d1 + d2 * d2;
  const R p = s1 * d1 + s2 * d2, q = s2 * d1 - s1 * d2;
  const R cs = R(2) * k.c[0] + R(4) * k.c[2] * S + R(2) * k.c[4] * D;
  const R cd = R(2) * k.c[1] + R(4) * k.c[3] * D + R(2) * k.c[4] * S;
  const R f4 = R(4) * k.c[5];
  R dV[4];
  dV[0] = cs * s1 + f4 * (p * d1 + q * d2);
  dV[1] = cs * s2 + f4 * (p * d2 - q * d1);
  dV[2] = cd * d1 + f4 * (p * s1 - q * s2);
  dV[3] = cd * d2 + f4 * (p * s2 + q * s1);
  G[4] = fxy[5] - fyy[4];
  G[5] = fxy[4] - fxx[5];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const int b = 1 - a;
    const R u = v[2 * a], w = v[2 * a + 1];
    R gu = dV[2 * a], gw = dV[2 * a + 1];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const R nj = j == 0 ? nu : -nu;
      const R P = X[a][j] + nj * X[b][j], Q = Y[a][j] + nj * Y[b][j];
      const R dP = dX[a][j] + nj * dX[b][j], dQ = dY[a][j] + nj * dY[b][j];
      gu -= A[j] * Q + dP;
      gw += A[j] * P - dQ;
      G[4 + j] += P * w - Q * u;
    }
    G[2 * a] = gu;
    G[2 * a + 1] = gw;
  }
}

// ------------------------------------------------------------------ energy differences
// Eq. 4 compares E_h(phi^{n+1}) with E_h(phi^n). Both energy densities are
// polynomials in (phi, d phi), so with a = phi^{n+1} and delta = phi^{n+1} - phi^n
// (exact in floating point: neighbouring values) the per-site difference
// e(a) - e(a - delta) expands exactly in delta and its derivatives. Evaluated in
// this form its rounding error is relative to the difference itself, not to e, so
// the arrest decision stays meaningful when the energy changes by far less than
// the rounding of e (FP32 near convergence). Identities used: for any Z that is a
// polynomial of the fields, Z(a)^2 - Z(a - delta)^2 = (2 Z(a) - dZ) dZ with
// dZ = Z(a) - Z(a - delta) written out exactly.

// Abelian Higgs: X_i = d_i psi_1 + A_i psi_2, Y_i = d_i psi_2 - A_i psi_1,
// B = d_1 A_2 - d_2 A_1, w = u^2 - |psi|^2; e = (X^2 + Y^2 + B^2)/2 + lambda/8 w^2.
template <typename R>
SS_HD R delta_density_ah(const Couplings<R>& k, const R* a, const R* ax, const R* ay,
                                              const R* d, const R* dx, const R* dy) {
  const R p1 = a[0], p2 = a[1], A1 = a[2], A2 = a[3];
  const R q1 = d[0], q2 = d[1], B1 = d[2], B2 = d[3];
  // new values
  const R X1 = ax[0] + A1 * p2, Y1 = ax[1] - A1 * p1;
  const R X2 = ay[0] + A2 * p2, Y2 = ay[1] - A2 * p1;
  const R B = ax[3] - ay[2];
  const R w = k.c[1] - (p1 * p1 + p2 * p2);
  // exact differences: A_i psi_c - (A_i - B_i)(psi_c - q_c) = A_i q_c + B_i psi_c - B_i q_c
  const R dX1 = dx[0] + (A1 * q2 + B1 * (p2 - q2));
  const R dY1 = dx[1] - (A1 * q1 + B1 * (p1 - q1));
  const R dX2 = dy[0] + (A2 * q2 + B2 * (p2 - q2));
  const R dY2 = dy[1] - (A2 * q1 + B2 * (p1 - q1));
  const R dB = dx[3] - dy[2];
  const R dw = -(q1 * (R(2) * p1 - q1) + q2 * (R(2) * p2 - q2));
  return R(0.5) * ((R(2) * X1 - dX1) * dX1 + (R(2) * Y1 - dY1) * dY1 + (R(2) * X2 - dX2) * dX2 +
                   (R(2) * Y2 - dY2) * dY2 + (R(2) * B - dB) * dB) +
         k.c[0] * R(0.125) * (R(2) * w - dw) * dw;
}

// Chiral magnet: every term is at most quadratic in (n, d n):
//   exchange  J sum_i d_i delta . (d_i a - d_i delta / 2)
//   DMI       D sum_i d_i . (a x d_i delta + delta x d_i a - delta x d_i delta)
//   anisotropy -K delta_3 (2 a_3 - delta_3),  Zeeman -h delta_3.
template <typename R>
SS_HD R delta_density_cm(const Couplings<R>& k, const R* a, const R* ax, const R* ay,
                                              const R* d, const R* dx, const R* dy) {
  R ex = R(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) ex += dx[c] * (ax[c] - R(0.5) * dx[c]) + dy[c] * (ay[c] - R(0.5) * dy[c]);
  R u1[3], u2[3], u3[3], w1[3], w2[3], w3[3];
  cross3(a, dx, u1);
  cross3(d, ax, u2);
  cross3(d, dx, u3);
  cross3(a, dy, w1);
  cross3(d, ay, w2);
  cross3(d, dy, w3);
  R dmi = R(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) dmi += k.c[4 + c] * (u1[c] + u2[c] - u3[c]) + k.c[7 + c] * (w1[c] + w2[c] - w3[c]);
  return k.c[0] * ex + k.c[1] * dmi - k.c[2] * d[2] * (R(2) * a[2] - d[2]) - k.c[3] * d[2];
}

// Baby Skyrme: with X = a_x x a_y of the new field and the exact difference
//   dX = X(a) - X(a - delta) = a_x x delta_y + delta_x x a_y - delta_x x delta_y,
//   sigma     sum_i d_i delta . (d_i a - d_i delta / 2)
//   Skyrme    kappa^2/2 (2 X - dX) . dX
//   potential -mu^2 delta_3 + nu^2/2 delta_1 (2 a_1 - delta_1).
template <typename R>
SS_HD R delta_density_bs(const Couplings<R>& k, const R* a, const R* ax, const R* ay, const R* d, const R* dx,
                         const R* dy) {
  R sig = R(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) sig += dx[c] * (ax[c] - R(0.5) * dx[c]) + dy[c] * (ay[c] - R(0.5) * dy[c]);
  R X[3], u1[3], u2[3], u3[3];
  cross3(ax, ay, X);
  cross3(ax, dy, u1);
  cross3(dx, ay, u2);
  cross3(dx, dy, u3);
  R sky = R(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const R dX = u1[c] + u2[c] - u3[c];
    sky += (R(2) * X[c] - dX) * dX;
  }
  return sig + R(0.5) * k.c[0] * sky - k.c[1] * d[2] + R(0.5) * k.c[2] * d[0] * (R(2) * a[0] - d[0]);
}

// BEC: with n = |psi|^2 and the exact difference dn = sum_c delta_c (2 a_c - delta_c),
//   kinetic   sum_i d_i delta . (d_i a - d_i delta / 2)
//   trap      r^2/2 dn,  interaction g/2 (2 n - dn) dn,  chemical potential -mu dn
//   rotation  -Omega [B(a, delta) + B(delta, a) - B(delta, delta)],
// B(p, q) = p_u D q_v - p_v D q_u being bilinear with B(a, a) the rotation density.
template <typename R>
SS_HD R delta_density_bec(const Couplings<R>& k, const R* a, const R* ax, const R* ay, const R* d, const R* dx,
                          const R* dy, R x, R y) {
  R kin = R(0);
#pragma unroll
  for (int c = 0; c < 2; ++c) kin += dx[c] * (ax[c] - R(0.5) * dx[c]) + dy[c] * (ay[c] - R(0.5) * dy[c]);
  const R n = a[0] * a[0] + a[1] * a[1];
  const R dn = d[0] * (R(2) * a[0] - d[0]) + d[1] * (R(2) * a[1] - d[1]);
  const R Da0 = x * ay[0] - y * ax[0], Da1 = x * ay[1] - y * ax[1];
  const R Dd0 = x * dy[0] - y * dx[0], Dd1 = x * dy[1] - y * dx[1];
  const R rot = (a[0] * Dd1 - a[1] * Dd0) + (d[0] * Da1 - d[1] * Da0) - (d[0] * Dd1 - d[1] * Dd0);
  return kin + (R(0.5) * (x * x + y * y) - k.c[2]) * dn + R(0.5) * k.c[0] * (R(2) * n - dn) * dn - k.c[1] * rot;
}

// s+id: exact differences of every factor (the Abelian Higgs identities per band),
//   dX_aj = d_j delta_u + A_j delta_w + delta_A_j (w - delta_w),
//   dY_aj = d_j delta_w - A_j delta_u - delta_A_j (u - delta_u),
// then 1/2 (2 X - dX) dX per square, X_s X_d - X_s' X_d' = dX_s X_d + X_s dX_d - dX_s dX_d
// for the mixed products, and likewise for S, D, p, q in the potential.
template <typename R>
SS_HD R delta_density_sid(const Couplings<R>& k, const R* a, const R* ax, const R* ay, const R* d, const R* dx,
                          const R* dy) {
  const R A[2] = {a[4], a[5]}, dA[2] = {d[4], d[5]};
  R X[2][2], Y[2][2], eX[2][2], eY[2][2];
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const R u = a[2 * b], w = a[2 * b + 1], du = d[2 * b], dw = d[2 * b + 1];
    const R gu[2] = {ax[2 * b], ay[2 * b]}, gw[2] = {ax[2 * b + 1], ay[2 * b + 1]};
    const R hu[2] = {dx[2 * b], dy[2 * b]}, hw[2] = {dx[2 * b + 1], dy[2 * b + 1]};
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      X[b][j] = gu[j] + A[j] * w;
      Y[b][j] = gw[j] - A[j] * u;
      eX[b][j] = hu[j] + (A[j] * dw + dA[j] * (w - dw));
      eY[b][j] = hw[j] - (A[j] * du + dA[j] * (u - du));
    }
  }
  R sq = R(0), mix = R(0);
#pragma unroll
  for (int j = 0; j < 2; ++j) {
#pragma unroll
    for (int b = 0; b < 2; ++b) sq += (R(2) * X[b][j] - eX[b][j]) * eX[b][j] + (R(2) * Y[b][j] - eY[b][j]) * eY[b][j];
    const R m = (eX[0][j] * X[1][j] + X[0][j] * eX[1][j] - eX[0][j] * eX[1][j]) +
                (eY[0][j] * Y[1][j] + Y[0][j] * eY[1][j] - eY[0][j] * eY[1][j]);
    mix += j == 0 ? m : -m;
  }
  const R B = ax[5] - ay[4], dB = dx[5] - dy[4];
  const R s1 = a[0], s2 = a[1], d1 = a[2], d2 = a[3];
  const R e1 = d[0], e2 = d[1], f1 = d[2], f2 = d[3];
  const R S = s1 * s1 + s2 * s2, D = d1 * d1 + d2 * d2;
  const R dS = e1 * (R(2) * s1 - e1) + e2 * (R(2) * s2 - e2);
  const R dD = f1 * (R(2) * d1 - f1) + f2 * (R(2) * d2 - f2);
  const R p = s1 * d1 + s2 * d2, q = s2 * d1 - s1 * d2;
  const R dp = (e1 * d1 + s1 * f1 - e1 * f1) + (e2 * d2 + s2 * f2 - e2 * f2);
  const R dq = (e2 * d1 + s2 * f1 - e2 * f1) - (e1 * d2 + s1 * f2 - e1 * f2);
  return R(0.5) * sq + k.c[6] * mix + R(0.5) * (R(2) * B - dB) * dB + k.c[0] * dS + k.c[1] * dD +
         k.c[2] * (R(2) * S - dS) * dS + k.c[3] * (R(2) * D - dD) * dD + k.c[4] * (dS * D + S * dD - dS * dD) +
         R(2) * k.c[5] * ((R(2) * p - dp) * dp - (R(2) * q - dq) * dq);
}

// Energy density, force and energy difference of theory TH. (x, y) carries the
// site-dependent extras: the BEC's site position; for the chiral magnet with
// demagnetisation the potential psi (density), its gradient (d_1 psi, d_2 psi) (force),
// and (psi, psi - psi_prev) (energy difference). Its magnetostatic part is written
// -mu_d/2 (rho - rho') (psi + psi'), which sums to E_ms(new) - E_ms(old) because the
// inverse Laplacian is symmetric: the small charge difference rho - rho' is formed
// exactly from the field difference, so the solver's rounding of psi enters relative
// to the energy change (the difference psi - psi' of two solves would carry it relative
// to E_ms and decide arrests by noise near convergence).
template <int TH, typename R>
SS_HD R density_at(const Couplings<R>& k, const R* v, const R* fx, const R* fy, R x = R(0), R y = R(0)) {
  if (TH == TH_CMD) return density_cm<R>(k, v, fx, fy) - R(0.5) * k.c[10] * x * (fx[0] + fy[1]);
  if (TH == TH_AH) return density_ah<R>(k, v, fx, fy);
  if (TH == TH_CM) return density_cm<R>(k, v, fx, fy);
  if (TH == TH_BS) return density_bs<R>(k, v, fx, fy);
  if (TH == TH_SID) return density_sid<R>(k, v, fx, fy);
  return density_bec<R>(k, v, fx, fy, x, y);
}
template <int TH, typename R>
SS_HD R delta_density_at(const Couplings<R>& k, const R* a, const R* ax, const R* ay, const R* d, const R* dx,
                         const R* dy, R x = R(0), R y = R(0)) {
  if (TH == TH_CMD)
    return delta_density_cm<R>(k, a, ax, ay, d, dx, dy) - R(0.5) * k.c[10] * (dx[0] + dy[1]) * (R(2) * x - y);
  if (TH == TH_AH) return delta_density_ah<R>(k, a, ax, ay, d, dx, dy);
  if (TH == TH_CM) return delta_density_cm<R>(k, a, ax, ay, d, dx, dy);
  if (TH == TH_BS) return delta_density_bs<R>(k, a, ax, ay, d, dx, dy);
  if (TH == TH_SID) return delta_density_sid<R>(k, a, ax, ay, d, dx, dy);
  return delta_density_bec<R>(k, a, ax, ay, d, dx, dy, x, y);
}
template <int TH, typename R>
SS_HD void force_of(const Couplings<R>& k, const R* v, const R* fx, const R* fy, const R* fxx, const R* fyy,
                    const R* fxy, R* G, R x = R(0), R y = R(0)) {
  if (TH == TH_AH) force_ah<R>(k, v, fx, fy, fxx, fyy, fxy, G);
  else if (TH == TH_CM) force_cm<R>(k, v, fx, fy, fxx, fyy, G);
  else if (TH == TH_CMD) force_cmd<R>(k, v, fx, fy, fxx, fyy, x, y, G);
  else if (TH == TH_BS) force_bs<R>(k, v, fx, fy, fxx, fyy, fxy, G);
  else if (TH == TH_SID) force_sid<R>(k, v, fx, fy, fxx, fyy, fxy, G);
  else force_bec<R>(k, v, fx, fy, fxx, fyy, x, y, G);
}

}  // namespace ss
