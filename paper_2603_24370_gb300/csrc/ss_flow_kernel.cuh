// ss_flow_kernel.cuh -- the arrested-Newton-flow step (arxiv 2603.24370, Sec. 3.2) as two
// fused passes over a batch of relaxation problems, and the gradient-descent step
// it is compared with as a third pass built from the same parts.
//
// One RK4 step of phi'' = -G(phi) (Eq. 3) on the first-order system (phi, v), with
// k_vi = -G(Y_i) at the stage inputs
//   Y_1 = phi,                       Y_2 = phi + dt/2 v,
//   Y_3 = phi + dt/2 v + dt^2/4 k_v1, Y_4 = phi + dt v + dt^2/2 k_v2,
//   phi' = phi + dt v + dt^2/6 (k_v1 + k_v2 + k_v3),
//   v'   = v + dt/6 (k_v1 + 2 k_v2 + 2 k_v3 + k_v4),
// is the textbook (k_phi, k_v) form with every k_phi eliminated. Y_1 and Y_2 need
// only (phi, v); Y_3 and Y_4 need only (phi, v, k_v1, k_v2). So a step is two passes
// with the ordinary width-2 halo and no recomputation:
//   pass 1  (stages 1, 2): reads phi, v (and phi^{n-1}), writes k_v1, k_v2;
//   pass 2  (stages 3, 4): reads phi, v, k_v1, k_v2, writes phi', v'
// (k_v3, k_v4 live in registers). Chiral magnet: every Y_i and phi' are normalised
// and v' tangent-projected (Sec. 3.2, constraint projection).
//
// Batches: every launch covers the tiles of all problems of a batch (uneven grid
// sizes and couplings, one theory and precision). Each tile reads its problem's
// descriptor; each problem selects its ping-pong buffers from its own step count,
// stops on its own (converged, non-finite, step limit), and its tiles are skipped
// from then on. A single-grid context is a batch of one.
//
// Pass 1 also reduces, per problem, E_h(phi), dx dy max|G| and the energy change
// since the previous field, dE = sum_I [e(phi^n) - e(phi^{n-1})], in the
// cancellation-free form of ss_device.cuh (phi^{n-1} is still intact in the other
// ping-pong buffer): a compensated pair per thread, summed over a block's run of
// consecutive tiles of one problem and reduced into a partial (one per run; a single
// problem has one run per block); the last arrival (arrival counter) sums the
// problem's partials in a fixed order (bitwise reproducible for a given grid) and
// decides on the device, with no host round trip:
//   arrest    = dE > 0, i.e. E_h(phi^n) > E_h(phi^{n-1})   (Eq. 4)
//   converged = dx dy max|G| < tol
// Pass 1 computes k_v2 with v before the arrest is known. That is exact either way:
// when the step is arrested v counts as zero, so Y_2 = Y_1 and k_v2 = k_v1, and
// pass 2 simply reads k_v1 in place of k_v2 (and zero in place of v).
//
// Compensated FP32 (LO): the field is stored as two FP32 planes, phi = hi + lo with
// |lo| <= ulp(hi)/2, and pass 2 adds each step's increment to lo and re-splits by
// TwoSum, so increments far below an ulp of the field still accumulate. With a
// single FP32 plane they are rounded away once the flow is slow, and the flow
// stalls above dx dy max|G| ~ 1e-6 while arresting every other step. The stage
// inputs are formed as hi + (lo + increment), normalised in split form for the
// chiral magnet, and rounded once to FP32 for the stencils.
//
// Gradient descent (pass 3), the first-order alternative Sec. 3.2 sets the flow
// against, read as the explicit Euler step of d phi / d tau = -G(phi):
//   phi^{n+1} = phi^n - dtau G(phi^n)   (chiral magnet: renormalised),
// one launch per step with the same tile staging, stencils, forces, reductions and
// device-side decision as pass 1: it reads phi^n, writes -G into k_v1 (so the
// force of the head field is always at hand) and phi^{n+1} into the other buffer,
// and the last tile of a problem advances its step count unless the field it
// evaluated has converged or the step budget is spent. Nothing is arrested; a rise
// E_h(phi^n) > E_h(phi^{n-1}) is counted (it means dtau is past the stability limit).
// The rise is judged on the two working-precision sums, not in the cancellation-free
// form of pass 1: that needs phi^{n-1}, whose buffer this launch is overwriting.
//
// Per block a tile of TX x TY sites is staged in shared memory with its halo, the
// stage inputs formed while loading (two sites per iteration, loads first). Each
// thread then walks RY rows of one column with a 5-row register window per
// component. Blocks stride over the batch's tiles; the grid is occupancy x SMs.
#pragma once
#include "ss_internal.h"
#include "ss_pack.cuh"

// Launch-shape knobs of the three passes: sites staged per iteration of the tile
// loading loop (their loads are all issued before any is used), and the resident
// blocks per SM the register allocation of the single-problem chiral-magnet FP32
// kernels must allow (1: no constraint; the other instances, whose descriptors
// occupy registers or whose working type is wider, would spill and keep their
// natural allocation).
// Defaults measured best at 4096^2: pass 1 gains 4% from 3 blocks / SM with two
// sites in flight, pass 2 6% from three sites in flight at 4 blocks / SM (against two
// at 5), the descent pass 4% from three sites in flight at 5 blocks / SM (against four
// at 6).
#ifndef SS_LU1
#define SS_LU1 2
#endif
// FP32 pass 1 sums E_h itself every SS_E_EVERY steps (a power of two), and on the first
// and last field of a run.
#ifndef SS_E_EVERY
#define SS_E_EVERY 16
#endif
// Vector staging units a thread's loop takes in one unrolled step in passes 1 / 2 / 3
// (their loads may be issued together).
#ifndef SS_VUNR1
#define SS_VUNR1 1
#endif
#ifndef SS_VUNR2
#define SS_VUNR2 1
#endif
#ifndef SS_VUNR3
#define SS_VUNR3 1
#endif
// Vector staging of passes 1 / 2 / 3 leaves out the units no stencil reads (1) or
// stages whole shared rows (0). At 4096^2 (chiral magnet, compensated; one GPU, both
// builds) leaving them out took pass 2 from 0.441 to 0.436 ms and the descent pass from
// 0.254 to 0.251 ms, and slowed pass 1 from 0.424 to 0.433 ms. (Forming pass 2's two
// stage inputs of a staged site as one packed pair measured 1% slower than the two
// scalar evaluations.)
#ifndef SS_VSKIP1
#define SS_VSKIP1 0
#endif
#ifndef SS_VSKIP2
#define SS_VSKIP2 1
#endif
#ifndef SS_VSKIP3
#define SS_VSKIP3 1
#endif
// FP32 pass 2 loads a site's stored values for the RK4 combination before computing
// the site's stage forces (1) or after them (0).
#ifndef SS_PF2
#define SS_PF2 0
#endif
#ifndef SS_LU2
#define SS_LU2 3
#endif
#ifndef SS_LU3
#define SS_LU3 3
#endif
#ifndef SS_MINB1
#define SS_MINB1 3
#endif
// Vector staging of tiles at the grid's edge, per pass (0: those take the scalar path).
#ifndef SS_VEDGE
#define SS_VEDGE 1
#endif
#ifndef SS_VEDGE1
#define SS_VEDGE1 SS_VEDGE
#endif
#ifndef SS_VEDGE2
#define SS_VEDGE2 SS_VEDGE
#endif
#ifndef SS_VEDGE3
#define SS_VEDGE3 SS_VEDGE
#endif
// Width (2 or 4 sites) of the vector units that stage tiles of FP32 grids whose rows
// start on 16-byte boundaries: compensated storage, plain FP32.
#ifndef SS_VW_LO
#define SS_VW_LO 2
#endif
#ifndef SS_VW_PLAIN
#define SS_VW_PLAIN 4
#endif
#ifndef SS_VW1_LO
#define SS_VW1_LO SS_VW_LO
#endif
#ifndef SS_VW2_LO
#define SS_VW2_LO SS_VW_LO
#endif
#ifndef SS_VW3_LO
#define SS_VW3_LO SS_VW_LO
#endif
#ifndef SS_MINB2
#define SS_MINB2 4
#endif
#ifndef SS_MINB3
#define SS_MINB3 5
#endif
// The kernels those bounds apply to: the FP32 kernels of theory SS_MINB_THEORY (a TH_*
// value; default the chiral magnet), single-problem launches, and batched launches too
// when SS_MINB_BATCH is 1. A theory's translation unit may set all of these before
// including this header.
#ifndef SS_MINB_THEORY
#define SS_MINB_THEORY 2
#endif
#ifndef SS_MINB_BATCH
#define SS_MINB_BATCH 0
#endif
// Batched launches may take bounds of their own (default: the single-problem ones).
#ifndef SS_MINB1B
#define SS_MINB1B SS_MINB1
#endif
#ifndef SS_MINB2B
#define SS_MINB2B SS_MINB2
#endif
#ifndef SS_MINB3B
#define SS_MINB3B SS_MINB3
#endif


namespace ss {

// Tile shape: TS = 0 (small) or 1 (large) selects the rows each thread walks,
// FP32 2 or 4 (tiles of 32 x 16 or 32 x 32 sites), FP64 1 or 2 (32 x 8 or 32 x 16).
// Shared rows: FP32 tiles keep 4 columns on each side (the stencils use 2), so that
// every row starts on a 16-byte boundary and the tile can be staged in float4 units;
// OX is the shared column of the tile's first site.
template <typename R, int TS>
struct FlowTile {
  static constexpr int RY = (sizeof(R) == 4 ? 2 : 1) << TS;  // rows per thread
  static constexpr int TX = 32, TY = BY * RY;
  static constexpr int OX = sizeof(R) == 4 ? 4 : 2;
  static constexpr int SX = TX + 2 * OX, SY = TY + 4, SXY = SX * SY;
  static constexpr int SW = TX + 4;  // staged sites per row (the tile and its halo)
};



// 1 / |n| for the unit-length projection: FP32 uses the hardware reciprocal square
// root refined by one Newton-Raphson step (y <- y (3 - x y^2) / 2), FP64 divides.
__device__ __forceinline__ float inv_norm(float x) {
  float y = rsqrtf(x);
  return y * (1.5f - 0.5f * x * y * y);
}
__device__ __forceinline__ double inv_norm(double x) { return 1.0 / sqrt(x); }

template <int C, typename R>
__device__ __forceinline__ void normalise(R* y) {
  const R s = inv_norm(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
#pragma unroll
  for (int c = 0; c < C; ++c) y[c] *= s;
}

// Split-form projection onto the unit sphere: given hi (FP32) and a small part t,
// return t' with hi + t' = (hi + t) / |hi + t| to about eps^2. With
// eta = |hi + t|^2 - 1 = (|hi|^2 - 1) + 2 hi.t + |t|^2, where |hi|^2 - 1 is formed
// exactly (error-free products and sums), 1/|hi + t| = 1 + rho with
// rho = -eta / (r (1 + r)), r = sqrt(1 + eta), and t' = t + rho (hi + t).
// rho enters only as a correction of size |eta| / 2, so a few ulps of relative
// error in it are harmless: r comes from the hardware reciprocal square root
// (r = x rsqrt(x)) and the quotient from the fast division, which keeps the IEEE
// division's range checks and slow path out of the kernels' inner loops.
__device__ __forceinline__ void normalise_split(const float* hi, float* t) {
  float p[3], e[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    p[c] = hi[c] * hi[c];
    e[c] = fmaf(hi[c], hi[c], -p[c]);
  }
  float s01, e01, s012, e012;
  two_sum_f(p[0], p[1], s01, e01);
  two_sum_f(s01, p[2], s012, e012);
  const float q = (s012 - 1.0f) + (e01 + e012 + e[0] + e[1] + e[2]);  // s012 - 1 is exact near 1
  const float ht = hi[0] * t[0] + hi[1] * t[1] + hi[2] * t[2];
  const float tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  const float eta = q + (2.0f * ht + tt);
  const float x = 1.0f + eta;
  const float r = x * rsqrtf(x);
  const float rho = __fdividef(-eta, r * (1.0f + r));
#pragma unroll
  for (int c = 0; c < 3; ++c) t[c] = t[c] + rho * (hi[c] + t[c]);
}

// Stage inputs of one site from its stored values: pass 1 Y_1 = phi, Y_2 = phi + dt/2 v
// and delta = phi^n - phi^{n-1}; pass 2 Y_3, Y_4; pass 3 phi. With compensated storage
// the small parts are formed first and added to the value once; unit vectors are
// normalised (split form) at sites of the interior.
template <int TH, typename R, int PASS, bool LO>
__device__ __forceinline__ void stage_site(const R* pv, const R* lv, const R* vv, const R* k1v, const R* k2v,
                                           const R* pp, const R* lp, bool inside, R hdt, R dt, R c3, R c4, R* ya,
                                           R* yb, R* yd) {
  constexpr int C = NComp<TH>::C;
  if (PASS == 1) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      // delta = phi^n - phi^{n-1} (differences of neighbouring values: exact per part)
      yd[c] = LO ? (pv[c] - pp[c]) + (lv[c] - lp[c]) : pv[c] - pp[c];
      ya[c] = LO ? lv[c] : pv[c];
      yb[c] = (LO ? lv[c] : pv[c]) + hdt * vv[c];
    }
    if (UnitVector<TH>::value && inside) {
      if constexpr (LO) normalise_split(pv, yb);
      else normalise<C>(yb);
    }
  } else if (PASS == 2) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const R base3 = hdt * vv[c] + c3 * k1v[c];
      const R base4 = dt * vv[c] + c4 * k2v[c];
      ya[c] = (LO ? lv[c] : pv[c]) + base3;
      yb[c] = (LO ? lv[c] : pv[c]) + base4;
    }
    if (UnitVector<TH>::value && inside) {
      if constexpr (LO) {
        normalise_split(pv, ya);
        normalise_split(pv, yb);
      } else {
        normalise<C>(ya);
        normalise<C>(yb);
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < C; ++c) ya[c] = LO ? lv[c] : pv[c];
  }
  if (LO) {  // stage inputs: value + small part, rounded once
#pragma unroll
    for (int c = 0; c < C; ++c) {
      ya[c] = pv[c] + ya[c];
      if (PASS != 3) yb[c] = pv[c] + yb[c];
    }
  }
}

// Vector units of VW = 2 or 4 consecutive FP32 sites (8- or 16-byte loads and stores).
template <int VW> struct VecOf;
template <> struct VecOf<2> { using T = float2; };
template <> struct VecOf<4> { using T = float4; };
template <int VW>
__device__ __forceinline__ typename VecOf<VW>::T ldv(const float* p) {
  return *reinterpret_cast<const typename VecOf<VW>::T*>(p);
}
template <int VW>
__device__ __forceinline__ void stv(float* p, const typename VecOf<VW>::T& v) {
  *reinterpret_cast<typename VecOf<VW>::T*>(p) = v;
}
template <typename V>
__device__ __forceinline__ float& vat(V& v, int j) { return (&v.x)[j]; }
template <int VW>
__device__ __forceinline__ typename VecOf<VW>::T vzero() { return typename VecOf<VW>::T{}; }

// Spacing factors and couplings broadcast to both lanes of a packed stage pair.
__device__ __forceinline__ Spacing<F2> bcast(const Spacing<float>& h) {
  return Spacing<F2>{F2(h.i12dx), F2(h.i12dy), F2(h.i12dx2), F2(h.i12dy2), F2(h.i144dxdy)};
}
__device__ __forceinline__ Couplings<F2> bcast(const Couplings<float>& k) {
  Couplings<F2> o;
#pragma unroll
  for (int i = 0; i < NCOUP; ++i) o.c[i] = F2(k.c[i]);
  return o;
}

// Sliding 5-row window over one component plane of the shared tile, for one
// column. MIX keeps the x-stencil of all five rows for the mixed derivative.
template <typename R, bool MIX>
struct Win {
  R c[5];   // centre values of rows y-2 .. y+2
  R g[5];   // MIX: unscaled Eq. 1 along x of rows y-2 .. y+2
  R xx[5];  // MIX: unscaled Eq. 2 along x of rows y-2 .. y+2

  __device__ __forceinline__ static void xterms(const R* P, R ce, R& gx, R& gxx) {
    const R m2 = P[-2], m1 = P[-1], p1 = P[1], p2 = P[2];
    gx = R(8) * (p1 - m1) - (p2 - m2);
    gxx = R(16) * ((p1 - ce) + (m1 - ce)) - ((p2 - ce) + (m2 - ce));
  }
  // P points at the row's centre.
  __device__ __forceinline__ void enter(const R* P, int slot) {
    const R ce = P[0];
    c[slot] = ce;
    if (MIX) xterms(P, ce, g[slot], xx[slot]);
  }
  __device__ __forceinline__ void shift() {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      c[k] = c[k + 1];
      if (MIX) { g[k] = g[k + 1]; xx[k] = xx[k + 1]; }
    }
  }
  __device__ __forceinline__ static R yd1(const R* a) { return R(8) * (a[3] - a[1]) - (a[4] - a[0]); }
  __device__ __forceinline__ static R yd2(const R* a) {
    return R(16) * ((a[3] - a[2]) + (a[1] - a[2])) - ((a[4] - a[2]) + (a[0] - a[2]));
  }
  // Derivatives at the window's centre row; Pc points at that row's centre.
  template <bool SECOND>
  __device__ __forceinline__ void derivs(const R* Pc, const Spacing<R>& h, R& v, R& fx, R& fy, R& fxx, R& fyy,
                                         R& fxy) const {
    R gx, gxx;
    if (MIX) {
      gx = g[2];
      gxx = xx[2];
    } else {
      xterms(Pc, c[2], gx, gxx);
    }
    v = c[2];
    fx = gx * h.i12dx;      // Eq. 1, x
    fy = yd1(c) * h.i12dy;  // Eq. 1, y
    if (SECOND) {
      fxx = gxx * h.i12dx2;     // Eq. 2, x
      fyy = yd2(c) * h.i12dy2;  // Eq. 2, y
    } else {
      fxx = fyy = R(0);
    }
    fxy = MIX ? (R(8) * (g[3] - g[1]) - (g[4] - g[0])) * h.i144dxdy : R(0);  // Eq. 1 in y of Eq. 1 in x
  }
};

// Window set of one stage input: all C components, with the x-stencils of every row
// kept for the mixed derivative where the theory needs it: the gauge field of the
// Abelian Higgs and s+id models, every component of the Baby Skyrme model.
template <int TH, int c>
struct NeedsMix {
  static constexpr bool value = TH == TH_BS || (TH == TH_AH && c >= 2) || (TH == TH_SID && c >= 4);
};

template <int TH, typename R, int SXY_, typename RP = R>
struct StageWin {
  static constexpr int C = NComp<TH>::C;
  static constexpr int SXY = SXY_;
  Win<R, NeedsMix<TH, 0>::value> w0;
  Win<R, NeedsMix<TH, 1>::value> w1;
  Win<R, NeedsMix<TH, 2>::value> w2;  // windows past C are never touched
  Win<R, NeedsMix<TH, 3>::value> w3;
  Win<R, NeedsMix<TH, 4>::value> w4;
  Win<R, NeedsMix<TH, 5>::value> w5;
  // chiral magnet with demagnetisation: the magnetostatic potential's tile, walked with
  // the stage input (pbase must be set before the first enter)
  Win<RP, false> wp;
  const RP* pbase = nullptr;

  __device__ __forceinline__ void enter(const R* tiles, int off, int slot) {
    if (TH == TH_CMD) wp.enter(pbase + off, slot);
    w0.enter(tiles + off, slot);
    w1.enter(tiles + SXY + off, slot);
    if (C > 2) w2.enter(tiles + 2 * SXY + off, slot);
    if (C > 3) w3.enter(tiles + 3 * SXY + off, slot);
    if (C > 4) w4.enter(tiles + 4 * SXY + off, slot);
    if (C > 5) w5.enter(tiles + 5 * SXY + off, slot);
  }
  __device__ __forceinline__ void shift() {
    if (TH == TH_CMD) wp.shift();
    w0.shift();
    w1.shift();
    if (C > 2) w2.shift();
    if (C > 3) w3.shift();
    if (C > 4) w4.shift();
    if (C > 5) w5.shift();
  }
  __device__ __forceinline__ void derivs(const R* tiles, int off, const Spacing<R>& h, R* v, R* fx, R* fy, R* fxx,
                                         R* fyy, R* fxy) const {
    w0.template derivs<true>(tiles + off, h, v[0], fx[0], fy[0], fxx[0], fyy[0], fxy[0]);
    w1.template derivs<true>(tiles + SXY + off, h, v[1], fx[1], fy[1], fxx[1], fyy[1], fxy[1]);
    if (C > 2) w2.template derivs<true>(tiles + 2 * SXY + off, h, v[2], fx[2], fy[2], fxx[2], fyy[2], fxy[2]);
    if (C > 3) w3.template derivs<true>(tiles + 3 * SXY + off, h, v[3], fx[3], fy[3], fxx[3], fyy[3], fxy[3]);
    if (C > 4) w4.template derivs<true>(tiles + 4 * SXY + off, h, v[4], fx[4], fy[4], fxx[4], fyy[4], fxy[4]);
    if (C > 5) w5.template derivs<true>(tiles + 5 * SXY + off, h, v[5], fx[5], fy[5], fxx[5], fyy[5], fxy[5]);
  }
  // the potential and its Eq. 1 gradient at the window's centre row
  __device__ __forceinline__ void psi_at(int off, const Spacing<RP>& h, RP& p, RP& px, RP& py) const {
    RP u0, u1, u2;
    wp.template derivs<false>(pbase + off, h, p, px, py, u0, u1, u2);
  }
};

// First derivatives only (the field difference of the arrest test).
template <int TH, typename R, int SXY_>
struct DiffWin {
  static constexpr int C = NComp<TH>::C;
  static constexpr int SXY = SXY_;
  Win<R, false> w[C];
  __device__ __forceinline__ void enter(const R* tiles, int off, int slot) {
#pragma unroll
    for (int c = 0; c < C; ++c) w[c].enter(tiles + c * SXY + off, slot);
  }
  __device__ __forceinline__ void shift() {
#pragma unroll
    for (int c = 0; c < C; ++c) w[c].shift();
  }
  __device__ __forceinline__ void derivs(const R* tiles, int off, const Spacing<R>& h, R* v, R* fx, R* fy) const {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      R unused0, unused1, unused2;
      w[c].template derivs<false>(tiles + c * SXY + off, h, v[c], fx[c], fy[c], unused0, unused1, unused2);
    }
  }
};

template <int TH, typename R>
__device__ __forceinline__ void force_at(const Couplings<R>& k, const R* v, const R* fx, const R* fy, const R* fxx,
                                         const R* fyy, const R* fxy, R* G, R x = R(0), R y = R(0)) {
  force_of<TH, R>(k, v, fx, fy, fxx, fyy, fxy, G, x, y);
}

// The RK4 combination at interior site s: phi' = phi + dt v + dt^2/6 (k1 + k2 + k3),
// the increment joining the stored remainder with compensated storage, and
// v' = v + dt/6 (k1 + 2 k2 + 2 k3 + k4); unit vectors are normalised (split form) and
// v' tangent-projected. Under a pending arrest v counts as zero and k2 as k1.
// The stored values the combination needs at site s (loaded before the stage forces
// are computed, so that their latency overlaps that work).
template <int TH, typename R>
struct SiteVals {
  R p0[NComp<TH>::C], l0[NComp<TH>::C], v0[NComp<TH>::C], k1[NComp<TH>::C], k2[NComp<TH>::C];
};
template <int TH, typename R, bool LO>
__device__ __forceinline__ void load_site(SiteVals<TH, R>& sv, const R* __restrict__ phi, const R* __restrict__ lo,
                                          const R* __restrict__ vel, const R* __restrict__ kv1,
                                          const R* __restrict__ kv2, size_t P, size_t s, bool arrest) {
#pragma unroll
  for (int c = 0; c < NComp<TH>::C; ++c) {
    sv.p0[c] = phi[c * P + s];
    sv.l0[c] = LO ? lo[c * P + s] : R(0);
    sv.v0[c] = arrest ? R(0) : vel[c * P + s];
    sv.k1[c] = kv1[c * P + s];
    sv.k2[c] = arrest ? sv.k1[c] : kv2[c * P + s];
  }
}
template <int TH, typename R, bool LO>
__device__ __forceinline__ void combine_loaded(const SiteVals<TH, R>& sv, R* __restrict__ phi_out,
                                               R* __restrict__ lo_out, R* __restrict__ v_out, size_t P, size_t s,
                                               R dt, R w6, R u6, const R* k3, const R* k4) {
  constexpr int C = NComp<TH>::C;
  R p0[C], q[C], vn[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    p0[c] = sv.p0[c];
    const R v0 = sv.v0[c], k1 = sv.k1[c], k2 = sv.k2[c];
    const R inc = dt * v0 + w6 * (k1 + k2 + k3[c]);
    q[c] = LO ? sv.l0[c] + inc : p0[c] + inc;
    vn[c] = v0 + u6 * (k1 + R(2) * (k2 + k3[c]) + k4[c]);
  }
  R pn[C], ln[C];
  if constexpr (LO) {
    if (UnitVector<TH>::value) normalise_split(p0, q);
#pragma unroll
    for (int c = 0; c < C; ++c) two_sum_f(p0[c], q[c], pn[c], ln[c]);  // hi' = fl(hi + small), lo' = rest
  } else {
#pragma unroll
    for (int c = 0; c < C; ++c) pn[c] = q[c];
    if (UnitVector<TH>::value) normalise<C>(pn);
  }
  if (UnitVector<TH>::value) {
    const R vp = vn[0] * pn[0] + vn[1] * pn[1] + vn[2] * pn[2];
#pragma unroll
    for (int c = 0; c < C; ++c) vn[c] -= vp * pn[c];
  }
#pragma unroll
  for (int c = 0; c < C; ++c) {
    phi_out[c * P + s] = pn[c];
    if (LO) lo_out[c * P + s] = ln[c];
    v_out[c * P + s] = vn[c];
  }
}
template <int TH, typename R, bool LO>
__device__ __forceinline__ void combine_site(const R* __restrict__ phi, const R* __restrict__ lo,
                                             const R* __restrict__ vel, const R* __restrict__ kv1,
                                             const R* __restrict__ kv2, R* __restrict__ phi_out,
                                             R* __restrict__ lo_out, R* __restrict__ v_out, size_t P, size_t s,
                                             bool arrest, R dt, R w6, R u6, const R* k3, const R* k4) {
  SiteVals<TH, R> sv;
  load_site<TH, R, LO>(sv, phi, lo, vel, kv1, kv2, P, s, arrest);
  combine_loaded<TH, R, LO>(sv, phi_out, lo_out, v_out, P, s, dt, w6, u6, k3, k4);
}

// Running maximum of |g| for a >= 0: on non-negative values the IEEE bit patterns
// order as unsigned integers, with every NaN above +Inf, so one integer max keeps
// the maximum and propagates NaN (as rmax does).
__device__ __forceinline__ float absmax(float a, float g) {
  return __uint_as_float(max(__float_as_uint(a), __float_as_uint(fabsf(g))));
}
__device__ __forceinline__ double absmax(double a, double g) {
  return __longlong_as_double((long long)max((unsigned long long)__double_as_longlong(a),
                                             (unsigned long long)__double_as_longlong(fabs(g))));
}
// Per-tile view of the problem, staged in shared memory by thread 0.
template <typename R>
struct TileCtx {
  ProbDesc<R> d;
  int p;         // problem index
  int skip;      // the problem has stopped (or, pass 1, its head is already evaluated)
  int cur;       // ping-pong parity of the current field
  int arrest;    // pass 2: the current velocity counts as zero
  int has_prev;  // pass 1: the other buffer holds the previous field
  int want_e;    // pass 1: sum E_h itself (else E_h = previous E_h + the exact change)
  int adv;       // pass 3: the step budget allows a new field
};

// Whether a pass skips the tiles of a problem: it has stopped, or (pass 1) its head is
// already evaluated, or (pass 2) its step budget is spent, or (descent) both.
template <int PASS>
__device__ __forceinline__ int tile_skip(const DevState* st) {
  const long long steps = st->steps;
  int skip = (st->converged | st->nonfinite) != 0;
  if (PASS == 1) skip |= (st->head_step == steps);
  else if (PASS == 2) skip |= (steps >= st->step_limit);
  else skip |= (st->head_step == steps && steps >= st->step_limit);  // evaluated, budget spent
  return skip;
}

// Batches: the first tile at or after `start` (stepping by `stride`) whose problem the
// pass does not skip, or `total`. Warp 0 tests 32 candidates per round (one ballot),
// so a block runs past the tiles of stopped problems without a block barrier per tile.
// A problem's record changes only when its last tile of the launch arrives, and every
// candidate is a tile this block has not processed yet, so the test is stable.
template <typename R, int PASS>
__device__ __forceinline__ int next_running(const ProbDesc<R>* __restrict__ probs, const int* __restrict__ tile_prob,
                                            int start, int stride, int total) {
  const int lane = threadIdx.x & 31;
  for (long long base = start; base < total; base += 32LL * stride) {
    const long long c = base + (long long)lane * stride;
    bool run = false;
    if (c < total) run = !tile_skip<PASS>(probs[tile_prob[c]].st);
    const unsigned m = __ballot_sync(0xffffffffu, run);
    if (m) return (int)(base + (long long)(__ffs(m) - 1) * stride);
  }
  return total;
}

// The per-tile flags of the view, from the problem's record.
template <typename R, int PASS>
__device__ __forceinline__ void set_tile_flags(TileCtx<R>& tc, const DevState* st) {
  const long long steps = st->steps;
  tc.skip = tile_skip<PASS>(st);
  tc.cur = (int)(steps & 1);
  tc.arrest = (PASS == 2) && (st->arrest != 0);
  tc.has_prev = (PASS == 1) && (steps > 0);
  // FP32 pass 1 sums E_h itself on the first field, every SS_E_EVERY-th step and on
  // the last field of a run; in between E_h = E_h(previous) + dE, the cancellation-free
  // change it sums anyway for Eq. 4 (drift over SS_E_EVERY steps: a few roundings of dE)
  tc.want_e = PASS != 1 || sizeof(R) == 8 || steps == 0 || (steps & (SS_E_EVERY - 1)) == 0 ||
              steps >= st->step_limit;
  tc.adv = (PASS == 3) && (steps < st->step_limit);
}

// Thread 0 stages the view of tile t. A problem's record changes only when its last
// tile of a launch arrives, so while any of its tiles is still unprocessed (as tile
// t is here) the view stays valid: it may be read ahead of use. A launch over a
// single problem passes its descriptor as a kernel parameter and stages only the
// record's flags.
template <typename R, int PASS, bool ONE>
__device__ __forceinline__ void load_tile_ctx(TileCtx<R>& tc, const ProbDesc<R>& one,
                                              const ProbDesc<R>* __restrict__ probs,
                                              const int* __restrict__ tile_prob, int t) {
  const DevState* st;
  if constexpr (ONE) {
    tc.p = 0;
    st = one.st;
  } else {
    const int p = tile_prob[t];
    tc.d = probs[p];
    tc.p = p;
    st = tc.d.st;
  }
  set_tile_flags<R, PASS>(tc, st);
}

// The same for a batch by the 32 lanes of warp 0 (t is uniform over the warp): the
// descriptor copied in 8-byte words in parallel, the record's flags by lane 0.
template <typename R, int PASS>
__device__ __forceinline__ void load_tile_ctx_warp(TileCtx<R>& tc, const ProbDesc<R>* __restrict__ probs,
                                                   const int* __restrict__ tile_prob, int t) {
  static_assert(sizeof(ProbDesc<R>) % 8 == 0, "the descriptor is copied in 8-byte words");
  const int lane = threadIdx.x & 31;
  const int p = tile_prob[t];
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(probs + p);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(&tc.d);
  for (int i = lane; i < (int)(sizeof(ProbDesc<R>) / 8); i += 32) dst[i] = src[i];
  if (lane == 0) {
    tc.p = p;
    set_tile_flags<R, PASS>(tc, probs[p].st);
  }
}

// One flow pass over every tile of a batch. ONE: the batch has a single problem,
// whose descriptor arrives as a kernel parameter, so its pointers, spacings and
// couplings are read as constant operands instead of occupying registers.
template <int TH, typename R, int PASS, bool ONE>
constexpr int pass_min_blocks() {
  return (TH == SS_MINB_THEORY && sizeof(R) == 4 && (ONE || SS_MINB_BATCH))
             ? (ONE ? (PASS == 1 ? SS_MINB1 : (PASS == 2 ? SS_MINB2 : SS_MINB3))
                    : (PASS == 1 ? SS_MINB1B : (PASS == 2 ? SS_MINB2B : SS_MINB3B)))
             : 1;
}

template <bool B>
struct BoolC {
  static constexpr bool value = B;
};

template <int TH, typename R, int PASS, bool LO, bool ONE, int TS>
__global__ void __launch_bounds__(NT, pass_min_blocks<TH, R, PASS, ONE>())
    k_pass(const __grid_constant__ ProbDesc<R> one, const ProbDesc<R>* __restrict__ probs,
           const int* __restrict__ tile_prob, int total_tiles) {
  using T = FlowTile<R, TS>;
  constexpr int C = NComp<TH>::C;
  constexpr int RY = T::RY;
  // FP32 flow passes evaluate their two stage inputs as packed pairs (ss_pack.cuh):
  // shared [C][SXY] planes of (Y_a, Y_b), one walk for both stages
  constexpr bool PK = sizeof(R) == 4 && PASS != 3;
  constexpr int PS = C * T::SXY;  // values per tile set
  extern __shared__ __align__(16) unsigned char smraw[];
  R* sm = reinterpret_cast<R*>(smraw);  // pass 1: [Y1 | Y2 | delta], pass 2: [Y3 | Y4], pass 3: [phi], (+ psi)
  __shared__ TileCtx<R> tcb[2];         // this tile's view and the next one's (read ahead)
  __shared__ R sred[(NT / 32) * 5];
  __shared__ double dred[RedSmem<2, 1>::n];
  __shared__ int s_last;
  const int tid = threadIdx.y * BX + threadIdx.x;
  R* const setA = sm;           // first stage input of the pass
  R* const setB = sm + PS;      // second stage input
  R* const setD = sm + 2 * PS;  // pass 1: phi^n - phi^{n-1}
  R* const setP = sm + (PASS == 1 ? 3 : (PASS == 2 ? 2 : 1)) * PS;  // demagnetisation: psi of phi^n
  // passes 1, 3: running sums over this block's consecutive tiles of one problem
  R es = R(0), ec = R(0), ds = R(0), dc = R(0), gmr = R(0);
  int run_lt0 = -1;  // local index of the first tile of the block's current run

  // The block's tiles: blockIdx.x, + gridDim.x, ... For a batch, warp 0 finds the next
  // tile of a running problem (s_next, one slot per buffer) while the block works on
  // the current one, so stopped problems cost no per-tile barrier.
  __shared__ int s_next[2];
  int t = blockIdx.x;
  if constexpr (ONE) {
    if (tid == 0 && t < total_tiles) load_tile_ctx<R, PASS, ONE>(tcb[0], one, probs, tile_prob, t);
  } else {
    if (tid < 32) {
      const int t0 = next_running<R, PASS>(probs, tile_prob, blockIdx.x, gridDim.x, total_tiles);
      if (tid == 0) s_next[0] = t0;
      if (t0 < total_tiles) load_tile_ctx_warp<R, PASS>(tcb[0], probs, tile_prob, t0);
    }
    __syncthreads();
    t = s_next[0];
  }
  int buf = 0;
  for (; t < total_tiles; t = ONE ? t + (int)gridDim.x : s_next[buf ^ 1], buf ^= 1) {
    __syncthreads();  // tcb[buf] is staged; the previous tile's shared reads are finished
    if constexpr (ONE) {
      const int tn1 = t + gridDim.x;
      if (tid == 0 && tn1 < total_tiles) load_tile_ctx<R, PASS, ONE>(tcb[buf ^ 1], one, probs, tile_prob, tn1);
    } else if (tid < 32) {
      // the common case: the block's next tile belongs to the same running problem, whose
      // view is this tile's (its record cannot change before that tile has run)
      const int cand = t + (int)gridDim.x;
      const bool same = cand < total_tiles && !tcb[buf].skip && tile_prob[cand] == tcb[buf].p;
      const int tn1 = same ? cand : next_running<R, PASS>(probs, tile_prob, cand, gridDim.x, total_tiles);
      if (tid == 0) s_next[buf ^ 1] = tn1;
      if (same) {
        static_assert(sizeof(TileCtx<R>) % 8 == 0, "the view is copied in 8-byte words");
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&tcb[buf]);
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(&tcb[buf ^ 1]);
        for (int i = tid; i < (int)(sizeof(TileCtx<R>) / 8); i += 32) dst[i] = src[i];
      } else if (tn1 < total_tiles) {
        load_tile_ctx_warp<R, PASS>(tcb[buf ^ 1], probs, tile_prob, tn1);
      }
    }
    const TileCtx<R>& tc = tcb[buf];
    if (tc.skip) {  // uniform over the block (batches: only if a record changed after the search)
      if (!ONE) __syncthreads();  // s_next[buf ^ 1] is read by the loop step
      continue;
    }
    const ProbDesc<R>& D = ONE ? one : tc.d;
    const int cur = tc.cur;
    const bool arrest = tc.arrest != 0;
    const bool has_prev = tc.has_prev != 0;
    const bool want_e = tc.want_e != 0;
    const bool adv = tc.adv != 0;
    const int nx = D.nx, ny = D.ny;
    const size_t P = (size_t)D.plane;
    const R* __restrict__ phi = D.phi[cur];
    const R* __restrict__ lo = D.lo[cur];
    const R* __restrict__ vel = D.v[cur];
    const R* __restrict__ phi_prev = D.phi[cur ^ 1];
    const R* __restrict__ lo_prev = D.lo[cur ^ 1];
    const R* __restrict__ psi = D.psi[cur];         // demagnetisation only
    const R* __restrict__ psi_prev = D.psi[cur ^ 1];
    R* __restrict__ kv1 = D.kv[0];
    R* __restrict__ kv2 = D.kv[1];
    const Spacing<R> h = D.h;
    Couplings<R> kc = D.k;
    if (TH == TH_BEC) kc.c[3] = R(D.st->mu_held);  // fixed atom number: the field's multiplier
    const R dt = D.dt, hdt = R(0.5) * dt;
    const R c3 = R(0.25) * dt * dt, c4 = R(0.5) * dt * dt;
    const int lt = t - D.tile0;  // tile index within the problem
    const int x0 = (lt % D.ntx) * T::TX, y0 = (lt / D.ntx) * T::TY;

    // ---- stage inputs over the tile and its halo
    constexpr int LU = PASS == 1 ? SS_LU1 : (PASS == 2 ? SS_LU2 : SS_LU3);
    bool vec = false;  // float4 staging: every loaded site in bounds, every used site in I
    if constexpr (sizeof(R) == 4) vec = D.vec && x0 >= 4 && x0 + T::TX + 4 <= nx && y0 >= 4 && y0 + T::TY + 4 <= ny;
    // the same units on tiles at the grid's edge (FP32 rows of whole 16-byte units): each
    // unit is wholly in or out of the grid (x0 - 4 and nx are multiples of it)
    constexpr bool VEDGE = PASS == 1 ? SS_VEDGE1 : (PASS == 2 ? SS_VEDGE2 : SS_VEDGE3);
    bool vedge = false;
    if constexpr (sizeof(R) == 4 && VEDGE) vedge = D.vec && !vec;
    if constexpr (sizeof(R) == 4) {
      // units of VW consecutive sites of one shared row (shared columns VW u ..,
      // sites x0 - 4 + VW u ..): one VW-wide load per stored plane, one VW-wide store
      // per staged plane. The stencils read shared columns OX - 2 .. OX + TX + 1; with
      // SS_VSKIPn units wholly outside them (the outermost two columns of each side,
      // with 2-site units) are not staged. Compensated storage loads twice the planes:
      // narrower units keep them in registers.
      constexpr int VW = LO ? (PASS == 1 ? SS_VW1_LO : (PASS == 2 ? SS_VW2_LO : SS_VW3_LO)) : SS_VW_PLAIN;
      using V = typename VecOf<VW>::T;
      constexpr bool VSKIP = PASS == 1 ? SS_VSKIP1 : (PASS == 2 ? SS_VSKIP2 : SS_VSKIP3);
      constexpr int U0 = VSKIP ? (T::OX - 2) / VW : 0;  // first and last unit staged
      constexpr int U1 = VSKIP ? (T::OX + T::TX + 1) / VW : T::SX / VW - 1;
      constexpr int UW = U1 - U0 + 1, NU = UW * T::SY;
      constexpr int VUNR = PASS == 1 ? SS_VUNR1 : (PASS == 2 ? SS_VUNR2 : SS_VUNR3);
      if (vec) {
#pragma unroll VUNR
        for (int u = tid; u < NU; u += NT) {
          const int ly = u / UW, ux = U0 + (u - ly * UW);
          const size_t s = (size_t)(y0 - 2 + ly) * nx + (size_t)(x0 - 4 + VW * ux);
          const int so = ly * T::SX + VW * ux;
          const V z = vzero<VW>();
          V P4[C], L4[C], V4[C], A4[C], B4[C], Z4 = z;
#pragma unroll
          for (int c = 0; c < C; ++c) {
            P4[c] = ldv<VW>(phi + c * P + s);
            L4[c] = LO ? ldv<VW>(lo + c * P + s) : z;
            V4[c] = (PASS != 3 && !arrest) ? ldv<VW>(vel + c * P + s) : z;
            if (PASS == 1) {  // the previous field (A: value, B: remainder)
              A4[c] = has_prev ? ldv<VW>(phi_prev + c * P + s) : P4[c];
              B4[c] = (LO && has_prev) ? ldv<VW>(lo_prev + c * P + s) : L4[c];
            } else if (PASS == 2) {  // k_v1, k_v2
              A4[c] = ldv<VW>(kv1 + c * P + s);
              B4[c] = arrest ? A4[c] : ldv<VW>(kv2 + c * P + s);
            }
          }
          if (TH == TH_CMD) Z4 = ldv<VW>(psi + s);
          V OA[C], OB[C], OD[C];
#pragma unroll
          for (int j = 0; j < VW; ++j) {
            R pv[C], lv[C], vv[C], aa[C], bb[C], ya[C], yb[C], yd[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
              pv[c] = vat(P4[c], j);
              lv[c] = vat(L4[c], j);
              vv[c] = vat(V4[c], j);
              aa[c] = vat(A4[c], j);
              bb[c] = vat(B4[c], j);
            }
            stage_site<TH, R, PASS, LO>(pv, lv, vv, aa, bb, aa, bb, true, hdt, dt, c3, c4, ya, yb, yd);
#pragma unroll
            for (int c = 0; c < C; ++c) {
              vat(OA[c], j) = ya[c];
              if (PASS != 3) vat(OB[c], j) = yb[c];
              if (PASS == 1) vat(OD[c], j) = yd[c];
            }
          }
#pragma unroll
          for (int c = 0; c < C; ++c) {
            if constexpr (PK) {  // interleaved (Y_a, Y_b) pairs
              float* ab = setA + 2 * (c * T::SXY + so);
#pragma unroll
              for (int j = 0; j < VW; j += 2)
                stv<4>(ab + 2 * j, make_float4(vat(OA[c], j), vat(OB[c], j), vat(OA[c], j + 1), vat(OB[c], j + 1)));
            } else {
              stv<VW>(setA + c * T::SXY + so, OA[c]);
              if (PASS != 3) stv<VW>(setB + c * T::SXY + so, OB[c]);
            }
            if (PASS == 1) stv<VW>(setD + c * T::SXY + so, OD[c]);
          }
          if (TH == TH_CMD) stv<VW>(setP + so, Z4);
        }
      }
      if constexpr (VEDGE) {
        if (vedge) {  // the loop above with each unit masked to the grid, each site to I
#pragma unroll 1
          for (int u = tid; u < NU; u += NT) {
            const int ly = u / UW, ux = U0 + (u - ly * UW);
            const int gy = y0 - 2 + ly, gx = x0 - 4 + VW * ux;  // the unit's first site
            const bool uin = (gy >= 0 && gy < ny && gx >= 0 && gx < nx);
            const size_t s = uin ? (size_t)gy * nx + (size_t)gx : 0;
            const int so = ly * T::SX + VW * ux;
            const V z = vzero<VW>();
            V P4[C], L4[C], V4[C], A4[C], B4[C], Z4 = z;
#pragma unroll
            for (int c = 0; c < C; ++c) {
              P4[c] = uin ? ldv<VW>(phi + c * P + s) : z;
              L4[c] = (LO && uin) ? ldv<VW>(lo + c * P + s) : z;
              V4[c] = (PASS != 3 && !arrest && uin) ? ldv<VW>(vel + c * P + s) : z;
              if (PASS == 1) {  // the previous field (A: value, B: remainder)
                A4[c] = (has_prev && uin) ? ldv<VW>(phi_prev + c * P + s) : P4[c];
                B4[c] = (LO && has_prev && uin) ? ldv<VW>(lo_prev + c * P + s) : L4[c];
              } else if (PASS == 2) {  // k_v1, k_v2
                A4[c] = uin ? ldv<VW>(kv1 + c * P + s) : z;
                B4[c] = arrest ? A4[c] : (uin ? ldv<VW>(kv2 + c * P + s) : z);
              }
            }
            if (TH == TH_CMD) Z4 = uin ? ldv<VW>(psi + s) : z;
            const bool row_in = (gy >= 2 && gy < ny - 2);
            V OA[C], OB[C], OD[C];
#pragma unroll
            for (int j = 0; j < VW; ++j) {
              // site in I: velocities and stage slopes are zero outside it, and the
              // unit-vector constraint is applied only inside it
              const bool ins = (uin && row_in && gx + j >= 2 && gx + j < nx - 2);
              R pv[C], lv[C], vv[C], aa[C], bb[C], ya[C], yb[C], yd[C];
#pragma unroll
              for (int c = 0; c < C; ++c) {
                pv[c] = vat(P4[c], j);
                lv[c] = vat(L4[c], j);
                vv[c] = ins ? vat(V4[c], j) : R(0);
                aa[c] = (PASS != 2 || ins) ? vat(A4[c], j) : R(0);
                bb[c] = (PASS != 2 || ins) ? vat(B4[c], j) : R(0);
              }
              stage_site<TH, R, PASS, LO>(pv, lv, vv, aa, bb, aa, bb, ins, hdt, dt, c3, c4, ya, yb, yd);
#pragma unroll
              for (int c = 0; c < C; ++c) {
                vat(OA[c], j) = ya[c];
                if (PASS != 3) vat(OB[c], j) = yb[c];
                if (PASS == 1) vat(OD[c], j) = yd[c];
              }
            }
#pragma unroll
            for (int c = 0; c < C; ++c) {
              if constexpr (PK) {  // interleaved (Y_a, Y_b) pairs
                float* ab = setA + 2 * (c * T::SXY + so);
#pragma unroll
                for (int j = 0; j < VW; j += 2)
                  stv<4>(ab + 2 * j, make_float4(vat(OA[c], j), vat(OB[c], j), vat(OA[c], j + 1), vat(OB[c], j + 1)));
              } else {
                stv<VW>(setA + c * T::SXY + so, OA[c]);
                if (PASS != 3) stv<VW>(setB + c * T::SXY + so, OB[c]);
              }
              if (PASS == 1) stv<VW>(setD + c * T::SXY + so, OD[c]);
            }
            if (TH == TH_CMD) stv<VW>(setP + so, Z4);
          }
        }
      }
    }
    // scalar staging (rows not 16-byte aligned, FP64; grid edges when SS_VEDGEn is 0): LU
    // sites per iteration, the loads of all LU sites issued before any is used
    constexpr int SWY = T::SW * T::SY;
    for (int base = tid; !vec && !vedge && base < SWY; base += LU * NT) {
      R pv[LU][C], lv[LU][C], vv[LU][C], k1v[LU][C], k2v[LU][C], pp[LU][C], lp[LU][C], pz[LU];
      bool in[LU], inside[LU];
#pragma unroll
      for (int u = 0; u < LU; ++u) {  // all global loads of the sites first
        const int idx = base + u * NT;
        const int ly = idx / T::SW, lx = idx - ly * T::SW;
        const int gx = x0 + lx - 2, gy = y0 + ly - 2;
        in[u] = idx < SWY && gx >= 0 && gx < nx && gy >= 0 && gy < ny;
        inside[u] = in[u] && gx >= 2 && gx < nx - 2 && gy >= 2 && gy < ny - 2;
        const size_t s = in[u] ? (size_t)gy * nx + gx : 0;
        if (TH == TH_CMD) pz[u] = in[u] ? psi[s] : R(0);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          pv[u][c] = in[u] ? phi[c * P + s] : R(0);
          lv[u][c] = (LO && in[u]) ? lo[c * P + s] : R(0);
          vv[u][c] = (PASS != 3 && inside[u] && !arrest) ? vel[c * P + s] : R(0);
          if (PASS == 1) {
            pp[u][c] = (has_prev && in[u]) ? phi_prev[c * P + s] : pv[u][c];
            lp[u][c] = (LO && has_prev && in[u]) ? lo_prev[c * P + s] : lv[u][c];
          } else if (PASS == 2) {
            k1v[u][c] = inside[u] ? kv1[c * P + s] : R(0);
            k2v[u][c] = inside[u] ? (arrest ? k1v[u][c] : kv2[c * P + s]) : R(0);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < LU; ++u) {
        const int idx = base + u * NT;
        if (idx >= SWY) break;
        const int ly = idx / T::SW, lx = idx - ly * T::SW;
        const int sh = ly * T::SX + lx + (T::OX - 2);  // shared index of the site
        R ya[C], yb[C], yd[C];
        stage_site<TH, R, PASS, LO>(pv[u], lv[u], vv[u], k1v[u], k2v[u], pp[u], lp[u], inside[u], hdt, dt, c3, c4,
                                    ya, yb, yd);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          if constexpr (PK) {
            setA[2 * (c * T::SXY + sh)] = ya[c];
            setA[2 * (c * T::SXY + sh) + 1] = yb[c];
          } else {
            setA[c * T::SXY + sh] = ya[c];
            if (PASS != 3) setB[c * T::SXY + sh] = yb[c];
          }
          if (PASS == 1) setD[c * T::SXY + sh] = has_prev ? yd[c] : R(0);
        }
        if (TH == TH_CMD) setP[sh] = pz[u];
      }
    }
    __syncthreads();

    // ---- column walk: RY rows of column threadIdx.x
    const int sx = threadIdx.x + T::OX, sy0 = threadIdx.y * RY + 2;
    const int gx = x0 + threadIdx.x, gyb = y0 + threadIdx.y * RY;
    const bool colok = gx >= 2 && gx < nx - 2;
    // site position, origin at the grid centre (only the BEC's trap and rotation use it)
    const R hy = D.hy;
    const R xs = TH == TH_BEC ? (R(gx) - R(0.5) * R(nx - 1)) * D.hx : R(0);
    auto ypos = [&](int r) { return TH == TH_BEC ? (R(gyb + r) - R(0.5) * R(ny - 1)) * hy : R(0); };

    if (PASS != 2) {
      if (PASS == 1) {
      if constexpr (PK) {
        // stages 1 and 2 in one walk over the pairs (Y_1, Y_2): k_v1, k_v2; at Y_1
        // also e, max|G| and e(phi^n) - e(phi^{n-1})
        const F2* ab = reinterpret_cast<const F2*>(setA);
        const Spacing<F2> h2 = bcast(h);
        const Couplings<F2> k2c = bcast(kc);
        StageWin<TH, F2, T::SXY, R> W;
        W.pbase = setP;
        DiffWin<TH, R, T::SXY> Dw;
#pragma unroll
        for (int s = 0; s < 5; ++s) {
          const int off = (sy0 - 2 + s) * T::SX + sx;
          W.enter(ab, off, s);
          if (has_prev) Dw.enter(setD, off, s);
        }
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          const int off = (sy0 + r) * T::SX + sx;
          const bool ok = colok && gyb + r >= 2 && gyb + r < ny - 2;
          F2 v[C], fx[C], fy[C], fxx[C], fyy[C], fxy[C], G[C];
          W.derivs(ab, off, h2, v, fx, fy, fxx, fyy, fxy);
          // site extras: the BEC's position; with demagnetisation psi and its gradient
          R q0 = xs, q1 = ypos(r), ps = R(0);
          if (TH == TH_CMD) W.psi_at(off, h, ps, q0, q1);
          force_at<TH, F2>(k2c, v, fx, fy, fxx, fyy, fxy, G, F2(q0), F2(q1));
          R va[C], fxa[C], fya[C];  // stage 1: the field and its first derivatives
#pragma unroll
          for (int c = 0; c < C; ++c) {
            va[c] = v[c].v.x;
            fxa[c] = fx[c].v.x;
            fya[c] = fy[c].v.x;
          }
          if (ok) {
            const size_t s = (size_t)(gyb + r) * nx + gx;
#pragma unroll
            for (int c = 0; c < C; ++c) {
              kv1[c * P + s] = -G[c].v.x;
              kv2[c * P + s] = -G[c].v.y;
              gmr = absmax(gmr, G[c].v.x);
            }
            if (want_e) {
              const R e = density_at<TH, R>(kc, va, fxa, fya, TH == TH_CMD ? ps : q0, q1);
              const R t1 = es + e;
              ec += (fabs(es) >= fabs(e)) ? (es - t1) + e : (e - t1) + es;
              es = t1;
            }
          }
          if (has_prev) {
            R dd[C], dxv[C], dyv[C];
            Dw.derivs(setD, off, h, dd, dxv, dyv);
            if (ok) {
              const R de = delta_density_at<TH, R>(
                  kc, va, fxa, fya, dd, dxv, dyv, TH == TH_CMD ? ps : q0,
                  TH == TH_CMD ? ps - psi_prev[(size_t)(gyb + r) * nx + gx] : q1);
              const R t2 = ds + de;
              dc += (fabs(ds) >= fabs(de)) ? (ds - t2) + de : (de - t2) + ds;
              ds = t2;
            }
          }
          if (r + 1 < RY) {
            const int noff = (sy0 + r + 3) * T::SX + sx;
            W.shift();
            W.enter(ab, noff, 4);
            if (has_prev) {
              Dw.shift();
              Dw.enter(setD, noff, 4);
            }
          }
        }
      } else {
      // stage 1 at Y_1 = phi: k_v1, e, max|G|, and e(phi^n) - e(phi^{n-1})
      {
        StageWin<TH, R, T::SXY> W;
        W.pbase = setP;
        DiffWin<TH, R, T::SXY> D;
#pragma unroll
        for (int s = 0; s < 5; ++s) {
          const int off = (sy0 - 2 + s) * T::SX + sx;
          W.enter(setA, off, s);
          if (has_prev) D.enter(setD, off, s);
        }
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          const int off = (sy0 + r) * T::SX + sx;
          const bool ok = colok && gyb + r >= 2 && gyb + r < ny - 2;
          R v[C], fx[C], fy[C], fxx[C], fyy[C], fxy[C], G[C];
          W.derivs(setA, off, h, v, fx, fy, fxx, fyy, fxy);
          // site extras: the BEC's position; with demagnetisation psi and its gradient
          R q0 = xs, q1 = ypos(r), ps = R(0);
          if (TH == TH_CMD) W.psi_at(off, h, ps, q0, q1);
          force_at<TH, R>(kc, v, fx, fy, fxx, fyy, fxy, G, q0, q1);
          if (ok) {
            const size_t s = (size_t)(gyb + r) * nx + gx;
#pragma unroll
            for (int c = 0; c < C; ++c) {
              kv1[c * P + s] = -G[c];
              gmr = absmax(gmr, G[c]);
            }
            if (want_e) {
              const R e = density_at<TH, R>(kc, v, fx, fy, TH == TH_CMD ? ps : q0, q1);
              const R t1 = es + e;
              ec += (fabs(es) >= fabs(e)) ? (es - t1) + e : (e - t1) + es;
              es = t1;
            }
          }
          if (has_prev) {
            R dd[C], dxv[C], dyv[C];
            D.derivs(setD, off, h, dd, dxv, dyv);
            if (ok) {
              const R de = delta_density_at<TH, R>(
                  kc, v, fx, fy, dd, dxv, dyv, TH == TH_CMD ? ps : q0,
                  TH == TH_CMD ? ps - psi_prev[(size_t)(gyb + r) * nx + gx] : q1);
              const R t2 = ds + de;
              dc += (fabs(ds) >= fabs(de)) ? (ds - t2) + de : (de - t2) + ds;
              ds = t2;
            }
          }
          if (r + 1 < RY) {
            const int noff = (sy0 + r + 3) * T::SX + sx;
            W.shift();
            W.enter(setA, noff, 4);
            if (has_prev) {
              D.shift();
              D.enter(setD, noff, 4);
            }
          }
        }
      }
      // stage 2 at Y_2 = phi + dt/2 v: k_v2
      {
        StageWin<TH, R, T::SXY> W;
        W.pbase = setP;
#pragma unroll
        for (int s = 0; s < 5; ++s) W.enter(setB, (sy0 - 2 + s) * T::SX + sx, s);
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          const int off = (sy0 + r) * T::SX + sx;
          R v[C], fx[C], fy[C], fxx[C], fyy[C], fxy[C], G[C];
          W.derivs(setB, off, h, v, fx, fy, fxx, fyy, fxy);
          // site extras: the BEC's position; with demagnetisation psi and its gradient
          R q0 = xs, q1 = ypos(r), ps = R(0);
          if (TH == TH_CMD) W.psi_at(off, h, ps, q0, q1);
          force_at<TH, R>(kc, v, fx, fy, fxx, fyy, fxy, G, q0, q1);
          if (colok && gyb + r >= 2 && gyb + r < ny - 2) {
            const size_t s = (size_t)(gyb + r) * nx + gx;
#pragma unroll
            for (int c = 0; c < C; ++c) kv2[c * P + s] = -G[c];
          }
          if (r + 1 < RY) {
            W.shift();
            W.enter(setB, (sy0 + r + 3) * T::SX + sx, 4);
          }
        }
      }
      }
      } else {
      // gradient descent at phi: -G into k_v1, e, max|G|, and phi - dtau G
      {
        StageWin<TH, R, T::SXY> W;
        W.pbase = setP;
#pragma unroll
        for (int s = 0; s < 5; ++s) W.enter(setA, (sy0 - 2 + s) * T::SX + sx, s);
        const R tau = D.tau;
        R* __restrict__ phi_out = D.phi[cur ^ 1];
        R* __restrict__ lo_out = D.lo[cur ^ 1];
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          const int off = (sy0 + r) * T::SX + sx;
          R v[C], fx[C], fy[C], fxx[C], fyy[C], fxy[C], G[C];
          W.derivs(setA, off, h, v, fx, fy, fxx, fyy, fxy);
          // site extras: the BEC's position; with demagnetisation psi and its gradient
          R q0 = xs, q1 = ypos(r), ps = R(0);
          if (TH == TH_CMD) W.psi_at(off, h, ps, q0, q1);
          force_at<TH, R>(kc, v, fx, fy, fxx, fyy, fxy, G, q0, q1);
          if (colok && gyb + r >= 2 && gyb + r < ny - 2) {
            const size_t s = (size_t)(gyb + r) * nx + gx;
#pragma unroll
            for (int c = 0; c < C; ++c) {
              kv1[c * P + s] = -G[c];
              gmr = absmax(gmr, G[c]);
            }
            const R e = density_at<TH, R>(kc, v, fx, fy, TH == TH_CMD ? ps : q0, q1);
            const R t1 = es + e;
            ec += (fabs(es) >= fabs(e)) ? (es - t1) + e : (e - t1) + es;
            es = t1;
            if (adv) {
              R p0[C], q[C], pn[C], ln[C];
#pragma unroll
              for (int c = 0; c < C; ++c) {
                p0[c] = phi[c * P + s];
                q[c] = (LO ? lo[c * P + s] : p0[c]) - tau * G[c];
              }
              if constexpr (LO) {
                if (UnitVector<TH>::value) normalise_split(p0, q);
#pragma unroll
                for (int c = 0; c < C; ++c) two_sum_f(p0[c], q[c], pn[c], ln[c]);
              } else {
#pragma unroll
                for (int c = 0; c < C; ++c) pn[c] = q[c];
                if (UnitVector<TH>::value) normalise<C>(pn);
              }
#pragma unroll
              for (int c = 0; c < C; ++c) {
                phi_out[c * P + s] = pn[c];
                if (LO) lo_out[c * P + s] = ln[c];
              }
            }
          }
          if (r + 1 < RY) {
            W.shift();
            W.enter(setA, (sy0 + r + 3) * T::SX + sx, 4);
          }
        }
      }
      }

      // ---- partials: the block keeps summing while its next tile belongs to the same
      // problem; otherwise it reduces and writes the running sums into the slot of its
      // run, and the runs are counted (no per-tile fence or counter). A problem's tiles
      // are one contiguous index range and a block walks its tiles in increasing order,
      // so each block's tiles of a problem form one run: a problem has min(grid, tiles)
      // runs, and the first tile of block b's run has local index (b - tile0) mod grid,
      // below that count (a single problem: the block index). The arrival that
      // completes the count reduces the problem's partials in slot order and decides.
      // (A block that still holds another tile of the problem can never be the last.)
      const ProbDesc<R>& d = D;
      if (run_lt0 < 0) run_lt0 = lt;
      const int tn = ONE ? t + (int)gridDim.x : s_next[buf ^ 1];  // written before the staging barrier
      const bool flush = ONE ? tn >= total_tiles : !(tn < total_tiles && tcb[buf ^ 1].p == tc.p);
      if (!flush) continue;
      const int slot = ONE ? (int)blockIdx.x : run_lt0;
      run_lt0 = -1;
      const int nslots = min((int)gridDim.x, d.ntiles);
      RPair<R> pe{es, ec}, pd{ds, dc};
      R pm = gmr;
      tile_reduce<R>(pe, pd, pm, sred);
      es = ec = ds = dc = gmr = R(0);  // the next run of tiles starts afresh
      if (tid == 0) {
        d.part[slot] = FlowPartial{(double)pe.s, (double)pe.c, (double)pd.s, (double)pd.c, (double)pm,
                                   {0.0, 0.0, 0.0}};
        if constexpr (ONE) {
          __threadfence();
          const unsigned prev = atomicAdd(&d.st->ticket, 1u);
          s_last = (prev == (unsigned)nslots - 1);
        }
      }
      if constexpr (!ONE) continue;  // a batch's partials are totalled by k_decide after the launch
      __syncthreads();
      if (s_last) {
        __threadfence();
        double tot[2] = {0.0, 0.0}, mtot = 0.0;  // the problem's sum of e, sum of e(new) - e(previous), max |G|
        if constexpr (sizeof(R) == 4) {
          // The partials hold float-float pairs exactly; the block totals them as
          // float-float pairs (TwoSum tree, ~2^-47 relative: far below the FP32
          // per-site rounding). An FP64 total costs this GPU 25-40 us per launch: its
          // FP64 pipe runs at a small fraction of the FP32 rate.
          RPair<R> acc{R(0), R(0)}, dacc{R(0), R(0)};
          R mm = R(0);
          for (int i = tid; i < nslots; i += NT) {
            const FlowPartial* q = d.part + i;
            acc = pair_add(acc, RPair<R>{R(__ldcg(&q->es)), R(__ldcg(&q->ec))});
            dacc = pair_add(dacc, RPair<R>{R(__ldcg(&q->ds)), R(__ldcg(&q->dc))});
            mm = rmax(mm, R(__ldcg(&q->m)));
          }
          tile_reduce<R>(acc, dacc, mm, sred);
          tot[0] = (double)acc.s + (double)acc.c;
          tot[1] = (double)dacc.s + (double)dacc.c;
          mtot = (double)mm;
        } else {
          DD acc{0.0, 0.0}, dacc{0.0, 0.0};
          double mm = 0.0;
          for (int i = tid; i < nslots; i += NT) {
            const FlowPartial* q = d.part + i;
            acc = dd_add(acc, DD{__ldcg(&q->es), __ldcg(&q->ec)});
            dacc = dd_add(dacc, DD{__ldcg(&q->ds), __ldcg(&q->dc)});
            mm = nanmax(mm, __ldcg(&q->m));
          }
          DD sv2[2] = {acc, dacc};
          double mv2[1] = {mm};
          block_reduce<2, 1>(sv2, mv2, dred);
          tot[0] = sv2[0].s + sv2[0].c;
          tot[1] = sv2[1].s + sv2[1].c;
          mtot = mv2[0];
        }
        if (tid == 0 && PASS == 1) {
          DevState* st = d.st;
          const double dE = d.area * tot[1];
          const double E = want_e ? d.area * tot[0] : st->E_last + dE;
          const double g = d.area * mtot;
          // Eq. 4, strict: E_h(phi^n) > E_h(phi^{n-1}); no previous field (E_last = +inf): no arrest
          const int arr = has_prev ? (dE > 0.0 ? 1 : 0) : (E > st->E_last ? 1 : 0);
          st->E_cur = E;
          st->dE = has_prev ? dE : 0.0;
          st->gmax = g;
          st->arrest = arr;
          st->arrests += arr;
          st->E_last = E;
          st->converged = (g < st->tol) ? 1 : 0;
          st->nonfinite = (isfinite(E) && isfinite(g) && isfinite(dE)) ? 0 : 1;
          st->head_step = st->steps;
          st->ticket = 0;
        } else if (tid == 0) {
          // descent: record the evaluated field, count a rise, then take the step
          // (its new field is already written) unless converged or out of budget
          DevState* st = d.st;
          const double E = d.area * tot[0];
          const double g = d.area * mtot;
          const double El = st->E_last;
          const int rose = E > El ? 1 : 0;  // E_last = +inf before the first field
          st->E_cur = E;
          st->dE = isfinite(El) ? E - El : 0.0;
          st->gmax = g;
          st->arrest = rose;
          st->arrests += rose;
          st->E_last = E;
          const int conv = (g < st->tol) ? 1 : 0;
          const int bad = (isfinite(E) && isfinite(g)) ? 0 : 1;
          st->converged = conv;
          st->nonfinite = bad;
          st->head_step = st->steps;
          if (!conv && !bad && st->steps < st->step_limit) st->steps += 1;
          st->ticket = 0;
        }
      }
    } else {
      if constexpr (PK) {
        // stages 3 and 4 in one walk over the pairs (Y_3, Y_4), then the RK4
        // combination at each site
        const F2* ab = reinterpret_cast<const F2*>(setA);
        const Spacing<F2> h2 = bcast(h);
        const Couplings<F2> k2c = bcast(kc);
        StageWin<TH, F2, T::SXY, R> W;
        W.pbase = setP;
#pragma unroll
        for (int s = 0; s < 5; ++s) W.enter(ab, (sy0 - 2 + s) * T::SX + sx, s);
        const R w6 = dt * dt / R(6), u6 = dt / R(6);
        R* __restrict__ phi_out = D.phi[cur ^ 1];
        R* __restrict__ lo_out = D.lo[cur ^ 1];
        R* __restrict__ v_out = D.v[cur ^ 1];
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          const int off = (sy0 + r) * T::SX + sx;
          const bool ok = colok && gyb + r >= 2 && gyb + r < ny - 2;
          const size_t s = (size_t)(gyb + r) * nx + gx;
          SiteVals<TH, R> sv;
          if (SS_PF2 && ok) load_site<TH, R, LO>(sv, phi, lo, vel, kv1, kv2, P, s, arrest);
          F2 v[C], fx[C], fy[C], fxx[C], fyy[C], fxy[C], G[C];
          W.derivs(ab, off, h2, v, fx, fy, fxx, fyy, fxy);
          // site extras: the BEC's position; with demagnetisation psi and its gradient
          R q0 = xs, q1 = ypos(r), ps = R(0);
          if (TH == TH_CMD) W.psi_at(off, h, ps, q0, q1);
          force_at<TH, F2>(k2c, v, fx, fy, fxx, fyy, fxy, G, F2(q0), F2(q1));
          if (ok) {
            R k3[C], k4[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
              k3[c] = -G[c].v.x;
              k4[c] = -G[c].v.y;
            }
            if (!SS_PF2) load_site<TH, R, LO>(sv, phi, lo, vel, kv1, kv2, P, s, arrest);
            combine_loaded<TH, R, LO>(sv, phi_out, lo_out, v_out, P, s, dt, w6, u6, k3, k4);
          }
          if (r + 1 < RY) {
            W.shift();
            W.enter(ab, (sy0 + r + 3) * T::SX + sx, 4);
          }
        }
      } else {
      // stage 3 at Y_3: k_v3 kept in registers
      R k3[RY][C];
      {
        StageWin<TH, R, T::SXY> W;
        W.pbase = setP;
#pragma unroll
        for (int s = 0; s < 5; ++s) W.enter(setA, (sy0 - 2 + s) * T::SX + sx, s);
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          const int off = (sy0 + r) * T::SX + sx;
          R v[C], fx[C], fy[C], fxx[C], fyy[C], fxy[C], G[C];
          W.derivs(setA, off, h, v, fx, fy, fxx, fyy, fxy);
          // site extras: the BEC's position; with demagnetisation psi and its gradient
          R q0 = xs, q1 = ypos(r), ps = R(0);
          if (TH == TH_CMD) W.psi_at(off, h, ps, q0, q1);
          force_at<TH, R>(kc, v, fx, fy, fxx, fyy, fxy, G, q0, q1);
#pragma unroll
          for (int c = 0; c < C; ++c) k3[r][c] = -G[c];
          if (r + 1 < RY) {
            W.shift();
            W.enter(setA, (sy0 + r + 3) * T::SX + sx, 4);
          }
        }
      }
      // stage 4 at Y_4, then the RK4 combination
      {
        StageWin<TH, R, T::SXY> W;
        W.pbase = setP;
#pragma unroll
        for (int s = 0; s < 5; ++s) W.enter(setB, (sy0 - 2 + s) * T::SX + sx, s);
        const R w6 = dt * dt / R(6), u6 = dt / R(6);
        R* __restrict__ phi_out = D.phi[cur ^ 1];
        R* __restrict__ lo_out = D.lo[cur ^ 1];
        R* __restrict__ v_out = D.v[cur ^ 1];
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          const int off = (sy0 + r) * T::SX + sx;
          R v[C], fx[C], fy[C], fxx[C], fyy[C], fxy[C], G[C];
          W.derivs(setB, off, h, v, fx, fy, fxx, fyy, fxy);
          // site extras: the BEC's position; with demagnetisation psi and its gradient
          R q0 = xs, q1 = ypos(r), ps = R(0);
          if (TH == TH_CMD) W.psi_at(off, h, ps, q0, q1);
          force_at<TH, R>(kc, v, fx, fy, fxx, fyy, fxy, G, q0, q1);
          if (colok && gyb + r >= 2 && gyb + r < ny - 2) {
            R k4[C];
#pragma unroll
            for (int c = 0; c < C; ++c) k4[c] = -G[c];
            combine_site<TH, R, LO>(phi, lo, vel, kv1, kv2, phi_out, lo_out, v_out, P, (size_t)(gyb + r) * nx + gx,
                                    arrest, dt, w6, u6, k3[r], k4);
          }
          if (r + 1 < RY) {
            W.shift();
            W.enter(setB, (sy0 + r + 3) * T::SX + sx, 4);
          }
        }
      }
      }
      // The step count selects the ping-pong buffers and gates every tile of this
      // problem, so it advances only when the problem's last run of tiles has arrived
      // (runs as in pass 1: a block's tiles of a problem are consecutive, one arrival
      // per run; its own stores need not be finished: nothing in this launch reads
      // them, and the next launch starts after this one ends).
      const int tn = ONE ? t + (int)gridDim.x : s_next[buf ^ 1];
      const bool run_ends = ONE ? tn >= total_tiles : !(tn < total_tiles && tcb[buf ^ 1].p == tc.p);
      if (run_ends && tid == 0) {
        __threadfence();
        DevState* st = D.st;
        const unsigned prev = atomicAdd(&st->ticket, 1u);
        if (prev == (unsigned)min((int)gridDim.x, D.ntiles) - 1) {
          st->ticket = 0;
          st->steps += 1;
        }
      }
    }
  }
}

// Batched passes 1 and 3 only leave each run's partial sums in its slot. This kernel,
// one block per problem, totals a problem's slots in slot order and decides as the
// single-problem path's last arrival does: Eq. 4 for pass 1, the descent step's record
// for pass 3. Inside the pass kernel the block that completed a problem's count did
// that work, so a block that fell behind completed one count after another (57 of
// the 256 decisions of the 256-problem set in one block, a fifth of the launch).
template <typename R, int PASS>
__global__ void __launch_bounds__(NT) k_decide(const ProbDesc<R>* __restrict__ probs, int nprob, int grid) {
  __shared__ R sred[(NT / 32) * 5];
  __shared__ double dred[RedSmem<2, 1>::n];
  const int p = blockIdx.x;
  if (p >= nprob) return;
  const ProbDesc<R>& d = probs[p];
  DevState* st = d.st;
  if (tile_skip<PASS>(st)) return;  // the pass did not run this problem (its flags as the pass saw them)
  const int tid = threadIdx.y * BX + threadIdx.x;
  const long long steps = st->steps;
  const bool has_prev = PASS == 1 && steps > 0;
  const bool want_e = PASS != 1 || sizeof(R) == 8 || steps == 0 || (steps & (SS_E_EVERY - 1)) == 0 ||
                      steps >= st->step_limit;
  const int nslots = min(grid, d.ntiles);
  double tot[2] = {0.0, 0.0}, mtot = 0.0;
  if constexpr (sizeof(R) == 4) {
    RPair<R> acc{R(0), R(0)}, dacc{R(0), R(0)};
    R mm = R(0);
    for (int i = tid; i < nslots; i += NT) {
      const FlowPartial* q = d.part + i;
      acc = pair_add(acc, RPair<R>{R(q->es), R(q->ec)});
      dacc = pair_add(dacc, RPair<R>{R(q->ds), R(q->dc)});
      mm = rmax(mm, R(q->m));
    }
    tile_reduce<R>(acc, dacc, mm, sred);
    tot[0] = (double)acc.s + (double)acc.c;
    tot[1] = (double)dacc.s + (double)dacc.c;
    mtot = (double)mm;
  } else {
    DD acc{0.0, 0.0}, dacc{0.0, 0.0};
    double mm = 0.0;
    for (int i = tid; i < nslots; i += NT) {
      const FlowPartial* q = d.part + i;
      acc = dd_add(acc, DD{q->es, q->ec});
      dacc = dd_add(dacc, DD{q->ds, q->dc});
      mm = nanmax(mm, q->m);
    }
    DD sv2[2] = {acc, dacc};
    double mv2[1] = {mm};
    block_reduce<2, 1>(sv2, mv2, dred);
    tot[0] = sv2[0].s + sv2[0].c;
    tot[1] = sv2[1].s + sv2[1].c;
    mtot = mv2[0];
  }
  if (tid != 0) return;
  if (PASS == 1) {
    const double dE = d.area * tot[1];
    const double E = want_e ? d.area * tot[0] : st->E_last + dE;
    const double g = d.area * mtot;
    // Eq. 4, strict: E_h(phi^n) > E_h(phi^{n-1}); no previous field (E_last = +inf): no arrest
    const int arr = has_prev ? (dE > 0.0 ? 1 : 0) : (E > st->E_last ? 1 : 0);
    st->E_cur = E;
    st->dE = has_prev ? dE : 0.0;
    st->gmax = g;
    st->arrest = arr;
    st->arrests += arr;
    st->E_last = E;
    st->converged = (g < st->tol) ? 1 : 0;
    st->nonfinite = (isfinite(E) && isfinite(g) && isfinite(dE)) ? 0 : 1;
    st->head_step = st->steps;
  } else {
    // descent: record the evaluated field, count a rise, then take the step (its new
    // field is already written) unless converged or out of budget
    const double E = d.area * tot[0];
    const double g = d.area * mtot;
    const double El = st->E_last;
    const int rose = E > El ? 1 : 0;  // E_last = +inf before the first field
    st->E_cur = E;
    st->dE = isfinite(El) ? E - El : 0.0;
    st->gmax = g;
    st->arrest = rose;
    st->arrests += rose;
    st->E_last = E;
    const int conv = (g < st->tol) ? 1 : 0;
    const int bad = (isfinite(E) && isfinite(g)) ? 0 : 1;
    st->converged = conv;
    st->nonfinite = bad;
    st->head_step = st->steps;
    if (!conv && !bad && st->steps < st->step_limit) st->steps += 1;
  }
  st->ticket = 0;
}

// ------------------------------------------------------------------ launchers
template <int TH, typename R, int TS>
static size_t pass_smem(int pass) {
  return ((size_t)(pass == 1 ? 3 : (pass == 2 ? 2 : 1)) * NComp<TH>::C + (TH == TH_CMD ? 1 : 0)) *
         FlowTile<R, TS>::SXY * sizeof(R);
}

template <int TH, typename R, bool LO, bool ONE, int TS>
static void pass_launch(const BatchLaunch& b, int pass, cudaStream_t s) {
  const ProbDesc<R>* probs = static_cast<const ProbDesc<R>*>(b.probs);
  const ProbDesc<R> one = ONE ? *static_cast<const ProbDesc<R>*>(b.one) : ProbDesc<R>{};
  const dim3 blk(BX, BY);
  if (pass == 1)
    k_pass<TH, R, 1, LO, ONE, TS><<<b.flow_blocks[0], blk, pass_smem<TH, R, TS>(1), s>>>(one, probs, b.tile_prob,
                                                                                          b.total_tiles);
  else if (pass == 2)
    k_pass<TH, R, 2, LO, ONE, TS><<<b.flow_blocks[1], blk, pass_smem<TH, R, TS>(2), s>>>(one, probs, b.tile_prob,
                                                                                          b.total_tiles);
  else
    k_pass<TH, R, 3, LO, ONE, TS><<<b.flow_blocks[2], blk, pass_smem<TH, R, TS>(3), s>>>(one, probs, b.tile_prob,
                                                                                          b.total_tiles);
  if constexpr (!ONE) {  // a batch's decisions, one block per problem
    if (pass == 1) k_decide<R, 1><<<b.nprob, blk, 0, s>>>(probs, b.nprob, b.flow_blocks[0]);
    else if (pass == 3) k_decide<R, 3><<<b.nprob, blk, 0, s>>>(probs, b.nprob, b.flow_blocks[2]);
  }
}
template <int TH, typename R, bool LO>
static cudaError_t pass_t(const BatchLaunch& b, int pass, cudaStream_t s) {
  if (pass < 1 || pass > 3) return cudaErrorInvalidValue;
  if (b.one) {
    if (b.ts) pass_launch<TH, R, LO, true, 1>(b, pass, s);
    else pass_launch<TH, R, LO, true, 0>(b, pass, s);
  } else {
    if (b.ts) pass_launch<TH, R, LO, false, 1>(b, pass, s);
    else pass_launch<TH, R, LO, false, 0>(b, pass, s);
  }
  return cudaGetLastError();
}
template <int TH>
static cudaError_t pass_th(const BatchLaunch& b, int pass, cudaStream_t s) {
  switch (b.prec) {
    case PREC_F32C: return pass_t<TH, float, true>(b, pass, s);
    case PREC_F64: return pass_t<TH, double, false>(b, pass, s);
    default: return pass_t<TH, float, false>(b, pass, s);
  }
}

// Opt the pass kernels into their dynamic shared memory and report how many blocks
// of each pass fit on one SM.
template <int TH, typename R, int PASS, bool LO, bool ONE, int TS>
static void one_occupancy(int* occ) {
  cudaFuncSetAttribute(k_pass<TH, R, PASS, LO, ONE, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)pass_smem<TH, R, TS>(PASS));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_pass<TH, R, PASS, LO, ONE, TS>, NT,
                                                pass_smem<TH, R, TS>(PASS));
}
template <int TH, typename R, bool LO, bool ONE, int TS>
static void pass_occupancy(int occ[3]) {
  one_occupancy<TH, R, 1, LO, ONE, TS>(&occ[0]);
  one_occupancy<TH, R, 2, LO, ONE, TS>(&occ[1]);
  one_occupancy<TH, R, 3, LO, ONE, TS>(&occ[2]);
}

template <int TH, bool ONE, int TS>
static void occupancy_th(int prec, int occ[3]) {
  switch (prec) {
    case PREC_F32C: pass_occupancy<TH, float, true, ONE, TS>(occ); break;
    case PREC_F64: pass_occupancy<TH, double, false, ONE, TS>(occ); break;
    default: pass_occupancy<TH, float, false, ONE, TS>(occ); break;
  }
}

template <int TH>
static void occupancy_sel(int prec, int ts, bool one, int occ[3]) {
  if (one) {
    if (ts) occupancy_th<TH, true, 1>(prec, occ);
    else occupancy_th<TH, true, 0>(prec, occ);
  } else {
    if (ts) occupancy_th<TH, false, 1>(prec, occ);
    else occupancy_th<TH, false, 0>(prec, occ);
  }
}

// One theory's pass launcher and occupancy query, instantiated in its own
// translation unit (ss_flow_<theory>.cu) so that the theories compile in parallel.
template <int TH>
cudaError_t launch_pass_theory(const BatchLaunch& b, int pass, cudaStream_t s) {
  return pass_th<TH>(b, pass, s);
}
template <int TH>
void occupancy_theory(int prec, int ts, bool one, int occ[3]) {
  occupancy_sel<TH>(prec, ts, one, occ);
}

}  // namespace ss
