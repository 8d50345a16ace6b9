// ss_flow.cu -- the arrested-Newton-flow step (arxiv 2603.24370, Sec. 3.2) as two
// fused passes over the grid.
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
// Pass 1 also reduces E_h(phi) (a compensated pair per thread, FP64 TwoSum warp
// trees, one partial per block, the last-arriving block sums the partials in a
// fixed order), dx dy max|G|, and the energy change since the previous field,
// dE = sum_I [e(phi^n) - e(phi^{n-1})] in the cancellation-free form of
// ss_device.cuh (phi^{n-1} is still intact in the other ping-pong buffer). Its last
// block then decides on the device, with no host round trip:
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

// Per block a tile of TX x TY sites is staged in shared memory with its halo, the
// stage inputs formed while loading (two sites per iteration, loads first). Each
// thread then walks RY rows of one column with a 5-row register window per
// component. Blocks stride over tiles; the grid is occupancy x SM count.
#include "ss_internal.h"

namespace ss {

template <typename R>
struct FlowTile {
  static constexpr int RY = sizeof(R) == 4 ? 4 : 2;  // rows per thread
  static constexpr int TX = 32, TY = BY * RY;
  static constexpr int SX = TX + 4, SY = TY + 4, SXY = SX * SY;
};

template <typename R>
struct PassArgs {
  const R* __restrict__ phi;       // phi^n (current field; hi part when compensated)
  const R* __restrict__ lo;        // LO: remainder part of phi^n
  const R* __restrict__ phi_prev;  // pass 1: phi^{n-1} (other ping-pong buffer)
  const R* __restrict__ lo_prev;   // LO pass 1: remainder part of phi^{n-1}
  const R* __restrict__ v;         // v^n
  const R* __restrict__ kv1;       // pass 2
  const R* __restrict__ kv2;       // pass 2
  R* __restrict__ kv1_out;         // pass 1
  R* __restrict__ kv2_out;         // pass 1
  R* __restrict__ phi_out;         // pass 2: phi^{n+1} (hi)
  R* __restrict__ lo_out;          // LO pass 2: remainder part of phi^{n+1}
  R* __restrict__ v_out;           // pass 2: v^{n+1}
  int nx, ny;
  size_t plane;
  int ntx, ntiles;
  R dt;
  Spacing<R> h;
  Couplings<R> k;
  double area;  // dx dy
  DevState* st;
  FlowPartial* part;
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

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

// Split-form projection onto the unit sphere: given hi (FP32) and a small part t,
// return t' with hi + t' = (hi + t) / |hi + t| to about eps^2. With
// eta = |hi + t|^2 - 1 = (|hi|^2 - 1) + 2 hi.t + |t|^2, where |hi|^2 - 1 is formed
// exactly (error-free products and sums), 1/|hi + t| = 1 + rho with
// rho = -eta / (r (1 + r)), r = sqrt(1 + eta), and t' = t + rho (hi + t).
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
  const float r = sqrtf(1.0f + eta);
  const float rho = -eta / (r * (1.0f + r));
#pragma unroll
  for (int c = 0; c < 3; ++c) t[c] = t[c] + rho * (hi[c] + t[c]);
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
    fx = gx * h.i12dx;        // Eq. 1, x
    fy = yd1(c) * h.i12dy;    // Eq. 1, y
    if (SECOND) {
      fxx = gxx * h.i12dx2;   // Eq. 2, x
      fyy = yd2(c) * h.i12dy2;  // Eq. 2, y
    } else {
      fxx = fyy = R(0);
    }
    fxy = MIX ? (R(8) * (g[3] - g[1]) - (g[4] - g[0])) * h.i144dxdy : R(0);  // Eq. 1 in y of Eq. 1 in x
  }
};

// Window set of one stage input: all C components, mixed derivatives for the gauge
// field of the Abelian Higgs model (components 2, 3).
template <int TH, typename R>
struct StageWin {
  static constexpr int C = NComp<TH>::C;
  static constexpr int SXY = FlowTile<R>::SXY;
  Win<R, false> w0, w1;
  Win<R, TH == TH_AH> w2;
  Win<R, TH == TH_AH> w3;  // unused for the chiral magnet

  __device__ __forceinline__ void enter(const R* tiles, int off, int slot) {
    w0.enter(tiles + off, slot);
    w1.enter(tiles + SXY + off, slot);
    w2.enter(tiles + 2 * SXY + off, slot);
    if (C == 4) w3.enter(tiles + 3 * SXY + off, slot);
  }
  __device__ __forceinline__ void shift() {
    w0.shift();
    w1.shift();
    w2.shift();
    if (C == 4) w3.shift();
  }
  __device__ __forceinline__ void derivs(const R* tiles, int off, const Spacing<R>& h, R* v, R* fx, R* fy, R* fxx,
                                         R* fyy, R* fxy) const {
    w0.template derivs<true>(tiles + off, h, v[0], fx[0], fy[0], fxx[0], fyy[0], fxy[0]);
    w1.template derivs<true>(tiles + SXY + off, h, v[1], fx[1], fy[1], fxx[1], fyy[1], fxy[1]);
    w2.template derivs<true>(tiles + 2 * SXY + off, h, v[2], fx[2], fy[2], fxx[2], fyy[2], fxy[2]);
    if (C == 4) w3.template derivs<true>(tiles + 3 * SXY + off, h, v[3], fx[3], fy[3], fxx[3], fyy[3], fxy[3]);
  }
};

// First derivatives only (the field difference of the arrest test): one plane set.
template <int TH, typename R>
struct DiffWin {
  static constexpr int C = NComp<TH>::C;
  static constexpr int SXY = FlowTile<R>::SXY;
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
                                         const R* fyy, const R* fxy, R* G) {
  if (TH == TH_AH) force_ah<R>(k, v, fx, fy, fxx, fyy, fxy, G);
  else force_cm<R>(k, v, fx, fy, fxx, fyy, G);
}

// Tile sets in shared memory (each C planes of SXY values): pass 1 [Y1 | Y2 | delta],
// pass 2 [Y3 | Y4]. LO: compensated FP32 storage (value + remainder planes).
template <int TH, typename R, int PASS, bool LO>
__global__ void __launch_bounds__(NT) k_pass(PassArgs<R> a) {
  using T = FlowTile<R>;
  constexpr int C = NComp<TH>::C;
  constexpr int RY = T::RY;
  constexpr int PS = C * T::SXY;  // values per tile set
  extern __shared__ __align__(16) unsigned char smraw[];
  R* sm = reinterpret_cast<R*>(smraw);
  __shared__ double sred[RedSmem<2, 1>::n];
  __shared__ int s_last;

  DevState* st = a.st;
  // Uniform over the grid (the record only changes between launches). Pass 1 runs
  // once per field; pass 2 stops at convergence, at a non-finite value and at the
  // step limit of the current call.
  if (st->converged | st->nonfinite) return;
  if (PASS == 1 ? (st->head_step == st->steps) : (st->steps >= st->step_limit)) return;
  const int tid = threadIdx.y * BX + threadIdx.x;
  const bool arrest = (PASS == 2) && (st->arrest != 0);
  const bool has_prev = (PASS == 1) && (st->steps > 0);
  const size_t P = a.plane;
  const R dt = a.dt, hdt = R(0.5) * a.dt;
  const R c3 = R(0.25) * dt * dt, c4 = R(0.5) * dt * dt;
  R* const setA = sm;           // first stage input of the pass
  R* const setB = sm + PS;      // second stage input
  R* const setD = sm + 2 * PS;  // pass 1: phi^n - phi^{n-1}

  R es = R(0), ec = R(0), ds = R(0), dc = R(0), gmr = R(0);

  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const int x0 = (t % a.ntx) * T::TX, y0 = (t / a.ntx) * T::TY;
    __syncthreads();  // the previous tile's shared reads are finished
    // ---- stage inputs over the tile and its halo, two sites per iteration
    for (int base = tid; base < T::SXY; base += 2 * NT) {
      R pv[2][C], lv[2][C], vv[2][C], k1v[2][C], k2v[2][C], pp[2][C], lp[2][C];
      bool in[2], inside[2];
      size_t sidx[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {  // all global loads of both sites first
        const int idx = base + u * NT;
        const int ly = idx / T::SX, lx = idx - ly * T::SX;
        const int gx = x0 + lx - 2, gy = y0 + ly - 2;
        in[u] = idx < T::SXY && gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny;
        inside[u] = in[u] && gx >= 2 && gx < a.nx - 2 && gy >= 2 && gy < a.ny - 2;
        const size_t s = in[u] ? (size_t)gy * a.nx + gx : 0;
        sidx[u] = s;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          pv[u][c] = in[u] ? a.phi[c * P + s] : R(0);
          lv[u][c] = (LO && in[u]) ? a.lo[c * P + s] : R(0);
          vv[u][c] = (inside[u] && !arrest) ? a.v[c * P + s] : R(0);
          if (PASS == 1) {
            pp[u][c] = (has_prev && in[u]) ? a.phi_prev[c * P + s] : pv[u][c];
            lp[u][c] = (LO && has_prev && in[u]) ? a.lo_prev[c * P + s] : lv[u][c];
          } else {
            k1v[u][c] = inside[u] ? a.kv1[c * P + s] : R(0);
            k2v[u][c] = inside[u] ? (arrest ? k1v[u][c] : a.kv2[c * P + s]) : R(0);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int idx = base + u * NT;
        if (idx >= T::SXY) break;
        R ya[C], yb[C], yd[C];
        if (PASS == 1) {
#pragma unroll
          for (int c = 0; c < C; ++c) {
            // delta = phi^n - phi^{n-1} (differences of neighbouring values: exact per part)
            yd[c] = LO ? (pv[u][c] - pp[u][c]) + (lv[u][c] - lp[u][c]) : pv[u][c] - pp[u][c];
            if (LO) {
              ya[c] = lv[u][c];
              yb[c] = lv[u][c] + hdt * vv[u][c];
            } else {
              ya[c] = pv[u][c];
              yb[c] = pv[u][c] + hdt * vv[u][c];
            }
          }
          if (TH == TH_CM && inside[u]) {
            if constexpr (LO) normalise_split(pv[u], yb);
            else normalise<C>(yb);
          }
          if (LO) {  // stage inputs: value + small part, rounded once
#pragma unroll
            for (int c = 0; c < C; ++c) {
              ya[c] = pv[u][c] + ya[c];
              yb[c] = pv[u][c] + yb[c];
            }
          }
        } else {
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const R base3 = hdt * vv[u][c] + c3 * k1v[u][c];
            const R base4 = dt * vv[u][c] + c4 * k2v[u][c];
            ya[c] = LO ? lv[u][c] + base3 : pv[u][c] + base3;
            yb[c] = LO ? lv[u][c] + base4 : pv[u][c] + base4;
          }
          if (TH == TH_CM && inside[u]) {
            if constexpr (LO) {
              normalise_split(pv[u], ya);
              normalise_split(pv[u], yb);
            } else {
              normalise<C>(ya);
              normalise<C>(yb);
            }
          }
          if (LO) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
              ya[c] = pv[u][c] + ya[c];
              yb[c] = pv[u][c] + yb[c];
            }
          }
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
          setA[c * T::SXY + idx] = ya[c];
          setB[c * T::SXY + idx] = yb[c];
          if (PASS == 1) setD[c * T::SXY + idx] = has_prev ? yd[c] : R(0);
        }
      }
    }
    __syncthreads();

    // ---- column walk: RY rows of column threadIdx.x
    const int sx = threadIdx.x + 2, sy0 = threadIdx.y * RY + 2;
    const int gx = x0 + threadIdx.x, gyb = y0 + threadIdx.y * RY;
    const bool colok = gx >= 2 && gx < a.nx - 2;

    if (PASS == 1) {
      // stage 1 at Y_1 = phi: k_v1, e, max|G|, and e(phi^n) - e(phi^{n-1})
      {
        StageWin<TH, R> W;
        DiffWin<TH, R> D;
#pragma unroll
        for (int s = 0; s < 5; ++s) {
          const int off = (sy0 - 2 + s) * T::SX + sx;
          W.enter(setA, off, s);
          if (has_prev) D.enter(setD, off, s);
        }
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          const int off = (sy0 + r) * T::SX + sx;
          const bool ok = colok && gyb + r >= 2 && gyb + r < a.ny - 2;
          R v[C], fx[C], fy[C], fxx[C], fyy[C], fxy[C], G[C];
          W.derivs(setA, off, a.h, v, fx, fy, fxx, fyy, fxy);
          force_at<TH, R>(a.k, v, fx, fy, fxx, fyy, fxy, G);
          if (ok) {
            const size_t s = (size_t)(gyb + r) * a.nx + gx;
#pragma unroll
            for (int c = 0; c < C; ++c) {
              a.kv1_out[c * P + s] = -G[c];
              const R ag = fabs(G[c]);
              gmr = (ag > gmr || ag != ag) ? ag : gmr;
            }
            const R e = (TH == TH_AH) ? density_ah<R>(a.k, v, fx, fy) : density_cm<R>(a.k, v, fx, fy);
            const R t1 = es + e;
            ec += (fabs(es) >= fabs(e)) ? (es - t1) + e : (e - t1) + es;
            es = t1;
          }
          if (has_prev) {
            R d[C], dxv[C], dyv[C];
            D.derivs(setD, off, a.h, d, dxv, dyv);
            if (ok) {
              const R de = (TH == TH_AH) ? delta_density_ah<R>(a.k, v, fx, fy, d, dxv, dyv)
                                         : delta_density_cm<R>(a.k, v, fx, fy, d, dxv, dyv);
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
        StageWin<TH, R> W;
#pragma unroll
        for (int s = 0; s < 5; ++s) W.enter(setB, (sy0 - 2 + s) * T::SX + sx, s);
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          const int off = (sy0 + r) * T::SX + sx;
          R v[C], fx[C], fy[C], fxx[C], fyy[C], fxy[C], G[C];
          W.derivs(setB, off, a.h, v, fx, fy, fxx, fyy, fxy);
          force_at<TH, R>(a.k, v, fx, fy, fxx, fyy, fxy, G);
          if (colok && gyb + r >= 2 && gyb + r < a.ny - 2) {
            const size_t s = (size_t)(gyb + r) * a.nx + gx;
#pragma unroll
            for (int c = 0; c < C; ++c) a.kv2_out[c * P + s] = -G[c];
          }
          if (r + 1 < RY) {
            W.shift();
            W.enter(setB, (sy0 + r + 3) * T::SX + sx, 4);
          }
        }
      }
    } else {
      // stage 3 at Y_3: k_v3 kept in registers
      R k3[RY][C];
      {
        StageWin<TH, R> W;
#pragma unroll
        for (int s = 0; s < 5; ++s) W.enter(setA, (sy0 - 2 + s) * T::SX + sx, s);
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          const int off = (sy0 + r) * T::SX + sx;
          R v[C], fx[C], fy[C], fxx[C], fyy[C], fxy[C], G[C];
          W.derivs(setA, off, a.h, v, fx, fy, fxx, fyy, fxy);
          force_at<TH, R>(a.k, v, fx, fy, fxx, fyy, fxy, G);
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
        StageWin<TH, R> W;
#pragma unroll
        for (int s = 0; s < 5; ++s) W.enter(setB, (sy0 - 2 + s) * T::SX + sx, s);
        const R w6 = dt * dt / R(6), u6 = dt / R(6);
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          const int off = (sy0 + r) * T::SX + sx;
          R v[C], fx[C], fy[C], fxx[C], fyy[C], fxy[C], G[C];
          W.derivs(setB, off, a.h, v, fx, fy, fxx, fyy, fxy);
          force_at<TH, R>(a.k, v, fx, fy, fxx, fyy, fxy, G);
          if (colok && gyb + r >= 2 && gyb + r < a.ny - 2) {
            const size_t s = (size_t)(gyb + r) * a.nx + gx;
            R p0[C], q[C], vn[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
              p0[c] = a.phi[c * P + s];
              const R v0 = arrest ? R(0) : a.v[c * P + s];
              const R k1 = a.kv1[c * P + s];
              const R k2 = arrest ? k1 : a.kv2[c * P + s];
              const R k4 = -G[c];
              // increment of phi; with compensated storage it joins the stored lo part
              const R inc = dt * v0 + w6 * (k1 + k2 + k3[r][c]);
              q[c] = LO ? a.lo[c * P + s] + inc : p0[c] + inc;
              vn[c] = v0 + u6 * (k1 + R(2) * (k2 + k3[r][c]) + k4);
            }
            R pn[C], ln[C];
            if constexpr (LO) {
              if (TH == TH_CM) normalise_split(p0, q);
#pragma unroll
              for (int c = 0; c < C; ++c) two_sum_f(p0[c], q[c], pn[c], ln[c]);  // hi' = fl(hi + small), lo' = rest
            } else {
#pragma unroll
              for (int c = 0; c < C; ++c) pn[c] = q[c];
              if (TH == TH_CM) normalise<C>(pn);
            }
            if (TH == TH_CM) {
              const R vp = vn[0] * pn[0] + vn[1] * pn[1] + vn[2] * pn[2];
#pragma unroll
              for (int c = 0; c < C; ++c) vn[c] -= vp * pn[c];
            }
#pragma unroll
            for (int c = 0; c < C; ++c) {
              a.phi_out[c * P + s] = pn[c];
              if (LO) a.lo_out[c * P + s] = ln[c];
              a.v_out[c * P + s] = vn[c];
            }
          }
          if (r + 1 < RY) {
            W.shift();
            W.enter(setB, (sy0 + r + 3) * T::SX + sx, 4);
          }
        }
      }
    }
  }

  if (PASS == 2) {
    if (blockIdx.x == 0 && tid == 0) st->steps += 1;  // single writer; read after this launch
    return;
  }

  // ---- energy / residual reduction and the on-device arrest + convergence decision
  DD sv[2] = {DD{(double)es, (double)ec}, DD{(double)ds, (double)dc}};
  double mv[1] = {(double)gmr};
  block_reduce<2, 1>(sv, mv, sred);
  if (tid == 0) {
    a.part[blockIdx.x] = FlowPartial{sv[0].s, sv[0].c, sv[1].s, sv[1].c, mv[0], {0.0, 0.0, 0.0}};
    __threadfence();
    const unsigned prev = atomicAdd(&st->ticket, 1u);
    s_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  DD acc{0.0, 0.0}, dacc{0.0, 0.0};
  double mm = 0.0;
  for (int i = tid; i < (int)gridDim.x; i += NT) {
    const FlowPartial* q = a.part + i;
    acc = dd_add(acc, DD{__ldcg(&q->es), __ldcg(&q->ec)});
    dacc = dd_add(dacc, DD{__ldcg(&q->ds), __ldcg(&q->dc)});
    mm = nanmax(mm, __ldcg(&q->m));
  }
  DD sv2[2] = {acc, dacc};
  double mv2[1] = {mm};
  block_reduce<2, 1>(sv2, mv2, sred);
  if (tid == 0) {
    const double E = a.area * (sv2[0].s + sv2[0].c);
    const double dE = a.area * (sv2[1].s + sv2[1].c);
    const double g = a.area * mv2[0];
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
  }
}

// ------------------------------------------------------------------ control kernels
__global__ void k_reset_state(DevState* st) {
  st->E_last = __longlong_as_double(0x7ff0000000000000LL);  // +inf: no arrest on the first step
  st->E_cur = 0.0;
  st->dE = 0.0;
  st->gmax = 0.0;
  st->tol = -1.0;
  st->steps = 0;
  st->arrests = 0;
  st->head_step = -1;
  st->step_limit = 0;
  st->arrest = 0;
  st->converged = 0;
  st->nonfinite = 0;
  st->ticket = 0;
  st->obs_ticket = 0;
}

// Start of a run: threshold, step budget, and the convergence verdict of an
// already-evaluated head under the new threshold.
__global__ void k_set_run(DevState* st, double tol, long long max_steps) {
  st->tol = tol;
  st->step_limit = st->steps + max_steps;
  st->converged = (st->head_step == st->steps && st->gmax < tol) ? 1 : 0;
}

template <typename R>
__global__ void k_scaled_copy(R* __restrict__ out, const R* __restrict__ in, size_t n, R scale) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = scale * in[i];
}

// ------------------------------------------------------------------ launchers
template <int TH, typename R>
static size_t pass_smem(int pass) {
  const int sets = pass == 1 ? 3 : 2;
  return (size_t)sets * NComp<TH>::C * FlowTile<R>::SXY * sizeof(R);
}

template <typename R>
static PassArgs<R> make_args(const LaunchCtx& c, int cur) {
  PassArgs<R> a{};
  const int nxt = cur ^ 1;
  a.phi = static_cast<const R*>(c.phi[cur]);
  a.lo = static_cast<const R*>(c.lo[cur]);
  a.phi_prev = static_cast<const R*>(c.phi[nxt]);
  a.lo_prev = static_cast<const R*>(c.lo[nxt]);
  a.v = static_cast<const R*>(c.v[cur]);
  a.kv1 = static_cast<const R*>(c.kv[0]);
  a.kv2 = static_cast<const R*>(c.kv[1]);
  a.kv1_out = static_cast<R*>(c.kv[0]);
  a.kv2_out = static_cast<R*>(c.kv[1]);
  a.phi_out = static_cast<R*>(c.phi[nxt]);
  a.lo_out = static_cast<R*>(c.lo[nxt]);
  a.v_out = static_cast<R*>(c.v[nxt]);
  a.nx = c.nx;
  a.ny = c.ny;
  a.plane = c.plane;
  a.ntx = (c.nx + FlowTile<R>::TX - 1) / FlowTile<R>::TX;
  a.ntiles = a.ntx * ((c.ny + FlowTile<R>::TY - 1) / FlowTile<R>::TY);
  a.dt = (R)c.dt;
  a.h.i12dx = (R)(1.0 / (12.0 * c.dx));
  a.h.i12dy = (R)(1.0 / (12.0 * c.dy));
  a.h.i12dx2 = (R)(1.0 / (12.0 * c.dx * c.dx));
  a.h.i12dy2 = (R)(1.0 / (12.0 * c.dy * c.dy));
  a.h.i144dxdy = (R)(1.0 / (144.0 * c.dx * c.dy));
  for (int i = 0; i < 10; ++i) a.k.c[i] = (R)c.coup[i];
  a.area = c.dx * c.dy;
  a.st = c.st;
  a.part = c.fpart;
  return a;
}

template <int TH, typename R, bool LO>
static cudaError_t pass_t(const LaunchCtx& c, int pass, int cur, cudaStream_t s) {
  const PassArgs<R> a = make_args<R>(c, cur);
  const dim3 blk(BX, BY);
  if (pass == 1) k_pass<TH, R, 1, LO><<<c.flow_blocks, blk, pass_smem<TH, R>(1), s>>>(a);
  else if (pass == 2) k_pass<TH, R, 2, LO><<<c.flow_blocks, blk, pass_smem<TH, R>(2), s>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <int TH>
static cudaError_t pass_th(const LaunchCtx& c, int pass, int cur, cudaStream_t s) {
  switch (c.prec) {
    case PREC_F32C: return pass_t<TH, float, true>(c, pass, cur, s);
    case PREC_F64: return pass_t<TH, double, false>(c, pass, cur, s);
    default: return pass_t<TH, float, false>(c, pass, cur, s);
  }
}

cudaError_t launch_pass(const LaunchCtx& c, int pass, int cur, cudaStream_t s) {
  return c.theory == TH_AH ? pass_th<TH_AH>(c, pass, cur, s) : pass_th<TH_CM>(c, pass, cur, s);
}

cudaError_t launch_reset_state(const LaunchCtx& c, cudaStream_t s) {
  k_reset_state<<<1, 1, 0, s>>>(c.st);
  return cudaGetLastError();
}

cudaError_t launch_set_run(const LaunchCtx& c, double tol, long long max_steps, cudaStream_t s) {
  k_set_run<<<1, 1, 0, s>>>(c.st, tol, max_steps);
  return cudaGetLastError();
}

cudaError_t launch_scaled_copy(const LaunchCtx& c, void* out, const void* in, double scale, cudaStream_t s) {
  const int C = c.theory == TH_AH ? 4 : 3;
  const size_t n = (size_t)C * c.plane;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = (int)((n + 255) / 256 < (size_t)nsm * 8 ? (n + 255) / 256 : (size_t)nsm * 8);
  if (c.prec != PREC_F64) k_scaled_copy<float><<<blocks, 256, 0, s>>>((float*)out, (const float*)in, n, (float)scale);
  else k_scaled_copy<double><<<blocks, 256, 0, s>>>((double*)out, (const double*)in, n, scale);
  return cudaGetLastError();
}

// Opt the pass kernels into their dynamic shared memory, then size the grid by
// the smaller occupancy of the two passes.
template <int TH, typename R, bool LO>
static int pass_occupancy() {
  cudaFuncSetAttribute(k_pass<TH, R, 1, LO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pass_smem<TH, R>(1));
  cudaFuncSetAttribute(k_pass<TH, R, 2, LO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pass_smem<TH, R>(2));
  int b1 = 0, b2 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_pass<TH, R, 1, LO>, NT, pass_smem<TH, R>(1));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_pass<TH, R, 2, LO>, NT, pass_smem<TH, R>(2));
  const int m = b1 < b2 ? b1 : b2;
  return m < 1 ? 1 : m;
}

template <int TH>
static int occupancy_th(int prec) {
  switch (prec) {
    case PREC_F32C: return pass_occupancy<TH, float, true>();
    case PREC_F64: return pass_occupancy<TH, double, false>();
    default: return pass_occupancy<TH, float, false>();
  }
}

int flow_grid(int theory, int prec, int nx, int ny) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int occ = theory == TH_AH ? occupancy_th<TH_AH>(prec) : occupancy_th<TH_CM>(prec);
  int ntiles;
  if (prec == PREC_F64)
    ntiles = ((nx + FlowTile<double>::TX - 1) / FlowTile<double>::TX) *
             ((ny + FlowTile<double>::TY - 1) / FlowTile<double>::TY);
  else
    ntiles = ((nx + FlowTile<float>::TX - 1) / FlowTile<float>::TX) *
             ((ny + FlowTile<float>::TY - 1) / FlowTile<float>::TY);
  const int g = nsm * occ;
  return ntiles < g ? ntiles : g;
}

}  // namespace ss
