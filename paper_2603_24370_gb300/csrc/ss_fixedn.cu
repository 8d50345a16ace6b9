// ss_fixedn.cu -- the rotating BEC at a fixed atom number N = int |psi|^2 (the BEC
// section: N is conserved and fixed by the normalisation of psi).
//
// The flow runs on the constraint surface N_h(psi) = dx dy sum_I |psi|^2 = N0 of the
// lattice functional at zero chemical potential. Every new field (psi, v) is
// refreshed before its step:
//   v   <- v - alpha psi on I,  alpha = sum_I v.psi / sum_I |psi|^2  (tangent to the surface;
//                                psi and the scaled psi point the same way),
//   psi <- s psi on I,          s = sqrt(N0 / N_h(psi))              (the halo keeps its values),
//   mu  =  sum_I G_0(psi).psi / (2 sum_I |psi|^2) of the scaled psi  (the Lagrange multiplier),
// and the step's RK stages take the force G_0 - 2 mu psi of the grand-canonical form at
// that mu (held through the step, like the demagnetising potential), which has no
// component along psi; the energy, its change and the arrest test (Eq. 4) are those
// of mu = 0. The previous field in the other ping-pong buffer is a refreshed field
// too, so Eq. 4 compares two fields of the same atom number.
//
// Three launches per refresh, every block skipping unless the problem holds a field
// not refreshed yet (its step count moved since the last refresh) and is running:
//   k_fn_sums   sum_I |psi|^2 and sum_I v.psi (compensated pairs, fixed order); the
//               last block derives s and alpha (a field without atoms stops the flow
//               as non-finite);
//   k_fn_mu     sum_I G_0(psi').psi' and sum_I |psi'|^2 over the scaled field psi' as
//               the flow will see it (the working type's rounding of s psi on I, psi on
//               the halo), staged per tile from the unscaled planes; the last block
//               stores mu;
//   k_fn_apply  psi <- s psi (re-split into value and remainder when compensated),
//               v <- v - alpha psi on I; the last block marks the field refreshed.
#include <cuda_runtime.h>

#include "ss_internal.h"

namespace ss {
namespace {

template <typename R>
struct FnArgs {
  R* phi[2];
  R* lo[2];  // compensated FP32: remainder planes (else null)
  R* v[2];
  int nx, ny;
  size_t plane;
  int ntx, ntiles;  // tiles of the staged kernel
  Spacing<R> h;
  R hx, hy;
  Couplings<R> k0;  // g, Omega; mu = 0
  double n0;        // the atom number held
  double area;      // dx dy
  DevState* st;
  ObsPartial* part;
};

// The last block to arrive (thread 0's view is broadcast through s_last).
__device__ __forceinline__ bool fn_arrive(DevState* st, int tid, int* s_last) {
  if (tid == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&st->fn_ticket, 1u);
    *s_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  const bool last = *s_last != 0;
  if (last) __threadfence();
  return last;
}

// Block sums of two per-thread pairs (thread 0 ends with them), in the working type:
// FP32 pairs for the FP32 kernels (this GPU's FP64 units would stall the SM for
// microseconds on an FP64 tree), FP64 pairs for FP64. sm holds (NT / 32) * 5 values.
template <typename R>
__device__ __forceinline__ void pair_block_sum(RPair<R>& a, RPair<R>& b, R* sm) {
  R m = R(0);
  tile_reduce<R>(a, b, m, sm);
}

// Block partials -> the fixed-order totals of two sums (last block); the partials hold
// the working type's pairs exactly, and are totalled as such (FP32: float-float pairs,
// ~2^-47 relative; an FP64 tree would hold this GPU's slow FP64 pipe for tens of us).
template <typename R>
__device__ __forceinline__ void fn_total(const ObsPartial* part, double& ta, double& tb, R* sm) {
  RPair<R> sa{R(0), R(0)}, sb{R(0), R(0)};
  const int tid = threadIdx.y * BX + threadIdx.x;
  for (int i = tid; i < (int)gridDim.x; i += NT) {
    sa = pair_add(sa, RPair<R>{R(__ldcg(&part[i].es)), R(__ldcg(&part[i].ec))});
    sb = pair_add(sb, RPair<R>{R(__ldcg(&part[i].fs)), R(__ldcg(&part[i].fc))});
  }
  pair_block_sum<R>(sa, sb, sm);
  ta = (double)sa.s + (double)sa.c;
  tb = (double)sb.s + (double)sb.c;
}

// Thread 0 writes the block's pairs as its partial.
template <typename R>
__device__ __forceinline__ void fn_partial(ObsPartial* p, const RPair<R>& a, const RPair<R>& b) {
  p->es = (double)a.s; p->ec = (double)a.c;
  p->fs = (double)b.s; p->fc = (double)b.c;
}

// Per-thread sums of products in the working type's extended precision: FP32 as a
// float-float pair (the product's rounding error recovered by FMA, the running sum by
// TwoSum), FP64 as a plain double. A thread sums tens of terms before the block tree
// of pairs, so both keep ~1e-13 relative, which the arrest test needs of the atom
// number, while the per-site work stays off the FP64 units (a small fraction of the
// FP32 rate on this GPU).
struct AccF {
  float h = 0.f, l = 0.f;
  __device__ __forceinline__ void add(float p, float e) {  // p + e, |e| << |p|
    const float t = h + p, bp = t - h;
    l += ((h - (t - bp)) + (p - bp)) + e;
    h = t;
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = a * b;
    add(p, fmaf(a, b, -p));
  }
  __device__ __forceinline__ void add_small(float x) { l += x; }
  __device__ __forceinline__ RPair<float> pair() const { return RPair<float>{h, l}; }
};
struct AccD {
  double s = 0.0;
  __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ void add_small(double x) { s += x; }
  __device__ __forceinline__ RPair<double> pair() const { return RPair<double>{s, 0.0}; }
};
template <typename R>
struct AccOf { using T = AccF; };
template <>
struct AccOf<double> { using T = AccD; };

// The scale factor in the working type: FP32 as a float pair (s = sh + sl).
struct ScaleF {
  float h, l;
  __device__ explicit ScaleF(double s) : h((float)s), l((float)(s - (double)(float)s)) {}
};
// y = s (hi + lo) as value + remainder: the product's rounding error recovered by FMA
// and the small cross terms added in FP32, then a fast TwoSum (|p| >= |e|), so the
// value is the FP32 rounding of s (hi + lo) to within the remainder's ~1e-14. Both
// the multiplier's staging and the in-place scaling call this, so they agree bitwise.
__device__ __forceinline__ void scale_split(const ScaleF& s, float hi, float lo, float& yh, float& yl) {
  const float p = s.h * hi;
  const float e = fmaf(s.h, hi, -p) + fmaf(s.h, lo, s.l * hi);
  yh = p + e;
  yl = e - (yh - p);
}
struct ScaleD {
  double v;
  __device__ explicit ScaleD(double s) : v(s) {}
};
__device__ __forceinline__ void scale_split(const ScaleD& s, double hi, double lo, double& yh, double& yl) {
  yh = s.v * (hi + lo);
  yl = 0.0;
}
template <typename R>
struct ScaleOf { using T = ScaleF; };
template <>
struct ScaleOf<double> { using T = ScaleD; };

template <typename R>
__global__ void __launch_bounds__(NT) k_fn_sums(FnArgs<R> a) {
  __shared__ R sred[(NT / 32) * 5];
  __shared__ int s_last;
  DevState* st = a.st;
  if (st->nonfinite || st->fn_step == st->steps) return;  // uniform: nothing changes them before the last block
  const int cur = (int)(st->steps & 1);
  const R* __restrict__ f = a.phi[cur];
  const R* __restrict__ lo = a.lo[cur];
  const R* __restrict__ v = a.v[cur];
  const int tid = threadIdx.y * BX + threadIdx.x;
  typename AccOf<R>::T an, av;
  // a block per interior row at a time, its threads along the row (no index division)
  for (int j = HALO + blockIdx.x; j < a.ny - HALO; j += gridDim.x)
    for (int i = HALO + tid; i < a.nx - HALO; i += NT) {
      const size_t s = (size_t)j * a.nx + i;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const R hi = f[c * a.plane + s], l = lo ? lo[c * a.plane + s] : R(0);
        an.add_prod(hi, hi);             // (hi + lo)^2 = hi^2 + 2 hi lo + (lo^2: below the sum's precision)
        an.add_small(R(2) * hi * l);
        av.add_prod(v[c * a.plane + s], hi);  // v.psi: the velocity's own precision suffices
      }
    }
  RPair<R> pn = an.pair(), pv = av.pair();
  pair_block_sum<R>(pn, pv, sred);
  if (tid == 0) fn_partial<R>(a.part + blockIdx.x, pn, pv);
  if (!fn_arrive(st, tid, &s_last)) return;
  double S, V;
  fn_total<R>(a.part, S, V, sred);
  if (tid == 0) {
    st->fn_ticket = 0;
    if (!(S > 0.0) || !isfinite(S) || !isfinite(V)) {
      st->nonfinite = 1;  // no atoms to scale: the flow stops
      return;
    }
    st->fn_scale = sqrt(a.n0 / (a.area * S));
    st->fn_alpha = V / S;
    st->fn_pending = 1;
  }
}

template <typename R>
__global__ void __launch_bounds__(NT) k_fn_mu(FnArgs<R> a) {
  constexpr int RPT = TY / BY;  // rows per thread
  __shared__ R sY[2][SY * SX];
  __shared__ R sred[(NT / 32) * 5];
  __shared__ int s_last;
  DevState* st = a.st;
  if (!st->fn_pending) return;
  const int cur = (int)(st->steps & 1);
  const R* __restrict__ f = a.phi[cur];
  const R* __restrict__ lo = a.lo[cur];
  const typename ScaleOf<R>::T sc(st->fn_scale);
  const int tid = threadIdx.y * BX + threadIdx.x;
  typename AccOf<R>::T ag, an;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const int x0 = (t % a.ntx) * TX, y0 = (t / a.ntx) * TY;
    __syncthreads();
    for (int idx = tid; idx < SX * SY; idx += NT) {
      const int lx = idx % SX, ly = idx / SX;
      const int gx = x0 + lx - HALO, gy = y0 + ly - HALO;
      const bool in = gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny;
      const bool inside = gx >= HALO && gx < a.nx - HALO && gy >= HALO && gy < a.ny - HALO;
      const size_t s = (size_t)gy * a.nx + gx;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        R y = R(0);
        if (in) {
          y = f[c * a.plane + s];
          if (inside) {  // what the flow will read after k_fn_apply
            R yl;
            scale_split(sc, y, lo ? lo[c * a.plane + s] : R(0), y, yl);
          }
        }
        sY[c][idx] = y;
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int lx = threadIdx.x, ly = threadIdx.y + r * BY;
      const int gx = x0 + lx, gy = y0 + ly;
      if (gx < HALO || gx >= a.nx - HALO || gy < HALO || gy >= a.ny - HALO) continue;
      const int sx = lx + HALO, sy = ly + HALO;
      R v[2], fx[2], fy[2], fxx[2], fyy[2], G[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const Deriv<R> d = stencil<R, true, false>(sY[c], sx, sy, a.h);
        v[c] = d.v; fx[c] = d.fx; fy[c] = d.fy; fxx[c] = d.fxx; fyy[c] = d.fyy;
      }
      const R x = (R(gx) - R(0.5) * R(a.nx - 1)) * a.hx, y = (R(gy) - R(0.5) * R(a.ny - 1)) * a.hy;
      force_bec<R>(a.k0, v, fx, fy, fxx, fyy, x, y, G);
      ag.add_prod(G[0], v[0]);
      ag.add_prod(G[1], v[1]);
      an.add_prod(v[0], v[0]);
      an.add_prod(v[1], v[1]);
    }
  }
  RPair<R> pg = ag.pair(), pn = an.pair();
  pair_block_sum<R>(pg, pn, sred);
  if (tid == 0) fn_partial<R>(a.part + blockIdx.x, pg, pn);
  if (!fn_arrive(st, tid, &s_last)) return;
  double tg, tn;
  fn_total<R>(a.part, tg, tn, sred);
  if (tid == 0) {
    st->fn_ticket = 0;
    st->mu_held = tg / (2.0 * tn);
  }
}

template <typename R>
__global__ void __launch_bounds__(NT) k_fn_apply(FnArgs<R> a) {
  __shared__ int s_last;
  DevState* st = a.st;
  if (!st->fn_pending) return;
  const int cur = (int)(st->steps & 1);
  R* __restrict__ f = a.phi[cur];
  R* __restrict__ lo = a.lo[cur];
  R* __restrict__ v = a.v[cur];
  const typename ScaleOf<R>::T sc(st->fn_scale);
  const R al = R(st->fn_alpha);
  const int tid = threadIdx.y * BX + threadIdx.x;
  for (int j = HALO + blockIdx.x; j < a.ny - HALO; j += gridDim.x)
    for (int i = HALO + tid; i < a.nx - HALO; i += NT) {
      const size_t s = (size_t)j * a.nx + i;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const size_t k = c * a.plane + s;
        const R hi = f[k], l = lo ? lo[k] : R(0);
        v[k] = v[k] - al * hi;  // alpha psi: the velocity's own precision suffices
        R yh, yl;
        scale_split(sc, hi, l, yh, yl);
        f[k] = yh;
        if (lo) lo[k] = yl;
      }
    }
  if (!fn_arrive(st, tid, &s_last)) return;
  if (tid == 0) {
    st->fn_ticket = 0;
    st->fn_pending = 0;
    st->fn_step = st->steps;
  }
}

template <typename R>
cudaError_t fixed_n_t(const FixedNLaunch& L, cudaStream_t s) {
  FnArgs<R> a{};
  for (int k = 0; k < 2; ++k) {
    a.phi[k] = static_cast<R*>(L.phi[k]);
    a.lo[k] = static_cast<R*>(L.lo[k]);
    a.v[k] = static_cast<R*>(L.v[k]);
  }
  a.nx = L.nx;
  a.ny = L.ny;
  a.plane = (size_t)L.nx * L.ny;
  a.ntx = (L.nx + TX - 1) / TX;
  a.ntiles = a.ntx * ((L.ny + TY - 1) / TY);
  a.h.i12dx = R(1.0 / (12.0 * L.dx));
  a.h.i12dy = R(1.0 / (12.0 * L.dy));
  a.h.i12dx2 = R(1.0 / (12.0 * L.dx * L.dx));
  a.h.i12dy2 = R(1.0 / (12.0 * L.dy * L.dy));
  a.h.i144dxdy = R(1.0 / (144.0 * L.dx * L.dy));
  a.hx = R(L.dx);
  a.hy = R(L.dy);
  a.k0.c[0] = R(L.g);
  a.k0.c[1] = R(L.omega);
  a.n0 = L.atoms;
  a.area = L.dx * L.dy;
  a.st = L.st;
  a.part = L.part;
  int g1 = L.ny - 2 * HALO;  // interior rows
  if (g1 > L.blocks) g1 = L.blocks;
  int g2 = a.ntiles < L.blocks ? a.ntiles : L.blocks;
  const dim3 blk(BX, BY);
  k_fn_sums<R><<<g1, blk, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_fn_mu<R><<<g2, blk, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_fn_apply<R><<<g1, blk, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fixed_n_refresh(const FixedNLaunch& L, cudaStream_t s) {
  return L.prec == PREC_F64 ? fixed_n_t<double>(L, s) : fixed_n_t<float>(L, s);
}

}  // namespace ss
