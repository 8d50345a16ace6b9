// ss_flow.cu -- the arrested-Newton-flow step (arxiv 2603.24370, Sec. 3.2).
//
// One RK4 step of phi'' = -G(phi) (Eq. 3) on the first-order system (phi, v) is
// four stage kernels. Writing k_vi = -G(Y_i) for the stage inputs Y_i, classic RK4
// reads
//   Y_1 = phi,  Y_2 = phi + dt/2 v,  Y_3 = phi + dt/2 v + dt^2/4 k_v1,
//   Y_4 = phi + dt v + dt^2/2 k_v2,
//   phi' = phi + dt v + dt^2/6 (k_v1 + k_v2 + k_v3),
//   v'   = v + dt/6 (k_v1 + 2 k_v2 + 2 k_v3 + k_v4),
// which is the textbook (k_phi, k_v) form with every k_phi eliminated, so no k_phi
// array is ever stored. Chiral magnet: every Y_i and phi' are normalised and v'
// is tangent-projected (Sec. 3.2, constraint projection).
//
// Stage 1 also reduces E_h(phi) (a compensated pair per thread, FP64 TwoSum warp
// trees, one partial per block, the last-arriving block sums the partials in a
// fixed order) and dx dy max|G|, and then decides on the device, with no host
// round trip:
//   arrest    = E_h(phi^n) > E_h(phi^{n-1})   (Eq. 4; stages 2-4 then use v = 0)
//   converged = dx dy max|G| < tol            (stages of later steps become no-ops)
// Because the arrest of step n-1 -> n is only needed by stage 2 of step n, zeroing
// v is lazy: no extra pass over memory.
//
// Each stage loads its input Y over a (TX+4) x (TY+4) shared tile (the width-2 halo
// of Eq. 1 / Eq. 2), evaluates Eq. 1, Eq. 2 and the mixed derivative from shared
// memory and writes C values per interior site. Blocks stride over tiles, so the
// grid is a multiple of the SM count and the reduction has one partial per block.
#include "ss_internal.h"

namespace ss {

template <typename R>
struct StageArgs {
  const R* __restrict__ phi;   // phi^n (current field)
  const R* __restrict__ v;     // v^n
  const R* __restrict__ kvin;  // stage 3: k_v1, stage 4: k_v2 (part of Y)
  const R* __restrict__ kv1;   // stage 4 combine
  const R* __restrict__ kv2;
  const R* __restrict__ kv3;
  R* __restrict__ kv_out;      // stages 1-3: k_vs
  R* __restrict__ phi_out;     // stage 4: phi^{n+1}
  R* __restrict__ v_out;       // stage 4: v^{n+1}
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

template <typename R>
__device__ __forceinline__ R ldcg(const R* p) {
  return __ldcg(p);
}

template <int TH, typename R, int STAGE>
__global__ void __launch_bounds__(NT) k_stage(StageArgs<R> a) {
  constexpr int C = NComp<TH>::C;
  __shared__ R sY[C][SY * SX];
  __shared__ double sred[(NT / 32) * 3];
  __shared__ int s_last;

  DevState* st = a.st;
  // Uniform over the grid (the record only changes between launches). Stage 1 runs
  // once per field; stages 2-4 stop at convergence, at a non-finite value and at
  // the step limit of the current call.
  if (st->converged | st->nonfinite) return;
  if (STAGE == 1 ? (st->head_step == st->steps) : (st->steps >= st->step_limit)) return;
  const int tid = threadIdx.y * BX + threadIdx.x;
  const bool arrest = (STAGE > 1) && (st->arrest != 0);
  const R cv = arrest ? R(0) : (STAGE == 4 ? a.dt : R(0.5) * a.dt);
  const R ck = STAGE == 3 ? R(0.25) * a.dt * a.dt : R(0.5) * a.dt * a.dt;
  const size_t P = a.plane;

  // Per-thread compensated pair in the working type; widened to FP64 once per
  // thread (the pair keeps the sum to O(n eps^2), so FP32 loses nothing material
  // over the few dozen sites a thread owns).
  R es = R(0), ec = R(0), gmr = R(0);

  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const int x0 = (t % a.ntx) * TX, y0 = (t / a.ntx) * TY;
    __syncthreads();  // the previous tile's shared reads are finished
    for (int idx = tid; idx < SX * SY; idx += NT) {
      const int lx = idx % SX, ly = idx / SX;
      const int gx = x0 + lx - HALO, gy = y0 + ly - HALO;
      R y[C];
      if (gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny) {
        const size_t s = (size_t)gy * a.nx + gx;
#pragma unroll
        for (int c = 0; c < C; ++c) y[c] = a.phi[c * P + s];
        // Halo sites have v = k_v = 0: their stage input is phi itself.
        if (STAGE > 1 && gx >= HALO && gx < a.nx - HALO && gy >= HALO && gy < a.ny - HALO) {
#pragma unroll
          for (int c = 0; c < C; ++c) {
            R u = y[c];
            if (!arrest) u += cv * a.v[c * P + s];
            if (STAGE > 2) u += ck * a.kvin[c * P + s];
            y[c] = u;
          }
          if (TH == TH_CM) {
            const R inv = rsqrt_t<R>(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
#pragma unroll
            for (int c = 0; c < C; ++c) y[c] *= inv;
          }
        }
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) y[c] = R(0);
      }
#pragma unroll
      for (int c = 0; c < C; ++c) sY[c][idx] = y[c];
    }
    __syncthreads();

#pragma unroll
    for (int r = 0; r < ROWS_PER_THREAD; ++r) {
      const int lx = threadIdx.x, ly = threadIdx.y + r * BY;
      const int gx = x0 + lx, gy = y0 + ly;
      if (gx < HALO || gx >= a.nx - HALO || gy < HALO || gy >= a.ny - HALO) continue;
      const int sx = lx + HALO, sy = ly + HALO;
      R v[C], fx[C], fy[C], fxx[C], fyy[C], fxy[C];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const Deriv<R> d = (TH == TH_AH && c >= 2) ? stencil<R, true, true>(sY[c], sx, sy, a.h)
                                                   : stencil<R, true, false>(sY[c], sx, sy, a.h);
        v[c] = d.v; fx[c] = d.fx; fy[c] = d.fy; fxx[c] = d.fxx; fyy[c] = d.fyy; fxy[c] = d.fxy;
      }
      R G[C];
      if (TH == TH_AH) force_ah<R>(a.k, v, fx, fy, fxx, fyy, fxy, G);
      else force_cm<R>(a.k, v, fx, fy, fxx, fyy, G);
      const size_t s = (size_t)gy * a.nx + gx;
      if (STAGE == 1) {
        const R e = (TH == TH_AH) ? density_ah<R>(a.k, v, fx, fy) : density_cm<R>(a.k, v, fx, fy);
        const R t = es + e;
        ec += (fabs(es) >= fabs(e)) ? (es - t) + e : (e - t) + es;
        es = t;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const R ag = fabs(G[c]);
          gmr = (ag > gmr || ag != ag) ? ag : gmr;
        }
      }
      if (STAGE < 4) {
#pragma unroll
        for (int c = 0; c < C; ++c) a.kv_out[c * P + s] = -G[c];
      } else {
        const R dt = a.dt, w = dt * dt / R(6), u = dt / R(6);
        R pn[C], vn[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const R p0 = a.phi[c * P + s];
          const R v0 = arrest ? R(0) : a.v[c * P + s];
          const R k1 = a.kv1[c * P + s], k2 = a.kv2[c * P + s], k3 = a.kv3[c * P + s], k4 = -G[c];
          pn[c] = p0 + dt * v0 + w * (k1 + k2 + k3);
          vn[c] = v0 + u * (k1 + R(2) * (k2 + k3) + k4);
        }
        if (TH == TH_CM) {
          const R inv = rsqrt_t<R>(pn[0] * pn[0] + pn[1] * pn[1] + pn[2] * pn[2]);
#pragma unroll
          for (int c = 0; c < C; ++c) pn[c] *= inv;
          const R vp = vn[0] * pn[0] + vn[1] * pn[1] + vn[2] * pn[2];
#pragma unroll
          for (int c = 0; c < C; ++c) vn[c] -= vp * pn[c];
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
          a.phi_out[c * P + s] = pn[c];
          a.v_out[c * P + s] = vn[c];
        }
      }
    }
  }

  if (STAGE == 4) {
    if (blockIdx.x == 0 && tid == 0) st->steps += 1;  // single writer; read after this launch
    return;
  }
  if (STAGE != 1) return;

  // ---- energy / residual reduction and the on-device arrest + convergence decision
  DD sv[1] = {DD{(double)es, (double)ec}};
  double mv[1] = {(double)gmr};
  block_reduce<1, 1>(sv, mv, sred);
  if (tid == 0) {
    a.part[blockIdx.x] = FlowPartial{sv[0].s, sv[0].c, mv[0], 0.0};
    __threadfence();
    const unsigned prev = atomicAdd(&st->ticket, 1u);
    s_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  DD acc{0.0, 0.0};
  double mm = 0.0;
  for (int i = tid; i < (int)gridDim.x; i += NT) {
    const double ps = ldcg(&a.part[i].s), pc = ldcg(&a.part[i].c), pm = ldcg(&a.part[i].m);
    acc = dd_add(acc, DD{ps, pc});
    mm = nanmax(mm, pm);
  }
  DD sv2[1] = {acc};
  double mv2[1] = {mm};
  block_reduce<1, 1>(sv2, mv2, sred);
  if (tid == 0) {
    const double E = a.area * (sv2[0].s + sv2[0].c);
    const double g = a.area * mv2[0];
    const int arr = (E > st->E_last) ? 1 : 0;  // Eq. 4, strict
    st->E_cur = E;
    st->gmax = g;
    st->arrest = arr;
    st->arrests += arr;
    st->E_last = E;
    st->converged = (g < st->tol) ? 1 : 0;
    st->nonfinite = (isfinite(E) && isfinite(g)) ? 0 : 1;
    st->head_step = st->steps;
    st->ticket = 0;
  }
}

// ------------------------------------------------------------------ control kernels
__global__ void k_reset_state(DevState* st) {
  st->E_last = __longlong_as_double(0x7ff0000000000000LL);  // +inf: no arrest on the first step
  st->E_cur = 0.0;
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
template <typename R>
static StageArgs<R> make_args(const LaunchCtx& c, int stage, int cur) {
  StageArgs<R> a{};
  const int nxt = cur ^ 1;
  a.phi = static_cast<const R*>(c.phi[cur]);
  a.v = static_cast<const R*>(c.v[cur]);
  a.kvin = stage == 3 ? static_cast<const R*>(c.kv[0]) : static_cast<const R*>(c.kv[1]);
  a.kv1 = static_cast<const R*>(c.kv[0]);
  a.kv2 = static_cast<const R*>(c.kv[1]);
  a.kv3 = static_cast<const R*>(c.kv[2]);
  a.kv_out = stage <= 3 ? static_cast<R*>(c.kv[stage - 1]) : nullptr;
  a.phi_out = static_cast<R*>(c.phi[nxt]);
  a.v_out = static_cast<R*>(c.v[nxt]);
  a.nx = c.nx;
  a.ny = c.ny;
  a.plane = c.plane;
  a.ntx = c.ntiles_x;
  a.ntiles = c.ntiles_x * c.ntiles_y;
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

template <int TH, typename R>
static cudaError_t stage_t(const LaunchCtx& c, int stage, int cur, cudaStream_t s) {
  const StageArgs<R> a = make_args<R>(c, stage, cur);
  const dim3 blk(BX, BY);
  switch (stage) {
    case 1: k_stage<TH, R, 1><<<c.flow_blocks, blk, 0, s>>>(a); break;
    case 2: k_stage<TH, R, 2><<<c.flow_blocks, blk, 0, s>>>(a); break;
    case 3: k_stage<TH, R, 3><<<c.flow_blocks, blk, 0, s>>>(a); break;
    case 4: k_stage<TH, R, 4><<<c.flow_blocks, blk, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_stage(const LaunchCtx& c, int stage, int cur, cudaStream_t s) {
  if (c.theory == TH_AH) return c.prec == 1 ? stage_t<TH_AH, float>(c, stage, cur, s) : stage_t<TH_AH, double>(c, stage, cur, s);
  return c.prec == 1 ? stage_t<TH_CM, float>(c, stage, cur, s) : stage_t<TH_CM, double>(c, stage, cur, s);
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
  if (c.prec == 1) k_scaled_copy<float><<<blocks, 256, 0, s>>>((float*)out, (const float*)in, n, (float)scale);
  else k_scaled_copy<double><<<blocks, 256, 0, s>>>((double*)out, (const double*)in, n, scale);
  return cudaGetLastError();
}

template <int TH, typename R>
static int occupancy_min() {
  int b1 = 0, b2 = 0, b3 = 0, b4 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_stage<TH, R, 1>, NT, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_stage<TH, R, 2>, NT, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b3, k_stage<TH, R, 3>, NT, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b4, k_stage<TH, R, 4>, NT, 0);
  int m = b1;
  if (b2 < m) m = b2;
  if (b3 < m) m = b3;
  if (b4 < m) m = b4;
  return m < 1 ? 1 : m;
}

int flow_grid(int theory, int prec, int ntiles) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int occ;
  if (theory == TH_AH) occ = prec == 1 ? occupancy_min<TH_AH, float>() : occupancy_min<TH_AH, double>();
  else occ = prec == 1 ? occupancy_min<TH_CM, float>() : occupancy_min<TH_CM, double>();
  const int g = nsm * occ;
  return ntiles < g ? ntiles : g;
}

}  // namespace ss
