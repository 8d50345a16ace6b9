// ss_observe.cu -- GPU-resident observables and initial data (arxiv 2603.24370,
// Sec. 2 "GPU-resident evaluation of observables", Sec. 3.3 reductions, Sec. 3.4
// initialisation).
//
// Observables are evaluated in FP64 arithmetic from the stored field (FP32 or
// FP64), with compensated sums and a fixed reduction order:
//   E_h  = dx dy sum_I e                              (Table 1 / Eq. 5 densities)
//   flux = dx dy sum_I (d_1 A_2 - d_2 A_1)            (Abelian Higgs, s+id)
//   Q    = (1/4pi) sum over plaquettes of the Berg-Luescher solid angles of the
//          two triangles (n00, n10, n11), (n00, n11, n01)   (chiral magnet, Baby Skyrme)
//   Q    = (1/2pi) sum of wrapped arg-psi steps around the boundary of I (Abelian Higgs;
//          s+id: arg Delta_s)
//   max_I |G|, max ||n| - 1|
//   N    = dx dy sum_I |psi|^2, L = dx dy sum_I Re(psi* L_z psi)   (BEC)
// A compensated FP32 field is read as value + remainder, exactly, in FP64.
#include <cmath>

#include "ss_internal.h"

namespace ss {

template <typename R>
struct ObsArgs {
  const R* __restrict__ phi;
  const R* __restrict__ lo;  // compensated FP32: remainder plane added in FP64 (else null)
  const R* __restrict__ psi; // chiral magnet with demagnetisation: magnetostatic potential (else null)
  int nx, ny;
  size_t plane;
  int ntx, ntiles;
  Spacing<double> h;
  double hx, hy;  // dx, dy
  Couplings<double> k;
  double area;
  DevState* st;
  ObsPartial* part;
};

__device__ __forceinline__ double dot3d(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Signed solid angle of the spherical triangle (a, b, c):
// tan(Omega / 2) = a.(b x c) / (1 + a.b + b.c + c.a)   (Berg and Luescher 1981).
__device__ __forceinline__ double solid_angle(const double* a, const double* b, const double* c) {
  double bc[3];
  cross3<double>(b, c, bc);
  return 2.0 * atan2(dot3d(a, bc), 1.0 + dot3d(a, b) + dot3d(b, c) + dot3d(c, a));
}

template <int TH, typename R>
__global__ void __launch_bounds__(NT) k_observables(ObsArgs<R> a) {
  constexpr int C = NComp<TH>::C;
  constexpr int CP = C + (TH == TH_CMD ? 1 : 0);  // + the potential plane
  __shared__ double sY[CP][SY * SX];
  __shared__ double sred[RedSmem<3, 2>::n];
  __shared__ int s_last;
  const int tid = threadIdx.y * BX + threadIdx.x;
  const size_t P = a.plane;
  DD se{0.0, 0.0}, sf{0.0, 0.0}, sq{0.0, 0.0};
  double gm = 0.0, nd = 0.0;

  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const int x0 = (t % a.ntx) * TX, y0 = (t / a.ntx) * TY;
    __syncthreads();
    for (int idx = tid; idx < SX * SY; idx += NT) {
      const int lx = idx % SX, ly = idx / SX;
      const int gx = x0 + lx - HALO, gy = y0 + ly - HALO;
      const bool in = gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny;
      const size_t s = (size_t)gy * a.nx + gx;
#pragma unroll
      for (int c = 0; c < C; ++c)
        sY[c][idx] = in ? (double)a.phi[c * P + s] + (a.lo ? (double)a.lo[c * P + s] : 0.0) : 0.0;
      if (TH == TH_CMD) sY[CP - 1][idx] = in ? (double)a.psi[s] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < ROWS_PER_THREAD; ++r) {
      const int lx = threadIdx.x, ly = threadIdx.y + r * BY;
      const int gx = x0 + lx, gy = y0 + ly;
      if (gx >= a.nx || gy >= a.ny) continue;
      const int sx = lx + HALO, sy = ly + HALO;
      if (UnitVector<TH>::value) {
        const int o = sy * SX + sx;
        const double n00[3] = {sY[0][o], sY[1][o], sY[2][o]};
        nd = nanmax(nd, fabs(sqrt(dot3d(n00, n00)) - 1.0));
        if (gx + 1 < a.nx && gy + 1 < a.ny) {
          double q[4][3];
          const int off[4] = {o, o + 1, o + 1 + SX, o + SX};  // (i,j) (i+1,j) (i+1,j+1) (i,j+1)
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const double x = sY[0][off[m]], y = sY[1][off[m]], z = sY[2][off[m]];
            const double inv = 1.0 / sqrt(x * x + y * y + z * z);
            q[m][0] = x * inv; q[m][1] = y * inv; q[m][2] = z * inv;
          }
          neumaier(sq, solid_angle(q[0], q[1], q[2]));
          neumaier(sq, solid_angle(q[0], q[2], q[3]));
        }
      }
      if (gx < HALO || gx >= a.nx - HALO || gy < HALO || gy >= a.ny - HALO) continue;
      double v[C], fx[C], fy[C], fxx[C], fyy[C], fxy[C];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const Deriv<double> d = ((TH == TH_AH && c >= 2) || TH == TH_BS || (TH == TH_SID && c >= 4))
                                    ? stencil<double, true, true>(sY[c], sx, sy, a.h)
                                    : stencil<double, true, false>(sY[c], sx, sy, a.h);
        v[c] = d.v; fx[c] = d.fx; fy[c] = d.fy; fxx[c] = d.fxx; fyy[c] = d.fyy; fxy[c] = d.fxy;
      }
      double G[C];
      if (TH == TH_AH) {
        force_ah<double>(a.k, v, fx, fy, fxx, fyy, fxy, G);
        neumaier(se, density_ah<double>(a.k, v, fx, fy));
        neumaier(sf, fx[3] - fy[2]);
      } else if (TH == TH_CMD) {  // E_ms density -mu_d/2 psi rho, force with mu_d grad psi
        const Deriv<double> pd = stencil<double, false, false>(sY[CP - 1], sx, sy, a.h);
        force_of<TH, double>(a.k, v, fx, fy, fxx, fyy, fxy, G, pd.fx, pd.fy);
        neumaier(se, density_at<TH, double>(a.k, v, fx, fy, pd.v, 0.0));
      } else if (TH == TH_SID) {
        force_of<TH, double>(a.k, v, fx, fy, fxx, fyy, fxy, G);
        neumaier(se, density_at<TH, double>(a.k, v, fx, fy));
        neumaier(sf, fx[5] - fy[4]);
      } else if (TH == TH_BEC) {
        const double x = (gx - 0.5 * (a.nx - 1)) * a.hx, y = (gy - 0.5 * (a.ny - 1)) * a.hy;
        force_of<TH, double>(a.k, v, fx, fy, fxx, fyy, fxy, G, x, y);
        neumaier(se, density_at<TH, double>(a.k, v, fx, fy, x, y));
        neumaier(sf, v[0] * v[0] + v[1] * v[1]);  // atoms
        neumaier(sq, v[0] * (x * fy[1] - y * fx[1]) - v[1] * (x * fy[0] - y * fx[0]));  // Re(psi* L_z psi)
      } else {
        force_of<TH, double>(a.k, v, fx, fy, fxx, fyy, fxy, G);
        neumaier(se, density_at<TH, double>(a.k, v, fx, fy));
      }
#pragma unroll
      for (int c = 0; c < C; ++c) gm = nanmax(gm, fabs(G[c]));
    }
  }

  DD sv[3] = {se, sf, sq};
  double mv[2] = {gm, nd};
  block_reduce<3, 2>(sv, mv, sred);
  if (tid == 0) {
    a.part[blockIdx.x] = ObsPartial{sv[0].s, sv[0].c, sv[1].s, sv[1].c, sv[2].s, sv[2].c, mv[0], mv[1]};
    __threadfence();
    const unsigned prev = atomicAdd(&a.st->obs_ticket, 1u);
    s_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  DD ae{0.0, 0.0}, af{0.0, 0.0}, aq{0.0, 0.0};
  double am = 0.0, an = 0.0;
  for (int i = tid; i < (int)gridDim.x; i += NT) {
    const ObsPartial* p = a.part + i;
    ae = dd_add(ae, DD{__ldcg(&p->es), __ldcg(&p->ec)});
    af = dd_add(af, DD{__ldcg(&p->fs), __ldcg(&p->fc)});
    aq = dd_add(aq, DD{__ldcg(&p->qs), __ldcg(&p->qc)});
    am = nanmax(am, __ldcg(&p->gm));
    an = nanmax(an, __ldcg(&p->nd));
  }
  DD sv2[3] = {ae, af, aq};
  double mv2[2] = {am, an};
  block_reduce<3, 2>(sv2, mv2, sred);
  if (tid == 0) {
    DevState* st = a.st;
    st->obs_energy = a.area * (sv2[0].s + sv2[0].c);
    st->obs_flux = (TH == TH_AH || TH == TH_SID) ? a.area * (sv2[1].s + sv2[1].c) : 0.0;
    st->obs_atoms = TH == TH_BEC ? a.area * (sv2[1].s + sv2[1].c) : 0.0;
    st->obs_lz = TH == TH_BEC ? a.area * (sv2[2].s + sv2[2].c) : 0.0;
    if (UnitVector<TH>::value) st->obs_charge = (sv2[2].s + sv2[2].c) / (4.0 * 3.14159265358979323846);
    if (TH == TH_BEC) st->obs_charge = 0.0;
    st->obs_gmax_raw = mv2[0];
    st->obs_normdev = mv2[1];
    st->obs_ticket = 0;
  }
}

// Winding of arg psi around the boundary loop of I, counter-clockwise, one block.
template <typename R>
__global__ void __launch_bounds__(NT) k_winding(const R* __restrict__ phi, int nx, int ny, size_t plane,
                                                DevState* st) {
  __shared__ double sred[RedSmem<1, 1>::n];
  const int tid = threadIdx.y * BX + threadIdx.x;
  const int a = nx - 5, b = ny - 5, L = 2 * a + 2 * b;
  auto site = [&](int k, int& i, int& j) {
    if (k < a) { i = 2 + k; j = 2; }
    else if (k < a + b) { i = nx - 3; j = 2 + (k - a); }
    else if (k < 2 * a + b) { i = nx - 3 - (k - a - b); j = ny - 3; }
    else { i = 2; j = ny - 3 - (k - 2 * a - b); }
  };
  const double PI = 3.14159265358979323846;
  DD acc{0.0, 0.0};
  for (int k = tid; k < L; k += NT) {
    int i0, j0, i1, j1;
    site(k, i0, j0);
    site((k + 1) % L, i1, j1);
    const size_t s0 = (size_t)j0 * nx + i0, s1 = (size_t)j1 * nx + i1;
    double d = atan2((double)phi[plane + s1], (double)phi[s1]) - atan2((double)phi[plane + s0], (double)phi[s0]);
    if (d > PI) d -= 2.0 * PI;
    if (d <= -PI) d += 2.0 * PI;
    neumaier(acc, d);
  }
  DD sv[1] = {acc};
  double mv[1] = {0.0};
  block_reduce<1, 1>(sv, mv, sred);
  if (tid == 0) st->obs_charge = (sv[0].s + sv[0].c) / (2.0 * PI);
}

// Initial data (Sec. 3.4 "model-specific ansatz"; standard forms, see soliton.h),
// evaluated in FP64 and rounded once to the storage type, into both field buffers.
// BEC: psi = sqrt(max(0, mu - r^2/2) / g) prod_k tanh(r_k/s_k)^{|n_k|} exp(i (n_k theta_k + chi_k))
// (Thomas-Fermi amplitude times vortex factors); q0 = g, q1 = mu.
// s+id: the Abelian Higgs vortex product scaled by the uniform minimum, Delta_s = q0 x it,
// Delta_d = q1 e^{i q2} x it (q2 the relative phase), A as for the Abelian Higgs model.
template <int TH, typename R>
__global__ void k_ansatz(R* __restrict__ f0, R* __restrict__ f1, int nx, int ny, size_t plane, double dx, double dy,
                         const double* __restrict__ sol, int ns, double q0, double q1, double q2) {
  const double PI = 3.14159265358979323846;
  for (size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x; s < plane; s += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(s % nx), j = (int)(s / nx);
    const double x = (i - 0.5 * (nx - 1)) * dx, y = (j - 0.5 * (ny - 1)) * dy;
    if (TH == TH_BEC) {
      double mod = sqrt(fmax(0.0, q1 - 0.5 * (x * x + y * y)) / q0), ph = 0.0;
      for (int k = 0; k < ns; ++k) {
        const double X = x - sol[5 * k], Y = y - sol[5 * k + 1];
        const double n = sol[5 * k + 2], sz = sol[5 * k + 3], chi = sol[5 * k + 4];
        mod *= pow(tanh(sqrt(X * X + Y * Y) / sz), fabs(n));
        ph += n * atan2(Y, X) + chi;
      }
      double sn, cs;
      sincos(ph, &sn, &cs);
      const R v[2] = {(R)(mod * cs), (R)(mod * sn)};
#pragma unroll
      for (int c = 0; c < 2; ++c) { f0[c * plane + s] = v[c]; f1[c * plane + s] = v[c]; }
    } else if (TH == TH_AH || TH == TH_SID) {
      double mod = 1.0, ph = 0.0, A1 = 0.0, A2 = 0.0;
      for (int k = 0; k < ns; ++k) {
        const double X = x - sol[5 * k], Y = y - sol[5 * k + 1];
        const double n = sol[5 * k + 2], sz = sol[5 * k + 3], chi = sol[5 * k + 4];
        const double r2 = X * X + Y * Y;
        const double t = tanh(sqrt(r2) / sz);
        mod *= pow(t, fabs(n));
        ph += n * atan2(Y, X) + chi;
        if (r2 > 0.0) {
          A1 += n * t * t * (-Y) / r2;
          A2 += n * t * t * X / r2;
        }
      }
      double sn, cs;
      sincos(ph, &sn, &cs);
      if (TH == TH_AH) {
        const R v[4] = {(R)(mod * cs), (R)(mod * sn), (R)A1, (R)A2};
#pragma unroll
        for (int c = 0; c < 4; ++c) { f0[c * plane + s] = v[c]; f1[c * plane + s] = v[c]; }
      } else {
        double sd, cd;
        sincos(ph + q2, &sd, &cd);
        const R v[6] = {(R)(q0 * mod * cs), (R)(q0 * mod * sn), (R)(q1 * mod * cd), (R)(q1 * mod * sd), (R)A1, (R)A2};
#pragma unroll
        for (int c = 0; c < 6; ++c) { f0[c * plane + s] = v[c]; f1[c * plane + s] = v[c]; }
      }
    } else {
      double n1 = 0.0, n2 = 0.0, n3 = 1.0;
      for (int k = 0; k < ns; ++k) {
        const double X = x - sol[5 * k], Y = y - sol[5 * k + 1];
        const double R0 = sol[5 * k + 3];
        const double r2 = X * X + Y * Y;
        if (r2 < R0 * R0) {
          const double r = sqrt(r2);
          const double fr = PI * (1.0 - r / R0), th = sol[5 * k + 2] * atan2(Y, X) + sol[5 * k + 4];
          n1 = sin(fr) * cos(th);
          n2 = sin(fr) * sin(th);
          n3 = cos(fr);
          break;
        }
      }
      const R v[3] = {(R)n1, (R)n2, (R)n3};
#pragma unroll
      for (int c = 0; c < 3; ++c) { f0[c * plane + s] = v[c]; f1[c * plane + s] = v[c]; }
    }
  }
}

// The compact skyrmions of the unit-vector theories (the last branch of k_ansatz) with
// the work proportional to the sites each soliton covers: a block takes a tile of
// 32 x 8 sites, first lists, in ascending order, the solitons whose disc reaches the
// tile's bounding box (widened by 1e-9 of the spacing), then each site scans only
// that list, with the same FP64 arithmetic and first-match rule as k_ansatz. A tile
// reached by more than ANS_CAP discs scans them all.
constexpr int ANS_CAP = 512;
template <typename R>
__global__ void __launch_bounds__(256) k_ansatz_compact(R* __restrict__ f0, R* __restrict__ f1, int nx, int ny,
                                                        size_t plane, double dx, double dy,
                                                        const double* __restrict__ sol, int ns) {
  const double PI = 3.14159265358979323846;
  __shared__ int list[ANS_CAP];
  __shared__ int wcnt[8];
  __shared__ int cnt;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int ntx = (nx + 31) / 32, nty = (ny + 7) / 8;
  for (int t = blockIdx.x; t < ntx * nty; t += gridDim.x) {
    const int i0 = (t % ntx) * 32, j0 = (t / ntx) * 8;
    const double ex = 1e-9 * dx, ey = 1e-9 * dy;
    const double xlo = (i0 - 0.5 * (nx - 1)) * dx - ex, xhi = (min(i0 + 31, nx - 1) - 0.5 * (nx - 1)) * dx + ex;
    const double ylo = (j0 - 0.5 * (ny - 1)) * dy - ey, yhi = (min(j0 + 7, ny - 1) - 0.5 * (ny - 1)) * dy + ey;
    if (tid == 0) cnt = 0;
    __syncthreads();
    for (int base = 0; base < ns; base += 256) {
      const int k = base + tid;
      bool hit = false;
      if (k < ns) {
        const double cx = sol[5 * k], cy = sol[5 * k + 1], R0 = sol[5 * k + 3];
        const double ddx = fmax(fmax(xlo - cx, cx - xhi), 0.0), ddy = fmax(fmax(ylo - cy, cy - yhi), 0.0);
        hit = ddx * ddx + ddy * ddy < R0 * R0;
      }
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (lane == 0) wcnt[w] = __popc(m);
      __syncthreads();
      int before = cnt;
      for (int q = 0; q < w; ++q) before += wcnt[q];
      const int pos = before + __popc(m & ((1u << lane) - 1u));
      if (hit && pos < ANS_CAP) list[pos] = k;
      __syncthreads();
      if (tid == 0) {
        int tot = 0;
        for (int q = 0; q < 8; ++q) tot += wcnt[q];
        cnt += tot;
      }
      __syncthreads();
    }
    const int nl = cnt;
    const int i = i0 + lane, j = j0 + w;
    if (i < nx && j < ny) {
      const size_t s = (size_t)j * nx + i;
      const double x = (i - 0.5 * (nx - 1)) * dx, y = (j - 0.5 * (ny - 1)) * dy;
      double n1 = 0.0, n2 = 0.0, n3 = 1.0;
      const bool all = nl > ANS_CAP;
      const int nk = all ? ns : nl;
      for (int q = 0; q < nk; ++q) {
        const int k = all ? q : list[q];
        const double X = x - sol[5 * k], Y = y - sol[5 * k + 1];
        const double R0 = sol[5 * k + 3];
        const double r2 = X * X + Y * Y;
        if (r2 < R0 * R0) {
          const double r = sqrt(r2);
          const double fr = PI * (1.0 - r / R0), th = sol[5 * k + 2] * atan2(Y, X) + sol[5 * k + 4];
          n1 = sin(fr) * cos(th);
          n2 = sin(fr) * sin(th);
          n3 = cos(fr);
          break;
        }
      }
      const R v[3] = {(R)n1, (R)n2, (R)n3};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        f0[c * plane + s] = v[c];
        f1[c * plane + s] = v[c];
      }
    }
    __syncthreads();  // the list is rebuilt for the next tile
  }
}

// ------------------------------------------------------------------ launchers
template <int TH, typename R>
static cudaError_t obs_t(const LaunchCtx& c, int cur, cudaStream_t s) {
  ObsArgs<R> a{};
  a.phi = static_cast<const R*>(c.phi[cur]);
  a.lo = static_cast<const R*>(c.lo[cur]);
  a.psi = static_cast<const R*>(c.psi[cur]);
  a.nx = c.nx;
  a.ny = c.ny;
  a.plane = c.plane;
  a.ntx = c.ntiles_x;
  a.ntiles = c.ntiles_x * c.ntiles_y;
  a.h.i12dx = 1.0 / (12.0 * c.dx);
  a.h.i12dy = 1.0 / (12.0 * c.dy);
  a.h.i12dx2 = 1.0 / (12.0 * c.dx * c.dx);
  a.h.i12dy2 = 1.0 / (12.0 * c.dy * c.dy);
  a.h.i144dxdy = 1.0 / (144.0 * c.dx * c.dy);
  a.hx = c.dx;
  a.hy = c.dy;
  for (int i = 0; i < NCOUP; ++i) a.k.c[i] = c.coup[i];
  a.area = c.dx * c.dy;
  a.st = c.st;
  a.part = c.opart;
  k_observables<TH, R><<<c.obs_blocks, dim3(BX, BY), 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (TH == TH_AH || TH == TH_SID) {  // winding of the first complex field
    k_winding<R><<<1, dim3(BX, BY), 0, s>>>(a.phi, c.nx, c.ny, c.plane, c.st);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_observables(const LaunchCtx& c, int cur, cudaStream_t s) {
  const bool f = c.prec != PREC_F64;  // every FP32 mode stores its (hi) field in float
  if (c.theory == TH_AH) return f ? obs_t<TH_AH, float>(c, cur, s) : obs_t<TH_AH, double>(c, cur, s);
  if (c.theory == TH_CM) return f ? obs_t<TH_CM, float>(c, cur, s) : obs_t<TH_CM, double>(c, cur, s);
  if (c.theory == TH_BS) return f ? obs_t<TH_BS, float>(c, cur, s) : obs_t<TH_BS, double>(c, cur, s);
  if (c.theory == TH_SID) return f ? obs_t<TH_SID, float>(c, cur, s) : obs_t<TH_SID, double>(c, cur, s);
  if (c.theory == TH_CMD) return f ? obs_t<TH_CMD, float>(c, cur, s) : obs_t<TH_CMD, double>(c, cur, s);
  return f ? obs_t<TH_BEC, float>(c, cur, s) : obs_t<TH_BEC, double>(c, cur, s);
}

// Uniform minimum of the s+id potential: the relative phase is pi/2 for b4 > 0 (else 0),
// which turns b3 into b3 - 2 |b4|; the two-band stationary point if both densities are
// positive, else the better one-band minimum (or the normal state). Returns sqrt(S),
// sqrt(D) and the phase.
static void sid_uniform_minimum(const double* k, double* rs, double* rd, double* phase) {
  const double a1 = k[0], a2 = k[1], b1 = k[2], b2 = k[3], b3 = k[4] - 2.0 * std::fabs(k[5]);
  *phase = k[5] > 0.0 ? 1.57079632679489661923 : 0.0;
  auto V = [&](double S, double D) { return a1 * S + a2 * D + b1 * S * S + b2 * D * D + b3 * S * D; };
  double bs = 0.0, bd = 0.0, bv = 0.0;
  auto take = [&](double S, double D) {
    if (S >= 0.0 && D >= 0.0 && V(S, D) < bv) { bs = S; bd = D; bv = V(S, D); }
  };
  const double det = 4.0 * b1 * b2 - b3 * b3;
  if (det != 0.0) take((-2.0 * b2 * a1 + b3 * a2) / det, (-2.0 * b1 * a2 + b3 * a1) / det);
  if (b1 > 0.0) take(-a1 / (2.0 * b1), 0.0);
  if (b2 > 0.0) take(0.0, -a2 / (2.0 * b2));
  *rs = std::sqrt(bs);
  *rd = std::sqrt(bd);
}

template <int TH, typename R>
static cudaError_t ansatz_t(const LaunchCtx& c, const double* sol, int n, cudaStream_t s) {
  const int blocks = (int)((c.plane + 255) / 256 < 4096 ? (c.plane + 255) / 256 : 4096);
  // BEC: g and mu; at a fixed atom number N the Thomas-Fermi mu of N atoms, sqrt(g N / pi)
  double q[3] = {c.coup[0], c.coup[4] > 0.0 ? std::sqrt(c.coup[0] * c.coup[4] / 3.14159265358979323846) : c.coup[2], 0.0};
  if (TH == TH_SID) sid_uniform_minimum(c.coup, &q[0], &q[1], &q[2]);
  if (TH == TH_CM) {  // compact skyrmions: each site scans only the discs near its tile
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long tiles = (long long)((c.nx + 31) / 32) * ((c.ny + 7) / 8);
    const int g = (int)(tiles < 8LL * nsm ? tiles : 8LL * nsm);
    k_ansatz_compact<R><<<g, 256, 0, s>>>(static_cast<R*>(c.phi[0]), static_cast<R*>(c.phi[1]), c.nx, c.ny, c.plane,
                                          c.dx, c.dy, sol, n);
    return cudaGetLastError();
  }
  k_ansatz<TH, R><<<blocks, 256, 0, s>>>(static_cast<R*>(c.phi[0]), static_cast<R*>(c.phi[1]), c.nx, c.ny, c.plane,
                                         c.dx, c.dy, sol, n, q[0], q[1], q[2]);
  return cudaGetLastError();
}

cudaError_t launch_ansatz(const LaunchCtx& c, const double* d_sol, int n, cudaStream_t s) {
  const bool f = c.prec != PREC_F64;
  if (c.theory == TH_AH) return f ? ansatz_t<TH_AH, float>(c, d_sol, n, s) : ansatz_t<TH_AH, double>(c, d_sol, n, s);
  if (c.theory == TH_BEC)
    return f ? ansatz_t<TH_BEC, float>(c, d_sol, n, s) : ansatz_t<TH_BEC, double>(c, d_sol, n, s);
  if (c.theory == TH_SID)
    return f ? ansatz_t<TH_SID, float>(c, d_sol, n, s) : ansatz_t<TH_SID, double>(c, d_sol, n, s);
  // both unit-vector theories take the compact skyrmion
  return f ? ansatz_t<TH_CM, float>(c, d_sol, n, s) : ansatz_t<TH_CM, double>(c, d_sol, n, s);
}

template <int TH, typename R>
static int obs_occ() {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_observables<TH, R>, NT, 0);
  return b < 1 ? 1 : b;
}

int obs_grid(int theory, int prec, int ntiles) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int occ;
  const bool f = prec != PREC_F64;
  if (theory == TH_AH) occ = f ? obs_occ<TH_AH, float>() : obs_occ<TH_AH, double>();
  else if (theory == TH_CM) occ = f ? obs_occ<TH_CM, float>() : obs_occ<TH_CM, double>();
  else if (theory == TH_BS) occ = f ? obs_occ<TH_BS, float>() : obs_occ<TH_BS, double>();
  else if (theory == TH_SID) occ = f ? obs_occ<TH_SID, float>() : obs_occ<TH_SID, double>();
  else if (theory == TH_CMD) occ = f ? obs_occ<TH_CMD, float>() : obs_occ<TH_CMD, double>();
  else occ = f ? obs_occ<TH_BEC, float>() : obs_occ<TH_BEC, double>();
  const int g = nsm * occ;
  return ntiles < g ? ntiles : g;
}

}  // namespace ss
