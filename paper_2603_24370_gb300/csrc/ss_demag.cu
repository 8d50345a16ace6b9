// ss_demag.cu -- magnetostatic potential of the chiral magnet (arxiv 2603.24370, Eq. 6).
//
// With psi = phi / (mu_0 M_s) the Poisson equation of Eq. 6 reads lap psi = div n (the
// in-plane components). On the lattice: L psi = rho on a Dirichlet box B containing the
// interior I, rho the Eq. 1 divergence of (n_1, n_2) on I and zero on the rest of B, L
// the 5-point Laplacian with psi = 0 on the nodes just outside B (standing in for the
// far field). Along each axis B has the first size N' >= N with N' + 1 free of prime
// factors above 7, floor((N' - N) / 2) sites below I and the rest above; only psi on I
// is kept (the plane's halo stays zero), and the flow's force, the Eq. 1 gradient of
// that plane, is the exact gradient of the energy for any such box. L is diagonalised
// by the 2D sine transform (DST-I) over B's Nx x Ny sites: mode (k, l) has the eigenvalue
//   lambda_kl = -(2 - 2 cos(pi k / (Nx + 1))) / dx^2 - (2 - 2 cos(pi l / (Ny + 1))) / dy^2,
// and DST-I is its own inverse up to 2 / (N + 1) per direction.
//
// A DST-I of length N is the imaginary part of a real FFT of the odd extension
// (0, s_1 .. s_N, 0, -s_N .. -s_1) of length M = 2 (N + 1): X_k = -2 i DST_k. The solve
// is four batched real FFTs (cuFFT, a plain library transform): along x for every row,
// along y for every column (after a tiled transpose), the division by lambda, and the
// same two transforms back. The kernels around them build the extensions, take the
// imaginary parts, transpose in 32 x 32 shared-memory tiles and scatter psi into the
// field-sized plane of the current ping-pong parity (read on the device from the flow
// record, so the solve can sit inside a captured step graph).
#include <cufft.h>

#include <cmath>
#include <new>
#include <vector>

#include "ss_internal.h"

namespace ss {

template <typename R>
struct FftOf;
template <>
struct FftOf<float> {
  using C = cufftComplex;
  static constexpr cufftType type = CUFFT_R2C;
  static cufftResult exec(cufftHandle p, float* in, C* out) { return cufftExecR2C(p, in, out); }
};
template <>
struct FftOf<double> {
  using C = cufftDoubleComplex;
  static constexpr cufftType type = CUFFT_D2Z;
  static cufftResult exec(cufftHandle p, double* in, C* out) { return cufftExecD2Z(p, in, out); }
};

struct DemagSolver {
  int nx = 0, ny = 0;
  int Nx = 0, Ny = 0;  // Dirichlet box sites per axis (>= the interior's nx - 4, ny - 4)
  int bx = 0, by = 0;  // box sites below I along x, y
  int Mx = 0, My = 0, Hx = 0, Hy = 0;
  int prec = 0;  // PREC_*: FP64 transforms for FP64 fields, FP32 otherwise
  double dx = 0, dy = 0;
  cufftHandle px = 0, py = 0;
  bool have_px = false, have_py = false;
  void* ext_x = nullptr;  // R [Ny][Mx] (box rows)
  void* cx = nullptr;     // complex [Ny][Hx]
  void* ext_y = nullptr;  // R [Nx][My]
  void* cy = nullptr;     // complex [Nx][Hy]
  void* lam = nullptr;    // R [Nx + Ny]: the x and y parts of lambda
};

// ---- kernels (R the transform type; F the field storage type, equal except that
// compensated FP32 adds the remainder plane)
// rho into the x-extension rows of the box (zero on the box's padding), with the two
// zero points of every row.
template <typename R>
__global__ void k_rho_ext(const R* __restrict__ phi0, const R* __restrict__ phi1, const R* __restrict__ lo0,
                          const R* __restrict__ lo1, const DevState* st, int nx, int ny, size_t plane, int Nx, int Ny,
                          int bx, int by, int Mx, R i12dx, R i12dy, R* __restrict__ ext) {
  const int cur = (int)(st->steps & 1);
  const R* __restrict__ f = cur ? phi1 : phi0;
  const R* __restrict__ lo = cur ? lo1 : lo0;
  // rows over blocks, the row's points over threads (no index division)
  for (int jp = blockIdx.x; jp < Ny; jp += gridDim.x)  // row 0 .. Ny-1  (j' - 1)
    for (int ip = threadIdx.x; ip < Nx + 2; ip += blockDim.x) {  // 0 .. Nx+1  (i')
      R* row = ext + (size_t)jp * Mx;
      const int i = ip + 1 - bx, j = jp + 2 - by;  // full-array site of box node (ip, jp + 1)
      if (ip == 0 || ip == Nx + 1 || i < 2 || i > nx - 3 || j < 2 || j > ny - 3) {  // zero node, padding
        row[ip] = R(0);
        if (ip != 0) row[Mx - ip] = R(0);
        continue;
      }
      const size_t s = (size_t)j * nx + i;
      auto d1 = [&](const R* p, size_t c, ptrdiff_t st1, R sc) {
        const R* q = p + c * plane + s;
        return (R(8) * (q[st1] - q[-st1]) - (q[2 * st1] - q[-2 * st1])) * sc;
      };
      R rho = d1(f, 0, 1, i12dx) + d1(f, 1, (ptrdiff_t)nx, i12dy);
      if (lo) rho += d1(lo, 0, 1, i12dx) + d1(lo, 1, (ptrdiff_t)nx, i12dy);
      row[ip] = rho;
      row[Mx - ip] = -rho;
    }
}

// -Im/2 of a row transform, written transposed as odd extensions of the columns:
// in [rows][H] (complex, k = 1..K used), out [K][Mo] with out[k-1][r+1] = value and
// out[k-1][Mo - r - 1] = -value, zeros at 0 and rows + 1. Optionally divided by
// (lam_in[k-1] + lam_out[r]) (not here) -- plain transposition via 32 x 32 tiles.
template <typename R, typename Cx>
__global__ void k_im_transpose_ext(const Cx* __restrict__ in, int rows, int H, int K, R* __restrict__ out, int Mo) {
  __shared__ R tile[32][33];
  const int k0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int r = r0 + dy, k = k0 + threadIdx.x;
    tile[dy][threadIdx.x] = (r < rows && k < K) ? -R(0.5) * in[(size_t)r * H + (k + 1)].y : R(0);
  }
  __syncthreads();
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int k = k0 + dy, r = r0 + threadIdx.x;
    if (k < K && r < rows) {
      const R v = tile[threadIdx.x][dy];
      R* o = out + (size_t)k * Mo;
      o[r + 1] = v;
      o[Mo - r - 1] = -v;
      if (r == 0) o[0] = R(0);
      if (r == rows - 1) o[rows + 1] = R(0);
    }
  }
}

// a / b: FP32 by the fast reciprocal (2 ulp; b is a sum of two negative eigenvalues,
// far from the range where it loses accuracy), FP64 exactly.
__device__ __forceinline__ float div_eig(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double div_eig(double a, double b) { return a / b; }

// In place along the same rows: b = -Im/2 / (lam_x[row] + lam_y[l]) written back as
// the odd extension of the row (for the inverse transform along y).
template <typename R, typename Cx>
__global__ void k_scale_ext(const Cx* __restrict__ in, int rows, int H, int L, const R* __restrict__ lamx,
                            const R* __restrict__ lamy, R* __restrict__ out, int Mo) {
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    const R lx = lamx[r];
    R* o = out + (size_t)r * Mo;
    const Cx* q = in + (size_t)r * H;
    for (int l = threadIdx.x; l < L + 2; l += blockDim.x) {
      if (l == 0 || l == L + 1) {
        o[l] = R(0);
        continue;
      }
      const R v = div_eig(-R(0.5) * q[l].y, lx + lamy[l - 1]);
      o[l] = v;
      o[Mo - l] = -v;
    }
  }
}

// psi = norm x (-Im/2) of the final row transform at I's box nodes, into the interior
// of the plane of the current parity (the halo stays zero).
template <typename R, typename Cx>
__global__ void k_scatter_psi(const Cx* __restrict__ in, int H, int nx, int ny, int bx, int by, R norm,
                              const DevState* st, R* __restrict__ psi0, R* __restrict__ psi1) {
  R* __restrict__ psi = (st->steps & 1) ? psi1 : psi0;
  for (int jp = blockIdx.x; jp < ny - 4; jp += gridDim.x)  // 0-based interior indices
    for (int ip = threadIdx.x; ip < nx - 4; ip += blockDim.x)
      psi[(size_t)(jp + 2) * nx + (ip + 2)] = norm * (-R(0.5) * in[(size_t)(jp + by) * H + (ip + 1 + bx)].y);
}

// ---- host side
namespace {

template <typename R>
cudaError_t solve_t(DemagSolver* d, const DevState* st, void* const phi[2], void* const lo[2], void* const psi[2],
                    cudaStream_t s) {
  using Cx = typename FftOf<R>::C;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = nsm * 8;
  R* ext_x = static_cast<R*>(d->ext_x);
  R* ext_y = static_cast<R*>(d->ext_y);
  Cx* cx = static_cast<Cx*>(d->cx);
  Cx* cy = static_cast<Cx*>(d->cy);
  const R* lam = static_cast<const R*>(d->lam);
  k_rho_ext<R><<<grid, 256, 0, s>>>(static_cast<const R*>(phi[0]), static_cast<const R*>(phi[1]),
                                    static_cast<const R*>(lo[0]), static_cast<const R*>(lo[1]), st, d->nx, d->ny,
                                    (size_t)d->nx * d->ny, d->Nx, d->Ny, d->bx, d->by, d->Mx,
                                    (R)(1.0 / (12.0 * d->dx)), (R)(1.0 / (12.0 * d->dy)), ext_x);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cufftSetStream(d->px, s);
  cufftSetStream(d->py, s);
  if (FftOf<R>::exec(d->px, ext_x, cx) != CUFFT_SUCCESS) return cudaErrorLaunchFailure;  // along x, every row
  const dim3 tb(32, 8);
  k_im_transpose_ext<R, Cx><<<dim3((d->Nx + 31) / 32, (d->Ny + 31) / 32), tb, 0, s>>>(cx, d->Ny, d->Hx, d->Nx, ext_y,
                                                                                        d->My);
  if (FftOf<R>::exec(d->py, ext_y, cy) != CUFFT_SUCCESS) return cudaErrorLaunchFailure;  // along y, every column
  k_scale_ext<R, Cx><<<grid, 256, 0, s>>>(cy, d->Nx, d->Hy, d->Ny, lam, lam + d->Nx, ext_y, d->My);
  if (FftOf<R>::exec(d->py, ext_y, cy) != CUFFT_SUCCESS) return cudaErrorLaunchFailure;  // back along y
  k_im_transpose_ext<R, Cx><<<dim3((d->Ny + 31) / 32, (d->Nx + 31) / 32), tb, 0, s>>>(cy, d->Nx, d->Hy, d->Ny, ext_x,
                                                                                        d->Mx);
  if (FftOf<R>::exec(d->px, ext_x, cx) != CUFFT_SUCCESS) return cudaErrorLaunchFailure;  // back along x
  const R norm = (R)((2.0 / (d->Nx + 1)) * (2.0 / (d->Ny + 1)));
  k_scatter_psi<R, Cx><<<grid, 256, 0, s>>>(cx, d->Hx, d->nx, d->ny, d->bx, d->by, norm, st,
                                            static_cast<R*>(psi[0]), static_cast<R*>(psi[1]));
  return cudaGetLastError();
}

template <typename R>
int create_t(DemagSolver* d) {
  using Cx = typename FftOf<R>::C;
  const size_t ex = sizeof(R) * (size_t)d->Ny * d->Mx, cxb = sizeof(Cx) * (size_t)d->Ny * d->Hx;
  const size_t ey = sizeof(R) * (size_t)d->Nx * d->My, cyb = sizeof(Cx) * (size_t)d->Nx * d->Hy;
  if (cudaMalloc(&d->ext_x, ex) != cudaSuccess || cudaMalloc(&d->cx, cxb) != cudaSuccess ||
      cudaMalloc(&d->ext_y, ey) != cudaSuccess || cudaMalloc(&d->cy, cyb) != cudaSuccess ||
      cudaMalloc(&d->lam, sizeof(R) * (size_t)(d->Nx + d->Ny)) != cudaSuccess)
    return -1;
  std::vector<R> lam((size_t)d->Nx + d->Ny);
  const double pi = 3.14159265358979323846;
  for (int k = 1; k <= d->Nx; ++k) lam[k - 1] = (R)(-(2.0 - 2.0 * std::cos(pi * k / (d->Nx + 1))) / (d->dx * d->dx));
  for (int l = 1; l <= d->Ny; ++l)
    lam[d->Nx + l - 1] = (R)(-(2.0 - 2.0 * std::cos(pi * l / (d->Ny + 1))) / (d->dy * d->dy));
  if (cudaMemcpy(d->lam, lam.data(), sizeof(R) * lam.size(), cudaMemcpyHostToDevice) != cudaSuccess) return -1;
  int n = d->Mx;
  if (cufftPlanMany(&d->px, 1, &n, nullptr, 1, d->Mx, nullptr, 1, d->Hx, FftOf<R>::type, d->Ny) != CUFFT_SUCCESS)
    return -2;
  d->have_px = true;
  n = d->My;
  if (cufftPlanMany(&d->py, 1, &n, nullptr, 1, d->My, nullptr, 1, d->Hy, FftOf<R>::type, d->Nx) != CUFFT_SUCCESS)
    return -2;
  d->have_py = true;
  return 0;
}

}  // namespace

namespace {
// The Dirichlet box along an axis of N interior sites: the smallest N' >= N whose
// N' + 1 has no prime factor above 7 (the transform length 2 (N' + 1) then factors
// into small primes; 2 (N + 1) with a large prime factor, as 2 (4092 + 1) = 2 x 4093,
// is several times slower), and floor((N' - N) / 2) of the extra sites below I.
void box_of(int N, int* Np, int* below) {
  int n = N;
  for (;; ++n) {
    int m = n + 1;
    for (int q = 2; q <= 7; ++q)
      while (m % q == 0) m /= q;
    if (m == 1) break;
  }
  *Np = n;
  *below = (n - N) / 2;
}
}  // namespace

int demag_create(DemagSolver** out, int nx, int ny, double dx, double dy, int prec) {
  *out = nullptr;
  DemagSolver* d = new (std::nothrow) DemagSolver();
  if (!d) return -1;
  d->nx = nx;
  d->ny = ny;
  box_of(nx - 4, &d->Nx, &d->bx);
  box_of(ny - 4, &d->Ny, &d->by);
  d->Mx = 2 * (d->Nx + 1);
  d->My = 2 * (d->Ny + 1);
  d->Hx = d->Mx / 2 + 1;
  d->Hy = d->My / 2 + 1;
  d->dx = dx;
  d->dy = dy;
  d->prec = prec;
  const int rc = prec == PREC_F64 ? create_t<double>(d) : create_t<float>(d);
  if (rc != 0) {
    demag_destroy(d);
    return rc;
  }
  *out = d;
  return 0;
}

void demag_destroy(DemagSolver* d) {
  if (!d) return;
  if (d->have_px) cufftDestroy(d->px);
  if (d->have_py) cufftDestroy(d->py);
  cudaFree(d->ext_x);
  cudaFree(d->cx);
  cudaFree(d->ext_y);
  cudaFree(d->cy);
  cudaFree(d->lam);
  delete d;
}

cudaError_t demag_solve(DemagSolver* d, const DevState* st, void* const phi[2], void* const lo[2], void* const psi[2],
                        cudaStream_t s) {
  return d->prec == PREC_F64 ? solve_t<double>(d, st, phi, lo, psi, s) : solve_t<float>(d, st, phi, lo, psi, s);
}

}  // namespace ss
