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
// The transforms are this file's own. A DST-I of length N is -Im/2 of the DFT of the
// odd extension y = (0, s_1 .. s_N, 0, -s_N .. -s_1) of length 2L, L = N + 1; that real
// DFT is one complex DFT of length L of z_n = y_2n + i y_2n+1, unpacked as
//   Y_k = E_k + e^{-i pi k / L} O_k,  E_k = (Z_k + conj Z_{L-k}) / 2,  O_k = (Z_k - conj Z_{L-k}) / 2i.
// The complex DFT is a Stockham autosort FFT (radix 16, 8, 4, 2, 3, 5, 7 stages, L being
// 7-smooth) held in shared memory: one thread block transforms one line, reading it
// once from global memory and writing it once. The solve is three line kernels and two
// tiled transposes:
//   rows:    rho (formed from the field on the fly) -> DST along x           -> T1 [Ny][Nx]
//   T1 -> T2 [Nx][Ny] (transpose)
//   columns: DST along y, division by lambda, DST along y again (in place)    -> T2
//   T2 -> T1 (transpose)
//   rows:    DST along x, the normalisation, psi on I into the current plane
// Twiddles are tabulated once in FP64 and rounded to the working type. The field's
// ping-pong parity is read on the device from the flow record, so the solve can sit
// inside a captured step graph.
#include <cmath>
#include <new>
#include <vector>

#include "ss_internal.h"

namespace ss {

namespace {

constexpr int DST_THREADS = 256;
// Radix-16 Stockham stages where the length allows (1) or radix 8 at most (0), and padded
// shared line buffers (1) or dense ones (0). The Poisson solve at 4096^2 (FP32, one GPU,
// all four builds): dense radix 8 0.778 ms, dense radix 16 0.817 ms, padded radix 8 0.724
// ms, padded radix 16 0.648 ms (0.659 ms with the radix-16 twiddles one product deep,
// the kept form: on a fixed 4096^2 field its FP32 demagnetisation energy is 3.1e-7 from
// the FP64 solve's, against 3.4e-7 with radix 8 and 3.6e-7 with products three deep).
#ifndef SS_DST_R16
#define SS_DST_R16 1
#endif
#ifndef SS_DST_PAD
#define SS_DST_PAD 1
#endif
constexpr int TW_FINE = 64;  // twiddles as coarse x fine factors: e^{-2 pi i t / L} = C[t / 64] F[t % 64]
constexpr int DST_MAX_STAGES = 24;

template <typename R>
struct Cx {
  R x, y;
};
template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
  return Cx<R>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename R>
__device__ __forceinline__ Cx<R> cadd(Cx<R> a, Cx<R> b) { return Cx<R>{a.x + b.x, a.y + b.y}; }
template <typename R>
__device__ __forceinline__ Cx<R> csub(Cx<R> a, Cx<R> b) { return Cx<R>{a.x - b.x, a.y - b.y}; }

// One line transform: radices of its Stockham stages, and its tables.
template <typename R>
struct LinePlan {
  int L;                            // complex DFT length (= N + 1)
  int nst;                          // stages
  int rad[DST_MAX_STAGES];          // radix of each stage (product = L)
  unsigned magic[DST_MAX_STAGES];   // ceil(2^32 / Ns) of each stage (0 when Ns = 1)
  int ncoarse;                      // ceil(L / 64)
  const Cx<R>* tw;                  // global: C[h] = e^{-2 pi i 64 h / L} (ncoarse), then F[l] = e^{-2 pi i l / L} (64)
  const Cx<R>* pw;                  // pw[k] = e^{-i pi k / L}, k <= L
};

// The twiddle table of a line, staged in shared memory once per block.
template <typename R>
struct Tw {
  const Cx<R>* c;
  const Cx<R>* f;
  __device__ __forceinline__ Cx<R> operator[](int t) const { return cmul(c[t / TW_FINE], f[t % TW_FINE]); }
};

// Shared line buffers hold element i at pz(i): one unused slot after every 16, so that a
// first stage's writes (each thread's RAD outputs at consecutive positions) and the
// strided accesses of later stages fall on different banks.
__host__ __device__ __forceinline__ int pz(int i) { return SS_DST_PAD ? i + (i >> 4) : i; }
__host__ __device__ __forceinline__ int pad_len(int L) { return SS_DST_PAD ? L + (L >> 4) + 1 : L; }

// j / Ns for the butterfly indices j < L <= 2^14 of a stage: with m = ceil(2^32 / Ns),
// floor(j m / 2^32) = floor(j / Ns) exactly because j Ns < 2^32.
__device__ __forceinline__ int div_ns(int j, int Ns, unsigned m) { return Ns == 1 ? j : (int)__umulhi((unsigned)j, m); }

// One Stockham stage of radix RAD (Ns = product of the earlier radices): butterfly j
// reads src[j + r L / RAD], twiddles r by e^{-2 pi i r (j mod Ns) / (Ns RAD)}, takes
// the RAD-point DFT and writes dst[(j / Ns) Ns RAD + j mod Ns + k Ns].
template <int RAD, typename R>
__device__ __forceinline__ void stockham_stage(const Cx<R>* __restrict__ src, Cx<R>* __restrict__ dst, int L, int Ns,
                                               unsigned magic, const Tw<R>& tw) {
  const int nb = L / RAD;
  const int step = L / (Ns * RAD);
  constexpr int UNR = (RAD <= 4 || RAD == 8) ? 2 : 1;  // two butterflies in flight where registers allow
  // radix-16 internal twiddles W16^1 and W16^3: (cos pi/8, -sin pi/8) and (sin pi/8, -cos pi/8)
  const R c8 = R(0.92387953251128675613), s8 = R(0.38268343236508977173), h = R(0.70710678118654752440);
#pragma unroll UNR
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    const int jd = div_ns(j, Ns, magic);
    const int jm = j - jd * Ns;
    Cx<R> v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[r] = src[pz(j + r * nb)];
    if (RAD == 16) {  // w^1, w^2, w^3, w^4, w^8, w^12 from the table, every other power one product of two
      const int t1 = jm * step;
      const Cx<R> w1 = tw[t1], w2 = tw[2 * t1], w3 = tw[3 * t1], w4 = tw[4 * t1], w8 = tw[8 * t1],
                  w12 = tw[12 * t1];
      const Cx<R> w[16] = {Cx<R>{R(1), R(0)}, w1, w2, w3, w4, cmul(w1, w4), cmul(w2, w4), cmul(w3, w4),
                           w8, cmul(w1, w8), cmul(w2, w8), cmul(w3, w8), w12, cmul(w1, w12), cmul(w2, w12),
                           cmul(w3, w12)};
#pragma unroll
      for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], w[r]);
    } else if (RAD == 8) {  // w^1, w^2, w^4 from the table, the other powers as their products
      const int t1 = jm * step;
      const Cx<R> w1 = tw[t1], w2 = tw[2 * t1], w4 = tw[4 * t1];
      const Cx<R> w3 = cmul(w1, w2);
      v[1] = cmul(v[1], w1);
      v[2] = cmul(v[2], w2);
      v[3] = cmul(v[3], w3);
      v[4] = cmul(v[4], w4);
      v[5] = cmul(v[5], cmul(w1, w4));
      v[6] = cmul(v[6], cmul(w2, w4));
      v[7] = cmul(v[7], cmul(w3, w4));
    } else {
#pragma unroll
      for (int r = 1; r < RAD; ++r) v[r] = cmul(v[r], tw[jm * r * step]);
    }
    Cx<R> o[RAD];
    if (RAD == 16) {  // 4 x 4: n = n2 + 4 n1, k = k1 + 4 k2
      // 4-point DFTs over n1, then the factors W16^(n2 k1), then 4-point DFTs over n2
      Cx<R> A[4][4];
#pragma unroll
      for (int n2 = 0; n2 < 4; ++n2) {
        const Cx<R> a = cadd(v[n2], v[n2 + 8]), b = csub(v[n2], v[n2 + 8]);
        const Cx<R> c = cadd(v[n2 + 4], v[n2 + 12]), d = csub(v[n2 + 4], v[n2 + 12]);
        A[n2][0] = cadd(a, c);
        A[n2][2] = csub(a, c);
        A[n2][1] = Cx<R>{b.x + d.y, b.y - d.x};  // b - i d
        A[n2][3] = Cx<R>{b.x - d.y, b.y + d.x};  // b + i d
      }
      auto mulw = [](Cx<R> z, R wr, R wi) { return Cx<R>{z.x * wr - z.y * wi, z.x * wi + z.y * wr}; };
      A[1][1] = mulw(A[1][1], c8, -s8);                          // W16^1
      A[1][2] = mulw(A[1][2], h, -h);                            // W16^2
      A[1][3] = mulw(A[1][3], s8, -c8);                          // W16^3
      A[2][1] = mulw(A[2][1], h, -h);                            // W16^2
      A[2][2] = Cx<R>{A[2][2].y, -A[2][2].x};                    // W16^4 = -i
      A[2][3] = mulw(A[2][3], -h, -h);                           // W16^6
      A[3][1] = mulw(A[3][1], s8, -c8);                          // W16^3
      A[3][2] = mulw(A[3][2], -h, -h);                           // W16^6
      A[3][3] = mulw(A[3][3], -c8, s8);                          // W16^9
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1) {
        const Cx<R> a = cadd(A[0][k1], A[2][k1]), b = csub(A[0][k1], A[2][k1]);
        const Cx<R> c = cadd(A[1][k1], A[3][k1]), d = csub(A[1][k1], A[3][k1]);
        o[k1] = cadd(a, c);
        o[k1 + 8] = csub(a, c);
        o[k1 + 4] = Cx<R>{b.x + d.y, b.y - d.x};   // b - i d
        o[k1 + 12] = Cx<R>{b.x - d.y, b.y + d.x};  // b + i d
      }
    } else if (RAD == 8) {  // three radix-2 levels; W8 = (1 - i) / sqrt 2, W8^3 = (-1 - i) / sqrt 2
      auto mi = [](Cx<R> z) { return Cx<R>{z.y, -z.x}; };  // z * (-i)
      const Cx<R> a0 = cadd(v[0], v[4]), a1 = csub(v[0], v[4]), a2 = cadd(v[2], v[6]), a3 = mi(csub(v[2], v[6]));
      const Cx<R> a4 = cadd(v[1], v[5]), a5 = csub(v[1], v[5]), a6 = cadd(v[3], v[7]), a7 = mi(csub(v[3], v[7]));
      const Cx<R> b0 = cadd(a0, a2), b2 = csub(a0, a2), b1 = cadd(a1, a3), b3 = csub(a1, a3);
      const Cx<R> b4 = cadd(a4, a6), b6 = mi(csub(a4, a6)), b5 = cadd(a5, a7), b7 = csub(a5, a7);
      const Cx<R> t5{h * (b5.x + b5.y), h * (b5.y - b5.x)};     // W8 b5
      const Cx<R> t7{h * (b7.y - b7.x), -h * (b7.x + b7.y)};    // W8^3 b7
      o[0] = cadd(b0, b4);
      o[4] = csub(b0, b4);
      o[2] = cadd(b2, b6);
      o[6] = csub(b2, b6);
      o[1] = cadd(b1, t5);
      o[5] = csub(b1, t5);
      o[3] = cadd(b3, t7);
      o[7] = csub(b3, t7);
    } else if (RAD == 2) {
      o[0] = cadd(v[0], v[1]);
      o[1] = csub(v[0], v[1]);
    } else if (RAD == 4) {
      const Cx<R> a = cadd(v[0], v[2]), b = csub(v[0], v[2]), c = cadd(v[1], v[3]), d = csub(v[1], v[3]);
      o[0] = cadd(a, c);
      o[2] = csub(a, c);
      o[1] = Cx<R>{b.x + d.y, b.y - d.x};  // b - i d
      o[3] = Cx<R>{b.x - d.y, b.y + d.x};  // b + i d
    } else {  // 3, 5, 7: the direct DFT with the table's roots of unity
#pragma unroll
      for (int k = 0; k < RAD; ++k) {
        Cx<R> acc = v[0];
#pragma unroll
        for (int r = 1; r < RAD; ++r) acc = cadd(acc, cmul(v[r], tw[((r * k) % RAD) * (L / RAD)]));
        o[k] = acc;
      }
    }
    const int idx = jd * Ns * RAD + jm;
#pragma unroll
    for (int k = 0; k < RAD; ++k) dst[pz(idx + k * Ns)] = o[k];
  }
}

// Copy a line's coarse and fine twiddle factors into shared memory at t (the block's
// first use of them follows a barrier).
template <typename R>
__device__ __forceinline__ Tw<R> stage_twiddles(Cx<R>* t, const LinePlan<R>& p) {
  for (int i = threadIdx.x; i < p.ncoarse + TW_FINE; i += blockDim.x) t[i] = p.tw[i];
  __syncthreads();
  return Tw<R>{t, t + p.ncoarse};
}

// DFT of the L complex values in a (scratch b): returns the buffer holding the result.
template <typename R>
__device__ Cx<R>* line_fft(Cx<R>* a, Cx<R>* b, const LinePlan<R>& p, const Tw<R>& tw) {
  int Ns = 1;
  for (int s = 0; s < p.nst; ++s) {
    const int rad = p.rad[s];
    const unsigned m = p.magic[s];
    if (rad == 16) stockham_stage<16, R>(a, b, p.L, Ns, m, tw);
    else if (rad == 8) stockham_stage<8, R>(a, b, p.L, Ns, m, tw);
    else if (rad == 4) stockham_stage<4, R>(a, b, p.L, Ns, m, tw);
    else if (rad == 2) stockham_stage<2, R>(a, b, p.L, Ns, m, tw);
    else if (rad == 3) stockham_stage<3, R>(a, b, p.L, Ns, m, tw);
    else if (rad == 5) stockham_stage<5, R>(a, b, p.L, Ns, m, tw);
    else stockham_stage<7, R>(a, b, p.L, Ns, m, tw);
    __syncthreads();
    Ns *= rad;
    Cx<R>* t = a;
    a = b;
    b = t;
  }
  return a;
}

// z_n = y_2n + i y_2n+1 of the odd extension of s_1 .. s_N (s(m) gives s_m, 1 <= m <= N):
// the N values are gathered once into tmp (L values of scratch, not z), then paired.
template <int UNR, typename R, typename S>
__device__ __forceinline__ void line_pack(Cx<R>* z, R* tmp, int L, S s) {
#pragma unroll UNR
  for (int m = 1 + threadIdx.x; m < L; m += blockDim.x) tmp[m] = s(m);  // UNR loads in flight per thread
  __syncthreads();
  auto y = [&](int m) -> R {
    if (m == 0 || m == L) return R(0);
    return m < L ? tmp[m] : -tmp[2 * L - m];
  };
  for (int n = threadIdx.x; n < L; n += blockDim.x) z[pz(n)] = Cx<R>{y(2 * n), y(2 * n + 1)};
}

// Every DST_k, k = 1 .. L - 1, to out(k, value), two at a time: k and L - k share the
// loads of Z_k, Z_{L-k} and the factor w_k = e^{-i pi k / L}, since E_{L-k} = conj E_k,
// O_{L-k} = conj O_k and w_{L-k} = -conj w_k give Im Y_{L-k} = -(Im E_k - Im(w_k O_k)).
template <int UNR, typename R, typename F>
__device__ __forceinline__ void line_dst_all(const Cx<R>* Z, int L, const Cx<R>* __restrict__ pw, F out) {
#pragma unroll UNR
  for (int k = 1 + threadIdx.x; 2 * k <= L; k += blockDim.x) {
    const Cx<R> zk = Z[pz(k)], zc = Z[pz(L - k)];
    const R Ey = R(0.5) * (zk.y - zc.y);
    const Cx<R> O{R(0.5) * (zk.y + zc.y), -R(0.5) * (zk.x - zc.x)};
    const Cx<R> w = pw[k];
    const R wo = w.x * O.y + w.y * O.x;  // Im(w_k O_k)
    out(k, -R(0.5) * (Ey + wo));
    if (2 * k != L) out(L - k, R(0.5) * (Ey - wo));
  }
}

// rho at box node (m, jp + 1) of an x line (m = 1 .. Nx): the Eq. 1 divergence of the
// in-plane field on I, zero on the box's padding.
template <typename R>
struct RhoRow {
  const R* f;
  const R* lo;
  int nx, ny, bx, by, jp;
  size_t plane;
  R i12dx, i12dy;
  __device__ __forceinline__ R operator()(int m) const {
    const int i = m + 1 - bx, j = jp + 2 - by;
    if (i < 2 || i > nx - 3 || j < 2 || j > ny - 3) return R(0);
    const size_t s = (size_t)j * nx + i;
    auto d1 = [&](const R* p, size_t c, ptrdiff_t st1, R sc) {
      const R* q = p + c * plane + s;
      return (R(8) * (q[st1] - q[-st1]) - (q[2 * st1] - q[-2 * st1])) * sc;
    };
    R rho = d1(f, 0, 1, i12dx) + d1(f, 1, (ptrdiff_t)nx, i12dy);
    if (lo) rho += d1(lo, 0, 1, i12dx) + d1(lo, 1, (ptrdiff_t)nx, i12dy);
    return rho;
  }
};

// Rows of the box along x: rho, its DST, into T1[Ny][Nx].
template <typename R>
__global__ void __launch_bounds__(DST_THREADS, sizeof(R) == 4 ? 3 : 1) k_dst_rho_rows(const R* __restrict__ phi0, const R* __restrict__ phi1,
                                                              const R* __restrict__ lo0, const R* __restrict__ lo1,
                                                              const DevState* st, int nx, int ny, size_t plane, int Nx,
                                                              int Ny, int bx, int by, R i12dx, R i12dy,
                                                              const LinePlan<R> p, R* __restrict__ T1) {
  extern __shared__ __align__(16) unsigned char dsm[];
  Cx<R>* a = reinterpret_cast<Cx<R>*>(dsm);
  Cx<R>* b = a + pad_len(p.L);
  const Tw<R> tw = stage_twiddles(b + pad_len(p.L), p);
  const int cur = (int)(st->steps & 1);
  RhoRow<R> rr{cur ? phi1 : phi0, cur ? lo1 : lo0, nx, ny, bx, by, 0, plane, i12dx, i12dy};
  for (int jp = blockIdx.x; jp < Ny; jp += gridDim.x) {
    rr.jp = jp;
    line_pack<2>(a, reinterpret_cast<R*>(b), p.L, rr);
    __syncthreads();
    const Cx<R>* Z = line_fft(a, b, p, tw);
    R* out = T1 + (size_t)jp * Nx;
    line_dst_all<2>(Z, p.L, p.pw, [&](int k, R v) { out[k - 1] = v; });
    __syncthreads();
  }
}

// Columns of the box (rows of T2[Nx][Ny]): DST along y, division by lambda_x + lambda_y,
// DST along y again, in place.
template <typename R>
__global__ void __launch_bounds__(DST_THREADS, sizeof(R) == 4 ? 3 : 1) k_dst_solve_cols(R* __restrict__ T2, int Nx, int Ny,
                                                                const R* __restrict__ lamx, const R* __restrict__ lamy,
                                                                const LinePlan<R> p) {
  extern __shared__ __align__(16) unsigned char dsm[];
  Cx<R>* a = reinterpret_cast<Cx<R>*>(dsm);
  Cx<R>* b = a + pad_len(p.L);
  const Tw<R> tw = stage_twiddles(b + pad_len(p.L), p);
  for (int r = blockIdx.x; r < Nx; r += gridDim.x) {
    R* line = T2 + (size_t)r * Ny;
    const R lx = lamx[r];
    line_pack<8>(a, reinterpret_cast<R*>(b), p.L, [&](int m) { return line[m - 1]; });
    __syncthreads();
    const Cx<R>* Z = line_fft(a, b, p, tw);
    // the divided coefficients, in the other buffer (as reals, index l = 1 .. Ny)
    Cx<R>* c = (Z == a) ? b : a;
    R* cr = reinterpret_cast<R*>(c);
    line_dst_all<2>(Z, p.L, p.pw, [&](int l, R v) { cr[l] = v / (lx + lamy[l - 1]); });
    __syncthreads();
    // the second transform's input: its gather is in place (each thread copies its own
    // entries), its pairs go to Z's buffer, free now
    Cx<R>* z2 = const_cast<Cx<R>*>(Z);
    line_pack<4>(z2, cr, p.L, [&](int m) { return cr[m]; });
    __syncthreads();
    const Cx<R>* Z2 = line_fft(z2, c, p, tw);
    line_dst_all<2>(Z2, p.L, p.pw, [&](int l, R v) { line[l - 1] = v; });
    __syncthreads();
  }
}

// Rows along x again: DST, the normalisation, and psi on I into the plane of the current
// parity (its halo stays zero).
template <typename R>
__global__ void __launch_bounds__(DST_THREADS, sizeof(R) == 4 ? 3 : 1) k_dst_psi_rows(const R* __restrict__ T1, int nx, int ny, int Nx, int Ny,
                                                              int bx, int by, R norm, const LinePlan<R> p,
                                                              const DevState* st, R* __restrict__ psi0,
                                                              R* __restrict__ psi1) {
  extern __shared__ __align__(16) unsigned char dsm[];
  Cx<R>* a = reinterpret_cast<Cx<R>*>(dsm);
  Cx<R>* b = a + pad_len(p.L);
  const Tw<R> tw = stage_twiddles(b + pad_len(p.L), p);
  R* __restrict__ psi = (st->steps & 1) ? psi1 : psi0;
  for (int jp = blockIdx.x; jp < Ny; jp += gridDim.x) {
    const int j = jp + 2 - by;  // full-array row of box row jp
    if (j < 2 || j > ny - 3) continue;  // uniform over the block
    const R* line = T1 + (size_t)jp * Nx;
    line_pack<8>(a, reinterpret_cast<R*>(b), p.L, [&](int m) { return line[m - 1]; });
    __syncthreads();
    const Cx<R>* Z = line_fft(a, b, p, tw);
    line_dst_all<2>(Z, p.L, p.pw, [&](int m, R v) {
      const int i = m + 1 - bx;  // the site of box column m
      if (i >= 2 && i <= nx - 3) psi[(size_t)j * nx + i] = norm * v;
    });
    __syncthreads();
  }
}

// out[c][r] = in[r][c] for an rows x cols array, through 32 x 32 shared tiles.
template <typename R>
__global__ void k_transpose(const R* __restrict__ in, int rows, int cols, R* __restrict__ out) {
  __shared__ R tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int r = r0 + dy, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[dy][threadIdx.x] = in[(size_t)r * cols + c];
  }
  __syncthreads();
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int c = c0 + dy, r = r0 + threadIdx.x;
    if (c < cols && r < rows) out[(size_t)c * rows + r] = tile[threadIdx.x][dy];
  }
}

// Radices of a 7-smooth length, sixteens, eights and fours first; 0 if L has another prime
// factor or needs too many stages.
int plan_radices(int L, int* rad) {
  int n = 0, m = L;
  while (m % 16 == 0 && SS_DST_R16 && n < DST_MAX_STAGES) { rad[n++] = 16; m /= 16; }
  while (m % 8 == 0 && n < DST_MAX_STAGES) { rad[n++] = 8; m /= 8; }
  while (m % 4 == 0 && n < DST_MAX_STAGES) { rad[n++] = 4; m /= 4; }
  const int ps[4] = {2, 3, 5, 7};
  for (int q : ps)
    while (m % q == 0 && n < DST_MAX_STAGES) { rad[n++] = q; m /= q; }
  return m == 1 ? n : 0;
}

}  // namespace

struct DemagSolver {
  int nx = 0, ny = 0;
  int Nx = 0, Ny = 0;  // Dirichlet box sites per axis (>= the interior's nx - 4, ny - 4)
  int bx = 0, by = 0;  // box sites below I along x, y
  int prec = 0;        // PREC_*: FP64 transforms for FP64 fields, FP32 otherwise
  double dx = 0, dy = 0;
  void* T1 = nullptr;   // R [Ny][Nx]
  void* T2 = nullptr;   // R [Nx][Ny]
  void* tab = nullptr;  // twiddles of both axes, then lambda_x, lambda_y
  int radx[DST_MAX_STAGES] = {0}, rady[DST_MAX_STAGES] = {0};
  int nstx = 0, nsty = 0;
  size_t off_twx = 0, off_pwx = 0, off_twy = 0, off_pwy = 0, off_lam = 0;  // element offsets into tab
  int occ = 1;  // resident blocks per SM of the line kernels
};

namespace {

template <typename R>
size_t line_smem(int L) { return sizeof(Cx<R>) * (2 * (size_t)pad_len(L) + (L + TW_FINE - 1) / TW_FINE + TW_FINE); }

template <typename R>
LinePlan<R> plan_of(const DemagSolver* d, int axis) {
  LinePlan<R> p{};
  const Cx<R>* t = static_cast<const Cx<R>*>(d->tab);
  p.L = (axis == 0 ? d->Nx : d->Ny) + 1;
  p.nst = axis == 0 ? d->nstx : d->nsty;
  long long Ns = 1;
  for (int s = 0; s < p.nst; ++s) {
    p.rad[s] = axis == 0 ? d->radx[s] : d->rady[s];
    p.magic[s] = Ns == 1 ? 0u : (unsigned)(((1ULL << 32) + (unsigned long long)Ns - 1) / (unsigned long long)Ns);
    Ns *= p.rad[s];
  }
  p.ncoarse = (p.L + TW_FINE - 1) / TW_FINE;
  p.tw = t + (axis == 0 ? d->off_twx : d->off_twy);
  p.pw = t + (axis == 0 ? d->off_pwx : d->off_pwy);
  return p;
}

template <typename R>
cudaError_t solve_t(DemagSolver* d, const DevState* st, void* const phi[2], void* const lo[2], void* const psi[2],
                    cudaStream_t s) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const LinePlan<R> px = plan_of<R>(d, 0), py = plan_of<R>(d, 1);
  R* T1 = static_cast<R*>(d->T1);
  R* T2 = static_cast<R*>(d->T2);
  const R* lam = reinterpret_cast<const R*>(static_cast<const Cx<R>*>(d->tab) + d->off_lam);
  // one wave of resident blocks striding over the lines
  const int gx = d->Ny < d->occ * nsm ? d->Ny : d->occ * nsm, gy = d->Nx < d->occ * nsm ? d->Nx : d->occ * nsm;
  k_dst_rho_rows<R><<<gx, DST_THREADS, line_smem<R>(px.L), s>>>(
      static_cast<const R*>(phi[0]), static_cast<const R*>(phi[1]), static_cast<const R*>(lo[0]),
      static_cast<const R*>(lo[1]), st, d->nx, d->ny, (size_t)d->nx * d->ny, d->Nx, d->Ny, d->bx, d->by,
      (R)(1.0 / (12.0 * d->dx)), (R)(1.0 / (12.0 * d->dy)), px, T1);
  const dim3 tb(32, 8);
  k_transpose<R><<<dim3((d->Nx + 31) / 32, (d->Ny + 31) / 32), tb, 0, s>>>(T1, d->Ny, d->Nx, T2);
  k_dst_solve_cols<R><<<gy, DST_THREADS, line_smem<R>(py.L), s>>>(T2, d->Nx, d->Ny, lam, lam + d->Nx, py);
  k_transpose<R><<<dim3((d->Ny + 31) / 32, (d->Nx + 31) / 32), tb, 0, s>>>(T2, d->Nx, d->Ny, T1);
  const R norm = (R)((2.0 / (d->Nx + 1)) * (2.0 / (d->Ny + 1)));
  k_dst_psi_rows<R><<<gx, DST_THREADS, line_smem<R>(px.L), s>>>(T1, d->nx, d->ny, d->Nx, d->Ny, d->bx, d->by, norm,
                                                                 px, st, static_cast<R*>(psi[0]),
                                                                 static_cast<R*>(psi[1]));
  return cudaGetLastError();
}

template <typename R>
int create_t(DemagSolver* d) {
  const int Lx = d->Nx + 1, Ly = d->Ny + 1;
  d->nstx = plan_radices(Lx, d->radx);
  d->nsty = plan_radices(Ly, d->rady);
  if (!d->nstx || !d->nsty) return -2;
  int dev = 0;
  size_t max_smem = 0;
  {
    int v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    max_smem = (size_t)v;
  }
  const size_t need = line_smem<R>(Lx > Ly ? Lx : Ly);
  if (need > max_smem || Lx > (1 << 14) || Ly > (1 << 14)) return -2;  // one line per block, exact index division
  if (cudaFuncSetAttribute(k_dst_rho_rows<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need) != cudaSuccess ||
      cudaFuncSetAttribute(k_dst_solve_cols<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_dst_psi_rows<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need) != cudaSuccess)
    return -2;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_dst_solve_cols<R>, DST_THREADS, need) != cudaSuccess)
    return -2;
  d->occ = occ < 1 ? 1 : occ;
  // tables: twiddle factors x (coarse, fine), pw_x [Lx + 1], the same for y, then lambda_x [Nx],
  // lambda_y [Ny] as R
  d->off_twx = 0;
  d->off_pwx = d->off_twx + (Lx + TW_FINE - 1) / TW_FINE + TW_FINE;
  d->off_twy = d->off_pwx + Lx + 1;
  d->off_pwy = d->off_twy + (Ly + TW_FINE - 1) / TW_FINE + TW_FINE;
  d->off_lam = d->off_pwy + Ly + 1;
  const size_t ncx = d->off_lam + (d->Nx + d->Ny + 1) / 2 + 1;  // lambdas packed two per complex slot
  std::vector<Cx<R>> t(ncx, Cx<R>{R(0), R(0)});
  const double pi = 3.14159265358979323846;
  auto fill = [&](size_t tw0, size_t pw0, int L) {
    const int nc = (L + TW_FINE - 1) / TW_FINE;
    for (int h = 0; h < nc; ++h)
      t[tw0 + h] = Cx<R>{(R)std::cos(2.0 * pi * TW_FINE * h / L), (R)(-std::sin(2.0 * pi * TW_FINE * h / L))};
    for (int l = 0; l < TW_FINE; ++l)
      t[tw0 + nc + l] = Cx<R>{(R)std::cos(2.0 * pi * l / L), (R)(-std::sin(2.0 * pi * l / L))};
    for (int k = 0; k <= L; ++k) t[pw0 + k] = Cx<R>{(R)std::cos(pi * k / L), (R)(-std::sin(pi * k / L))};
  };
  fill(d->off_twx, d->off_pwx, Lx);
  fill(d->off_twy, d->off_pwy, Ly);
  R* lam = reinterpret_cast<R*>(t.data() + d->off_lam);
  for (int k = 1; k <= d->Nx; ++k) lam[k - 1] = (R)(-(2.0 - 2.0 * std::cos(pi * k / Lx)) / (d->dx * d->dx));
  for (int l = 1; l <= d->Ny; ++l) lam[d->Nx + l - 1] = (R)(-(2.0 - 2.0 * std::cos(pi * l / Ly)) / (d->dy * d->dy));
  const size_t tb = sizeof(R) * (size_t)d->Nx * d->Ny;
  if (cudaMalloc(&d->T1, tb) != cudaSuccess || cudaMalloc(&d->T2, tb) != cudaSuccess ||
      cudaMalloc(&d->tab, sizeof(Cx<R>) * t.size()) != cudaSuccess)
    return -1;
  if (cudaMemcpy(d->tab, t.data(), sizeof(Cx<R>) * t.size(), cudaMemcpyHostToDevice) != cudaSuccess) return -1;
  return 0;
}

// The Dirichlet box along an axis of N interior sites: the smallest N' >= N whose
// N' + 1 has no prime factor above 7 (the line transform of length N' + 1 then runs
// in stages of radix 4, 2, 3, 5, 7; a length with a large prime factor, as
// 4092 + 1 = 4093, has no such factoring), and floor((N' - N) / 2) of the extra sites
// below I.
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
  cudaFree(d->T1);
  cudaFree(d->T2);
  cudaFree(d->tab);
  delete d;
}

cudaError_t demag_solve(DemagSolver* d, const DevState* st, void* const phi[2], void* const lo[2], void* const psi[2],
                        cudaStream_t s) {
  return d->prec == PREC_F64 ? solve_t<double>(d, st, phi, lo, psi, s) : solve_t<float>(d, st, phi, lo, psi, s);
}

}  // namespace ss
