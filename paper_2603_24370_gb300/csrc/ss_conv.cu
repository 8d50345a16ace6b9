// ss_conv.cu -- tensor-core 3x3 convolutions of the learned initialiser (tcgen05,
// TMA, TMEM), BF16 operands with FP32 accumulation.
//
// Forward and input-gradient convolutions are implicit GEMMs: one CTA computes a
// 128-pixel x Cout output tile, M = pixels, N = output channels, K = 9 taps x input
// channels in groups of 8. For each K-group the TMA loads a box of 8 channels x 128
// pixels straight from the NHWC activation at the tap's shifted coordinates; the
// tensor-map bounds supply the zero padding, so no im2col copy is ever written. The
// matching 8-wide slice of the weights ([Cout][9 Cin], K contiguous) is a second box.
// Both land in the K-major no-swizzle layout that tcgen05.mma reads directly.
//
// The weight gradient contracts over pixels: M = output channels, N = input channels
// of one tap, K = pixels. Its operands are channel-major copies (made by the
// memory-bound kernels) so that K is contiguous; the tap's row shift is a TMA
// coordinate and its column shift selects one of three pre-shifted copies.
//
// The convolution kernel is persistent with three warp roles (see k_conv3x3_p); the
// weight gradient uses one CTA per (tap, pixel range): warp 0 allocates TMEM and
// lane 0 drives the TMA pipeline, warp 1 lane 0 issues the MMAs, then all four warps
// drain the accumulator (warp w owns TMEM lanes 32w..32w+31, one row per thread).
// Every mbarrier wait is bounded: on time-out the kernel records the failure in
// `err`, waits (bounded) for its copies in flight, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "ss_net_internal.h"
#include "ss_umma.cuh"

namespace ss {
namespace {

using namespace umma;

constexpr int BM = 128;     // tile rows (pixels, or output channels for the weight gradient)
constexpr int GPS = 8;      // K-groups of 8 values per pipeline stage (BK = 64)
constexpr int STAGES = 3;
constexpr uint64_t WAIT_NS = 2000000000ull;  // 2 s per wait

__host__ __device__ constexpr int tmem_cols(int bn) { return bn <= 32 ? 32 : bn <= 64 ? 64 : bn <= 128 ? 128 : 256; }
template <int BN>
__host__ __device__ constexpr int stage_bytes() {
  return GPS * (BM + BN) * 16;
}
// Dynamic shared memory: the stages and 1 KB for aligning the base. The MMA reads
// of a stage stay inside it: A spans 16 row groups x SBO 128 B plus K-groups at
// LBO 2048 B, B likewise with LBO = BN * 16 B.
template <int BN>
constexpr size_t conv_smem() {
  return (size_t)STAGES * stage_bytes<BN>() + 1024;
}

struct ConvArgs {
  int N, H, W, Cin, Cout;
  int mode;
  const float* bias;
  void* out;
  int out_cs, out_coff;
  int* err;
  // CONV_GRAD_RELU
  const __nv_bfloat16* mask;
  int mask_cs, mask_off;
  __nv_bfloat16* dyT;
  float* dbias;
  long long P;
};

struct WgradArgs {
  int N, H, W, Cout, Cin;
  int groups_per_cta;  // K-groups (8 pixels each) per CTA, even
  int total_groups;
  float* dw;
  int* err;
};

__device__ __forceinline__ void record_fail(int* err, int code) { atomicCAS(err, 0, code); }

// The producer's last wait: every TMA it issued has landed (bounded).
__device__ __forceinline__ void drain_stages(uint64_t* full, int issued) {
  for (int s = 0; s < STAGES && s < issued; ++s) {
    const int last = s + STAGES * ((issued - 1 - s) / STAGES);
    mbar_wait(&full[s], (uint32_t)((last / STAGES) & 1), WAIT_NS);
  }
}

// ---------------------------------------------------------------- persistent conv
// The same implicit GEMM, persistent: each CTA walks tiles blockIdx.x, +gridDim.x,
// ... with three roles (192 threads): warp 0 lane 0 streams the activation boxes
// (and, once, the whole weight matrix when it fits in shared memory) through a
// STAGES-deep ring; warp 1 lane 0 issues the MMAs into one of two TMEM
// accumulators; warps 2..5 drain the other accumulator into the epilogue, so a
// tile's epilogue overlaps the next tile's MMAs. TMEM lanes: warp w reads the
// quarter w % 4. Every wait is bounded (2 s); on time-out the roles stop, the
// failure is recorded in `err`, TMEM is freed and the kernel returns.
constexpr int P_STAGES = 4;
constexpr int W_RESIDENT_MAX = 64 * 1024;  // weight bytes kept in shared memory

__host__ __device__ constexpr int ptcols(int bn) {
  return 2 * bn <= 32 ? 32 : 2 * bn <= 64 ? 64 : 2 * bn <= 128 ? 128 : 2 * bn <= 256 ? 256 : 512;
}

struct PConvArgs {
  ConvArgs c;
  int tiles;
  int resident;  // 1: all weight groups in shared memory, loaded once
  int wbytes;    // BN * K * 2
  int halo;      // 1: halo staging (rows of at least 128 pixels), 2: row-halo staging
                 // (narrower rows); both with resident weights
};

// Halo staging. For rows of at least 128 pixels a tile is 128 pixels of one image row.
// Per pair of 8-channel groups, two TMA boxes of {8 channels, 130 pixels, 3 rows}
// (the tile's pixels, one more on each side, the rows above and below; zero outside
// the image) hold every input the tile's nine taps read. In a box, pixel x of row r
// sits at r * HROW + x * 16 bytes, so the A operand of tap (dy, dx) is the box read
// from byte dy * HROW + dx * 16 on: 128 rows at a 16-byte pitch, the K-major
// no-swizzle layout with the K-adjacent group in the pair's other box (LBO = HSLOT).
// Against one box per tap and group this moves a third of the bytes from L2.
#ifndef SS_CONV_RHALO
#define SS_CONV_RHALO 1
#endif
constexpr int HROW = 130 * 16;   // one row of a halo box
constexpr int HBOX = 3 * HROW;   // box bytes: 6240
constexpr int HSLOT = 49 * 128;  // a box's slot, 128-byte aligned: 6272

// Row-halo staging, for rows narrower than 128 pixels (a tile is 128 / W whole image
// rows). A shift along x would carry a tile row's last pixel into the next row, so
// each column shift dx gets its own box {8 channels, W pixels, rows + 2} starting at
// x = dx - 1 (zero outside the image), and the row shift dy is the start offset
// dy * W * 16 bytes inside it: 128 rows at a 16-byte pitch again. Per pair of channel
// groups six boxes, [group][dx], hold the nine taps (LBO = three boxes).
__host__ __device__ inline int rbox_bytes(int W) { return ((128 / W + 2) * W * 16 + 127) & ~127; }

template <int BN>
__global__ void __launch_bounds__(192) k_conv3x3_p(const __grid_constant__ CUtensorMap mx,
                                                   const __grid_constant__ CUtensorMap mw, const PConvArgs pa) {
  extern __shared__ unsigned char smraw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  const ConvArgs& a = pa.c;
  constexpr int A_BYTES = GPS * BM * 16;
  constexpr int TCOLS = ptcols(BN);
  const bool resident = pa.resident != 0;
  const bool halo = pa.halo == 1, rhalo = pa.halo == 2;  // both imply resident
  const int RB = rhalo ? rbox_bytes(a.W) : 0;
  const int stage = halo ? 2 * HSLOT : rhalo ? 6 * RB : A_BYTES + (resident ? 0 : GPS * BN * 16);
  unsigned char* wsm = smem + P_STAGES * stage;  // resident weights: group g at g * BN * 16
  __shared__ __align__(8) uint64_t full[P_STAGES], empty[P_STAGES], tfull[2], tempty[2], wbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  __shared__ float sbias[BN];  // CONV_GRAD_RELU: this CTA's per-channel sums
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = threadIdx.x; c < BN; c += blockDim.x) sbias[c] = 0.f;

  const int W = a.W, H = a.H;
  const int Wt = W < BM ? W : BM;
  const int rows = BM / Wt;
  const int tpr = W / Wt;
  const int tpi = (H / rows) * tpr;
  const int cg = a.Cin >> 3;
  const int G = 9 * cg;
  const int nkb = (halo || rhalo) ? cg / 2 : (G + GPS - 1) / GPS;  // ring entries per tile

  if (threadIdx.x == 0) {
    for (int s = 0; s < P_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    mbar_init(&wbar, 1);
    s_fail = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base, TCOLS);
    tmem_relinquish();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    if (lane == 0) {  // ---- producer
      if (resident) {
        mbar_arrive_expect_tx(&wbar, (uint32_t)(G * BN * 16));
        for (int g = 0; g < G; ++g) tma_load_2d(wsm + g * (BN * 16), &mw, &wbar, g * 8, 0);
      }
      int q = 0;  // k-blocks issued so far (ring position)
      for (int t = blockIdx.x; t < pa.tiles && !*static_cast<volatile int*>(&s_fail); t += gridDim.x) {
        const int n = t / tpi, r = t % tpi;
        const int y0 = (r / tpr) * rows, x0 = (r % tpr) * Wt;
        for (int kb = 0; kb < nkb; ++kb, ++q) {
          const int s = q % P_STAGES;
          if (!mbar_wait(&empty[s], (uint32_t)(((q / P_STAGES) & 1) ^ 1), WAIT_NS)) {
            record_fail(a.err, 21);
            s_fail = 1;
            break;
          }
          unsigned char* sa = smem + s * stage;
          if (halo) {  // channel groups 2 kb and 2 kb + 1, every tap
            mbar_arrive_expect_tx(&full[s], (uint32_t)(2 * HBOX));
            tma_load_4d(sa, &mx, &full[s], 16 * kb, x0 - 1, y0 - 1, n);
            tma_load_4d(sa + HSLOT, &mx, &full[s], 16 * kb + 8, x0 - 1, y0 - 1, n);
            continue;
          }
          if (rhalo) {  // channel groups 2 kb and 2 kb + 1, one box per column shift
            mbar_arrive_expect_tx(&full[s], (uint32_t)(6 * (rows + 2) * Wt * 16));
            for (int gi = 0; gi < 2; ++gi)
              for (int dxi = 0; dxi < 3; ++dxi)
                tma_load_4d(sa + (gi * 3 + dxi) * RB, &mx, &full[s], 16 * kb + 8 * gi, x0 + dxi - 1, y0 - 1, n);
            continue;
          }
          unsigned char* sb = sa + A_BYTES;
          const int g0 = kb * GPS, ng = min(GPS, G - g0);
          mbar_arrive_expect_tx(&full[s], (uint32_t)(ng * (BM + (resident ? 0 : BN)) * 16));
          for (int j = 0; j < ng; ++j) {
            const int gg = g0 + j, tap = gg / cg, c0 = (gg - tap * cg) * 8;
            tma_load_4d(sa + j * (BM * 16), &mx, &full[s], c0, x0 + tap % 3 - 1, y0 + tap / 3 - 1, n);
            if (!resident) tma_load_2d(sb + j * (BN * 16), &mw, &full[s], gg * 8, 0);
          }
        }
      }
      // every issued copy has landed before the CTA may end (bounded)
      for (int s = 0; s < P_STAGES && s < q; ++s) {
        const int last = s + P_STAGES * ((q - 1 - s) / P_STAGES);
        mbar_wait(&full[s], (uint32_t)((last / P_STAGES) & 1), WAIT_NS);
      }
      if (resident) mbar_wait(&wbar, 0, WAIT_NS);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer
      constexpr uint32_t idesc = idesc_bf16(BM, BN);
      bool ok = !resident || mbar_wait(&wbar, 0, WAIT_NS);
      if (!ok) {
        record_fail(a.err, 22);
        s_fail = 1;
      }
      const uint32_t wbase = smem_u32(wsm);
      int q = 0, it = 0;
      for (int t = blockIdx.x; ok && t < pa.tiles && !*static_cast<volatile int*>(&s_fail); t += gridDim.x, ++it) {
        const int b = it & 1;
        if (!mbar_wait(&tempty[b], (uint32_t)(((it >> 1) & 1) ^ 1), WAIT_NS)) {
          record_fail(a.err, 23);
          s_fail = 1;
          break;
        }
        fence_after_sync();
        const uint32_t acc = tmem + (uint32_t)(b * BN);
        for (int kb = 0; kb < nkb; ++kb, ++q) {
          const int s = q % P_STAGES;
          if (!mbar_wait(&full[s], (uint32_t)((q / P_STAGES) & 1), WAIT_NS)) {
            record_fail(a.err, 24);
            s_fail = 1;
            ok = false;
            break;
          }
          fence_after_sync();
          const uint32_t sa = smem_u32(smem + s * stage), sb = sa + A_BYTES;
          if (rhalo) {
            for (int tap = 0; tap < 9; ++tap) {
              const uint64_t ad =
                  sdesc(sa + (uint32_t)((tap % 3) * RB + (tap / 3) * Wt * 16), (uint32_t)(3 * RB), 128);
              const uint64_t bd = sdesc(wbase + (uint32_t)((tap * cg + 2 * kb) * (BN * 16)), BN * 16, 128);
              mma_bf16(acc, ad, bd, idesc, (kb > 0 || tap > 0) ? 1u : 0u);
            }
            mma_commit(&empty[s]);
            continue;
          }
          if (halo) {
            for (int tap = 0; tap < 9; ++tap) {
              const uint64_t ad = sdesc(sa + (uint32_t)((tap / 3) * HROW + (tap % 3) * 16), HSLOT, 128);
              const uint64_t bd = sdesc(wbase + (uint32_t)((tap * cg + 2 * kb) * (BN * 16)), BN * 16, 128);
              mma_bf16(acc, ad, bd, idesc, (kb > 0 || tap > 0) ? 1u : 0u);
            }
            mma_commit(&empty[s]);
            continue;
          }
          const int g0 = kb * GPS, ng = min(GPS, G - g0);
          for (int j = 0; j < ng; j += 2) {
            const uint64_t ad = sdesc(sa + j * (BM * 16), BM * 16, 128);
            const uint64_t bd = resident ? sdesc(wbase + (g0 + j) * (BN * 16), BN * 16, 128)
                                         : sdesc(sb + j * (BN * 16), BN * 16, 128);
            mma_bf16(acc, ad, bd, idesc, (kb > 0 || j > 0) ? 1u : 0u);
          }
          mma_commit(&empty[s]);
        }
        mma_commit(&tfull[b]);
      }
    }
  } else {
    // ---- epilogue warps 2..5: TMEM lane quarter warp % 4
    const int qd = warp & 3;
    const int m = qd * 32 + lane;
    int it = 0;
    for (int t = blockIdx.x; t < pa.tiles; t += gridDim.x, ++it) {
      const int b = it & 1;
      bool ok = mbar_wait(&tfull[b], (uint32_t)((it >> 1) & 1), WAIT_NS);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) {
          record_fail(a.err, 25);
          s_fail = 1;
        }
        break;
      }
      fence_after_sync();
      const int n = t / tpi, r = t % tpi;
      const int y0 = (r / tpr) * rows, x0 = (r % tpr) * Wt;
      const int yy = y0 + m / Wt, xx = x0 + m % Wt;
      const size_t pix = ((size_t)n * H + yy) * W + xx;
      const uint32_t trow = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(b * BN);
#pragma unroll 1
      for (int c = 0; c < BN; c += 16) {
        float v[16];
        tmem_ld16(trow + (uint32_t)c, v);
        if (c >= a.Cout) continue;
        if (a.mode == CONV_GRAD_RELU) {
          // the previous layer's ReLU: its BF16 output at this pixel masks the gradient
          const uint4* mk = reinterpret_cast<const uint4*>(a.mask + pix * a.mask_cs + a.mask_off + c);
          const uint4 mq[2] = {mk[0], mk[1]};
          const __nv_bfloat16* mb = reinterpret_cast<const __nv_bfloat16*>(mq);
          uint32_t w[8];
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (!(__bfloat162float(mb[i]) > 0.f)) v[i] = 0.f;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
            w[i] = *reinterpret_cast<uint32_t*>(&b2);
          }
          uint4* o4 = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(a.out) + pix * a.out_cs + a.out_coff + c);
          o4[0] = make_uint4(w[0], w[1], w[2], w[3]);
          o4[1] = make_uint4(w[4], w[5], w[6], w[7]);
          const __nv_bfloat16* wb = reinterpret_cast<const __nv_bfloat16*>(w);
#pragma unroll
          for (int i = 0; i < 16; ++i) {  // channel-major: a warp's 32 pixels are consecutive
            a.dyT[(size_t)(c + i) * a.P + pix] = wb[i];
            float sum = v[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane == 0) atomicAdd(&sbias[c + i], sum);
          }
          continue;
        }
        if (a.mode == CONV_BF16_BIAS_RELU) {
          __nv_bfloat16* o = static_cast<__nv_bfloat16*>(a.out) + pix * a.out_cs + a.out_coff + c;
          uint32_t w[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float lo = fmaxf(v[2 * i] + __ldg(a.bias + c + 2 * i), 0.f);
            const float hi = fmaxf(v[2 * i + 1] + __ldg(a.bias + c + 2 * i + 1), 0.f);
            __nv_bfloat162 b2 = __floats2bfloat162_rn(lo, hi);
            w[i] = *reinterpret_cast<uint32_t*>(&b2);
          }
          uint4* o4 = reinterpret_cast<uint4*>(o);
          o4[0] = make_uint4(w[0], w[1], w[2], w[3]);
          o4[1] = make_uint4(w[4], w[5], w[6], w[7]);
        } else {
          float* o = static_cast<float*>(a.out) + pix * a.out_cs + a.out_coff + c;
          const bool bb = a.mode == CONV_F32_BIAS;
#pragma unroll
          for (int i = 0; i < 16; i += 4) {
            float4 qv;
            qv.x = v[i] + (bb ? __ldg(a.bias + c + i) : 0.f);
            qv.y = v[i + 1] + (bb ? __ldg(a.bias + c + i + 1) : 0.f);
            qv.z = v[i + 2] + (bb ? __ldg(a.bias + c + i + 2) : 0.f);
            qv.w = v[i + 3] + (bb ? __ldg(a.bias + c + i + 3) : 0.f);
            *reinterpret_cast<float4*>(o + i) = qv;
          }
        }
      }
      // the accumulator is read: hand it back to the MMA issuer
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
    }
  }
  fence_before_sync();
  __syncthreads();
  if (a.mode == CONV_GRAD_RELU)
    for (int c = threadIdx.x; c < a.Cout; c += blockDim.x) atomicAdd(a.dbias + c, sbias[c]);
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tmem, TCOLS);
  }
}

// ---------------------------------------------------------------- weight gradient
template <int BN>
__global__ void __launch_bounds__(128) k_wgrad3x3(const __grid_constant__ CUtensorMap mdy,
                                                  const __grid_constant__ CUtensorMap mx0,
                                                  const __grid_constant__ CUtensorMap mx1,
                                                  const __grid_constant__ CUtensorMap mx2, const WgradArgs a) {
  extern __shared__ unsigned char smraw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  constexpr int A_BYTES = GPS * BM * 16;
  constexpr int STAGE = stage_bytes<BN>();
  constexpr int TCOLS = tmem_cols(BN);
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], accum;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  const int tap = blockIdx.y, dy = tap / 3 - 1, dx = tap % 3 - 1;
  const CUtensorMap* mx = dx < 0 ? &mx0 : (dx == 0 ? &mx1 : &mx2);
  const int q0 = blockIdx.x * a.groups_per_cta;
  const int q1 = min(q0 + a.groups_per_cta, a.total_groups);
  const int G = q1 - q0;
  const int nkb = G > 0 ? (G + GPS - 1) / GPS : 0;
  const int HW = a.H * a.W;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&accum, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base, TCOLS);
    tmem_relinquish();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    int issued = 0;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(&empty[s], (uint32_t)(((kb / STAGES) & 1) ^ 1), WAIT_NS)) {
        record_fail(a.err, 11);
        break;
      }
      unsigned char* sa = smem + s * STAGE;
      unsigned char* sb = sa + A_BYTES;
      const int g0 = q0 + kb * GPS, ng = min(GPS, q1 - g0);
      mbar_arrive_expect_tx(&full[s], (uint32_t)(ng * (BM + BN) * 16));
      for (int j = 0; j < ng; ++j) {
        const int p = (g0 + j) * 8;
        const int nn = p / HW, rem = p - nn * HW;
        const int y = rem / a.W, x = rem - y * a.W;
        tma_load_4d(sa + j * (BM * 16), &mdy, &full[s], x, y, nn, 0);
        tma_load_4d(sb + j * (BN * 16), mx, &full[s], x, y + dy, nn, 0);
      }
      issued = kb + 1;
    }
    drain_stages(full, issued);
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(&full[s], (uint32_t)((kb / STAGES) & 1), WAIT_NS)) {
        record_fail(a.err, 12);
        break;
      }
      fence_after_sync();
      const uint32_t sa = smem_u32(smem + s * STAGE), sb = sa + A_BYTES;
      const int ng = min(GPS, q1 - (q0 + kb * GPS));
      for (int j = 0; j < ng; j += 2) {
        const uint64_t ad = sdesc(sa + j * (BM * 16), BM * 16, 128);
        const uint64_t bd = sdesc(sb + j * (BN * 16), BN * 16, 128);
        mma_bf16(tmem, ad, bd, idesc, (kb > 0 || j > 0) ? 1u : 0u);
      }
      mma_commit(&empty[s]);
    }
    mma_commit(&accum);
  }
  __syncwarp();

  bool ok = nkb > 0 ? mbar_wait(&accum, 0, WAIT_NS) : false;
  ok = __all_sync(0xffffffffu, ok);
  fence_after_sync();
  if (!ok) {
    if (lane == 0 && nkb > 0) record_fail(a.err, 13);
  } else {
    const int co = warp * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c = 0; c < BN; c += 16) {
      float v[16];
      tmem_ld16(trow + (uint32_t)c, v);
      if (co < a.Cout) {
        float* d = a.dw + ((size_t)co * 9 + tap) * a.Cin + c;
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (c + i < a.Cin) atomicAdd(d + i, v[i]);
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tmem, TCOLS);
  }
}


// ---------------------------------------------------------------- weight gradient, 64-pixel K-blocks
// For rows of at least 64 pixels: each K-block is 64 consecutive pixels of one image
// row, fetched as one 128-byte-swizzled TMA box per operand (the output gradient,
// M = 128 rows of output channels, zero beyond Cout; and the shifted input of each
// tap, N = Cin rows). With 9 Cin <= 512 TMEM columns one CTA accumulates all nine
// taps (TPC = 9), so the output-gradient tile is loaded once per K-block.
struct WgSwArgs {
  int N, H, W, Cout, Cin;
  int kb_per_cta, total_kb;
  int stages;
  float* dw;
  int* err;
};

template <int BN, int TPC>
__global__ void __launch_bounds__(128) k_wgrad_sw(const __grid_constant__ CUtensorMap mdy,
                                                  const __grid_constant__ CUtensorMap mx0,
                                                  const __grid_constant__ CUtensorMap mx1,
                                                  const __grid_constant__ CUtensorMap mx2, const WgSwArgs a) {
  extern __shared__ unsigned char smraw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  constexpr int A_BYTES = BM * 128;
  constexpr int B_BYTES = BN * 128;
  constexpr int STAGE = A_BYTES + TPC * B_BYTES;
  constexpr int NCOL = TPC * BN;
  constexpr int TCOLS = NCOL <= 32 ? 32 : NCOL <= 64 ? 64 : NCOL <= 128 ? 128 : NCOL <= 256 ? 256 : 512;
  constexpr int MAXS = 4;
  __shared__ __align__(8) uint64_t full[MAXS], empty[MAXS], accum;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S = a.stages;
  const int tap0 = blockIdx.y * TPC;
  const int kb0 = blockIdx.x * a.kb_per_cta;
  const int kb1 = min(kb0 + a.kb_per_cta, a.total_kb);
  const int nkb = kb1 > kb0 ? kb1 - kb0 : 0;
  const int HW = a.H * a.W;

  if (threadIdx.x == 0) {
    for (int s = 0; s < MAXS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&accum, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base, TCOLS);
    tmem_relinquish();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    int issued = 0;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % S;
      if (!mbar_wait(&empty[s], (uint32_t)(((i / S) & 1) ^ 1), WAIT_NS)) {
        record_fail(a.err, 31);
        break;
      }
      unsigned char* sa = smem + s * STAGE;
      const int p0 = (kb0 + i) * 64;
      const int n = p0 / HW, rem = p0 - n * HW;
      const int y = rem / a.W, x = rem - y * a.W;
      mbar_arrive_expect_tx(&full[s], (uint32_t)STAGE);
      tma_load_4d(sa, &mdy, &full[s], x, y, n, 0);
#pragma unroll
      for (int j = 0; j < TPC; ++j) {
        const int tap = tap0 + j, dy = tap / 3 - 1, dx = tap % 3 - 1;
        const CUtensorMap* mx = dx < 0 ? &mx0 : (dx == 0 ? &mx1 : &mx2);
        tma_load_4d(sa + A_BYTES + j * B_BYTES, mx, &full[s], x, y + dy, n, 0);
      }
      issued = i + 1;
    }
    for (int s = 0; s < S && s < issued; ++s) {
      const int last = s + S * ((issued - 1 - s) / S);
      mbar_wait(&full[s], (uint32_t)((last / S) & 1), WAIT_NS);
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    for (int i = 0; i < nkb; ++i) {
      const int s = i % S;
      if (!mbar_wait(&full[s], (uint32_t)((i / S) & 1), WAIT_NS)) {
        record_fail(a.err, 32);
        break;
      }
      fence_after_sync();
      const uint32_t sa = smem_u32(smem + s * STAGE);
#pragma unroll
      for (int j = 0; j < TPC; ++j) {
        const uint32_t sb = sa + A_BYTES + j * B_BYTES;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma_bf16(tmem + (uint32_t)(j * BN), sdesc_sw128(sa + kk * 32), sdesc_sw128(sb + kk * 32), idesc,
                   (i > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(&empty[s]);
    }
    mma_commit(&accum);
  }
  __syncwarp();

  bool ok = nkb > 0 ? mbar_wait(&accum, 0, WAIT_NS) : false;
  ok = __all_sync(0xffffffffu, ok);
  fence_after_sync();
  if (!ok) {
    if (lane == 0 && nkb > 0) record_fail(a.err, 33);
  } else {
    const int co = warp * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int j = 0; j < TPC; ++j) {
#pragma unroll 1
      for (int c = 0; c < BN; c += 16) {
        float v[16];
        tmem_ld16(trow + (uint32_t)(j * BN + c), v);
        if (co < a.Cout) {  // 16-byte vector atomics (dw rows are 16-byte aligned: Cin % 16 == 0)
          float4* d = reinterpret_cast<float4*>(a.dw + ((size_t)co * 9 + tap0 + j) * a.Cin + c);
#pragma unroll
          for (int q = 0; q < 4; ++q) atomicAdd(d + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
        }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tmem, TCOLS);
  }
}

// ---------------------------------------------------------------- weight gradient, tap rows
// For rows of at least 64 pixels and 9 Cin <= 512: the M rows of the contraction are
// the (tap, input channel) pairs, N the output channels, K 64 pixels of one image row
// per K-block. The nine shifted input boxes of a K-block ({64 pixels, Cin channels}
// each, 128-byte swizzle) are stacked, so rows 128 g .. 128 g + 127 of the stack are
// the A operand of accumulator g; the last accumulator runs past the stack into bytes
// whose products land in TMEM rows that are never read (the allocation is padded so
// those reads stay inside it). The output-gradient box ({64 pixels, Cout channels}) is
// B. Against one 128-row tile of output channels per tap (k_wgrad_sw) this issues
// ceil(9 Cin / 128) instead of nine MMAs per K step and loads no zero rows.
// The nine shifted input boxes of a K-block as three boxes of three rows each, one per
// column shift (1), or one box per tap (0).
#ifndef SS_WG_ROWS3
#define SS_WG_ROWS3 1
#endif
struct WgRowArgs {
  int N, H, W, Cout, Cin;
  int kb_per_cta, total_kb;
  int stages, groups, stage_bytes, tcols;
  float* dw;
  int* err;
};

template <int BN>
__global__ void __launch_bounds__(128) k_wgrad_rows(const __grid_constant__ CUtensorMap mdy,
                                                    const __grid_constant__ CUtensorMap mx0,
                                                    const __grid_constant__ CUtensorMap mx1,
                                                    const __grid_constant__ CUtensorMap mx2, const WgRowArgs a) {
  extern __shared__ unsigned char smraw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  constexpr int MAXS = 4;
  __shared__ __align__(8) uint64_t full[MAXS], empty[MAXS], accum;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S = a.stages, G = a.groups, STAGE = a.stage_bytes;
  const int Cin = a.Cin, XB = Cin * 128;  // one tap's box
  const int A_BYTES = 9 * XB;             // a multiple of 1 KB (Cin % 16 == 0)
  const int kb0 = blockIdx.x * a.kb_per_cta;
  const int kb1 = min(kb0 + a.kb_per_cta, a.total_kb);
  const int nkb = kb1 > kb0 ? kb1 - kb0 : 0;
  const int HW = a.H * a.W;

  if (threadIdx.x == 0) {
    for (int s = 0; s < MAXS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&accum, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base, (uint32_t)a.tcols);
    tmem_relinquish();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {  // ---- producer
    int issued = 0;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % S;
      if (!mbar_wait(&empty[s], (uint32_t)(((i / S) & 1) ^ 1), WAIT_NS)) {
        record_fail(a.err, 41);
        break;
      }
      unsigned char* sa = smem + s * STAGE;
      const int p0 = (kb0 + i) * 64;
      const int n = p0 / HW, rem = p0 - n * HW;
      const int y = rem / a.W, x = rem - y * a.W;
      mbar_arrive_expect_tx(&full[s], (uint32_t)(A_BYTES + BN * 128));
      if (SS_WG_ROWS3) {  // per column shift one box of rows y - 1 .. y + 1: stack row (dx, ci, dy)
        tma_load_4d(sa, &mx0, &full[s], x, y - 1, n, 0);
        tma_load_4d(sa + 3 * XB, &mx1, &full[s], x, y - 1, n, 0);
        tma_load_4d(sa + 6 * XB, &mx2, &full[s], x, y - 1, n, 0);
      } else {  // one box per tap: stack row (tap, ci)
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
          const int dy = tap / 3 - 1, dx = tap % 3 - 1;
          const CUtensorMap* mx = dx < 0 ? &mx0 : (dx == 0 ? &mx1 : &mx2);
          tma_load_4d(sa + tap * XB, mx, &full[s], x, y + dy, n, 0);
        }
      }
      tma_load_4d(sa + A_BYTES, &mdy, &full[s], x, y, n, 0);
      issued = i + 1;
    }
    for (int s = 0; s < S && s < issued; ++s) {
      const int last = s + S * ((issued - 1 - s) / S);
      mbar_wait(&full[s], (uint32_t)((last / S) & 1), WAIT_NS);
    }
  } else if (warp == 1 && lane == 0) {  // ---- MMA issuer
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    for (int i = 0; i < nkb; ++i) {
      const int s = i % S;
      if (!mbar_wait(&full[s], (uint32_t)((i / S) & 1), WAIT_NS)) {
        record_fail(a.err, 42);
        break;
      }
      fence_after_sync();
      const uint32_t sa = smem_u32(smem + s * STAGE), sb = sa + (uint32_t)A_BYTES;
      for (int g = 0; g < G; ++g) {
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma_bf16(tmem + (uint32_t)(g * BN), sdesc_sw128(sa + (uint32_t)(g * BM * 128 + kk * 32)),
                   sdesc_sw128(sb + kk * 32), idesc, (i > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(&empty[s]);
    }
    mma_commit(&accum);
  }
  __syncwarp();

  bool ok = nkb > 0 ? mbar_wait(&accum, 0, WAIT_NS) : false;
  ok = __all_sync(0xffffffffu, ok);
  fence_after_sync();
  if (!ok) {
    if (lane == 0 && nkb > 0) record_fail(a.err, 43);
  } else {
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int g = 0; g < G; ++g) {
      const int r = g * BM + warp * 32 + lane;  // stack row
      int tap, ci;
      if (SS_WG_ROWS3) {  // (column shift, input channel, row shift)
        const int dxi = r / (3 * Cin), rem = r - dxi * 3 * Cin;
        ci = rem / 3;
        tap = (rem - 3 * ci) * 3 + dxi;
      } else {  // (tap, input channel)
        tap = r / Cin;
        ci = r - tap * Cin;
      }
#pragma unroll 1
      for (int c = 0; c < BN; c += 16) {
        float v[16];
        tmem_ld16(trow + (uint32_t)(g * BN + c), v);
        if (r < 9 * Cin) {
          float* d = a.dw + (size_t)tap * Cin + ci;
#pragma unroll
          for (int q = 0; q < 16; ++q) atomicAdd(d + (size_t)(c + q) * 9 * Cin, v[q]);
        }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tmem, (uint32_t)a.tcols);
  }
}

template <int BN>
cudaError_t wgrad_rows_launch(const CUtensorMap& mdy, const CUtensorMap* mx, WgRowArgs a, cudaStream_t s) {
  const int A_BYTES = 9 * a.Cin * 128;
  a.groups = (9 * a.Cin + BM - 1) / BM;
  a.stage_bytes = A_BYTES + BN * 128;  // a multiple of 1 KB
  int cols = a.groups * BN;
  a.tcols = cols <= 32 ? 32 : cols <= 64 ? 64 : cols <= 128 ? 128 : cols <= 256 ? 256 : 512;
  int stages = (100 * 1024) / a.stage_bytes;
  stages = stages < 2 ? 2 : (stages > 4 ? 4 : stages);
  a.stages = stages;
  // the last accumulator's A rows run up to groups x 16 KB past the last stage's start
  const int over = a.groups * BM * 128 - a.stage_bytes;
  const size_t smem = (size_t)stages * a.stage_bytes + (over > 0 ? over : 0) + 1024;
  static int max_smem_set = 0;
  if ((int)smem > max_smem_set) {
    cudaError_t e = cudaFuncSetAttribute(k_wgrad_rows<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    max_smem_set = (int)smem;
  }
  int dev = 0, nsm = 0, sm_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  int per_sm = sm_smem / (int)(smem + 1024);
  if (per_sm > 512 / a.tcols) per_sm = 512 / a.tcols;
  if (per_sm > 2) per_sm = 2;
  if (per_sm < 1) per_sm = 1;
  int splits = nsm * per_sm;
  a.kb_per_cta = (a.total_kb + splits - 1) / splits;
  if (a.kb_per_cta < 4) a.kb_per_cta = 4;
  splits = (a.total_kb + a.kb_per_cta - 1) / a.kb_per_cta;
  k_wgrad_rows<BN><<<splits, 128, smem, s>>>(mdy, mx[0], mx[1], mx[2], a);
  return cudaGetLastError();
}

template <int BN, int TPC>
cudaError_t wgrad_sw_launch(const CUtensorMap& mdy, const CUtensorMap* mx, WgSwArgs a, cudaStream_t s) {
  constexpr int STAGE = BM * 128 + TPC * BN * 128;
  int stages = (110 * 1024) / STAGE;
  stages = stages < 2 ? 2 : (stages > 4 ? 4 : stages);
  a.stages = stages;
  const size_t smem = (size_t)stages * STAGE + 1024;
  static int max_smem_set = 0;
  if ((int)smem > max_smem_set) {
    cudaError_t e = cudaFuncSetAttribute(k_wgrad_sw<BN, TPC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    max_smem_set = (int)smem;
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int ytaps = 9 / TPC;
  // one wave: every CTA adds its partial sums once, so fewer, longer CTAs also mean
  // fewer atomics on the same weight-gradient entries
  int splits = (nsm + ytaps - 1) / ytaps;
  a.kb_per_cta = (a.total_kb + splits - 1) / splits;
  if (a.kb_per_cta < 4) a.kb_per_cta = 4;
  splits = (a.total_kb + a.kb_per_cta - 1) / a.kb_per_cta;
  k_wgrad_sw<BN, TPC><<<dim3(splits, ytaps), 128, smem, s>>>(mdy, mx[0], mx[1], mx[2], a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- tensor maps
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// BF16 tensor map of rank r: dims[0] innermost (elements), strides in bytes for
// dims 1..r-1, box per dim; out-of-bounds elements read as zero.
cudaError_t make_map(CUtensorMap* m, const void* base, int r, const cuuint64_t* dims, const cuuint64_t* strides,
                     const cuuint32_t* box, bool swizzle128 = false) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  const CUresult rc = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)r, const_cast<void*>(base), dims, strides,
                         box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return rc == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN>
cudaError_t conv_launch_p(const CUtensorMap& mx, const CUtensorMap* mxh, const CUtensorMap& mw, const ConvArgs& a,
                          int tiles, int K, cudaStream_t s) {
  PConvArgs pa{a, tiles, 0, BN * K * 2, 0};
  pa.resident = pa.wbytes <= W_RESIDENT_MAX ? 1 : 0;
  pa.halo = (mxh != nullptr && pa.resident) ? (a.W % 128 == 0 ? 1 : 2) : 0;
  const size_t stage = pa.halo == 1   ? (size_t)2 * HSLOT
                       : pa.halo == 2 ? (size_t)6 * rbox_bytes(a.W)
                                      : (size_t)GPS * BM * 16 + (pa.resident ? 0 : GPS * BN * 16);
  const size_t smem = (size_t)P_STAGES * stage + (pa.resident ? (size_t)pa.wbytes : 0) + 1024;
  static int max_smem_set = 0;  // per instantiation, under g_attr_mu
  if ((int)smem > max_smem_set) {
    cudaError_t e = cudaFuncSetAttribute(k_conv3x3_p<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    max_smem_set = (int)smem;
  }
  // CTAs per SM from the shared-memory budget (1 KB reserved per CTA), the 512 TMEM
  // columns and the thread limit
  int dev = 0, nsm = 0, sm_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const int by_smem = sm_smem / (int)(smem + 2048);
  const int by_tmem = 512 / ptcols(BN);
  int per_sm = by_smem < by_tmem ? by_smem : by_tmem;
  if (per_sm > 2048 / 192) per_sm = 2048 / 192;
  if (per_sm < 1) per_sm = 1;
  const int grid = tiles < nsm * per_sm ? tiles : nsm * per_sm;
  k_conv3x3_p<BN><<<grid, 192, smem, s>>>(pa.halo ? *mxh : mx, mw, pa);
  return cudaGetLastError();
}

template <int BN>
cudaError_t wgrad_launch(const CUtensorMap& mdy, const CUtensorMap* mx, const WgradArgs& a, int splits, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(k_wgrad3x3<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv_smem<BN>());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_wgrad3x3<BN><<<dim3(splits, 9), 128, conv_smem<BN>(), s>>>(mdy, mx[0], mx[1], mx[2], a);
  return cudaGetLastError();
}

std::mutex g_attr_mu;

}  // namespace

cudaError_t conv3x3_tc(const Act& x, const void* w, int Cout, int mode, const float* bias, const Act& out, int* err,
                       cudaStream_t s, const GradRelu* gr) {
  const int W = x.W, H = x.H;
  if (x.C % 16 || x.off % 8 || x.cs % 8 || (W < 128 ? (128 % W || W % 8) : W % 128) || (H * W) % 128 ||
      out.N != x.N || out.H != H || out.W != W || out.off % 8 || out.cs % 8 || out.C != Cout)
    return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(x.p) & 15) || (reinterpret_cast<uintptr_t>(w) & 15) ||
      (reinterpret_cast<uintptr_t>(out.p) & 15))
    return cudaErrorInvalidValue;
  // activation view: dims {C, W, H, N}; the base is moved to the view's first channel
  CUtensorMap mx, mw;
  const char* xb = static_cast<const char*>(x.p) + (size_t)x.off * 2;
  const cuuint64_t xd[4] = {(cuuint64_t)x.C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)x.N};
  const cuuint64_t xs[3] = {(cuuint64_t)x.cs * 2, (cuuint64_t)x.cs * 2 * W, (cuuint64_t)x.cs * 2 * W * H};
  const int Wt = W < 128 ? W : 128;
  const cuuint32_t xbox[4] = {8, (cuuint32_t)Wt, (cuuint32_t)(128 / Wt), 1};
  cudaError_t e = make_map(&mx, xb, 4, xd, xs, xbox);
  if (e != cudaSuccess) return e;
  CUtensorMap mxh;  // halo boxes (rows of at least 128 pixels) or row-halo boxes (narrower rows)
  const bool halo = W % 128 == 0 || SS_CONV_RHALO;
  if (W % 128 == 0) {
    const cuuint32_t hbox[4] = {8, 130, 3, 1};
    e = make_map(&mxh, xb, 4, xd, xs, hbox);
    if (e != cudaSuccess) return e;
  } else if (halo) {
    const cuuint32_t rbox[4] = {8, (cuuint32_t)W, (cuuint32_t)(128 / W + 2), 1};
    e = make_map(&mxh, xb, 4, xd, xs, rbox);
    if (e != cudaSuccess) return e;
  }
  const int K = 9 * x.C;
  const cuuint64_t wd[2] = {(cuuint64_t)K, (cuuint64_t)Cout};
  const cuuint64_t ws[1] = {(cuuint64_t)K * 2};
  ConvArgs a{x.N, H, W, x.C, Cout, mode, bias, static_cast<char*>(out.p), out.cs, out.off, err,
             nullptr, 0, 0, nullptr, nullptr, (long long)x.N * H * W};
  if (mode == CONV_GRAD_RELU) {
    const Act& m = gr ? gr->mask : out;
    if (!gr || !gr->dyT || !gr->dbias || !m.p || m.N != x.N || m.H != H || m.W != W || m.C != Cout || m.cs % 8 ||
        m.off % 8 || (reinterpret_cast<uintptr_t>(m.p) & 15))
      return cudaErrorInvalidValue;
    a.mask = static_cast<const __nv_bfloat16*>(m.p);
    a.mask_cs = m.cs;
    a.mask_off = m.off;
    a.dyT = static_cast<__nv_bfloat16*>(gr->dyT);
    a.dbias = gr->dbias;
  }
  const int tiles = x.N * H * W / 128;
  std::lock_guard<std::mutex> lock(g_attr_mu);
#define SS_CONV_CASE(BNV)                                   \
  case BNV: {                                               \
    const cuuint32_t wbox[2] = {8, (cuuint32_t)BNV};        \
    e = make_map(&mw, w, 2, wd, ws, wbox);                  \
    if (e != cudaSuccess) return e;                         \
    return conv_launch_p<BNV>(mx, halo ? &mxh : nullptr, mw, a, tiles, K, s); \
  }
  switch (Cout) {
    SS_CONV_CASE(16)
    SS_CONV_CASE(32)
    SS_CONV_CASE(48)
    SS_CONV_CASE(80)
    SS_CONV_CASE(96)
    SS_CONV_CASE(144)
    default:
      return cudaErrorInvalidValue;
  }
#undef SS_CONV_CASE
}

cudaError_t wgrad3x3_tc(const void* dyT, const void* xT, int N, int H, int W, int Cout, int Cin, float* dw, int* err,
                        cudaStream_t s) {
  const long long P = (long long)N * H * W;
  if (W % 8 || P % 16 || Cout < 1 || Cout > 128 || P >= (1LL << 31)) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(dyT) & 15) || (reinterpret_cast<uintptr_t>(xT) & 15)) return cudaErrorInvalidValue;
  CUtensorMap mdy, mx[3];
  const cuuint64_t dd[4] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N, (cuuint64_t)Cout};
  const cuuint64_t st[3] = {(cuuint64_t)W * 2, (cuuint64_t)W * H * 2, (cuuint64_t)P * 2};
  const cuuint64_t xd[4] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N, (cuuint64_t)Cin};
  cudaError_t e;
  if (W % 64 == 0 && Cin % 16 == 0 && Cin <= 48 && (Cout == 16 || Cout == 32 || Cout == 48 || Cout == 96)) {
    // (tap, input channel) rows: 64-pixel K-blocks in 128-byte-swizzled boxes
    WgRowArgs a{N, H, W, Cout, Cin, 0, (int)(P / 64), 0, 0, 0, 0, dw, err};
    const cuuint32_t xbox[4] = {64, SS_WG_ROWS3 ? 3u : 1u, 1, (cuuint32_t)Cin};
    for (int d = 0; d < 3; ++d) {
      e = make_map(&mx[d], static_cast<const char*>(xT) + (size_t)d * Cin * P * 2, 4, xd, st, xbox, true);
      if (e != cudaSuccess) return e;
    }
    const cuuint32_t dbox[4] = {64, 1, 1, (cuuint32_t)Cout};
    e = make_map(&mdy, dyT, 4, dd, st, dbox, true);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    switch (Cout) {
      case 16: return wgrad_rows_launch<16>(mdy, mx, a, s);
      case 32: return wgrad_rows_launch<32>(mdy, mx, a, s);
      case 48: return wgrad_rows_launch<48>(mdy, mx, a, s);
      default: return wgrad_rows_launch<96>(mdy, mx, a, s);
    }
  }
  if (W % 64 == 0) {  // 64-pixel K-blocks in 128-byte-swizzled boxes
    const cuuint32_t dbox[4] = {64, 1, 1, 128};
    e = make_map(&mdy, dyT, 4, dd, st, dbox, true);
    if (e != cudaSuccess) return e;
    WgSwArgs a{N, H, W, Cout, Cin, 0, (int)(P / 64), 0, dw, err};
    std::lock_guard<std::mutex> lock(g_attr_mu);
#define SS_WGS_CASE(BNV, TPCV)                                                                          \
  case BNV: {                                                                                           \
    const cuuint32_t xbox[4] = {64, 1, 1, (cuuint32_t)BNV};                                             \
    for (int d = 0; d < 3; ++d) {                                                                       \
      e = make_map(&mx[d], static_cast<const char*>(xT) + (size_t)d * Cin * P * 2, 4, xd, st, xbox, true); \
      if (e != cudaSuccess) return e;                                                                   \
    }                                                                                                   \
    return wgrad_sw_launch<BNV, TPCV>(mdy, mx, a, s);                                                   \
  }
    switch (Cin) {
      SS_WGS_CASE(16, 9)
      SS_WGS_CASE(32, 9)
      SS_WGS_CASE(48, 9)
      SS_WGS_CASE(80, 1)
      SS_WGS_CASE(96, 1)
      SS_WGS_CASE(144, 1)
      default:
        return cudaErrorInvalidValue;
    }
#undef SS_WGS_CASE
  }
  const cuuint32_t dbox[4] = {8, 1, 1, 128};
  e = make_map(&mdy, dyT, 4, dd, st, dbox);
  if (e != cudaSuccess) return e;
  // K-groups split over CTAs: about 4 waves of 9-tap grids over 152 SMs, even counts
  const int total = (int)(P / 8);
  int splits = (152 * 4 + 8) / 9;
  int gpc = (total + splits - 1) / splits;
  gpc = (gpc + 1) & ~1;
  if (gpc < 16) gpc = 16;
  splits = (total + gpc - 1) / gpc;
  WgradArgs a{N, H, W, Cout, Cin, gpc, total, dw, err};
  std::lock_guard<std::mutex> lock(g_attr_mu);
#define SS_WG_CASE(BNV)                                                                      \
  case BNV: {                                                                                \
    const cuuint32_t xbox[4] = {8, 1, 1, (cuuint32_t)BNV};                                   \
    for (int d = 0; d < 3; ++d) {                                                            \
      e = make_map(&mx[d], static_cast<const char*>(xT) + (size_t)d * Cin * P * 2, 4, xd, st, xbox); \
      if (e != cudaSuccess) return e;                                                        \
    }                                                                                        \
    return wgrad_launch<BNV>(mdy, mx, a, splits, s);                                         \
  }
  switch (Cin) {
    SS_WG_CASE(16)
    SS_WG_CASE(32)
    SS_WG_CASE(48)
    SS_WG_CASE(80)
    SS_WG_CASE(96)
    SS_WG_CASE(144)
    default:
      return cudaErrorInvalidValue;
  }
#undef SS_WG_CASE
}


// ---------------------------------------------------------------- wait self-test
// The bounded mbarrier wait of the kernels above, on a barrier nothing completes:
// it gives up after limit_ns and records code 99 (the failure path of a stalled copy).
__global__ void k_wait_selftest(uint64_t limit_ns, int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0, limit_ns)) record_fail(err, 99);
}

cudaError_t wait_selftest(uint64_t limit_ns, int* err, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(limit_ns, err);
  return cudaGetLastError();
}

}  // namespace ss
