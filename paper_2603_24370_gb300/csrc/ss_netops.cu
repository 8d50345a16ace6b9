// ss_netops.cu -- the memory-bound layers of the learned initialiser: 2x2 average
// pooling, nearest-neighbour upsampling, ReLU gradients, bias gradients, the
// channel-major (and column-shifted) copies the weight-gradient contraction reads,
// and gradient routing through the decoder's concatenations. Each kernel is a
// grid-stride loop over elements with 16-byte accesses along channels where the
// layout allows it.
#include <cuda_bf16.h>

#include "ss_net_internal.h"

namespace ss {
namespace {

int grid_for(size_t n, int threads = 256) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t b = (n + threads - 1) / threads;
  const size_t cap = (size_t)nsm * 8;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

__device__ __forceinline__ const __nv_bfloat16* act_ptr(const Act& a, size_t pix) {
  return static_cast<const __nv_bfloat16*>(a.p) + pix * a.cs + a.off;
}
__device__ __forceinline__ __nv_bfloat16* act_wptr(const Act& a, size_t pix) {
  return static_cast<__nv_bfloat16*>(a.p) + pix * a.cs + a.off;
}

// xT[d][c][pix] = x[pix shifted by dx = d - 1 along x][c]; one thread per (pix, 8 channels)
__global__ void k_shifted_transpose(const Act x, __nv_bfloat16* __restrict__ xT) {
  const size_t P = (size_t)x.N * x.H * x.W;
  const int cg = x.C / 8;
  const size_t total = P * cg;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t pix = i / cg;
    const int c0 = (int)(i - pix * cg) * 8;
    const int xx = (int)(pix % x.W);
    const uint4 v = *reinterpret_cast<const uint4*>(act_ptr(x, pix) + c0);
    const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&v);
    // x at column xx feeds copy d at column xx - (d - 1)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int xd = xx - (d - 1);
      if (xd < 0 || xd >= x.W) continue;
      const size_t q = pix - xx + xd;
      __nv_bfloat16* o = xT + (size_t)d * x.C * P;
#pragma unroll
      for (int k = 0; k < 8; ++k) o[(size_t)(c0 + k) * P + q] = e[k];
    }
    // the column that no source reaches in each shifted copy is zero
    if (xx == 0) {  // copy d = 2 (dx = +1) at column W - 1
      __nv_bfloat16* o = xT + (size_t)2 * x.C * P;
#pragma unroll
      for (int k = 0; k < 8; ++k) o[(size_t)(c0 + k) * P + pix + x.W - 1] = __float2bfloat16(0.f);
    }
    if (xx == x.W - 1) {  // copy d = 0 (dx = -1) at column 0
#pragma unroll
      for (int k = 0; k < 8; ++k) xT[(size_t)(c0 + k) * P + pix - (x.W - 1)] = __float2bfloat16(0.f);
    }
  }
}

// dy_bf16 = bf16(dy * mask), dyT = the same, channel-major; dbias += sum over pixels.
// One block handles a run of pixels for all channels; per-channel partial sums in
// shared memory, one atomic per channel per block.
__global__ void k_relu_grad(const float* __restrict__ dy, const Act yact, int has_mask, size_t P, int C,
                            __nv_bfloat16* __restrict__ dyb, __nv_bfloat16* __restrict__ dyT, float* __restrict__ dbias) {
  extern __shared__ float sb[];
  for (int c = threadIdx.x; c < C; c += blockDim.x) sb[c] = 0.f;
  __syncthreads();
  const size_t total = P * C;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t pix = i / C;
    const int c = (int)(i - pix * C);
    float g = dy[i];
    if (has_mask && !(__bfloat162float(act_ptr(yact, pix)[c]) > 0.f)) g = 0.f;
    const __nv_bfloat16 b = __float2bfloat16(g);
    dyb[i] = b;
    dyT[(size_t)c * P + pix] = b;
    atomicAdd(&sb[c], g);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) atomicAdd(&dbias[c], sb[c]);
}

__global__ void k_avgpool2(const Act x, const Act out) {
  const size_t Po = (size_t)out.N * out.H * out.W;
  const int cg = out.C / 8;
  const size_t total = Po * cg;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t po = i / cg;
    const int c0 = (int)(i - po * cg) * 8;
    const int xo = (int)(po % out.W);
    const size_t t = po / out.W;
    const int yo = (int)(t % out.H);
    const int n = (int)(t / out.H);
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const size_t pi = ((size_t)n * x.H + 2 * yo + (q >> 1)) * x.W + 2 * xo + (q & 1);
      const uint4 v = *reinterpret_cast<const uint4*>(act_ptr(x, pi) + c0);
      const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] += __bfloat162float(e[k]);
    }
    uint4 o;
    __nv_bfloat16* oe = reinterpret_cast<__nv_bfloat16*>(&o);
#pragma unroll
    for (int k = 0; k < 8; ++k) oe[k] = __float2bfloat16(0.25f * acc[k]);
    *reinterpret_cast<uint4*>(act_wptr(out, po) + c0) = o;
  }
}

// Four channels per thread (C % 4 == 0): 16-byte loads and stores.
__global__ void k_avgpool2_backward(const float* __restrict__ dout, int N, int Ho, int Wo, int C,
                                    float* __restrict__ dx) {
  const int C4 = C / 4;
  const size_t total = (size_t)N * (2 * Ho) * (2 * Wo) * C4;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t pix = i / C4;
    const int c = (int)(i - pix * C4) * 4;
    const int xx = (int)(pix % (2 * Wo));
    const size_t t = pix / (2 * Wo);
    const int yy = (int)(t % (2 * Ho));
    const int n = (int)(t / (2 * Ho));
    const float4 g = *reinterpret_cast<const float4*>(dout + (((size_t)n * Ho + yy / 2) * Wo + xx / 2) * C + c);
    float4* d = reinterpret_cast<float4*>(dx + pix * C + c);
    float4 v = *d;
    v.x += 0.25f * g.x;
    v.y += 0.25f * g.y;
    v.z += 0.25f * g.z;
    v.w += 0.25f * g.w;
    *d = v;
  }
}

__global__ void k_upsample2(const Act x, const Act out) {
  const size_t Po = (size_t)out.N * out.H * out.W;
  const int cg = out.C / 8;
  const size_t total = Po * cg;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t po = i / cg;
    const int c0 = (int)(i - po * cg) * 8;
    const int xo = (int)(po % out.W);
    const size_t t = po / out.W;
    const int yo = (int)(t % out.H);
    const int n = (int)(t / out.H);
    const size_t pi = ((size_t)n * x.H + yo / 2) * x.W + xo / 2;
    *reinterpret_cast<uint4*>(act_wptr(out, po) + c0) = *reinterpret_cast<const uint4*>(act_ptr(x, pi) + c0);
  }
}

// Four channels per thread (C, cs and off multiples of 4): 16-byte loads and stores.
__global__ void k_upsample2_backward(const float* __restrict__ dup, int cs, int off, int N, int H, int W, int C,
                                     float* __restrict__ dx) {
  const int C4 = C / 4;
  const size_t total = (size_t)N * H * W * C4;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t pix = i / C4;
    const int c = (int)(i - pix * C4) * 4;
    const int xx = (int)(pix % W);
    const size_t t = pix / W;
    const int yy = (int)(t % H);
    const int n = (int)(t / H);
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const size_t pu = ((size_t)n * (2 * H) + 2 * yy + (q >> 1)) * (2 * W) + 2 * xx + (q & 1);
      const float4 u = *reinterpret_cast<const float4*>(dup + pu * cs + off + c);
      s.x += u.x;
      s.y += u.y;
      s.z += u.z;
      s.w += u.w;
    }
    *reinterpret_cast<float4*>(dx + pix * C + c) = s;
  }
}

// Four channels per thread (C, cs and off multiples of 4).
__global__ void k_add_slice(const float* __restrict__ src, int cs, int off, size_t P, int C, float* __restrict__ dst) {
  const int C4 = C / 4;
  const size_t total = P * C4;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t pix = i / C4;
    const int c = (int)(i - pix * C4) * 4;
    const float4 u = *reinterpret_cast<const float4*>(src + pix * cs + off + c);
    float4* d = reinterpret_cast<float4*>(dst + pix * C + c);
    float4 v = *d;
    v.x += u.x;
    v.y += u.y;
    v.z += u.z;
    v.w += u.w;
    *d = v;
  }
}

// One image row per block: the row's C channels are staged in shared memory as
// [C][W + 2] (the padding staggers the channels across banks), then each thread
// writes 8 consecutive pixels of one channel of one shifted copy as a 16-byte store.
__global__ void k_shifted_transpose_rows(const Act x, __nv_bfloat16* __restrict__ xT) {
  extern __shared__ __nv_bfloat16 row[];  // [C][W + 2]
  const size_t P = (size_t)x.N * x.H * x.W;
  const int W = x.W, C = x.C, cg = C / 8, RS = W + 2;
  const int nrows = x.N * x.H;
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  for (int rr = blockIdx.x; rr < nrows; rr += gridDim.x) {
    const size_t pix0 = (size_t)rr * W;
    __syncthreads();  // the previous row's reads are done
    for (int i = threadIdx.x; i < W * cg; i += blockDim.x) {
      const int xx = i / cg, c0 = (i - xx * cg) * 8;
      const uint4 v = *reinterpret_cast<const uint4*>(act_ptr(x, pix0 + xx) + c0);
      const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
      for (int k = 0; k < 8; ++k) row[(c0 + k) * RS + xx] = e[k];
    }
    __syncthreads();
    const int chunks = W / 8;
    for (int i = threadIdx.x; i < 3 * C * chunks; i += blockDim.x) {
      const int d = i / (C * chunks), rem = i - d * C * chunks;
      const int c = rem / chunks, x0 = (rem - c * chunks) * 8;
      uint4 o;
      __nv_bfloat16* oe = reinterpret_cast<__nv_bfloat16*>(&o);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int src = x0 + k + d - 1;  // copy d holds x[x + d - 1]
        oe[k] = (src >= 0 && src < W) ? row[c * RS + src] : zero;
      }
      *reinterpret_cast<uint4*>(xT + ((size_t)d * C + c) * P + pix0 + x0) = o;
    }
  }
}

// dy (FP32 NHWC) -> masked gradient: BF16 NHWC (dyb) and channel-major (dyT), and the
// bias gradient. A block takes 128 pixels at a time: four channels per thread in NHWC
// order (16-byte loads of dy, 8-byte loads of the mask and stores of dyb), staged in
// shared memory as [128][C + 1] FP32 (the odd pitch keeps the channel-major reads free
// of bank conflicts), then written channel-major. A warp's 32 channel-major values
// share one channel, so they are summed by shuffles into one shared atomic; one
// global atomic per channel per block at the end.
constexpr int RG_TP = 128;  // pixels per tile, a multiple of 32
__global__ void k_relu_grad_tiles(const float* __restrict__ dy, const Act yact, int has_mask, size_t P, int C,
                                  __nv_bfloat16* __restrict__ dyb, __nv_bfloat16* __restrict__ dyT,
                                  float* __restrict__ dbias) {
  extern __shared__ unsigned char rg_smem[];
  const int GS = C + 1;
  float* g = reinterpret_cast<float*>(rg_smem);  // [RG_TP][GS] FP32
  float* csum = g + RG_TP * GS;                  // [C]
  for (int c = threadIdx.x; c < C; c += blockDim.x) csum[c] = 0.f;
  const int C4 = C / 4;
  const size_t ntiles = (P + RG_TP - 1) / RG_TP;
  for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const size_t pix0 = tile * RG_TP;
    const int np = (int)((P - pix0) < (size_t)RG_TP ? (P - pix0) : (size_t)RG_TP);
    __syncthreads();
    for (int i = threadIdx.x; i < np * C4; i += blockDim.x) {  // NHWC order: coalesced
      const int pp = i / C4, c = (i - pp * C4) * 4;
      const size_t e = (pix0 + pp) * C + c;
      float4 v = *reinterpret_cast<const float4*>(dy + e);
      if (has_mask) {
        const uint2 m = *reinterpret_cast<const uint2*>(act_ptr(yact, pix0 + pp) + c);
        const float2 m01 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&m.x));
        const float2 m23 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&m.y));
        if (!(m01.x > 0.f)) v.x = 0.f;
        if (!(m01.y > 0.f)) v.y = 0.f;
        if (!(m23.x > 0.f)) v.z = 0.f;
        if (!(m23.y > 0.f)) v.w = 0.f;
      }
      float* gr = g + pp * GS + c;
      gr[0] = v.x;
      gr[1] = v.y;
      gr[2] = v.z;
      gr[3] = v.w;
      __nv_bfloat162 b01 = __floats2bfloat162_rn(v.x, v.y), b23 = __floats2bfloat162_rn(v.z, v.w);
      uint2 o;
      o.x = *reinterpret_cast<uint32_t*>(&b01);
      o.y = *reinterpret_cast<uint32_t*>(&b23);
      *reinterpret_cast<uint2*>(dyb + e) = o;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < C * np; i += blockDim.x) {  // channel-major: coalesced
      const int c = i / np, pp = i - c * np;
      const float v = g[pp * GS + c];
      dyT[(size_t)c * P + pix0 + pp] = __float2bfloat16(v);
      if (np == RG_TP) {  // the warp's lanes hold 32 pixels of channel c
        float w = v;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&csum[c], w);
      } else {
        atomicAdd(&csum[c], v);
      }
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) atomicAdd(&dbias[c], csum[c]);
}

bool act_ok(const Act& a) { return a.p && a.C % 8 == 0 && a.cs % 8 == 0 && a.off % 8 == 0 && a.off + a.C <= a.cs; }

}  // namespace

cudaError_t shifted_transpose(const Act& x, void* xT, cudaStream_t s) {
  if (!act_ok(x)) return cudaErrorInvalidValue;
  const size_t row_bytes = (size_t)x.C * (x.W + 2) * sizeof(__nv_bfloat16);
  if (row_bytes <= 48 * 1024 && x.W % 8 == 0) {  // one image row per block, staged in shared memory
    const int rows = x.N * x.H;
    k_shifted_transpose_rows<<<grid_for((size_t)rows * 256) < rows ? grid_for((size_t)rows * 256) : rows, 256,
                               row_bytes, s>>>(x, static_cast<__nv_bfloat16*>(xT));
    return cudaGetLastError();
  }
  const size_t n = (size_t)x.N * x.H * x.W * (x.C / 8);
  k_shifted_transpose<<<grid_for(n), 256, 0, s>>>(x, static_cast<__nv_bfloat16*>(xT));
  return cudaGetLastError();
}

cudaError_t relu_grad(const float* dy, const Act* y_act, int N, int H, int W, int C, void* dy_bf16, void* dyT,
                      float* dbias, cudaStream_t s) {
  const size_t P = (size_t)N * H * W;
  Act y{};
  if (y_act) y = *y_act;
  const size_t smem = ((size_t)RG_TP * (C + 1) + C) * sizeof(float);
  if (smem <= 48 * 1024 && C % 4 == 0) {
    const size_t ntiles = (P + RG_TP - 1) / RG_TP;
    int blocks = grid_for(ntiles * 256);
    if ((size_t)blocks > ntiles) blocks = (int)ntiles;
    k_relu_grad_tiles<<<blocks, 256, smem, s>>>(dy, y, y_act != nullptr, P, C, static_cast<__nv_bfloat16*>(dy_bf16),
                                                static_cast<__nv_bfloat16*>(dyT), dbias);
    return cudaGetLastError();
  }
  k_relu_grad<<<grid_for(P * C), 256, C * sizeof(float), s>>>(dy, y, y_act != nullptr, P, C,
                                                              static_cast<__nv_bfloat16*>(dy_bf16),
                                                              static_cast<__nv_bfloat16*>(dyT), dbias);
  return cudaGetLastError();
}

cudaError_t avgpool2(const Act& x, const Act& out, cudaStream_t s) {
  if (!act_ok(x) || !act_ok(out) || out.C != x.C || out.H * 2 != x.H || out.W * 2 != x.W) return cudaErrorInvalidValue;
  const size_t n = (size_t)out.N * out.H * out.W * (out.C / 8);
  k_avgpool2<<<grid_for(n), 256, 0, s>>>(x, out);
  return cudaGetLastError();
}

bool f4_ok(const float* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

cudaError_t avgpool2_backward(const float* dout, int N, int Ho, int Wo, int C, float* dx, cudaStream_t s) {
  if (C % 4 || !f4_ok(dout) || !f4_ok(dx)) return cudaErrorInvalidValue;
  const size_t n = (size_t)N * 4 * Ho * Wo * (C / 4);
  k_avgpool2_backward<<<grid_for(n), 256, 0, s>>>(dout, N, Ho, Wo, C, dx);
  return cudaGetLastError();
}

cudaError_t upsample2(const Act& x, const Act& out, cudaStream_t s) {
  if (!act_ok(x) || !act_ok(out) || out.C != x.C || out.H != 2 * x.H || out.W != 2 * x.W) return cudaErrorInvalidValue;
  const size_t n = (size_t)out.N * out.H * out.W * (out.C / 8);
  k_upsample2<<<grid_for(n), 256, 0, s>>>(x, out);
  return cudaGetLastError();
}

cudaError_t upsample2_backward(const float* dup, int cs, int off, int N, int H, int W, int C, float* dx,
                               cudaStream_t s) {
  if (C % 4 || cs % 4 || off % 4 || !f4_ok(dup) || !f4_ok(dx)) return cudaErrorInvalidValue;
  const size_t n = (size_t)N * H * W * (C / 4);
  k_upsample2_backward<<<grid_for(n), 256, 0, s>>>(dup, cs, off, N, H, W, C, dx);
  return cudaGetLastError();
}

cudaError_t add_slice(const float* src, int cs, int off, int N, int H, int W, int C, float* dst, cudaStream_t s) {
  if (C % 4 || cs % 4 || off % 4 || !f4_ok(src) || !f4_ok(dst)) return cudaErrorInvalidValue;
  const size_t P = (size_t)N * H * W;
  k_add_slice<<<grid_for(P * (C / 4)), 256, 0, s>>>(src, cs, off, P, C, dst);
  return cudaGetLastError();
}

}  // namespace ss
