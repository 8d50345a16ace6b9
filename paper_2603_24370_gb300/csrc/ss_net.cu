// ss_net.cu -- the learned initialiser: a 4-level convolutional U-Net that maps an
// ansatz field (and its couplings) to a correction towards the relaxed field, and
// its training (forward, backward, Adam) on the GPU.
//
// Architecture (channels 16, 32, 48, 96; every convolution 3x3, zero padding, ReLU
// except the last): two convolutions per level, 2x2 average pooling down, nearest
// x2 upsampling up, the encoder output of each level concatenated with the
// upsampled decoder input. The input holds the theory's field components and one
// plane per coupling, zero-padded to 16 channels; the output's first C channels
// are the correction. With these widths the network has 304,720 parameters (the
// last layer computes 16 channels; those beyond C keep zero weights, since the loss
// never reaches them).
//
// Convolutions run on the tensor cores (ss_conv.cu), BF16 operands and FP32
// accumulation; weights are kept in FP32 (the Adam state too) and re-rounded to
// BF16 after each update. Activations are BF16, gradients FP32 until they feed a
// contraction.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "soliton.h"
#include "soliton_net.h"
#include "ss_internal.h"
#include "ss_net_internal.h"

using namespace ss;

namespace {

constexpr int NL = 15;          // convolutions
constexpr int CIN_PAD = 16;     // input channels (fields + coupling planes, zero-padded)
constexpr int COUT_LAST = 16;   // output channels computed (the first C are used)
constexpr uint32_t NET_MAGIC = 0x4E455431u;  // "1TEN"

struct LayerDef {
  int cin, cout, level;
  bool relu;
};
// conv index -> (input channels, output channels, level)
constexpr LayerDef LAYERS[NL] = {
    {16, 16, 0, true},  {16, 16, 0, true},  {16, 32, 1, true},  {32, 32, 1, true},  {32, 48, 2, true},
    {48, 48, 2, true},  {48, 96, 3, true},  {96, 96, 3, true},  {144, 48, 2, true}, {48, 48, 2, true},
    {80, 32, 1, true},  {32, 32, 1, true},  {48, 16, 0, true},  {16, 16, 0, true},  {16, 16, 0, false}};

thread_local std::string g_net_err;
int nfail(int code, const std::string& m) {
  g_net_err = m;
  set_last_error(m);
  return code;
}

// ---------------------------------------------------------------- small kernels
// NHWC BF16 input: field components of the SoA planes, then one plane per coupling.
__global__ void k_pack_input(const float* __restrict__ fields, int C, const float* __restrict__ coup, int ncoup,
                             int B, int S, __nv_bfloat16* __restrict__ in) {
  const size_t P = (size_t)S * S;
  const size_t total = (size_t)B * P;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / P, q = i - b * P;
    __nv_bfloat16 v[CIN_PAD];
#pragma unroll
    for (int c = 0; c < CIN_PAD; ++c) {
      float x = 0.f;
      if (c < C) x = fields[(b * C + c) * P + q];
      else if (c < C + ncoup) x = coup[b * ncoup + (c - C)];
      v[c] = __float2bfloat16(x);
    }
    uint4* o = reinterpret_cast<uint4*>(in + i * CIN_PAD);
    o[0] = *reinterpret_cast<uint4*>(&v[0]);
    o[1] = *reinterpret_cast<uint4*>(&v[8]);
  }
}

// loss = mean over interior sites and the first C channels of (out - target)^2 with
// target = relaxed - ansatz; dout = its gradient (zero elsewhere). Fields: SoA [B][C][S][S].
__global__ void k_mse(const float* __restrict__ out, const float* __restrict__ ansatz,
                      const float* __restrict__ relaxed, int C, int B, int S, float* __restrict__ dout,
                      double* __restrict__ loss) {
  __shared__ double red[8];
  const size_t P = (size_t)S * S;
  const size_t total = (size_t)B * P;
  const double inv = 1.0 / ((double)B * (S - 4) * (S - 4) * C);
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / P, q = i - b * P;
    const int y = (int)(q / S), x = (int)(q % S);
    const bool inside = x >= 2 && x < S - 2 && y >= 2 && y < S - 2;
    // the pixel's 16 output channels as four 16-byte loads and stores
    const float4* o4 = reinterpret_cast<const float4*>(out + i * COUT_LAST);
    float4* g4 = reinterpret_cast<float4*>(dout + i * COUT_LAST);
#pragma unroll
    for (int v = 0; v < COUT_LAST / 4; ++v) {
      float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (inside && 4 * v < C) {
        const float4 ov = o4[v];
        const float on[4] = {ov.x, ov.y, ov.z, ov.w};
        float gg[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int c = 4 * v + k;
          if (c < C) {
            const size_t f = (b * C + c) * P + q;
            const float d = on[k] - (relaxed[f] - ansatz[f]);
            acc += (double)d * d;
            gg[k] = (float)(2.0 * inv) * d;
          }
        }
        gv = make_float4(gg[0], gg[1], gg[2], gg[3]);
      }
      g4[v] = gv;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    atomicAdd(loss, s * inv);
  }
}

// init = ansatz + correction on the interior, the ansatz on the halo (Dirichlet);
// chiral magnet: unit length restored.
__global__ void k_apply(const float* __restrict__ ansatz, const float* __restrict__ out, int C, int B, int S,
                        int normalise, float* __restrict__ init) {
  const size_t P = (size_t)S * S;
  const size_t total = (size_t)B * P;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / P, q = i - b * P;
    const int y = (int)(q / S), x = (int)(q % S);
    const bool inside = x >= 2 && x < S - 2 && y >= 2 && y < S - 2;
    float v[4];
    for (int c = 0; c < C; ++c) v[c] = ansatz[(b * C + c) * P + q] + (inside ? out[i * COUT_LAST + c] : 0.f);
    if (normalise && inside) {
      float n2 = 0.f;
      for (int c = 0; c < C; ++c) n2 += v[c] * v[c];
      const float r = n2 > 0.f ? 1.f / sqrtf(n2) : 0.f;
      for (int c = 0; c < C; ++c) v[c] *= r;
    }
    for (int c = 0; c < C; ++c) init[(b * C + c) * P + q] = v[c];
  }
}

struct LayerView {
  int cin, cout;
  long long woff, boff;  // offsets into the parameter vector
  long long wbo, wto;    // offsets of the BF16 copies (elements)
};
struct LayerTable {
  LayerView l[NL];
};

// BF16 copies of every layer's weights: wb[co][tap * cin + ci] = W[co][tap][ci],
// wt[ci][tap * cout + co] = W[co][8 - tap][ci] (the input-gradient convolution).
__global__ void k_pack_weights(const float* __restrict__ theta, const LayerTable T, long long n,
                               __nv_bfloat16* __restrict__ wbf) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int L = -1;
#pragma unroll 1
    for (int k = 0; k < NL; ++k)
      if (i >= T.l[k].woff && i < T.l[k].boff) L = k;
    if (L < 0) continue;
    const LayerView& v = T.l[L];
    const long long j = i - v.woff;
    const int ci = (int)(j % v.cin);
    const int tap = (int)((j / v.cin) % 9);
    const int co = (int)(j / (9LL * v.cin));
    const __nv_bfloat16 w = __float2bfloat16(theta[i]);
    wbf[v.wbo + j] = w;
    wbf[v.wto + (long long)ci * 9 * v.cout + (long long)(8 - tap) * v.cout + co] = w;
  }
}

// Adam (Kingma & Ba 2015, Algorithm 1) over the flat parameter vector. omb1, omb2 are
// 1 - beta1, 1 - beta2 and c1, c2 the bias corrections 1 - beta1^t, 1 - beta2^t of
// update t, each formed in FP64 and rounded once (1.f - 0.999f would be 1.3e-5 off).
__global__ void k_adam(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float omb1, float omb2,
                       float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + omb1 * gi;
    const float vi = b2 * v[i] + omb2 * (gi * gi);
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

int grid_of(size_t n) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  size_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  return (int)(b < (size_t)nsm * 8 ? b : (size_t)nsm * 8);
}

// SplitMix64 (Steele, Lea, Flood 2014) and Box-Muller normals for the initial weights.
struct Rng {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
  double normal() {
    const double u = uniform(), w = uniform();
    return std::sqrt(-2.0 * std::log(u)) * std::cos(6.283185307179586 * w);
  }
};

}  // namespace

struct ss_net {
  int theory = 0, C = 0, ncoup = 0;
  int S = 0, maxB = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  LayerTable T{};
  long long nparam = 0, nwbf = 0;
  long long t = 0;  // Adam steps taken
  // device memory (one allocation)
  void* base = nullptr;
  float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16* wbf = nullptr;
  int* err = nullptr;
  double* loss = nullptr;
  float* coup = nullptr;  // [maxB * ncoup]
  // activations (BF16 NHWC) and their gradients (FP32 NHWC)
  Act in0, e1a, cat1, p1, e2a, cat2, p2, e3a, cat3, p3, b1, bb, d3a, d3, d2a, d2, d1a, d1;
  float* out = nullptr;  // FP32 [B][S][S][16]
  float *g_out, *g_d1, *g_d1a, *g_cat1, *g_d2, *g_d2a, *g_cat2, *g_d3, *g_d3a, *g_cat3, *g_b, *g_b1, *g_p3, *g_e3,
      *g_e3a, *g_p2, *g_e2, *g_e2a, *g_p1, *g_e1, *g_e1a;
  void *dyb = nullptr, *dyT = nullptr, *xT = nullptr, *xT1 = nullptr;
  void *dyb1 = nullptr, *dyT1 = nullptr;  // the masked output gradients, alternating by layer
  // backward: the weight gradients' shifted channel-major input copies are made on a
  // second stream, one layer ahead, into two alternating buffers (xT, xT1)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_start = nullptr, ev_x[2] = {nullptr, nullptr}, ev_w[2] = {nullptr, nullptr};
  double* h_loss = nullptr;  // pinned
  int* h_err = nullptr;      // pinned
};

namespace {

Act view(const Act& a, int B, int off, int C) {
  Act r = a;
  r.N = B;
  r.off = off;
  r.C = C;
  return r;
}
Act batch(const Act& a, int B) {
  Act r = a;
  r.N = B;
  return r;
}

#define NET_CK(call)                                                                                      \
  do {                                                                                                    \
    cudaError_t e_ = (call);                                                                              \
    if (e_ != cudaSuccess) return nfail(SS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int conv(ss_net* n, int L, const Act& x, const Act& y, int B) {
  const LayerView& lv = n->T.l[L];
  const Act xi = batch(x, B), yo = batch(y, B);
  NET_CK(conv3x3_tc(xi, n->wbf + lv.wbo, lv.cout, CONV_BF16_BIAS_RELU, n->theta + lv.boff, yo, n->err, n->stream));
  return SS_OK;
}

int forward(ss_net* n, int B) {
  const int S = n->S;
  int rc;
  if ((rc = conv(n, 0, n->in0, n->e1a, B))) return rc;
  const Act e1 = view(n->cat1, B, 32, 16);
  if ((rc = conv(n, 1, n->e1a, e1, B))) return rc;
  NET_CK(avgpool2(e1, batch(n->p1, B), n->stream));
  if ((rc = conv(n, 2, n->p1, n->e2a, B))) return rc;
  const Act e2 = view(n->cat2, B, 48, 32);
  if ((rc = conv(n, 3, n->e2a, e2, B))) return rc;
  NET_CK(avgpool2(e2, batch(n->p2, B), n->stream));
  if ((rc = conv(n, 4, n->p2, n->e3a, B))) return rc;
  const Act e3 = view(n->cat3, B, 96, 48);
  if ((rc = conv(n, 5, n->e3a, e3, B))) return rc;
  NET_CK(avgpool2(e3, batch(n->p3, B), n->stream));
  if ((rc = conv(n, 6, n->p3, n->b1, B))) return rc;
  if ((rc = conv(n, 7, n->b1, n->bb, B))) return rc;
  NET_CK(upsample2(batch(n->bb, B), view(n->cat3, B, 0, 96), n->stream));
  if ((rc = conv(n, 8, n->cat3, n->d3a, B))) return rc;
  if ((rc = conv(n, 9, n->d3a, n->d3, B))) return rc;
  NET_CK(upsample2(batch(n->d3, B), view(n->cat2, B, 0, 48), n->stream));
  if ((rc = conv(n, 10, n->cat2, n->d2a, B))) return rc;
  if ((rc = conv(n, 11, n->d2a, n->d2, B))) return rc;
  NET_CK(upsample2(batch(n->d2, B), view(n->cat1, B, 0, 32), n->stream));
  if ((rc = conv(n, 12, n->cat1, n->d1a, B))) return rc;
  if ((rc = conv(n, 13, n->d1a, n->d1, B))) return rc;
  const LayerView& lv = n->T.l[14];
  Act o{n->out, B, S, S, COUT_LAST, COUT_LAST, 0};
  NET_CK(conv3x3_tc(batch(n->d1, B), n->wbf + lv.wbo, COUT_LAST, CONV_F32_BIAS, n->theta + lv.boff, o, n->err,
                    n->stream));
  return SS_OK;
}

// Backward through conv L, the k-th of the backward pass: gradient gy (FP32 NHWC, cout
// channels) of its output y (mask: y's BF16 values, or none for the linear last layer),
// input x. Writes the weight and bias gradients and, if gx is given, the input gradient
// (FP32 NHWC). The shifted copies of x go to buffer k % 2 on the side stream, after the
// weight gradient of layer k - 2 has read that buffer. The masked output gradient
// (BF16 NHWC and channel-major) alternates between two buffer pairs by k.
// fused_in: the previous call already left it in pair k % 2 (and added the bias
// gradient). fuse_out: x is the ReLU output of conv L - 1, the next call: the input
// gradient is formed through that ReLU straight into pair (k + 1) % 2, with conv L - 1's
// bias gradient, and gx is not written.
int conv_backward(ss_net* n, int k, int L, const Act& x, const Act* y, const float* gy, float* gx, int B,
                  bool fused_in = false, bool fuse_out = false) {
  const LayerView& lv = n->T.l[L];
  const Act xi = batch(x, B);
  Act yb;
  if (y) yb = batch(*y, B);
  void* xT = (k & 1) ? n->xT1 : n->xT;
  void* dyb = (k & 1) ? n->dyb1 : n->dyb;
  void* dyT = (k & 1) ? n->dyT1 : n->dyT;
  if (k >= 2) NET_CK(cudaStreamWaitEvent(n->side, n->ev_w[k & 1], 0));
  NET_CK(shifted_transpose(xi, xT, n->side));
  NET_CK(cudaEventRecord(n->ev_x[k & 1], n->side));
  if (!fused_in)
    NET_CK(relu_grad(gy, y ? &yb : nullptr, B, xi.H, xi.W, lv.cout, dyb, dyT, n->grad + lv.boff, n->stream));
  NET_CK(cudaStreamWaitEvent(n->stream, n->ev_x[k & 1], 0));
  NET_CK(wgrad3x3_tc(dyT, xT, B, xi.H, xi.W, lv.cout, lv.cin, n->grad + lv.woff, n->err, n->stream));
  NET_CK(cudaEventRecord(n->ev_w[k & 1], n->stream));
  Act dy{dyb, B, xi.H, xi.W, lv.cout, lv.cout, 0};
  if (fuse_out) {
    GradRelu g;
    g.mask = xi;
    g.dyT = (k & 1) ? n->dyT : n->dyT1;
    g.dbias = n->grad + n->T.l[L - 1].boff;
    Act o{(k & 1) ? n->dyb : n->dyb1, B, xi.H, xi.W, lv.cin, lv.cin, 0};
    NET_CK(conv3x3_tc(dy, n->wbf + lv.wto, lv.cin, CONV_GRAD_RELU, nullptr, o, n->err, n->stream, &g));
  } else if (gx) {
    Act gxa{gx, B, xi.H, xi.W, lv.cin, lv.cin, 0};
    NET_CK(conv3x3_tc(dy, n->wbf + lv.wto, lv.cin, CONV_F32, nullptr, gxa, n->err, n->stream));
  }
  return SS_OK;
}

int backward(ss_net* n, int B) {
  const int S = n->S;
  const cudaStream_t s = n->stream;
  int rc;
  NET_CK(cudaMemsetAsync(n->grad, 0, sizeof(float) * n->nparam, s));
  // the forward activations are complete: the side stream may start copying them
  NET_CK(cudaEventRecord(n->ev_start, s));
  NET_CK(cudaStreamWaitEvent(n->side, n->ev_start, 0));
  int k = 0;
  const Act e1 = view(n->cat1, B, 32, 16), e2 = view(n->cat2, B, 48, 32), e3 = view(n->cat3, B, 96, 48);
  if ((rc = conv_backward(n, k++, 14, n->d1, nullptr, n->g_out, n->g_d1, B, false, true))) return rc;
  if ((rc = conv_backward(n, k++, 13, n->d1a, &n->d1, n->g_d1, n->g_d1a, B, true, true))) return rc;
  if ((rc = conv_backward(n, k++, 12, n->cat1, &n->d1a, n->g_d1a, n->g_cat1, B, true, false))) return rc;
  NET_CK(upsample2_backward(n->g_cat1, 48, 0, B, S / 2, S / 2, 32, n->g_d2, s));
  if ((rc = conv_backward(n, k++, 11, n->d2a, &n->d2, n->g_d2, n->g_d2a, B, false, true))) return rc;
  if ((rc = conv_backward(n, k++, 10, n->cat2, &n->d2a, n->g_d2a, n->g_cat2, B, true, false))) return rc;
  NET_CK(upsample2_backward(n->g_cat2, 80, 0, B, S / 4, S / 4, 48, n->g_d3, s));
  if ((rc = conv_backward(n, k++, 9, n->d3a, &n->d3, n->g_d3, n->g_d3a, B, false, true))) return rc;
  if ((rc = conv_backward(n, k++, 8, n->cat3, &n->d3a, n->g_d3a, n->g_cat3, B, true, false))) return rc;
  NET_CK(upsample2_backward(n->g_cat3, 144, 0, B, S / 8, S / 8, 96, n->g_b, s));
  if ((rc = conv_backward(n, k++, 7, n->b1, &n->bb, n->g_b, n->g_b1, B, false, true))) return rc;
  if ((rc = conv_backward(n, k++, 6, n->p3, &n->b1, n->g_b1, n->g_p3, B, true, false))) return rc;
  // level 2 encoder output: concatenation slice + pooling path
  NET_CK(cudaMemsetAsync(n->g_e3, 0, sizeof(float) * (size_t)B * (S / 4) * (S / 4) * 48, s));
  NET_CK(add_slice(n->g_cat3, 144, 96, B, S / 4, S / 4, 48, n->g_e3, s));
  NET_CK(avgpool2_backward(n->g_p3, B, S / 8, S / 8, 48, n->g_e3, s));
  if ((rc = conv_backward(n, k++, 5, n->e3a, &e3, n->g_e3, n->g_e3a, B, false, true))) return rc;
  if ((rc = conv_backward(n, k++, 4, n->p2, &n->e3a, n->g_e3a, n->g_p2, B, true, false))) return rc;
  NET_CK(cudaMemsetAsync(n->g_e2, 0, sizeof(float) * (size_t)B * (S / 2) * (S / 2) * 32, s));
  NET_CK(add_slice(n->g_cat2, 80, 48, B, S / 2, S / 2, 32, n->g_e2, s));
  NET_CK(avgpool2_backward(n->g_p2, B, S / 4, S / 4, 32, n->g_e2, s));
  if ((rc = conv_backward(n, k++, 3, n->e2a, &e2, n->g_e2, n->g_e2a, B, false, true))) return rc;
  if ((rc = conv_backward(n, k++, 2, n->p1, &n->e2a, n->g_e2a, n->g_p1, B, true, false))) return rc;
  NET_CK(cudaMemsetAsync(n->g_e1, 0, sizeof(float) * (size_t)B * S * S * 16, s));
  NET_CK(add_slice(n->g_cat1, 48, 32, B, S, S, 16, n->g_e1, s));
  NET_CK(avgpool2_backward(n->g_p1, B, S / 2, S / 2, 16, n->g_e1, s));
  if ((rc = conv_backward(n, k++, 1, n->e1a, &e1, n->g_e1, n->g_e1a, B, false, true))) return rc;
  if ((rc = conv_backward(n, k++, 0, n->in0, &n->e1a, n->g_e1a, nullptr, B, true, false))) return rc;
  return SS_OK;
}

int pack_weights(ss_net* n) {
  k_pack_weights<<<grid_of((size_t)n->nparam), 256, 0, n->stream>>>(n->theta, n->T, n->nparam, n->wbf);
  NET_CK(cudaGetLastError());
  return SS_OK;
}

// Device-side failure flags of the tensor-core kernels (bounded waits that gave up).
int check_err(ss_net* n) {
  NET_CK(cudaMemcpyAsync(n->h_err, n->err, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
  NET_CK(cudaStreamSynchronize(n->stream));
  if (*n->h_err) {
    const int code = *n->h_err;
    cudaMemsetAsync(n->err, 0, sizeof(int), n->stream);
    return nfail(SS_ERR_TIMEOUT, "tensor-core kernel gave up waiting (code " + std::to_string(code) + ")");
  }
  return SS_OK;
}

int check_batch(const ss_net* n, int B) {
  if (!n) return nfail(SS_ERR_ARG, "net is NULL");
  if (B < 1 || B > n->maxB) return nfail(SS_ERR_ARG, "batch must be in [1, max_batch]");
  return SS_OK;
}

void net_free(ss_net* n) {
  if (!n) return;
  if (n->stream) cudaStreamSynchronize(n->stream);
  if (n->base) cudaFree(n->base);
  if (n->h_loss) cudaFreeHost(n->h_loss);
  if (n->h_err) cudaFreeHost(n->h_err);
  if (n->side) {
    cudaStreamSynchronize(n->side);
    cudaStreamDestroy(n->side);
  }
  for (cudaEvent_t e : {n->ev_start, n->ev_x[0], n->ev_x[1], n->ev_w[0], n->ev_w[1]})
    if (e) cudaEventDestroy(e);
  if (n->own_stream && n->stream) cudaStreamDestroy(n->stream);
  delete n;
}

}  // namespace

extern "C" int ss_net_create(ss_net** out, int theory, int size, int max_batch, unsigned long long seed,
                             void* cuda_stream) {
  if (!out) return nfail(SS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (theory != SS_ABELIAN_HIGGS && theory != SS_CHIRAL_MAGNET) return nfail(SS_ERR_ARG, "unknown theory");
  if (size < 128 || size % 128 != 0 || size > 4096)
    return nfail(SS_ERR_ARG, "size must be a multiple of 128 in [128, 4096]");
  if (max_batch < 1 || (long long)max_batch * size * size > (1LL << 28))
    return nfail(SS_ERR_ARG, "max_batch must be >= 1 with max_batch * size^2 <= 2^28");
  ss_net* n = new (std::nothrow) ss_net();
  if (!n) return nfail(SS_ERR_NOMEM, "host allocation failed");
  n->theory = theory;
  n->C = theory == SS_ABELIAN_HIGGS ? 4 : 3;
  n->ncoup = theory == SS_ABELIAN_HIGGS ? 1 : 0;
  n->S = size;
  n->maxB = max_batch;
  if (cuda_stream) {
    n->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete n;
      return nfail(SS_ERR_CUDA, "stream creation failed");
    }
    n->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&n->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&n->ev_start, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&n->ev_x[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&n->ev_x[1], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&n->ev_w[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&n->ev_w[1], cudaEventDisableTiming) != cudaSuccess) {
    net_free(n);
    return nfail(SS_ERR_CUDA, "stream or event creation failed");
  }
  // parameter layout: per layer W [cout][9][cin] then b [cout]
  long long off = 0, wo = 0;
  for (int L = 0; L < NL; ++L) {
    LayerView& v = n->T.l[L];
    v.cin = LAYERS[L].cin;
    v.cout = LAYERS[L].cout;
    v.woff = off;
    v.boff = off + 9LL * v.cin * v.cout;
    off = v.boff + v.cout;
    v.wbo = wo;
    v.wto = wo + 9LL * v.cin * v.cout;
    wo = v.wto + 9LL * v.cin * v.cout;
  }
  n->nparam = off;
  n->nwbf = wo;

  // one allocation for everything
  const long long B = max_batch, S = size, P0 = B * S * S;
  std::vector<std::pair<void**, size_t>> plan;
  auto add = [&](void** p, size_t bytes) { plan.push_back({p, (bytes + 255) & ~size_t(255)}); };
  add((void**)&n->theta, sizeof(float) * off);
  add((void**)&n->grad, sizeof(float) * off);
  add((void**)&n->m, sizeof(float) * off);
  add((void**)&n->v, sizeof(float) * off);
  add((void**)&n->wbf, sizeof(__nv_bfloat16) * wo);
  add((void**)&n->err, 256);
  add((void**)&n->loss, 256);
  add((void**)&n->coup, sizeof(float) * (B * 4 + 8));
  struct ActSpec {
    Act* a;
    int level, C;
  };
  const ActSpec acts[] = {{&n->in0, 0, 16},  {&n->e1a, 0, 16}, {&n->cat1, 0, 48}, {&n->p1, 1, 16}, {&n->e2a, 1, 32},
                          {&n->cat2, 1, 80}, {&n->p2, 2, 32},  {&n->e3a, 2, 48},  {&n->cat3, 2, 144}, {&n->p3, 3, 48},
                          {&n->b1, 3, 96},   {&n->bb, 3, 96},  {&n->d3a, 2, 48},  {&n->d3, 2, 48},  {&n->d2a, 1, 32},
                          {&n->d2, 1, 32},   {&n->d1a, 0, 16}, {&n->d1, 0, 16}};
  for (const ActSpec& a : acts) {
    const long long h = S >> a.level;
    *a.a = Act{nullptr, (int)B, (int)h, (int)h, a.C, a.C, 0};
    add(&a.a->p, sizeof(__nv_bfloat16) * B * h * h * a.C);
  }
  add((void**)&n->out, sizeof(float) * P0 * COUT_LAST);
  struct GSpec {
    float** g;
    int level, C;
  };
  const GSpec gs[] = {{&n->g_out, 0, 16}, {&n->g_d1, 0, 16},  {&n->g_d1a, 0, 16}, {&n->g_cat1, 0, 48},
                      {&n->g_d2, 1, 32},  {&n->g_d2a, 1, 32}, {&n->g_cat2, 1, 80}, {&n->g_d3, 2, 48},
                      {&n->g_d3a, 2, 48}, {&n->g_cat3, 2, 144}, {&n->g_b, 3, 96},  {&n->g_b1, 3, 96},
                      {&n->g_p3, 3, 48},  {&n->g_e3, 2, 48},  {&n->g_e3a, 2, 48}, {&n->g_p2, 2, 32},
                      {&n->g_e2, 1, 32},  {&n->g_e2a, 1, 32}, {&n->g_p1, 1, 16},  {&n->g_e1, 0, 16},
                      {&n->g_e1a, 0, 16}};
  for (const GSpec& g : gs) {
    const long long h = S >> g.level;
    add((void**)g.g, sizeof(float) * B * h * h * g.C);
  }
  add(&n->dyb, sizeof(__nv_bfloat16) * P0 * 16);
  add(&n->dyT, sizeof(__nv_bfloat16) * P0 * 16);
  add(&n->dyb1, sizeof(__nv_bfloat16) * P0 * 16);
  add(&n->dyT1, sizeof(__nv_bfloat16) * P0 * 16);
  add(&n->xT, sizeof(__nv_bfloat16) * P0 * 3 * 48);
  add(&n->xT1, sizeof(__nv_bfloat16) * P0 * 3 * 48);
  size_t total = 0;
  for (auto& e : plan) total += e.second;
  if (cudaMalloc(&n->base, total) != cudaSuccess) {
    net_free(n);
    return nfail(SS_ERR_NOMEM, "device allocation of " + std::to_string(total) + " bytes failed");
  }
  char* q = static_cast<char*>(n->base);
  for (auto& e : plan) {
    *e.first = q;
    q += e.second;
  }
  if (cudaMallocHost(&n->h_loss, sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&n->h_err, sizeof(int)) != cudaSuccess) {
    net_free(n);
    return nfail(SS_ERR_NOMEM, "pinned host allocation failed");
  }
  // zero-initialised state (this also zeroes the unused output channels' weights)
  if (cudaMemsetAsync(n->base, 0, total, n->stream) != cudaSuccess) {
    net_free(n);
    return nfail(SS_ERR_CUDA, "memset failed");
  }
  // He-normal weights (std sqrt(2 / fan_in), fan_in over the channels that carry
  // data), zero biases; the last layer starts at zero so the initial correction is 0
  std::vector<float> h((size_t)off, 0.f);
  Rng rng{seed};
  for (int L = 0; L < NL - 1; ++L) {
    const LayerView& v = n->T.l[L];
    const int fan_cin = L == 0 ? n->C + n->ncoup : v.cin;
    const double sd = std::sqrt(2.0 / (9.0 * fan_cin));
    for (int co = 0; co < v.cout; ++co)
      for (int tap = 0; tap < 9; ++tap)
        for (int ci = 0; ci < v.cin; ++ci) {
          const double z = rng.normal();
          if (L == 0 && ci >= fan_cin) continue;
          h[(size_t)(v.woff + ((long long)co * 9 + tap) * v.cin + ci)] = (float)(sd * z);
        }
  }
  if (cudaMemcpyAsync(n->theta, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice, n->stream) != cudaSuccess ||
      pack_weights(n) != SS_OK || cudaStreamSynchronize(n->stream) != cudaSuccess) {
    net_free(n);
    return nfail(SS_ERR_CUDA, "weight initialisation failed");
  }
  *out = n;
  return SS_OK;
}

extern "C" int ss_net_destroy(ss_net* n) {
  net_free(n);
  return SS_OK;
}

extern "C" const char* ss_net_last_error(void) { return g_net_err.c_str(); }

extern "C" long long ss_net_num_params(const ss_net* n) { return n ? n->nparam : -1; }

extern "C" int ss_net_get_params(ss_net* n, float* host_out) {
  if (!n || !host_out) return nfail(SS_ERR_ARG, "NULL argument");
  NET_CK(cudaMemcpyAsync(host_out, n->theta, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost, n->stream));
  NET_CK(cudaStreamSynchronize(n->stream));
  return SS_OK;
}

extern "C" int ss_net_set_params(ss_net* n, const float* host_in) {
  if (!n || !host_in) return nfail(SS_ERR_ARG, "NULL argument");
  NET_CK(cudaMemcpyAsync(n->theta, host_in, sizeof(float) * n->nparam, cudaMemcpyHostToDevice, n->stream));
  int rc = pack_weights(n);
  if (rc) return rc;
  NET_CK(cudaStreamSynchronize(n->stream));
  return SS_OK;
}

// Input packing without the host synchronisation of the public call (the coupling
// values are staged in the network's own device buffer).
int pack(ss_net* n, const float* fields, const double* couplings, int batch, void* input) {
  if (n->ncoup > 0) {
    if (!couplings) return nfail(SS_ERR_ARG, "couplings are required for this theory");
    std::vector<float> c((size_t)batch * n->ncoup);
    for (size_t i = 0; i < c.size(); ++i) c[i] = (float)couplings[i];
    NET_CK(cudaMemcpyAsync(n->coup, c.data(), sizeof(float) * c.size(), cudaMemcpyHostToDevice, n->stream));
    NET_CK(cudaStreamSynchronize(n->stream));  // the staging vector goes out of scope
  }
  k_pack_input<<<grid_of((size_t)batch * n->S * n->S), 256, 0, n->stream>>>(
      fields, n->C, n->coup, n->ncoup, batch, n->S, static_cast<__nv_bfloat16*>(input));
  NET_CK(cudaGetLastError());
  return SS_OK;
}

extern "C" int ss_net_pack(ss_net* n, const float* fields, const double* couplings, int batch, void* input) {
  int rc = check_batch(n, batch);
  if (rc) return rc;
  if (!fields || !input) return nfail(SS_ERR_ARG, "NULL argument");
  if ((rc = pack(n, fields, couplings, batch, input))) return rc;
  NET_CK(cudaStreamSynchronize(n->stream));
  return SS_OK;
}

extern "C" int ss_net_forward(ss_net* n, const float* ansatz, const double* couplings, int batch, float* out) {
  int rc = check_batch(n, batch);
  if (rc) return rc;
  if (!ansatz) return nfail(SS_ERR_ARG, "ansatz is NULL");
  if ((rc = pack(n, ansatz, couplings, batch, n->in0.p))) return rc;
  if ((rc = forward(n, batch))) return rc;
  if (out)
    NET_CK(cudaMemcpyAsync(out, n->out, sizeof(float) * (size_t)batch * n->S * n->S * COUT_LAST,
                           cudaMemcpyDeviceToDevice, n->stream));
  return check_err(n);
}

// Loss and parameter gradient at the current weights (no update).
extern "C" int ss_net_gradients(ss_net* n, const float* ansatz, const double* couplings, const float* relaxed,
                                int batch, float* grad_out, double* loss_out) {
  int rc = check_batch(n, batch);
  if (rc) return rc;
  if (!ansatz || !relaxed) return nfail(SS_ERR_ARG, "NULL argument");
  if ((rc = pack(n, ansatz, couplings, batch, n->in0.p))) return rc;
  if ((rc = forward(n, batch))) return rc;
  NET_CK(cudaMemsetAsync(n->loss, 0, sizeof(double), n->stream));
  k_mse<<<grid_of((size_t)batch * n->S * n->S), 256, 0, n->stream>>>(n->out, ansatz, relaxed, n->C, batch, n->S,
                                                                      n->g_out, n->loss);
  NET_CK(cudaGetLastError());
  if ((rc = backward(n, batch))) return rc;
  if (grad_out)
    NET_CK(cudaMemcpyAsync(grad_out, n->grad, sizeof(float) * n->nparam, cudaMemcpyDeviceToDevice, n->stream));
  NET_CK(cudaMemcpyAsync(n->h_loss, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
  if ((rc = check_err(n))) return rc;
  if (loss_out) *loss_out = *n->h_loss;
  return SS_OK;
}

// One Adam update of the parameters from the gradient `g` (device, nparam floats),
// then the BF16 weight copies are re-packed.
static int adam_update(ss_net* n, const float* g, float lr) {
  n->t += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - std::pow(b1, (double)n->t)), c2 = (float)(1.0 - std::pow(b2, (double)n->t));
  k_adam<<<grid_of((size_t)n->nparam), 256, 0, n->stream>>>(n->theta, g, n->m, n->v, n->nparam, lr, (float)b1,
                                                            (float)b2, (float)(1.0 - b1), (float)(1.0 - b2), 1e-8f,
                                                            c1, c2);
  NET_CK(cudaGetLastError());
  return pack_weights(n);
}

extern "C" int ss_net_train_step(ss_net* n, const float* ansatz, const double* couplings, const float* relaxed,
                                 int batch, float lr, double* loss_out) {
  if (!(lr > 0.f) || !std::isfinite(lr)) return nfail(SS_ERR_ARG, "lr must be positive and finite");
  int rc = ss_net_gradients(n, ansatz, couplings, relaxed, batch, nullptr, loss_out);
  if (rc) return rc;
  return adam_update(n, n->grad, lr);
}

extern "C" int ss_net_apply_gradients(ss_net* n, const float* grad, float lr) {
  if (!n || !grad) return nfail(SS_ERR_ARG, "NULL argument");
  if (!(lr > 0.f) || !std::isfinite(lr)) return nfail(SS_ERR_ARG, "lr must be positive and finite");
  int rc = adam_update(n, grad, lr);
  if (rc) return rc;
  return check_err(n);
}

extern "C" int ss_net_get_optimizer_state(ss_net* n, float* m_host, float* v_host, long long* steps) {
  if (!n) return nfail(SS_ERR_ARG, "NULL argument");
  if (m_host) NET_CK(cudaMemcpyAsync(m_host, n->m, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost, n->stream));
  if (v_host) NET_CK(cudaMemcpyAsync(v_host, n->v, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost, n->stream));
  NET_CK(cudaStreamSynchronize(n->stream));
  if (steps) *steps = n->t;
  return SS_OK;
}

extern "C" int ss_net_predict(ss_net* n, const float* ansatz, const double* couplings, int batch, float* init) {
  int rc = check_batch(n, batch);
  if (rc) return rc;
  if (!ansatz || !init) return nfail(SS_ERR_ARG, "NULL argument");
  if ((rc = pack(n, ansatz, couplings, batch, n->in0.p))) return rc;
  if ((rc = forward(n, batch))) return rc;
  k_apply<<<grid_of((size_t)batch * n->S * n->S), 256, 0, n->stream>>>(
      ansatz, n->out, n->C, batch, n->S, n->theory == SS_CHIRAL_MAGNET, init);
  NET_CK(cudaGetLastError());
  return check_err(n);
}

extern "C" int ss_net_save(ss_net* n, const char* path) {
  if (!n || !path) return nfail(SS_ERR_ARG, "NULL argument");
  std::vector<float> h((size_t)n->nparam);
  int rc = ss_net_get_params(n, h.data());
  if (rc) return rc;
  FILE* f = std::fopen(path, "wb");
  if (!f) return nfail(SS_ERR_ARG, std::string("cannot open ") + path);
  const int32_t hdr[4] = {(int32_t)NET_MAGIC, n->theory, n->S, 1};
  const int64_t np = n->nparam;
  bool ok = std::fwrite(hdr, sizeof(hdr), 1, f) == 1 && std::fwrite(&np, sizeof(np), 1, f) == 1 &&
            std::fwrite(h.data(), sizeof(float), h.size(), f) == h.size();
  ok = (std::fclose(f) == 0) && ok;
  return ok ? SS_OK : nfail(SS_ERR_ARG, std::string("write failed: ") + path);
}

extern "C" int ss_net_load(ss_net* n, const char* path) {
  if (!n || !path) return nfail(SS_ERR_ARG, "NULL argument");
  FILE* f = std::fopen(path, "rb");
  if (!f) return nfail(SS_ERR_ARG, std::string("cannot open ") + path);
  int32_t hdr[4];
  int64_t np = 0;
  std::vector<float> h((size_t)n->nparam);
  bool ok = std::fread(hdr, sizeof(hdr), 1, f) == 1 && std::fread(&np, sizeof(np), 1, f) == 1;
  ok = ok && hdr[0] == (int32_t)NET_MAGIC && hdr[1] == n->theory && np == n->nparam &&
       std::fread(h.data(), sizeof(float), h.size(), f) == h.size();
  std::fclose(f);
  if (!ok) return nfail(SS_ERR_ARG, std::string("not a network file of this theory and shape: ") + path);
  return ss_net_set_params(n, h.data());
}

// Direct access to the tensor-core convolutions, for testing them in isolation.
extern "C" int ss_conv3x3(const void* x, int N, int H, int W, int Cin, const void* w, int Cout, const float* bias,
                          int mode, void* out, void* cuda_stream) {
  if (!x || !w || !out || (mode != CONV_F32 && !bias)) return nfail(SS_ERR_ARG, "NULL argument");
  if (mode < 0 || mode > 2) return nfail(SS_ERR_ARG, "mode must be 0, 1 or 2");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int* d_err = nullptr;
  NET_CK(cudaMalloc(&d_err, sizeof(int)));
  Act xa{const_cast<void*>(x), N, H, W, Cin, Cin, 0};
  Act oa{out, N, H, W, Cout, Cout, 0};
  int h = 0;
  cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = conv3x3_tc(xa, w, Cout, mode, bias, oa, d_err, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_err);
  if (e != cudaSuccess) return nfail(e == cudaErrorInvalidValue ? SS_ERR_ARG : SS_ERR_CUDA,
                                     std::string("ss_conv3x3: ") + cudaGetErrorString(e));
  if (h) return nfail(SS_ERR_TIMEOUT, "ss_conv3x3: a wait gave up (code " + std::to_string(h) + ")");
  return SS_OK;
}

extern "C" int ss_conv3x3_wgrad(const void* dy, const void* x, int N, int H, int W, int Cout, int Cin, float* dw,
                                void* cuda_stream) {
  if (!dy || !x || !dw) return nfail(SS_ERR_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const size_t P = (size_t)N * H * W;
  void *dyT = nullptr, *xT = nullptr, *dyb = nullptr;
  float* db = nullptr;
  int* d_err = nullptr;
  NET_CK(cudaMalloc(&d_err, sizeof(int)));
  NET_CK(cudaMalloc(&dyT, P * Cout * 2));
  NET_CK(cudaMalloc(&dyb, P * Cout * 2));
  NET_CK(cudaMalloc(&xT, P * Cin * 2 * 3));
  NET_CK(cudaMalloc(&db, sizeof(float) * Cout));
  NET_CK(cudaMemsetAsync(d_err, 0, sizeof(int), s));
  NET_CK(cudaMemsetAsync(dw, 0, sizeof(float) * 9 * Cin * Cout, s));
  NET_CK(cudaMemsetAsync(db, 0, sizeof(float) * Cout, s));
  Act xa{const_cast<void*>(x), N, H, W, Cin, Cin, 0};
  cudaError_t e = relu_grad(static_cast<const float*>(dy), nullptr, N, H, W, Cout, dyb, dyT, db, s);
  if (e == cudaSuccess) e = shifted_transpose(xa, xT, s);
  if (e == cudaSuccess) e = wgrad3x3_tc(dyT, xT, N, H, W, Cout, Cin, dw, d_err, s);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dyT);
  cudaFree(dyb);
  cudaFree(xT);
  cudaFree(db);
  cudaFree(d_err);
  if (e != cudaSuccess) return nfail(e == cudaErrorInvalidValue ? SS_ERR_ARG : SS_ERR_CUDA,
                                     std::string("ss_conv3x3_wgrad: ") + cudaGetErrorString(e));
  if (h) return nfail(SS_ERR_TIMEOUT, "ss_conv3x3_wgrad: a wait gave up (code " + std::to_string(h) + ")");
  return SS_OK;
}

extern "C" int ss_wait_selftest(int limit_us, void* cuda_stream) {
  if (limit_us < 1 || limit_us > 1000000) return nfail(SS_ERR_ARG, "limit_us must be in 1..1000000");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int* d_err = nullptr;
  NET_CK(cudaMalloc(&d_err, sizeof(int)));
  int h = 0;
  cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = wait_selftest((uint64_t)limit_us * 1000ull, d_err, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_err);
  if (e != cudaSuccess) return nfail(SS_ERR_CUDA, std::string("ss_wait_selftest: ") + cudaGetErrorString(e));
  if (h) return nfail(SS_ERR_TIMEOUT, "ss_wait_selftest: the wait gave up as it must (code " + std::to_string(h) + ")");
  return nfail(SS_ERR_STATE, "ss_wait_selftest: the wait completed although nothing signals it");
}
