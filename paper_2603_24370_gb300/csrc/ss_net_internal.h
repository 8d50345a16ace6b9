// ss_net_internal.h -- launch interfaces of the learned initialiser's kernels
// (ss_conv.cu: tensor-core convolutions; ss_netops.cu: the memory-bound layers).
//
// Activations are NHWC BF16 with the channel count a multiple of 16; a tensor may be
// a channel slice [off, off + C) of a wider buffer of `cs` channels per pixel (the
// decoder's concatenations are such buffers). Convolutions are 3x3, stride 1, zero
// padding 1. Weights are stored [Cout][tap][Cin] with tap = 3 (dy + 1) + (dx + 1).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace ss {

// An NHWC BF16 (or FP32) activation view.
struct Act {
  void* p = nullptr;  // buffer base
  int N = 0, H = 0, W = 0;
  int C = 0;    // channels of the view
  int cs = 0;   // channels per pixel of the buffer
  int off = 0;  // first channel of the view
};

enum ConvMode {
  CONV_BF16_BIAS_RELU = 0,  // out (bf16) = relu(acc + bias)
  CONV_F32_BIAS = 1,        // out (fp32) = acc + bias
  CONV_F32 = 2,             // out (fp32) = acc          (input gradients)
  CONV_GRAD_RELU = 3,       // input gradient through the previous layer's ReLU (GradRelu)
};

// CONV_GRAD_RELU: g = acc * (mask > 0) (mask: that layer's BF16 output, the view read
// as this convolution's output shape) goes out as BF16 NHWC (out), BF16 channel-major
// dyT [Cout][N][H][W], and its sum over pixels is added to dbias [Cout]: what
// relu_grad makes of the FP32 input gradient, without writing it.
struct GradRelu {
  Act mask;
  void* dyT = nullptr;
  float* dbias = nullptr;
};

// out[n, y, x, co] = epilogue( sum_{tap, ci} x[n, y + dy, x + dx, ci] * w[co, tap, ci] )
// w: BF16 [Cout][9 * Cin] (K ordering tap-major). Cout must be one of 16, 32, 48, 80,
// 96, 144; Cin a multiple of 16; H * W a multiple of 128 with W a multiple of 32 (W < 128)
// or of 128. `err` (device int) is set non-zero when a wait in the kernel gives up.
cudaError_t conv3x3_tc(const Act& x, const void* w, int Cout, int mode, const float* bias, const Act& out, int* err,
                       cudaStream_t s, const GradRelu* gr = nullptr);

// dw[co, tap, ci] += sum_{n, y, x} dyT[co, n, y, x] * xT[dx][ci, n, y + dy, x]
// dyT: BF16 [Cout][N][H][W]; xT: BF16 [3][Cin][N][H][W], copy dx + 1 holding the
// input shifted by dx along x (zero where x + dx leaves the image). dw: FP32
// [Cout][9][Cin], accumulated with atomics (zero it first). Cin one of 16, 32, 48,
// 80, 96, 144; Cout <= 128; N * H * W a multiple of 16, W a multiple of 8.
cudaError_t wgrad3x3_tc(const void* dyT, const void* xT, int N, int H, int W, int Cout, int Cin, float* dw, int* err,
                        cudaStream_t s);

// The kernels' bounded mbarrier wait on a barrier nothing completes: records code 99
// in `err` after limit_ns (tests the time-out path without stalling the device).
cudaError_t wait_selftest(uint64_t limit_ns, int* err, cudaStream_t s);

// ---- memory-bound layers (ss_netops.cu)
// xT[dx + 1][c, n, y, x] = x[n, y, x + dx, c] (0 outside), dx = -1, 0, 1.
cudaError_t shifted_transpose(const Act& x, void* xT, cudaStream_t s);
// dyT[c, n, y, x] = bf16(dy[n, y, x, c] * (mask ? (y_act[n, y, x, c] > 0) : 1)) and
// dy_bf16 (NHWC, C channels) the same values: the input of the input-gradient
// convolution. dy: FP32 NHWC with C channels; y_act: the layer's BF16 output view.
cudaError_t relu_grad(const float* dy, const Act* y_act, int N, int H, int W, int C, void* dy_bf16, void* dyT,
                      float* dbias, cudaStream_t s);
// out = 2x2 average of x (out spatial size H/2 x W/2)
cudaError_t avgpool2(const Act& x, const Act& out, cudaStream_t s);
// dx (FP32 NHWC, C channels) += dout / 4 broadcast over each 2x2 block
cudaError_t avgpool2_backward(const float* dout, int N, int Ho, int Wo, int C, float* dx, cudaStream_t s);
// out (view at 2H x 2W) = nearest-neighbour x2 upsampling of x
cudaError_t upsample2(const Act& x, const Act& out, cudaStream_t s);
// dx (FP32 NHWC, C channels, H x W) = sum over each 2x2 block of the slice [off, off + C)
// of dup (FP32, cs channels per pixel, 2H x 2W)
cudaError_t upsample2_backward(const float* dup, int cs, int off, int N, int H, int W, int C, float* dx,
                               cudaStream_t s);
// dst (FP32 NHWC, C channels) += slice [off, off + C) of src (FP32, cs channels)
cudaError_t add_slice(const float* src, int cs, int off, int N, int H, int W, int C, float* dst, cudaStream_t s);

}  // namespace ss
