/* soliton_net.h -- C-ABI of the learned initialiser of libsoliton.so.
 *
 * The paper starts every relaxation from a model-specific ansatz (Sec. 4.1, the
 * "initial field" step of the workflow) and lets the arrested Newton flow (Sec. 3.2)
 * do all of the work. It has no learned component. This part adds one: a
 * convolutional U-Net, trained on configurations that the flow itself relaxed, maps
 * an ansatz (and the couplings) to a correction; ansatz + correction is the initial
 * field, the flow then finishes the solve as before and remains the judge of energy
 * and charge (starting from the plain ansatz is the fallback).
 *
 * Network: 4 levels with 16, 32, 48, 96 channels, two 3x3 convolutions per level
 * (ReLU), 2x2 average pooling, nearest x2 upsampling, skip concatenations, a final
 * linear 3x3 convolution; 304,720 parameters (the last layer computes 16 channels,
 * those beyond C keep zero weights). Inputs: the field components (Abelian
 * Higgs: Re psi, Im psi, A_1, A_2; chiral magnet: n_1, n_2, n_3) and one constant
 * plane per coupling (Abelian Higgs: lambda), BF16, zero-padded to 16 channels.
 * Convolutions run on the tensor cores with BF16 operands and FP32 accumulation;
 * parameters and the Adam state are FP32.
 *
 * Layouts. Fields: FP32, a batch of B problems of size x size sites each, SoA planes
 * [B][C][size][size] (x fastest), the solver's layout, halo included. Network input:
 * BF16 NHWC [B][size][size][16]. Network output: FP32 NHWC [B][size][size][16], the
 * first C channels are the correction. All pointers marked "device" are device
 * memory owned by the caller and must stay valid until the call returns. Every call
 * is ordered on the network's stream and returns after its results are complete,
 * unless stated otherwise. Return codes as in soliton.h.
 */
#ifndef SOLITON_NET_H
#define SOLITON_NET_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ss_net ss_net;

/* Create a network for `theory` (SS_ABELIAN_HIGGS: C = 4, one coupling lambda;
 * SS_CHIRAL_MAGNET: C = 3, no coupling plane, outputs renormalised to |n| = 1) on
 * size x size grids (size a multiple of 128, 128..4096), for batches of up to
 * max_batch problems (max_batch * size^2 <= 2^28). Weights are He-normal from a
 * SplitMix64 stream seeded by `seed`, biases zero, the last layer zero (the initial
 * correction is 0). `cuda_stream`: borrowed cudaStream_t, or NULL for a private
 * stream. The network owns all device memory it allocates (parameters, Adam state,
 * activations and gradients for max_batch), freed by ss_net_destroy.
 * Errors: SS_ERR_ARG, SS_ERR_NOMEM, SS_ERR_CUDA. */
int ss_net_create(ss_net** out, int theory, int size, int max_batch, unsigned long long seed, void* cuda_stream);
int ss_net_destroy(ss_net* net);
/* Message of the last failed ss_net_* call of this thread. */
const char* ss_net_last_error(void);
/* Number of FP32 parameters (layer by layer: W[cout][9][cin], then b[cout]). */
long long ss_net_num_params(const ss_net* net);
/* Copy the parameters to / from a host array of ss_net_num_params floats. */
int ss_net_get_params(ss_net* net, float* host_out);
int ss_net_set_params(ss_net* net, const float* host_in);
/* Save / load the parameters (binary: magic, theory, size, version, count, FP32
 * values). Loading checks theory and parameter count. Errors: SS_ERR_ARG. */
int ss_net_save(ss_net* net, const char* path);
int ss_net_load(ss_net* net, const char* path);

/* Network input (device, BF16 NHWC [batch][size][size][16]) from fields (device,
 * FP32 SoA [batch][C][size][size]) and `couplings` (host, batch values for the
 * Abelian Higgs lambda; may be NULL for the chiral magnet). */
int ss_net_pack(ss_net* net, const float* fields, const double* couplings, int batch, void* input);
/* Forward pass on the input packed from `ansatz` (device, FP32 SoA) and `couplings`
 * (as ss_net_pack); `out` (device, FP32 NHWC [batch][size][size][16]) may be NULL. */
int ss_net_forward(ss_net* net, const float* ansatz, const double* couplings, int batch, float* out);
/* Loss = mean over the interior sites (the halo of width 2 excluded) and the first
 * C channels of (output - (relaxed - ansatz))^2, where the output is the network's
 * on the input packed from `ansatz` and `couplings`, and `relaxed` (device, FP32 SoA
 * [batch][C][size][size]) is the flow's relaxed field of the same problems; its
 * gradient with respect to every parameter into `grad_out` (device,
 * ss_net_num_params floats; may be NULL) and the loss into *loss_out (host; may be
 * NULL). The weights are not changed. */
int ss_net_gradients(ss_net* net, const float* ansatz, const double* couplings, const float* relaxed, int batch,
                     float* grad_out, double* loss_out);
/* ss_net_gradients followed by one Adam update (beta1 0.9, beta2 0.999, eps 1e-8,
 * bias-corrected) with learning rate lr. The update is enqueued on the network's
 * stream and completes before the next call on it. */
int ss_net_train_step(ss_net* net, const float* ansatz, const double* couplings, const float* relaxed, int batch,
                      float lr, double* loss_out);
/* One Adam update (the same as ss_net_train_step's) from a caller-supplied gradient
 * `grad` (device, ss_net_num_params floats, read only), e.g. gradients accumulated
 * over several batches or summed across ranks. Adam (Kingma & Ba 2015, Algorithm 1)
 * in FP32: m <- 0.9 m + 0.1 g, v <- 0.999 v + 0.001 g^2, theta <- theta - lr
 * (m / (1 - 0.9^t)) / (sqrt(v / (1 - 0.999^t)) + 1e-8), t the update count from 1.
 * The paper has no learned part; this call serves the network's training. Enqueued
 * on the network's stream; returns after the update has completed. Errors:
 * SS_ERR_ARG (NULL, lr not positive and finite), SS_ERR_CUDA. */
int ss_net_apply_gradients(ss_net* net, const float* grad, float lr);
/* Copy the Adam moments m and v (host arrays of ss_net_num_params floats; either may
 * be NULL) and the number of updates taken (may be NULL). Synchronises the stream. */
int ss_net_get_optimizer_state(ss_net* net, float* m_host, float* v_host, long long* steps);
/* Initial fields (device, FP32 SoA [batch][C][size][size]) = ansatz + correction on
 * the interior, the ansatz itself on the halo (the Dirichlet values stay exact);
 * chiral magnet: renormalised to unit length. `ansatz` (device) in the same layout. */
int ss_net_predict(ss_net* net, const float* ansatz, const double* couplings, int batch, float* init);

/* The tensor-core convolution on its own (no counterpart in the paper; for testing):
 * out[n,y,x,co] = sum_{dy,dx,ci} x[n,y+dy,x+dx,ci] w[co,3(dy+1)+(dx+1),ci] (zero
 * padding), then mode 0: relu(. + bias) stored BF16; 1: . + bias stored FP32; 2: .
 * stored FP32 (bias unused). x: device BF16 NHWC [N][H][W][Cin], Cin a multiple of
 * 16; w: device BF16 [Cout][9][Cin]; Cout in {16, 32, 48, 80, 96, 144}; W a multiple
 * of 128, or W in {8, 16, 32, 64}; H * W a multiple of 128; out: device NHWC with
 * Cout channels. Synchronises `cuda_stream`. Errors: SS_ERR_ARG, SS_ERR_CUDA,
 * SS_ERR_TIMEOUT (a bounded wait inside the kernel gave up). */
int ss_conv3x3(const void* x, int N, int H, int W, int Cin, const void* w, int Cout, const float* bias, int mode,
               void* out, void* cuda_stream);
/* Weight gradient of that convolution: dw[co,tap,ci] = sum_{n,y,x} bf16(dy[n,y,x,co])
 * x[n,y+dy_tap,x+dx_tap,ci]. dy: device FP32 NHWC [N][H][W][Cout] (rounded to BF16
 * before the contraction), x: device BF16 NHWC [N][H][W][Cin], dw: device FP32
 * [Cout][9][Cin] (overwritten). Cin in {16, 32, 48, 80, 96, 144}, Cout <= 128, W a
 * multiple of 8, N H W a multiple of 16. Synchronises `cuda_stream`. */
int ss_conv3x3_wgrad(const void* dy, const void* x, int N, int H, int W, int Cout, int Cin, float* dw,
                     void* cuda_stream);

/* Self-test of the failure path (no counterpart in the paper): runs the bounded
 * mbarrier wait that every tensor-core kernel uses, on a barrier that nothing
 * completes, with a limit of limit_us microseconds (1..1e6). The wait gives up, the
 * kernel records the failure and returns, and the call reports SS_ERR_TIMEOUT, the
 * code the network calls return when one of their waits gives up; the device stays
 * usable. Returns SS_ERR_STATE if the wait completed. Synchronises `cuda_stream`. */
int ss_wait_selftest(int limit_us, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SOLITON_NET_H */
