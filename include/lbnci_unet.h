/*
 * lbnci_unet.h -- C ABI of the warm-start surrogate: a convolutional U-Net (Ronneberger,
 * Fischer and Brox, MICCAI 2015) with BF16 weights and activations, FP32 accumulation,
 * trained with Adam (Kingma and Ba, ICLR 2015) by the library's own forward and backward
 * kernels (sm_103a).
 *
 * The paper (arXiv:2003.11069) has no surrogate: the network only predicts a relaxed
 * packed-emulsion state (order parameter psi and velocity) from which the lattice
 * Boltzmann step of lbnci.h is started; the lattice Boltzmann run then continues to
 * convergence and remains the judge of the prediction.
 *
 * Network (levels L, base width C): widths C_l = C 2^l, l = 0..L-1.
 *   encoder l < L-1 : conv3x3 + ReLU, conv3x3 + ReLU (= skip_l), 2x2 max pool
 *   bottom  l = L-1 : conv3x3 + ReLU, conv3x3 + ReLU
 *   decoder l = L-2..0 : nearest 2x upsampling, conv3x3 to C_l + ReLU,
 *                        concatenation [that output, skip_l], conv3x3 + ReLU, conv3x3 + ReLU
 *   head : 1x1 convolution to out_ch channels (no activation), FP32 output.
 * Every 3x3 convolution pads with zeros beyond the first and last image row (the channel
 * walls) and periodically along x (the flow direction). Max-pool ties go to the first
 * element of the window in the order (0,0), (0,1), (1,0), (1,1).
 *
 * Images are NHWC FP32 arrays x[b][y][x][c] (c fastest), b < batch, y < H, x < W.
 *
 * Parameters are one flat FP32 vector: for each layer in the order enc0a, enc0b, ...,
 * enc{L-1}a, enc{L-1}b, then for l = L-2 down to 0: up_l, dec_la, dec_lb, then head --
 * the weight (3x3: [C_out][3][3][C_in], taps (dy, dx) = -1..+1; head: [C_out][C_in])
 * followed by the bias [C_out]. Weights are rounded to BF16 for the kernels; the FP32
 * vector is the master copy that Adam updates.
 *
 * Loss: L = (1/P) sum_p sum_j lam_j (y_pj - t_pj)^2, P = batch H W pixels.
 * Adam: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; theta -= lr mh/(sqrt(vh) + eps) with
 * mh = m/(1-b1^t), vh = v/(1-b2^t), t = the number of updates so far.
 *
 * Errors: every call returns an lb_status (lbnci.h); nothing aborts or traps. A handle is
 * not thread-safe. All work is enqueued on the configured stream; calls that return host
 * values synchronise it.
 */
#ifndef LBNCI_UNET_H
#define LBNCI_UNET_H

#include <stddef.h>

#include "lbnci.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int levels;     /* resolution levels L, 2..6 */
  int base;       /* channels at the finest level, a multiple of 32 */
  int in_ch;      /* input channels, 1..32 */
  int out_ch;     /* output channels, 1..8 */
  int H, W;       /* image size; multiples of 2^(L-1) */
  int max_batch;  /* largest batch any call may pass (sizes the activation buffers) */
  void* stream;   /* cudaStream_t; NULL = legacy default stream */
} lbu_config;

typedef struct lbu_net lbu_net;

/* Number of layers and the weight shape of layer i: {C_out, kh, kw, C_in} (kh = kw = 1 for
 * the head). Pure host functions. */
int lbu_layer_count(const lbu_config* cfg);
lb_status lbu_layer_shape(const lbu_config* cfg, int layer, int shape[4]);
/* Total number of FP32 parameters (weights and biases). */
lb_status lbu_param_count(const lbu_config* cfg, long long* count);

/* Create a network on the current CUDA device; parameters start at zero. The library
 * owns every buffer it allocates (about max_batch * H * W * 1.1 KB at base 32). */
lb_status lbu_create(const lbu_config* cfg, lbu_net** out);
void lbu_destroy(lbu_net* net);
const char* lbu_last_error(const lbu_net* net);
/* Kernel launches enqueued by this handle so far. */
long long lbu_kernel_launches(const lbu_net* net);

/* Copy the flat FP32 parameter vector in or out (host or device pointer) and reset the
 * Adam state (moments and step count) on set. */
lb_status lbu_set_params(lbu_net* net, const float* params, int on_device);
lb_status lbu_get_params(lbu_net* net, float* params, int on_device);
/* Adam hyper-parameters (defaults 0.9, 0.999, 1e-8). */
lb_status lbu_set_adam(lbu_net* net, float b1, float b2, float eps);

/* Inference: y[batch][H][W][out_ch] = net(x[batch][H][W][in_ch]). x and y are both host
 * (on_device = 0) or both device pointers. */
lb_status lbu_forward(lbu_net* net, const float* x, int batch, float* y, int on_device);

/* One forward and backward pass on samples idx[0..batch-1] of the device arrays
 * X[n][H][W][in_ch] and T[n][H][W][out_ch] (idx == NULL: samples 0..batch-1); lam[out_ch]
 * are the channel weights of the loss (NULL: all 1, host pointer). Writes the loss
 * (host, may be NULL: no synchronisation) and, when grads != NULL, the gradient of every
 * parameter (device pointer, flat layout). */
lb_status lbu_loss_grad(lbu_net* net, const float* X, const float* T, const int* idx, int batch,
                        const float* lam, float* loss, float* grads);

/* lbu_loss_grad followed by one Adam update of the parameters with learning rate lr. */
lb_status lbu_train_step(lbu_net* net, const float* X, const float* T, const int* idx, int batch,
                         const float* lam, float lr, float* loss);

/* Single 3x3 convolution (the kernel every layer uses), device pointers, for tests:
 * y[p][o] (BF16 bits, pixel stride y_stride elements) = act(b[o] + sum w[o][t][c] x[...])
 * with x BF16 [batch][h][w][c] (pixel stride x_stride, image h x w, or h/2 x w/2 when
 * upsample = 1: nearest 2x upsampling on the fly), w BF16 [C_out][9][C_in], b FP32 or
 * NULL, act = ReLU when relu = 1. C_in and C_out multiples of 32; strides multiples of 8.
 * The convolutions run on mma.sync tensor-core instructions; with the environment
 * variable LBNCI_UNET_MMA=tcgen05 (read at every launch) they run on tcgen05.mma with the
 * accumulator in tensor memory instead. That kernel's waits are bounded: an expired wait
 * leaves its output unwritten and sets a device error word, which the next lbu_forward
 * (host output), lbu_loss_grad or lbu_train_step (with a loss pointer) reports as
 * LB_ECUDA after it synchronises. */
lb_status lbu_conv3x3(const unsigned short* x, int x_stride, int batch, int h, int w, int c_in,
                      int upsample, const unsigned short* wgt, const float* bias, int relu,
                      unsigned short* y, int y_stride, int c_out, void* stream);

/* Weight gradient of that convolution: dw[o][t][c] (FP32, [C_out][9][C_in]) =
 * sum_p dy[p][o] xpad[p + tap t][c] and db[o] = sum_p dy[p][o] (db may be NULL).
 * work: device scratch of at least lbu_conv3x3_wgrad_work(...) bytes. */
size_t lbu_conv3x3_wgrad_work(int batch, int h, int w, int c_in, int c_out);
lb_status lbu_conv3x3_wgrad(const unsigned short* x, int x_stride, int batch, int h, int w, int c_in,
                            int upsample, const unsigned short* dy, int dy_stride, int c_out,
                            float* dw, float* db, void* work, size_t work_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif
