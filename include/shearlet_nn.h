/*
 * shearlet_nn.h - C ABI of the learned parts built around the shearlet
 * transform (libshearlet): kernels to train and run
 *   (1) a threshold predictor for the unrolled inpainting iteration of
 *       Sec. 4.3 (per-subband thresholds delta_{t,i}), and
 *   (2) a residual CNN on shearlet coefficients after the learned proximal
 *       operators of Sec. 4.4 (Id + W3 A W2 A W1, 3x3 convolutions, PReLU).
 *
 * Conventions: float32, NCHW contiguous device tensors, caller-owned; every
 * call launches on `stream` (cudaStream_t as void*) and returns shl_status
 * (SHL_EINVAL for bad arguments before any launch, SHL_ECUDA if a launch
 * failed; shl_nn_last_error() gives text).  Reductions are deterministic:
 * per-CTA partial sums in a caller workspace, combined in a fixed order.
 */
#ifndef SHEARLET_NN_H
#define SHEARLET_NN_H

#include <stddef.h>

#include "shearlet.h"

#ifdef __cplusplus
extern "C" {
#endif

const char* shl_nn_last_error(void);

/* 3x3 convolution, zero padding 1 (the affine maps W_{w,b} of Sec. 4.4):
 * out[b][o][y][x] = bias[o] + sum_{i,dy,dx} w[o][i][dy][dx] in[b][i][y+dy-1][x+dx-1].
 * in [B][Ci][H][W], w [Co][Ci][3][3], bias [Co] or NULL, out [B][Co][H][W]. */
shl_status shl_nn_conv3x3_forward(const float* in, const float* w, const float* bias, float* out,
                                  int B, int Ci, int Co, int H, int W, void* stream);
/* Workspace (floats) for the two backward calls. */
size_t shl_nn_conv3x3_workspace_floats(int B, int Ci, int Co, int H, int W);
/* gin = d loss / d in given gout = d loss / d out (convolution with the flipped,
 * channel-transposed weights). ws: shl_nn_conv3x3_workspace_floats floats. */
shl_status shl_nn_conv3x3_backward_data(const float* gout, const float* w, float* gin, int B,
                                        int Ci, int Co, int H, int W, float* ws, void* stream);
/* gw [Co][Ci][3][3] and gb [Co] (gb may be NULL); Ci <= 64. */
shl_status shl_nn_conv3x3_backward_weight(const float* in, const float* gout, float* gw, float* gb,
                                          int B, int Ci, int Co, int H, int W, float* ws,
                                          void* stream);

/* The same 3x3 convolution on the tensor cores (tcgen05): bfloat16 operands
 * (inputs and weights rounded to nearest even), float32 accumulation, so
 * the result equals the convolution of the bfloat16-rounded tensors up to
 * float32 summation order.  Supported when shl_nn_conv3x3_tc_supported()
 * (1 <= Ci, Co <= 48 and W a multiple of 128) and the input (gout for the
 * backward call) is 16-byte aligned; SHL_EINVAL otherwise. */
int shl_nn_conv3x3_tc_supported(int Ci, int Co, int H, int W);
shl_status shl_nn_conv3x3_forward_tc(const float* in, const float* w, const float* bias,
                                     float* out, int B, int Ci, int Co, int H, int W,
                                     void* stream);
/* gin for the convolution with w [Co][Ci][3][3] (flipped, channel-transposed
 * weights), on the tensor cores; no workspace. */
shl_status shl_nn_conv3x3_backward_data_tc(const float* gout, const float* w, float* gin, int B,
                                           int Ci, int Co, int H, int W, void* stream);
/* Weight (and bias) gradient on the tensor cores: gw = sum over pixels of
 * gout x shifted input with both rounded to bfloat16, float32 accumulation
 * (per-CTA partials in ws, summed in a fixed order); gb (may be NULL) in
 * float32 from the unrounded gout.  Supported when
 * shl_nn_conv3x3_wgrad_tc_supported() (3 Ci <= 128, Co <= 48, W a multiple
 * of 128) and in, gout are 16-byte aligned; ws holds
 * shl_nn_conv3x3_backward_weight_tc_workspace_floats() floats. */
int shl_nn_conv3x3_wgrad_tc_supported(int Ci, int Co, int H, int W);
size_t shl_nn_conv3x3_backward_weight_tc_workspace_floats(int B, int Ci, int Co, int H, int W);
shl_status shl_nn_conv3x3_backward_weight_tc(const float* in, const float* gout, float* gw,
                                             float* gb, int B, int Ci, int Co, int H, int W,
                                             float* ws, void* stream);
/* Synchronises `stream`, then reports SHL_ETIMEOUT if a tensor-core
 * convolution on this device gave up waiting for its MMAs (bounded wait)
 * since the last call, clearing the flag. */
shl_status shl_nn_tc_status(void* stream);
const char* shl_nn_tc_last_error(void);

/* PReLU A(x) = x (x >= 0), a x (x < 0) with one slope a[0] per layer
 * (Sec. 4.4 writes the negative branch as -c x, i.e. a = -c). */
shl_status shl_nn_prelu_forward(const float* x, const float* a, float* y, long long n, void* stream);
size_t shl_nn_reduce_workspace_floats(long long n);
/* gx and ga[0] = sum_{x<0} gy x; ws: shl_nn_reduce_workspace_floats floats. */
shl_status shl_nn_prelu_backward(const float* x, const float* a, const float* gy, float* gx,
                                 float* ga, long long n, float* ws, void* stream);

/* Average pooling by an integer factor f (H, W divisible by f). */
shl_status shl_nn_avgpool(const float* x, float* y, int B, int C, int H, int W, int f, void* stream);
/* Global average pooling [B][C][HW] -> [B][C] and its backward. */
shl_status shl_nn_gap_forward(const float* x, float* y, int B, int C, int HW, void* stream);
shl_status shl_nn_gap_backward(const float* gy, float* gx, int B, int C, int HW, void* stream);

/* y[b][o] = b[o] + sum_i x[b][i] w[o][i]; backward gives gx (may be NULL), gw, gb. */
shl_status shl_nn_linear_forward(const float* x, const float* w, const float* b, float* y, int B,
                                 int I, int O, void* stream);
shl_status shl_nn_linear_backward(const float* x, const float* w, const float* gy, float* gx,
                                  float* gw, float* gb, int B, int I, int O, void* stream);

/* softplus(x) = log(1 + e^x) (keeps predicted thresholds positive). */
shl_status shl_nn_softplus_forward(const float* x, float* y, long long n, void* stream);
shl_status shl_nn_softplus_backward(const float* x, const float* gy, float* gx, long long n,
                                    void* stream);

/* Relaxed hard threshold y = c sigmoid((|c| / d_s - 1) / tau) for each of
 * nsub subbands of HW values, d_s = delta[s] * scale[s % K] (scale [K] or NULL,
 * e.g. the filters' RMS for thresholds given relative to RMS_i; tau relative to
 * the threshold); tends to the hard threshold T_d of Sec. 4.2 as tau -> 0.
 * c is float32 or (c_bf16 != 0) bfloat16. */
shl_status shl_nn_gate_forward(const void* c, int c_bf16, const float* delta, const float* scale,
                               int K, float tau, float* y, int nsub, long long HW, void* stream);
size_t shl_nn_gate_workspace_floats(int nsub);
/* gc (float32 c only) and gdelta [nsub] (d loss / d delta); ws:
 * shl_nn_gate_workspace_floats floats. */
shl_status shl_nn_gate_backward(const float* c, const float* delta, const float* scale, int K,
                                float tau, const float* gy, float* gc, float* gdelta, int nsub,
                                long long HW, float* ws, void* stream);

/* out[0] = sum (a - b)^2 (divide by n for the mean); ws: reduce workspace. */
shl_status shl_nn_mse_forward(const float* a, const float* b, float* out, long long n, float* ws,
                              void* stream);
/* ga = 2 gscale[0] (a - b) / n. */
shl_status shl_nn_mse_backward(const float* a, const float* b, const float* gscale, float* ga,
                               long long n, void* stream);

/* One Adam step with bias correction (step counts from 1). */
shl_status shl_nn_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1,
                       float b2, float eps, int step, void* stream);

/* Inpainting residual input u = mask (f_masked - f) + f (Alg. of Sec. 4.3) and
 * its backward gf = (1 - mask) gu; mask uint8 in {0, 1}. */
shl_status shl_nn_mask_mix(const float* f_masked, const unsigned char* mask, const float* f,
                           float* u, long long n, void* stream);
shl_status shl_nn_mask_mix_backward(const unsigned char* mask, const float* gu, float* gf,
                                    long long n, void* stream);

/* bfloat16 <-> float32 conversion (x_bf16 != 0: bf16 -> f32, else f32 -> bf16, RNE). */
shl_status shl_nn_cast(const void* x, int x_bf16, void* y, long long n, void* stream);
/* Thresholds of the unrolled inpainting iteration (Sec. 4.3) from predictions
 * relative to RMS_i: out[t][b][k] = d[b][t][k] * scale[k]. */
shl_status shl_nn_scale_thresholds(const float* d, const float* scale, float* out, int B, int T,
                                   int K, void* stream);
/* y += a x */
shl_status shl_nn_axpy(const float* x, float a, float* y, long long n, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SHEARLET_NN_H */
