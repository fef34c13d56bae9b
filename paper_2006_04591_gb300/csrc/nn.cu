// nn.cu - training and inference kernels of the learned parts.
//
// Two small networks sit around the shearlet transform:
//  * a threshold predictor (avgpool, 4 x [3x3 conv + PReLU], global average
//    pool, linear, softplus) giving per-subband thresholds of the unrolled
//    inpainting iteration, trained through a relaxed hard threshold;
//  * a residual 3-layer CNN on shearlet coefficients (the learned proximal
//    operator pattern of Sec. 4.4: Id + W A W A W with PReLU A).
// All tensors are float32 NCHW, contiguous.  Every reduction is deterministic
// (per-CTA partial sums combined in a fixed order; no atomics).
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "../../include/shearlet_nn.h"

namespace {

thread_local const char* g_nn_err = "";

shl_status nn_fail(shl_status s, const char* m) {
  g_nn_err = m;
  return s;
}
shl_status nn_launch(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_nn_err = where;
    return SHL_ECUDA;
  }
  return SHL_OK;
}
inline cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
inline int blocks(long long n, int t) { return (int)std::min<long long>((n + t - 1) / t, 1 << 20); }

// ------------------------------------------------------------ conv 3x3
// Output tile 64 x 16 pixels x 8 output channels per CTA; 256 threads, each
// computes 4 horizontally adjacent pixels for the 8 channels.  Input
// channels are consumed 4 at a time through shared memory.
constexpr int CX = 64, CY = 16, COT = 8, CIC = 4;

__global__ void __launch_bounds__(256) k_conv3x3(const float* __restrict__ in,
                                                 const float* __restrict__ w,
                                                 const float* __restrict__ bias,
                                                 float* __restrict__ out, int Ci, int Co, int H,
                                                 int W) {
  __shared__ float tile[CIC][CY + 2][CX + 2];
  __shared__ float wt[CIC][COT][9];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int tiles_x = (W + CX - 1) / CX;
  const int x0 = (blockIdx.x % tiles_x) * CX, y0 = (blockIdx.x / tiles_x) * CY;
  const int co0 = blockIdx.y * COT;
  const int b = blockIdx.z;
  float acc[COT][4];
#pragma unroll
  for (int o = 0; o < COT; ++o)
#pragma unroll
    for (int p = 0; p < 4; ++p) acc[o][p] = 0.f;
  const float* inb = in + (size_t)b * Ci * H * W;
  for (int c0 = 0; c0 < Ci; c0 += CIC) {
    for (int idx = threadIdx.x; idx < CIC * (CY + 2) * (CX + 2); idx += 256) {
      const int cc = idx / ((CY + 2) * (CX + 2));
      const int rem = idx % ((CY + 2) * (CX + 2));
      const int yy = rem / (CX + 2), xx = rem % (CX + 2);
      const int gy = y0 + yy - 1, gx = x0 + xx - 1, ci = c0 + cc;
      float v = 0.f;
      if (ci < Ci && gy >= 0 && gy < H && gx >= 0 && gx < W) v = inb[((size_t)ci * H + gy) * W + gx];
      tile[cc][yy][xx] = v;
    }
    for (int idx = threadIdx.x; idx < CIC * COT * 9; idx += 256) {
      const int cc = idx / (COT * 9), rem = idx % (COT * 9), o = rem / 9, k = rem % 9;
      const int ci = c0 + cc, co = co0 + o;
      wt[cc][o][k] = (ci < Ci && co < Co) ? w[((size_t)co * Ci + ci) * 9 + k] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int cc = 0; cc < CIC; ++cc) {
      float v[3][6];
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 6; ++dx) v[dy][dx] = tile[cc][ty + dy][4 * tx + dx];
#pragma unroll
      for (int o = 0; o < COT; ++o) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          const float wv = wt[cc][o][k];
#pragma unroll
          for (int p = 0; p < 4; ++p) acc[o][p] = fmaf(wv, v[k / 3][k % 3 + p], acc[o][p]);
        }
      }
    }
    __syncthreads();
  }
  const int y = y0 + ty;
  if (y >= H) return;
#pragma unroll
  for (int o = 0; o < COT; ++o) {
    const int co = co0 + o;
    if (co >= Co) break;
    const float bv = bias ? bias[co] : 0.f;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int x = x0 + 4 * tx + p;
      if (x < W) out[(((size_t)b * Co + co) * H + y) * W + x] = acc[o][p] + bv;
    }
  }
}

// w'[ci][co][2-dy][2-dx] = w[co][ci][dy][dx]: backward-data is a convolution
// of the output gradient with the flipped, channel-transposed weights.
__global__ void k_flip(const float* __restrict__ w, float* __restrict__ wf, int Ci, int Co) {
  const int n = Ci * Co * 9;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    const int co = idx / (Ci * 9), rem = idx % (Ci * 9), ci = rem / 9, k = rem % 9;
    wf[((size_t)ci * Co + co) * 9 + (8 - k)] = w[idx];
  }
}

// Weight gradient partial sums: CTA g accumulates, over the pixel tiles it
// owns, gw[co][ci][k] for one group of 8 output channels; thread t owns
// entries t, t + 256, ... of the group's COT * Ci * 9 (+ COT bias) entries.
constexpr int WTX = 32, WTY = 8;
__global__ void __launch_bounds__(256) k_conv_wgrad(const float* __restrict__ in,
                                                    const float* __restrict__ gout,
                                                    float* __restrict__ partial, int B, int Ci,
                                                    int Co, int H, int W) {
  extern __shared__ float sm[];
  float* go = sm;                                  // [COT][WTY][WTX]
  float* xt = go + COT * WTY * WTX;                // [Ci][WTY+2][WTX+2]
  const int co0 = blockIdx.y * COT;
  const int nent = COT * Ci * 9 + COT;
  const int tiles_x = (W + WTX - 1) / WTX, tiles_y = (H + WTY - 1) / WTY;
  const long long ntiles = (long long)B * tiles_x * tiles_y;
  constexpr int MAXE = 24;                         // entries per thread (Ci <= 64)
  float acc[MAXE];
#pragma unroll
  for (int e = 0; e < MAXE; ++e) acc[e] = 0.f;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int b = (int)(t / (tiles_x * tiles_y));
    const int rem = (int)(t % (tiles_x * tiles_y));
    const int y0 = (rem / tiles_x) * WTY, x0 = (rem % tiles_x) * WTX;
    for (int idx = threadIdx.x; idx < COT * WTY * WTX; idx += 256) {
      const int o = idx / (WTY * WTX), r2 = idx % (WTY * WTX), yy = r2 / WTX, xx = r2 % WTX;
      const int co = co0 + o, y = y0 + yy, x = x0 + xx;
      go[idx] = (co < Co && y < H && x < W) ? gout[(((size_t)b * Co + co) * H + y) * W + x] : 0.f;
    }
    for (int idx = threadIdx.x; idx < Ci * (WTY + 2) * (WTX + 2); idx += 256) {
      const int ci = idx / ((WTY + 2) * (WTX + 2)), r2 = idx % ((WTY + 2) * (WTX + 2));
      const int yy = r2 / (WTX + 2), xx = r2 % (WTX + 2);
      const int y = y0 + yy - 1, x = x0 + xx - 1;
      xt[idx] = (y >= 0 && y < H && x >= 0 && x < W) ? in[(((size_t)b * Ci + ci) * H + y) * W + x] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < MAXE; ++e) {
      const int ent = threadIdx.x + e * 256;
      if (ent >= nent) break;
      float s = acc[e];
      if (ent < COT * Ci * 9) {
        const int o = ent / (Ci * 9), r2 = ent % (Ci * 9), ci = r2 / 9, k = r2 % 9;
        const int dy = k / 3, dx = k % 3;
        const float* g = go + o * WTY * WTX;
        const float* xv = xt + ci * (WTY + 2) * (WTX + 2);
        for (int yy = 0; yy < WTY; ++yy)
          for (int xx = 0; xx < WTX; ++xx) s = fmaf(g[yy * WTX + xx], xv[(yy + dy) * (WTX + 2) + xx + dx], s);
      } else {
        const float* g = go + (ent - COT * Ci * 9) * WTY * WTX;
        for (int q = 0; q < WTY * WTX; ++q) s += g[q];
      }
      acc[e] = s;
    }
    __syncthreads();
  }
  float* P = partial + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * nent;
#pragma unroll
  for (int e = 0; e < MAXE; ++e) {
    const int ent = threadIdx.x + e * 256;
    if (ent < nent) P[ent] = acc[e];
  }
}

__global__ void k_conv_wgrad_reduce(const float* __restrict__ partial, float* __restrict__ gw,
                                    float* __restrict__ gb, int nparts, int Ci, int Co) {
  const int groups = (Co + COT - 1) / COT;
  const int nent = COT * Ci * 9 + COT;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < groups * nent;
       idx += gridDim.x * blockDim.x) {
    const int g = idx / nent, ent = idx % nent;
    float s = 0.f;
    for (int p = 0; p < nparts; ++p) s += partial[((size_t)g * nparts + p) * nent + ent];
    if (ent < COT * Ci * 9) {
      const int o = ent / (Ci * 9), r2 = ent % (Ci * 9);
      const int co = g * COT + o;
      if (co < Co) gw[(size_t)co * Ci * 9 + r2] = s;
    } else {
      const int co = g * COT + (ent - COT * Ci * 9);
      if (co < Co && gb) gb[co] = s;
    }
  }
}

// ------------------------------------------------------------ elementwise
__global__ void k_prelu_fwd(const float* __restrict__ x, const float* __restrict__ a,
                            float* __restrict__ y, long long n, int vec) {
  const float s = a[0];
  const long long n4 = vec ? n / 4 : 0;               // float4 body (16-byte aligned pointers)
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride) {
    float4 v = __ldcs(reinterpret_cast<const float4*>(x) + i);
    v.x = v.x >= 0.f ? v.x : s * v.x;
    v.y = v.y >= 0.f ? v.y : s * v.y;
    v.z = v.z >= 0.f ? v.z : s * v.z;
    v.w = v.w >= 0.f ? v.w : s * v.w;
    reinterpret_cast<float4*>(y)[i] = v;
  }
  for (long long i = 4 * n4 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
    const float v = x[i];
    y[i] = v >= 0.f ? v : s * v;
  }
}

// gx = gy * (x >= 0 ? 1 : a); partial[cta] = sum over the CTA's elements of gy * x (x < 0).
__global__ void __launch_bounds__(256) k_prelu_bwd(const float* __restrict__ x,
                                                   const float* __restrict__ a,
                                                   const float* __restrict__ gy,
                                                   float* __restrict__ gx,
                                                   float* __restrict__ partial, long long n,
                                                   int vec) {
  const float s = a[0];
  float acc = 0.f;
  const long long n4 = vec ? n / 4 : 0;               // float4 body (16-byte aligned pointers)
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride) {
    const float4 v = __ldcs(reinterpret_cast<const float4*>(x) + i);
    const float4 g = __ldcs(reinterpret_cast<const float4*>(gy) + i);
    float4 o;
    o.x = v.x >= 0.f ? g.x : s * g.x;
    o.y = v.y >= 0.f ? g.y : s * g.y;
    o.z = v.z >= 0.f ? g.z : s * g.z;
    o.w = v.w >= 0.f ? g.w : s * g.w;
    reinterpret_cast<float4*>(gx)[i] = o;
    if (v.x < 0.f) acc = fmaf(g.x, v.x, acc);
    if (v.y < 0.f) acc = fmaf(g.y, v.y, acc);
    if (v.z < 0.f) acc = fmaf(g.z, v.z, acc);
    if (v.w < 0.f) acc = fmaf(g.w, v.w, acc);
  }
  for (long long i = 4 * n4 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
    const float v = x[i], g = gy[i];
    gx[i] = v >= 0.f ? g : s * g;
    if (v < 0.f) acc = fmaf(g, v, acc);
  }
  __shared__ float red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Sum of n partial values into out[0] (one CTA, fixed order).
__global__ void __launch_bounds__(256) k_sum(const float* __restrict__ p, int n, float* out) {
  __shared__ float red[256];
  float acc = 0.f;
  for (int i = threadIdx.x; i < n; i += 256) acc += p[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

__global__ void k_avgpool(const float* __restrict__ x, float* __restrict__ y, long long BC, int H,
                          int W, int f) {
  const int Ho = H / f, Wo = W / f;
  const long long n = BC * Ho * Wo;
  const float inv = 1.f / (f * f);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long bc = i / (Ho * Wo);
    const int r = (int)(i % (Ho * Wo)), yo = r / Wo, xo = r % Wo;
    const float* p = x + (bc * H + (long long)yo * f) * W + (long long)xo * f;
    float s = 0.f;
    for (int dy = 0; dy < f; ++dy)
      for (int dx = 0; dx < f; ++dx) s += p[(long long)dy * W + dx];
    y[i] = s * inv;
  }
}

// Global average pool: one CTA per (b, c).
__global__ void __launch_bounds__(256) k_gap_fwd(const float* __restrict__ x, float* __restrict__ y,
                                                 int HW) {
  __shared__ float red[256];
  const float* p = x + (size_t)blockIdx.x * HW;
  float acc = 0.f;
  for (int i = threadIdx.x; i < HW; i += 256) acc += p[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) y[blockIdx.x] = red[0] / HW;
}

__global__ void k_gap_bwd(const float* __restrict__ gy, float* __restrict__ gx, long long BC,
                          int HW) {
  const long long n = BC * HW;
  const float inv = 1.f / HW;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    gx[i] = gy[i / HW] * inv;
}

// y[b][o] = bias[o] + sum_i x[b][i] w[o][i]
__global__ void k_linear_fwd(const float* __restrict__ x, const float* __restrict__ w,
                             const float* __restrict__ bias, float* __restrict__ y, int B, int I,
                             int O) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < B * O; idx += gridDim.x * blockDim.x) {
    const int b = idx / O, o = idx % O;
    float s = bias ? bias[o] : 0.f;
    for (int i = 0; i < I; ++i) s = fmaf(x[(size_t)b * I + i], w[(size_t)o * I + i], s);
    y[idx] = s;
  }
}

// gx = gy W; gw = gy^T x; gb = sum_b gy (each entry one thread, fixed order).
__global__ void k_linear_bwd(const float* __restrict__ x, const float* __restrict__ w,
                             const float* __restrict__ gy, float* __restrict__ gx,
                             float* __restrict__ gw, float* __restrict__ gb, int B, int I, int O) {
  const int n1 = B * I, n2 = O * I, n3 = O;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n1 + n2 + n3;
       idx += gridDim.x * blockDim.x) {
    if (idx < n1) {
      const int b = idx / I, i = idx % I;
      float s = 0.f;
      for (int o = 0; o < O; ++o) s = fmaf(gy[(size_t)b * O + o], w[(size_t)o * I + i], s);
      if (gx) gx[idx] = s;
    } else if (idx < n1 + n2) {
      const int e = idx - n1, o = e / I, i = e % I;
      float s = 0.f;
      for (int b = 0; b < B; ++b) s = fmaf(gy[(size_t)b * O + o], x[(size_t)b * I + i], s);
      gw[e] = s;
    } else {
      const int o = idx - n1 - n2;
      float s = 0.f;
      for (int b = 0; b < B; ++b) s += gy[(size_t)b * O + o];
      gb[o] = s;
    }
  }
}

__device__ __forceinline__ float softplus_f(float v) {
  return fmaxf(v, 0.f) + log1pf(expf(-fabsf(v)));
}
__device__ __forceinline__ float sigmoid_f(float v) { return 1.f / (1.f + expf(-v)); }

__global__ void k_softplus_fwd(const float* __restrict__ x, float* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = softplus_f(x[i]);
}
__global__ void k_softplus_bwd(const float* __restrict__ x, const float* __restrict__ gy,
                               float* __restrict__ gx, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    gx[i] = gy[i] * sigmoid_f(x[i]);
}

// Relaxed hard threshold y = c sigmoid((|c| / delta - 1) / tau), delta per
// (b, k); tau is relative to the threshold, so the relaxation is scale-free.
// The threshold of subband s is delta[s] * scale[s % K] (scale may be null).
template <bool BF16>
__global__ void k_gate_fwd(const void* __restrict__ c, const float* __restrict__ delta,
                           const float* __restrict__ scale, int K, float tau,
                           float* __restrict__ y, long long HW) {
  const long long sub = blockIdx.y;
  const float id = 1.f / (delta[sub] * (scale ? scale[sub % K] : 1.f)), it = 1.f / tau;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HW;
       i += (long long)gridDim.x * blockDim.x) {
    const long long o = sub * HW + i;
    const float v = BF16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(c)[o])
                         : static_cast<const float*>(c)[o];
    y[o] = v * sigmoid_f(fmaf(fabsf(v), id, -1.f) * it);
  }
}

// With s = sigmoid(r), r = (|c| / delta - 1) / tau, s' = s (1 - s):
//   gc = gy (s + |c| s' / (delta tau)),
//   gdelta = sum gy c s' (-|c| / (delta^2 tau))  (per-CTA partials).
// (with a scale, gdelta[s] also carries the factor scale[s % K])
__global__ void __launch_bounds__(256) k_gate_bwd(const float* __restrict__ c,
                                                  const float* __restrict__ delta,
                                                  const float* __restrict__ scale, int K,
                                                  float tau, const float* __restrict__ gy,
                                                  float* __restrict__ gc,
                                                  float* __restrict__ partial, long long HW) {
  const long long sub = blockIdx.y;
  const float sc = scale ? scale[sub % K] : 1.f;
  const float id = 1.f / (delta[sub] * sc), it = 1.f / tau;
  float acc = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HW;
       i += (long long)gridDim.x * blockDim.x) {
    const long long o = sub * HW + i;
    const float v = c[o], g = gy[o];
    const float a = fabsf(v);
    const float s = sigmoid_f(fmaf(a, id, -1.f) * it);
    const float ds = s * (1.f - s) * it * id;          // s' / (delta tau)
    gc[o] = g * (s + a * ds);
    acc = fmaf(-g * v * a * id * sc, ds, acc);
  }
  __shared__ float red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[sub * gridDim.x + blockIdx.x] = red[0];
}

// out[s] = sum_j partial[s][j], one thread per row, fixed order.
__global__ void k_rowsum(const float* __restrict__ partial, float* __restrict__ out, int rows,
                         int cols) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int j = 0; j < cols; ++j) s += partial[(size_t)r * cols + j];
    out[r] = s;
  }
}

__global__ void __launch_bounds__(256) k_mse_partial(const float* __restrict__ a,
                                                     const float* __restrict__ b,
                                                     float* __restrict__ partial, long long n) {
  float acc = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float d = a[i] - b[i];
    acc = fmaf(d, d, acc);
  }
  __shared__ float red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_mse_bwd(const float* __restrict__ a, const float* __restrict__ b,
                          const float* __restrict__ gscale, float* __restrict__ ga, long long n) {
  const float s = 2.f * gscale[0] / (float)n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    ga[i] = s * (a[i] - b[i]);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// u = mask ? f_masked : f  (= mask (f_masked - f) + f); backward gf = (1 - mask) gu.
__global__ void k_mask_mix(const float* __restrict__ fm, const uint8_t* __restrict__ mask,
                           const float* __restrict__ f, float* __restrict__ u, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    u[i] = mask[i] ? fm[i] : f[i];
}
__global__ void k_mask_mix_bwd(const uint8_t* __restrict__ mask, const float* __restrict__ gu,
                               float* __restrict__ gf, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    gf[i] = mask[i] ? 0.f : gu[i];
}

__global__ void k_bf16_to_f32(const __nv_bfloat16* __restrict__ x, float* __restrict__ y,
                              long long n, int vec) {
  const long long n8 = vec ? n / 8 : 0;               // 16-byte body (16-byte aligned pointers)
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n8; i += stride) {
    const uint4 h = __ldcs(reinterpret_cast<const uint4*>(x) + i);
    const __nv_bfloat162* p = reinterpret_cast<const __nv_bfloat162*>(&h);
    const float2 a = __bfloat1622float2(p[0]), b = __bfloat1622float2(p[1]);
    const float2 c = __bfloat1622float2(p[2]), d = __bfloat1622float2(p[3]);
    reinterpret_cast<float4*>(y)[2 * i] = make_float4(a.x, a.y, b.x, b.y);
    reinterpret_cast<float4*>(y)[2 * i + 1] = make_float4(c.x, c.y, d.x, d.y);
  }
  for (long long i = 8 * n8 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride)
    y[i] = __bfloat162float(x[i]);
}
__global__ void k_f32_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y,
                              long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

__global__ void k_axpy(const float* __restrict__ x, float a, float* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = fmaf(a, x[i], y[i]);
}

// out[t][b][k] = d[b][t][k] * scale[k]
__global__ void k_scale_thresholds(const float* __restrict__ d, const float* __restrict__ scale,
                                   float* __restrict__ out, int B, int T, int K) {
  const int n = B * T * K;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int b = i / (T * K), r = i % (T * K), t = r / K, k = r % K;
    out[((size_t)t * B + b) * K + k] = d[i] * scale[k];
  }
}

constexpr int RED_CTAS = 1024;

}  // namespace

extern "C" {

const char* shl_nn_last_error(void) { return g_nn_err; }

shl_status shl_nn_conv3x3_forward(const float* in, const float* w, const float* bias, float* out,
                                  int B, int Ci, int Co, int H, int W, void* stream) {
  if (!in || !w || !out || B < 0 || Ci < 1 || Co < 1 || H < 1 || W < 1)
    return nn_fail(SHL_EINVAL, "conv3x3_forward: bad arguments");
  if (B == 0) return SHL_OK;
  dim3 grid(((W + CX - 1) / CX) * ((H + CY - 1) / CY), (Co + COT - 1) / COT, B);
  k_conv3x3<<<grid, 256, 0, S(stream)>>>(in, w, bias, out, Ci, Co, H, W);
  return nn_launch("conv3x3_forward");
}

size_t shl_nn_conv3x3_workspace_floats(int B, int Ci, int Co, int H, int W) {
  (void)B; (void)H; (void)W;
  const size_t groups = (Co + COT - 1) / COT;
  const size_t nent = (size_t)COT * Ci * 9 + COT;
  return std::max((size_t)Ci * Co * 9, groups * 256 * nent);
}

shl_status shl_nn_conv3x3_backward_data(const float* gout, const float* w, float* gin, int B,
                                        int Ci, int Co, int H, int W, float* ws, void* stream) {
  if (!gout || !w || !gin || !ws || B < 0) return nn_fail(SHL_EINVAL, "conv3x3_backward_data: bad arguments");
  if (B == 0) return SHL_OK;
  k_flip<<<blocks((long long)Ci * Co * 9, 256), 256, 0, S(stream)>>>(w, ws, Ci, Co);
  dim3 grid(((W + CX - 1) / CX) * ((H + CY - 1) / CY), (Ci + COT - 1) / COT, B);
  k_conv3x3<<<grid, 256, 0, S(stream)>>>(gout, ws, nullptr, gin, Co, Ci, H, W);
  return nn_launch("conv3x3_backward_data");
}

shl_status shl_nn_conv3x3_backward_weight(const float* in, const float* gout, float* gw, float* gb,
                                          int B, int Ci, int Co, int H, int W, float* ws,
                                          void* stream) {
  if (!in || !gout || !gw || !ws || B < 1 || Ci > 64 || Ci < 1)
    return nn_fail(SHL_EINVAL, "conv3x3_backward_weight: bad arguments (Ci must be 1..64)");
  const int nparts = 256;
  const size_t sm = sizeof(float) * ((size_t)COT * WTY * WTX + (size_t)Ci * (WTY + 2) * (WTX + 2));
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(k_conv_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  dim3 grid(nparts, (Co + COT - 1) / COT);
  k_conv_wgrad<<<grid, 256, sm, S(stream)>>>(in, gout, ws, B, Ci, Co, H, W);
  const int groups = (Co + COT - 1) / COT, nent = COT * Ci * 9 + COT;
  k_conv_wgrad_reduce<<<blocks((long long)groups * nent, 256), 256, 0, S(stream)>>>(ws, gw, gb, nparts,
                                                                                  Ci, Co);
  return nn_launch("conv3x3_backward_weight");
}

shl_status shl_nn_prelu_forward(const float* x, const float* a, float* y, long long n, void* stream) {
  if (!x || !a || !y || n < 0) return nn_fail(SHL_EINVAL, "prelu_forward: bad arguments");
  if (n == 0) return SHL_OK;
  const int vec = aligned16(x) && aligned16(y);
  k_prelu_fwd<<<blocks(vec ? (n + 3) / 4 : n, 256), 256, 0, S(stream)>>>(x, a, y, n, vec);
  return nn_launch("prelu_forward");
}

size_t shl_nn_reduce_workspace_floats(long long n) {
  (void)n;
  return RED_CTAS;
}

shl_status shl_nn_prelu_backward(const float* x, const float* a, const float* gy, float* gx,
                                 float* ga, long long n, float* ws, void* stream) {
  if (!x || !a || !gy || !gx || !ga || !ws || n < 0) return nn_fail(SHL_EINVAL, "prelu_backward: bad arguments");
  const int g = std::max(1, std::min(RED_CTAS, blocks(n, 256)));
  const int vec = aligned16(x) && aligned16(gy) && aligned16(gx);
  k_prelu_bwd<<<g, 256, 0, S(stream)>>>(x, a, gy, gx, ws, n, vec);
  k_sum<<<1, 256, 0, S(stream)>>>(ws, g, ga);
  return nn_launch("prelu_backward");
}

shl_status shl_nn_avgpool(const float* x, float* y, int B, int C, int H, int W, int f,
                          void* stream) {
  if (!x || !y || f < 1 || H % f || W % f) return nn_fail(SHL_EINVAL, "avgpool: bad arguments");
  const long long n = (long long)B * C * (H / f) * (W / f);
  if (n == 0) return SHL_OK;
  k_avgpool<<<blocks(n, 256), 256, 0, S(stream)>>>(x, y, (long long)B * C, H, W, f);
  return nn_launch("avgpool");
}

shl_status shl_nn_gap_forward(const float* x, float* y, int B, int C, int HW, void* stream) {
  if (!x || !y || HW < 1) return nn_fail(SHL_EINVAL, "gap_forward: bad arguments");
  if (B * C == 0) return SHL_OK;
  k_gap_fwd<<<B * C, 256, 0, S(stream)>>>(x, y, HW);
  return nn_launch("gap_forward");
}

shl_status shl_nn_gap_backward(const float* gy, float* gx, int B, int C, int HW, void* stream) {
  if (!gy || !gx || HW < 1) return nn_fail(SHL_EINVAL, "gap_backward: bad arguments");
  const long long n = (long long)B * C * HW;
  if (n == 0) return SHL_OK;
  k_gap_bwd<<<blocks(n, 256), 256, 0, S(stream)>>>(gy, gx, (long long)B * C, HW);
  return nn_launch("gap_backward");
}

shl_status shl_nn_linear_forward(const float* x, const float* w, const float* b, float* y, int B,
                                 int I, int O, void* stream) {
  if (!x || !w || !y) return nn_fail(SHL_EINVAL, "linear_forward: bad arguments");
  if (B * O == 0) return SHL_OK;
  k_linear_fwd<<<blocks((long long)B * O, 128), 128, 0, S(stream)>>>(x, w, b, y, B, I, O);
  return nn_launch("linear_forward");
}

shl_status shl_nn_linear_backward(const float* x, const float* w, const float* gy, float* gx,
                                  float* gw, float* gb, int B, int I, int O, void* stream) {
  if (!x || !w || !gy || !gw || !gb) return nn_fail(SHL_EINVAL, "linear_backward: bad arguments");
  k_linear_bwd<<<blocks((long long)B * I + (long long)O * I + O, 128), 128, 0, S(stream)>>>(
      x, w, gy, gx, gw, gb, B, I, O);
  return nn_launch("linear_backward");
}

shl_status shl_nn_softplus_forward(const float* x, float* y, long long n, void* stream) {
  if (!x || !y) return nn_fail(SHL_EINVAL, "softplus_forward: bad arguments");
  if (n == 0) return SHL_OK;
  k_softplus_fwd<<<blocks(n, 256), 256, 0, S(stream)>>>(x, y, n);
  return nn_launch("softplus_forward");
}

shl_status shl_nn_softplus_backward(const float* x, const float* gy, float* gx, long long n,
                                    void* stream) {
  if (!x || !gy || !gx) return nn_fail(SHL_EINVAL, "softplus_backward: bad arguments");
  if (n == 0) return SHL_OK;
  k_softplus_bwd<<<blocks(n, 256), 256, 0, S(stream)>>>(x, gy, gx, n);
  return nn_launch("softplus_backward");
}

shl_status shl_nn_gate_forward(const void* c, int c_bf16, const float* delta, const float* scale,
                               int K, float tau, float* y, int nsub, long long HW, void* stream) {
  if (!c || !delta || !y || !(tau > 0.f) || nsub < 0 || (scale && K < 1))
    return nn_fail(SHL_EINVAL, "gate_forward: bad arguments");
  if (nsub == 0 || HW == 0) return SHL_OK;
  dim3 grid(std::max(1, std::min(64, blocks(HW, 256))), nsub);
  if (c_bf16) k_gate_fwd<true><<<grid, 256, 0, S(stream)>>>(c, delta, scale, K, tau, y, HW);
  else k_gate_fwd<false><<<grid, 256, 0, S(stream)>>>(c, delta, scale, K, tau, y, HW);
  return nn_launch("gate_forward");
}

size_t shl_nn_gate_workspace_floats(int nsub) { return (size_t)nsub * 64; }

shl_status shl_nn_gate_backward(const float* c, const float* delta, const float* scale, int K,
                                float tau, const float* gy, float* gc, float* gdelta, int nsub,
                                long long HW, float* ws, void* stream) {
  if (!c || !delta || !gy || !gc || !gdelta || !ws || !(tau > 0.f) || (scale && K < 1))
    return nn_fail(SHL_EINVAL, "gate_backward: bad arguments");
  if (nsub == 0) return SHL_OK;
  const int g = std::max(1, std::min(64, blocks(HW, 256)));
  dim3 grid(g, nsub);
  k_gate_bwd<<<grid, 256, 0, S(stream)>>>(c, delta, scale, K, tau, gy, gc, ws, HW);
  k_rowsum<<<blocks(nsub, 128), 128, 0, S(stream)>>>(ws, gdelta, nsub, g);
  return nn_launch("gate_backward");
}

shl_status shl_nn_mse_forward(const float* a, const float* b, float* out, long long n, float* ws,
                              void* stream) {
  if (!a || !b || !out || !ws || n < 1) return nn_fail(SHL_EINVAL, "mse_forward: bad arguments");
  const int g = std::max(1, std::min(RED_CTAS, blocks(n, 256)));
  k_mse_partial<<<g, 256, 0, S(stream)>>>(a, b, ws, n);
  k_sum<<<1, 256, 0, S(stream)>>>(ws, g, out);
  return nn_launch("mse_forward");   // out = sum of squares; divide by n on the host
}

shl_status shl_nn_mse_backward(const float* a, const float* b, const float* gscale, float* ga,
                               long long n, void* stream) {
  if (!a || !b || !gscale || !ga || n < 1) return nn_fail(SHL_EINVAL, "mse_backward: bad arguments");
  k_mse_bwd<<<blocks(n, 256), 256, 0, S(stream)>>>(a, b, gscale, ga, n);
  return nn_launch("mse_backward");
}

shl_status shl_nn_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1,
                       float b2, float eps, int step, void* stream) {
  if (!p || !g || !m || !v || step < 1) return nn_fail(SHL_EINVAL, "adam: bad arguments");
  if (n == 0) return SHL_OK;
  const double c1 = 1.0 / (1.0 - std::pow((double)b1, step));
  const double c2 = 1.0 / (1.0 - std::pow((double)b2, step));
  k_adam<<<blocks(n, 256), 256, 0, S(stream)>>>(p, g, m, v, n, lr, b1, b2, eps, (float)c1, (float)c2);
  return nn_launch("adam");
}

shl_status shl_nn_mask_mix(const float* f_masked, const unsigned char* mask, const float* f,
                           float* u, long long n, void* stream) {
  if (!f_masked || !mask || !f || !u) return nn_fail(SHL_EINVAL, "mask_mix: bad arguments");
  if (n == 0) return SHL_OK;
  k_mask_mix<<<blocks(n, 256), 256, 0, S(stream)>>>(f_masked, mask, f, u, n);
  return nn_launch("mask_mix");
}

shl_status shl_nn_mask_mix_backward(const unsigned char* mask, const float* gu, float* gf,
                                    long long n, void* stream) {
  if (!mask || !gu || !gf) return nn_fail(SHL_EINVAL, "mask_mix_backward: bad arguments");
  if (n == 0) return SHL_OK;
  k_mask_mix_bwd<<<blocks(n, 256), 256, 0, S(stream)>>>(mask, gu, gf, n);
  return nn_launch("mask_mix_backward");
}

shl_status shl_nn_cast(const void* x, int x_bf16, void* y, long long n, void* stream) {
  if (!x || !y) return nn_fail(SHL_EINVAL, "cast: bad arguments");
  if (n == 0) return SHL_OK;
  if (x_bf16) {
    const int vec = aligned16(x) && aligned16(y);
    k_bf16_to_f32<<<blocks(vec ? (n + 7) / 8 : n, 256), 256, 0, S(stream)>>>(
        static_cast<const __nv_bfloat16*>(x), static_cast<float*>(y), n, vec);
  } else
    k_f32_to_bf16<<<blocks(n, 256), 256, 0, S(stream)>>>(static_cast<const float*>(x),
                                                         static_cast<__nv_bfloat16*>(y), n);
  return nn_launch("cast");
}

shl_status shl_nn_scale_thresholds(const float* d, const float* scale, float* out, int B, int T,
                                   int K, void* stream) {
  if (!d || !scale || !out || B < 0 || T < 0 || K < 0) return nn_fail(SHL_EINVAL, "scale_thresholds: bad arguments");
  if (B * T * K == 0) return SHL_OK;
  k_scale_thresholds<<<blocks((long long)B * T * K, 256), 256, 0, S(stream)>>>(d, scale, out, B, T, K);
  return nn_launch("scale_thresholds");
}

shl_status shl_nn_axpy(const float* x, float a, float* y, long long n, void* stream) {
  if (!x || !y) return nn_fail(SHL_EINVAL, "axpy: bad arguments");
  if (n == 0) return SHL_OK;
  k_axpy<<<blocks(n, 256), 256, 0, S(stream)>>>(x, a, y, n);
  return nn_launch("axpy");
}

}  // extern "C"
