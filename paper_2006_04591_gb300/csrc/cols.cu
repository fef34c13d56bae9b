// cols.cu - column passes over half spectra [N][Mh] (Mh = M/2 + 1).
//
// A CTA owns a tile of TW adjacent columns.  Thread (c, j) holds rows
// j + u*T of column c, so every global access of a warp covers TW adjacent
// complex values of one row.  Modes:
//
//   COL_FWD        X = FFT_y(U) in place (image spectra, decomposition).
//   COL_DEC_INV    Z_s = IFFT_y(G_i * scale [* 1/W] * X_b) for the chunk's
//                  subbands s = b K + i; the filter multiply of Sec. 3.4 is
//                  applied as the column is loaded.
//   COL_REC_ACC    acc_b (+)= sum_{i in chunk} G_i * FFT_y(U_s): the subband
//                  sum of the reconstruction, in registers, in order of i.
//   COL_FINAL_INV  acc_b = IFFT_y(acc_b * scale [* 1/W]) in place: the dual
//                  frame weights of the reconstruction (Sec. 3.4).
#include "fft_core.cuh"
#include "internal.h"

namespace shl {

template <int LOG_N>
struct ColCfg {
  static constexpr int N = 1 << LOG_N;
  static constexpr int R = N < 16 ? N : 16;
  static constexpr int T = N / R;                       // threads per column
  static constexpr int TWc = (512 / T) < 1 ? 1 : ((512 / T) > 32 ? 32 : (512 / T));
  static constexpr int THREADS = TWc * T;
};

template <int LOG_N, int MODE>
__global__ void __launch_bounds__(ColCfg<LOG_N>::THREADS) k_cols(ColArgs a) {
  using C = ColCfg<LOG_N>;
  extern __shared__ float2 smem[];
  const int tid = threadIdx.x;
  const int c = tid % C::TWc, j = tid / C::TWc;
  const int col = blockIdx.x * C::TWc + c;
  const bool valid = col < a.Mh;
  const size_t plane = (size_t)C::N * a.Mh;
  ColLine sm{smem + c, C::TWc};

  float2 v[C::R];

  if constexpr (MODE == COL_FWD || MODE == COL_FINAL_INV) {
    float2* d = a.data + (size_t)blockIdx.y * plane;
#pragma unroll
    for (int u = 0; u < C::R; ++u) {
      const int row = j + u * C::T;
      float2 z = valid ? d[(size_t)row * a.Mh + col] : make_float2(0.f, 0.f);
      if (MODE == COL_FINAL_INV && valid) {
        float s = a.scale;
        if (a.invW) s *= __ldg(a.invW + (size_t)row * a.Mh + col);
        z = cscale(z, s);
      }
      v[u] = z;
    }
    if constexpr (MODE == COL_FWD) fft_line<C::N, C::R, -1>(v, sm, j, a.tw);
    else fft_line<C::N, C::R, +1>(v, sm, j, a.tw);
    if (valid) {
#pragma unroll
      for (int u = 0; u < C::R; ++u) d[(size_t)(j + u * C::T) * a.Mh + col] = v[u];
    }
  } else if constexpr (MODE == COL_DEC_INV) {
    const int s = a.s0 + blockIdx.y;
    const int b = s / a.K, i = s % a.K;
    const float2* X = a.data + (size_t)b * plane;
    const float* G = a.G + (size_t)i * plane;
#pragma unroll
    for (int u = 0; u < C::R; ++u) {
      const size_t o = (size_t)(j + u * C::T) * a.Mh + col;
      float2 z = make_float2(0.f, 0.f);
      if (valid) {
        float g = __ldg(G + o) * a.scale;
        if (a.invW) g *= __ldg(a.invW + o);
        z = cscale(X[o], g);
      }
      v[u] = z;
    }
    fft_line<C::N, C::R, +1>(v, sm, j, a.tw);
    if (valid) {
      float2* out = a.out + (size_t)blockIdx.y * plane;
#pragma unroll
      for (int u = 0; u < C::R; ++u) out[(size_t)(j + u * C::T) * a.Mh + col] = v[u];
    }
  } else {  // COL_REC_ACC
    const int b = a.b_lo + blockIdx.y;
    const int s_begin = max(a.s0, b * a.K), s_end = min(a.s0 + a.S, (b + 1) * a.K);
    float2 acc[C::R];
#pragma unroll
    for (int u = 0; u < C::R; ++u) acc[u] = make_float2(0.f, 0.f);
    for (int s = s_begin; s < s_end; ++s) {
      const float2* U = a.in + (size_t)(s - a.s0) * plane;
      const float* G = a.G + (size_t)(s - b * a.K) * plane;
#pragma unroll
      for (int u = 0; u < C::R; ++u)
        v[u] = valid ? U[(size_t)(j + u * C::T) * a.Mh + col] : make_float2(0.f, 0.f);
      fft_line<C::N, C::R, -1>(v, sm, j, a.tw);
      if (valid) {
#pragma unroll
        for (int u = 0; u < C::R; ++u) {
          const float g = __ldg(G + (size_t)(j + u * C::T) * a.Mh + col);
          acc[u].x = fmaf(g, v[u].x, acc[u].x);
          acc[u].y = fmaf(g, v[u].y, acc[u].y);
        }
      }
    }
    if (valid) {
      float2* A = a.acc + (size_t)b * plane;
      const bool first = (s_begin == b * a.K);
#pragma unroll
      for (int u = 0; u < C::R; ++u) {
        const size_t o = (size_t)(j + u * C::T) * a.Mh + col;
        A[o] = first ? acc[u] : cadd(A[o], acc[u]);
      }
    }
  }
}

template <int LOG_N>
static cudaError_t cols_dispatch(ColMode mode, const ColArgs& a, int grid_y, cudaStream_t st) {
  using C = ColCfg<LOG_N>;
  const dim3 grid((a.Mh + C::TWc - 1) / C::TWc, grid_y);
  const size_t sm = (size_t)C::N * C::TWc * sizeof(float2);
  if (grid_y == 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  switch (mode) {
#define SHL_COL_CASE(MD)                                                                  \
  case MD:                                                                                \
    if (sm > 48 * 1024)                                                                   \
      e = cudaFuncSetAttribute(k_cols<LOG_N, MD>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                               (int)sm);                                                  \
    if (e != cudaSuccess) return e;                                                       \
    k_cols<LOG_N, MD><<<grid, C::THREADS, sm, st>>>(a);                                   \
    break;
    SHL_COL_CASE(COL_FWD)
    SHL_COL_CASE(COL_DEC_INV)
    SHL_COL_CASE(COL_REC_ACC)
    SHL_COL_CASE(COL_FINAL_INV)
#undef SHL_COL_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_cols(int N, ColMode mode, const ColArgs& a, int grid_y, cudaStream_t st) {
  switch (ilog2(N)) {
    case 4: return cols_dispatch<4>(mode, a, grid_y, st);
    case 5: return cols_dispatch<5>(mode, a, grid_y, st);
    case 6: return cols_dispatch<6>(mode, a, grid_y, st);
    case 7: return cols_dispatch<7>(mode, a, grid_y, st);
    case 8: return cols_dispatch<8>(mode, a, grid_y, st);
    case 9: return cols_dispatch<9>(mode, a, grid_y, st);
    case 10: return cols_dispatch<10>(mode, a, grid_y, st);
    case 11: return cols_dispatch<11>(mode, a, grid_y, st);
    default: return cudaErrorInvalidValue;
  }
}

// Per-subband max |c| (optionally divided by RMS_i): one CTA per subband.
template <bool BF16>
__global__ void __launch_bounds__(256) k_absmax(const void* coeffs, int K, size_t elems,
                                                const float* rms, float* out) {
  const int s = blockIdx.x;
  float m = 0.f;
  if constexpr (BF16) {
    const __nv_bfloat16* p = static_cast<const __nv_bfloat16*>(coeffs) + (size_t)s * elems;
    for (size_t e = threadIdx.x; e < elems; e += blockDim.x) m = fmaxf(m, fabsf(__bfloat162float(p[e])));
  } else {
    const float* p = static_cast<const float*>(coeffs) + (size_t)s * elems;
    for (size_t e = threadIdx.x; e < elems; e += blockDim.x) m = fmaxf(m, fabsf(__ldg(p + e)));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float r = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, red[w]);
    out[s] = rms ? r / rms[s % K] : r;
  }
}

cudaError_t launch_absmax(const void* coeffs, bool bf16, int nsub, int K, size_t elems,
                          const float* rms, float* out, cudaStream_t st) {
  if (nsub == 0) return cudaSuccess;
  if (bf16) k_absmax<true><<<nsub, 256, 0, st>>>(coeffs, K, elems, rms, out);
  else k_absmax<false><<<nsub, 256, 0, st>>>(coeffs, K, elems, rms, out);
  return cudaGetLastError();
}

}  // namespace shl
