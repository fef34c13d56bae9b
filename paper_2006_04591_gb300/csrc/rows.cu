// rows.cu - row passes of the 2D real FFTs.
//
// k_rows_r2c: a real line of length M is packed as z[n] = x[2n] + i x[2n+1],
// transformed with a length-M/2 complex FFT, and unpacked into the half
// spectrum X[k], k = 0..M/2, using the conjugate-pair split
//   E[k] = (Z[k] + conj Z[M/2-k]) / 2,  O[k] = -i (Z[k] - conj Z[M/2-k]) / 2,
//   X[k] = E[k] + exp(-2 pi i k / M) O[k].
// The hard threshold of the reconstruction (Sec. 4.2) and the inpainting
// residual u = mask (f_masked - f_est) + f_est (Sec. 4.3) are applied to the
// reals as they are loaded.
//
// k_rows_c2r: the inverse.  From the half spectrum it forms
//   Z[k] = (X[k] + conj X[M/2-k]) + i exp(+2 pi i k / M) (X[k] - conj X[M/2-k]),
// runs the unnormalised length-M/2 inverse FFT and writes x[2n] = Re z[n],
// x[2n+1] = Im z[n], which is M times the normalised inverse (callers fold
// the 1/(N M) of IFFT2 into the filter or dual-weight factors).
#include "fft_core.cuh"
#include "internal.h"

namespace shl {

constexpr int ROW_THREADS = 256;

template <int LOG_M>
struct RowCfg {
  static constexpr int M = 1 << LOG_M;
  static constexpr int L = M / 2;                       // complex line length
  static constexpr int R = L < 16 ? L : 16;
  static constexpr int T = L / R;                       // threads per line
  static constexpr int LPC = ROW_THREADS / T;           // lines per CTA
  static constexpr int WORDS = RowLine::words(L);
  static constexpr int Mh = M / 2 + 1;
};

template <int LOG_M, int INM, bool THRESH>
__global__ void __launch_bounds__(ROW_THREADS) k_rows_r2c(RowR2CArgs a) {
  using C = RowCfg<LOG_M>;
  extern __shared__ float2 smem[];
  const int tid = threadIdx.x;
  const int ll = tid / C::T, j = tid % C::T;
  const int line = blockIdx.x * C::LPC + ll;
  const bool valid = line < a.nlines;
  RowLine sm{smem + ll * C::WORDS};

  float tau = 0.f;
  if (THRESH && valid) tau = __ldg(a.thresh + line / a.N);

  float2 v[C::R];
#pragma unroll
  for (int u = 0; u < C::R; ++u) {
    const int p = j + u * C::T;
    float2 z = make_float2(0.f, 0.f);
    if (valid) {
      const size_t off = (size_t)line * C::M + 2 * p;
      if constexpr (INM == IN_F32) {
        z = __ldg(reinterpret_cast<const float2*>(static_cast<const float*>(a.in) + off));
      } else if constexpr (INM == IN_BF16) {
        __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(
            static_cast<const __nv_bfloat16*>(a.in) + off);
        z = __bfloat1622float2(h);
      } else {
        float2 fm = __ldg(reinterpret_cast<const float2*>(static_cast<const float*>(a.in) + off));
        float2 fe = __ldg(reinterpret_cast<const float2*>(a.fest + off));
        uchar2 mk = *reinterpret_cast<const uchar2*>(a.mask + off);
        z.x = mk.x ? fm.x : fe.x;   // m (fm - fe) + fe with m in {0, 1}
        z.y = mk.y ? fm.y : fe.y;
      }
      if (THRESH) {
        if (fabsf(z.x) < tau) z.x = 0.f;
        if (fabsf(z.y) < tau) z.y = 0.f;
      }
    }
    v[u] = z;
  }

  fft_line<C::L, C::R, -1>(v, sm, j, a.tw);

  __syncthreads();
#pragma unroll
  for (int u = 0; u < C::R; ++u) sm.at(j + u * C::T) = v[u];
  __syncthreads();
  if (!valid) return;
  float2* out = a.out + (size_t)line * C::Mh;
#pragma unroll
  for (int u = 0; u < C::R; ++u) {
    const int k = j + u * C::T;
    const float2 A = v[u];
    const float2 B = sm.at((C::L - k) & (C::L - 1));
    const float2 E = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y - B.y));
    // O = -i (A - conj B) / 2 = ((A.y + B.y), -(A.x - B.x)) / 2
    const float2 O = make_float2(0.5f * (A.y + B.y), -0.5f * (A.x - B.x));
    const float2 w = twiddle<-1>(a.tw, k, LOG_M);
    out[k] = cadd(E, cmul(O, w));
    if (k == 0) out[C::L] = make_float2(A.x - A.y, 0.f);
  }
}

template <int LOG_M, bool BF16OUT>
__global__ void __launch_bounds__(ROW_THREADS) k_rows_c2r(RowC2RArgs a) {
  using C = RowCfg<LOG_M>;
  extern __shared__ float2 smem[];
  const int tid = threadIdx.x;
  const int ll = tid / C::T, j = tid % C::T;
  const int line = blockIdx.x * C::LPC + ll;
  const bool valid = line < a.nlines;
  RowLine sm{smem + ll * C::WORDS};

  const float2* in = a.in + (size_t)line * C::Mh;
  float2 v[C::R];
#pragma unroll
  for (int u = 0; u < C::R; ++u) {
    const int k = j + u * C::T;
    float2 z = make_float2(0.f, 0.f);
    if (valid) {
      const float2 A = in[k];
      const float2 B = in[C::L - k];
      // (A + conj B) + i w (A - conj B), w = exp(+2 pi i k / M)
      const float2 S = make_float2(A.x + B.x, A.y - B.y);
      const float2 D = make_float2(A.x - B.x, A.y + B.y);
      const float2 wd = cmul(D, twiddle<+1>(a.tw, k, LOG_M));
      z = make_float2(S.x - wd.y, S.y + wd.x);
    }
    v[u] = z;
  }

  fft_line<C::L, C::R, +1>(v, sm, j, a.tw);

  if (!valid) return;
  const size_t base = (size_t)line * C::M;
#pragma unroll
  for (int u = 0; u < C::R; ++u) {
    const int p = j + u * C::T;
    if constexpr (BF16OUT) {
      *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(a.out) + base + 2 * p) =
          __floats2bfloat162_rn(v[u].x, v[u].y);
    } else {
      *reinterpret_cast<float2*>(static_cast<float*>(a.out) + base + 2 * p) = v[u];
    }
  }
}

template <int LOG_M>
static cudaError_t r2c_dispatch(InMode mode, bool thresh, const RowR2CArgs& a, cudaStream_t st) {
  using C = RowCfg<LOG_M>;
  const int grid = (a.nlines + C::LPC - 1) / C::LPC;
  const size_t sm = (size_t)C::LPC * C::WORDS * sizeof(float2);
  if (grid == 0) return cudaSuccess;
  if (mode == IN_MASKED) {
    k_rows_r2c<LOG_M, IN_MASKED, false><<<grid, ROW_THREADS, sm, st>>>(a);
  } else if (mode == IN_BF16) {
    if (thresh) k_rows_r2c<LOG_M, IN_BF16, true><<<grid, ROW_THREADS, sm, st>>>(a);
    else k_rows_r2c<LOG_M, IN_BF16, false><<<grid, ROW_THREADS, sm, st>>>(a);
  } else {
    if (thresh) k_rows_r2c<LOG_M, IN_F32, true><<<grid, ROW_THREADS, sm, st>>>(a);
    else k_rows_r2c<LOG_M, IN_F32, false><<<grid, ROW_THREADS, sm, st>>>(a);
  }
  return cudaGetLastError();
}

template <int LOG_M>
static cudaError_t c2r_dispatch(bool bf16, const RowC2RArgs& a, cudaStream_t st) {
  using C = RowCfg<LOG_M>;
  const int grid = (a.nlines + C::LPC - 1) / C::LPC;
  const size_t sm = (size_t)C::LPC * C::WORDS * sizeof(float2);
  if (grid == 0) return cudaSuccess;
  if (bf16) k_rows_c2r<LOG_M, true><<<grid, ROW_THREADS, sm, st>>>(a);
  else k_rows_c2r<LOG_M, false><<<grid, ROW_THREADS, sm, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_rows_r2c(int M, InMode mode, bool thresh, const RowR2CArgs& a,
                            cudaStream_t st) {
  switch (ilog2(M)) {
    case 4: return r2c_dispatch<4>(mode, thresh, a, st);
    case 5: return r2c_dispatch<5>(mode, thresh, a, st);
    case 6: return r2c_dispatch<6>(mode, thresh, a, st);
    case 7: return r2c_dispatch<7>(mode, thresh, a, st);
    case 8: return r2c_dispatch<8>(mode, thresh, a, st);
    case 9: return r2c_dispatch<9>(mode, thresh, a, st);
    case 10: return r2c_dispatch<10>(mode, thresh, a, st);
    case 11: return r2c_dispatch<11>(mode, thresh, a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_rows_c2r(int M, bool bf16_out, const RowC2RArgs& a, cudaStream_t st) {
  switch (ilog2(M)) {
    case 4: return c2r_dispatch<4>(bf16_out, a, st);
    case 5: return c2r_dispatch<5>(bf16_out, a, st);
    case 6: return c2r_dispatch<6>(bf16_out, a, st);
    case 7: return c2r_dispatch<7>(bf16_out, a, st);
    case 8: return c2r_dispatch<8>(bf16_out, a, st);
    case 9: return c2r_dispatch<9>(bf16_out, a, st);
    case 10: return c2r_dispatch<10>(bf16_out, a, st);
    case 11: return c2r_dispatch<11>(bf16_out, a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace shl
