// fft_core.cuh - register/shared-memory FFT building blocks for sm_103a.
//
// A length-L complex line is spread over T = L/R threads; thread j holds the
// R elements at positions j + u*T (u = 0..R-1) in registers.  Each pass of
// the Stockham autosort algorithm does one radix-R butterfly per thread in
// registers and exchanges the line through shared memory; the final pass
// leaves thread j holding outputs j + u*T in natural order, the same layout
// the first pass reads, so lines can be loaded from and stored to global
// memory with coalesced accesses in both directions.
//
// Twiddles come from a table tw[q] = exp(-2 pi i q / TW_P) built on the host
// in float64 and rounded once to float32 (no device sin/cos).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "internal.h"

namespace shl {

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// cos(2 pi k / 16), k = 0..4 (exact closed forms: 1, cos(pi/8), sqrt(2)/2,
// sin(pi/8), 0).  Other angles follow by symmetry.
constexpr double C16_1 = 0.92387953251128675613;  // sqrt(2 + sqrt 2) / 2
constexpr double C16_2 = 0.70710678118654752440;  // sqrt(2) / 2
constexpr double C16_3 = 0.38268343236508977173;  // sqrt(2 - sqrt 2) / 2

__host__ __device__ constexpr double cos16(int k) {
  k = ((k % 16) + 16) % 16;
  return k == 0 ? 1.0 : k == 1 ? C16_1 : k == 2 ? C16_2 : k == 3 ? C16_3 : k == 4 ? 0.0
       : k < 8 ? -cos16(8 - k) : k == 8 ? -1.0 : cos16(16 - k);
}
__host__ __device__ constexpr double sin16(int k) { return cos16(k - 4); }

// a * exp(SIGN * 2 pi i * K16 / 16), SIGN = -1 forward, +1 inverse.
// Multiples of 90 degrees are swaps / negations, 45 degrees uses one scale.
template <int K16, int SIGN>
__device__ __forceinline__ float2 rot16(float2 a) {
  constexpr int k = ((K16 * SIGN) % 16 + 16) % 16;
  if constexpr (k == 0) return a;
  else if constexpr (k == 4) return make_float2(-a.y, a.x);
  else if constexpr (k == 8) return make_float2(-a.x, -a.y);
  else if constexpr (k == 12) return make_float2(a.y, -a.x);
  else if constexpr (k == 2 || k == 6 || k == 10 || k == 14) {
    constexpr float s = (float)C16_2;
    // (cos + i sin) with |cos| = |sin| = s
    constexpr float c = (float)cos16(k), si = (float)sin16(k);
    return make_float2((a.x * (c > 0 ? 1.f : -1.f) - a.y * (si > 0 ? 1.f : -1.f)) * s,
                       (a.x * (si > 0 ? 1.f : -1.f) + a.y * (c > 0 ? 1.f : -1.f)) * s);
  } else {
    constexpr float c = (float)cos16(k), s = (float)sin16(k);
    return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
  }
}

template <int N> struct BitRev {
  static __host__ __device__ constexpr int rev(int x) {
    int r = 0;
    for (int b = 1; b < N; b <<= 1) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
  }
};

// In-register DFT of size R (power of two <= 16), natural order in and out.
// Radix-2 decimation in frequency followed by a compile-time bit reversal.
template <int R, int SIGN>
__device__ __forceinline__ void dft_reg(float2* v) {
  if constexpr (R == 1) return;
#pragma unroll
  for (int span = R / 2; span >= 1; span >>= 1) {
#pragma unroll
    for (int start = 0; start < R; start += 2 * span) {
#pragma unroll
      for (int q = 0; q < span; ++q) {
        float2 a = v[start + q], b = v[start + q + span];
        v[start + q] = cadd(a, b);
        float2 d = csub(a, b);
        // twiddle exp(SIGN 2 pi i q / (2 span)) = 16th-roots index q*16/(2 span)
        switch (q * (16 / (2 * span))) {
          case 0: v[start + q + span] = d; break;
          case 1: v[start + q + span] = rot16<1, SIGN>(d); break;
          case 2: v[start + q + span] = rot16<2, SIGN>(d); break;
          case 3: v[start + q + span] = rot16<3, SIGN>(d); break;
          case 4: v[start + q + span] = rot16<4, SIGN>(d); break;
          case 5: v[start + q + span] = rot16<5, SIGN>(d); break;
          case 6: v[start + q + span] = rot16<6, SIGN>(d); break;
          case 7: v[start + q + span] = rot16<7, SIGN>(d); break;
          default: break;
        }
      }
    }
  }
  float2 t[R];
#pragma unroll
  for (int i = 0; i < R; ++i) t[i] = v[i];
#pragma unroll
  for (int i = 0; i < R; ++i) v[i] = t[BitRev<R>::rev(i)];
}

// Twiddle exp(SIGN 2 pi i e / D) for D a power of two dividing TW_P.
template <int SIGN>
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int e, int logD) {
  int q = (e & ((1 << logD) - 1)) << (LOG_TW_P - logD);
  float2 w = __ldg(tw + q);
  return SIGN < 0 ? w : make_float2(w.x, -w.y);
}

// Shared-memory view of one line for the exchanges.
//   RowLine: a contiguous line, one padding slot every 16 elements.
//   ColLine: column c of a tile stored [position][TW]; no padding needed.
struct RowLine {
  float2* base;
  __device__ __forceinline__ float2& at(int p) const { return base[p + (p >> 4)]; }
  static __host__ __device__ constexpr int words(int L) { return L + L / 16; }
};
struct ColLine {
  float2* base;  // &tile[0][c]
  int tw;        // tile width
  __device__ __forceinline__ float2& at(int p) const { return base[p * tw]; }
};

// Full length-L FFT of the line held as v[u] = x[j + u*T].  All T threads of
// every line in the CTA must call this together (it contains __syncthreads).
template <int L, int R, int SIGN, class LINE>
__device__ __forceinline__ void fft_line(float2 (&v)[R], const LINE& sm, int j,
                                         const float2* __restrict__ tw) {
  constexpr int T = L / R;
  constexpr int LOG_L = ilog2(L), LOG_R = ilog2(R);
  constexpr int NFULL = LOG_L / LOG_R;
  constexpr int LAST = 1 << (LOG_L - NFULL * LOG_R);
#pragma unroll
  for (int st = 0; st < NFULL; ++st) {
    const int logNs = st * LOG_R;
    const int Ns = 1 << logNs;
    if (st > 0) {
      const int k = j & (Ns - 1);
#pragma unroll
      for (int u = 1; u < R; ++u) v[u] = cmul(v[u], twiddle<SIGN>(tw, u * k, logNs + LOG_R));
    }
    dft_reg<R, SIGN>(v);
    if (st < NFULL - 1 || LAST > 1) {
      const int idxD = ((j >> logNs) << (logNs + LOG_R)) + (j & (Ns - 1));
      __syncthreads();
#pragma unroll
      for (int u = 0; u < R; ++u) sm.at(idxD + u * Ns) = v[u];
      __syncthreads();
#pragma unroll
      for (int u = 0; u < R; ++u) v[u] = sm.at(j + u * T);
    }
  }
  if constexpr (LAST > 1) {
    constexpr int Q = R / LAST;
    constexpr int logNs = LOG_L - ilog2(LAST);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int k = (j + q * T) & ((1 << logNs) - 1);
      float2 w[LAST];
#pragma unroll
      for (int m = 0; m < LAST; ++m) {
        w[m] = v[q + m * Q];
        if (m > 0) w[m] = cmul(w[m], twiddle<SIGN>(tw, m * k, LOG_L));
      }
      dft_reg<LAST, SIGN>(w);
#pragma unroll
      for (int m = 0; m < LAST; ++m) v[q + m * Q] = w[m];
    }
  }
}

__device__ __forceinline__ float bf16_to_f(__nv_bfloat16 h) { return __bfloat162float(h); }

}  // namespace shl
