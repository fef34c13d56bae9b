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

// cos(2 pi k / 32) for k = 0..8, closed forms: 1, cos(pi/16), cos(pi/8),
// cos(3pi/16), sqrt(2)/2, sin(3pi/16), sin(pi/8), sin(pi/16), 0.  Every
// other 32nd root of unity follows by symmetry.
constexpr double C32[9] = {
    1.0,
    0.98078528040323044913,   // cos(pi/16) = sqrt(2 + sqrt(2 + sqrt 2)) / 2
    0.92387953251128675613,   // cos(pi/8)  = sqrt(2 + sqrt 2) / 2
    0.83146961230254523708,   // cos(3pi/16) = sqrt(2 + sqrt(2 - sqrt 2)) / 2
    0.70710678118654752440,   // sqrt(2) / 2
    0.55557023301960222474,   // sin(3pi/16) = sqrt(2 - sqrt(2 - sqrt 2)) / 2
    0.38268343236508977173,   // sin(pi/8)  = sqrt(2 - sqrt 2) / 2
    0.19509032201612826785,   // sin(pi/16) = sqrt(2 - sqrt(2 + sqrt 2)) / 2
    0.0};

__host__ __device__ constexpr double cos32(int k) {
  k = ((k % 32) + 32) % 32;
  return k <= 8 ? C32[k] : k < 16 ? -C32[16 - k] : k <= 24 ? -C32[k - 16] : C32[32 - k];
}
__host__ __device__ constexpr double sin32(int k) { return cos32(k - 8); }

// a * exp(SIGN * 2 pi i * K / 32), SIGN = -1 forward, +1 inverse.
// Multiples of 90 degrees are swaps / negations, odd multiples of 45 degrees
// use one scale; the rest a full complex multiply by constants.
template <int K, int SIGN>
__device__ __forceinline__ float2 rot32(float2 a) {
  constexpr int k = ((K * SIGN) % 32 + 32) % 32;
  if constexpr (k == 0) return a;
  else if constexpr (k == 8) return make_float2(-a.y, a.x);
  else if constexpr (k == 16) return make_float2(-a.x, -a.y);
  else if constexpr (k == 24) return make_float2(a.y, -a.x);
  else if constexpr (k % 4 == 0) {
    constexpr float s = (float)C32[4];
    constexpr float sc = cos32(k) > 0 ? 1.f : -1.f, ss = sin32(k) > 0 ? 1.f : -1.f;
    return make_float2((sc * a.x - ss * a.y) * s, (ss * a.x + sc * a.y) * s);
  } else {
    constexpr float c = (float)cos32(k), s = (float)sin32(k);
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

// In-register DFT of size R (power of two <= 32), natural order in and out.
// Radix-2 decimation in frequency followed by a compile-time bit reversal.
template <int R, int SIGN>
__device__ __forceinline__ void dft_reg(float2* v) {
  if constexpr (R == 1) return;
  else {
#pragma unroll
    for (int span = R / 2; span >= 1; span >>= 1) {
#pragma unroll
      for (int start = 0; start < R; start += 2 * span) {
#pragma unroll
        for (int q = 0; q < span; ++q) {
          float2 a = v[start + q], b = v[start + q + span];
          v[start + q] = cadd(a, b);
          float2 d = csub(a, b);
          // twiddle exp(SIGN 2 pi i q / (2 span)), in 32nds: q * 16 / span
          float2 r;
          switch (q * (16 / span)) {
#define SHL_ROT(Q) case Q: r = rot32<Q, SIGN>(d); break;
            SHL_ROT(0) SHL_ROT(1) SHL_ROT(2) SHL_ROT(3) SHL_ROT(4) SHL_ROT(5) SHL_ROT(6)
            SHL_ROT(7) SHL_ROT(8) SHL_ROT(9) SHL_ROT(10) SHL_ROT(11) SHL_ROT(12) SHL_ROT(13)
            SHL_ROT(14) SHL_ROT(15)
#undef SHL_ROT
            default: r = d; break;
          }
          v[start + q + span] = r;
        }
      }
    }
    float2 t[R];
#pragma unroll
    for (int i = 0; i < R; ++i) t[i] = v[i];
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = t[BitRev<R>::rev(i)];
  }
}

// Twiddle exp(SIGN 2 pi i e / D) for D a power of two dividing TW_P.
template <int SIGN>
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int e, int logD) {
  int q = (e & ((1 << logD) - 1)) << (LOG_TW_P - logD);
  float2 w = __ldg(tw + q);
  return SIGN < 0 ? w : make_float2(w.x, -w.y);
}

__device__ __forceinline__ float bf16_to_f(__nv_bfloat16 h) { return __bfloat162float(h); }

}  // namespace shl
