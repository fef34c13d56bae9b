// warp_fft.cuh - FFT of one contiguous line by a group of lanes.
//
// A line of L complex values is held by T = L/R lanes (R <= 32), lane j
// owning positions j + u*T.  Groups of T <= 32 lanes sit inside one warp and
// synchronise with __syncwarp; a group of 64 lanes (two warps) uses a named
// barrier.  The Stockham exchanges go through a group-private shared-memory
// line padded by one slot every R elements, which keeps every exchange free
// of bank conflicts.  No CTA-wide barrier is involved, so warps of a CTA
// progress independently.
#pragma once

#include "fft_core.cuh"

namespace shl {

template <int L, int R>
struct LineCfg {
  static constexpr int T = L / R;                   // lanes per line
  static constexpr int LOG_L = ilog2(L), LOG_R = ilog2(R);
  static constexpr int NFULL = LOG_L / LOG_R;
  static constexpr int LAST = 1 << (LOG_L - NFULL * LOG_R);
  static constexpr int WORDS = L + L / R;           // padded line in shared memory
  static_assert(T >= 1 && T <= 64, "line group must fit two warps");
};

// Radix for a line of length L: 32 for the longest lines, else 16.
template <int L> struct LineRadix {
  static constexpr int R = L >= 1024 ? 32 : (L < 16 ? L : 16);
};

__device__ __forceinline__ int pad_index(int p, int logR) { return p + (p >> logR); }

// Synchronise the lanes of one line group, and only those: groups that share
// a warp may run different numbers of loop iterations, so a group narrower
// than a warp synchronises with the mask of its own T aligned lanes.  A group
// spanning two warps uses named barrier bar_id (1..15) over its 64 threads.
template <int T>
__device__ __forceinline__ void group_sync(int bar_id) {
  if constexpr (T < 32) {
    const unsigned lane = threadIdx.x & 31u;
    __syncwarp(((1u << T) - 1u) << (lane & ~(unsigned)(T - 1)));
  } else if constexpr (T == 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(T) : "memory");
  }
}

// Per-lane twiddles of one line FFT, staged in shared memory as [..][lane]
// so that a lane group reads them as consecutive words (one conflict-free
// access per stage and element) instead of scattered table loads.
//   stages st = 1..NFULL-1: w(st, u, j) = exp(-2 pi i u (j mod Ns) / (Ns R)),
//   last stage (radix LAST): w(q, m, j) = exp(-2 pi i m ((j + qT) mod Ns) / L).
// Inverse transforms use the conjugates.
template <int L, int R>
struct LineTw {
  using C = LineCfg<L, R>;
  static constexpr int T = C::T;
  static constexpr int Q = C::LAST > 1 ? R / C::LAST : 0;
  static constexpr int STAGE_WORDS = (C::NFULL - 1) * (R - 1) * T;
  static constexpr int LAST_WORDS = C::LAST > 1 ? Q * (C::LAST - 1) * T : 0;
  static constexpr int WORDS = STAGE_WORDS + LAST_WORDS;

  static __device__ void fill(float2* sm, const float2* __restrict__ tw, int tid, int nthreads) {
    for (int idx = tid; idx < WORDS; idx += nthreads) {
      int e, logD;
      if (idx < STAGE_WORDS) {
        const int st = 1 + idx / ((R - 1) * T);
        const int rem = idx % ((R - 1) * T);
        const int u = 1 + rem / T, j = rem % T;
        const int logNs = st * C::LOG_R;
        e = u * (j & ((1 << logNs) - 1));
        logD = logNs + C::LOG_R;
      } else {
        if constexpr (C::LAST > 1) {
          const int rem = idx - STAGE_WORDS;
          const int qm = rem / T, j = rem % T;
          const int q = qm / (C::LAST - 1), m = 1 + qm % (C::LAST - 1);
          const int logNs = C::LOG_L - ilog2(C::LAST);
          e = m * ((j + q * T) & ((1 << logNs) - 1));
          logD = C::LOG_L;
        } else {
          e = 0;
          logD = 1;
        }
      }
      sm[idx] = twiddle<-1>(tw, e, logD);
    }
  }
};

template <int SIGN>
__device__ __forceinline__ float2 stw(const float2* p) {
  const float2 w = *p;
  return SIGN < 0 ? w : make_float2(w.x, -w.y);
}

// In-place FFT of the line held as v[u] = x[j + u*T]; on return v[u] =
// X[j + u*T].  SIGN = -1 forward, +1 inverse (unnormalised).  sm is the
// group's padded line buffer (LineCfg::WORDS float2); stw_sm holds the
// staged twiddles of LineTw<L, R>.
// Padded position of element p + u * stride when the base p is fixed per lane
// and stride is a multiple of R: pad(p) + u * (stride + stride / R).
template <int R>
__device__ __forceinline__ int pad_base(int p) { return p + (p >> ilog2(R)); }

template <int L, int R, int SIGN>
__device__ __forceinline__ void line_fft(float2 (&v)[R], float2* sm, int j, int bar_id,
                                         const float2* __restrict__ stw_sm) {
  using C = LineCfg<L, R>;
  using W = LineTw<L, R>;
  constexpr int T = C::T;
  constexpr bool T_ALIGNED = (T % R) == 0;         // read stride is a multiple of R
  const int rbase = pad_base<R>(j);
#pragma unroll
  for (int st = 0; st < C::NFULL; ++st) {
    const int logNs = st * C::LOG_R;
    const int Ns = 1 << logNs;
    if (st > 0) {
      const float2* w = stw_sm + (st - 1) * (R - 1) * T + j;
#pragma unroll
      for (int u = 1; u < R; ++u) v[u] = cmul(v[u], stw<SIGN>(w + (u - 1) * T));
    }
    dft_reg<R, SIGN>(v);
    if (st < C::NFULL - 1 || C::LAST > 1) {
      group_sync<T>(bar_id);
      if (st == 0) {
        // positions j R + u: padded j (R + 1) + u
        float2* wp = sm + j * (R + 1);
#pragma unroll
        for (int u = 0; u < R; ++u) wp[u] = v[u];
      } else {
        const int idxD = ((j >> logNs) << (logNs + C::LOG_R)) + (j & (Ns - 1));
        float2* wp = sm + pad_base<R>(idxD);
#pragma unroll
        for (int u = 0; u < R; ++u) wp[u * (Ns + Ns / R)] = v[u];
      }
      group_sync<T>(bar_id);
      if constexpr (T_ALIGNED) {
        const float2* rp = sm + rbase;
#pragma unroll
        for (int u = 0; u < R; ++u) v[u] = rp[u * (T + T / R)];
      } else {
#pragma unroll
        for (int u = 0; u < R; ++u) v[u] = sm[pad_index(j + u * T, C::LOG_R)];
      }
    }
  }
  if constexpr (C::LAST > 1) {
    constexpr int LAST = C::LAST;
    constexpr int Q = R / LAST;
    const float2* wl = stw_sm + W::STAGE_WORDS + j;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      float2 w[LAST];
#pragma unroll
      for (int m = 0; m < LAST; ++m) {
        w[m] = v[q + m * Q];
        if (m > 0) w[m] = cmul(w[m], stw<SIGN>(wl + (q * (LAST - 1) + (m - 1)) * T));
      }
      dft_reg<LAST, SIGN>(w);
#pragma unroll
      for (int m = 0; m < LAST; ++m) v[q + m * Q] = w[m];
    }
  }
}

// Per-lane twiddle bases of the 256- and 512-point lines (R = 16): for lane
// j, [0..3] b, b^2, b^4, b^8 with b = exp(-2 pi i (j mod 16) / 256) (the
// middle-stage twiddles b^u), [4] w0 = exp(-2 pi i j / 512) (the last stage
// of the 512-point line, and with the 32nd roots of unity the real-FFT split
// of a 512-point real row).  Stored [5][T], from the float64-built table.
template <int L, int R>
struct LineTwB {
  static constexpr int T = L / R;
  static constexpr bool OK = (L == 512 || L == 256) && R == 16;
  static constexpr int WORDS = 5 * T;
  static __device__ void fill(float2* sm, const float2* __restrict__ tw, int tid, int nthreads) {
    for (int idx = tid; idx < WORDS; idx += nthreads) {
      const int k = idx / T, j = idx - (idx / T) * T, m = j & 15;
      sm[idx] = __ldg(tw + (k < 4 ? m * (16 << k) : j * 8));
    }
  }
};

// line_fft for the 256- and 512-point lines with the twiddles formed from
// the lane's five bases (LineTwB) in registers: the same Stockham passes and
// exchanges, 4 or 5 shared-memory loads per line instead of 15 or 23
// (middle stage b^u: products of at most two bases; last stage of 512:
// w0 times the 16th roots of unity).
template <int L, int R, int SIGN>
__device__ __forceinline__ void line_fft_b(float2 (&v)[R], float2* sm, int j, int bar_id,
                                           const float2* __restrict__ twb) {
  static_assert(LineTwB<L, R>::OK, "bases exist for 256 and 512 points, radix 16");
  constexpr int T = L / R;
  auto cj = [](float2 a) { return SIGN < 0 ? a : make_float2(a.x, -a.y); };
  dft_reg<R, SIGN>(v);
  group_sync<T>(bar_id);
  {
    float2* wp = sm + j * (R + 1);
#pragma unroll
    for (int u = 0; u < R; ++u) wp[u] = v[u];
  }
  group_sync<T>(bar_id);
  const float2* rp = sm + pad_base<R>(j);
#pragma unroll
  for (int u = 0; u < R; ++u) v[u] = rp[u * (T + T / R)];
  {
    float2 w[R];
    w[1] = cj(twb[j]); w[2] = cj(twb[T + j]); w[4] = cj(twb[2 * T + j]); w[8] = cj(twb[3 * T + j]);
    w[3] = cmul(w[2], w[1]); w[5] = cmul(w[4], w[1]); w[6] = cmul(w[4], w[2]);
    w[7] = cmul(w[4], w[3]); w[9] = cmul(w[8], w[1]); w[10] = cmul(w[8], w[2]);
    w[11] = cmul(w[8], w[3]); w[12] = cmul(w[8], w[4]); w[13] = cmul(w[8], w[5]);
    w[14] = cmul(w[8], w[6]); w[15] = cmul(w[8], w[7]);
#pragma unroll
    for (int u = 1; u < R; ++u) v[u] = cmul(v[u], w[u]);
  }
  dft_reg<R, SIGN>(v);
  if constexpr (L == 512) {
    group_sync<T>(bar_id);
    {
      float2* wp = sm + pad_base<R>(((j >> 4) << 8) + (j & 15));
#pragma unroll
      for (int u = 0; u < R; ++u) wp[u * (R + 1)] = v[u];
    }
    group_sync<T>(bar_id);
#pragma unroll
    for (int u = 0; u < R; ++u) v[u] = rp[u * (T + T / R)];
    const float2 w0 = cj(twb[4 * T + j]);
#pragma unroll
    for (int q = 0; q < R / 2; ++q) {
      float2 x1 = cmul(v[q + R / 2], w0);
      switch (q) {            // times exp(SIGN 2 pi i q / 16)
        case 1: x1 = rot32<2, SIGN>(x1); break;
        case 2: x1 = rot32<4, SIGN>(x1); break;
        case 3: x1 = rot32<6, SIGN>(x1); break;
        case 4: x1 = rot32<8, SIGN>(x1); break;
        case 5: x1 = rot32<10, SIGN>(x1); break;
        case 6: x1 = rot32<12, SIGN>(x1); break;
        case 7: x1 = rot32<14, SIGN>(x1); break;
        default: break;
      }
      const float2 x0 = v[q];
      v[q] = cadd(x0, x1);
      v[q + R / 2] = csub(x0, x1);
    }
  }
}

// line_fft or, where the lane bases exist, line_fft_b.
template <int L, int R, int SIGN>
__device__ __forceinline__ void line_fft_any(float2 (&v)[R], float2* sm, int j, int bar_id,
                                             const float2* __restrict__ stw_sm,
                                             const float2* __restrict__ twb) {
  if constexpr (LineTwB<L, R>::OK) line_fft_b<L, R, SIGN>(v, sm, j, bar_id, twb);
  else line_fft<L, R, SIGN>(v, sm, j, bar_id, stw_sm);
}

// Store v[u] (natural positions j + u T) into the padded line buffer.
template <int L, int R>
__device__ __forceinline__ void line_store(const float2 (&v)[R], float2* sm, int j) {
  constexpr int T = L / R;
  if constexpr (T % R == 0) {
    float2* p = sm + pad_base<R>(j);
#pragma unroll
    for (int u = 0; u < R; ++u) p[u * (T + T / R)] = v[u];
  } else {
#pragma unroll
    for (int u = 0; u < R; ++u) sm[pad_index(j + u * T, ilog2(R))] = v[u];
  }
}

// Load the mirrored elements X[(L - (j + u T)) mod L], u = 0..R-1, from the
// padded line buffer (the conjugate-pair partners of the real-FFT split).
template <int L, int R>
__device__ __forceinline__ void line_load_mirror(float2 (&out)[R], const float2* sm, int j) {
  constexpr int T = L / R;
  if constexpr (T % R == 0) {
    // j > 0: L - j - uT = (T - j) + (R - 1 - u) T;  j == 0: ((R - u) mod R) T
    constexpr int S = T + T / R;
    const float2* p = sm + (j > 0 ? pad_base<R>(T - j) : 0);
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int off = j > 0 ? (R - 1 - u) * S : ((R - u) & (R - 1)) * S;
      out[u] = p[off];
    }
  } else {
#pragma unroll
    for (int u = 0; u < R; ++u) out[u] = sm[pad_index((L - (j + u * T)) & (L - 1), ilog2(R))];
  }
}

}  // namespace shl
