// general.cu - transform kernels for any image size and for complex
// Hermitian filter spectra: the decomposition, reconstruction and adjoint of
// Sec. 3.4 on row-major half-spectrum planes [N][M/2+1] in natural DFT order
// (real images and Hermitian filters give Hermitian spectra, so columns
// 0..M/2 determine the rest).
//
//   k_rows<ROW_FWD>     real rows (threshold-on-read or masked input) ->
//                       forward row DFT -> half-spectrum planes.
//   k_rows<ROW_INV>     Hermitian rows -> inverse row DFT -> real part * scale
//                       -> float32 / bfloat16.
//   k_rows<ROW_SHRINK>  in place: inverse row DFT -> hard threshold ->
//                       forward row DFT (denoise / IHT).
//   k_cols<COL_FWD>     in-place forward column DFT (image spectra).
//   k_cols<COL_DEC>     G_i * X_b [* 1/W] formed in the load, inverse column
//                       DFT, stored to the staging planes.
//   k_cols<COL_REC>     per image: forward column DFT of each staged subband,
//                       conj(G_i) multiply, fixed-order sum in registers;
//                       then 1/W and the inverse column DFT.
//
// A row CTA transforms C lines, each holding two real rows of one plane (real
// and imaginary parts of one complex DFT).  A column CTA owns C adjacent
// columns of one plane and reads and writes them as C * 8-byte runs of each
// row.  Lines live in shared memory with pitch P + 1 float2, so that the
// column tiles hit distinct banks.
//
// Line DFT.  Length P = r_1 r_2 ... r_s (all factors <= 61): Stockham's
// autosort FFT,
//   out[g Ns R + q Ns + k] = sum_{m<R} in[g Ns + k + m P/R] w^(m (k + q Ns) P/(Ns R)),
// w = exp(-2 pi i / P), R the stage radix, Ns the product of the earlier
// radices, 0 <= k < Ns, 0 <= q < R: each thread twiddles one butterfly's R
// inputs by w^(m k P/(Ns R)) and runs the length-R DFT in registers (radix
// 2, 3, 4, 8 in closed form, 5 and 7 against the table's roots; larger prime
// radices one output per thread).  A length with a prime factor above 61
// goes through Bluestein's chirp-z identity n k = (n^2 + k^2 - (k - n)^2)/2:
//   X[k] = c[k] sum_n (x[n] c[n]) conj(c[k - n]),  c[n] = exp(-i pi n^2 / L),
// a circular convolution of length P (power of two >= 2L - 1) evaluated with
// two length-P FFTs against the precomputed DFT_P of the chirp kernel.  The
// inverse DFT is conj(DFT(conj x)) (exact in floating point), so one forward
// plan serves both directions.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>

#include "general.h"

namespace shl {
namespace gen {
namespace {

constexpr int ROW_THREADS = 256;
constexpr int COL_THREADS = 256;
constexpr int MAX_LINES = 16;          // lines per CTA
constexpr int ROW_ELEMS = 2048;        // target C * P of a row CTA (32 KB of lines)
constexpr size_t COL_SMEM_CAP = 72 * 1024;   // the two line buffers of a column CTA
constexpr int COL_LINES_MAX = 6;        // columns per CTA (4, 6, 8 measured at 480..512 rows)
constexpr int COL_ACC = 16;            // accumulator elements per thread (C * N <= 16 * 256)

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {   // conj(a) * b
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 conj2(float2 a) { return make_float2(a.x, -a.y); }

// floor(n / d) for 0 <= n < 2^22, given r = 1/d rounded to nearest: n + 1/2
// lies at least 1/(2d) from a multiple of d, and the two float roundings move
// (n + 1/2) r by less than (n + 1/2)/d * 2^-23 < 1/(2d).
__device__ __forceinline__ int qdiv(int n, float r) {
  return __float2int_rz(((float)n + 0.5f) * r);
}

// ---------------------------------------------------------- butterflies
// In-register forward DFTs of length R (sign -1).
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  const float2 t = a;
  a = make_float2(t.x + b.x, t.y + b.y);
  b = make_float2(t.x - b.x, t.y - b.y);
}
__device__ __forceinline__ void dft4(float2& a, float2& b, float2& c, float2& d) {
  const float2 t0 = make_float2(a.x + c.x, a.y + c.y), t1 = make_float2(a.x - c.x, a.y - c.y);
  const float2 t2 = make_float2(b.x + d.x, b.y + d.y), t3 = make_float2(b.x - d.x, b.y - d.y);
  a = make_float2(t0.x + t2.x, t0.y + t2.y);
  c = make_float2(t0.x - t2.x, t0.y - t2.y);
  b = make_float2(t1.x + t3.y, t1.y - t3.x);      // t1 - i t3
  d = make_float2(t1.x - t3.y, t1.y + t3.x);      // t1 + i t3
}

template <int R>
struct Dft;
template <>
struct Dft<2> {
  __device__ __forceinline__ static void run(float2 (&v)[2], const float2*, int) { dft2(v[0], v[1]); }
};
template <>
struct Dft<4> {
  __device__ __forceinline__ static void run(float2 (&v)[4], const float2*, int) {
    dft4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct Dft<8> {   // two length-4 DFTs of the even and odd samples, then w8^k
  __device__ __forceinline__ static void run(float2 (&v)[8], const float2*, int) {
    constexpr float h = 0.70710678118654752440f;
    dft4(v[0], v[2], v[4], v[6]);
    dft4(v[1], v[3], v[5], v[7]);
    const float2 o1 = make_float2(h * (v[3].x + v[3].y), h * (v[3].y - v[3].x));   // w8 o1
    const float2 o2 = make_float2(v[5].y, -v[5].x);                                // w8^2 o2
    const float2 o3 = make_float2(h * (v[7].y - v[7].x), -h * (v[7].x + v[7].y));  // w8^3 o3
    const float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
    v[0] = make_float2(e0.x + o0.x, e0.y + o0.y);
    v[4] = make_float2(e0.x - o0.x, e0.y - o0.y);
    v[1] = make_float2(e1.x + o1.x, e1.y + o1.y);
    v[5] = make_float2(e1.x - o1.x, e1.y - o1.y);
    v[2] = make_float2(e2.x + o2.x, e2.y + o2.y);
    v[6] = make_float2(e2.x - o2.x, e2.y - o2.y);
    v[3] = make_float2(e3.x + o3.x, e3.y + o3.y);
    v[7] = make_float2(e3.x - o3.x, e3.y - o3.y);
  }
};
template <>
struct Dft<3> {
  __device__ __forceinline__ static void run(float2 (&v)[3], const float2*, int) {
    constexpr float h = 0.86602540378443864676f;   // sin(2 pi / 3)
    const float2 s = make_float2(v[1].x + v[2].x, v[1].y + v[2].y);
    const float2 d = make_float2(v[1].x - v[2].x, v[1].y - v[2].y);
    const float2 m = make_float2(v[0].x - 0.5f * s.x, v[0].y - 0.5f * s.y);
    v[0] = make_float2(v[0].x + s.x, v[0].y + s.y);
    v[1] = make_float2(m.x + h * d.y, m.y - h * d.x);
    v[2] = make_float2(m.x - h * d.y, m.y + h * d.x);
  }
};
// Odd prime R (5, 7): X_q = sum_m v_m w_R^(q m mod R), the roots read from the
// length-P table (w_R = w^(P/R)).
template <int R>
struct Dft {
  __device__ __forceinline__ static void run(float2 (&v)[R], const float2* tw, int PR) {
    float2 om[R];
#pragma unroll
    for (int j = 1; j < R; ++j) om[j] = __ldg(tw + j * PR);
    float2 out[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      float2 acc = v[0];
#pragma unroll
      for (int m = 1; m < R; ++m) {
        const float2 w = om[(q * m) % R == 0 ? 1 : (q * m) % R];
        if ((q * m) % R == 0) {
          acc.x += v[m].x;
          acc.y += v[m].y;
        } else {
          acc.x = fmaf(v[m].x, w.x, fmaf(-v[m].y, w.y, acc.x));
          acc.y = fmaf(v[m].x, w.y, fmaf(v[m].y, w.x, acc.y));
        }
      }
      out[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = out[q];
  }
};

// 8-byte asynchronous global -> shared copies (cp.async) and their waits.
__device__ __forceinline__ void gcp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void gcp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void gcp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// One Stockham stage of radix R, one butterfly j = g Ns + k per thread:
// twiddle input m by w^(m k P/(Ns R)), DFT_R, store output q at
// g Ns R + q Ns + k.
template <int R>
__device__ __forceinline__ void stage_r(const float2* src, float2* dst, int C, int pitch, int P,
                                        int Ns, const float2* tw) {
  const int nb = P / R, tstep = P / (Ns * R);
  const float rnb = __frcp_rn((float)nb), rNs = __frcp_rn((float)Ns);
  for (int t = threadIdx.x; t < C * nb; t += blockDim.x) {
    const int l = qdiv(t, rnb), j = t - l * nb;
    const int g = qdiv(j, rNs), k = j - g * Ns;
    const float2* s = src + l * pitch + j;
    float2 v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = s[m * nb];
    if (Ns > 1) {
      const int e = k * tstep;                      // m e < P for m < R
#pragma unroll
      for (int m = 1; m < R; ++m) v[m] = cmul(v[m], __ldg(tw + m * e));
    }
    Dft<R>::run(v, tw, nb);
    float2* d = dst + l * pitch + g * Ns * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) d[q * Ns] = v[q];
  }
}

// Radix R > 7: one output element per thread, the R-term sum in a loop.
__device__ void stage_generic(const float2* src, float2* dst, int C, int pitch, int P, int R,
                              int Ns, const float2* tw) {
  const int stride = P / R, span = Ns * R, tstep = P / span;
  const float rP = __frcp_rn((float)P);
  const float rNs = __frcp_rn((float)Ns), rR = __frcp_rn((float)R);
  for (int idx = threadIdx.x; idx < C * P; idx += blockDim.x) {
    const int l = qdiv(idx, rP), o = idx - l * P;
    const int qg = qdiv(o, rNs), k = o - qg * Ns;
    const int g = qdiv(qg, rR), q = qg - g * R;
    const float2* s = src + l * pitch + g * Ns + k;
    const int base = (k + q * Ns) * tstep;       // < P
    float2 acc = s[0];
    int ex = 0;
    for (int m = 1; m < R; ++m) {
      ex += base;
      if (ex >= P) ex -= P;
      const float2 w = __ldg(tw + ex), v = s[m * stride];
      acc.x = fmaf(v.x, w.x, fmaf(-v.y, w.y, acc.x));
      acc.y = fmaf(v.x, w.y, fmaf(v.y, w.x, acc.y));
    }
    dst[l * pitch + o] = acc;
  }
}

// Forward FFT of length p.P on C lines at src[l * pitch + e], ping-ponging
// with dst; returns the buffer that holds the result.  Stockham stages
// (stage radix R, Ns = product of the earlier radices):
//   out[g Ns R + q Ns + k] = sum_m in[g Ns + k + m P/R] w^(m (k + q Ns) P/(Ns R)).
// Every stage ends with a barrier; the caller has synchronised after
// writing src.
__device__ float2* stockham(float2* src, float2* dst, int C, int pitch, const LinePlan& p) {
  const int P = p.P;
  int Ns = 1;
  for (int st = 0; st < p.nst; ++st) {
    const int R = p.radix[st];
    switch (R) {
      case 2: stage_r<2>(src, dst, C, pitch, P, Ns, p.tw); break;
      case 3: stage_r<3>(src, dst, C, pitch, P, Ns, p.tw); break;
      case 4: stage_r<4>(src, dst, C, pitch, P, Ns, p.tw); break;
      case 5: stage_r<5>(src, dst, C, pitch, P, Ns, p.tw); break;
      case 7: stage_r<7>(src, dst, C, pitch, P, Ns, p.tw); break;
      case 8: stage_r<8>(src, dst, C, pitch, P, Ns, p.tw); break;
      default: stage_generic(src, dst, C, pitch, P, R, Ns, p.tw); break;
    }
    __syncthreads();
    float2* t = src;
    src = dst;
    dst = t;
    Ns *= R;
  }
  return src;
}

// Forward DFT of length p.L of the C lines at buf[l * pitch + n], n < L
// (entries L..P-1 need not be set).  Returns the buffer holding X[k] at
// [l * pitch + k], k < L.  Begins and ends with a barrier.
__device__ float2* line_dft(float2* buf, float2* alt, int C, int pitch, const LinePlan& p) {
  __syncthreads();
  if (!p.bluestein) return stockham(buf, alt, C, pitch, p);
  const int P = p.P, L = p.L;
  const float rP = __frcp_rn((float)P);
  for (int idx = threadIdx.x; idx < C * P; idx += blockDim.x) {
    const int l = qdiv(idx, rP), n = idx - l * P;
    float2* e = buf + l * pitch + n;
    *e = n < L ? cmul(*e, __ldg(p.chirp + n)) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2* r = stockham(buf, alt, C, pitch, p);
  for (int idx = threadIdx.x; idx < C * P; idx += blockDim.x) {
    const int l = qdiv(idx, rP), n = idx - l * P;
    float2* e = r + l * pitch + n;
    *e = conj2(cmul(*e, __ldg(p.kern + n)));     // conj(FFT(a) * DFT_P(h) / P)
  }
  __syncthreads();
  float2* r2 = stockham(r, r == buf ? alt : buf, C, pitch, p);
  for (int idx = threadIdx.x; idx < C * P; idx += blockDim.x) {
    const int l = qdiv(idx, rP), n = idx - l * P;
    if (n < L) {
      float2* e = r2 + l * pitch + n;
      *e = cmul(__ldg(p.chirp + n), conj2(*e));  // c[k] (a conv h)[k]
    }
  }
  __syncthreads();
  return r2;
}

// ------------------------------------------------------------------ rows
enum RowKind : int { ROW_FWD = 0, ROW_INV = 1, ROW_SHRINK = 2 };

struct RowArgs {
  LinePlan pm;               // rows: length M
  const void* in;            // ROW_FWD: [nplanes][N][M] reals (f_masked when masked)
  const uint8_t* mask;       // ROW_FWD masked
  const float* fest;         // ROW_FWD masked
  const float* thresh;       // [nplanes] or null (ROW_FWD), [nplanes] (ROW_SHRINK)
  float2* z;                 // half-spectrum planes [nplanes][N][M/2+1]: ROW_FWD out,
                             // ROW_INV in, ROW_SHRINK in / out
  void* out;                 // ROW_INV: float32 / bfloat16 [nplanes][N][M]
  float scale;               // ROW_INV, ROW_SHRINK: 1/(N M)
  int N, nplanes, C, pitch;
  int mode;                  // ROW_FWD: RowIn; ROW_INV: 1 = bfloat16 out
};

// Two real rows share one complex line DFT: rows 2m and 2m+1 of a plane go
// into the real and imaginary parts (the last row of an odd-height plane is
// paired with zeros).  Forward: z = x_a + i x_b, Z = DFT(z), X_a[k] =
// (Z[k] + conj Z[-k])/2, X_b[k] = (Z[k] - conj Z[-k])/(2i).  Inverse (real
// part wanted): IDFT(T_a + i T_b) = x_a + i x_b for Hermitian T_a, T_b.  The
// pairing depends only on (plane, row), never on how planes are chunked.
template <int KIND>
__global__ void __launch_bounds__(ROW_THREADS) k_rows(const RowArgs a) {
  extern __shared__ float2 sm[];
  __shared__ int s_ra[MAX_LINES];       // global index of the line's first row
  __shared__ int s_hb[MAX_LINES];       // 1: the line has a second row
  __shared__ float s_tau[MAX_LINES];    // threshold of the line's plane
  const LinePlan& p = a.pm;
  const int M = p.L, Mh = M / 2 + 1;                  // row length, stored half width
  const int Np = (a.N + 1) / 2;                       // lines per plane
  const int L0 = blockIdx.x * a.C;
  const int C = min(a.C, Np * a.nplanes - L0);
  float2* buf = sm;
  float2* alt = sm + (size_t)a.C * a.pitch;
  if (threadIdx.x < C) {
    const int lg = L0 + threadIdx.x, pl = lg / Np, m = lg - pl * Np;
    s_ra[threadIdx.x] = pl * a.N + 2 * m;
    s_hb[threadIdx.x] = 2 * m + 1 < a.N;
    s_tau[threadIdx.x] = a.thresh ? __ldg(a.thresh + pl) : 0.f;
  }
  __syncthreads();
  const float rM = __frcp_rn((float)M);
  for (int idx = threadIdx.x; idx < C * M; idx += blockDim.x) {
    const int l = qdiv(idx, rM), e = idx - l * M;
    const bool hb = s_hb[l];
    float2 v;
    if constexpr (KIND == ROW_FWD) {
      const size_t ga = (size_t)s_ra[l] * M + e, gb = ga + M;
      float xa, xb = 0.f;
      if (a.mode == RIN_BF16) {
        const __nv_bfloat16* in = static_cast<const __nv_bfloat16*>(a.in);
        xa = __bfloat162float(in[ga]);
        if (hb) xb = __bfloat162float(in[gb]);
      } else if (a.mode == RIN_MASKED) {
        const float* in = static_cast<const float*>(a.in);
        xa = a.mask[ga] ? in[ga] : a.fest[ga];
        if (hb) xb = a.mask[gb] ? in[gb] : a.fest[gb];
      } else {
        const float* in = static_cast<const float*>(a.in);
        xa = in[ga];
        if (hb) xb = in[gb];
      }
      if (a.thresh) {                                  // ties kept
        if (fabsf(xa) < s_tau[l]) xa = 0.f;
        if (fabsf(xb) < s_tau[l]) xb = 0.f;
      }
      v = make_float2(xa, xb);
    } else {
      // Hermitian rows from their stored half: T[e] for e < Mh, conj T[M - e]
      // above; the DC and (even M) Nyquist bins keep their real parts only.
      const bool up = e >= Mh;
      const int eh = up ? M - e : e;
      const size_t ga = (size_t)s_ra[l] * Mh + eh, gb = ga + Mh;
      float2 ta = a.z[ga], tb = hb ? a.z[gb] : make_float2(0.f, 0.f);
      if (up) { ta.y = -ta.y; tb.y = -tb.y; }
      if (e == 0 || 2 * e == M) { ta.y = 0.f; tb.y = 0.f; }
      v = make_float2(ta.x - tb.y, -(ta.y + tb.x));   // conj(T_a + i T_b)
    }
    buf[l * a.pitch + e] = v;
  }
  float2* res = line_dft(buf, alt, C, a.pitch, p);      // conj of the inverse for INV / SHRINK
  if constexpr (KIND == ROW_SHRINK) {
    float2* other = res == buf ? alt : buf;
    for (int idx = threadIdx.x; idx < C * M; idx += blockDim.x) {
      const int l = qdiv(idx, rM), e = idx - l * M;
      const float2 r = res[l * a.pitch + e];
      float ca = r.x * a.scale, cb = -r.y * a.scale;  // x_a, x_b
      if (fabsf(ca) < s_tau[l]) ca = 0.f;
      if (fabsf(cb) < s_tau[l]) cb = 0.f;
      other[l * a.pitch + e] = make_float2(ca, cb);
    }
    res = line_dft(other, res, C, a.pitch, p);
  }
  if constexpr (KIND == ROW_INV) {
    for (int idx = threadIdx.x; idx < C * M; idx += blockDim.x) {
      const int l = qdiv(idx, rM), e = idx - l * M;
      const bool hb = s_hb[l];
      const size_t ga = (size_t)s_ra[l] * M + e, gb = ga + M;
      const float2 r = res[l * a.pitch + e];
      const float xa = r.x * a.scale, xb = -r.y * a.scale;
      if (a.mode) {
        __nv_bfloat16* out = static_cast<__nv_bfloat16*>(a.out);
        out[ga] = __float2bfloat16_rn(xa);
        if (hb) out[gb] = __float2bfloat16_rn(xb);
      } else {
        float* out = static_cast<float*>(a.out);
        out[ga] = xa;
        if (hb) out[gb] = xb;
      }
    }
  } else {                                            // half spectra of both rows
    const float rMh = __frcp_rn((float)Mh);
    for (int idx = threadIdx.x; idx < C * Mh; idx += blockDim.x) {
      const int l = qdiv(idx, rMh), e = idx - l * Mh;
      const size_t ga = (size_t)s_ra[l] * Mh + e, gb = ga + Mh;
      const float2 zk = res[l * a.pitch + e], zn = res[l * a.pitch + (e ? M - e : 0)];
      a.z[ga] = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
      if (s_hb[l]) a.z[gb] = make_float2(0.5f * (zk.y + zn.y), 0.5f * (zn.x - zk.x));
    }
  }
}

// --------------------------------------------------------------- columns
enum ColKind : int { COL_FWD = 0, COL_DEC = 1, COL_REC = 2, COL_FIN = 3 };

struct ColArgs {
  LinePlan pn;               // columns: length N
  const float2* X;           // COL_DEC: image spectra [B][N][W]
  float2* T;                 // COL_DEC out / COL_REC in: staging [S][N][W]
  float2* A;                 // COL_FWD planes (in place) / COL_REC accumulators [B][N][W]
  const void* G;             // float [K][N][W] or float2 [K][N][W]
  const float* invW;         // [N][W] or null
  int W, K, s0, S, C, pitch, cplx;   // W = M/2 + 1 stored columns
  int groups;                // COL_REC / COL_FIN: subband groups per image (blockIdx.z)
};

// Subbands [sa, sb) of image b in the chunk s0 .. s0+S-1, and their group g
// of `groups`: [lo, hi) (possibly empty).
struct RecRange {
  int b, sa, sb, lo, hi;
  bool first, last;
};
__device__ __forceinline__ RecRange rec_range(const ColArgs& a, int img, int g) {
  RecRange r;
  r.b = a.s0 / a.K + img;
  r.sa = max(a.s0, r.b * a.K);
  r.sb = min(a.s0 + a.S, (r.b + 1) * a.K);
  r.first = r.sa == r.b * a.K;
  r.last = r.sb == (r.b + 1) * a.K;
  const int n = r.sb - r.sa;
  r.lo = r.sa + (g * n) / a.groups;
  r.hi = r.sa + ((g + 1) * n) / a.groups;
  return r;
}

__device__ __forceinline__ float2 filter_at(const ColArgs& a, int i, size_t e, size_t plane) {
  if (a.cplx) return __ldg(static_cast<const float2*>(a.G) + (size_t)i * plane + e);
  return make_float2(__ldg(static_cast<const float*>(a.G) + (size_t)i * plane + e), 0.f);
}

// A column CTA owns columns col0 .. col0+C-1 of one plane (or image).  Thread
// t owns tile elements idx = t + u * blockDim.x, (y, c) = (idx / C, idx % C),
// at offset y * W + col0 + c of a plane, in every loop below, so the
// reconstruction keeps its running sum for those elements in registers.
template <int KIND>
__global__ void __launch_bounds__(COL_THREADS) k_cols(const ColArgs a) {
  extern __shared__ float2 sm[];
  const LinePlan& p = a.pn;
  const int N = p.L, W = a.W;
  const size_t plane = (size_t)N * W;
  const int col0 = blockIdx.x * a.C;
  const int C = min(a.C, W - col0);
  const int NC = N * C;
  float2* buf = sm;
  float2* alt = sm + (size_t)a.C * a.pitch;
  const float rC = __frcp_rn((float)C);
  if constexpr (KIND == COL_FWD) {
    float2* pl = a.A + (size_t)blockIdx.y * plane;
    for (int idx = threadIdx.x; idx < NC; idx += blockDim.x) {
      const int y = qdiv(idx, rC), c = idx - y * C;
      buf[c * a.pitch + y] = pl[(size_t)y * W + col0 + c];
    }
    float2* res = line_dft(buf, alt, C, a.pitch, p);
    for (int idx = threadIdx.x; idx < NC; idx += blockDim.x) {
      const int y = qdiv(idx, rC), c = idx - y * C;
      pl[(size_t)y * W + col0 + c] = res[c * a.pitch + y];
    }
  } else if constexpr (KIND == COL_DEC) {
    const int s = a.s0 + blockIdx.y, b = s / a.K, i = s - b * a.K;
    const float2* Xb = a.X + (size_t)b * plane;
    for (int idx = threadIdx.x; idx < NC; idx += blockDim.x) {
      const int y = qdiv(idx, rC), c = idx - y * C;
      const size_t e = (size_t)y * W + col0 + c;
      float2 v = cmul(filter_at(a, i, e, plane), Xb[e]);
      if (a.invW) {
        const float w = __ldg(a.invW + e);
        v.x *= w;
        v.y *= w;
      }
      buf[c * a.pitch + y] = conj2(v);
    }
    float2* res = line_dft(buf, alt, C, a.pitch, p);
    float2* Ts = a.T + (size_t)blockIdx.y * plane;
    for (int idx = threadIdx.x; idx < NC; idx += blockDim.x) {
      const int y = qdiv(idx, rC), c = idx - y * C;
      Ts[(size_t)y * W + col0 + c] = conj2(res[c * a.pitch + y]);
    }
  } else if constexpr (KIND == COL_REC) {
    // group blockIdx.z of image blockIdx.y: its subbands' column DFTs times
    // conj(G_i), summed in order of i in registers, written over the
    // columns of the group's first staging plane (which only this CTA reads).
    // Three tile buffers rotate: subband s is transformed in `in` (with `al`
    // as the Stockham partner) while the staged columns of subband s + 1 are
    // copied (cp.async) into `nx`.
    const RecRange r = rec_range(a, blockIdx.y, blockIdx.z);
    if (r.lo >= r.hi) return;
    float2 acc[COL_ACC];
#pragma unroll
    for (int u = 0; u < COL_ACC; ++u) acc[u] = make_float2(0.f, 0.f);
    float2* in = sm + 2 * (size_t)a.C * a.pitch;
    float2* al = buf;
    float2* nx = alt;
    for (int s = r.lo - 1; s < r.hi; ++s) {
      if (s >= r.lo) gcp_wait_all();        // this thread's copies of subband s
      if (s + 1 < r.hi) {                   // nx was last read before the loop's closing barrier
        const float2* Ts = a.T + (size_t)(s + 1 - a.s0) * plane;
        float2* dst = s >= r.lo ? nx : in;
        for (int idx = threadIdx.x; idx < NC; idx += blockDim.x) {
          const int y = qdiv(idx, rC), c = idx - y * C;
          gcp_async8(dst + c * a.pitch + y, Ts + (size_t)y * W + col0 + c);
        }
        gcp_commit();
      }
      if (s < r.lo) continue;
      const int i = s - r.b * a.K;
      float2* res = line_dft(in, al, C, a.pitch, p);   // begins with a barrier
#pragma unroll
      for (int u = 0; u < COL_ACC; ++u) {
        const int idx = threadIdx.x + u * COL_THREADS;
        if (idx < NC) {
          const int y = qdiv(idx, rC), c = idx - y * C;
          const float2 t = cmulc(filter_at(a, i, (size_t)y * W + col0 + c, plane),
                                 res[c * a.pitch + y]);
          acc[u].x += t.x;
          acc[u].y += t.y;
        }
      }
      __syncthreads();
      float2* const t = in;                 // rotate: next input, its partner, the next target
      in = nx;
      nx = al;
      al = t;
    }
    float2* part = a.T + (size_t)(r.lo - a.s0) * plane;
#pragma unroll
    for (int u = 0; u < COL_ACC; ++u) {
      const int idx = threadIdx.x + u * COL_THREADS;
      if (idx < NC) {
        const int y = qdiv(idx, rC), c = idx - y * C;
        part[(size_t)y * W + col0 + c] = acc[u];
      }
    }
  } else {
    // COL_FIN, image blockIdx.y: acc = (partial sum in A_b unless the chunk
    // holds the image's first subband) + the groups' partials in group
    // order; on the image's last subband acc * 1/W is inverse column
    // transformed into A_b, else stored there as the new partial sum
    const RecRange r0 = rec_range(a, blockIdx.y, 0);
    float2* Ab = a.A + (size_t)r0.b * plane;
    for (int idx = threadIdx.x; idx < NC; idx += blockDim.x) {
      const int y = qdiv(idx, rC), c = idx - y * C;
      const size_t e = (size_t)y * W + col0 + c;
      float2 v = r0.first ? make_float2(0.f, 0.f) : Ab[e];
      for (int g = 0; g < a.groups; ++g) {
        const RecRange r = rec_range(a, blockIdx.y, g);
        if (r.lo < r.hi) {
          const float2 t = a.T[(size_t)(r.lo - a.s0) * plane + e];
          v.x += t.x;
          v.y += t.y;
        }
      }
      if (!r0.last) {
        Ab[e] = v;
      } else {
        if (a.invW) {
          const float w = __ldg(a.invW + e);
          v.x *= w;
          v.y *= w;
        }
        buf[c * a.pitch + y] = conj2(v);
      }
    }
    if (!r0.last) return;
    float2* res = line_dft(buf, alt, C, a.pitch, p);
    for (int idx = threadIdx.x; idx < NC; idx += blockDim.x) {
      const int y = qdiv(idx, rC), c = idx - y * C;
      Ab[(size_t)y * W + col0 + c] = conj2(res[c * a.pitch + y]);
    }
  }
}

// ------------------------------------------------------------ host side
using cd = std::complex<double>;
constexpr double PI = 3.14159265358979323846264338327950288;

// In-place radix-2 FFT in float64 (n a power of two), sign -1 forward.
void fft_pow2(std::vector<cd>& x, int sign) {
  const int n = (int)x.size();
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(x[i], x[j]);
  }
  for (int len = 2; len <= n; len <<= 1)
    for (int k = 0; k < len / 2; ++k) {
      const double a = sign * 2.0 * PI * k / len;
      const cd w(std::cos(a), std::sin(a));
      for (int s = 0; s < n; s += len) {
        const cd u = x[s + k], v = x[s + k + len / 2] * w;
        x[s + k] = u + v;
        x[s + k + len / 2] = u - v;
      }
    }
}

float2 to_f2(cd v) { return make_float2((float)v.real(), (float)v.imag()); }

// Stage radices of a length whose prime factors are all <= MAX_DIRECT_PRIME:
// the factor 2^t as radix-8 stages and one radix-4 or radix-2 stage for the
// rest, then the odd primes.
void radices_of(int n, LinePlan* p) {
  std::vector<int> r;
  int twos = 0;
  while (n % 2 == 0) { n /= 2; ++twos; }
  for (; twos >= 3; twos -= 3) r.push_back(8);
  if (twos) r.push_back(1 << twos);
  for (int f = 3; n > 1; f += 2)
    while (n % f == 0) { r.push_back(f); n /= f; }
  p->nst = (int)r.size();
  for (int s = 0; s < p->nst; ++s) p->radix[s] = r[s];
}

int largest_prime_factor(int n) {
  int big = 1;
  for (int f = 2; (long long)f * f <= n; ++f)
    while (n % f == 0) { big = f; n /= f; }
  return n > 1 ? std::max(big, n) : big;
}

// Launches k, first raising its dynamic shared-memory limit to what this
// launch asks for (the attribute is per function and device; a launch that
// needs no more than the default 48 KB leaves it alone).
template <typename Args>
cudaError_t launch(void (*k)(Args), dim3 grid, int threads, size_t smem, cudaStream_t st,
                   const Args& a) {
  if (grid.x == 0 || grid.y == 0) return cudaSuccess;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
  }
  k<<<grid, threads, smem, st>>>(a);
  return cudaGetLastError();
}

// CTAs of a row pass: (N + 1) / 2 row-pair lines per plane, C per CTA.
unsigned row_grid(int N, int nplanes, int C) {
  const long long lines = (long long)((N + 1) / 2) * nplanes;
  return (unsigned)((lines + C - 1) / C);
}

int row_lines(const LinePlan& pm) {
  return std::max(1, std::min(MAX_LINES, ROW_ELEMS / pm.P));
}

// Columns per CTA: at most COL_LINES_MAX (more CTAs per SM beat longer
// column runs), two line buffers within COL_SMEM_CAP (one CTA per line when
// a single column needs more), and C * N <= 16 * 256 so that the
// reconstruction's running sum fits its registers.
int col_lines(const LinePlan& pn, int W) {
  const size_t per = 2 * (size_t)(pn.P + 1) * sizeof(float2);
  int c = (int)std::min<size_t>(COL_LINES_MAX, std::max<size_t>(1, COL_SMEM_CAP / per));
  c = std::min(c, std::max(1, COL_ACC * COL_THREADS / pn.L));
  return std::min(c, W);
}

}  // namespace

LineTables make_line_tables(int L) {
  LineTables t;
  LinePlan& p = t.plan;
  p = LinePlan{};
  p.L = L;
  p.bluestein = largest_prime_factor(L) > MAX_DIRECT_PRIME;
  p.P = L;
  if (p.bluestein) {
    p.P = 1;
    while (p.P < 2 * L - 1) p.P <<= 1;
  }
  radices_of(p.P, &p);
  const int P = p.P;
  t.off_tw = 0;
  t.data.resize(P);
  for (int q = 0; q < P; ++q) {
    const double a = -2.0 * PI * q / P;
    t.data[q] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  if (p.bluestein) {
    std::vector<cd> c(L), h(P, cd(0.0, 0.0));
    for (int n = 0; n < L; ++n) {
      const long long q = ((long long)n * n) % (2LL * L);   // exp(-i pi n^2 / L), reduced
      const double a = -PI * (double)q / L;
      c[n] = cd(std::cos(a), std::sin(a));
    }
    for (int m = 0; m < L; ++m) {
      h[m] = std::conj(c[m]);
      if (m) h[P - m] = std::conj(c[m]);
    }
    fft_pow2(h, -1);
    t.off_chirp = t.data.size();
    for (int n = 0; n < L; ++n) t.data.push_back(to_f2(c[n]));
    t.off_kern = t.data.size();
    for (int k = 0; k < P; ++k) t.data.push_back(to_f2(h[k] / (double)P));
  }
  return t;
}

void place_line_tables(LineTables* t, const float2* dev) {
  t->plan.tw = dev + t->off_tw;
  t->plan.chirp = t->plan.bluestein ? dev + t->off_chirp : nullptr;
  t->plan.kern = t->plan.bluestein ? dev + t->off_kern : nullptr;
}

cudaError_t launch_rows_fwd(const LinePlan& pm, RowIn mode, const void* in, const uint8_t* mask,
                            const float* fest, const float* thresh, float2* out, int N,
                            int nplanes, cudaStream_t st) {
  RowArgs a{};
  a.pm = pm; a.in = in; a.mask = mask; a.fest = fest; a.thresh = thresh; a.z = out;
  a.N = N; a.nplanes = nplanes; a.C = row_lines(pm); a.pitch = pm.P + 1; a.mode = mode;
  const size_t smem = 2 * (size_t)a.C * a.pitch * sizeof(float2);
  return launch(k_rows<ROW_FWD>, dim3(row_grid(N, nplanes, a.C)), ROW_THREADS, smem, st, a);
}

cudaError_t launch_rows_inv(const LinePlan& pm, const float2* in, void* out, bool bf16,
                            float scale, int N, int nplanes, cudaStream_t st) {
  RowArgs a{};
  a.pm = pm; a.z = const_cast<float2*>(in); a.out = out; a.scale = scale;
  a.N = N; a.nplanes = nplanes; a.C = row_lines(pm); a.pitch = pm.P + 1; a.mode = bf16 ? 1 : 0;
  const size_t smem = 2 * (size_t)a.C * a.pitch * sizeof(float2);
  return launch(k_rows<ROW_INV>, dim3(row_grid(N, nplanes, a.C)), ROW_THREADS, smem, st, a);
}

cudaError_t launch_rows_shrink(const LinePlan& pm, float2* z, const float* thresh, float scale,
                               int N, int nplanes, cudaStream_t st) {
  RowArgs a{};
  a.pm = pm; a.z = z; a.thresh = thresh; a.scale = scale;
  a.N = N; a.nplanes = nplanes; a.C = row_lines(pm); a.pitch = pm.P + 1;
  const size_t smem = 2 * (size_t)a.C * a.pitch * sizeof(float2);
  return launch(k_rows<ROW_SHRINK>, dim3(row_grid(N, nplanes, a.C)), ROW_THREADS, smem, st, a);
}

cudaError_t launch_cols_fwd(const LinePlan& pn, float2* X, int W, int nplanes, cudaStream_t st) {
  ColArgs a{};
  a.pn = pn; a.A = X; a.W = W; a.C = col_lines(pn, W); a.pitch = pn.P + 1;
  const size_t smem = 2 * (size_t)a.C * a.pitch * sizeof(float2);
  return launch(k_cols<COL_FWD>, dim3((W + a.C - 1) / a.C, nplanes), COL_THREADS, smem, st, a);
}

cudaError_t launch_cols_dec(const LinePlan& pn, const float2* X, float2* T, const void* G,
                            bool cplx, const float* invW, int W, int K, int s0, int S,
                            cudaStream_t st) {
  ColArgs a{};
  a.pn = pn; a.X = X; a.T = T; a.G = G; a.cplx = cplx; a.invW = invW;
  a.W = W; a.K = K; a.s0 = s0; a.S = S; a.C = col_lines(pn, W); a.pitch = pn.P + 1;
  const size_t smem = 2 * (size_t)a.C * a.pitch * sizeof(float2);
  return launch(k_cols<COL_DEC>, dim3((W + a.C - 1) / a.C, S), COL_THREADS, smem, st, a);
}

cudaError_t launch_cols_rec(const LinePlan& pn, float2* T, float2* A, const void* G,
                            bool cplx, const float* invW, int W, int K, int s0, int S,
                            cudaStream_t st) {
  ColArgs a{};
  a.pn = pn; a.T = T; a.A = A; a.G = G; a.cplx = cplx; a.invW = invW;
  a.W = W; a.K = K; a.s0 = s0; a.S = S; a.C = col_lines(pn, W); a.pitch = pn.P + 1;
  const int nimg = S > 0 ? (s0 + S - 1) / K - s0 / K + 1 : 0;
  const size_t smem = 2 * (size_t)a.C * a.pitch * sizeof(float2);
  const size_t smem_rec = 3 * (size_t)a.C * a.pitch * sizeof(float2);   // + the prefetch buffer
  const unsigned cb = (unsigned)((W + a.C - 1) / a.C);
  // subband groups per image: about four waves of CTAs (smem-bound residency)
  // with at least ceil(K / 16) subbands a group, so that one image's K
  // transforms are spread over the GPU instead of running in one CTA
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long per_sm = std::max<long long>(1, (228 * 1024) / (long long)(smem_rec + 1024));
  const long long want = 4LL * std::max(sms, 1) * per_sm;
  const long long base = std::max<long long>(1, (long long)cb * nimg);
  a.groups = (int)std::max<long long>(1, std::min<long long>({(want + base - 1) / base, 16,
                                                              std::min(S, K)}));
  cudaError_t e = launch(k_cols<COL_REC>, dim3(cb, nimg, a.groups), COL_THREADS, smem_rec, st, a);
  if (e) return e;
  return launch(k_cols<COL_FIN>, dim3(cb, nimg), COL_THREADS, smem, st, a);
}

}  // namespace gen
}  // namespace shl
