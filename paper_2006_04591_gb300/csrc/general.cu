// general.cu - transform kernels for any image size and for complex
// Hermitian filter spectra: the decomposition, reconstruction and adjoint of
// Sec. 3.4 on full complex planes [N][M] in natural DFT order.
//
//   k_rows<ROW_FWD>     real rows (threshold-on-read or masked input) ->
//                       forward row DFT -> complex planes.
//   k_rows<ROW_INV>     complex rows -> inverse row DFT -> real part * scale
//                       -> float32 / bfloat16.
//   k_rows<ROW_SHRINK>  in place: inverse row DFT -> real part * scale ->
//                       hard threshold -> forward row DFT (denoise / IHT).
//   k_cols<COL_FWD>     in-place forward column DFT (image spectra).
//   k_cols<COL_DEC>     G_i * X_b [* 1/W] formed in the load, inverse column
//                       DFT, stored to the staging planes.
//   k_cols<COL_REC>     per image: forward column DFT of each staged subband,
//                       conj(G_i) multiply, fixed-order sum in shared memory;
//                       then 1/W and the inverse column DFT.
//
// Each CTA owns C whole lines of one pass in shared memory (line pitch P + 1
// float2, so that the C-column tiles of the column passes hit distinct
// banks).  A column CTA reads and writes its C adjacent columns as C * 8-byte
// runs of each row (128 B at C = 16).
//
// Line DFT.  Length P = r_1 r_2 ... r_s (all factors <= 61): Stockham's
// autosort FFT, one output element per thread and stage:
//   out[g Ns R + q Ns + k] = sum_{m<R} in[g Ns + k + m P/R] w^(m (k + q Ns) P/(Ns R)),
// w = exp(-2 pi i / P), R the stage radix, Ns the product of the earlier
// radices, 0 <= k < Ns, 0 <= q < R.  A length with a larger prime factor
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
constexpr int COL_THREADS = 512;
constexpr int MAX_LINES = 16;          // lines per CTA
constexpr int ROW_ELEMS = 4096;        // target C * P of a row CTA (64 KB of lines)
constexpr size_t COL_SMEM_CAP = 200 * 1024;

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

// Forward FFT of length p.P on C lines at src[l * pitch + e], ping-ponging
// with dst; returns the buffer that holds the result.  Every stage ends with
// a barrier; the caller has synchronised after writing src.
__device__ float2* stockham(float2* src, float2* dst, int C, int pitch, const LinePlan& p) {
  const int P = p.P;
  const float rP = __frcp_rn((float)P);
  int Ns = 1;
  for (int st = 0; st < p.nst; ++st) {
    const int R = p.radix[st];
    const int stride = P / R, span = Ns * R, tstep = P / span;
    const float rNs = __frcp_rn((float)Ns), rR = __frcp_rn((float)R);
    for (int idx = threadIdx.x; idx < C * P; idx += blockDim.x) {
      const int l = qdiv(idx, rP), o = idx - l * P;
      const int qg = qdiv(o, rNs), k = o - qg * Ns;
      const int g = qdiv(qg, rR), q = qg - g * R;
      const float2* s = src + l * pitch + g * Ns + k;
      const int base = (k + q * Ns) * tstep;     // < P
      float2 acc = s[0];
      int ex = 0;
      for (int m = 1; m < R; ++m) {
        ex += base;
        if (ex >= P) ex -= P;
        const float2 w = __ldg(p.tw + ex), v = s[m * stride];
        acc.x = fmaf(v.x, w.x, fmaf(-v.y, w.y, acc.x));
        acc.y = fmaf(v.x, w.y, fmaf(v.y, w.x, acc.y));
      }
      dst[l * pitch + o] = acc;
    }
    __syncthreads();
    float2* t = src;
    src = dst;
    dst = t;
    Ns = span;
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
  float2* z;                 // complex planes: ROW_FWD out, ROW_INV in, ROW_SHRINK in/out
  void* out;                 // ROW_INV: float32 / bfloat16 [nplanes][N][M]
  float scale;               // ROW_INV, ROW_SHRINK: 1/(N M)
  int N, nplanes, C, pitch;
  int mode;                  // ROW_FWD: RowIn; ROW_INV: 1 = bfloat16 out
};

template <int KIND>
__global__ void __launch_bounds__(ROW_THREADS) k_rows(const RowArgs a) {
  extern __shared__ float2 sm[];
  __shared__ float s_tau[MAX_LINES];
  const LinePlan& p = a.pm;
  const int M = p.L;
  const int rows = a.N * a.nplanes;
  const int r0 = blockIdx.x * a.C;
  const int C = min(a.C, rows - r0);
  float2* buf = sm;
  float2* alt = sm + (size_t)a.C * a.pitch;
  if (threadIdx.x < C)
    s_tau[threadIdx.x] = a.thresh ? __ldg(a.thresh + (r0 + (int)threadIdx.x) / a.N) : 0.f;
  __syncthreads();
  const float rM = __frcp_rn((float)M);
  for (int idx = threadIdx.x; idx < C * M; idx += blockDim.x) {
    const int l = qdiv(idx, rM), e = idx - l * M;
    const size_t g = (size_t)(r0 + l) * M + e;
    float2 v;
    if constexpr (KIND == ROW_FWD) {
      float x;
      if (a.mode == RIN_BF16)
        x = __bfloat162float(static_cast<const __nv_bfloat16*>(a.in)[g]);
      else if (a.mode == RIN_MASKED)
        x = a.mask[g] ? static_cast<const float*>(a.in)[g] : a.fest[g];
      else
        x = static_cast<const float*>(a.in)[g];
      if (a.thresh && fabsf(x) < s_tau[l]) x = 0.f;   // ties kept
      v = make_float2(x, 0.f);
    } else {
      v = conj2(a.z[g]);                              // inverse DFT by conjugation
    }
    buf[l * a.pitch + e] = v;
  }
  float2* res = line_dft(buf, alt, C, a.pitch, p);
  if constexpr (KIND == ROW_SHRINK) {
    float2* other = res == buf ? alt : buf;
    for (int idx = threadIdx.x; idx < C * M; idx += blockDim.x) {
      const int l = qdiv(idx, rM), e = idx - l * M;
      float c = res[l * a.pitch + e].x * a.scale;     // Re IDFT = Re conj(DFT(conj z))
      if (fabsf(c) < s_tau[l]) c = 0.f;
      other[l * a.pitch + e] = make_float2(c, 0.f);
    }
    res = line_dft(other, res, C, a.pitch, p);
  }
  for (int idx = threadIdx.x; idx < C * M; idx += blockDim.x) {
    const int l = qdiv(idx, rM), e = idx - l * M;
    const size_t g = (size_t)(r0 + l) * M + e;
    const float2 v = res[l * a.pitch + e];
    if constexpr (KIND == ROW_INV) {
      const float x = v.x * a.scale;
      if (a.mode) static_cast<__nv_bfloat16*>(a.out)[g] = __float2bfloat16_rn(x);
      else static_cast<float*>(a.out)[g] = x;
    } else {
      a.z[g] = v;
    }
  }
}

// --------------------------------------------------------------- columns
enum ColKind : int { COL_FWD = 0, COL_DEC = 1, COL_REC = 2 };

struct ColArgs {
  LinePlan pn;               // columns: length N
  const float2* X;           // COL_DEC: image spectra [B][N][M]
  float2* T;                 // COL_DEC out / COL_REC in: staging [S][N][M]
  float2* A;                 // COL_FWD planes (in place) / COL_REC accumulators [B][N][M]
  const void* G;             // float [K][N][M] or float2 [K][N][M]
  const float* invW;         // [N][M] or null
  int M, K, s0, S, C, pitch, cplx;
};

__device__ __forceinline__ float2 filter_at(const ColArgs& a, int i, size_t e, size_t plane) {
  if (a.cplx) return __ldg(static_cast<const float2*>(a.G) + (size_t)i * plane + e);
  return make_float2(__ldg(static_cast<const float*>(a.G) + (size_t)i * plane + e), 0.f);
}

template <int KIND>
__global__ void __launch_bounds__(COL_THREADS) k_cols(const ColArgs a) {
  extern __shared__ float2 sm[];
  const LinePlan& p = a.pn;
  const int N = p.L, M = a.M;
  const size_t plane = (size_t)N * M;
  const int col0 = blockIdx.x * a.C;
  const int C = min(a.C, M - col0);
  float2* buf = sm;
  float2* alt = sm + (size_t)a.C * a.pitch;
  const float rC = __frcp_rn((float)C);
  // Thread idx owns tile element (y, c) = (idx / C, idx % C) in every loop
  // below, at global offset y * M + col0 + c of a plane.
  if constexpr (KIND == COL_FWD) {
    float2* pl = a.A + (size_t)blockIdx.y * plane;
    for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
      const int y = qdiv(idx, rC), c = idx - y * C;
      buf[c * a.pitch + y] = pl[(size_t)y * M + col0 + c];
    }
    float2* res = line_dft(buf, alt, C, a.pitch, p);
    for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
      const int y = qdiv(idx, rC), c = idx - y * C;
      pl[(size_t)y * M + col0 + c] = res[c * a.pitch + y];
    }
  } else if constexpr (KIND == COL_DEC) {
    const int s = a.s0 + blockIdx.y, b = s / a.K, i = s - b * a.K;
    const float2* Xb = a.X + (size_t)b * plane;
    for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
      const int y = qdiv(idx, rC), c = idx - y * C;
      const size_t e = (size_t)y * M + col0 + c;
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
    for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
      const int y = qdiv(idx, rC), c = idx - y * C;
      Ts[(size_t)y * M + col0 + c] = conj2(res[c * a.pitch + y]);
    }
  } else {
    float2* acc = sm + 2 * (size_t)a.C * a.pitch;
    const int b = a.s0 / a.K + blockIdx.y;
    const int sa = max(a.s0, b * a.K), sb = min(a.s0 + a.S, (b + 1) * a.K);
    const bool first = sa == b * a.K, last = sb == (b + 1) * a.K;
    float2* Ab = a.A + (size_t)b * plane;
    for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
      const int y = qdiv(idx, rC), c = idx - y * C;
      acc[c * a.pitch + y] = first ? make_float2(0.f, 0.f) : Ab[(size_t)y * M + col0 + c];
    }
    for (int s = sa; s < sb; ++s) {
      const int i = s - b * a.K;
      const float2* Ts = a.T + (size_t)(s - a.s0) * plane;
      for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
        const int y = qdiv(idx, rC), c = idx - y * C;
        buf[c * a.pitch + y] = Ts[(size_t)y * M + col0 + c];
      }
      float2* res = line_dft(buf, alt, C, a.pitch, p);
      for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
        const int y = qdiv(idx, rC), c = idx - y * C;
        const float2 t = cmulc(filter_at(a, i, (size_t)y * M + col0 + c, plane),
                               res[c * a.pitch + y]);
        float2& u = acc[c * a.pitch + y];
        u.x += t.x;
        u.y += t.y;
      }
      __syncthreads();
    }
    if (!last) {
      for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
        const int y = qdiv(idx, rC), c = idx - y * C;
        Ab[(size_t)y * M + col0 + c] = acc[c * a.pitch + y];
      }
      return;
    }
    for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
      const int y = qdiv(idx, rC), c = idx - y * C;
      float2 v = acc[c * a.pitch + y];
      if (a.invW) {
        const float w = __ldg(a.invW + (size_t)y * M + col0 + c);
        v.x *= w;
        v.y *= w;
      }
      buf[c * a.pitch + y] = conj2(v);
    }
    float2* res = line_dft(buf, alt, C, a.pitch, p);
    for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
      const int y = qdiv(idx, rC), c = idx - y * C;
      Ab[(size_t)y * M + col0 + c] = conj2(res[c * a.pitch + y]);
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
// pairs of 2 merged into radix 4, then the odd primes.
void radices_of(int n, LinePlan* p) {
  std::vector<int> r;
  int twos = 0;
  while (n % 2 == 0) { n /= 2; ++twos; }
  for (; twos >= 2; twos -= 2) r.push_back(4);
  if (twos) r.push_back(2);
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

int row_lines(const LinePlan& pm) {
  return std::max(1, std::min(MAX_LINES, ROW_ELEMS / pm.P));
}

int col_lines(const LinePlan& pn, int M, int buffers) {
  const size_t per = (size_t)buffers * (pn.P + 1) * sizeof(float2);
  const int c = (int)std::min<size_t>(MAX_LINES, std::max<size_t>(1, COL_SMEM_CAP / per));
  return std::min(c, M);
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
  const int rows = N * nplanes;
  const size_t smem = 2 * (size_t)a.C * a.pitch * sizeof(float2);
  return launch(k_rows<ROW_FWD>, dim3((rows + a.C - 1) / a.C), ROW_THREADS, smem, st, a);
}

cudaError_t launch_rows_inv(const LinePlan& pm, const float2* in, void* out, bool bf16,
                            float scale, int N, int nplanes, cudaStream_t st) {
  RowArgs a{};
  a.pm = pm; a.z = const_cast<float2*>(in); a.out = out; a.scale = scale;
  a.N = N; a.nplanes = nplanes; a.C = row_lines(pm); a.pitch = pm.P + 1; a.mode = bf16 ? 1 : 0;
  const int rows = N * nplanes;
  const size_t smem = 2 * (size_t)a.C * a.pitch * sizeof(float2);
  return launch(k_rows<ROW_INV>, dim3((rows + a.C - 1) / a.C), ROW_THREADS, smem, st, a);
}

cudaError_t launch_rows_shrink(const LinePlan& pm, float2* z, const float* thresh, float scale,
                               int N, int nplanes, cudaStream_t st) {
  RowArgs a{};
  a.pm = pm; a.z = z; a.thresh = thresh; a.scale = scale;
  a.N = N; a.nplanes = nplanes; a.C = row_lines(pm); a.pitch = pm.P + 1;
  const int rows = N * nplanes;
  const size_t smem = 2 * (size_t)a.C * a.pitch * sizeof(float2);
  return launch(k_rows<ROW_SHRINK>, dim3((rows + a.C - 1) / a.C), ROW_THREADS, smem, st, a);
}

cudaError_t launch_cols_fwd(const LinePlan& pn, float2* X, int M, int nplanes, cudaStream_t st) {
  ColArgs a{};
  a.pn = pn; a.A = X; a.M = M; a.C = col_lines(pn, M, 2); a.pitch = pn.P + 1;
  const size_t smem = 2 * (size_t)a.C * a.pitch * sizeof(float2);
  return launch(k_cols<COL_FWD>, dim3((M + a.C - 1) / a.C, nplanes), COL_THREADS, smem, st, a);
}

cudaError_t launch_cols_dec(const LinePlan& pn, const float2* X, float2* T, const void* G,
                            bool cplx, const float* invW, int M, int K, int s0, int S,
                            cudaStream_t st) {
  ColArgs a{};
  a.pn = pn; a.X = X; a.T = T; a.G = G; a.cplx = cplx; a.invW = invW;
  a.M = M; a.K = K; a.s0 = s0; a.S = S; a.C = col_lines(pn, M, 2); a.pitch = pn.P + 1;
  const size_t smem = 2 * (size_t)a.C * a.pitch * sizeof(float2);
  return launch(k_cols<COL_DEC>, dim3((M + a.C - 1) / a.C, S), COL_THREADS, smem, st, a);
}

cudaError_t launch_cols_rec(const LinePlan& pn, const float2* T, float2* A, const void* G,
                            bool cplx, const float* invW, int M, int K, int s0, int S,
                            cudaStream_t st) {
  ColArgs a{};
  a.pn = pn; a.T = const_cast<float2*>(T); a.A = A; a.G = G; a.cplx = cplx; a.invW = invW;
  a.M = M; a.K = K; a.s0 = s0; a.S = S; a.C = col_lines(pn, M, 3); a.pitch = pn.P + 1;
  const int nimg = S > 0 ? (s0 + S - 1) / K - s0 / K + 1 : 0;
  const size_t smem = 3 * (size_t)a.C * a.pitch * sizeof(float2);
  return launch(k_cols<COL_REC>, dim3((M + a.C - 1) / a.C, nimg), COL_THREADS, smem, st, a);
}

}  // namespace gen
}  // namespace shl
