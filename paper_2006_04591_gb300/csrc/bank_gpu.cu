// bank_gpu.cu - float64 construction of the digital shearlet system on the
// GPU (Sec. 2.1 and 3.4; the filter-construction step the paper times as
// its first experiment).  Same construction and readings as the host
// builder (bank_build.cpp):
//   unsheared psi_j(w1, w2) = P(a1 w1, a2 w2) g_{J-j}(w1) h_{J-j-1+l}(w2),
//   digital shear S^d_k along x1 in the (x2, w1) domain: each row x2 times
//       sum_{r < 2^l} h_l(w_r)^2 exp(+i w_r k x2), w_r = 2 pi (p1 + r M)/(M 2^l),
//   cone 2 = cone 1 on the transposed grid, low-pass h_J (x) h_J, spectra
//   made exactly even.
// Every column p1 of a cone-1 filter is independent (its shear acts along
// x1, i.e. per w1): one CTA builds one column -- the column spectrum, an
// inverse DFT along w2, the shear multiplier, a forward DFT -- in shared
// memory (radix-2, float64).  Later kernels make the spectra even, transpose
// cone 2, and derive the float32 tables the transform kernels read.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "internal.h"

namespace shl {
namespace {

struct LowPass {
  double b[5];
};

__device__ __forceinline__ double lp_H(const LowPass& F, double w) {
  double s = F.b[0];
#pragma unroll
  for (int m = 1; m < 5; ++m) s += F.b[m] * cos(m * w);
  return s;
}
__device__ __forceinline__ double lp_Hj(const LowPass& F, int j, double w) {
  double s = 1.0;
  for (int k = 0; k < j; ++k) s *= lp_H(F, ldexp(w, k));
  return s;
}
__device__ __forceinline__ double lp_Gj(const LowPass& F, int j, double w) {
  return lp_H(F, ldexp(w, j - 1) + M_PI) * lp_Hj(F, j - 1, w);
}
__device__ __forceinline__ double fan(double w1, double w2) {
  const double t = 0.5 * (cos(w2) - cos(w1));
  const double a = 0.5 * (1.0 + t);
  return a * a * (2.0 - t);
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-place radix-2 FFT of x[0..n) in shared memory, tw[k] = exp(-2 pi i k / n)
// for k < n / 2; sign -1 forward, +1 inverse (unnormalised).
__device__ void fft_smem(double2* x, int n, int logn, const double2* tw, int sign) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int j = (int)(__brev((unsigned)i) >> (32 - logn));
    if (i < j) {
      const double2 t = x[i];
      x[i] = x[j];
      x[j] = t;
    }
  }
  __syncthreads();
  for (int s = 1; s <= logn; ++s) {
    const int half = 1 << (s - 1);
    for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
      const int grp = b >> (s - 1), pos = b & (half - 1);
      const int i0 = grp * 2 * half + pos, i1 = i0 + half;
      double2 w = tw[pos << (logn - s)];
      if (sign > 0) w.y = -w.y;
      const double2 a = x[i0], c = zmul(x[i1], w);
      x[i0] = make_double2(a.x + c.x, a.y + c.y);
      x[i1] = make_double2(a.x - c.x, a.y - c.y);
    }
    __syncthreads();
  }
}

struct ColArgs {
  LowPass F;
  double* out;        // [Nr][Mc], real part of the sheared spectrum
  int j, J, l, k, Nr, Mc, logNr;
};

// One column p1 = blockIdx.x of a cone-1 filter on an Nr x Mc grid.
__global__ void __launch_bounds__(256) k_bank_col(ColArgs a) {
  extern __shared__ double2 sm[];
  double2* col = sm;                  // [Nr]
  double2* tw = sm + a.Nr;            // [Nr / 2]
  double* h2 = reinterpret_cast<double*>(tw + a.Nr / 2);   // [2^l]
  const int p1 = blockIdx.x, tid = threadIdx.x;
  const double a1 = ldexp(1.0, a.J - a.j - 1), a2 = a1 * ldexp(1.0, a.l);
  const double w1 = 2.0 * M_PI * p1 / a.Mc;
  const int U = 1 << a.l;
  for (int q = tid; q < a.Nr / 2; q += blockDim.x) {
    double s, c;
    sincospi(-2.0 * q / a.Nr, &s, &c);
    tw[q] = make_double2(c, s);
  }
  for (int r = tid; r < U; r += blockDim.x) {
    const double w = 2.0 * M_PI * (p1 + (double)r * a.Mc) / ((double)a.Mc * U);
    const double h = lp_Hj(a.F, a.l, w);
    h2[r] = h * h;
  }
  const double gx = lp_Gj(a.F, a.J - a.j, w1);
  for (int p2 = tid; p2 < a.Nr; p2 += blockDim.x) {
    const double w2 = 2.0 * M_PI * p2 / a.Nr;
    col[p2] = make_double2(fan(a1 * w1, a2 * w2) * gx * lp_Hj(a.F, a.J - a.j - 1 + a.l, w2), 0.0);
  }
  __syncthreads();
  fft_smem(col, a.Nr, a.logNr, tw, +1);              // -> x2 rows of column w1
  for (int x2 = tid; x2 < a.Nr; x2 += blockDim.x) {
    const int c2 = x2 < a.Nr / 2 ? x2 : x2 - a.Nr;
    double2 t = make_double2(0.0, 0.0);
    for (int r = 0; r < U; ++r) {
      const double w = 2.0 * M_PI * (p1 + (double)r * a.Mc) / ((double)a.Mc * U);
      double s, c;
      sincos(w * a.k * c2, &s, &c);
      t.x += h2[r] * c;
      t.y += h2[r] * s;
    }
    const double2 v = col[x2];
    const double inv = 1.0 / a.Nr;
    col[x2] = zmul(make_double2(v.x * inv, v.y * inv), t);
  }
  __syncthreads();
  fft_smem(col, a.Nr, a.logNr, tw, -1);
  for (int p2 = tid; p2 < a.Nr; p2 += blockDim.x) a.out[(size_t)p2 * a.Mc + p1] = col[p2].x;
}

// dst[y][x] (N x M) = even part of src: cone 1 src is [N][M]; cone 2 src is
// the transposed-grid filter [M][N], dst[y][x] = src[x][y].
__global__ void k_bank_even(const double* __restrict__ src, double* __restrict__ dst, int N, int M,
                            int transposed) {
  const size_t n = (size_t)N * M;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int y = (int)(e / M), x = (int)(e % M);
    const int yq = (N - y) % N, xq = (M - x) % M;
    const double a = transposed ? src[(size_t)x * N + y] : src[(size_t)y * M + x];
    const double b = transposed ? src[(size_t)xq * N + yq] : src[(size_t)yq * M + xq];
    dst[e] = 0.5 * (a + b);
  }
}

__global__ void k_bank_lowpass(LowPass F, double* __restrict__ dst, int J, int N, int M) {
  const size_t n = (size_t)N * M;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int y = (int)(e / M), x = (int)(e % M);
    dst[e] = lp_Hj(F, J, 2.0 * M_PI * x / M) * lp_Hj(F, J, 2.0 * M_PI * y / N);
  }
}

// W = sum_i G_i^2 (float64, filters summed in order), its float32 inverse on
// the transposed half spectrum, and a count of points with W <= 0.
__global__ void k_bank_dual(const double* __restrict__ S, int K, int N, int M,
                            double* __restrict__ W, float* __restrict__ invW,
                            unsigned* __restrict__ bad) {
  const int Mh = M / 2 + 1;
  const size_t n = (size_t)N * M;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    double w = 0.0;
    for (int i = 0; i < K; ++i) {
      const double g = S[(size_t)i * n + e];
      w += g * g;
    }
    W[e] = w;
    if (!(w > 0.0)) atomicAdd(bad, 1u);
    const int y = (int)(e / M), x = (int)(e % M);
    if (x < Mh) invW[(size_t)x * N + y] = (float)(1.0 / w);
  }
}

// G[i][kx][ky] = float(S[i][ky][kx]) for kx <= M/2.
__global__ void k_bank_pack(const double* __restrict__ S, float* __restrict__ G, int K, int N, int M) {
  const int Mh = M / 2 + 1;
  const size_t per = (size_t)Mh * N, n = (size_t)K * per;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / per);
    const size_t r = e - (size_t)i * per;
    const int kx = (int)(r / N), ky = (int)(r % N);
    G[e] = (float)S[((size_t)i * N + ky) * M + kx];
  }
}

// RMS_i = sqrt(sum G_i^2 / (N M)): one CTA per filter, fixed thread mapping
// and tree order.
__global__ void __launch_bounds__(256) k_bank_rms(const double* __restrict__ S, int N, int M,
                                                  double* __restrict__ rms) {
  const size_t n = (size_t)N * M;
  const double* g = S + (size_t)blockIdx.x * n;
  double s = 0.0;
  for (size_t e = threadIdx.x; e < n; e += blockDim.x) s += g[e] * g[e];
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) rms[blockIdx.x] = sqrt(red[0] / (double)n);
}

int log2i(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

}  // namespace

cudaError_t build_bank_device(int rows, int cols, int n_scales, const int* shear_levels, int full,
                              const std::vector<BankItem>& items, double* d_spectra,
                              double* d_tmp, double* d_w, double* d_rms, float* d_G,
                              float* d_invW, unsigned* d_bad, cudaStream_t st) {
  (void)shear_levels;
  (void)full;
  LowPass F;
  maxflat_coeffs(F.b);
  const int N = rows, M = cols, J = n_scales, K = (int)items.size();
  const size_t plane = (size_t)N * M;
  const int eg = 1024;   // grid of the elementwise kernels
  cudaError_t e;
  for (int i = 0; i < K; ++i) {
    const BankItem& it = items[i];
    double* dst = d_spectra + (size_t)i * plane;
    if (it.cone == 0) {
      k_bank_lowpass<<<eg, 256, 0, st>>>(F, dst, J, N, M);
    } else {
      const bool t = it.cone == 2;
      ColArgs a;
      a.F = F;
      a.out = d_tmp;
      a.j = it.scale - 1;
      a.J = J;
      a.l = it.l;
      a.k = it.k;
      a.Nr = t ? M : N;
      a.Mc = t ? N : M;
      a.logNr = log2i(a.Nr);
      const size_t sm = sizeof(double2) * ((size_t)a.Nr + a.Nr / 2) + sizeof(double) * (1u << it.l);
      if (sm > 48 * 1024 &&
          (e = cudaFuncSetAttribute(k_bank_col, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
        return e;
      k_bank_col<<<a.Mc, 256, sm, st>>>(a);
      k_bank_even<<<eg, 256, 0, st>>>(d_tmp, dst, N, M, t ? 1 : 0);
    }
    if ((e = cudaGetLastError())) return e;
  }
  if ((e = cudaMemsetAsync(d_bad, 0, sizeof(unsigned), st))) return e;
  k_bank_dual<<<eg, 256, 0, st>>>(d_spectra, K, N, M, d_w, d_invW, d_bad);
  k_bank_pack<<<eg, 256, 0, st>>>(d_spectra, d_G, K, N, M);
  k_bank_rms<<<K, 256, 0, st>>>(d_spectra, N, M, d_rms);
  return cudaGetLastError();
}

}  // namespace shl
