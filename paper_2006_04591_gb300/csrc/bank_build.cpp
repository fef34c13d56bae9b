// bank_build.cpp - float64 host construction of the digital shearlet system
// (Sec. 2.1 and 3.4 of the paper; ``getshearletsystem2D``).
//
// Construction (readings where the paper is silent or garbled are marked):
//   h   9-tap symmetric low-pass, H(w) = b0 + sum_{m=1..4} b_m cos(m w),
//       maximally flat at DC (H(0)=1, H''(0)=H''''(0)=0), H(pi)=0 and
//       |H(pi/2)| = 1/sqrt(2): the paper's order-8 "maxflat" design with its
//       3 dB point at half Nyquist, solved here as a 5x5 linear system.
//   g   mirror high-pass g(n) = (-1)^n h(n), G(w) = H(w + pi).
//   h_j(w) = prod_{k<j} H(2^k w);  g_j(w) = G(2^{j-1} w) h_{j-1}(w)  (Sec. 2.1).
//   P   fan filter: maximally flat half-band polynomial
//       Hmf(t) = ((1+t)/2)^2 (2-t) under the McClellan substitution
//       t = (cos w2 - cos w1)/2 (diamond modulated by (-1)^{n1}).
//   scale j (0 = coarsest) of J, shear level l = l_j (default ceil((j+1)/2)):
//       unsheared psi_j = P(a1 w1, a2 w2) g_{J-j}(w1) h_{J-j-1+l}(w2),
//       a1 = 2^{J-j-1}, a2 = a1 2^l  (reading of p_j * W_j, Eq. 2.6).
//   digital shear S^d_k (Eqs. 2.4-2.5) along x1 on the circular grid: each
//       row x2 of the x2-space / w1-frequency array is multiplied by
//       sum_{r<2^l} h_l(w_r)^2 exp(+i w_r k x2), w_r = 2 pi (p1 + r M)/(M 2^l),
//       which is upsample-by-2^l, convolve 2^l h_l, shift k x2, convolve h_l,
//       downsample, written in the frequency domain.
//   cone 2 = cone 1 built on the transposed grid, transposed back; low-pass
//       h_J (x) h_J.  Every spectrum is made exactly real and even.
//   order: low-pass; per scale cone 1 (k = -2^l..2^l), cone 2
//       (k = -(2^l-1)..2^l-1, or +-2^l when full).
#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace shl {
namespace {

using cd = std::complex<double>;
constexpr double PI = 3.14159265358979323846264338327950288;

// ---------------------------------------------------------------- filters
struct Filters {
  double b[5];

  Filters() {
    // rows: H(0)=1, sum m^2 b_m = 0, sum m^4 b_m = 0, H(pi)=0, H(pi/2)=1/sqrt2
    double A[5][6];
    for (int m = 0; m < 5; ++m) {
      A[0][m] = 1.0;
      A[1][m] = double(m * m);
      A[2][m] = double(m * m * m * m);
      A[3][m] = (m % 2) ? -1.0 : 1.0;
      A[4][m] = (m % 4 == 0) ? 1.0 : (m % 4 == 2) ? -1.0 : 0.0;
    }
    A[0][5] = 1.0; A[1][5] = 0.0; A[2][5] = 0.0; A[3][5] = 0.0;
    A[4][5] = 1.0 / std::sqrt(2.0);
    for (int c = 0; c < 5; ++c) {              // Gaussian elimination, pivoting
      int p = c;
      for (int r = c + 1; r < 5; ++r)
        if (std::fabs(A[r][c]) > std::fabs(A[p][c])) p = r;
      for (int k = 0; k < 6; ++k) std::swap(A[c][k], A[p][k]);
      for (int r = 0; r < 5; ++r) {
        if (r == c) continue;
        const double f = A[r][c] / A[c][c];
        for (int k = c; k < 6; ++k) A[r][k] -= f * A[c][k];
      }
    }
    for (int m = 0; m < 5; ++m) b[m] = A[m][5] / A[m][m];
  }
  double H(double w) const {
    double s = b[0];
    for (int m = 1; m < 5; ++m) s += b[m] * std::cos(m * w);
    return s;
  }
  double Gh(double w) const { return H(w + PI); }
  double Hj(int j, double w) const {
    double s = 1.0;
    for (int k = 0; k < j; ++k) s *= H(std::ldexp(w, k));
    return s;
  }
  double Gj(int j, double w) const { return Gh(std::ldexp(w, j - 1)) * Hj(j - 1, w); }
  static double fan(double w1, double w2) {
    const double t = 0.5 * (std::cos(w2) - std::cos(w1));
    const double a = 0.5 * (1.0 + t);
    return a * a * (2.0 - t);
  }
};

// In-place iterative radix-2 FFT of length n (power of two), sign -1 forward.
void fft_pow2(cd* x, int n, int sign) {
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(x[i], x[j]);
  }
  for (int len = 2; len <= n; len <<= 1) {
    const double ang = sign * 2.0 * PI / len;
    for (int k = 0; k < len / 2; ++k) {
      const cd w(std::cos(ang * k), std::sin(ang * k));
      for (int s = 0; s < n; s += len) {
        const cd a = x[s + k], bb = x[s + k + len / 2] * w;
        x[s + k] = a + bb;
        x[s + k + len / 2] = a - bb;
      }
    }
  }
}

// Unnormalised DFT of any length n, in place (sign -1 forward).  Powers of
// two go straight to fft_pow2; other lengths use Bluestein's identity
// n k = (n^2 + k^2 - (k - n)^2) / 2, a circular convolution of length
// m = the power of two >= 2n - 1 with the chirp exp(sign i pi t^2 / n).
void fft1d(cd* x, int n, int sign) {
  if ((n & (n - 1)) == 0) { fft_pow2(x, n, sign); return; }
  int m = 1;
  while (m < 2 * n - 1) m <<= 1;
  std::vector<cd> c(n), a(m, cd(0.0, 0.0)), h(m, cd(0.0, 0.0));
  for (int t = 0; t < n; ++t) {
    const long long q = ((long long)t * t) % (2LL * n);
    const double ang = sign * PI * (double)q / n;
    c[t] = cd(std::cos(ang), std::sin(ang));
  }
  for (int t = 0; t < n; ++t) a[t] = x[t] * c[t];
  for (int t = 0; t < n; ++t) {
    h[t] = std::conj(c[t]);
    if (t) h[m - t] = std::conj(c[t]);
  }
  fft_pow2(a.data(), m, -1);
  fft_pow2(h.data(), m, -1);
  for (int t = 0; t < m; ++t) a[t] *= h[t];
  fft_pow2(a.data(), m, +1);
  for (int t = 0; t < n; ++t) x[t] = c[t] * a[t] / (double)m;
}

// One cone-1 filter on an Nr x Mc grid (rows = x2/w2, cols = x1/w1).
std::vector<double> cone1(const Filters& F, int j, int J, int l, int k, int Nr, int Mc) {
  const double a1 = std::ldexp(1.0, J - j - 1), a2 = a1 * std::ldexp(1.0, l);
  std::vector<cd> col(Nr);
  std::vector<cd> mixed((size_t)Nr * Mc);
  // unsheared spectrum, then inverse DFT along w2 (columns) -> x2 rows
  for (int p1 = 0; p1 < Mc; ++p1) {
    const double w1 = 2.0 * PI * p1 / Mc;
    const double gx = F.Gj(J - j, w1);
    for (int p2 = 0; p2 < Nr; ++p2) {
      const double w2 = 2.0 * PI * p2 / Nr;
      col[p2] = cd(Filters::fan(a1 * w1, a2 * w2) * gx * F.Hj(J - j - 1 + l, w2), 0.0);
    }
    fft1d(col.data(), Nr, +1);
    for (int x2 = 0; x2 < Nr; ++x2) mixed[(size_t)x2 * Mc + p1] = col[x2] / double(Nr);
  }
  // digital shear in the (x2, w1) domain
  const int U = 1 << l;
  std::vector<double> h2((size_t)U * Mc);
  for (int r = 0; r < U; ++r)
    for (int p1 = 0; p1 < Mc; ++p1) {
      const double w = 2.0 * PI * (p1 + (double)r * Mc) / ((double)Mc * U);
      const double h = F.Hj(l, w);
      h2[(size_t)r * Mc + p1] = h * h;
    }
  for (int x2 = 0; x2 < Nr; ++x2) {
    const int c2 = x2 < Nr / 2 ? x2 : x2 - Nr;
    for (int p1 = 0; p1 < Mc; ++p1) {
      cd t(0.0, 0.0);
      for (int r = 0; r < U; ++r) {
        const double w = 2.0 * PI * (p1 + (double)r * Mc) / ((double)Mc * U);
        const double ph = w * k * c2;
        t += h2[(size_t)r * Mc + p1] * cd(std::cos(ph), std::sin(ph));
      }
      mixed[(size_t)x2 * Mc + p1] *= t;
    }
  }
  // forward DFT along x2, keep the real part, make exactly even
  std::vector<double> out((size_t)Nr * Mc);
  for (int p1 = 0; p1 < Mc; ++p1) {
    for (int x2 = 0; x2 < Nr; ++x2) col[x2] = mixed[(size_t)x2 * Mc + p1];
    fft1d(col.data(), Nr, -1);
    for (int p2 = 0; p2 < Nr; ++p2) out[(size_t)p2 * Mc + p1] = col[p2].real();
  }
  std::vector<double> ev((size_t)Nr * Mc);
  for (int p2 = 0; p2 < Nr; ++p2)
    for (int p1 = 0; p1 < Mc; ++p1) {
      const int q2 = (Nr - p2) % Nr, q1 = (Mc - p1) % Mc;
      ev[(size_t)p2 * Mc + p1] = 0.5 * (out[(size_t)p2 * Mc + p1] + out[(size_t)q2 * Mc + q1]);
    }
  return ev;
}

}  // namespace

void maxflat_coeffs(double b[5]) {
  const Filters F;
  for (int m = 0; m < 5; ++m) b[m] = F.b[m];
}

const char* bank_items(int n_scales, const int* shear_levels, int full,
                       std::vector<BankItem>* items) {
  static thread_local std::string err;
  if (n_scales < 1 || n_scales > 8) return (err = "n_scales must be in [1, 8]").c_str();
  items->clear();
  items->push_back({0, 0, 0, 0});
  for (int j = 0; j < n_scales; ++j) {
    const int l = shear_levels ? shear_levels[j] : (j + 2) / 2;   // ceil((j+1)/2)
    if (l < 0 || l > 4) return (err = "shear levels must be in [0, 4]").c_str();
    const int kmax1 = 1 << l, kmax2 = full ? (1 << l) : (1 << l) - 1;
    for (int k = -kmax1; k <= kmax1; ++k) items->push_back({1, j + 1, k, l});
    for (int k = -kmax2; k <= kmax2; ++k) items->push_back({2, j + 1, k, l});
  }
  return "";
}

const char* build_shearlet_bank(int rows, int cols, int n_scales, const int* shear_levels,
                                int full, HostBank* out) {
  std::vector<BankItem> items;
  const char* e = bank_items(n_scales, shear_levels, full, &items);
  if (*e) return e;
  const int J = n_scales, N = rows, M = cols;
  const int K = (int)items.size();
  Filters F;
  out->rows = N; out->cols = M; out->K = K;
  out->spectra.assign((size_t)K * N * M, 0.0);
  out->idx.assign((size_t)K * 3, 0);
  for (int i = 0; i < K; ++i) {
    out->idx[3 * i] = items[i].cone;
    out->idx[3 * i + 1] = items[i].scale;
    out->idx[3 * i + 2] = items[i].k;
  }
  auto work = [&](int i) {
    double* dst = out->spectra.data() + (size_t)i * N * M;
    const BankItem& it = items[i];
    if (it.cone == 0) {
      for (int p2 = 0; p2 < N; ++p2)
        for (int p1 = 0; p1 < M; ++p1)
          dst[(size_t)p2 * M + p1] = F.Hj(J, 2.0 * PI * p1 / M) * F.Hj(J, 2.0 * PI * p2 / N);
    } else if (it.cone == 1) {
      std::vector<double> g = cone1(F, it.scale - 1, J, it.l, it.k, N, M);
      std::memcpy(dst, g.data(), g.size() * sizeof(double));
    } else {
      std::vector<double> g = cone1(F, it.scale - 1, J, it.l, it.k, M, N);  // M x N
      for (int p2 = 0; p2 < N; ++p2)
        for (int p1 = 0; p1 < M; ++p1) dst[(size_t)p2 * M + p1] = g[(size_t)p1 * N + p2];
    }
  };
  unsigned hw = std::thread::hardware_concurrency();
  const int nth = (int)std::max(1u, std::min(hw ? hw : 1u, 16u));
  std::vector<std::thread> pool;
  for (int t = 0; t < nth; ++t)
    pool.emplace_back([&, t]() { for (int i = t; i < K; i += nth) work(i); });
  for (auto& th : pool) th.join();
  return "";
}

}  // namespace shl
