// fused.cu - paired-subband transform kernels: both passes of a 2D transform
// in one persistent launch of thread-block clusters, with the plane between
// the passes kept in a per-cluster slot that stays in L2.
//
// Pairing (Sec. 3.4 decomposition and reconstruction for real images and a
// real, even filter bank).  The coefficients c_s of every subband are real,
// so two subbands s, s' of one image travel as one complex plane
// z = c_s + i c_s':
//   decomposition   z = IFFT2( X * (G_s + i G_s') )       (X = FFT2(image))
//   reconstruction  H = sum_i G_i FFT2(c_i)  over the half plane kx <= M/2,
//                   each pair adding  a Z + conj(a) Q,  Z = FFT2(z)[kx][ky],
//                   Q = conj(Z[-kx][-ky]),  a = (G_s - i G_s') / 2.
// A real row needs no real-FFT split: a complex line FFT of length M is the
// whole row transform of two subbands.  Both identities follow from
// FFT2(real c)[-k] = conj FFT2(c)[k] and G_i[-k] = G_i[k].
//
// The plane of a pair is N x M complex.  Full-plane column kx > M/2 is not
// formed from mirrored half-plane data: for the decomposition
//   IFFT_y( X[M-kx] (G_s + i G_s')[M-kx] ) = conj( a - i b ),
//   a = IFFT_y(X[kx] G_s[kx]),  b = IFFT_y(X[kx] G_s'[kx]),
// and for the reconstruction Q[kx][ky] = FFT_y( conj slot[M-kx] )[ky], so
// every lane keeps its own ky; columns 0 and M/2 mirror onto themselves and
// take Q from the mirrored line in shared memory.
//
// Cluster of C CTAs (one per SM), one pair ("unit") at a time, units of an
// image consecutive.  The cluster's slot holds the plane as [kx][y] (y
// contiguous, N * M * 8 bytes):
//   k_pair_dec  A: jobs kx = 0..M/2-1 (kx = 0 also makes column M/2); lane
//                  group g < JPR computes a, g >= JPR computes b of job
//                  (g mod JPR); they swap through shared memory and write
//                  columns kx and M - kx of the slot.
//               B: TRW-row tiles of the slot (cp.async, 8-byte swizzled, two
//                  stages) -> inverse row FFT -> real part to c_s, imaginary
//                  part to c_s' (float32 or bfloat16 RNE).
//   k_pair_rec  A: rows of c_s, c_s' (thresholded on read) -> forward row
//                  FFT -> swizzled tile -> slot columns.
//               B: job kx: group g < JPR transforms slot column kx, group
//                  g >= JPR the conjugated column M - kx; g < JPR adds
//                  a Z + conj(a) Q to the cluster's partial plane of the image.
//   k_pair_final  per image: partial planes in cluster order -> x scale [/W]
//                  -> inverse column FFT; the real rows follow with
//                  k_rows_c2r_t.
// Hardware cluster barriers separate the passes (release / acquire at cluster
// scope); every CTA of a cluster runs the same units, so every barrier is
// reached by all of them.
#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "warp_fft.cuh"

namespace shl {
namespace fz {

__device__ __forceinline__ int cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return (int)r;
}
__device__ __forceinline__ int cl_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return (int)r;
}
__device__ __forceinline__ int cl_id() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return (int)r;
}
__device__ __forceinline__ int cl_count() {
  unsigned r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return (int)r;
}
// Split cluster barrier: arrive publishes this thread's prior memory
// operations (release), wait returns once every thread of the cluster has
// arrived and makes their writes visible (acquire).
__device__ __forceinline__ void cl_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cl_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Natural-order values v[u] = x[j + u T] back from a padded line buffer
// written by line_store (the same addressing).
template <int L, int R>
__device__ __forceinline__ void line_load(float2 (&v)[R], const float2* sm, int j) {
  constexpr int T = L / R;
  if constexpr (T % R == 0) {
    const float2* p = sm + pad_base<R>(j);
#pragma unroll
    for (int u = 0; u < R; ++u) v[u] = p[u * (T + T / R)];
  } else {
#pragma unroll
    for (int u = 0; u < R; ++u) v[u] = sm[pad_index(j + u * T, ilog2(R))];
  }
}

// Twiddle bases of one lane for line_fft512 (j = lane), from the float64-
// built table tw[q] = exp(-2 pi i q / 4096): b^(1,2,4,8) with
// b = exp(-2 pi i (j mod 16) / 256) for the middle stage, and
// w0 = exp(-2 pi i j / 512) for the last one.
struct Tw512 {
  float2 b1, b2, b4, b8, w0;
};
__device__ __forceinline__ Tw512 tw512_load(const float2* __restrict__ tw, int j) {
  const int m = j & 15;
  return Tw512{__ldg(tw + m * 16), __ldg(tw + m * 32), __ldg(tw + m * 64), __ldg(tw + m * 128),
               __ldg(tw + j * 8)};
}

// 512-point FFT of one line held by one warp, v[u] = x[j + 32 u] in and
// X[j + 32 u] out (SIGN -1 forward, +1 inverse, unnormalised): the same
// radix-16, radix-16, radix-2 Stockham passes and shared-memory exchanges as
// line_fft<512, 16>, with the twiddles formed in registers instead of loaded
// (middle stage: b^u as products of b, b^2, b^4, b^8, at most two roundings;
// last stage: w0 times the constant 16th roots of unity).
template <int SIGN>
__device__ __forceinline__ void line_fft512(float2 (&v)[16], float2* sm, int j, const Tw512& t) {
  constexpr int R = 16, T = 32;
  auto cj = [](float2 a) { return SIGN < 0 ? a : make_float2(a.x, -a.y); };
  dft_reg<R, SIGN>(v);
  __syncwarp();
  {
    float2* wp = sm + j * (R + 1);
#pragma unroll
    for (int u = 0; u < R; ++u) wp[u] = v[u];
  }
  __syncwarp();
  const float2* rp = sm + pad_base<R>(j);
#pragma unroll
  for (int u = 0; u < R; ++u) v[u] = rp[u * (T + T / R)];
  {
    float2 w[R];
    w[1] = cj(t.b1); w[2] = cj(t.b2); w[4] = cj(t.b4); w[8] = cj(t.b8);
    w[3] = cmul(w[2], w[1]); w[5] = cmul(w[4], w[1]); w[6] = cmul(w[4], w[2]);
    w[7] = cmul(w[4], w[3]); w[9] = cmul(w[8], w[1]); w[10] = cmul(w[8], w[2]);
    w[11] = cmul(w[8], w[3]); w[12] = cmul(w[8], w[4]); w[13] = cmul(w[8], w[5]);
    w[14] = cmul(w[8], w[6]); w[15] = cmul(w[8], w[7]);
#pragma unroll
    for (int u = 1; u < R; ++u) v[u] = cmul(v[u], w[u]);
  }
  dft_reg<R, SIGN>(v);
  __syncwarp();
  {
    float2* wp = sm + pad_base<R>(((j >> 4) << 8) + (j & 15));
#pragma unroll
    for (int u = 0; u < R; ++u) wp[u * (R + 1)] = v[u];
  }
  __syncwarp();
#pragma unroll
  for (int u = 0; u < R; ++u) v[u] = rp[u * (T + T / R)];
  const float2 w0 = cj(t.w0);
#pragma unroll
  for (int q = 0; q < R / 2; ++q) {
    float2 x1 = cmul(v[q + R / 2], w0);
    switch (q) {              // times exp(SIGN 2 pi i q / 16)
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

}  // namespace fz

// Square planes L x L (N = M = L), one lane group = one warp (T = 32).
template <int LOG_L>
struct PairCfg {
  static constexpr int L = 1 << LOG_L;
  static constexpr int Mh = L / 2 + 1;
  static constexpr int R = LineRadix<L>::R;
  using C = LineCfg<L, R>;
  static constexpr int T = C::T;
  static constexpr int THREADS = 512;
  static constexpr int NG = THREADS / T;        // lane groups (warps)
  static constexpr int JPR = NG / 2;            // column jobs per round
  static constexpr int TRW = NG;                // rows per tile, one per group
  static constexpr size_t WORDS = C::WORDS;     // padded line buffer of one group
  static constexpr size_t LINE_W = (size_t)NG * WORDS;
  static constexpr size_t TW_W = ((size_t)LineTw<L, R>::WORDS + 1) & ~size_t(1);
  static constexpr size_t TILE_W = (size_t)L * TRW;
  // decomposition: line buffers, then two stages used by pass A as X lines
  // [JPR+1][L] float2 + G lines [JPR+1][2][L] float and by pass B as row tiles
  static constexpr size_t DSTAGE_A = 2 * (size_t)(JPR + 1) * L;
  static constexpr size_t DSTAGE_W = DSTAGE_A > TILE_W ? DSTAGE_A : TILE_W;
  static constexpr size_t DEC_SMEM = sizeof(float2) * (LINE_W + 2 * DSTAGE_W);
  // reconstruction: two sets of group buffers (each group's staged input,
  // then its line buffer), then a region that holds pass A's output tile or
  // pass B's two G stages [JPR+1][2][L] float
  static constexpr size_t RG_W = (size_t)(JPR + 1) * L;
  static constexpr size_t RT_W = 2 * RG_W > TILE_W ? 2 * RG_W : TILE_W;
  static constexpr size_t REC_SMEM = sizeof(float2) * (2 * LINE_W + RT_W);
  static_assert(T == 32, "one warp per line");
  static_assert((TRW & (TRW - 1)) == 0 && (JPR & (JPR - 1)) == 0, "groups must be powers of two");
  static_assert(DEC_SMEM <= 227 * 1024 && REC_SMEM <= 227 * 1024, "shared memory");
};

struct PairArgs {
  const float2* X;       // dec: image half spectra [B][Mh][L] (kx-major)
  const float* G;        // [K][Mh][L] real half spectra, kx-major
  const float* invW;     // dec: [Mh][L] for the dual-weighted decomposition, else null
  void* coeffs;          // [B][K][L][L] float32 or bfloat16
  const float* thresh;   // rec: [B][K] or null
  float2* slots;         // [clusters][L][L] (kx-major planes)
  float2* parts;         // rec: [clusters + B - 1][Mh][L] partial half planes
  const float2* tw;
  float scale;
  int K, P, units;       // P = ceil(K / 2) pairs per image, units = B * P
};

namespace fz {
__device__ __forceinline__ void cp16(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// The 2 * 32 threads of warps g and g ^ JPR (a partner pair).
__device__ __forceinline__ void pair_sync(int id) {
  asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory");
}

// Unit u -> image b and its pair of filters s, s2 (s2 = -1: no partner).
__device__ __forceinline__ void unit_of(const PairArgs& a, int u, int* b, int* s, int* s2) {
  *b = u / a.P;
  const int q = u - *b * a.P;
  *s = 2 * q;
  *s2 = 2 * q + 1 < a.K ? 2 * q + 1 : -1;
}

// Lines of a column round: jobs jx0 .. jx0 + JPR - 1, and for jx0 == 0 also
// column L/2 as line JPR.  X lines [JPR+1][L] float2 into Xs (when Xs is not
// null), G lines [JPR+1][2][L] float of filters s, s2 into Gs (s2 < 0: only
// f = 0).  Each thread copies fixed 16-byte offsets of a fixed set of lines.
template <int L, int JPR>
__device__ __forceinline__ void stage_columns(float2* Xs, float* Gs, const float2* Xb,
                                              const float* G, int Mh, int s, int s2, int jx0,
                                              int tid) {
  static_assert(L == 512 && JPR == 8, "chunk mapping of 512 threads");
  const int nf = s2 >= 0 ? 2 : 1;
  if (Xs) {                                 // 256 chunks a line: 2 lines per pass
    const int o = tid & 255, l0 = tid >> 8;
    const float2* src = Xb + (size_t)(jx0 + l0) * L + 2 * o;
    float2* dst = Xs + (size_t)l0 * L + 2 * o;
#pragma unroll
    for (int i = 0; i < JPR / 2; ++i) cp16(dst + (size_t)2 * i * L, src + (size_t)2 * i * L);
  }
  {                                         // 128 chunks a line: 4 lines per pass
    const int o = tid & 127, q0 = tid >> 7;
    if (nf == 2) {                          // line q = 2 i + f
      const int f = q0 & 1, i0 = q0 >> 1;
      const float* src = G + ((size_t)(s + f) * Mh + jx0 + i0) * L + 4 * o;
      float* dst = Gs + ((size_t)2 * i0 + f) * L + 4 * o;
#pragma unroll
      for (int i = 0; i < JPR / 2; ++i) cp16(dst + (size_t)4 * i * L, src + (size_t)2 * i * L);
    } else {
      const float* src = G + ((size_t)s * Mh + jx0 + q0) * L + 4 * o;
      float* dst = Gs + (size_t)2 * q0 * L + 4 * o;
#pragma unroll
      for (int i = 0; i < JPR / 4; ++i) cp16(dst + (size_t)8 * i * L, src + (size_t)4 * i * L);
    }
  }
  if (jx0 == 0) {                           // column L/2 as line JPR
    if (Xs && tid < 256) cp16(Xs + (size_t)JPR * L + 2 * tid, Xb + (size_t)(L / 2) * L + 2 * tid);
    if (tid < 128 * nf) {
      const int f = tid >> 7, o = tid & 127;
      cp16(Gs + ((size_t)2 * JPR + f) * L + 4 * o, G + ((size_t)(s + f) * Mh + L / 2) * L + 4 * o);
    }
  }
}
}  // namespace fz

// ------------------------------------------------------------ decomposition
template <int LOG_L, bool BF16, bool DUAL>
__global__ void __launch_bounds__(512, 1) k_pair_dec(PairArgs a) {
  using P = PairCfg<LOG_L>;
  constexpr int L = P::L, R = P::R, T = P::T, JPR = P::JPR, TRW = P::TRW, Mh = P::Mh;
  extern __shared__ __align__(16) float2 smem[];
  float2* lines = smem;
  float2* stg0 = lines + P::LINE_W;
  const int tid = threadIdx.x, g = tid / T, j = tid % T;
  float2* line = lines + (size_t)g * P::WORDS;
  const int C = fz::cl_size(), r = fz::cl_rank(), cid = fz::cl_id(), ncl = fz::cl_count();
  const fz::Tw512 tw5 = fz::tw512_load(a.tw, j);
  const int u0 = (int)((long long)cid * a.units / ncl);
  const int u1 = (int)((long long)(cid + 1) * a.units / ncl);
  float2* slot = a.slots + (size_t)cid * L * L;
  const int JPC = (L / 2) / C, RPC = L / C, nA = JPC / JPR, ntile = RPC / TRW;
  const bool bpart = g >= JPR;
  const int gi = g & (JPR - 1);
  auto stage = [&](int k) { return stg0 + (size_t)(k & 1) * P::DSTAGE_W; };
  auto stage_g = [&](int k) { return reinterpret_cast<float*>(stage(k) + (size_t)(JPR + 1) * L); };
  if (u0 < u1) {                              // first unit's first column round
    int b, s, s2;
    fz::unit_of(a, u0, &b, &s, &s2);
    fz::stage_columns<L, JPR>(stage(0), stage_g(0), a.X + (size_t)b * Mh * L, a.G, Mh, s, s2,
                              r * JPC, tid);
  }
  fz::cp_commit();

  for (int u = u0; u < u1; ++u) {
    int b, s, s2;
    fz::unit_of(a, u, &b, &s, &s2);
    const float2* Xb = a.X + (size_t)b * Mh * L;

    // -------- pass A: inverse column FFTs of the pair's plane -> slot.
    // Round k reads stage k & 1; nA and ntile are even, so every unit
    // starts on stage 0.  One CTA barrier a round: after it every thread's
    // copies of round k have landed and every group has finished round k - 1,
    // whose stage then takes round k + 1.
    for (int k = 0; k < nA; ++k) {
      const int jx0 = r * JPC + k * JPR;
      fz::cp_wait<0>();
      __syncthreads();
      if (k + 1 < nA)
        fz::stage_columns<L, JPR>(stage(k + 1), stage_g(k + 1), Xb, a.G, Mh, s, s2, jx0 + JPR, tid);
      fz::cp_commit();
      const float2* S = stage(k);
      const float* Gs = stage_g(k);
      const int jx = jx0 + gi;
      // group g < JPR: full-plane column jx, X (G_s + i G_s') at ky;
      // group g >= JPR: column L - jx, conj(X) (G_s + i G_s') at -ky of the
      // same staged lines (Hermitian X, even G); job 0: columns 0 and L/2
      const bool mirror = bpart && jx != 0;
      const int li = (jx == 0 && bpart) ? JPR : gi;
      const int col = jx == 0 ? (bpart ? L / 2 : 0) : (bpart ? L - jx : jx);
      const int kw = jx == 0 ? col : jx;         // half-plane column of the weights
      const float2* xl = S + (size_t)li * L;
      const float* g1 = Gs + (size_t)li * 2 * L;
      float2 v[R];
#pragma unroll
      for (int e = 0; e < R; ++e) {
        const int p = j + e * T;
        const int m = mirror ? ((L - p) & (L - 1)) : p;
        const float sc = DUAL ? a.scale * __ldg(a.invW + (size_t)kw * L + m) : a.scale;
        const float h1 = g1[m] * sc, h2 = s2 >= 0 ? g1[L + m] * sc : 0.f;
        float2 x = xl[m];
        if (mirror) x.y = -x.y;
        v[e] = make_float2(fmaf(x.x, h1, -x.y * h2), fmaf(x.x, h2, x.y * h1));
      }
      fz::line_fft512<+1>(v, line, j, tw5);
      if (k == 0 && u > u0) fz::cl_wait();   // every CTA has read the previous unit's slot
      float2* dst = slot + (size_t)col * L + j;
#pragma unroll
      for (int e = 0; e < R; ++e) dst[e * T] = v[e];
    }
    fz::cl_arrive();
    fz::cl_wait();                           // slot complete

    // -------- pass B: TRW-row tiles -> inverse row FFT -> coefficient rows.
    // Thread tid copies row rr = tid % TRW of kx = tid / TRW + (512 / TRW) i.
    const int y0c = r * RPC;
    const int rr = tid & (TRW - 1), kx0 = tid / TRW;
    constexpr int KXS = 512 / TRW;
    auto issue = [&](float2* dst, int y0) {
      const float2* src = slot + (size_t)kx0 * L + y0 + rr;
      float2* d = dst + kx0 * TRW + (rr ^ (kx0 & (TRW - 1)));
#pragma unroll
      for (int i = 0; i < L / KXS; ++i)      // (kx0 + KXS i) & (TRW - 1) == kx0 & (TRW - 1)
        fz::cp_async8(d + (size_t)i * KXS * TRW, src + (size_t)i * KXS * L);
    };
    issue(stage(0), y0c);
    fz::cp_commit();
    const size_t sub1 = (size_t)b * a.K + s;
    for (int t = 0; t < ntile; ++t) {
      fz::cp_wait<0>();
      __syncthreads();
      if (t + 1 < ntile) {
        issue(stage(t + 1), y0c + (t + 1) * TRW);
      } else {
        fz::cl_arrive();                     // this CTA's slot reads are complete
        if (u + 1 < u1) {                    // next unit's first column round
          int b2, s_, s2_;
          fz::unit_of(a, u + 1, &b2, &s_, &s2_);
          fz::stage_columns<L, JPR>(stage(t + 1), stage_g(t + 1), a.X + (size_t)b2 * Mh * L, a.G, Mh,
                                    s_, s2_, r * JPC, tid);
        }
      }
      fz::cp_commit();
      const float2* cur = stage(t);
      const int y = y0c + t * TRW + g;
      float2 v[R];
#pragma unroll
      for (int e = 0; e < R; ++e) {
        const int p = j + e * T;
        v[e] = cur[p * TRW + (g ^ (p & (TRW - 1)))];
      }
      fz::line_fft512<+1>(v, line, j, tw5);
      const size_t row1 = (sub1 * L + y) * L + j;
      const size_t row2 = row1 + (size_t)L * L;
      if constexpr (BF16) {
        __nv_bfloat16* o = static_cast<__nv_bfloat16*>(a.coeffs);
#pragma unroll
        for (int e = 0; e < R; ++e) o[row1 + e * T] = __float2bfloat16_rn(v[e].x);
        if (s2 >= 0) {
#pragma unroll
          for (int e = 0; e < R; ++e) o[row2 + e * T] = __float2bfloat16_rn(v[e].y);
        }
      } else {
        float* o = static_cast<float*>(a.coeffs);
#pragma unroll
        for (int e = 0; e < R; ++e) __stcs(o + row1 + e * T, v[e].x);
        if (s2 >= 0) {
#pragma unroll
          for (int e = 0; e < R; ++e) __stcs(o + row2 + e * T, v[e].y);
        }
      }
    }
  }
  fz::cp_wait<0>();
  if (u1 > u0) fz::cl_wait();                // pairs the last unit's arrive
}

// ----------------------------------------------------------- reconstruction
// Accumulator of the half-plane columns of this CTA's jobs in tensor memory:
// the job of group gi (< JPR) in round k owns TMEM columns
// 256 (gi / 4) + 32 k .. + 31 of lanes 32 (gi % 4) + j, in which warp gi adds
// its elements 0..7 (words 0..15) and warp gi + JPR, which shares the lane
// quadrant, elements 8..15 (words 16..31); the self-mirrored column 0 takes
// all 32 words from warp 0.
#define SHL_TM_LD32(R, ADDR)                                                                  \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "                                     \
               "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"                     \
               "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"    \
               : "=r"((R)[0]), "=r"((R)[1]), "=r"((R)[2]), "=r"((R)[3]), "=r"((R)[4]),        \
                 "=r"((R)[5]), "=r"((R)[6]), "=r"((R)[7]), "=r"((R)[8]), "=r"((R)[9]),        \
                 "=r"((R)[10]), "=r"((R)[11]), "=r"((R)[12]), "=r"((R)[13]), "=r"((R)[14]),   \
                 "=r"((R)[15]), "=r"((R)[16]), "=r"((R)[17]), "=r"((R)[18]), "=r"((R)[19]),   \
                 "=r"((R)[20]), "=r"((R)[21]), "=r"((R)[22]), "=r"((R)[23]), "=r"((R)[24]),   \
                 "=r"((R)[25]), "=r"((R)[26]), "=r"((R)[27]), "=r"((R)[28]), "=r"((R)[29]),   \
                 "=r"((R)[30]), "=r"((R)[31])                                                 \
               : "r"(ADDR)                                                                    \
               : "memory")
#define SHL_TM_ST32(ADDR, R)                                                                  \
  asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "                               \
               "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"                    \
               "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"           \
               ::"r"(ADDR), "r"((R)[0]), "r"((R)[1]), "r"((R)[2]), "r"((R)[3]), "r"((R)[4]),  \
                 "r"((R)[5]), "r"((R)[6]), "r"((R)[7]), "r"((R)[8]), "r"((R)[9]),             \
                 "r"((R)[10]), "r"((R)[11]), "r"((R)[12]), "r"((R)[13]), "r"((R)[14]),        \
                 "r"((R)[15]), "r"((R)[16]), "r"((R)[17]), "r"((R)[18]), "r"((R)[19]),        \
                 "r"((R)[20]), "r"((R)[21]), "r"((R)[22]), "r"((R)[23]), "r"((R)[24]),        \
                 "r"((R)[25]), "r"((R)[26]), "r"((R)[27]), "r"((R)[28]), "r"((R)[29]),        \
                 "r"((R)[30]), "r"((R)[31])                                                   \
               : "memory")

#define SHL_TM_LD16(R, ADDR)                                                                  \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "                                     \
               "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"             \
               : "=r"((R)[0]), "=r"((R)[1]), "=r"((R)[2]), "=r"((R)[3]), "=r"((R)[4]),        \
                 "=r"((R)[5]), "=r"((R)[6]), "=r"((R)[7]), "=r"((R)[8]), "=r"((R)[9]),        \
                 "=r"((R)[10]), "=r"((R)[11]), "=r"((R)[12]), "=r"((R)[13]), "=r"((R)[14]),   \
                 "=r"((R)[15])                                                                \
               : "r"(ADDR)                                                                    \
               : "memory")
#define SHL_TM_ST16(ADDR, R)                                                                  \
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "                               \
               "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"                   \
               ::"r"(ADDR), "r"((R)[0]), "r"((R)[1]), "r"((R)[2]), "r"((R)[3]), "r"((R)[4]),  \
                 "r"((R)[5]), "r"((R)[6]), "r"((R)[7]), "r"((R)[8]), "r"((R)[9]),             \
                 "r"((R)[10]), "r"((R)[11]), "r"((R)[12]), "r"((R)[13]), "r"((R)[14]),        \
                 "r"((R)[15])                                                                 \
               : "memory")

template <int LOG_L, bool BF16, bool THRESH>
__global__ void __launch_bounds__(512, 1) k_pair_rec(PairArgs a) {
  using P = PairCfg<LOG_L>;
  constexpr int L = P::L, R = P::R, T = P::T, JPR = P::JPR, TRW = P::TRW, Mh = P::Mh;
  static_assert(2 * R == 32, "one TMEM access of 32 words per line");
  extern __shared__ __align__(16) float2 smem[];
  __shared__ uint32_t s_tmem;
  float2* set0 = smem;                                  // group buffers, two sets
  float2* tile = set0 + 2 * P::LINE_W;                  // pass A output tile
  const int tid = threadIdx.x, g = tid / T, j = tid % T;
  const int C = fz::cl_size(), r = fz::cl_rank(), cid = fz::cl_id(), ncl = fz::cl_count();
  auto buf_of = [&](int k, int grp) { return set0 + (size_t)(k & 1) * P::LINE_W + (size_t)grp * P::WORDS; };
  auto gstage = [&](int k) { return reinterpret_cast<float*>(tile + (size_t)(k & 1) * P::RG_W); };
  const fz::Tw512 tw5 = fz::tw512_load(a.tw, j);
  if (g == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     fz::smem_u32(&s_tmem)), "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  // warp g and its partner g ^ JPR share lane quadrant g % 4; the job of
  // group gi = g % JPR owns columns 256 (gi / 4) + 32 k .. + 31 in round k
  const uint32_t tjob = tmem + ((uint32_t)(32 * (g & 3)) << 16) + (uint32_t)(((g & (JPR - 1)) >> 2) & 1) * 256u;
  const uint32_t tacc = tjob;
  const int u0 = (int)((long long)cid * a.units / ncl);
  const int u1 = (int)((long long)(cid + 1) * a.units / ncl);
  float2* slot = a.slots + (size_t)cid * L * L;
  const int JPC = (L / 2) / C, RPC = L / C, nA = JPC / JPR, ntile = RPC / TRW;
  const bool bpart = g >= JPR;
  const int gi = g & (JPR - 1);
  // pass A input of tile t: rows y0 .. y0 + TRW - 1 of subbands s and s2,
  // row y0 + grp into group grp's buffer of set t & 1 (subband s in its
  // first half, s2 in its second)
  auto issue_rows = [&](int u, int t) {
    int b, s, s2;
    fz::unit_of(a, u, &b, &s, &s2);
    const size_t sub1 = (size_t)b * a.K + s;
    constexpr int ESZ = BF16 ? 2 : 4;
    constexpr int RC = L * ESZ / 16;             // 16-byte chunks of a row
    constexpr int RPP = 512 / RC;                // rows (group, f) a pass
    const int o = tid % RC, q0 = tid / RC;
    const int nq = (s2 >= 0 ? 2 : 1) * TRW;
    const int y0 = r * RPC + t * TRW;
    const char* base = static_cast<const char*>(a.coeffs);
    for (int q = q0; q < nq; q += RPP) {         // q = 2 grp + f (f = 0 only without s2)
      const int f = s2 >= 0 ? (q & 1) : 0, grp = s2 >= 0 ? (q >> 1) : q;
      char* d = reinterpret_cast<char*>(buf_of(t, grp)) + (size_t)f * L * ESZ + (size_t)o * 16;
      fz::cp16(d, base + (((sub1 + f) * L + y0 + grp) * L) * ESZ + (size_t)o * 16);
    }
  };
  if (u0 < u1) issue_rows(u0, 0);
  fz::cp_commit();

  for (int u = u0; u < u1; ++u) {
    int b, s, s2;
    fz::unit_of(a, u, &b, &s, &s2);
    const int q = s / 2;
    const size_t sub1 = (size_t)b * a.K + s;
    float tau1 = 0.f, tau2 = 0.f;
    if (THRESH) {
      tau1 = __ldg(a.thresh + sub1);
      if (s2 >= 0) tau2 = __ldg(a.thresh + sub1 + 1);
    }
    const bool first = (u == u0) || (q == 0);       // first unit of this image here
    const bool last = (u + 1 == u1) || (q + 1 == a.P);

    // -------- pass A: coefficient rows -> forward row FFT -> slot columns
    const int y0c = r * RPC;
    for (int t = 0; t < ntile; ++t) {
      const int y0 = y0c + t * TRW;
      fz::cp_wait<0>();
      __syncthreads();                       // tile t landed; tile t - 1 fully done
      if (t + 1 < ntile) issue_rows(u, t + 1);
      fz::cp_commit();
      float2* buf = buf_of(t, g);
      float2 v[R];
      if constexpr (BF16) {
        const __nv_bfloat16* in = reinterpret_cast<const __nv_bfloat16*>(buf);
#pragma unroll
        for (int e = 0; e < R; ++e) {
          const int p = j + e * T;
          float c1 = __bfloat162float(in[p]);
          float c2 = s2 >= 0 ? __bfloat162float(in[L + p]) : 0.f;
          if (THRESH) {
            if (fabsf(c1) < tau1) c1 = 0.f;
            if (fabsf(c2) < tau2) c2 = 0.f;
          }
          v[e] = make_float2(c1, c2);
        }
      } else {
        const float* in = reinterpret_cast<const float*>(buf);
#pragma unroll
        for (int e = 0; e < R; ++e) {
          const int p = j + e * T;
          float c1 = in[p];
          float c2 = s2 >= 0 ? in[L + p] : 0.f;
          if (THRESH) {
            if (fabsf(c1) < tau1) c1 = 0.f;
            if (fabsf(c2) < tau2) c2 = 0.f;
          }
          v[e] = make_float2(c1, c2);
        }
      }
      fz::line_fft512<-1>(v, buf, j, tw5);
#pragma unroll
      for (int e = 0; e < R; ++e) {
        const int p = j + e * T;
        tile[p * TRW + (g ^ (p & (TRW - 1)))] = v[e];
      }
      __syncthreads();
      if (t == 0 && u > u0) fz::cl_wait();   // every CTA has read the previous unit's slot
      {
        // thread: kx = tid / 8 + 64 i, row pair m2 = 2 (tid % 8)
        const int kxa = tid >> 3, m2 = 2 * (tid & 7);
        const int sw = kxa & (TRW - 1);      // (kxa + 64 i) & 15 == kxa & 15
        const float2* tl = tile + kxa * TRW;
        float2* dst = slot + (size_t)kxa * L + y0 + m2;
#pragma unroll
        for (int i = 0; i < L / 64; ++i) {
          const float2 lo = tl[i * 64 * TRW + (m2 ^ sw)], hi = tl[i * 64 * TRW + ((m2 + 1) ^ sw)];
          *reinterpret_cast<float4*>(dst + (size_t)i * 64 * L) = make_float4(lo.x, lo.y, hi.x, hi.y);
        }
      }
    }
    fz::cl_arrive();
    fz::cl_wait();                           // slot complete

    // -------- pass B: column FFTs, pair combination, partial sum of the image.
    // Round k: group g's column staged in buf_of(k, g) (then its line
    // buffer), filters in gstage(k).
    auto issue_cols = [&](int k) {
      const int jx0 = r * JPC + k * JPR;
      constexpr int XC = L * 8 / 16;               // 256 chunks a column, 2 columns a pass
      const int o = tid & (XC - 1), g0 = tid >> 8;
#pragma unroll
      for (int i = 0; i < P::NG / 2; ++i) {
        const int gg = g0 + 2 * i, jj = jx0 + (gg & (JPR - 1));
        const int cc = jj == 0 ? (gg >= JPR ? L / 2 : 0) : (gg >= JPR ? L - jj : jj);
        fz::cp16(buf_of(k, gg) + 2 * o, slot + (size_t)cc * L + 2 * o);
      }
      fz::stage_columns<L, JPR>(nullptr, gstage(k), nullptr, a.G, Mh, s, s2, jx0, tid);
    };
    issue_cols(0);
    fz::cp_commit();
    float2* part = a.parts + (size_t)(cid + b) * Mh * L;
    for (int k = 0; k < nA; ++k) {
      fz::cp_wait<0>();
      __syncthreads();                       // round k landed; round k - 1 fully done
      if (k + 1 < nA) {
        issue_cols(k + 1);
      } else {
        fz::cl_arrive();                     // this CTA's slot reads are complete
        if (u + 1 < u1) issue_rows(u + 1, 0);  // next unit's first input tile
      }
      fz::cp_commit();
      float2* buf = buf_of(k, g);
      const float* Gs = gstage(k);
      const int jx = r * JPC + k * JPR + gi;
      const bool special = jx == 0;
      float2 v[R];
#pragma unroll
      for (int e = 0; e < R; ++e) {
        const float2 z = buf[j + e * T];
        v[e] = (bpart && !special) ? make_float2(z.x, -z.y) : z;
      }
      fz::line_fft512<-1>(v, buf, j, tw5);
      line_store<L, R>(v, buf, j);
      if (special) {
        // self-mirrored column (0 in group 0, L/2 in group JPR): Q[ky] = conj Z[-ky]
        __syncwarp();
        float2 Q[R];
        line_load_mirror<L, R>(Q, buf, j);
        const float* g1 = Gs + (size_t)(bpart ? JPR : 0) * 2 * L;
        uint32_t cw[2 * R];
#pragma unroll
        for (int e = 0; e < R; ++e) {
          const int p = j + e * T;
          const float h1 = g1[p], h2 = s2 >= 0 ? g1[L + p] : 0.f;
          const float2 Zp = v[e], Qp = make_float2(Q[e].x, -Q[e].y);
          cw[2 * e] = __float_as_uint(fmaf(h1, Zp.x + Qp.x, h2 * (Zp.y - Qp.y)));
          cw[2 * e + 1] = __float_as_uint(fmaf(h1, Zp.y + Qp.y, -h2 * (Zp.x - Qp.x)));
        }
        if (!bpart) {            // column 0: tensor memory, all 32 words
          const uint32_t ta = tacc + (uint32_t)k * 32u;
          if (!first) {
            uint32_t old[2 * R];
            SHL_TM_LD32(old, ta);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int w = 0; w < 2 * R; ++w)
              cw[w] = __float_as_uint(__uint_as_float(cw[w]) + __uint_as_float(old[w]));
          }
          if (last) {
            float2* pc = part + j;
#pragma unroll
            for (int e = 0; e < R; ++e)
              pc[e * T] = make_float2(__uint_as_float(cw[2 * e]), __uint_as_float(cw[2 * e + 1]));
          } else {
            SHL_TM_ST32(ta, cw);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          }
        } else {                 // column L/2: partial plane in global memory
          float2* pc = part + (size_t)(L / 2) * L + j;
#pragma unroll
          for (int e = 0; e < R; ++e) {
            float2 c = make_float2(__uint_as_float(cw[2 * e]), __uint_as_float(cw[2 * e + 1]));
            if (!first) c = cadd(c, pc[e * T]);
            pc[e * T] = c;
          }
        }
      } else {
        // job jx: Z = FFT(slot[jx]) in group gi, Q = FFT(conj slot[L - jx]) in
        // group gi + JPR; after the swap group gi combines elements 0..7 and
        // group gi + JPR elements 8..15 (words 16 h .. 16 h + 15 of the job's
        // TMEM columns, in the lanes both warps share)
        fz::pair_sync(1 + gi);
        const int h = bpart ? 1 : 0;
        const float2* own = buf + pad_base<R>(j);
        const float2* oth = buf_of(k, g ^ JPR) + pad_base<R>(j);
        const float* g1 = Gs + (size_t)gi * 2 * L;
        uint32_t cw[R];
#pragma unroll
        for (int e2 = 0; e2 < R / 2; ++e2) {
          const int e = (R / 2) * h + e2;
          const int p = j + e * T;
          const float2 A = own[e * (T + T / R)], Bv = oth[e * (T + T / R)];
          const float2 Zp = bpart ? Bv : A, Qp = bpart ? A : Bv;
          const float h1 = g1[p], h2 = s2 >= 0 ? g1[L + p] : 0.f;
          cw[2 * e2] = __float_as_uint(fmaf(h1, Zp.x + Qp.x, h2 * (Zp.y - Qp.y)));
          cw[2 * e2 + 1] = __float_as_uint(fmaf(h1, Zp.y + Qp.y, -h2 * (Zp.x - Qp.x)));
        }
        const uint32_t ta = tjob + (uint32_t)k * 32u + 16u * (uint32_t)h;
        if (!first) {
          uint32_t old[R];
          SHL_TM_LD16(old, ta);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int w = 0; w < R; ++w)
            cw[w] = __float_as_uint(__uint_as_float(cw[w]) + __uint_as_float(old[w]));
        }
        if (last) {              // image segment done: partial plane column
          float2* pc = part + (size_t)jx * L + j + (size_t)(R / 2) * h * T;
#pragma unroll
          for (int e2 = 0; e2 < R / 2; ++e2)
            pc[e2 * T] = make_float2(__uint_as_float(cw[2 * e2]), __uint_as_float(cw[2 * e2 + 1]));
        } else {
          SHL_TM_ST16(ta, cw);
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
      }
    }
  }
  fz::cp_wait<0>();
  if (u1 > u0) fz::cl_wait();                // pairs the last unit's arrive
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (g == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
}

// ------------------------------------------------------------- image lines
// Cluster that owns unit v when `units` units are split into `ncl`
// contiguous ranges [floor(c units / ncl), floor((c + 1) units / ncl)).
__host__ __device__ __forceinline__ int pair_cluster_of(int v, int units, int ncl) {
  return (int)(((long long)(v + 1) * ncl - 1) / units);
}

struct PairFinalArgs {
  const float2* parts;   // [clusters + B - 1][Mh][L]
  float2* A;             // [B][Mh][L] image spectrum lines, then their inverse column FFT
  const float* invW;     // [Mh][L] or null (adjoint)
  const float2* tw;
  float scale;           // applied with the factor 1/2 of the pair weights
  int B, P, units, ncl;
};

template <int LOG_L>
__global__ void __launch_bounds__(256) k_pair_final(PairFinalArgs f) {
  using P = PairCfg<LOG_L>;
  constexpr int L = P::L, R = P::R, T = P::T, Mh = P::Mh;
  constexpr int NGF = 256 / T;
  extern __shared__ __align__(16) float2 smem[];
  float2* twl = smem + (size_t)NGF * P::C::WORDS;
  const int g = threadIdx.x / T, j = threadIdx.x % T;
  float2* line = smem + (size_t)g * P::C::WORDS;
  LineTw<L, R>::fill(twl, f.tw, threadIdx.x, 256);
  __syncthreads();
  const int items = f.B * Mh;
  for (int it = blockIdx.x * NGF + g; it < items; it += gridDim.x * NGF) {
    const int b = it / Mh, kx = it - b * Mh;
    const int c0 = pair_cluster_of(b * f.P, f.units, f.ncl);
    const int c1 = pair_cluster_of((b + 1) * f.P - 1, f.units, f.ncl);
    float2 v[R];
#pragma unroll
    for (int e = 0; e < R; ++e) v[e] = make_float2(0.f, 0.f);
    for (int c = c0; c <= c1; ++c) {        // partial planes in cluster order
      const float2* pp = f.parts + ((size_t)(c + b) * Mh + kx) * L;
#pragma unroll
      for (int e = 0; e < R; ++e) v[e] = cadd(v[e], pp[j + e * T]);
    }
#pragma unroll
    for (int e = 0; e < R; ++e) {
      float sc = 0.5f * f.scale;
      if (f.invW) sc *= __ldg(f.invW + (size_t)kx * L + j + e * T);
      v[e] = cscale(v[e], sc);
    }
    line_fft<L, R, +1>(v, line, j, 1 + g, twl);
    float2* o = f.A + ((size_t)b * Mh + kx) * L;
#pragma unroll
    for (int e = 0; e < R; ++e) o[j + e * T] = v[e];
  }
}

// ------------------------------------------------------------------ launch
namespace {

int env_int(const char* k, int d) {
  const char* e = std::getenv(k);
  return e ? std::atoi(e) : d;
}

// Cluster size: 4 CTAs (SHL_PAIR_C = 8 overrides).  The reconstruction keeps
// JPC / JPR <= 8 rounds of accumulator columns per warp in tensor memory, and
// both kernels alternate their stages over an even number of rounds and
// tiles, so C is 4 or 8 at 512 x 512.
int pair_cluster_size() {
  static const int c = [] {
    const int v = env_int("SHL_PAIR_C", 4);
    return (v == 4 || v == 8) ? v : 4;
  }();
  return c;
}

template <typename Kern>
cudaError_t max_clusters(Kern kern, size_t smem, int C, int* out) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C * 64);
  cfg.blockDim = dim3(512);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(out, kern, &cfg);
}

template <typename Kern>
cudaError_t launch_cluster(Kern kern, size_t smem, int C, int ncl, const PairArgs& a,
                           cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C * ncl);
  cfg.blockDim = dim3(512);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

// Co-resident clusters of the paired kernels per device (both kernels take
// the same shared memory and one CTA per SM).
std::mutex g_mu;
int g_ncl[64] = {};

template <int LOG_L>
cudaError_t query_clusters(int C, int* out) {
  int a = 0, b = 0;
  cudaError_t e = max_clusters(k_pair_dec<LOG_L, false, false>, PairCfg<LOG_L>::DEC_SMEM, C, &a);
  if (!e) e = max_clusters(k_pair_rec<LOG_L, false, false>, PairCfg<LOG_L>::REC_SMEM, C, &b);
  *out = std::min(a, b);
  return e;
}

}  // namespace

bool pair_supported(int N, int M) { return N == M && N == 512; }

cudaError_t pair_max_clusters(int L, int* ncl) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ncl[dev]) {
    int n = 0;
    const int C = pair_cluster_size();
    switch (L) {
      case 512: e = query_clusters<9>(C, &n); break;
      default: return cudaErrorInvalidValue;
    }
    if (e) return e;
    if (n < 1) return cudaErrorInvalidConfiguration;
    g_ncl[dev] = n;
  }
  *ncl = g_ncl[dev];
  return cudaSuccess;
}

int pair_clusters_for(int ncl_max, int units) { return std::max(1, std::min(ncl_max, units)); }

cudaError_t launch_pair_dec(int L, bool bf16, const float2* X, const float* G, const float* invW,
                            void* coeffs, float2* slots, int ncl, float scale, int K, int B,
                            const float2* tw, cudaStream_t st) {
  PairArgs a{};
  a.X = X; a.G = G; a.invW = invW; a.coeffs = coeffs; a.slots = slots; a.tw = tw;
  a.scale = scale; a.K = K; a.P = (K + 1) / 2; a.units = B * a.P;
  if (a.units == 0) return cudaSuccess;
  const int C = pair_cluster_size();
  cudaError_t e;
#define SHL_PDEC(LG, BF, DU)                                                             \
  {                                                                                      \
    using Pc = PairCfg<LG>;                                                              \
    if ((e = cudaFuncSetAttribute(k_pair_dec<LG, BF, DU>,                                \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Pc::DEC_SMEM))) \
      return e;                                                                          \
    return launch_cluster(k_pair_dec<LG, BF, DU>, Pc::DEC_SMEM, C, ncl, a, st);          \
  }
  if (L == 512) {
    if (bf16) {
      if (invW) SHL_PDEC(9, true, true) else SHL_PDEC(9, true, false)
    } else {
      if (invW) SHL_PDEC(9, false, true) else SHL_PDEC(9, false, false)
    }
  }
#undef SHL_PDEC
  return cudaErrorInvalidValue;
}

cudaError_t launch_pair_rec(int L, bool bf16, const void* coeffs, const float* thresh,
                            const float* G, float2* slots, float2* parts, int ncl, int K, int B,
                            const float2* tw, cudaStream_t st) {
  PairArgs a{};
  a.G = G; a.coeffs = const_cast<void*>(coeffs); a.thresh = thresh; a.slots = slots;
  a.parts = parts; a.tw = tw; a.K = K; a.P = (K + 1) / 2; a.units = B * a.P;
  if (a.units == 0) return cudaSuccess;
  const int C = pair_cluster_size();
  cudaError_t e;
#define SHL_PREC(LG, BF, TH)                                                             \
  {                                                                                      \
    using Pc = PairCfg<LG>;                                                              \
    if ((e = cudaFuncSetAttribute(k_pair_rec<LG, BF, TH>,                                \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Pc::REC_SMEM))) \
      return e;                                                                          \
    return launch_cluster(k_pair_rec<LG, BF, TH>, Pc::REC_SMEM, C, ncl, a, st);          \
  }
  if (L == 512) {
    if (bf16) {
      if (thresh) SHL_PREC(9, true, true) else SHL_PREC(9, true, false)
    } else {
      if (thresh) SHL_PREC(9, false, true) else SHL_PREC(9, false, false)
    }
  }
#undef SHL_PREC
  return cudaErrorInvalidValue;
}

cudaError_t launch_pair_final(int L, const float2* parts, float2* A, const float* invW, float scale,
                              int K, int B, int ncl, const float2* tw, cudaStream_t st) {
  PairFinalArgs f{};
  f.parts = parts; f.A = A; f.invW = invW; f.tw = tw; f.scale = scale;
  f.B = B; f.P = (K + 1) / 2; f.units = B * f.P; f.ncl = ncl;
  if (f.units == 0) return cudaSuccess;
  cudaError_t e;
#define SHL_PFIN(LG)                                                                     \
  if (L == (1 << LG)) {                                                                  \
    using Pc = PairCfg<LG>;                                                              \
    constexpr int NGF = 256 / Pc::T;                                                     \
    const size_t sm = sizeof(float2) * ((size_t)NGF * Pc::C::WORDS + LineTw<Pc::L, Pc::R>::WORDS); \
    if ((e = cudaFuncSetAttribute(k_pair_final<LG>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  (int)sm)))                                             \
      return e;                                                                          \
    const int items = B * Pc::Mh;                                                        \
    const int grid = std::max(1, (items + NGF - 1) / NGF);                               \
    k_pair_final<LG><<<grid, 256, sm, st>>>(f);                                          \
    return cudaGetLastError();                                                           \
  }
  SHL_PFIN(9)
#undef SHL_PFIN
  return cudaErrorInvalidValue;
}

}  // namespace shl
