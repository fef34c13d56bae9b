// fast.cu - the transform kernels (warp-line design).
//
// Half spectra live "transposed": H[kx][ky], kx = 0..M/2 (Mh lines), ky =
// 0..N-1 contiguous, so that every column transform runs along one
// contiguous line owned by a lane group (line_fft).  Row transforms run on
// the image rows and move to / from the transposed layout through a
// 16-row shared-memory tile, whose global side is written or read as 128-byte
// runs.
//
//   k_rows_r2c_t  real rows (image, masked image or coefficients with
//                 threshold-on-read) -> R2C -> H planes.
//   k_rows_c2r_t  H planes -> C2R -> real rows (float32 or bfloat16).
//   k_lines_fwd   in-place forward column FFT of H lines (image spectra).
//   k_dec_lines   Z = IFFT_y(G_i * scale [* 1/W] * X_b) per subband line
//                 (the filter multiply of Sec. 3.4 fused into the load).
//   k_rec_lines   one CTA per (image, kx): lane groups split the chunk's
//                 filters, FFT_y each staged line (the next one prefetched
//                 with cp.async), multiply by G_i, sum in registers; the CTA
//                 adds the partial sums in fixed order, and on the image's
//                 last chunk applies scale [* 1/W] and the inverse column
//                 FFT (Sec. 3.4 reconstruction).
//   k_rows_shrink_t  in place on staged half spectra: C2R rows -> hard
//                 threshold in registers -> R2C rows (fused denoise / IHT).
//   k_dec_pipe    opt-in: k_dec_lines + k_rows_c2r_t in one cooperative
//                 launch over an L2-resident staging ring.
//
// Real-row packing: z[n] = x[2n] + i x[2n+1] with a length-M/2 complex FFT
// and the conjugate-pair split (the standard real-FFT identities):
//   R2C: X[k] = E[k] + exp(-2 pi i k/M) O[k], E = (Z[k] + conj Z[L-k]) / 2,
//        O = -i (Z[k] - conj Z[L-k]) / 2, X[L] = Re Z[0] - Im Z[0];
//   C2R: Z[k] = (X[k] + conj X[L-k]) + i exp(+2 pi i k/M) (X[k] - conj X[L-k]),
//        x[2n] + i x[2n+1] = unnormalised IFFT_L(Z)[n] (= M times the
//        normalised inverse; 1/(N M) is folded into filter or weight factors).
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "check.cuh"
#include "warp_fft.cuh"

SHL_CHECK_WORD_DEFINE

namespace shl {


// ------------------------------------------------------------------ rows
// The row kernels are persistent: each CTA walks tiles of 16 rows and keeps
// the next tile's input landing in shared memory (cp.async, two stages)
// while it transforms the current one.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Bounded device waits (the pipelined decomposition's flags, the row tiles'
// bulk copies) record here why they gave up: bit 0 a pipelined-pass wait,
// bit 1 a row-tile copy; shl_sync reads and clears it.
__device__ unsigned int g_pipe_err = 0;
constexpr unsigned WAIT_PIPE = 1u, WAIT_TILE = 2u;
constexpr unsigned TILE_SPIN_LIMIT = 1u << 22;   // try_wait rounds, each suspends briefly

// Row tiles of the R2C passes are contiguous runs of global memory (TR whole
// rows), so one thread moves each with a single bulk copy (TMA,
// cp.async.bulk) that completes on an mbarrier with its byte count, in
// place of per-thread 16-byte cp.async: source and destination 16-byte
// aligned, size a multiple of 16.
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                          unsigned long long* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(b)) : "memory");
}
// true once phase `parity` of the barrier has completed; false after
// TILE_SPIN_LIMIT rounds (the caller records the error and stops).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* b, unsigned parity) {
  const unsigned a = smem_addr(b);
  for (unsigned i = 0; i < TILE_SPIN_LIMIT; ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done) : "r"(a), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

// Copy `bytes` (multiple of 16) from gmem to smem with all threads of the CTA.
__device__ __forceinline__ void cta_copy_async(void* dst, const void* src, int bytes, int tid,
                                               int nthreads) {
  char* d = static_cast<char*>(dst);
  const char* s = static_cast<const char*>(src);
  for (int c = tid * 16; c < bytes; c += nthreads * 16) cp_async16(d + c, s + c);
}

// Split factor exp(-2 pi i p / M), p = j + u T, of the real-row transforms:
// for M = 512 (T = 16 lanes) the lane base w0 = exp(-2 pi i j / 512) times
// the 32nd root exp(-2 pi i u / 32) (u is a constant in the unrolled
// loops); otherwise the staged table.
template <int LOG_M, int T>
__device__ __forceinline__ float2 split_tw(const float2* ptw, const float2* twb, int j, int u) {
  if constexpr (LOG_M == 9 && T == 16) {
    const float2 w0 = twb[4 * T + j];
    switch (u) {
#define SHL_SPLIT(U) case U: return rot32<U, -1>(w0);
      SHL_SPLIT(0) SHL_SPLIT(1) SHL_SPLIT(2) SHL_SPLIT(3) SHL_SPLIT(4) SHL_SPLIT(5) SHL_SPLIT(6)
      SHL_SPLIT(7) SHL_SPLIT(8) SHL_SPLIT(9) SHL_SPLIT(10) SHL_SPLIT(11) SHL_SPLIT(12)
      SHL_SPLIT(13) SHL_SPLIT(14) SHL_SPLIT(15)
#undef SHL_SPLIT
      default: return ptw[j + u * T];
    }
  } else {
    return ptw[j + u * T];
  }
}

template <int LOG_M>
struct RowsT {
  static constexpr int M = 1 << LOG_M;
  static constexpr int L = M / 2;
  static constexpr int R = LineRadix<L>::R;
  using C = LineCfg<L, R>;
  static constexpr int T = C::T;
  static constexpr int TR = M >= 2048 ? 8 : 16;   // rows per tile
  static constexpr int TP = TR + 1;               // padded transpose-tile pitch
  static constexpr int LPC = (TR * T) >= 32 ? TR : 32 / T;  // lines incl. idle ones
  static constexpr int THREADS = LPC * T;
  static constexpr int Mh = L + 1;
  static constexpr int CPITCH = TR + 2;           // c2r input tile pitch (16-byte rows)
  static constexpr int CPITCH16 = TR + 2;         // bfloat16 stage: pitch in bfloat162 words (8-byte rows)
  // the transpose tile reuses the line buffers (separated by __syncthreads)
  static constexpr size_t LINES = (size_t)LPC * C::WORDS, TILE = (size_t)Mh * TP;
  static constexpr size_t WORK = sizeof(float2) * (LINES > TILE ? LINES : TILE);
  static constexpr size_t CSTAGE = sizeof(float2) * (size_t)Mh * CPITCH;
  static constexpr size_t CSTAGE16 = (4 * (size_t)Mh * CPITCH16 + 15) / 16 * 16;
  static constexpr size_t SMEM_CAP = 224 * 1024;
  static constexpr int MINB = M <= 512 ? 2 : 1;    // CTAs per SM the sizes allow
  // twiddles: line stages, split factors exp(-2 pi i p / M), lane bases
  static constexpr size_t TWB = sizeof(float2) * ((size_t)LineTw<L, R>::WORDS + L + LineTwB<L, R>::WORDS);
  static constexpr int CNST = 2 * CSTAGE + WORK + TWB <= SMEM_CAP ? 2 : 1;   // c2r pipeline depth
  static constexpr int CNST16 = 2 * CSTAGE16 + WORK + TWB <= SMEM_CAP ? 2 : 1;
  static_assert(CSTAGE + WORK + TWB <= SMEM_CAP, "c2r tile does not fit shared memory");
};

template <int INM>
struct RowInput {  // bytes of one 16-row input tile per stream
  static constexpr int ESZ = INM == IN_BF16 ? 2 : 4;
};

struct RowsTArgs {
  const void* in;            // [nsub][N][M] reals, or f_masked
  const uint8_t* mask;       // masked mode
  const float* fest;         // masked mode
  const float* thresh;       // [nsub] or null
  float2* out;               // [nsub][Mh][N]
  const float2* tw;
  int N, nsub;
};

template <int LOG_M, int INM>
__host__ __device__ constexpr size_t r2c_stage_bytes() {
  return INM == IN_MASKED ? (size_t)RowsT<LOG_M>::TR * (1 << LOG_M) * (4 + 4 + 1)
                          : (size_t)RowsT<LOG_M>::TR * (1 << LOG_M) * RowInput<INM>::ESZ;
}
// r2c pipeline depth: 2 (double-buffered), 1, or 0 (inputs read straight
// from global memory when even one staged tile does not fit).
// Three CTAs per SM (24 warps) where one staged tile, the work buffers and
// the twiddles fit a third of the SM's shared memory and the input is not
// the masked triple: one stage, refilled as soon as its rows are in
// registers, so the next tile's copy still overlaps the current transform.
template <int LOG_M, int INM>
__host__ __device__ constexpr bool r2c_occ3() {
  using P = RowsT<LOG_M>;
  return INM != IN_MASKED && 3 * (r2c_stage_bytes<LOG_M, INM>() + P::WORK + P::TWB + 1024 + 64) <=
                                 228 * 1024;
}
template <int LOG_M, int INM>
__host__ __device__ constexpr int r2c_nst() {
  using P = RowsT<LOG_M>;
  constexpr size_t SB = r2c_stage_bytes<LOG_M, INM>(), REST = P::WORK + P::TWB;
  if (r2c_occ3<LOG_M, INM>()) return 1;
  return 2 * SB + REST <= P::SMEM_CAP ? 2 : (SB + REST <= P::SMEM_CAP ? 1 : 0);
}
template <int LOG_M, int INM>
__host__ __device__ constexpr int r2c_minb() {
  return r2c_occ3<LOG_M, INM>() ? 3 : RowsT<LOG_M>::MINB;
}

// Thread 0: start the bulk copies of tile t into `stage`, completing on
// `bar` (one arrival carrying their byte count).  The stage's earlier
// readers have passed a CTA barrier.
template <int LOG_M, int INM>
__device__ __forceinline__ void r2c_issue(const RowsTArgs& a, char* stage, int t,
                                          unsigned long long* bar) {
  using P = RowsT<LOG_M>;
  const int tiles_per_sub = a.N / P::TR;
  const int s = t / tiles_per_sub, y0 = (t % tiles_per_sub) * P::TR;
  const size_t row0 = (size_t)s * a.N + y0;
  constexpr int n = P::TR * P::M;
  if (!SHL_IN(row0 + P::TR - 1, (size_t)a.nsub * a.N, CHK_R2C_IN)) {
    mbar_arrive_tx(bar, 0);                  // completes the phase without data
    return;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if constexpr (INM == IN_MASKED) {
    mbar_arrive_tx(bar, n * 9);
    bulk_load(stage, static_cast<const float*>(a.in) + row0 * P::M, n * 4, bar);
    bulk_load(stage + n * 4, a.fest + row0 * P::M, n * 4, bar);
    bulk_load(stage + n * 8, a.mask + row0 * P::M, n, bar);
  } else {
    constexpr int esz = RowInput<INM>::ESZ;
    mbar_arrive_tx(bar, n * esz);
    bulk_load(stage, static_cast<const char*>(a.in) + row0 * P::M * esz, n * esz, bar);
  }
}

// Forward half of a row tile: v[u] = z[j + u T] (two reals packed per
// complex) of row r -> R2C (line FFT and conjugate-pair split) -> the
// transposed tile in shared memory -> out[kx * N + row] for the TR rows.
// Ends with a CTA barrier, after which the line and tile buffers are free.
template <int LOG_M>
__device__ __forceinline__ void r2c_tile_finish(float2 (&v)[RowsT<LOG_M>::R], float2* line,
                                                float2* tile, const float2* twl, const float2* ptw,
                                                float2* out, int N, int r, int j, bool valid,
                                                int tid, bool store_ok = true) {
  using P = RowsT<LOG_M>;
  constexpr int T = P::T, R = P::R, L = P::L, Mh = P::Mh, TR = P::TR, TP = P::TP;
  const float2* twb = ptw + L;                             // lane bases after the split factors
  line_fft_any<L, R, -1>(v, line, j, 1 + r, twl, twb);

  // conjugate-pair split needs Z[L - k]: publish the natural-order line
  group_sync<T>(1 + r);
  line_store<L, R>(v, line, j);
  group_sync<T>(1 + r);
  float2 mir[R];
  line_load_mirror<L, R>(mir, line, j);
  const float2 nyq = make_float2(v[0].x - v[0].y, 0.f);   // X[L], kept by lane j == 0
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const float2 A = v[u], B = mir[u];
    const float2 E = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y - B.y));
    const float2 O = make_float2(0.5f * (A.y + B.y), -0.5f * (A.x - B.x));
    v[u] = cadd(E, cmul(O, split_tw<LOG_M, T>(ptw, twb, j, u)));
  }
  __syncthreads();                       // line buffers become the tile
  if (valid) {
#pragma unroll
    for (int u = 0; u < R; ++u) tile[(j + u * T) * TP + r] = v[u];
    if (j == 0) tile[L * TP + r] = nyq;
  }
  __syncthreads();
  // transposed store: two rows of one kx per 16-byte store
  for (int idx = tid; idx < Mh * (TR / 2); idx += P::THREADS) {
    const int kx = idx / (TR / 2), q = 2 * (idx % (TR / 2));
    const float2 lo = tile[kx * TP + q], hi = tile[kx * TP + q + 1];
    if (store_ok)
      *reinterpret_cast<float4*>(out + (size_t)kx * N + q) = make_float4(lo.x, lo.y, hi.x, hi.y);
  }
  __syncthreads();
}

template <int LOG_M, int INM, bool THRESH>
__global__ void __launch_bounds__(RowsT<LOG_M>::THREADS, (r2c_minb<LOG_M, INM>())) k_rows_r2c_t(RowsTArgs a) {
  using P = RowsT<LOG_M>;
  constexpr int T = P::T, R = P::R, L = P::L, Mh = P::Mh, M = P::M;
  constexpr int TR = P::TR;
  constexpr size_t SB = r2c_stage_bytes<LOG_M, INM>();
  constexpr int NST = r2c_nst<LOG_M, INM>();
  constexpr bool EARLY = r2c_occ3<LOG_M, INM>();   // one stage, refilled after the read
  extern __shared__ __align__(16) float2 smem[];
  char* stages = reinterpret_cast<char*>(smem);
  float2* work = reinterpret_cast<float2*>(stages + (size_t)NST * SB);
  float2* tile = work;
  float2* twl = work + P::WORK / sizeof(float2);          // line-FFT twiddles
  float2* ptw = twl + LineTw<L, R>::WORDS;                 // exp(-2 pi i p / M), p < L
  const int tid = threadIdx.x;
  const int r = tid / T, j = tid % T;
  const bool valid = r < TR;
  float2* line = work + (size_t)r * P::C::WORDS;
  const int tiles_per_sub = a.N / TR;
  const int ntiles = a.nsub * tiles_per_sub;

  __shared__ unsigned long long full[2];   // one mbarrier per stage
  if (tid == 0) {
    mbar_init(&full[0]);
    mbar_init(&full[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  LineTw<L, R>::fill(twl, a.tw, tid, P::THREADS);
  for (int p = tid; p < L; p += P::THREADS) ptw[p] = twiddle<-1>(a.tw, p, LOG_M);
  LineTwB<L, R>::fill(ptw + L, a.tw, tid, P::THREADS);
  __syncthreads();
  if ((NST == 2 || EARLY) && tid == 0 && blockIdx.x < ntiles)
    r2c_issue<LOG_M, INM>(a, stages, blockIdx.x, &full[0]);
  int k = 0;
  int pending = (NST == 2 || EARLY) && blockIdx.x < ntiles ? 1 : 0;   // copies issued, not waited on
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
    if constexpr (EARLY) {
      const bool ok = mbar_wait_bounded(&full[0], k & 1);     // tile k, the stage's k-th use
      --pending;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          atomicOr(&g_pipe_err, WAIT_TILE);
          mbar_wait_bounded(&full[0], k & 1);   // the copy that ran out: let it land
        }
        return;
      }
    } else if constexpr (NST > 0) {
      const int tn = NST == 2 ? t + gridDim.x : t;
      if (tn < ntiles) {
        if (tid == 0) r2c_issue<LOG_M, INM>(a, stages + ((k + 1) % NST) * SB, tn, &full[(k + 1) % NST]);
        ++pending;
      }
      // tile k's copy: stage k % NST, its (k / NST)-th use
      const bool ok = mbar_wait_bounded(&full[k % NST], (k / NST) & 1);
      --pending;
      if (__syncthreads_or(!ok)) {             // the same decision in every thread
        if (tid == 0) {
          atomicOr(&g_pipe_err, WAIT_TILE);
          // a copy still in flight targets the other stage: let it land
          if (pending > 0) mbar_wait_bounded(&full[(k + 1) % NST], ((k + 1) / NST) & 1);
        }
        return;
      }
    } else {
      __syncthreads();
    }
    const int s = t / tiles_per_sub, y0 = (t % tiles_per_sub) * TR;
    // tile input: staged in shared memory, or the global rows themselves
    const char* cur = NST > 0 ? stages + (k % (NST > 0 ? NST : 1)) * SB : nullptr;
    const size_t grow0 = ((size_t)s * a.N + y0) * M;
    constexpr int n = TR * M;
    const float2* src_f = NST > 0 ? reinterpret_cast<const float2*>(cur)
                                  : reinterpret_cast<const float2*>(static_cast<const float*>(a.in) + grow0);
    const __nv_bfloat162* src_h = NST > 0 ? reinterpret_cast<const __nv_bfloat162*>(cur)
                                          : reinterpret_cast<const __nv_bfloat162*>(
                                                static_cast<const __nv_bfloat16*>(a.in) + grow0);
    const float2* src_e = NST > 0 ? reinterpret_cast<const float2*>(cur + n * 4)
                                  : reinterpret_cast<const float2*>(a.fest ? a.fest + grow0 : nullptr);
    const uchar2* src_m = NST > 0 ? reinterpret_cast<const uchar2*>(cur + n * 8)
                                  : reinterpret_cast<const uchar2*>(a.mask ? a.mask + grow0 : nullptr);
    float tau = 0.f;
    if (THRESH) tau = SHL_IN(s, a.nsub, CHK_R2C_IN) ? __ldg(a.thresh + s) : 0.f;
    const int rr = valid ? r : 0;
    const bool tile_ok = SHL_IN((size_t)s * a.N + y0 + TR - 1, (size_t)a.nsub * a.N, CHK_R2C_OUT);

    float2 v[R];
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int p = j + u * T;
      float2 z;
      if constexpr (INM == IN_F32) {
        z = src_f[rr * (M / 2) + p];
      } else if constexpr (INM == IN_BF16) {
        z = __bfloat1622float2(src_h[rr * (M / 2) + p]);
      } else {
        const float2 fm = src_f[rr * (M / 2) + p];
        const float2 fe = src_e[rr * (M / 2) + p];
        const uchar2 mk = src_m[rr * (M / 2) + p];
        z.x = mk.x ? fm.x : fe.x;   // mask (f_masked - f_est) + f_est, mask in {0, 1}
        z.y = mk.y ? fm.y : fe.y;
      }
      if (THRESH) {
        if (fabsf(z.x) < tau) z.x = 0.f;
        if (fabsf(z.y) < tau) z.y = 0.f;
      }
      v[u] = valid ? z : make_float2(0.f, 0.f);
    }
    if constexpr (EARLY) {
      // the stage is in registers: refill it with the next tile now
      __syncthreads();
      const int tn = t + gridDim.x;
      if (tn < ntiles) {
        if (tid == 0) r2c_issue<LOG_M, INM>(a, stages, tn, &full[0]);
        ++pending;
      }
    }

    r2c_tile_finish<LOG_M>(v, line, tile, twl, ptw, a.out + (size_t)s * Mh * a.N + y0, a.N, r, j,
                           valid, tid, tile_ok);    // ends with a barrier: tile and stage reusable
  }
}

struct RowsTC2RArgs {
  const void* in;            // [nsub][Mh][N] float2, or bfloat162 (bfloat16 staging)
  void* out;                 // [nsub][N][M]
  const float2* tw;
  int N, nsub;
};

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gmem_src) : "memory");
}

// Stage tile t's TR rows of every kx: 16-byte (float2 staging) or 8-byte
// (bfloat16 staging, S16) chunks of two rows.
template <int LOG_M, bool S16 = false>
__device__ __forceinline__ void c2r_issue(const RowsTC2RArgs& a, float2* stage, int t, int tid) {
  using P = RowsT<LOG_M>;
  const int tiles_per_sub = a.N / P::TR;
  const int s = t / tiles_per_sub, y0 = (t % tiles_per_sub) * P::TR;
  constexpr int CH = P::TR / 2;                       // two-row chunks per kx row
  if (!SHL_IN((size_t)s * a.N + y0 + P::TR - 1, (size_t)a.nsub * a.N, CHK_C2R_IN)) return;
  if constexpr (S16) {
    const __nv_bfloat162* in =
        static_cast<const __nv_bfloat162*>(a.in) + (size_t)s * P::Mh * a.N + y0;
    __nv_bfloat162* st = reinterpret_cast<__nv_bfloat162*>(stage);
    for (int c = tid; c < P::Mh * CH; c += P::THREADS) {
      const int kx = c / CH, q = c % CH;
      cp_async8(st + kx * P::CPITCH16 + 2 * q, in + (size_t)kx * a.N + 2 * q);
    }
  } else {
    const float2* in = static_cast<const float2*>(a.in) + (size_t)s * P::Mh * a.N + y0;
    for (int c = tid; c < P::Mh * CH; c += P::THREADS) {
      const int kx = c / CH, q = c % CH;
      cp_async16(stage + kx * P::CPITCH + 2 * q, in + (size_t)kx * a.N + 2 * q);
    }
  }
}

// C2R of one TR-row tile staged as tile[kx * CPITCH + row]: on return v[u]
// holds (x[2p], x[2p+1]), p = j + u T, of row r of the tile (lanes j of
// group r); unnormalised (the 1/(N M) sits in the filter or weight factors).
// The split of row r of the staged tile (reads the stage, leaves v[u] =
// Z[j + u T] of the line before its inverse FFT).
template <int LOG_M, bool S16 = false>
__device__ __forceinline__ void c2r_tile_load(const float2* tile, const float2* ptw, int r,
                                              int j, bool valid, float2 (&v)[RowsT<LOG_M>::R]) {
  using P = RowsT<LOG_M>;
  constexpr int T = P::T, R = P::R, L = P::L, CP = S16 ? P::CPITCH16 : P::CPITCH;
  const int rr = valid ? r : 0;
  auto at = [&](int i) -> float2 {
    if constexpr (S16) return __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(tile)[i]);
    else return tile[i];
  };
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int kk = j + u * T;
    const float2 A = at(kk * CP + rr);
    const float2 B = at((L - kk) * CP + rr);
    const float2 S = make_float2(A.x + B.x, A.y - B.y);
    const float2 D = make_float2(A.x - B.x, A.y + B.y);
    const float2 wd = cmulc(D, split_tw<LOG_M, T>(ptw, ptw + L, j, u));   // D * exp(+2 pi i k / M)
    v[u] = valid ? make_float2(S.x - wd.y, S.y + wd.x) : make_float2(0.f, 0.f);
  }
}

template <int LOG_M, bool S16 = false>
__device__ __forceinline__ void c2r_tile_compute(const float2* tile, float2* line,
                                                 const float2* twl, const float2* ptw, int r,
                                                 int j, bool valid,
                                                 float2 (&v)[RowsT<LOG_M>::R]) {
  using P = RowsT<LOG_M>;
  c2r_tile_load<LOG_M, S16>(tile, ptw, r, j, valid, v);
  line_fft_any<P::L, P::R, +1>(v, line, j, 1 + r, twl, ptw + P::L);
}

// Row r of the inverse FFT's output v to out + base (float32 or bfloat16).
template <int LOG_M, bool BF16OUT>
__device__ __forceinline__ void c2r_store_row(const float2 (&v)[RowsT<LOG_M>::R], void* out,
                                              size_t base, int j) {
  using P = RowsT<LOG_M>;
#pragma unroll
  for (int u = 0; u < P::R; ++u) {
    const int p = j + u * P::T;
    if constexpr (BF16OUT) {
      __nv_bfloat162 h = __floats2bfloat162_rn(v[u].x, v[u].y);
      __stcs(reinterpret_cast<unsigned int*>(static_cast<__nv_bfloat16*>(out) + base + 2 * p),
             *reinterpret_cast<unsigned int*>(&h));
    } else {
      __stcs(reinterpret_cast<float2*>(static_cast<float*>(out) + base + 2 * p), v[u]);
    }
  }
}

// C2R of one staged tile and the store of row r to out + base.
template <int LOG_M, bool BF16OUT, bool S16 = false>
__device__ __forceinline__ void c2r_tile_body(const float2* tile, float2* line,
                                              const float2* twl, const float2* ptw, void* out,
                                              size_t base, int r, int j, bool valid) {
  using P = RowsT<LOG_M>;
  constexpr int T = P::T, R = P::R;
  float2 v[R];
  c2r_tile_compute<LOG_M, S16>(tile, line, twl, ptw, r, j, valid, v);
  if (valid) {
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int p = j + u * T;
      if constexpr (BF16OUT) {
        __nv_bfloat162 h = __floats2bfloat162_rn(v[u].x, v[u].y);
        __stcs(reinterpret_cast<unsigned int*>(static_cast<__nv_bfloat16*>(out) + base + 2 * p),
               *reinterpret_cast<unsigned int*>(&h));
      } else {
        __stcs(reinterpret_cast<float2*>(static_cast<float*>(out) + base + 2 * p), v[u]);
      }
    }
  }
}

// S16: the staged half spectra are bfloat16 (the bfloat16 decomposition).
// Three CTAs per SM where one staged tile, the work buffers and the
// twiddles fit a third of the SM's shared memory: one stage, refilled once
// the tile's split has read it (c2r_t sizes the launch accordingly).
template <int LOG_M, bool S16>
__host__ __device__ constexpr bool c2r_occ3() {
  using P = RowsT<LOG_M>;
  return 3 * ((S16 ? P::CSTAGE16 : P::CSTAGE) + P::WORK + P::TWB + 1024) <= 228 * 1024;
}
template <int LOG_M, bool S16>
__host__ __device__ constexpr int c2r_nst() {
  using P = RowsT<LOG_M>;
  return c2r_occ3<LOG_M, S16>() ? 1 : (S16 ? P::CNST16 : P::CNST);
}

template <int LOG_M, bool BF16OUT, bool S16>
__global__ void __launch_bounds__(RowsT<LOG_M>::THREADS, (c2r_occ3<LOG_M, S16>() ? 3 : RowsT<LOG_M>::MINB))
    k_rows_c2r_t(RowsTC2RArgs a) {
  using P = RowsT<LOG_M>;
  constexpr int T = P::T, R = P::R, L = P::L, TR = P::TR, NST = c2r_nst<LOG_M, S16>();
  constexpr bool EARLY = c2r_occ3<LOG_M, S16>();
  constexpr size_t SW = (S16 ? P::CSTAGE16 : P::CSTAGE) / sizeof(float2);
  extern __shared__ __align__(16) float2 smem[];
  float2* stages = smem;
  float2* work = smem + NST * SW;
  float2* twl = work + P::WORK / sizeof(float2);
  float2* ptw = twl + LineTw<L, R>::WORDS;
  const int tid = threadIdx.x;
  const int r = tid / T, j = tid % T;
  const bool valid = r < TR;
  const int rr = valid ? r : 0;
  float2* line = work + (size_t)r * P::C::WORDS;
  const int tiles_per_sub = a.N / TR;
  const int ntiles = a.nsub * tiles_per_sub;

  LineTw<L, R>::fill(twl, a.tw, tid, P::THREADS);
  for (int p = tid; p < L; p += P::THREADS) ptw[p] = twiddle<-1>(a.tw, p, LOG_M);
  LineTwB<L, R>::fill(ptw + L, a.tw, tid, P::THREADS);
  if ((NST == 2 || EARLY) && blockIdx.x < ntiles) c2r_issue<LOG_M, S16>(a, stages, blockIdx.x, tid);
  cp_async_commit();
  int k = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
    if constexpr (EARLY) {
      cp_async_wait0();
      __syncthreads();
      const int s = t / tiles_per_sub, y0 = (t % tiles_per_sub) * TR;
      float2 v[R];
      c2r_tile_load<LOG_M, S16>(stages, ptw, r, j, valid, v);
      __syncthreads();                     // the stage is read: refill it with the next tile
      if (t + (int)gridDim.x < ntiles) c2r_issue<LOG_M, S16>(a, stages, t + gridDim.x, tid);
      cp_async_commit();
      line_fft_any<L, R, +1>(v, line, j, 1 + r, twl, ptw + L);
      if (valid && SHL_IN((size_t)s * a.N + y0 + rr, (size_t)a.nsub * a.N, CHK_C2R_OUT))
        c2r_store_row<LOG_M, BF16OUT>(v, a.out, ((size_t)s * a.N + y0 + rr) * P::M, j);
      continue;
    }
    const int tn = NST == 2 ? t + gridDim.x : t;
    if (tn < ntiles) c2r_issue<LOG_M, S16>(a, stages + ((k + 1) % NST) * SW, tn, tid);
    cp_async_commit();
    if (NST == 2) cp_async_wait1(); else cp_async_wait0();
    __syncthreads();
    const float2* tile = stages + (k % NST) * SW;
    const int s = t / tiles_per_sub, y0 = (t % tiles_per_sub) * TR;

    c2r_tile_body<LOG_M, BF16OUT, S16>(tile, line, twl, ptw, a.out,
                                       ((size_t)s * a.N + y0 + rr) * P::M, r, j,
                                       valid && SHL_IN((size_t)s * a.N + y0 + rr,
                                                       (size_t)a.nsub * a.N, CHK_C2R_OUT));
    __syncthreads();                       // stage reuse
  }
  cp_async_wait0();
}

// Row pass of the fused denoise / IHT step, in place on the staged half
// spectra of the chunk: each TR-row tile is C2R'd to its coefficient rows in
// registers, hard-thresholded (T_delta of Sec. 4.2: zero |c| < thresh[s],
// ties kept, the same float32 compare as the threshold-on-read R2C), and
// R2C'd back to the same place.  The coefficients never reach memory.
struct RowsShrinkArgs {
  float2* z;                 // [nsub][Mh][N], read and rewritten
  const float* thresh;       // [nsub]
  const float2* tw;
  int N, nsub;
};

template <int LOG_M>
__global__ void __launch_bounds__(RowsT<LOG_M>::THREADS, RowsT<LOG_M>::MINB)
k_rows_shrink_t(RowsShrinkArgs a) {
  using P = RowsT<LOG_M>;
  constexpr int T = P::T, R = P::R, L = P::L, Mh = P::Mh, TR = P::TR, NST = P::CNST;
  extern __shared__ __align__(16) float2 smem[];
  float2* stages = smem;
  float2* work = smem + NST * (P::CSTAGE / sizeof(float2));
  float2* twl = work + P::WORK / sizeof(float2);
  float2* ptw = twl + LineTw<L, R>::WORDS;
  const int tid = threadIdx.x;
  const int r = tid / T, j = tid % T;
  const bool valid = r < TR;
  float2* line = work + (size_t)r * P::C::WORDS;
  const int tiles_per_sub = a.N / TR;
  const int ntiles = a.nsub * tiles_per_sub;
  constexpr size_t SW = P::CSTAGE / sizeof(float2);
  const RowsTC2RArgs ca{a.z, nullptr, a.tw, a.N, a.nsub};

  LineTw<L, R>::fill(twl, a.tw, tid, P::THREADS);
  for (int p = tid; p < L; p += P::THREADS) ptw[p] = twiddle<-1>(a.tw, p, LOG_M);
  LineTwB<L, R>::fill(ptw + L, a.tw, tid, P::THREADS);
  if (NST == 2 && blockIdx.x < ntiles) c2r_issue<LOG_M>(ca, stages, blockIdx.x, tid);
  cp_async_commit();
  int k = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
    const int tn = NST == 2 ? t + gridDim.x : t;
    if (tn < ntiles) c2r_issue<LOG_M>(ca, stages + ((k + 1) % NST) * SW, tn, tid);
    cp_async_commit();
    if (NST == 2) cp_async_wait1(); else cp_async_wait0();
    __syncthreads();
    const int s = t / tiles_per_sub, y0 = (t % tiles_per_sub) * TR;
    float2 v[R];
    c2r_tile_compute<LOG_M>(stages + (k % NST) * SW, line, twl, ptw, r, j, valid, v);
    const float tau = SHL_IN(s, a.nsub, CHK_SHRINK) ? __ldg(a.thresh + s) : 0.f;
#pragma unroll
    for (int u = 0; u < R; ++u) {
      if (fabsf(v[u].x) < tau) v[u].x = 0.f;
      if (fabsf(v[u].y) < tau) v[u].y = 0.f;
    }
    // the forward line FFT reuses the group's own line buffer after a group
    // sync; the CTA-wide tile reuse is fenced inside r2c_tile_finish
    r2c_tile_finish<LOG_M>(v, line, work, twl, ptw, a.z + (size_t)s * Mh * a.N + y0, a.N, r, j,
                           valid, tid);    // ends with a barrier: tile and stage reusable
  }
  cp_async_wait0();
}

// ----------------------------------------------------------------- lines
// (Radix 32 for the 512-point column lines, one shared-memory exchange
// instead of two, measured slower at 512 x 512: 0.554 / 0.662 ms against
// 0.534 / 0.571 ms for decomposition / reconstruction of 16 images; the
// extra registers leave one CTA per SM.)
template <int LOG_N>
struct LinesT {
  static constexpr int N = 1 << LOG_N;
  static constexpr int R = LineRadix<N>::R;
  using C = LineCfg<N, R>;
  static constexpr int T = C::T;
  static constexpr int THREADS = 256;
  static constexpr int NG = THREADS / T;              // lane groups per CTA
  static constexpr size_t SMEM_LINES = sizeof(float2) * (size_t)NG * C::WORDS;
  static constexpr size_t TWB = sizeof(float2) * ((size_t)LineTw<N, R>::WORDS + LineTwB<N, R>::WORDS);
};

struct LinesArgs {
  float2* data;              // FWD: [nlines][N] in place; DEC: image spectra [B][Mh][N]
  void* out;                 // DEC: staging [S][Mh][N], float2 (or bfloat162 with s16)
  const float* G;            // [K][Mh][N]
  const float* invW;         // [Mh][N] or null
  const float2* tw;
  float scale;
  int Mh, K, s0, nlines;
  int nimg;                  // image planes of data (checked build)
  int s16;                   // DEC: bfloat16 staging (the bfloat16 decomposition)
};

template <int LOG_N>
__global__ void __launch_bounds__(256) k_lines_fwd(LinesArgs a) {
  using P = LinesT<LOG_N>;
  constexpr int T = P::T, R = P::R, N = P::N;
  extern __shared__ float2 smem[];
  const int g = threadIdx.x / T, j = threadIdx.x % T;
  float2* line = smem + (size_t)g * P::C::WORDS;
  float2* twl = smem + (size_t)P::NG * P::C::WORDS;
  float2* twb = twl + LineTw<N, R>::WORDS;
  LineTw<N, R>::fill(twl, a.tw, threadIdx.x, P::THREADS);
  LineTwB<N, R>::fill(twb, a.tw, threadIdx.x, P::THREADS);
  __syncthreads();
  for (int q = blockIdx.x * P::NG + g; q < a.nlines; q += gridDim.x * P::NG) {
    if (!SHL_IN(q, a.nlines, CHK_LINES)) break;
    float2* d = a.data + (size_t)q * N;
    float2 v[R];
#pragma unroll
    for (int u = 0; u < R; ++u) v[u] = d[j + u * T];
    line_fft_any<N, R, -1>(v, line, j, 1 + g, twl, twb);
#pragma unroll
    for (int u = 0; u < R; ++u) d[j + u * T] = v[u];
  }
}

// One lane group handles one kx line for DEC_FPG consecutive subbands of the
// chunk: the image-spectrum line is loaded once per image and the next
// filter's G line is fetched before the current FFT.
constexpr int DEC_FPG = 4;

// One lane group: kx line `kx` of the chunk subbands sl0..sl1-1 (global
// subband s0 + sl, image s / K, filter s mod K) into out[sl][kx][:].
template <int LOG_N, bool S16 = false>
__device__ __forceinline__ void dec_group(const float2* X, void* out, const float* Gall,
                                          const float* invW, float scale, int Mh, int K, int s0,
                                          int sl0, int sl1, int kx, float2* line, const float2* twl,
                                          int j, int g, int nimg = 0x7fffffff,
                                          int nstage = 0x7fffffff) {
  using P = LinesT<LOG_N>;
  constexpr int T = P::T, R = P::R, N = P::N;
  const float* W = invW ? invW + (size_t)kx * N : nullptr;
  float2 Xl[R];
  float gn[R];
  int b_loaded = -1;
  {
    const int s = s0 + sl0, b = s / K, i = s - b * K;
    const float* G = Gall + ((size_t)i * Mh + kx) * N;
    const bool ok = SHL_IN((size_t)i * Mh + kx, (size_t)K * Mh, CHK_DEC_G);
#pragma unroll
    for (int u = 0; u < R; ++u) gn[u] = ok ? __ldg(G + j + u * T) : 0.f;
  }
  for (int sl = sl0; sl < sl1; ++sl) {
    const int s = s0 + sl, b = s / K;
    if (b != b_loaded) {                              // image spectrum line, once per image
      const float2* Xp = X + ((size_t)b * Mh + kx) * N;
      const bool ok = SHL_IN((size_t)b * Mh + kx, (size_t)nimg * Mh, CHK_DEC_X);
#pragma unroll
      for (int u = 0; u < R; ++u) Xl[u] = ok ? Xp[j + u * T] : make_float2(0.f, 0.f);
      b_loaded = b;
    }
    float gc[R];
#pragma unroll
    for (int u = 0; u < R; ++u) gc[u] = gn[u];
    if (sl + 1 < sl1) {                               // prefetch the next filter's line
      const int s2 = s + 1, i2 = s2 - (s2 / K) * K;
      const float* G2 = Gall + ((size_t)i2 * Mh + kx) * N;
      const bool ok = SHL_IN((size_t)i2 * Mh + kx, (size_t)K * Mh, CHK_DEC_G);
#pragma unroll
      for (int u = 0; u < R; ++u) gn[u] = ok ? __ldg(G2 + j + u * T) : 0.f;
    }
    float2 v[R];
#pragma unroll
    for (int u = 0; u < R; ++u) {
      float gv = gc[u] * scale;
      if (W) gv *= __ldg(W + j + u * T);
      v[u] = cscale(Xl[u], gv);
    }
    line_fft_any<N, R, +1>(v, line, j, 1 + g, twl, twl + LineTw<N, R>::WORDS);
    if (SHL_IN((size_t)sl * Mh + kx, (size_t)nstage * Mh, CHK_DEC_OUT)) {
      if constexpr (S16) {
        __nv_bfloat162* o = static_cast<__nv_bfloat162*>(out) + ((size_t)sl * Mh + kx) * N;
#pragma unroll
        for (int u = 0; u < R; ++u) o[j + u * T] = __floats2bfloat162_rn(v[u].x, v[u].y);
      } else {
        float2* o = static_cast<float2*>(out) + ((size_t)sl * Mh + kx) * N;
#pragma unroll
        for (int u = 0; u < R; ++u) o[j + u * T] = v[u];
      }
    }
  }
}

template <int LOG_N, bool S16>
__global__ void __launch_bounds__(256) k_dec_lines(LinesArgs a) {
  using P = LinesT<LOG_N>;
  constexpr int T = P::T, R = P::R, N = P::N;
  extern __shared__ float2 smem[];
  const int g = threadIdx.x / T, j = threadIdx.x % T;
  float2* line = smem + (size_t)g * P::C::WORDS;
  float2* twl = smem + (size_t)P::NG * P::C::WORDS;
  LineTw<N, R>::fill(twl, a.tw, threadIdx.x, P::THREADS);
  LineTwB<N, R>::fill(twl + LineTw<N, R>::WORDS, a.tw, threadIdx.x, P::THREADS);
  __syncthreads();
  const int S = a.nlines / a.Mh;                        // subbands in the chunk
  const int ngroups = (S + DEC_FPG - 1) / DEC_FPG;
  const int items = ngroups * a.Mh;
  for (int q = blockIdx.x * P::NG + g; q < items; q += gridDim.x * P::NG) {
    const int m = q / a.Mh, kx = q - m * a.Mh;
    const int sl0 = m * DEC_FPG, sl1 = min(S, sl0 + DEC_FPG);
    dec_group<LOG_N, S16>(a.data, a.out, a.G, a.invW, a.scale, a.Mh, a.K, a.s0, sl0, sl1, kx, line,
                          twl, j, g, a.nimg, S);
  }
}

struct RecLinesArgs {
  const float2* stage;       // [Sc][Mh][N] row spectra of the chunk's subbands
  float2* acc;               // [B][Mh][N] partial sums, then the image lines
  const float* G;            // [K][Mh][N]
  const float* invW;         // [Mh][N] or null (adjoint)
  const float2* tw;
  float scale;
  int Mh, K, s0, Sc, b_lo;
  int nimg;                  // image planes of acc (checked build)
};

template <int LOG_N>
__global__ void __launch_bounds__(256, LinesT<LOG_N>::R >= 32 ? 1 : 2) k_rec_lines(RecLinesArgs a) {
  using P = LinesT<LOG_N>;
  constexpr int T = P::T, R = P::R, N = P::N, NG = P::NG;
  extern __shared__ float2 smem[];
  float2* red = smem + (size_t)NG * P::C::WORDS;     // [NG][N] partial sums
  float2* twl = red + (size_t)NG * N;
  const int g = threadIdx.x / T, j = threadIdx.x % T;
  float2* line = smem + (size_t)g * P::C::WORDS;
  float2* twb = twl + LineTw<N, R>::WORDS;
  LineTw<N, R>::fill(twl, a.tw, threadIdx.x, P::THREADS);
  LineTwB<N, R>::fill(twb, a.tw, threadIdx.x, P::THREADS);
  __syncthreads();
  const int kx = blockIdx.x;
  const int b = a.b_lo + blockIdx.y;
  const int s_begin = max(a.s0, b * a.K), s_end = min(a.s0 + a.Sc, (b + 1) * a.K);
  const bool first = s_begin == b * a.K, last = s_end == (b + 1) * a.K;

  float2 acc[R];
#pragma unroll
  for (int u = 0; u < R; ++u) acc[u] = make_float2(0.f, 0.f);
  // Each group's row of `red` (free until the reduction below) holds the
  // next staged line, fetched with cp.async while the current one is
  // transformed.
  float2* pre = red + (size_t)g * N;
  auto fetch = [&](int s) {
    const float2* U = a.stage + ((size_t)(s - a.s0) * a.Mh + kx) * N;
    if (!SHL_IN((size_t)(s - a.s0) * a.Mh + kx, (size_t)a.Sc * a.Mh, CHK_REC_STAGE)) return;
    for (int c = j; c < N / 2; c += T) cp_async16(pre + 2 * c, U + 2 * c);
  };
  if (s_begin + g < s_end) fetch(s_begin + g);
  cp_async_commit();
  for (int s = s_begin + g; s < s_end; s += NG) {
    const float* G = a.G + ((size_t)(s - b * a.K) * a.Mh + kx) * N;
    const bool gok = SHL_IN((size_t)(s - b * a.K) * a.Mh + kx, (size_t)a.K * a.Mh, CHK_REC_G);
    cp_async_wait0();                       // this lane's copies of line s
    group_sync<T>(1 + g);                   // ... and the whole group's
    float2 v[R];
#pragma unroll
    for (int u = 0; u < R; ++u) v[u] = pre[j + u * T];
    group_sync<T>(1 + g);                   // line read before it is overwritten
    if (s + NG < s_end) fetch(s + NG);
    cp_async_commit();
    line_fft_any<N, R, -1>(v, line, j, 1 + g, twl, twb);
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const float gv = gok ? __ldg(G + j + u * T) : 0.f;
      acc[u].x = fmaf(gv, v[u].x, acc[u].x);
      acc[u].y = fmaf(gv, v[u].y, acc[u].y);
    }
  }
  cp_async_wait0();
  group_sync<T>(1 + g);                     // no copy into this row is pending
#pragma unroll
  for (int u = 0; u < R; ++u) red[(size_t)g * N + j + u * T] = acc[u];
  __syncthreads();
  float2* A = a.acc + ((size_t)b * a.Mh + kx) * N;
  if (!SHL_IN((size_t)b * a.Mh + kx, (size_t)a.nimg * a.Mh, CHK_REC_ACC)) A = red + (size_t)(NG - 1) * N;
  for (int p = threadIdx.x; p < N; p += P::THREADS) {
    float2 sum = red[p];
    for (int q = 1; q < NG; ++q) sum = cadd(sum, red[(size_t)q * N + p]);
    if (!first) sum = cadd(A[p], sum);
    if (!last) {
      A[p] = sum;
    } else {
      float sc = a.scale;
      if (a.invW) sc *= __ldg(a.invW + (size_t)kx * N + p);
      red[p] = cscale(sum, sc);
    }
  }
  if (!last) return;
  __syncthreads();
  if (g == 0) {
    float2 v[R];
#pragma unroll
    for (int u = 0; u < R; ++u) v[u] = red[j + u * T];
    line_fft_any<N, R, +1>(v, line, j, 1, twl, twb);
#pragma unroll
    for (int u = 0; u < R; ++u) A[j + u * T] = v[u];
  }
}

// ------------------------------------------------- pipelined decomposition
// k_dec_pipe runs both passes of the decomposition in one cooperative,
// persistent launch.  The subbands are cut into chunks of CS; chunk c is
// staged in ring slot c mod NS (NS * CS planes, 25 MB at 512 x 512 with the
// defaults), which stays in L2 while the coefficients stream out with
// evict-first stores: the staging round trip costs L2, not DRAM, bandwidth.
// Each CTA has one role:
//   COL CTAs claim COL items in chunk order: DEC_FPG subbands x NG kx lines
//     of a chunk (filter multiply and inverse column FFT, dec_group) into
//     the chunk's ring slot, after the ROW tiles of the chunk that used the
//     slot NS chunks earlier are done;
//   ROW CTAs claim TR-row tiles in subband order (C2R rows, c2r_tile_body)
//     with a two-stage cp.async pipeline: the next tile is fetched while the
//     current one is transformed, as soon as every COL item of its chunk is
//     done.
// The CTAs of both roles share the SMs, so the column pass's arithmetic and
// the row pass's memory traffic overlap.  The dependencies run from lower to
// higher chunks only (ROW c after COL c, COL c after ROW c - NS), items are
// claimed in chunk order, and the cooperative launch keeps every CTA
// resident, so every wait ends.  Each wait is also bounded: when it runs
// out the CTA sets g_pipe_err, and every CTA leaves at its next claim.
constexpr unsigned PIPE_SPIN_LIMIT = 1u << 21;   // ~0.3-1 s with the back-off below

struct DecPipeArgs {
  const float2* X;           // image spectra [B][Mh][N]
  float2* ring;              // [NS][CS][Mh][N]
  void* out;                 // coefficients [total][N][M]
  const float* G;            // [K][Mh][N]
  const float* invW;         // [Mh][N] or null
  const float2* tw;
  unsigned* ctl;             // [0] COL claims, [1] ROW claims, [4 + c] COL done, [4 + nchunks + c] ROW done
  float scale;
  int Mh, K, total, CS, NS, nchunks, ncol_ctas;
  unsigned stall;            // 0; 1 makes every ROW wait unsatisfiable (tests the bounded wait)
};

template <int LOG_N, int LOG_M>
struct DecPipeT {
  using RP = RowsT<LOG_M>;
  static constexpr int N = 1 << LOG_N;
  static constexpr int THREADS = RP::THREADS;
  static constexpr int RL = LinesT<LOG_N>::R;
  using CL = LineCfg<N, RL>;
  static constexpr int TL = CL::T;
  static constexpr int NG = THREADS / TL;          // column lines per COL item
  static_assert(NG >= 1 && THREADS % TL == 0, "column line groups must tile the CTA");
  static constexpr int TPS = N / RP::TR;           // row tiles per subband
  // two CTAs per SM where the registers of both passes allow it
  static constexpr int MINB = (THREADS >= 512 || LOG_N >= 10) ? 1 : 2;
  // shared memory, float2 words: the role's twiddles, then its buffers
  // (ROW: two C2R stages + row line buffers; COL: column line buffers)
  static constexpr size_t TWR = (size_t)LineTw<RP::L, RP::R>::WORDS + RP::L + LineTwB<RP::L, RP::R>::WORDS;
  static constexpr size_t TWL = (size_t)LineTw<N, RL>::WORDS + LineTwB<N, RL>::WORDS;
  static constexpr size_t TW = TWR > TWL ? TWR : TWL;
  static constexpr size_t STW = RP::CSTAGE / sizeof(float2);
  static constexpr size_t ROWW = 2 * STW + (size_t)RP::LPC * RP::C::WORDS;
  static constexpr size_t COLW = (size_t)NG * CL::WORDS;
  static constexpr size_t SMEM = sizeof(float2) * (TW + (ROWW > COLW ? ROWW : COLW));
  static_assert(SMEM <= 227 * 1024, "pipelined decomposition does not fit shared memory");
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0: wait until *flag >= target.  false = gave up (error recorded).
__device__ __noinline__ bool pipe_wait(const unsigned* flag, unsigned target) {
  for (unsigned spin = 0;; ++spin) {
    if (ld_acquire_u32(flag) >= target) return true;
    if (*(volatile unsigned*)&g_pipe_err) return false;
    if (spin >= PIPE_SPIN_LIMIT) {
      atomicOr(&g_pipe_err, WAIT_PIPE);
      return false;
    }
    if (spin > 32) __nanosleep(128);
  }
}

// Thread 0, after the CTA's barrier: publish one finished item.
__device__ __forceinline__ void pipe_signal(unsigned* flag) {
  __threadfence();
  atomicAdd(flag, 1u);
}

// Issue the cp.async copies of ROW tile t (subband-major over the batch)
// from its ring slot into a C2R stage.
template <int LOG_N, int LOG_M>
__device__ __forceinline__ void pipe_row_issue(const DecPipeArgs& a, float2* stage, int t, int tid) {
  using P = DecPipeT<LOG_N, LOG_M>;
  using RP = typename P::RP;
  constexpr int N = P::N, TR = RP::TR, Mh = RP::Mh, CH = TR / 2;   // 16-byte chunks per kx row
  const int sub = t / P::TPS, y0 = (t - sub * P::TPS) * TR;
  const int c = sub / a.CS, sl = sub - c * a.CS;
  const float2* in = a.ring + ((size_t)(c % a.NS) * a.CS + sl) * ((size_t)Mh * N) + y0;
  for (int q = tid; q < Mh * CH; q += P::THREADS) {
    const int kx = q / CH, h = q - kx * CH;
    cp_async16(stage + kx * RP::CPITCH + 2 * h, in + (size_t)kx * N + 2 * h);
  }
  cp_async_commit();
}

template <int LOG_N, int LOG_M, bool BF16OUT>
__global__ void __launch_bounds__(DecPipeT<LOG_N, LOG_M>::THREADS, DecPipeT<LOG_N, LOG_M>::MINB)
k_dec_pipe(DecPipeArgs a) {
  using P = DecPipeT<LOG_N, LOG_M>;
  using RP = typename P::RP;
  constexpr int N = P::N, NG = P::NG, TL = P::TL, RL = P::RL;
  constexpr int TR = RP::TR, TRow = RP::T, L = RP::L, Mh = RP::Mh, M = RP::M;
  extern __shared__ __align__(16) float2 smem[];
  float2* tws = smem;                                  // the role's twiddles
  float2* area = smem + P::TW;
  __shared__ int s_item, s_next, s_ok, s_rdy;
  const int tid = threadIdx.x;
  const int NCB = (Mh + NG - 1) / NG;
  const int NCOL = ((a.CS + DEC_FPG - 1) / DEC_FPG) * NCB;   // COL items per chunk
  unsigned* col_done = a.ctl + 4;
  unsigned* row_done = a.ctl + 4 + a.nchunks;
  const size_t plane = (size_t)Mh * N;

  if ((int)blockIdx.x < a.ncol_ctas) {
    // ------------------------------------------------------------ COL role
    LineTw<N, RL>::fill(tws, a.tw, tid, P::THREADS);
    LineTwB<N, RL>::fill(tws + LineTw<N, RL>::WORDS, a.tw, tid, P::THREADS);
    const int items = a.nchunks * NCOL;
    const int g = tid / TL, j = tid % TL;
    unsigned ahead = tid == 0 ? atomicAdd(a.ctl + 0, 1u) : 0u;   // one claim ahead
    for (;;) {
      __syncthreads();                                 // twiddles ready / item done
      if (tid == 0) {
        int it = *(volatile unsigned*)&g_pipe_err ? -1 : (int)ahead;
        int ok = 1;
        if (it >= 0 && it < items) {
          ahead = atomicAdd(a.ctl + 0, 1u);
          const int c = it / NCOL;
          if (c >= a.NS) {
            const int cp = c - a.NS;
            ok = pipe_wait(row_done + cp, (unsigned)(min(a.CS, a.total - cp * a.CS) * P::TPS));
          }
        }
        s_item = it;
        s_ok = ok;
      }
      __syncthreads();
      const int it = s_item;
      if (it < 0 || it >= items || !s_ok) break;
      const int c = it / NCOL, o = it - c * NCOL;
      const int Sc = min(a.CS, a.total - c * a.CS);
      const int m = o / NCB, kb = o - m * NCB;
      const int sl0 = m * DEC_FPG, sl1 = min(Sc, sl0 + DEC_FPG);
      const int kx = kb * NG + g;
      if (kx < Mh && sl0 < sl1)
        dec_group<LOG_N>(a.X, a.ring + (size_t)(c % a.NS) * a.CS * plane, a.G, a.invW, a.scale,
                         Mh, a.K, c * a.CS, sl0, sl1, kx, area + (size_t)g * P::CL::WORDS, tws, j, g);
      __syncthreads();
      if (tid == 0) pipe_signal(col_done + c);
    }
    return;
  }

  // -------------------------------------------------------------- ROW role
  float2* twr = tws;                                   // row line twiddles
  float2* ptw = twr + LineTw<L, RP::R>::WORDS;         // exp(-2 pi i p / M)
  float2* stages = area;                               // two C2R stages
  float2* rlines = area + 2 * P::STW;                  // row line buffers
  LineTw<L, RP::R>::fill(twr, a.tw, tid, P::THREADS);
  for (int p = tid; p < L; p += P::THREADS) ptw[p] = twiddle<-1>(a.tw, p, LOG_M);
  LineTwB<L, RP::R>::fill(ptw + L, a.tw, tid, P::THREADS);
  const int ntiles = a.total * P::TPS;
  const unsigned need = (unsigned)NCOL + a.stall;      // COL items per chunk
  const int r = tid / TRow, j = tid % TRow;
  const bool valid = r < TR;
  const int rr = valid ? r : 0;
  if (tid == 0) s_next = *(volatile unsigned*)&g_pipe_err ? ntiles : (int)atomicAdd(a.ctl + 1, 1u);
  __syncthreads();
  int cur = s_next;
  bool cur_issued = false;
  int buf = 0;
  while (cur < ntiles) {
    // claim the next tile; prefetch it if its chunk is complete already
    if (tid == 0) {
      int ok = 1;
      if (!cur_issued) ok = pipe_wait(col_done + cur / P::TPS / a.CS, need);
      int nx = ntiles, rdy = 0;
      if (ok && !*(volatile unsigned*)&g_pipe_err) {
        nx = (int)atomicAdd(a.ctl + 1, 1u);
        if (nx < ntiles) rdy = ld_acquire_u32(col_done + nx / P::TPS / a.CS) >= need;
      }
      s_next = nx;
      s_rdy = rdy;
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) break;
    const int nx = s_next;
    const bool rdy = s_rdy != 0;
    if (!cur_issued) pipe_row_issue<LOG_N, LOG_M>(a, stages + buf * P::STW, cur, tid);
    if (rdy) {
      pipe_row_issue<LOG_N, LOG_M>(a, stages + (buf ^ 1) * P::STW, nx, tid);
      cp_async_wait1();
    } else {
      cp_async_wait0();
    }
    __syncthreads();
    const int sub = cur / P::TPS, y0 = (cur - sub * P::TPS) * TR;
    c2r_tile_body<LOG_M, BF16OUT>(stages + buf * P::STW, rlines + (size_t)r * RP::C::WORDS, twr,
                                  ptw, a.out, ((size_t)sub * N + y0 + rr) * M, r, j, valid);
    __syncthreads();                                   // stage reuse, tile stored
    if (tid == 0) pipe_signal(row_done + sub / a.CS);
    cur = nx;
    cur_issued = rdy;
    buf ^= 1;
  }
  cp_async_wait0();
}

// --------------------------------------------------------------- launch
template <typename K>
static cudaError_t prep(K kernel, size_t smem) {
  if (smem > 48 * 1024)
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

static int sm_count() {
  static int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return n;
}

template <int LOG_M>
static cudaError_t r2c_t(InMode mode, bool th, const RowsTArgs& a, cudaStream_t st) {
  using P = RowsT<LOG_M>;
  const int ntiles = a.nsub * (a.N / P::TR);
  if (ntiles == 0) return cudaSuccess;
  cudaError_t e;
#define SHL_LAUNCH(INM, TH)                                                         \
  do {                                                                              \
    const size_t sm = r2c_nst<LOG_M, INM>() * r2c_stage_bytes<LOG_M, INM>() + P::WORK + P::TWB; \
    const int grid = std::min(ntiles, sm_count() * r2c_minb<LOG_M, INM>());         \
    if ((e = prep(k_rows_r2c_t<LOG_M, INM, TH>, sm))) return e;                     \
    k_rows_r2c_t<LOG_M, INM, TH><<<grid, P::THREADS, sm, st>>>(a);                   \
  } while (0)
  if (mode == IN_MASKED) SHL_LAUNCH(IN_MASKED, false);
  else if (mode == IN_BF16) { if (th) SHL_LAUNCH(IN_BF16, true); else SHL_LAUNCH(IN_BF16, false); }
  else { if (th) SHL_LAUNCH(IN_F32, true); else SHL_LAUNCH(IN_F32, false); }
#undef SHL_LAUNCH
  return cudaGetLastError();
}

template <int LOG_M>
static cudaError_t c2r_t(bool bf16, bool s16, const RowsTC2RArgs& a, cudaStream_t st) {
  using P = RowsT<LOG_M>;
  const int ntiles = a.nsub * (a.N / P::TR);
  if (ntiles == 0) return cudaSuccess;
  cudaError_t e;
#define SHL_C2R(B, S)                                                                     \
  if (bf16 == B && s16 == S) {                                                            \
    const size_t sm = c2r_nst<LOG_M, S>() * (S ? P::CSTAGE16 : P::CSTAGE) + P::WORK + P::TWB; \
    const int g = std::min(ntiles, sm_count() * (c2r_occ3<LOG_M, S>() ? 3 : P::MINB));    \
    if ((e = prep(k_rows_c2r_t<LOG_M, B, S>, sm))) return e;                              \
    k_rows_c2r_t<LOG_M, B, S><<<g, P::THREADS, sm, st>>>(a);                              \
    return cudaGetLastError();                                                            \
  }
  SHL_C2R(true, true) SHL_C2R(true, false) SHL_C2R(false, false)
#undef SHL_C2R
  return cudaErrorInvalidValue;                 // bfloat16 staging only with bfloat16 output
}

template <int LOG_M>
static cudaError_t shrink_t(const RowsShrinkArgs& a, cudaStream_t st) {
  using P = RowsT<LOG_M>;
  const int ntiles = a.nsub * (a.N / P::TR);
  if (ntiles == 0) return cudaSuccess;
  const int grid = std::min(ntiles, sm_count() * P::MINB);
  const size_t sm = P::CNST * P::CSTAGE + P::WORK + P::TWB;
  cudaError_t e;
  if ((e = prep(k_rows_shrink_t<LOG_M>, sm))) return e;
  k_rows_shrink_t<LOG_M><<<grid, P::THREADS, sm, st>>>(a);
  return cudaGetLastError();
}

template <int LOG_N>
static cudaError_t lines_t(int mode, const LinesArgs& a, const RecLinesArgs& ra, int grid_y,
                           cudaStream_t st) {
  using P = LinesT<LOG_N>;
  cudaError_t e;
  if (mode == 0 || mode == 1) {
    if (a.nlines == 0) return cudaSuccess;
    const int work = mode == 1 ? ((a.nlines / a.Mh + DEC_FPG - 1) / DEC_FPG) * a.Mh : a.nlines;
    const size_t sm = P::SMEM_LINES + P::TWB;
    // persistent grid-stride: exactly the CTAs that fit at once, so that no
    // partial last wave is left
    int per_sm = 0;
    if (mode == 0) {
      if ((e = prep(k_lines_fwd<LOG_N>, sm))) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lines_fwd<LOG_N>, P::THREADS, sm);
    } else if (a.s16) {
      if ((e = prep(k_dec_lines<LOG_N, true>, sm))) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dec_lines<LOG_N, true>, P::THREADS, sm);
    } else {
      if ((e = prep(k_dec_lines<LOG_N, false>, sm))) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dec_lines<LOG_N, false>, P::THREADS, sm);
    }
    if (e) return e;
    const int grid = std::max(1, std::min((work + P::NG - 1) / P::NG, std::max(per_sm, 1) * sm_count()));
    if (mode == 0) k_lines_fwd<LOG_N><<<grid, P::THREADS, sm, st>>>(a);
    else if (a.s16) k_dec_lines<LOG_N, true><<<grid, P::THREADS, sm, st>>>(a);
    else k_dec_lines<LOG_N, false><<<grid, P::THREADS, sm, st>>>(a);
  } else {
    const size_t sm = P::SMEM_LINES + sizeof(float2) * (size_t)P::NG * P::N + P::TWB;
    if ((e = prep(k_rec_lines<LOG_N>, sm))) return e;
    k_rec_lines<LOG_N><<<dim3(ra.Mh, grid_y), P::THREADS, sm, st>>>(ra);
  }
  return cudaGetLastError();
}

#define SHL_SWITCH_LOG(LOGV, CALL)                 \
  switch (LOGV) {                                  \
    case 4: return CALL(4);                        \
    case 5: return CALL(5);                        \
    case 6: return CALL(6);                        \
    case 7: return CALL(7);                        \
    case 8: return CALL(8);                        \
    case 9: return CALL(9);                        \
    case 10: return CALL(10);                      \
    case 11: return CALL(11);                      \
    default: return cudaErrorInvalidValue;         \
  }

cudaError_t launch_rows_r2c_t(int M, InMode mode, bool thresh, const void* in, const uint8_t* mask,
                              const float* fest, const float* th, float2* out, int N, int nsub,
                              const float2* tw, cudaStream_t st) {
  RowsTArgs a{in, mask, fest, th, out, tw, N, nsub};
#define CALL(X) r2c_t<X>(mode, thresh, a, st)
  SHL_SWITCH_LOG(ilog2(M), CALL)
#undef CALL
}

cudaError_t launch_rows_c2r_t(int M, bool bf16, const void* in, void* out, int N, int nsub,
                              const float2* tw, cudaStream_t st, bool s16) {
  RowsTC2RArgs a{in, out, tw, N, nsub};
#define CALL(X) c2r_t<X>(bf16, s16, a, st)
  SHL_SWITCH_LOG(ilog2(M), CALL)
#undef CALL
}

cudaError_t launch_rows_shrink_t(int M, float2* z, const float* thresh, int N, int nsub,
                                 const float2* tw, cudaStream_t st) {
  RowsShrinkArgs a{z, thresh, tw, N, nsub};
#define CALL(X) shrink_t<X>(a, st)
  SHL_SWITCH_LOG(ilog2(M), CALL)
#undef CALL
}

cudaError_t launch_lines_fwd(int N, float2* data, int nlines, const float2* tw, cudaStream_t st) {
  LinesArgs a{};
  a.data = data; a.nlines = nlines; a.tw = tw;
  RecLinesArgs ra{};
#define CALL(X) lines_t<X>(0, a, ra, 0, st)
  SHL_SWITCH_LOG(ilog2(N), CALL)
#undef CALL
}

cudaError_t launch_dec_lines(int N, const float2* X, void* out, const float* G, const float* invW,
                             float scale, int Mh, int K, int s0, int S, const float2* tw,
                             cudaStream_t st, int nimg, bool s16) {
  LinesArgs a{};
  a.data = const_cast<float2*>(X); a.out = out; a.G = G; a.invW = invW; a.tw = tw;
  a.scale = scale; a.Mh = Mh; a.K = K; a.s0 = s0; a.nlines = S * Mh; a.nimg = nimg;
  a.s16 = s16 ? 1 : 0;
  RecLinesArgs ra{};
#define CALL(X) lines_t<X>(1, a, ra, 0, st)
  SHL_SWITCH_LOG(ilog2(N), CALL)
#undef CALL
}

cudaError_t launch_rec_lines(int N, const float2* stage, float2* acc, const float* G,
                             const float* invW, float scale, int Mh, int K, int s0, int Sc,
                             const float2* tw, cudaStream_t st, int nimg) {
  LinesArgs a{};
  RecLinesArgs ra{stage, acc, G, invW, tw, scale, Mh, K, s0, Sc, s0 / K, nimg};
  const int b_hi = (s0 + Sc - 1) / K;
  const int gy = Sc > 0 ? b_hi - ra.b_lo + 1 : 0;
  if (gy == 0) return cudaSuccess;
#define CALL(X) lines_t<X>(2, a, ra, gy, st)
  SHL_SWITCH_LOG(ilog2(N), CALL)
#undef CALL
}

// ------------------------------------------------------- pipelined launch
template <int LOG_N, int LOG_M, bool BF16>
static cudaError_t dec_pipe_t(const DecPipeArgs& a0, float col_frac, cudaStream_t st) {
  using P = DecPipeT<LOG_N, LOG_M>;
  auto kern = k_dec_pipe<LOG_N, LOG_M, BF16>;
  cudaError_t e;
  if ((e = prep(kern, P::SMEM))) return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, P::THREADS, P::SMEM)))
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = per_sm * sm_count();
  if (grid < 2) return cudaErrorInvalidConfiguration;
  DecPipeArgs args = a0;
  args.ncol_ctas = std::min(grid - 1, std::max(1, (int)std::lround(col_frac * grid)));
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kern), dim3(grid),
                                     dim3(P::THREADS), params, P::SMEM, st);
}

// Column length 1024 needs 32 complex values per lane in the column pass,
// which does not fit beside the row pass at two CTAs per SM (it spills);
// those sizes keep the two-launch path.
bool dec_pipe_supported(int N, int M) { return N == 512 && (M == 512 || M == 1024); }

size_t dec_pipe_ctl_bytes(int nchunks) { return sizeof(unsigned) * (4 + 2 * (size_t)nchunks); }

cudaError_t launch_dec_pipe(int N, int M, bool bf16, const float2* X, float2* ring, void* out,
                            const float* G, const float* invW, float scale, int K, int total,
                            int CS, int NS, float col_frac, unsigned* ctl, const float2* tw,
                            cudaStream_t st) {
  if (total == 0) return cudaSuccess;
  if (!dec_pipe_supported(N, M) || CS < 1 || NS < 2 || !(col_frac > 0.f && col_frac < 1.f))
    return cudaErrorInvalidValue;
  DecPipeArgs a{};
  a.X = X; a.ring = ring; a.out = out; a.G = G; a.invW = invW; a.tw = tw; a.ctl = ctl;
  a.scale = scale; a.Mh = M / 2 + 1; a.K = K; a.total = total; a.CS = CS; a.NS = NS;
  a.nchunks = (total + CS - 1) / CS;
  // SHL_PIPE_STALL_TEST=1 (read per call): the ROW items wait for one COL
  // item more than exist, so every wait runs out; used to test that the
  // bounded waits end the launch and shl_sync reports SHL_ETIMEOUT.
  const char* stall = std::getenv("SHL_PIPE_STALL_TEST");
  a.stall = (stall && stall[0] == '1') ? 1u : 0u;
  cudaError_t e = cudaMemsetAsync(ctl, 0, dec_pipe_ctl_bytes(a.nchunks), st);
  if (e) return e;
#define SHL_PIPE(LN, LM)                                                        \
  if (N == (1 << LN) && M == (1 << LM))                                          \
    return bf16 ? dec_pipe_t<LN, LM, true>(a, col_frac, st) : dec_pipe_t<LN, LM, false>(a, col_frac, st);
  SHL_PIPE(9, 9) SHL_PIPE(9, 10)
#undef SHL_PIPE
  return cudaErrorInvalidValue;
}

// Reads and clears the checked build's guard word of the current device
// (always 0 without SHL_CHECKED).
cudaError_t read_check_word(unsigned* word) {
#ifdef SHL_CHECKED
  cudaError_t e = cudaMemcpyFromSymbol(word, g_shl_check, sizeof(unsigned));
  if (e == cudaSuccess && *word) {
    const unsigned zero = 0;
    e = cudaMemcpyToSymbol(g_shl_check, &zero, sizeof(unsigned));
  }
  return e;
#else
  *word = 0;
  return cudaSuccess;
#endif
}

// Reads and clears the pipelined-wait error flag of the current device.
cudaError_t read_pipe_error(unsigned* flag) {
  cudaError_t e = cudaMemcpyFromSymbol(flag, g_pipe_err, sizeof(unsigned));
  if (e == cudaSuccess && *flag) {
    const unsigned zero = 0;
    e = cudaMemcpyToSymbol(g_pipe_err, &zero, sizeof(unsigned));
  }
  return e;
}

// Per-subband max |c| (optionally divided by RMS_i): one CTA per subband.
template <bool BF16>
__global__ void __launch_bounds__(256) k_absmax(const void* coeffs, int K, size_t elems,
                                                const float* rms, float* out) {
  const int s = blockIdx.x;
  float m = 0.f;
  if (!SHL_IN(s % K, K, CHK_ABSMAX)) return;
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

// Iterative-hard-thresholding schedule (Sec. 4.3, Alg. inpainting): one CTA
// per image; delta_0 = max_i a[b][i] (a = max |c_i| / RMS_i), then
// th[t][b][i] = delta_0 lambda^t RMS_i, lambda = (delta_min / delta_0)^(1/(T-1)),
// in float64 and rounded once.
__global__ void __launch_bounds__(256) k_iht_schedule(const float* a, const float* rms, int K, int B,
                                                      int T, double delta_min, float* th) {
  const int b = blockIdx.x;
  float m = 0.f;
  for (int i = threadIdx.x; i < K; i += blockDim.x) m = fmaxf(m, a[(size_t)b * K + i]);
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float red[8];
  __shared__ double s_d0, s_lam;
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float r = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, red[w]);
    s_d0 = (double)r;
    s_lam = (T > 1 && r > 0.f) ? pow(delta_min / (double)r, 1.0 / (T - 1)) : 1.0;
  }
  __syncthreads();
  const double d0 = s_d0, lam = s_lam;
  for (int e = threadIdx.x; e < T * K; e += blockDim.x) {
    const int t = e / K, i = e - t * K;
    th[((size_t)t * B + b) * K + i] = (float)(d0 * pow(lam, (double)t) * (double)rms[i]);
  }
}

cudaError_t launch_iht_schedule(const float* a, const float* rms, int K, int B, int T,
                                double delta_min, float* th, cudaStream_t st) {
  if (B == 0 || T == 0) return cudaSuccess;
  k_iht_schedule<<<B, 256, 0, st>>>(a, rms, K, B, T, delta_min, th);
  return cudaGetLastError();
}

cudaError_t launch_absmax(const void* coeffs, bool bf16, int nsub, int K, size_t elems,
                          const float* rms, float* out, cudaStream_t st) {
  if (nsub == 0) return cudaSuccess;
  if (bf16) k_absmax<true><<<nsub, 256, 0, st>>>(coeffs, K, elems, rms, out);
  else k_absmax<false><<<nsub, 256, 0, st>>>(coeffs, K, elems, rms, out);
  return cudaGetLastError();
}

}  // namespace shl
