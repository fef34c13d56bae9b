// tc_dft.cu - the column pass of the bfloat16-output decomposition on the
// tensor cores (tcgen05, bfloat16 operands, float32 accumulation in TMEM).
//
// Same result as k_dec_lines for 512-point columns: for every line l =
// (subband s, column frequency kx) of the chunk,
//   Z_l[y] = sum_ky V_l[ky] exp(+2 pi i ky y / 512),
//   V_l[ky] = X_b[kx][ky] * G_i[kx][ky] * scale [* 1/W[kx][ky]]
// (the filter product and inverse column transform of Sec. 3.4), written to
// the float32 staging plane for the row pass.  The 512-point DFT is split as
// ky = n1 + 16 n2, y = k2 + 32 k1 (Cooley-Tukey, 32 x 16):
//   stage 1  Y[k2][n1] = sum_n2 exp(2 pi i n2 k2 / 32) V[n1 + 16 n2]
//   twiddle  T[k2][n1] = exp(2 pi i n1 k2 / 512) Y[k2][n1]
//   stage 2  Z[k2 + 32 k1] = sum_n1 exp(2 pi i n1 k1 / 16) T[k2][n1]
// Each stage is one real GEMM on complex data written as (re, im) pairs,
// [re; im](out) = [[C, -S], [S, C]] [re; im](in), with the DFT matrix on one
// side and a tile of 8 lines on the other:
//   stage 1  D1[2 k2 + c][(l, n1)] = sum_{(n2, c')} F32[2 k2 + c][2 n2 + c'] V[(l, n1)][2 n2 + c']
//            (M = 128: rows 64..127 repeat rows 0..63, N = 8 lines x 16 n1 = 128, K = 64)
//   stage 2  D2[(l, k2)][2 k1 + c] = sum_{(n1, c')} T[(l, k2)][2 n1 + c'] F16[2 k1 + c][2 n1 + c']
//            (two M = 128 tiles of 4 lines x 32 k2, N = 32, K = 32)
// One thread fetches the next tile's spectrum and filter lines (contiguous
// 4 KB and 2 KB runs) with bulk copies (TMA) while the current tile runs its
// stages; the CTA forms V from them.  Operands sit in shared memory in the
// no-swizzle K-major core-matrix layout [K / 8][row][8 elements] (16 bytes
// per row and 8-element group).  Between
// the stages every thread reads one TMEM lane (a k2 and a re/im component)
// of D1, takes the other component from its neighbour lane, applies the
// twiddle and writes T as the stage-2 A operand; the stage-2 accumulators
// reuse D1's columns.  The waits on the MMAs' mbarrier are bounded: when
// one runs out the kernel records it (read by shl_sync), waits once more
// for the MMAs and copies in flight, frees its TMEM and returns.
//
// bfloat16 operands (8-bit mantissa) bound the relative error of Z near
// 2^-8; this pass serves only the decomposition whose coefficients are
// stored in bfloat16, where the storage rounding is of the same size.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "check.cuh"
#include "internal.h"

namespace shl {
namespace {

SHL_CHECK_WORD_DEFINE

__device__ unsigned int g_dft_err = 0;

constexpr int TD_N = 512;
constexpr int TD_LINES = 8;                    // lines per tile
constexpr int TD_THREADS = 256;
constexpr unsigned TD_SPIN_LIMIT = 1u << 22;
constexpr uint32_t TD_COLS = 128;              // TMEM columns (D1; D2 reuses 0..63)

// shared-memory layout (bytes); LBO = stride between K groups
constexpr uint32_t A1_LBO = 128 * 16;          // F32 real form, 128 rows x 64 K
constexpr uint32_t A1_BYTES = 8 * A1_LBO;
constexpr uint32_t B1_LBO = 128 * 16;          // V, 128 rows (l, n1) x 64 K
constexpr uint32_t B1_BYTES = 8 * B1_LBO;
constexpr uint32_t A2_LBO = 128 * 16 + 32;     // T, 128 rows x 32 K per tile; +32 spreads banks
constexpr uint32_t A2_TILE = 4 * A2_LBO;
constexpr uint32_t A2_BYTES = 2 * A2_TILE;
constexpr uint32_t B2_LBO = 32 * 16;           // F16 real form, 32 rows x 32 K
constexpr uint32_t B2_BYTES = 4 * B2_LBO;
constexpr uint32_t RX_BYTES = TD_LINES * TD_N * 8;   // the tile's spectrum lines, float2
constexpr uint32_t RG_BYTES = TD_LINES * TD_N * 4;   // its filter lines, float
constexpr uint32_t OFF_A1 = 0, OFF_B1 = OFF_A1 + A1_BYTES, OFF_A2 = OFF_B1 + B1_BYTES,
                   OFF_B2 = OFF_A2 + A2_BYTES, OFF_TW = OFF_B2 + B2_BYTES,
                   OFF_RX = OFF_TW + 32 * 16 * 8, OFF_RG = OFF_RX + RX_BYTES;
constexpr uint32_t TD_SMEM = OFF_RG + RG_BYTES;

struct DftArgs {
  const float2* X;       // image spectra [nimg][Mh][512]
  float2* out;           // staging [S][Mh][512]
  const float* G;        // [K][Mh][512]
  const float* invW;     // [Mh][512] or null
  const float2* tw;      // exp(-2 pi i q / TW_P)
  float scale;
  int Mh, K, s0, nlines, nimg;
};

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor, no swizzle, version 1.
__device__ __forceinline__ uint64_t mdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: float32 D, bfloat16 A and B, K-major.
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t pk(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ float2 tw_pos(const float2* tw, int e, int logD) {
  const int q = (e & ((1 << logD) - 1)) << (LOG_TW_P - logD);
  const float2 w = __ldg(tw + q);
  return make_float2(w.x, -w.y);                 // exp(+2 pi i e / 2^logD)
}

__device__ __forceinline__ bool wait_bounded(uint32_t bar, uint32_t parity) {
  for (unsigned i = 0; i < TD_SPIN_LIMIT; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

__device__ __forceinline__ void arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// Warp 0: bulk copies (TMA) of the spectrum and filter lines of tile `tile`
// into RX / RG, completing on `bar`: lane 0 arms the barrier with the byte
// count, then lane l < 8 copies spectrum line l and lane 8 + l filter line l
// (lines past the end are skipped).
__device__ __forceinline__ void fetch_tile(const DftArgs& a, int tile, uint32_t rx, uint32_t rg,
                                           uint32_t bar, int lane) {
  const int l0 = tile * TD_LINES;
  const int n = min(TD_LINES, a.nlines - l0);
  if (lane == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    arrive_tx(bar, (uint32_t)n * TD_N * 12);
  }
  __syncwarp();
  const int l = lane & 7;
  if (lane < 16 && l < n) {
    const int sl0 = l0 / a.Mh, kx0 = l0 - sl0 * a.Mh;
    const bool wrap = kx0 + l >= a.Mh;
    const int kx = wrap ? kx0 + l - a.Mh : kx0 + l;
    const int s = a.s0 + sl0 + (wrap ? 1 : 0), b = s / a.K, i = s - b * a.K;
    if (lane < 8) {
      const bool ok = SHL_IN((size_t)b * a.Mh + kx, (size_t)a.nimg * a.Mh, CHK_TC_X);
      // a guarded-out line reads line 0 instead (the checked build has flagged it)
      bulk_load(rx + l * TD_N * 8, a.X + (ok ? ((size_t)b * a.Mh + kx) * TD_N : 0), TD_N * 8, bar);
    } else {
      const bool ok = SHL_IN((size_t)i * a.Mh + kx, (size_t)a.K * a.Mh, CHK_TC_G);
      bulk_load(rg + l * TD_N * 4, a.G + (ok ? ((size_t)i * a.Mh + kx) * TD_N : 0), TD_N * 4, bar);
    }
  }
}

#define TD_LD16(R, ADDR)                                                                    \
  asm volatile(                                                                             \
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "                                             \
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"                     \
      : "=r"((R)[0]), "=r"((R)[1]), "=r"((R)[2]), "=r"((R)[3]), "=r"((R)[4]), "=r"((R)[5]), \
        "=r"((R)[6]), "=r"((R)[7]), "=r"((R)[8]), "=r"((R)[9]), "=r"((R)[10]),              \
        "=r"((R)[11]), "=r"((R)[12]), "=r"((R)[13]), "=r"((R)[14]), "=r"((R)[15])           \
      : "r"(ADDR)                                                                           \
      : "memory")

__global__ void __launch_bounds__(TD_THREADS, 2) k_dec_lines_tc(DftArgs a) {
  extern __shared__ __align__(128) uint8_t sm[];
  __shared__ __align__(8) uint64_t mbar[2];        // [0] MMAs, [1] line copies
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t* A1 = sm + OFF_A1;
  uint8_t* B1 = sm + OFF_B1;
  uint8_t* A2 = sm + OFF_A2;
  uint8_t* B2 = sm + OFF_B2;
  float2* TW = reinterpret_cast<float2*>(sm + OFF_TW);
  const float2* RX = reinterpret_cast<const float2*>(sm + OFF_RX);
  const float* RG = reinterpret_cast<const float*>(sm + OFF_RG);
  const int ntiles = (a.nlines + TD_LINES - 1) / TD_LINES;

  // constant operands: F32 (rows 2 k2 + c, repeated for rows 64..127), F16,
  // and the twiddles exp(2 pi i n1 k2 / 512)
  for (int it = tid; it < 128 * 8; it += TD_THREADS) {
    const int m = it >> 3, g = it & 7;             // row, K group (n2 = 4 g .. 4 g + 3)
    const int k2 = (m & 63) >> 1, c = m & 1;
    uint32_t w[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float2 e = tw_pos(a.tw, (4 * g + t) * k2, 5);
      w[t] = c == 0 ? pk(e.x, -e.y) : pk(e.y, e.x);
    }
    *reinterpret_cast<uint4*>(A1 + g * A1_LBO + m * 16) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  for (int it = tid; it < 32 * 4; it += TD_THREADS) {
    const int n = it >> 2, g = it & 3;             // row 2 k1 + c, K group (n1 = 4 g .. 4 g + 3)
    const int k1 = n >> 1, c = n & 1;
    uint32_t w[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float2 e = tw_pos(a.tw, (4 * g + t) * k1, 4);
      w[t] = c == 0 ? pk(e.x, -e.y) : pk(e.y, e.x);
    }
    *reinterpret_cast<uint4*>(B2 + g * B2_LBO + n * 16) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  for (int it = tid; it < 32 * 16; it += TD_THREADS) TW[it] = tw_pos(a.tw, (it >> 4) * (it & 15), 9);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&tmem_slot)), "r"(TD_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  const uint32_t bar = su32(&mbar[0]), rbar = su32(&mbar[1]);
  const uint32_t rx = su32(sm + OFF_RX), rg = su32(sm + OFF_RG);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(rbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0 && (int)blockIdx.x < ntiles) fetch_tile(a, blockIdx.x, rx, rg, rbar, lane);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t a1 = su32(A1), b1 = su32(B1), a2 = su32(A2), b2 = su32(B2);

  // this thread's D1 lane: quarter q, k2 = 16 (q & 1) + lane / 2, component c
  const int q = warp & 3, c = lane & 1, k2 = 16 * (q & 1) + (lane >> 1);
  const int lpair = (q >> 1) + 2 * (warp >> 2);    // D1 lines 2 lpair, 2 lpair + 1
  float2 tw8[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) tw8[u] = TW[k2 * 16 + u + 8 * c];
  // conversion items (l, n1, g): this thread's share n1, g fixed, l = lc, lc + 2, ...
  const int n1 = tid & 15, g = (tid >> 4) & 7, lc = tid >> 7;

  uint32_t phase = 0, rphase = 0;
  int inflight = (int)blockIdx.x < ntiles ? 1 : 0;   // line copies issued and not waited on
  bool failed = false, mma_pending = false;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int l0 = tile * TD_LINES;
    bool ok = wait_bounded(rbar, rphase);
    if (__syncthreads_or(!ok)) { failed = true; break; }
    rphase ^= 1u;
    inflight = 0;
    // V = X * G * scale [* 1/W] -> bfloat16 B1 rows (l, n1), K group g = n2 4 g .. 4 g + 3
    const int sl0 = l0 / a.Mh, kx0 = l0 - sl0 * a.Mh;
#pragma unroll
    for (int k = 0; k < TD_LINES / 2; ++k) {
      const int l = lc + 2 * k;
      uint32_t w[4] = {0u, 0u, 0u, 0u};
      if (l0 + l < a.nlines) {
        const float* Wp = nullptr;
        if (a.invW) {
          const int kx = kx0 + l >= a.Mh ? kx0 + l - a.Mh : kx0 + l;
          Wp = a.invW + (size_t)kx * TD_N;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int ky = n1 + 16 * (4 * g + t);
          const float2 x = RX[l * TD_N + ky];
          float gv = RG[l * TD_N + ky] * a.scale;
          if (Wp) gv *= __ldg(Wp + ky);
          w[t] = pk(x.x * gv, x.y * gv);
        }
      }
      *reinterpret_cast<uint4*>(B1 + g * B1_LBO + (l * 16 + n1) * 16) =
          make_uint4(w[0], w[1], w[2], w[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    __syncthreads();                                 // B1 written, RX / RG read
    if (warp == 0) {
      if (lane == 0) {
        fence_after();
#pragma unroll
        for (int s = 0; s < 4; ++s)                  // stage 1: 4 K steps of 16
          mma(tmem, mdesc(a1 + 2 * s * A1_LBO, A1_LBO, 128),
              mdesc(b1 + 2 * s * B1_LBO, B1_LBO, 128), idesc(128, 128), s > 0);
        commit(bar);
      }
      __syncwarp();
      const int next = tile + gridDim.x;             // lands during this tile's stages
      if (next < ntiles) fetch_tile(a, next, rx, rg, rbar, lane);
    }
    inflight = tile + (int)gridDim.x < ntiles ? 1 : 0;
    ok = wait_bounded(bar, phase);
    if (__syncthreads_or(!ok)) { failed = mma_pending = true; break; }
    phase ^= 1u;
    fence_after();

    // D1 -> twiddled T -> A2 (lane pairs swap components: c = 0 forms n1 0..7, c = 1 n1 8..15)
    uint32_t d1[2][16];
    TD_LD16(d1[0], tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * lpair));
    TD_LD16(d1[1], tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * lpair + 16));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int l = 2 * lpair + h;
      const uint32_t* v = d1[h];
      float re[8], im[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float send = __uint_as_float(c ? v[u] : v[u + 8]);
        const float got = __shfl_xor_sync(0xffffffffu, send, 1);
        const float mine = __uint_as_float(c ? v[u + 8] : v[u]);
        const float yr = c ? got : mine, yi = c ? mine : got;
        re[u] = yr * tw8[u].x - yi * tw8[u].y;
        im[u] = yr * tw8[u].y + yi * tw8[u].x;
      }
      const int mt = l >> 2, r2 = (l & 3) * 32 + k2;
      uint8_t* dst = A2 + mt * A2_TILE + (2 * c) * A2_LBO + r2 * 16;
      *reinterpret_cast<uint4*>(dst) =
          make_uint4(pk(re[0], im[0]), pk(re[1], im[1]), pk(re[2], im[2]), pk(re[3], im[3]));
      *reinterpret_cast<uint4*>(dst + A2_LBO) =
          make_uint4(pk(re[4], im[4]), pk(re[5], im[5]), pk(re[6], im[6]), pk(re[7], im[7]));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    __syncthreads();
    if (tid == 0) {                                  // stage 2: 2 M tiles x 2 K steps
      fence_after();
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int s = 0; s < 2; ++s)
          mma(tmem + (uint32_t)(32 * mt), mdesc(a2 + mt * A2_TILE + 2 * s * A2_LBO, A2_LBO, 128),
              mdesc(b2 + 2 * s * B2_LBO, B2_LBO, 128), idesc(128, 32), s > 0);
      commit(bar);
    }
    ok = wait_bounded(bar, phase);
    if (__syncthreads_or(!ok)) { failed = mma_pending = true; break; }
    phase ^= 1u;
    fence_after();

    // D2 -> staging: warp w reads line 4 (w / 4) + q, lane k2: Z[k2 + 32 k1], k1 = 0..15
    {
      const int mt = warp >> 2, line = l0 + 4 * mt + q;
      uint32_t v[32];
      TD_LD16(v, tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * mt));
      TD_LD16(v + 16, tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * mt + 16));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (line < a.nlines && SHL_IN(line, a.nlines, CHK_TC_OUT)) {
        float2* o = a.out + (size_t)line * TD_N + lane;
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1)
          o[32 * k1] = make_float2(__uint_as_float(v[2 * k1]), __uint_as_float(v[2 * k1 + 1]));
      }
    }
    fence_before();                                  // TMEM reads done before the next MMAs
  }
  if (failed && tid == 0) {
    atomicOr(&g_dft_err, 1u);
    if (mma_pending) wait_bounded(bar, phase);       // the MMAs whose wait ran out
    if (inflight) wait_bounded(rbar, rphase);        // line copies still in flight
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TD_COLS)
                 : "memory");
}

}  // namespace

// A tile's 8 lines span at most two subbands when Mh >= 8.
bool dec_lines_tc_supported(int N, int Mh) { return N == TD_N && Mh >= TD_LINES; }

cudaError_t launch_dec_lines_tc(int N, const float2* X, float2* out, const float* G,
                                const float* invW, float scale, int Mh, int K, int s0, int S,
                                const float2* tw, cudaStream_t st, int nimg) {
  if (S == 0) return cudaSuccess;
  if (!dec_lines_tc_supported(N, Mh) || S < 0) return cudaErrorInvalidValue;
  static int nsm[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (nsm[dev] == 0) {
    if ((e = cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev))) return e;
    if ((e = cudaFuncSetAttribute(k_dec_lines_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)TD_SMEM)))
      return e;
  }
  DftArgs a{X, out, G, invW, tw, scale, Mh, K, s0, S * Mh, nimg};
  const int ntiles = (a.nlines + TD_LINES - 1) / TD_LINES;
  const int grid = ntiles < 2 * nsm[dev] ? ntiles : 2 * nsm[dev];   // two CTAs per SM
  k_dec_lines_tc<<<grid, TD_THREADS, TD_SMEM, st>>>(a);
  return cudaGetLastError();
}

cudaError_t read_dft_error(unsigned* flag) {
  cudaError_t e = cudaMemcpyFromSymbol(flag, g_dft_err, sizeof(unsigned));
  if (e == cudaSuccess && *flag) {
    const unsigned zero = 0;
    e = cudaMemcpyToSymbol(g_dft_err, &zero, sizeof(unsigned));
  }
  return e;
}

cudaError_t read_check_word_tc(unsigned* word) {
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

}  // namespace shl
