// tc_dft.cu - the column pass of the bfloat16-output decomposition on the
// tensor cores (tcgen05, bfloat16 operands, float32 accumulation in TMEM).
//
// Same result as k_dec_lines for 512-point columns: for every line l =
// (subband s, column frequency kx) of the chunk,
//   Z_l[y] = sum_ky V_l[ky] exp(+2 pi i ky y / 512),
//   V_l[ky] = X_b[kx][ky] * G_i[kx][ky] * scale [* 1/W[kx][ky]]
// (the filter product and inverse column transform of Sec. 3.4), written to
// the staging plane of the row pass (bfloat16 pairs, or float2).  The
// 512-point DFT is split as ky = n1 + 16 n2, y = k2 + 32 k1 (Cooley-Tukey,
// 32 x 16):
//   stage 1  Y[k2][n1] = sum_n2 exp(2 pi i n2 k2 / 32) V[n1 + 16 n2]
//   twiddle  T[k2][n1] = exp(2 pi i n1 k2 / 512) Y[k2][n1]
//   stage 2  Z[k2 + 32 k1] = sum_n1 exp(2 pi i n1 k1 / 16) T[k2][n1]
// Each stage is one real GEMM on complex data written as (re, im) pairs,
// [re; im](out) = [[C, -S], [S, C]] [re; im](in), with the DFT matrix on one
// side and a tile of 8 lines on the other (two column frequencies of four
// subbands of one image, tile_at):
//   stage 1  D1[2 k2 + c][(l, n1)] = sum_{(n2, c')} F32[2 k2 + c][2 n2 + c'] V[(l, n1)][2 n2 + c']
//            (M = 128: rows 64..127 repeat rows 0..63, N = 8 lines x 16 n1 = 128, K = 64)
//   stage 2  D2[(l, k2)][2 k1 + c] = sum_{(n1, c')} T[(l, k2)][2 n1 + c'] F16[2 k1 + c][2 n1 + c']
//            (two M = 128 tiles of 4 lines x 32 k2, N = 32, K = 32)
// Operands sit in shared memory in the no-swizzle K-major core-matrix
// layout [K / 8][row][8 elements] (16 bytes per row and 8-element group).
// The work of a tile is split over warp roles that run concurrently on
// different tiles: one warp copies the tile's two spectrum lines and its
// four filters' line pairs (contiguous runs) with bulk copies (TMA); eight
// warps form V from them; one thread issues both stages' MMAs; four warps
// read D1 (every thread one TMEM lane, a k2 and a re/im component, the
// other component from its neighbour lane), apply the twiddle and write T;
// four warps read D2 and store the lines.  Line slots, V, D1, T and D2 are
// two-slot rings handed between the roles by mbarriers (MMA completion
// through tcgen05.commit).  Every wait is bounded: when one runs out the
// kernel records it (read by shl_sync), the other roles stop at their next
// wait, the copies and MMAs in flight are waited for, and TMEM is freed.
//
// bfloat16 operands (8-bit mantissa) bound the relative error of Z near
// 2^-8; this pass serves only the decomposition whose coefficients are
// stored in bfloat16, where the storage rounding is of the same size.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "check.cuh"
#include "internal.h"

namespace shl {
namespace {

SHL_CHECK_WORD_DEFINE

__device__ unsigned int g_dft_err = 0;

constexpr int TD_N = 512;
constexpr int TD_LINES = 8;                    // lines per tile
// Roles by warp: 0-3 read out stage 1 (TMEM lane quarters 0-3), 4-7 read out
// stage 2 and store, 8-15 form the stage-1 operand, 16 copies lines, 17
// issues the MMAs.  Each hand-over is a two-slot ring of mbarrier pairs.
constexpr int W_RD1 = 0, W_RD2 = 4, W_CONV = 8, W_COPY = 16, W_MMA = 17;
constexpr int TD_THREADS = 18 * 32;
constexpr int GROUP = 128;                     // threads of a read-out role
constexpr int CGROUP = 256;                    // threads of the conversion role
constexpr unsigned TD_SPIN_LIMIT = 1u << 22;
// TMEM: D1 of even / odd tiles at columns 0 / 128, D2 at 256 / 320
constexpr uint32_t TD_COLS = 512;
constexpr uint32_t D1_COL = 0, D2_COL = 256;

// shared-memory layout (bytes); LBO = stride between K groups.  The line
// slots, V (B1) and T (A2) are two-slot rings: tile k uses slot k & 1.
constexpr uint32_t A1_LBO = 128 * 16;          // F32 real form, 128 rows x 64 K
constexpr uint32_t A1_BYTES = 8 * A1_LBO;
constexpr uint32_t B1_LBO = 128 * 16;          // V, 128 rows (l, n1) x 64 K
constexpr uint32_t B1_BYTES = 8 * B1_LBO;
constexpr uint32_t A2_LBO = 128 * 16 + 32;     // T, 128 rows x 32 K per M tile; +32 spreads banks
constexpr uint32_t A2_TILE = 4 * A2_LBO;
constexpr uint32_t A2_BYTES = 2 * A2_TILE;
constexpr uint32_t B2_LBO = 32 * 16;           // F16 real form, 32 rows x 32 K
constexpr uint32_t B2_BYTES = 4 * B2_LBO;
constexpr uint32_t RX_BYTES = 2 * TD_N * 8;          // a tile's two spectrum lines, float2
constexpr uint32_t RG_BYTES = TD_LINES * TD_N * 4;   // its 4 x 2 filter lines [j][h], float
constexpr uint32_t RAW_BYTES = RX_BYTES + RG_BYTES;
constexpr uint32_t OFF_A1 = 0, OFF_B2 = OFF_A1 + A1_BYTES, OFF_TW = OFF_B2 + B2_BYTES,
                   OFF_B1 = OFF_TW + 32 * 16 * 8, OFF_A2 = OFF_B1 + 2 * B1_BYTES,
                   OFF_RAW = OFF_A2 + 2 * A2_BYTES;
constexpr uint32_t TD_SMEM = OFF_RAW + 2 * RAW_BYTES;
static_assert(TD_SMEM <= 227 * 1024, "tensor-core column pass does not fit shared memory");

// mbarriers, two slots each: FULL / EMPTY of the line slots, V, D1, T, D2
enum : int { RAW_FULL = 0, RAW_EMPTY = 2, B1_FULL = 4, B1_EMPTY = 6, D1_FULL = 8, D1_EMPTY = 10,
             A2_FULL = 12, A2_EMPTY = 14, D2_FULL = 16, D2_EMPTY = 18, NBAR = 20 };

struct DftArgs {
  const float2* X;       // image spectra [nimg][Mh][512]
  void* out;             // staging [S][Mh][512], float2 or (s16) bfloat162
  const float* G;        // [K][Mh][512]
  const float* invW;     // [Mh][512] or null
  const float2* tw;      // exp(-2 pi i q / TW_P)
  float scale;
  int Mh, K, s0, nimg;
  int s16;               // bfloat16 staging
  int S, b_lo, gmax, npairs, ntiles;   // the chunk's subbands; tiling (tile_at)
};

// Tile t of a chunk: image b = b_lo + t / (gmax npairs); its subbands
// s .. s + 3 (s = the image's first subband in the chunk + 4 f) and column
// frequencies kx, kx + 1 (kx = 2 p).  Line l = 2 j + h of the tile is
// (subband s + j, column frequency kx + h); nj / nh of the four subbands /
// two column frequencies exist (nj = 0 for a tile past the image's last
// subband: an empty tile).  The two spectrum lines serve all four filters.
struct Tile {
  int b, s, kx, nj, nh;
};
__device__ __forceinline__ Tile tile_at(const DftArgs& a, int t) {
  Tile r;
  const int per_img = a.gmax * a.npairs;
  const int bi = t / per_img, rem = t - bi * per_img;
  const int f = rem / a.npairs, p = rem - f * a.npairs;
  r.b = a.b_lo + bi;
  const int sa = max(a.s0, r.b * a.K), sb = min(a.s0 + a.S, (r.b + 1) * a.K);
  r.s = sa + 4 * f;
  r.nj = max(0, min(4, sb - r.s));
  r.kx = 2 * p;
  r.nh = min(2, a.Mh - r.kx);
  return r;
}

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

// One warp: bulk copies (TMA) of tile t's lines into RX / RG, completing on
// `bar`.  Lane 0 arms the barrier with the byte count (zero for an empty
// tile) and copies the two spectrum lines, one contiguous run; lane 1 + j
// copies filter j's two lines, another.
__device__ __forceinline__ void fetch_tile(const DftArgs& a, int t, uint32_t rx, uint32_t rg,
                                           uint32_t bar, int lane) {
  const Tile T = tile_at(a, t);
  if (lane == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    arrive_tx(bar, T.nj > 0 ? (uint32_t)(T.nh * TD_N * (8 + 4 * T.nj)) : 0u);
  }
  __syncwarp();
  if (T.nj == 0) return;
  const int i0 = T.s - T.b * a.K;
  if (lane == 0) {
    const bool ok = SHL_IN((size_t)T.b * a.Mh + T.kx + T.nh - 1, (size_t)a.nimg * a.Mh, CHK_TC_X);
    // a guarded-out run reads line 0 instead (the checked build has flagged it)
    bulk_load(rx, a.X + (ok ? ((size_t)T.b * a.Mh + T.kx) * TD_N : 0), (uint32_t)T.nh * TD_N * 8, bar);
  } else if (lane <= T.nj) {
    const int j = lane - 1;
    const bool ok = SHL_IN((size_t)(i0 + j) * a.Mh + T.kx + T.nh - 1, (size_t)a.K * a.Mh, CHK_TC_G);
    bulk_load(rg + j * 2 * TD_N * 4, a.G + (ok ? ((size_t)(i0 + j) * a.Mh + T.kx) * TD_N : 0),
              (uint32_t)T.nh * TD_N * 4, bar);
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

// Wait for phase `parity` of mbarrier `bar`.  false when the wait runs out
// (the role records it in *fail) or another role has failed: the caller's
// role then stops.
__device__ __forceinline__ bool role_wait(uint32_t bar, uint32_t parity, volatile int* fail) {
  for (unsigned i = 0; i < TD_SPIN_LIMIT; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
    if ((i & 255u) == 255u && *fail) return false;
  }
  *fail = 1;
  return false;
}

// role_wait taken by a whole warp: every lane goes on or every lane stops.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int* fail) {
  return __all_sync(0xffffffffu, role_wait(bar, parity, fail));
}

__device__ __forceinline__ void arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// One CTA per SM walks the tiles blockIdx.x + k gridDim.x, k = 0 .. nk-1,
// each role at its own pace:
//   copy warp     lines of tile k -> line slot k & 1          (after the slot is empty)
//   conversion    V = X G scale [/W] of tile k -> B1 slot      (after its lines arrived)
//   MMA thread    stage 1 of tile k -> D1 slot, then stage 2 of tile k-1 -> D2 slot
//   read-out 1    D1 of tile k, twiddled -> T (A2 slot)
//   read-out 2    D2 of tile k -> staging rows
// Every slot is handed on by a FULL mbarrier and back by an EMPTY one (MMA
// completion arrives through tcgen05.commit), so up to two tiles are in
// each stage at once and the stages overlap across tiles.
__global__ void __launch_bounds__(TD_THREADS, 1) k_dec_lines_tc(DftArgs a) {
  extern __shared__ __align__(128) uint8_t sm[];
  __shared__ __align__(8) uint64_t mb[NBAR];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail, s_copies, s_mma1, s_mma2;   // failure flag; tiles issued per async unit
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t* A1 = sm + OFF_A1;
  uint8_t* B2 = sm + OFF_B2;
  float2* TW = reinterpret_cast<float2*>(sm + OFF_TW);
  const int ntiles = a.ntiles;
  const int nk = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  auto tile_of = [&](int k) { return (int)blockIdx.x + k * (int)gridDim.x; };
  auto bar = [&](int i) { return su32(&mb[i]); };
  volatile int* fail = &s_fail;

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
  if (tid == 0) {
    for (int i = 0; i < NBAR; ++i) {
      const int kind = i & ~1;
      const unsigned count = (kind == RAW_EMPTY || kind == B1_FULL) ? CGROUP
                             : (kind == D1_EMPTY || kind == A2_FULL || kind == D2_EMPTY) ? GROUP
                                                                                           : 1;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(i)), "r"(count) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
    s_copies = s_mma1 = s_mma2 = 0;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // constant operands
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp >= W_RD1 && warp < W_RD1 + 4) {
    // stage-1 read-out: thread (quarter q, lane) holds row 32 q + lane of D1,
    // i.e. k2 = 16 (q & 1) + lane / 2 and component c = lane & 1 (rows 64..127
    // repeat 0..63: quarters 0, 1 take lines 0-3, quarters 2, 3 lines 4-7)
    const int q = warp & 3, c = lane & 1, k2 = 16 * (q & 1) + (lane >> 1);
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    float2 tw8[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) tw8[u] = TW[k2 * 16 + u + 8 * c];
    for (int k = 0; k < nk; ++k) {
      const int s = k & 1;
      const uint32_t ph = (k >> 1) & 1;
      if (!warp_wait(bar(D1_FULL + s), ph, fail) || !warp_wait(bar(A2_EMPTY + s), ph ^ 1, fail))
        break;
      fence_after();
      uint8_t* A2 = sm + OFF_A2 + s * A2_BYTES;
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int lpair = 2 * (q >> 1) + i;          // lines 2 lpair, 2 lpair + 1
        uint32_t d1v[2][16];
        const uint32_t d1 = tmem + lanes + D1_COL + (uint32_t)(128 * s + 32 * lpair);
        TD_LD16(d1v[0], d1);
        TD_LD16(d1v[1], d1 + 16u);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (i == 1) {                                // this thread's reads of D1 are done
          fence_before();
          arrive(bar(D1_EMPTY + s));
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int l = 2 * lpair + h;
          const uint32_t* v = d1v[h];
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
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      arrive(bar(A2_FULL + s));
    }
  } else if (warp >= W_RD2 && warp < W_RD2 + 4) {
    // stage-2 read-out: quarter q holds rows (l & 3) 32 + k2 of both M tiles,
    // i.e. lines 4 mt + q, k2 = lane; columns 2 k1 + c
    const int q = warp & 3;
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    for (int k = 0; k < nk; ++k) {
      const int s = k & 1;
      if (!warp_wait(bar(D2_FULL + s), (k >> 1) & 1, fail)) break;
      fence_after();
      uint32_t v[2][32];
      const uint32_t d2 = tmem + lanes + D2_COL + (uint32_t)(64 * s);
      TD_LD16(v[0], d2);
      TD_LD16(v[0] + 16, d2 + 16u);
      TD_LD16(v[1], d2 + 32u);
      TD_LD16(v[1] + 16, d2 + 48u);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      fence_before();
      arrive(bar(D2_EMPTY + s));
      const Tile T = tile_at(a, tile_of(k));
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int j = (4 * mt + q) >> 1, h = q & 1;    // tile line 4 mt + q = 2 j + h
        const int line = (T.s + j - a.s0) * a.Mh + T.kx + h;
        if (j < T.nj && h < T.nh && SHL_IN(line, (size_t)a.S * a.Mh, CHK_TC_OUT)) {
          if (a.s16) {
            __nv_bfloat162* o = static_cast<__nv_bfloat162*>(a.out) + (size_t)line * TD_N + lane;
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1)
              o[32 * k1] = __floats2bfloat162_rn(__uint_as_float(v[mt][2 * k1]),
                                                 __uint_as_float(v[mt][2 * k1 + 1]));
          } else {
            float2* o = static_cast<float2*>(a.out) + (size_t)line * TD_N + lane;
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1)
              o[32 * k1] = make_float2(__uint_as_float(v[mt][2 * k1]), __uint_as_float(v[mt][2 * k1 + 1]));
          }
        }
      }
    }
  } else if (warp >= W_CONV && warp < W_CONV + 8) {
    // V[(l, n1)][(n2, c)]: thread (n1, g, h) forms n2 = 4 g .. 4 g + 3 of the
    // four lines l = 2 j + h of column frequency kx + h, reading its
    // spectrum values (and 1/W) once for the four filters
    const int ct = tid - W_CONV * 32;
    const int n1 = ct & 15, g = (ct >> 4) & 7, h = ct >> 7;
    for (int k = 0; k < nk; ++k) {
      const int s = k & 1;
      const uint32_t ph = (k >> 1) & 1;
      if (!warp_wait(bar(RAW_FULL + s), ph, fail) || !warp_wait(bar(B1_EMPTY + s), ph ^ 1, fail))
        break;
      const Tile T = tile_at(a, tile_of(k));
      const float2* RX = reinterpret_cast<const float2*>(sm + OFF_RAW + s * RAW_BYTES);
      const float* RG = reinterpret_cast<const float*>(sm + OFF_RAW + s * RAW_BYTES + RX_BYTES);
      uint8_t* B1 = sm + OFF_B1 + s * B1_BYTES;
      const bool hv = h < T.nh;
      // (slots of lines that do not exist hold stale data, read in bounds
      // and replaced by zeros)
      float2 xv[4];
      float wv[4] = {1.f, 1.f, 1.f, 1.f};
#pragma unroll
      for (int t = 0; t < 4; ++t) xv[t] = RX[h * TD_N + n1 + 16 * (4 * g + t)];
      if (a.invW && hv) {
#pragma unroll
        for (int t = 0; t < 4; ++t) wv[t] = __ldg(a.invW + (size_t)(T.kx + h) * TD_N + n1 + 16 * (4 * g + t));
      }
      uint4 pkd[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float gq[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) gq[t] = RG[(2 * j + h) * TD_N + n1 + 16 * (4 * g + t)];
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if (j < T.nj && hv) {
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const float gv = gq[t] * a.scale * wv[t];
            w[t] = pk(xv[t].x * gv, xv[t].y * gv);
          }
        }
        pkd[j] = make_uint4(w[0], w[1], w[2], w[3]);
      }
      arrive(bar(RAW_EMPTY + s));                    // the line slot is read
#pragma unroll
      for (int j = 0; j < 4; ++j)
        *reinterpret_cast<uint4*>(B1 + g * B1_LBO + ((2 * j + h) * 16 + n1) * 16) = pkd[j];
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      arrive(bar(B1_FULL + s));
    }
  } else if (warp == W_COPY) {
    for (int k = 0; k < nk; ++k) {
      const int s = k & 1;
      if (!warp_wait(bar(RAW_EMPTY + s), ((k >> 1) & 1) ^ 1, fail)) break;
      fetch_tile(a, tile_of(k), su32(sm + OFF_RAW + s * RAW_BYTES),
                 su32(sm + OFF_RAW + s * RAW_BYTES + RX_BYTES), bar(RAW_FULL + s), lane);
      if (lane == 0) s_copies = k + 1;
    }
  } else if (warp == W_MMA && lane == 0) {
    const uint32_t a1 = su32(A1), b2 = su32(B2);
    for (int k = 0; k <= nk; ++k) {
      if (k < nk) {                                  // stage 1 of tile k
        const int s = k & 1;
        const uint32_t ph = (k >> 1) & 1;
        if (!role_wait(bar(B1_FULL + s), ph, fail) || !role_wait(bar(D1_EMPTY + s), ph ^ 1, fail))
          break;
        fence_after();
        const uint32_t b1 = su32(sm + OFF_B1 + s * B1_BYTES), d1 = tmem + D1_COL + (uint32_t)(128 * s);
#pragma unroll
        for (int st = 0; st < 4; ++st)
          mma(d1, mdesc(a1 + 2 * st * A1_LBO, A1_LBO, 128), mdesc(b1 + 2 * st * B1_LBO, B1_LBO, 128),
              idesc(128, 128), st > 0);
        commit(bar(D1_FULL + s));
        commit(bar(B1_EMPTY + s));
        s_mma1 = k + 1;
      }
      if (k >= 1) {                                  // stage 2 of tile k - 1
        const int j = k - 1, s = j & 1;
        const uint32_t ph = (j >> 1) & 1;
        if (!role_wait(bar(A2_FULL + s), ph, fail) || !role_wait(bar(D2_EMPTY + s), ph ^ 1, fail))
          break;
        fence_after();
        const uint32_t a2 = su32(sm + OFF_A2 + s * A2_BYTES);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int st = 0; st < 2; ++st)
            mma(tmem + D2_COL + (uint32_t)(64 * s + 32 * mt),
                mdesc(a2 + mt * A2_TILE + 2 * st * A2_LBO, A2_LBO, 128),
                mdesc(b2 + 2 * st * B2_LBO, B2_LBO, 128), idesc(128, 32), st > 0);
        commit(bar(D2_FULL + s));
        commit(bar(A2_EMPTY + s));
        s_mma2 = j + 1;
      }
    }
  }

  __syncthreads();
  if (s_fail) {
    // a wait ran out: let the copies and MMAs still in flight land (bounded)
    // before TMEM is freed and the CTA's shared memory released
    if (tid == 0) {
      atomicOr(&g_dft_err, 1u);
      for (int s = 0; s < 2; ++s) {
        const int kc = s_copies - 1 - ((s_copies - 1 - s) & 1);   // last copied tile in slot s
        if (kc >= 0) wait_bounded(bar(RAW_FULL + s), (kc >> 1) & 1);
      }
      if (s_mma1 > 0) wait_bounded(bar(D1_FULL + ((s_mma1 - 1) & 1)), ((s_mma1 - 1) >> 1) & 1);
      if (s_mma2 > 0) wait_bounded(bar(D2_FULL + ((s_mma2 - 1) & 1)), ((s_mma2 - 1) >> 1) & 1);
    }
    __syncthreads();
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TD_COLS)
                 : "memory");
}

}  // namespace

// 512-point columns; planes with fewer than 8 stored column frequencies keep
// the CUDA-core pass (the range the pass is tested on).
bool dec_lines_tc_supported(int N, int Mh) { return N == TD_N && Mh >= TD_LINES; }

cudaError_t launch_dec_lines_tc(int N, const float2* X, void* out, const float* G,
                                const float* invW, float scale, int Mh, int K, int s0, int S,
                                const float2* tw, cudaStream_t st, int nimg, bool s16) {
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
  DftArgs a{X, out, G, invW, tw, scale, Mh, K, s0, nimg, s16 ? 1 : 0};
  // tiles: per image of the chunk, groups of 4 of its subbands x pairs of
  // column frequencies (the groups start at the image's first subband)
  a.S = S;
  a.b_lo = s0 / K;
  a.npairs = (Mh + 1) / 2;
  a.gmax = 0;
  for (int b = a.b_lo; b <= (s0 + S - 1) / K; ++b) {
    const int sa = std::max(s0, b * K), sb = std::min(s0 + S, (b + 1) * K);
    a.gmax = std::max(a.gmax, (sb - sa + 3) / 4);
  }
  const long long nt = (long long)((s0 + S - 1) / K - a.b_lo + 1) * a.gmax * a.npairs;
  if (nt > 0x7fffffffLL) return cudaErrorInvalidValue;
  a.ntiles = (int)nt;
  const int ntiles = a.ntiles;
  const int grid = ntiles < nsm[dev] ? ntiles : nsm[dev];   // one CTA per SM
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
