// nn_tc.cu - 3x3 convolutions of the learned parts on the tensor cores
// (tcgen05, bfloat16 operands, float32 accumulation in tensor memory).
//
// Implicit GEMM per tile of 128 consecutive output pixels of one image row:
//   D[m][n] = sum_{tap, ci} P_tap[m][ci] * W_tap[n][ci]
// with P_tap[m][ci] = in[ci][y + dy - 1][x0 + m + dx - 1] (zero padding).
// The CTA stages input rows as bfloat16 in the no-swizzle K-major
// core-matrix layout [ci/8][pixel][8 ci] (16 bytes per pixel and channel
// group), loading groups of 4 pixels (float4, or two float2 when the width is
// not a multiple of 4), into a ring of four rows.  Consecutive pixels are 16 bytes apart, so
// the A operand of tap (dy, dx) is the same staged rows with its start
// address moved by dx * 16 bytes: no im2col copy.  The weights sit in the
// same layout [tap][ci/8][n][8 ci] for the whole launch.  One thread issues
// the 9 * Ci/16 MMAs (M = 128, N = Cout padded to 16, K = 16) into a TMEM
// accumulator and commits them to an mbarrier; warps w and w + 4 then read
// TMEM lanes 32 (w % 4) .. + 31 (= pixels), each one half of the columns
// (= output channels), and store the NCHW output rows.  The wait
// on the mbarrier is bounded: when it runs out the kernel records the
// error (read by shl_nn_tc_status), frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>

#include "../../include/shearlet_nn.h"

namespace {

__device__ unsigned int g_tc_err = 0;

constexpr int TC_M = 128;            // output pixels per tile (MMA M)
constexpr int CONV_THREADS = 256;    // warps w and w + 4 share TMEM lanes 32 (w % 4)
// Staged pixels per row: x0 - 4 .. x0 + 131 (x0 a multiple of 128), in groups
// of 4 (load4: zero outside the row, so the last tile of a row whose width
// is not a multiple of 128 is ragged); output pixel m, tap dx reads staged
// pixel m + dx + 3.  Widths are even (float2 halves stay 8-byte aligned).
constexpr int PW = TC_M + 8;
constexpr int PX0 = 3;
constexpr unsigned TC_SPIN_LIMIT = 1u << 22;

struct ConvTcArgs {
  const float* in;      // [B][Cin][H][W]
  const float* w;       // forward: [Cout][Cin][3][3]; flip: [Cin][Cout][3][3]
  const float* bias;    // [Cout] or null
  float* out;           // [B][Cout][H][W]
  int B, Cin, Cout, H, W;
  int flip;             // 1: convolution with the flipped, channel-transposed weights
  int rows_per_unit;    // output rows one CTA walks down per unit
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of tcgen05, no swizzle: start address,
// leading-dimension byte offset (between core matrices along K), stride
// byte offset (between 8-row groups along M or N), descriptor version 1.
__device__ __forceinline__ uint64_t mdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: float32 accumulator, bfloat16 A and
// B, both K-major, N and M.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float wval(const ConvTcArgs& a, int n, int k, int dy, int dx) {
  // n: output channel, k: input channel of this convolution
  return a.flip ? __ldg(a.w + (((size_t)k * a.Cout + n) * 3 + (2 - dy)) * 3 + (2 - dx))
                : __ldg(a.w + (((size_t)n * a.Cin + k) * 3 + dy) * 3 + dx);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  for (unsigned i = 0; i < TC_SPIN_LIMIT; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

#define SHL_TMEM_LD16(R, ADDR)                                                              \
  asm volatile(                                                                             \
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "                                             \
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"                     \
      : "=r"((R)[0]), "=r"((R)[1]), "=r"((R)[2]), "=r"((R)[3]), "=r"((R)[4]), "=r"((R)[5]), \
        "=r"((R)[6]), "=r"((R)[7]), "=r"((R)[8]), "=r"((R)[9]), "=r"((R)[10]),              \
        "=r"((R)[11]), "=r"((R)[12]), "=r"((R)[13]), "=r"((R)[14]), "=r"((R)[15])           \
      : "r"(ADDR)                                                                           \
      : "memory")

#define SHL_TMEM_LD8(R, ADDR)                                                               \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"      \
               : "=r"((R)[0]), "=r"((R)[1]), "=r"((R)[2]), "=r"((R)[3]), "=r"((R)[4]),         \
                 "=r"((R)[5]), "=r"((R)[6]), "=r"((R)[7])                                      \
               : "r"(ADDR)                                                                     \
               : "memory")

template <int CG, int NP>
struct ConvTcT {
  static_assert(CG % 2 == 0 && NP % 16 == 0 && NP >= 16 && NP <= 128, "tile shape");
  static constexpr int KS = CG / 2;                          // K steps of 16 per tap
  static constexpr int SLOTS = 4;                            // input-row ring
  static constexpr size_t WBYTES = (size_t)9 * CG * NP * 16;  // [tap][cg][n][8]
  static constexpr size_t RBYTES = (size_t)CG * PW * 16;      // one row: [cg][px][8]
  static constexpr size_t SMEM = WBYTES + SLOTS * RBYTES;    // descriptors stay inside
  static constexpr uint32_t NCOLS = NP <= 32 ? 32 : (NP <= 64 ? 64 : 128);   // TMEM columns (power of 2)
  // two CTAs per SM where their shared memory fits (228 KB, 1 KB reserved each)
  static constexpr int MINB = 2 * (SMEM + 1024) <= 228 * 1024 ? 2 : 1;
};

// Staging of one input row in two halves (global loads into registers, then
// bfloat16 conversion and shared-memory stores), so that the loads of the
// next row are in flight while the current row's MMAs and epilogue run.
// Row gy of image b, pixels x0-4..x0+131 -> bfloat16 [cg][px][8]; one item =
// 4 pixels x 8 channels (8 float4 loads, 4 16-byte stores); zeros outside the
// image.
template <int CG>
struct ConvRegs {
  static constexpr int ITEMS = (CG * (PW / 4) + CONV_THREADS - 1) / CONV_THREADS;
  float4 v[ITEMS][8];
};

// Pixels gx .. gx + 3 (gx a multiple of 4) of the row starting at `row`, zero
// outside 0 .. W - 1: one float4 when W is a multiple of 4 (the group then
// lies wholly inside or wholly outside the row), else (W even, rows 8-byte
// aligned) two float2 halves, each wholly inside or outside.
__device__ __forceinline__ float4 load4(const float* row, int gx, int W) {
  if ((W & 3) == 0)
    return gx >= 0 && gx < W ? __ldg(reinterpret_cast<const float4*>(row + gx))
                             : make_float4(0.f, 0.f, 0.f, 0.f);
  const float2 lo = gx >= 0 && gx < W ? __ldg(reinterpret_cast<const float2*>(row + gx))
                                      : make_float2(0.f, 0.f);
  const float2 hi = gx + 2 >= 0 && gx + 2 < W ? __ldg(reinterpret_cast<const float2*>(row + gx + 2))
                                              : make_float2(0.f, 0.f);
  return make_float4(lo.x, lo.y, hi.x, hi.y);
}

template <int CG>
__device__ __forceinline__ void conv_load_row(const ConvTcArgs& a, ConvRegs<CG>& R, int b, int gy,
                                              int x0, int tid) {
  constexpr int PG = PW / 4;
  const size_t cs = (size_t)a.H * a.W;
  const bool rok = gy >= 0 && gy < a.H;
#pragma unroll
  for (int k = 0; k < ConvRegs<CG>::ITEMS; ++k) {
    const int idx = tid + k * CONV_THREADS;
    const int cg = idx / PG, q = idx - cg * PG;
    const int gx = x0 - 4 + 4 * q;
    const bool ok = rok && idx < CG * PG;
    const float* row = a.in + (((size_t)b * a.Cin + cg * 8) * a.H + (ok ? gy : 0)) * a.W;
#pragma unroll
    for (int c = 0; c < 8; ++c)
      R.v[k][c] = (ok && cg * 8 + c < a.Cin) ? load4(row + c * cs, gx, a.W)
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

template <int CG>
__device__ __forceinline__ void conv_store_row(const ConvRegs<CG>& R, uint8_t* dst, int tid) {
  constexpr int PG = PW / 4;
#pragma unroll
  for (int k = 0; k < ConvRegs<CG>::ITEMS; ++k) {
    const int idx = tid + k * CONV_THREADS;
    if (idx < CG * PG) {
      const int cg = idx / PG, q = idx - cg * PG;
      const float4* v = R.v[k];
      uint8_t* d = dst + ((size_t)cg * PW + 4 * q) * 16;
      *reinterpret_cast<uint4*>(d) =
          make_uint4(pack_bf16(v[0].x, v[1].x), pack_bf16(v[2].x, v[3].x),
                     pack_bf16(v[4].x, v[5].x), pack_bf16(v[6].x, v[7].x));
      *reinterpret_cast<uint4*>(d + 16) =
          make_uint4(pack_bf16(v[0].y, v[1].y), pack_bf16(v[2].y, v[3].y),
                     pack_bf16(v[4].y, v[5].y), pack_bf16(v[6].y, v[7].y));
      *reinterpret_cast<uint4*>(d + 32) =
          make_uint4(pack_bf16(v[0].z, v[1].z), pack_bf16(v[2].z, v[3].z),
                     pack_bf16(v[4].z, v[5].z), pack_bf16(v[6].z, v[7].z));
      *reinterpret_cast<uint4*>(d + 48) =
          make_uint4(pack_bf16(v[0].w, v[1].w), pack_bf16(v[2].w, v[3].w),
                     pack_bf16(v[4].w, v[5].w), pack_bf16(v[6].w, v[7].w));
    }
  }
}

// A CTA takes units of (image, 128-pixel column, run of a.rows_per_unit
// rows) and walks down the rows with a ring of four staged input rows: row
// y + 2 is staged while the MMAs of row y run, so each output row costs one
// new input row.
template <int CG, int NP>
__global__ void __launch_bounds__(CONV_THREADS, (ConvTcT<CG, NP>::MINB)) k_conv3x3_tc(ConvTcArgs a) {
  using P = ConvTcT<CG, NP>;
  extern __shared__ __align__(128) uint8_t sm[];
  uint8_t* wsm = sm;
  uint8_t* ring = sm + P::WBYTES;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // weights -> bfloat16 [tap][cg][n][8], zero beyond Cin / Cout
  for (int idx = tid; idx < 9 * CG * NP; idx += CONV_THREADS) {
    const int t = idx / (CG * NP), rem = idx - t * CG * NP, cg = rem / NP, n = rem - cg * NP;
    const int dy = t / 3, dx = t - dy * 3;
    uint32_t pk[4];
#pragma unroll
    for (int c = 0; c < 8; c += 2) {
      const int k0 = cg * 8 + c;
      const float v0 = (n < a.Cout && k0 < a.Cin) ? wval(a, n, k0, dy, dx) : 0.f;
      const float v1 = (n < a.Cout && k0 + 1 < a.Cin) ? wval(a, n, k0 + 1, dy, dx) : 0.f;
      pk[c / 2] = pack_bf16(v0, v1);
    }
    *reinterpret_cast<uint4*>(wsm + (size_t)idx * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(P::NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_bf16(TC_M, NP);
  const uint32_t wbase = smem_u32(wsm), rbase = smem_u32(ring);
  const size_t cs = (size_t)a.H * a.W;

  const int tiles_x = (a.W + TC_M - 1) / TC_M;
  const int RU = a.rows_per_unit;
  const int runs = (a.H + RU - 1) / RU;
  const int nunits = a.B * tiles_x * runs;
  uint32_t phase = 0;
  ConvRegs<CG> R;
  for (int u = blockIdx.x; u < nunits && !s_fail; u += gridDim.x) {
    const int b = u / (tiles_x * runs), rem = u - b * tiles_x * runs;
    const int xt = rem / runs, y0 = (rem - xt * runs) * RU, y1 = min(a.H, y0 + RU);
    const int x0 = xt * TC_M;
    // the three rows of the first output row (the previous unit's MMAs are
    // done), then the loads of row y0 + 2 start
    for (int gy = y0 - 1; gy <= y0 + 1; ++gy) {
      conv_load_row<CG>(a, R, b, gy, x0, tid);
      conv_store_row<CG>(R, ring + (size_t)((gy + 4) & 3) * P::RBYTES, tid);
    }
    if (y0 + 1 < y1) conv_load_row<CG>(a, R, b, y0 + 2, x0, tid);
    for (int y = y0; y < y1; ++y) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // staged rows -> async proxy
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
#pragma unroll
        for (int t = 0; t < 9; ++t) {
          const int dy = t / 3, dx = t - dy * 3;
          const uint32_t row = rbase + (uint32_t)(((y + dy - 1 + 4) & 3) * P::RBYTES);
#pragma unroll
          for (int s = 0; s < P::KS; ++s) {
            const uint64_t ad = mdesc(row + (uint32_t)(((2 * s) * PW + dx + PX0) * 16), PW * 16, 128);
            const uint64_t bd = mdesc(wbase + (uint32_t)(((t * CG + 2 * s) * NP) * 16), NP * 16, 128);
            const uint32_t acc = (t | s) != 0;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
          }
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar))
            : "memory");
      }
      // row y + 2 (loaded last iteration) goes to the slot of row y - 2, which
      // no MMA in flight reads; then the loads of row y + 3 start
      if (y + 1 < y1) {
        conv_store_row<CG>(R, ring + (size_t)((y + 2) & 3) * P::RBYTES, tid);
        if (y + 2 < y1) conv_load_row<CG>(a, R, b, y + 3, x0, tid);
      }
      if (!mbar_wait(smem_u32(&mbar), phase)) {
        atomicOr(&g_tc_err, 1u);
        s_fail = 1;
      }
      phase ^= 1u;
      __syncthreads();
      if (s_fail) break;
      tc_fence_after();
      // warp w reads TMEM lanes 32 (w % 4) .. + 31 (= pixels), columns
      // (w / 4) NP/2 .. + NP/2 - 1 (= output channels)
      constexpr int HC = NP / 2;
      const int quarter = warp & 3, n0 = (warp >> 2) * HC;
      uint32_t acc[HC];
#pragma unroll
      for (int q = 0; q < HC / 8; ++q)
        SHL_TMEM_LD8(acc + 8 * q, tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(n0 + 8 * q));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const int px = x0 + quarter * 32 + lane;     // the last tile of a row may be ragged
      float* o = a.out + (((size_t)b * a.Cout) * a.H + y) * a.W + px;
#pragma unroll
      for (int n = 0; n < HC; ++n) {
        const int ch = n0 + n;
        if (ch < a.Cout && px < a.W)
          o[ch * cs] = __uint_as_float(acc[n]) + (a.bias ? __ldg(a.bias + ch) : 0.f);
      }
      tc_fence_before();   // TMEM reads done before the next row's MMAs (barrier at loop top)
    }
    __syncthreads();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(P::NCOLS)
                 : "memory");
}

// ----------------------------------------------------------- weight gradient
// gw[o][i][dy][dx] = sum_{b,y,x} gout[b][o][y][x] in[b][i][y+dy-1][x+dx-1].
// Per unit of 128 consecutive pixels of one row (K = pixels, 16 per MMA):
//   A_dy[r][p] = in[i][y+dy-1][x0+p+dx-1], r = dx * Cin + i  (3 Cin <= 128 rows)
//   B[o][p]    = gout[o][y][x0+p]                             (NP rows)
//   D_dy[r][o] += sum_p A_dy[r][p] B[o][p]                    (TMEM columns dy * NP + o)
// both staged as bfloat16 K-major core matrices [pixel/8][row][8 pixels].
// A CTA accumulates all its units in TMEM and writes one partial
// gw[o][i][dy][dx]; k_wgrad_reduce sums the partials in CTA order.
struct WgradTcArgs {
  const float* in;      // [B][Cin][H][W]
  const float* gout;    // [B][Cout][H][W]
  float* part;          // [gridDim.x][Cout * Cin * 9 + Cout]: weight then bias partials
  int B, Cin, Cout, H, W;
  int rows_per_unit;    // output rows one CTA walks down per unit
};

template <int NP>
struct WgradTcT {
  static constexpr int THREADS = 256;                       // 8 warps stage, 4 read TMEM
  static constexpr int PG = TC_M / 8;                       // pixel groups per unit row
  static constexpr int SLOTS = 4;                           // input-row ring
  static constexpr size_t ABYTES = (size_t)PG * 128 * 16;   // one input row: [pg][r][8]
  static constexpr size_t BBYTES = (size_t)PG * NP * 16;    // one gout row: [pg][o][8]
  static constexpr size_t SMEM = SLOTS * ABYTES + 2 * BBYTES;
  static constexpr uint32_t NCOLS =
      3 * NP <= 64 ? 64 : (3 * NP <= 128 ? 128 : (3 * NP <= 256 ? 256 : 512));
  static constexpr int BITEMS = (NP * PG + THREADS - 1) / THREADS;   // gout items per thread
  static constexpr int IITEMS = (42 * PG + THREADS - 1) / THREADS;   // input items (Cin <= 42)
};

// Staging of the weight-gradient operands in two halves, so that the global
// loads of the next rows are in flight while the MMAs of the current row
// run: *_load fills registers, *_store converts them to bfloat16 and writes
// shared memory.  Item idx -> (pixel group pg = idx / C, channel idx % C):
// consecutive threads write consecutive 16-byte rows (no bank conflicts).
template <int NP>
struct WgradRegs {
  float e[WgradTcT<NP>::IITEMS][10];     // input: pixels x0+8pg-1 .. x0+8pg+8
  float4 g[WgradTcT<NP>::BITEMS][2];     // gout: pixels x0+8pg .. x0+8pg+7
};

template <int NP>
__device__ __forceinline__ void wgrad_load_in(const WgradTcArgs& a, WgradRegs<NP>& R, int b, int gy,
                                              int x0, int tid) {
  using P = WgradTcT<NP>;
  const bool rok = gy >= 0 && gy < a.H;
#pragma unroll
  for (int k = 0; k < P::IITEMS; ++k) {
    const int idx = tid + k * P::THREADS;
    float* e = R.e[k];
    if (rok && idx < a.Cin * P::PG) {
      const int pg = idx / a.Cin, i = idx - pg * a.Cin;
      const int xs = x0 + 8 * pg;
      const float* row = a.in + (((size_t)b * a.Cin + i) * a.H + gy) * a.W;
      if ((a.W & 3) == 0 && xs + 8 <= a.W) {
        const float4 v0 = __ldg(reinterpret_cast<const float4*>(row + xs));
        const float4 v1 = __ldg(reinterpret_cast<const float4*>(row + xs + 4));
        e[0] = xs > 0 ? __ldg(row + xs - 1) : 0.f;
        e[1] = v0.x; e[2] = v0.y; e[3] = v0.z; e[4] = v0.w;
        e[5] = v1.x; e[6] = v1.y; e[7] = v1.z; e[8] = v1.w;
        e[9] = xs + 8 < a.W ? __ldg(row + xs + 8) : 0.f;
      } else {                       // ragged last tile, or rows not 16-byte aligned
#pragma unroll
        for (int j = 0; j < 10; ++j) {
          const int x = xs - 1 + j;
          e[j] = x >= 0 && x < a.W ? __ldg(row + x) : 0.f;
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < 10; ++c) e[c] = 0.f;
    }
  }
}

// -> the three shifted copies A[r = dx * Cin + i][p] = in[i][gy][x0 + p + dx - 1]
template <int NP>
__device__ __forceinline__ void wgrad_store_in(const WgradTcArgs& a, const WgradRegs<NP>& R,
                                               uint8_t* dst, int tid) {
  using P = WgradTcT<NP>;
#pragma unroll
  for (int k = 0; k < P::IITEMS; ++k) {
    const int idx = tid + k * P::THREADS;
    if (idx < a.Cin * P::PG) {
      const int pg = idx / a.Cin, i = idx - pg * a.Cin;
      const float* e = R.e[k];
      uint8_t* d = dst + ((size_t)pg * 128 + i) * 16;
#pragma unroll
      for (int dx = 0; dx < 3; ++dx)   // pixel x0+8pg+j-1+dx = e[j + dx]
        *reinterpret_cast<uint4*>(d + (size_t)dx * a.Cin * 16) =
            make_uint4(pack_bf16(e[dx], e[dx + 1]), pack_bf16(e[dx + 2], e[dx + 3]),
                       pack_bf16(e[dx + 4], e[dx + 5]), pack_bf16(e[dx + 6], e[dx + 7]));
    }
  }
}

template <int NP>
__device__ __forceinline__ void wgrad_load_gout(const WgradTcArgs& a, WgradRegs<NP>& R, int b,
                                                int y, int x0, int tid) {
  using P = WgradTcT<NP>;
#pragma unroll
  for (int k = 0; k < P::BITEMS; ++k) {
    const int idx = tid + k * P::THREADS;
    if (idx < a.Cout * P::PG) {
      const int pg = idx / a.Cout, o = idx - pg * a.Cout;
      const int xs = x0 + 8 * pg;
      const float* row = a.gout + (((size_t)b * a.Cout + o) * a.H + y) * a.W;
      if ((a.W & 3) == 0 && xs + 8 <= a.W) {
        R.g[k][0] = __ldg(reinterpret_cast<const float4*>(row + xs));
        R.g[k][1] = __ldg(reinterpret_cast<const float4*>(row + xs + 4));
      } else {                       // ragged last tile, or rows not 16-byte aligned
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = xs + j < a.W ? __ldg(row + xs + j) : 0.f;
        R.g[k][0] = make_float4(v[0], v[1], v[2], v[3]);
        R.g[k][1] = make_float4(v[4], v[5], v[6], v[7]);
      }
    }
  }
}

// -> B[o][p] = gout[o][y][x0 + p]; bsum[k] gathers this thread's float32
// bias partial (item k always has channel (tid + k THREADS) mod Cout)
template <int NP>
__device__ __forceinline__ void wgrad_store_gout(const WgradTcArgs& a, const WgradRegs<NP>& R,
                                                 uint8_t* dst, int tid,
                                                 float (&bsum)[WgradTcT<NP>::BITEMS]) {
  using P = WgradTcT<NP>;
#pragma unroll
  for (int k = 0; k < P::BITEMS; ++k) {
    const int idx = tid + k * P::THREADS;
    if (idx < a.Cout * P::PG) {
      const int pg = idx / a.Cout, o = idx - pg * a.Cout;
      const float4 v0 = R.g[k][0], v1 = R.g[k][1];
      bsum[k] += ((v0.x + v0.y) + (v0.z + v0.w)) + ((v1.x + v1.y) + (v1.z + v1.w));
      *reinterpret_cast<uint4*>(dst + ((size_t)pg * NP + o) * 16) =
          make_uint4(pack_bf16(v0.x, v0.y), pack_bf16(v0.z, v0.w), pack_bf16(v1.x, v1.y),
                     pack_bf16(v1.z, v1.w));
    }
  }
}

// A CTA takes units of (image, 128-pixel column, run of a.rows_per_unit
// output rows) and walks down the rows: input rows in a ring of four slots
// (row y + 2 staged while the MMAs of row y run), gout rows double-buffered;
// every MMA of the launch accumulates into the same three TMEM tiles.
template <int NP>
__global__ void __launch_bounds__(WgradTcT<NP>::THREADS, 1) k_wgrad_tc(WgradTcArgs a) {
  using P = WgradTcT<NP>;
  extern __shared__ __align__(128) uint8_t sm[];
  uint8_t* As = sm;                           // SLOTS x [pg][128][8]
  uint8_t* Bs = sm + P::SLOTS * P::ABYTES;    // 2 x [pg][NP][8]
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // rows r >= 3 Cin and o >= Cout stay zero for the whole launch
  for (size_t q = tid; q < P::SMEM / 16; q += P::THREADS)
    reinterpret_cast<uint4*>(sm)[q] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(P::NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_bf16(TC_M, NP);
  const uint32_t abase = smem_u32(As), bbase = smem_u32(Bs);
  const int tiles_x = (a.W + TC_M - 1) / TC_M;
  const int RU = a.rows_per_unit;
  const int runs = (a.H + RU - 1) / RU;
  const int nunits = a.B * tiles_x * runs;
  uint32_t phase = 0;
  bool first = true;
  float bsum[P::BITEMS];   // bias partials of this thread's fixed gout items, float32
#pragma unroll
  for (int k = 0; k < P::BITEMS; ++k) bsum[k] = 0.f;
  WgradRegs<NP> R;

  for (int u = blockIdx.x; u < nunits && !s_fail; u += gridDim.x) {
    const int b = u / (tiles_x * runs), rem = u - b * tiles_x * runs;
    const int xt = rem / runs, y0 = (rem - xt * runs) * RU, y1 = min(a.H, y0 + RU);
    const int x0 = xt * TC_M;
    // the previous unit's MMAs are done: stage rows y0-1..y0+1 and gout row
    // y0, then start the loads of input row y0+2 and gout row y0+1
    for (int gy = y0 - 1; gy <= y0 + 1; ++gy) {
      wgrad_load_in<NP>(a, R, b, gy, x0, tid);
      wgrad_store_in<NP>(a, R, As + (size_t)((gy + 4) & 3) * P::ABYTES, tid);
    }
    wgrad_load_gout<NP>(a, R, b, y0, x0, tid);
    wgrad_store_gout<NP>(a, R, Bs + (size_t)(y0 & 1) * P::BBYTES, tid, bsum);
    if (y0 + 1 < y1) {
      wgrad_load_in<NP>(a, R, b, y0 + 2, x0, tid);
      wgrad_load_gout<NP>(a, R, b, y0 + 1, x0, tid);
    }
    for (int y = y0; y < y1; ++y) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
          const uint32_t arow = abase + (uint32_t)(((y + dy - 1 + 4) & 3) * P::ABYTES);
          const uint32_t brow = bbase + (uint32_t)((y & 1) * P::BBYTES);
#pragma unroll
          for (int s = 0; s < P::PG / 2; ++s) {
            const uint64_t ad = mdesc(arow + (uint32_t)(2 * s * 128 * 16), 128 * 16, 128);
            const uint64_t bd = mdesc(brow + (uint32_t)(2 * s * NP * 16), NP * 16, 128);
            const uint32_t acc = (first && s == 0) ? 0u : 1u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
                    tmem + (uint32_t)(dy * NP)),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
          }
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar))
            : "memory");
      }
      first = false;
      // the rows loaded last iteration go to slots no MMA in flight reads:
      // input row y + 2 to the slot of row y - 2, gout row y + 1 to the other
      // B buffer (row y - 1's); then the loads of the rows after them start
      if (y + 1 < y1) {
        wgrad_store_in<NP>(a, R, As + (size_t)((y + 2) & 3) * P::ABYTES, tid);
        wgrad_store_gout<NP>(a, R, Bs + (size_t)((y + 1) & 1) * P::BBYTES, tid, bsum);
        if (y + 2 < y1) {
          wgrad_load_in<NP>(a, R, b, y + 3, x0, tid);
          wgrad_load_gout<NP>(a, R, b, y + 2, x0, tid);
        }
      }
      if (!mbar_wait(smem_u32(&mbar), phase)) {
        atomicOr(&g_tc_err, 1u);
        s_fail = 1;
      }
      phase ^= 1u;
      __syncthreads();
      if (s_fail) break;
    }
    __syncthreads();
  }
  // bias partial of this CTA: item partials through shared memory (the
  // staging area is free: every MMA has completed), summed per channel in
  // pixel-group order
  float* bred = reinterpret_cast<float*>(sm);
#pragma unroll
  for (int k = 0; k < P::BITEMS; ++k) {
    const int idx = tid + k * P::THREADS;
    if (idx < a.Cout * P::PG) bred[idx] = bsum[k];
  }
  __syncthreads();
  const size_t stride = (size_t)a.Cout * a.Cin * 9 + a.Cout;
  if (tid < a.Cout) {   // items of channel o: idx = pg * Cout + o
    float s = 0.f;
    for (int pg = 0; pg < P::PG; ++pg) s += bred[pg * a.Cout + tid];
    a.part[(size_t)blockIdx.x * stride + (size_t)a.Cout * a.Cin * 9 + tid] = s;
  }
  // epilogue (warps 0-3): lane r = dx * Cin + i, columns dy * NP + o
  if (!s_fail && warp < 4) {
    tc_fence_after();
    const int r = warp * 32 + lane;
    const int dx = r / a.Cin, i = r - dx * a.Cin;
    float* part = a.part + (size_t)blockIdx.x * stride;
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
#pragma unroll 1
      for (int q = 0; q < NP / 16; ++q) {          // 16 columns (output channels) at a time
        uint32_t acc[16];
        SHL_TMEM_LD16(acc, tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(dy * NP + 16 * q));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (dx < 3) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int o = 16 * q + j;
            if (o < a.Cout)
              part[(((size_t)o * a.Cin + i) * 3 + dy) * 3 + dx] =
                  blockIdx.x < nunits ? __uint_as_float(acc[j]) : 0.f;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(P::NCOLS)
                 : "memory");
}

// Sum the per-CTA partials in CTA order: entries e < nw are the weight
// gradient, the next Cout the bias gradient (written only if gb != null).
__global__ void k_wgrad_reduce(const float* __restrict__ part, float* __restrict__ gw,
                               float* __restrict__ gb, int nparts, int nw, int nb) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = nw + nb;
  if (e >= n) return;
  float s = 0.f;
  for (int c = 0; c < nparts; ++c) s += part[(size_t)c * n + e];
  if (e < nw) gw[e] = s;
  else if (gb) gb[e - nw] = s;
}

// One CTA per SM (the row ring takes ~150 KB of shared memory); rows per
// unit: about four units per CTA, 4..32 rows.
void wgrad_plan(int B, int H, int W, int* grid, int* rows_per_unit) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  sms = std::max(sms, 1);
  const long long strips = (long long)B * ((W + TC_M - 1) / TC_M);
  const int ru = (int)std::min<long long>(
      H, std::max(4LL, std::min(32LL, strips * H / std::max(1LL, 4LL * sms))));
  const long long nunits = strips * ((H + ru - 1) / ru);
  *grid = (int)std::max(1LL, std::min(nunits, (long long)sms));
  *rows_per_unit = ru;
}

template <int NP>
cudaError_t launch_wgrad(const WgradTcArgs& a, int grid, cudaStream_t st) {
  using P = WgradTcT<NP>;
  static_assert(P::SMEM + 1024 > 228 * 1024 / 2, "one CTA per SM keeps TMEM use at NCOLS");
  auto k = k_wgrad_tc<NP>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::SMEM);
  if (e) return e;
  k<<<grid, P::THREADS, P::SMEM, st>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------- warp-specialised forward conv
// The same convolution as k_conv3x3_tc with the roles split between warps
// and handed over through mbarriers, so that loads, MMAs and stores of
// different rows overlap:
//   warps 5..7 (producers)  stage input rows into a ring of WS_SLOTS slots;
//                           slot s: full[s] (96 producer arrivals) /
//                           empty[s] (released by the MMA commit of the
//                           last output row that reads it);
//   warp 4, lane 0 (MMA)    per output row waits for its three rows and a
//                           free accumulator, issues the 9 Ci/16 MMAs into
//                           one of two TMEM accumulators, commits to
//                           accf[buffer] and to empty[] of the row it no
//                           longer needs;
//   warps 0..3 (epilogue)   wait accf, read their 32 TMEM lanes, add the
//                           bias, store the NCHW row, arrive on acce.
// Every wait is bounded; on a timeout the role records the error and
// leaves its loop, the MMA thread drains its MMAs, and the CTA frees TMEM.
constexpr int WS_SLOTS = 6;
constexpr int WS_PROD = 96;   // producer threads (warps 5..7)

template <int CG, int NP>
struct ConvWsT {
  static constexpr size_t WBYTES = (size_t)9 * CG * NP * 16;
  static constexpr size_t RBYTES = (size_t)CG * PW * 16;
  static constexpr size_t SMEM = WBYTES + WS_SLOTS * RBYTES;
  static constexpr uint32_t NCOLS = 2 * NP <= 32 ? 32 : (2 * NP <= 64 ? 64 : 128);
};

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(b))
               : "memory");
}

// One input row (pixels x0-4..x0+131, bfloat16 [cg][px][8]) staged by the 96
// producer threads, two items of 4 pixels x 8 channels in flight per thread.
template <int CG>
__device__ __forceinline__ void ws_stage_row(const ConvTcArgs& a, uint8_t* dst, int b, int gy,
                                             int x0, int ptid) {
  constexpr int PG = PW / 4, NI = CG * PG;
  const size_t cs = (size_t)a.H * a.W;
  const bool rok = gy >= 0 && gy < a.H;
  for (int base = ptid; base < NI; base += 2 * WS_PROD) {
    float4 v[2][8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int idx = base + h * WS_PROD;
      const int cg = idx / PG, q = idx - cg * PG;
      const int gx = x0 - 4 + 4 * q;
      const bool ok = rok && idx < NI && gx >= 0 && gx < a.W;
      const float* src =
          a.in + (((size_t)b * a.Cin + cg * 8) * a.H + (ok ? gy : 0)) * a.W + (ok ? gx : 0);
#pragma unroll
      for (int c = 0; c < 8; ++c)
        v[h][c] = (ok && cg * 8 + c < a.Cin) ? __ldg(reinterpret_cast<const float4*>(src + c * cs))
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int idx = base + h * WS_PROD;
      if (idx < NI) {
        const int cg = idx / PG, q = idx - cg * PG;
        const float4* w = v[h];
        uint8_t* d = dst + ((size_t)cg * PW + 4 * q) * 16;
        *reinterpret_cast<uint4*>(d) =
            make_uint4(pack_bf16(w[0].x, w[1].x), pack_bf16(w[2].x, w[3].x),
                       pack_bf16(w[4].x, w[5].x), pack_bf16(w[6].x, w[7].x));
        *reinterpret_cast<uint4*>(d + 16) =
            make_uint4(pack_bf16(w[0].y, w[1].y), pack_bf16(w[2].y, w[3].y),
                       pack_bf16(w[4].y, w[5].y), pack_bf16(w[6].y, w[7].y));
        *reinterpret_cast<uint4*>(d + 32) =
            make_uint4(pack_bf16(w[0].z, w[1].z), pack_bf16(w[2].z, w[3].z),
                       pack_bf16(w[4].z, w[5].z), pack_bf16(w[6].z, w[7].z));
        *reinterpret_cast<uint4*>(d + 48) =
            make_uint4(pack_bf16(w[0].w, w[1].w), pack_bf16(w[2].w, w[3].w),
                       pack_bf16(w[4].w, w[5].w), pack_bf16(w[6].w, w[7].w));
      }
    }
  }
}

template <int CG, int NP>
__global__ void __launch_bounds__(CONV_THREADS, 2) k_conv3x3_ws(ConvTcArgs a) {
  using P = ConvWsT<CG, NP>;
  constexpr int KS = CG / 2;
  extern __shared__ __align__(128) uint8_t sm[];
  uint8_t* wsm = sm;
  uint8_t* ring = sm + P::WBYTES;
  __shared__ __align__(8) uint64_t full[WS_SLOTS], empty[WS_SLOTS], accf[2], acce[2], done;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // weights -> bfloat16 [tap][cg][n][8], zero beyond Cin / Cout
  for (int idx = tid; idx < 9 * CG * NP; idx += CONV_THREADS) {
    const int t = idx / (CG * NP), rem = idx - t * CG * NP, cg = rem / NP, n = rem - cg * NP;
    const int dy = t / 3, dx = t - dy * 3;
    uint32_t pk[4];
#pragma unroll
    for (int c = 0; c < 8; c += 2) {
      const int k0 = cg * 8 + c;
      const float v0 = (n < a.Cout && k0 < a.Cin) ? wval(a, n, k0, dy, dx) : 0.f;
      const float v1 = (n < a.Cout && k0 + 1 < a.Cin) ? wval(a, n, k0 + 1, dy, dx) : 0.f;
      pk[c / 2] = pack_bf16(v0, v1);
    }
    *reinterpret_cast<uint4*>(wsm + (size_t)idx * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(P::NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < WS_SLOTS; ++s) {
      mbar_init(&full[s], WS_PROD);
      mbar_init(&empty[s], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&accf[k], 1);
      mbar_init(&acce[k], 128);
    }
    mbar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // weights -> async proxy
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const size_t cs = (size_t)a.H * a.W;
  const int tiles_x = (a.W + TC_M - 1) / TC_M;
  const int RU = a.rows_per_unit;
  const int runs = (a.H + RU - 1) / RU;
  const int nunits = a.B * tiles_x * runs;

  if (warp >= 5) {
    // ------------------------------------------------------------ producers
    const int ptid = tid - 5 * 32;
    unsigned p = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
      const int b = u / (tiles_x * runs), rem = u - b * tiles_x * runs;
      const int xt = rem / runs, y0 = (rem - xt * runs) * RU, y1 = min(a.H, y0 + RU);
      for (int gy = y0 - 1; gy <= y1 && ok; ++gy, ++p) {
        const unsigned s = p % WS_SLOTS;
        if (!mbar_wait(smem_u32(&empty[s]), ((p / WS_SLOTS) & 1u) ^ 1u)) {
          atomicOr(&g_tc_err, 1u);
          ok = false;
          break;
        }
        ws_stage_row<CG>(a, ring + (size_t)s * P::RBYTES, b, gy, xt * TC_M, ptid);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&full[s]);
      }
    }
  } else if (warp == 4) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(TC_M, NP);
      const uint32_t wbase = smem_u32(wsm), rbase = smem_u32(ring);
      unsigned p = 0, q = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        const int rem = u % (tiles_x * runs);
        const int xt = rem / runs, y0 = (rem - xt * runs) * RU, y1 = min(a.H, y0 + RU);
        const int n_out = y1 - y0;
        for (int j = 0; j < n_out && ok; ++j, ++q) {
          for (int dy = 0; dy < 3 && ok; ++dy) {
            const unsigned r = p + j + dy;
            ok = mbar_wait(smem_u32(&full[r % WS_SLOTS]), (r / WS_SLOTS) & 1u);
          }
          if (ok) ok = mbar_wait(smem_u32(&acce[q & 1]), ((q >> 1) & 1u) ^ 1u);
          if (!ok) {
            atomicOr(&g_tc_err, 1u);
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + (q & 1) * NP;
#pragma unroll
          for (int t = 0; t < 9; ++t) {
            const int dy = t / 3, dx = t - dy * 3;
            const uint32_t row = rbase + (uint32_t)(((p + j + dy) % WS_SLOTS) * P::RBYTES);
#pragma unroll
            for (int s = 0; s < KS; ++s) {
              const uint64_t ad = mdesc(row + (uint32_t)(((2 * s) * PW + dx + PX0) * 16), PW * 16, 128);
              const uint64_t bd = mdesc(wbase + (uint32_t)(((t * CG + 2 * s) * NP) * 16), NP * 16, 128);
              const uint32_t acc = (t | s) != 0;
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                  : "memory");
            }
          }
          tc_commit(&accf[q & 1]);
          tc_commit(&empty[(p + j) % WS_SLOTS]);       // input row y - 1 is done with
        }
        if (!ok) break;
        tc_commit(&empty[(p + n_out) % WS_SLOTS]);     // the unit's last two input rows
        tc_commit(&empty[(p + n_out + 1) % WS_SLOTS]);
        p += n_out + 2;
      }
      tc_commit(&done);                                // drain every MMA issued
      if (!mbar_wait(smem_u32(&done), 0)) atomicOr(&g_tc_err, 1u);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    unsigned q = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
      const int b = u / (tiles_x * runs), rem = u - b * tiles_x * runs;
      const int xt = rem / runs, y0 = (rem - xt * runs) * RU, y1 = min(a.H, y0 + RU);
      for (int y = y0; y < y1; ++y, ++q) {
        if (!mbar_wait(smem_u32(&accf[q & 1]), (q >> 1) & 1u)) {
          atomicOr(&g_tc_err, 1u);
          ok = false;
          break;
        }
        tc_fence_after();
        uint32_t acc[NP];
#pragma unroll
        for (int k = 0; k < NP / 16; ++k)
          SHL_TMEM_LD16(acc + 16 * k,
                        tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((q & 1) * NP + 16 * k));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        tc_fence_before();
        mbar_arrive(&acce[q & 1]);
        float* o = a.out + (((size_t)b * a.Cout) * a.H + y) * a.W + xt * TC_M + warp * 32 + lane;
#pragma unroll
        for (int n = 0; n < NP; ++n)
          if (n < a.Cout) o[n * cs] = __uint_as_float(acc[n]) + (a.bias ? __ldg(a.bias + n) : 0.f);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(P::NCOLS)
                 : "memory");
}

template <int CG, int NP>
cudaError_t launch_tc(const ConvTcArgs& a, cudaStream_t st) {
  using P = ConvTcT<CG, NP>;
  auto k = k_conv3x3_tc<CG, NP>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::SMEM);
  if (e) return e;
  // CTAs per SM for the grid size: the shared-memory bound (228 KB per SM,
  // 1 KB reserved per CTA) and the register bound, at most 8 and at most 512
  // TMEM columns.  No CTA
  // waits on another, so the count only sizes the grid.
  int per_sm = (int)((228u * 1024u) / (P::SMEM + 1024u + 256u));
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, k) == cudaSuccess && fa.numRegs > 0)
    per_sm = std::min(per_sm, 65536 / (fa.numRegs * CONV_THREADS));
  per_sm = std::max(1, std::min({per_sm, 8, (int)(512 / P::NCOLS)}));
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int slots = per_sm * std::max(sms, 1);
  // rows per unit: about four units per CTA, 4..32 rows (two extra input
  // rows are staged per unit)
  const long long strips = (long long)a.B * ((a.W + TC_M - 1) / TC_M);
  const long long rows = strips * a.H;
  ConvTcArgs args = a;
  args.rows_per_unit = (int)std::max(4LL, std::min(32LL, rows / std::max(1LL, 4LL * slots)));
  args.rows_per_unit = std::min(args.rows_per_unit, a.H);
  const long long nunits = strips * ((a.H + args.rows_per_unit - 1) / args.rows_per_unit);
  const int grid = (int)std::max(1LL, std::min(nunits, (long long)slots));
  k<<<grid, CONV_THREADS, P::SMEM, st>>>(args);
  return cudaGetLastError();
}

template <int CG, int NP>
cudaError_t launch_ws(const ConvTcArgs& a, cudaStream_t st) {
  using P = ConvWsT<CG, NP>;
  auto k = k_conv3x3_ws<CG, NP>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::SMEM);
  if (e) return e;
  int per_sm = (int)((228u * 1024u) / (P::SMEM + 1024u + 512u));
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, k) == cudaSuccess && fa.numRegs > 0)
    per_sm = std::min(per_sm, 65536 / (fa.numRegs * CONV_THREADS));
  per_sm = std::max(1, std::min({per_sm, 8, (int)(512 / P::NCOLS)}));
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int slots = per_sm * std::max(sms, 1);
  // rows per unit: about two units per CTA, 8..64 rows (two extra input rows
  // are staged per unit)
  const long long strips = (long long)a.B * ((a.W + TC_M - 1) / TC_M);
  ConvTcArgs args = a;
  args.rows_per_unit = (int)std::max(8LL, std::min(64LL, strips * a.H / std::max(1LL, 2LL * slots)));
  args.rows_per_unit = std::min(args.rows_per_unit, a.H);
  const long long nunits = strips * ((a.H + args.rows_per_unit - 1) / args.rows_per_unit);
  const int grid = (int)std::max(1LL, std::min(nunits, (long long)slots));
  k<<<grid, CONV_THREADS, P::SMEM, st>>>(args);
  return cudaGetLastError();
}

// SHL_CONV_WS=1 selects the warp-specialised kernel.  It is opt-in: at
// 32 x 33 -> 32 x 256 x 256 it measured 0.282 ms against 0.194 ms for
// k_conv3x3_tc, whose 256 threads all stage operands (three producer warps
// do not keep enough loads in flight).
bool conv_ws_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("SHL_CONV_WS");
    return e && e[0] == '1';
  }();
  return on;
}

int round16(int v) { return (v + 15) / 16 * 16; }

// Tile of one call: CG 8-channel input groups, NP output channels (padded to
// 16).  Narrow layers take the exact tile (and the warp-specialised variant
// when it is switched on); layers with up to 112 input and 32 output
// channels, or 32 input and 112 output channels, take a wider tile with the
// extra channels zero.  false: no tile takes the shape.
bool tc_tile(int Ci, int Co, int* cg, int* np) {
  if (Ci < 1 || Co < 1) return false;
  *cg = round16(Ci) / 8;
  *np = round16(Co);
  if (*cg <= 6 && *np <= 48) return true;
  if (*cg <= 14 && *np <= 32) {
    *np = 32;
    return true;
  }
  if (*cg <= 4 && *np <= 112) {
    *cg = 4;
    *np = *np <= 64 ? 64 : (*np <= 96 ? 96 : 112);
    return true;
  }
  return false;
}

cudaError_t dispatch(const ConvTcArgs& a, cudaStream_t st) {
  int cg = 0, np = 0;
  if (!tc_tile(a.Cin, a.Cout, &cg, &np)) return cudaErrorInvalidValue;
  const bool ws = conv_ws_enabled() && a.W % TC_M == 0;   // the variant takes whole tiles only
#define SHL_TC(CGV, NPV)                                                                \
  if (cg == CGV && np == NPV) return ws ? launch_ws<CGV, NPV>(a, st) : launch_tc<CGV, NPV>(a, st);
#define SHL_TC_WIDE(CGV, NPV) \
  if (cg == CGV && np == NPV) return launch_tc<CGV, NPV>(a, st);
  SHL_TC(2, 16) SHL_TC(2, 32) SHL_TC(2, 48)
  SHL_TC(4, 16) SHL_TC(4, 32) SHL_TC(4, 48)
  SHL_TC(6, 16) SHL_TC(6, 32) SHL_TC(6, 48)
  SHL_TC_WIDE(8, 32) SHL_TC_WIDE(10, 32) SHL_TC_WIDE(12, 32) SHL_TC_WIDE(14, 32)
  SHL_TC_WIDE(4, 64) SHL_TC_WIDE(4, 96) SHL_TC_WIDE(4, 112)
#undef SHL_TC_WIDE
#undef SHL_TC
  return cudaErrorInvalidValue;
}

thread_local const char* g_tc_msg = "";

shl_status tc_run(const ConvTcArgs& a, void* stream, const char* where) {
  if (a.B == 0) return SHL_OK;
  cudaError_t e = dispatch(a, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    g_tc_msg = where;
    return SHL_ECUDA;
  }
  return SHL_OK;
}

}  // namespace

extern "C" {

int shl_nn_conv3x3_tc_supported(int Ci, int Co, int H, int W) {
  int cg = 0, np = 0;
  return tc_tile(Ci, Co, &cg, &np) && H >= 1 && W >= 16 && W % 2 == 0;
}

shl_status shl_nn_conv3x3_forward_tc(const float* in, const float* w, const float* bias,
                                     float* out, int B, int Ci, int Co, int H, int W,
                                     void* stream) {
  if (!in || !w || !out || B < 0 || !shl_nn_conv3x3_tc_supported(Ci, Co, H, W) ||
      (reinterpret_cast<uintptr_t>(in) & 15u)) {
    g_tc_msg = "conv3x3_forward_tc: bad arguments, unsupported shape or input not 16-byte aligned";
    return SHL_EINVAL;
  }
  const ConvTcArgs a{in, w, bias, out, B, Ci, Co, H, W, 0, 1};
  return tc_run(a, stream, "conv3x3_forward_tc: launch failed");
}

shl_status shl_nn_conv3x3_backward_data_tc(const float* gout, const float* w, float* gin, int B,
                                           int Ci, int Co, int H, int W, void* stream) {
  if (!gout || !w || !gin || B < 0 || !shl_nn_conv3x3_tc_supported(Co, Ci, H, W) ||
      (reinterpret_cast<uintptr_t>(gout) & 15u)) {
    g_tc_msg = "conv3x3_backward_data_tc: bad arguments, unsupported shape or gout not 16-byte aligned";
    return SHL_EINVAL;
  }
  // gin = conv(gout, flipped and channel-transposed w): Cin = Co, Cout = Ci
  const ConvTcArgs a{gout, w, nullptr, gin, B, Co, Ci, H, W, 1, 1};
  return tc_run(a, stream, "conv3x3_backward_data_tc: launch failed");
}

int shl_nn_conv3x3_wgrad_tc_supported(int Ci, int Co, int H, int W) {
  return Ci >= 1 && 3 * Ci <= 128 && Co >= 1 && Co <= 96 && H >= 1 && W >= 16 && W % 2 == 0;
}

size_t shl_nn_conv3x3_backward_weight_tc_workspace_floats(int B, int Ci, int Co, int H, int W) {
  if (B < 1 || !shl_nn_conv3x3_wgrad_tc_supported(Ci, Co, H, W)) return 0;
  int grid = 0, ru = 0;
  wgrad_plan(B, H, W, &grid, &ru);
  return (size_t)grid * ((size_t)Co * Ci * 9 + Co);
}

shl_status shl_nn_conv3x3_backward_weight_tc(const float* in, const float* gout, float* gw,
                                             float* gb, int B, int Ci, int Co, int H, int W,
                                             float* ws, void* stream) {
  if (!in || !gout || !gw || !ws || B < 1 || !shl_nn_conv3x3_wgrad_tc_supported(Ci, Co, H, W) ||
      ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(gout)) & 15u)) {
    g_tc_msg = "conv3x3_backward_weight_tc: bad arguments, unsupported shape or misaligned input";
    return SHL_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int grid = 0, ru = 0;
  wgrad_plan(B, H, W, &grid, &ru);
  const WgradTcArgs a{in, gout, ws, B, Ci, Co, H, W, ru};
  const int np = round16(Co);          // 49..96 output channels: the 96-wide tile
  cudaError_t e = np == 16 ? launch_wgrad<16>(a, grid, st)
                : np == 32 ? launch_wgrad<32>(a, grid, st)
                : np == 48 ? launch_wgrad<48>(a, grid, st)
                           : launch_wgrad<96>(a, grid, st);
  if (e == cudaSuccess) {
    const int nw = Co * Ci * 9;
    k_wgrad_reduce<<<(nw + Co + 255) / 256, 256, 0, st>>>(ws, gw, gb, grid, nw, Co);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    g_tc_msg = "conv3x3_backward_weight_tc: launch failed";
    return SHL_ECUDA;
  }
  return SHL_OK;
}

shl_status shl_nn_tc_status(void* stream) {
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    g_tc_msg = "shl_nn_tc_status: stream synchronisation failed";
    return SHL_ECUDA;
  }
  unsigned flag = 0;
  if (cudaMemcpyFromSymbol(&flag, g_tc_err, sizeof(flag)) != cudaSuccess) return SHL_ECUDA;
  if (flag) {
    const unsigned zero = 0;
    cudaMemcpyToSymbol(g_tc_err, &zero, sizeof(zero));
    g_tc_msg = "a tensor-core convolution gave up waiting for its MMAs";
    return SHL_ETIMEOUT;
  }
  return SHL_OK;
}

const char* shl_nn_tc_last_error(void) { return g_tc_msg; }

}  // extern "C"
