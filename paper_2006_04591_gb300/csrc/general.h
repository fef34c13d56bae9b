// general.h - the transform for any image size (1..4096 per side) and for
// complex Hermitian filter spectra: declarations shared by api.cpp and
// general.cu.
//
// The power-of-two kernels of fast.cu keep real, even spectra in transposed
// half-spectrum planes.  This path keeps row-major half-spectrum planes
// [N][M/2+1] (columns kx = 0..M/2 of the natural-order spectrum; the rest
// follows from Hermitian symmetry, which holds for real images and Hermitian
// filters), complex filter values where the bank has them, and computes
// every line DFT in shared memory with a mixed-radix Stockham FFT (all prime
// factors <= 61), or with Bluestein's chirp-z algorithm (a larger prime
// factor: the length-L DFT becomes a circular convolution of length P = the
// power of two >= 2L - 1).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

namespace shl {
namespace gen {

constexpr int MAX_LEN = 4096;     // longest side
constexpr int MAX_STAGES = 16;
constexpr int MAX_DIRECT_PRIME = 61;

// Forward DFT of length L, X[k] = sum_n x[n] exp(-2 pi i n k / L); the
// inverse is taken as conj(DFT(conj(x))).  Pointers refer to device tables.
struct LinePlan {
  int L;                     // transform length
  int P;                     // working length (L, or Bluestein's power of two)
  int bluestein;             // 1: chirp-z through a length-P FFT
  int nst;                   // Stockham stages of the length-P FFT
  int radix[MAX_STAGES];     // their radices (product P)
  const float2* tw;          // [P]  exp(-2 pi i q / P)
  const float2* chirp;       // [L]  exp(-i pi n^2 / L)              (Bluestein)
  const float2* kern;        // [P]  DFT_P(h) / P, h[m] = conj chirp[|m|] (Bluestein)
};

// Host-side tables of one length, computed in float64 and rounded; offsets
// (in float2 units) of tw / chirp / kern inside `data`.
struct LineTables {
  LinePlan plan{};
  std::vector<float2> data;
  size_t off_tw = 0, off_chirp = 0, off_kern = 0;
};
// Builds the plan and tables of length L (1 <= L <= MAX_LEN).
LineTables make_line_tables(int L);
// Points the plan at the tables after `data` was copied to `dev`.
void place_line_tables(LineTables* t, const float2* dev);

// Real-row input of the forward row pass.
enum RowIn : int { RIN_F32 = 0, RIN_BF16 = 1, RIN_MASKED = 2 };

// Row passes (rows of length M, plan pm) between real planes [nplanes][N][M]
// and half-spectrum planes [nplanes][N][M/2+1].
//   rows_fwd:    real rows (thresholded on read when thresh != null, one
//                threshold per plane; masked: mask ? f_masked : f_est) ->
//                row DFTs, columns 0..M/2 -> out.
//   rows_inv:    Hermitian row spectra (from their halves) -> inverse row
//                DFT -> real part * scale -> float32 or bfloat16 out.
//   rows_shrink: in place: inverse row DFT -> real part * scale -> zero
//                |c| < thresh[plane] -> forward row DFT.
cudaError_t launch_rows_fwd(const LinePlan& pm, RowIn mode, const void* in, const uint8_t* mask,
                            const float* fest, const float* thresh, float2* out, int N,
                            int nplanes, cudaStream_t st);
cudaError_t launch_rows_inv(const LinePlan& pm, const float2* in, void* out, bool bf16,
                            float scale, int N, int nplanes, cudaStream_t st);
cudaError_t launch_rows_shrink(const LinePlan& pm, float2* z, const float* thresh, float scale,
                               int N, int nplanes, cudaStream_t st);

// Column passes (columns of length N, plan pn) on half-spectrum planes of
// W = M/2 + 1 columns.
//   cols_fwd: in-place forward column DFT of nplanes planes.
//   cols_dec: T[s - s0] = inverse column DFT of G_i * X_b [* 1/W] for the
//             subbands s = s0 .. s0+S-1 (b = s / K, i = s % K).
//   cols_rec: for each image b with subbands in s0 .. s0+S-1, split into
//             groups of consecutive subbands (one CTA per column block,
//             image and group): the group's sum_i conj(G_i) * column
//             DFT(T[s - s0]) in order of i, written over its first staging
//             plane; then acc = (partial sum in A_b unless the chunk holds
//             the image's first subband) + the group sums in group order; on
//             the image's last subband acc is multiplied by 1/W (when invW)
//             and inverse column transformed into A_b, else stored there as
//             the new partial sum.  T is overwritten.
// G is float [K][N][W] (real spectra) or float2 [K][N][W] (complex), 1/W
// float [N][W]: the columns kx = 0..M/2 of the natural-order tables.
cudaError_t launch_cols_fwd(const LinePlan& pn, float2* X, int W, int nplanes, cudaStream_t st);
cudaError_t launch_cols_dec(const LinePlan& pn, const float2* X, float2* T, const void* G,
                            bool cplx, const float* invW, int W, int K, int s0, int S,
                            cudaStream_t st);
cudaError_t launch_cols_rec(const LinePlan& pn, float2* T, float2* A, const void* G,
                            bool cplx, const float* invW, int W, int K, int s0, int S,
                            cudaStream_t st);

}  // namespace gen
}  // namespace shl
