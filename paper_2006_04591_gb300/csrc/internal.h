// internal.h - declarations shared by the C-ABI layer and the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "../../include/shearlet.h"

namespace shl {

constexpr int TW_P = 4096;      // twiddle table length: exp(-2 pi i q / TW_P)
constexpr int LOG_TW_P = 12;

// Input handling of the row R2C pass.
enum InMode : int {
  IN_F32 = 0,      // float32 reals
  IN_BF16 = 1,     // bfloat16 reals
  IN_MASKED = 2,   // u = mask * (f_masked - f_est) + f_est, float32
};

// Launchers of fast.cu.  Half-spectrum planes are stored transposed,
// [Mh][N] with Mh = M/2 + 1 and the N column-frequency values contiguous.
cudaError_t launch_rows_r2c_t(int M, InMode mode, bool thresh, const void* in, const uint8_t* mask,
                              const float* fest, const float* th, float2* out, int N, int nsub,
                              const float2* tw, cudaStream_t st);
// s16: the staged planes are bfloat16 (bfloat16 output only).
cudaError_t launch_rows_c2r_t(int M, bool bf16, const void* in, void* out, int N, int nsub,
                              const float2* tw, cudaStream_t st, bool s16 = false);
// In place on [nsub][Mh][N] half spectra: C2R rows -> zero |c| < thresh[s]
// -> R2C rows (the fused threshold of the denoise / IHT step).
cudaError_t launch_rows_shrink_t(int M, float2* z, const float* thresh, int N, int nsub,
                                 const float2* tw, cudaStream_t st);
cudaError_t launch_lines_fwd(int N, float2* data, int nlines, const float2* tw, cudaStream_t st);
// nimg: image planes of X / acc (bounds of the checked build); s16: write
// the staged planes as bfloat16 (the bfloat16 decomposition).
cudaError_t launch_dec_lines(int N, const float2* X, void* out, const float* G, const float* invW,
                             float scale, int Mh, int K, int s0, int S, const float2* tw,
                             cudaStream_t st, int nimg, bool s16 = false);
cudaError_t launch_rec_lines(int N, const float2* stage, float2* acc, const float* G,
                             const float* invW, float scale, int Mh, int K, int s0, int Sc,
                             const float2* tw, cudaStream_t st, int nimg);
// Column pass of the bfloat16-output decomposition on the tensor cores
// (tc_dft.cu, N = 512 only): the same staging planes as launch_dec_lines
// (s16: bfloat16 planes).
bool dec_lines_tc_supported(int N, int Mh);
cudaError_t launch_dec_lines_tc(int N, const float2* X, void* out, const float* G,
                                const float* invW, float scale, int Mh, int K, int s0, int S,
                                const float2* tw, cudaStream_t st, int nimg, bool s16 = false);
// Error flag of its bounded MMA waits and its checked-build guard word,
// read and cleared.
cudaError_t read_dft_error(unsigned* flag);
cudaError_t read_check_word_tc(unsigned* word);
// Pipelined decomposition (both passes in one cooperative launch over a
// ring of NS staging chunks of CS subbands, col_frac of the CTAs on the
// column pass); sizes with dec_pipe_supported.
bool dec_pipe_supported(int N, int M);
size_t dec_pipe_ctl_bytes(int nchunks);
cudaError_t launch_dec_pipe(int N, int M, bool bf16, const float2* X, float2* ring, void* out,
                            const float* G, const float* invW, float scale, int K, int total,
                            int CS, int NS, float col_frac, unsigned* ctl, const float2* tw,
                            cudaStream_t st);
cudaError_t read_pipe_error(unsigned* flag);
// Guard word of the checked build (fast.cu), read and cleared; 0 otherwise.
cudaError_t read_check_word(unsigned* word);

// Paired-subband kernels of fused.cu (square planes, see pair_supported):
// one persistent cluster launch per direction, the plane between the passes
// in a per-cluster slot of L * L * 8 bytes.
bool pair_supported(int N, int M);
// Co-resident clusters of the paired kernels on the current device.
cudaError_t pair_max_clusters(int L, int* ncl);
// Clusters a launch over `units` pairs uses.
int pair_clusters_for(int ncl_max, int units);
cudaError_t launch_pair_dec(int L, bool bf16, const float2* X, const float* G, const float* invW,
                            void* coeffs, float2* slots, int ncl, float scale, int K, int B,
                            const float2* tw, cudaStream_t st);
// Writes the partial half planes [ncl + B - 1][Mh][L] of each image.
cudaError_t launch_pair_rec(int L, bool bf16, const void* coeffs, const float* thresh,
                            const float* G, float2* slots, float2* parts, int ncl, int K, int B,
                            const float2* tw, cudaStream_t st);
// Sums the partial planes of each image in cluster order, applies
// scale [* 1/W] and the inverse column FFT into A [B][Mh][L].
cudaError_t launch_pair_final(int L, const float2* parts, float2* A, const float* invW, float scale,
                              int K, int B, int ncl, const float2* tw, cudaStream_t st);
cudaError_t launch_absmax(const void* coeffs, bool bf16, int nsub, int K, size_t elems,
                          const float* rms, float* out, cudaStream_t st);
cudaError_t launch_iht_schedule(const float* a, const float* rms, int K, int B, int T,
                                double delta_min, float* th, cudaStream_t st);

// Helpers of api.cpp used by noalloc.cu.
shl_status set_error(shl_status s, const char* msg);
shl_status bank_geometry(const shl_bank* b, int* device, size_t* plane_bytes);
// shl_decompose with at most `stage_subbands_max` per-subband staging planes
// after the batch's image spectra in ws.
shl_status decompose_staged(const shl_bank* b, const float* x, int batch, void* coeffs,
                            shl_dtype dtype, int flags, void* ws, size_t ws_bytes, void* stream,
                            int stage_subbands_max);

// Filters of a bank in order: cone 0 (low-pass), then per scale cone 1
// (k = -2^l..2^l) and cone 2 (k = -(2^l-1)..2^l-1, or +-2^l when full).
struct BankItem { int cone, scale, k, l; };
const char* bank_items(int n_scales, const int* shear_levels, int full,
                       std::vector<BankItem>* items);
// Coefficients b_0..b_4 of the maximally flat low-pass H(w) = b0 + sum b_m cos(m w).
void maxflat_coeffs(double b[5]);

// float64 construction on the current device (bank_gpu.cu): spectra
// [K][N][M] natural order into d_spectra (d_tmp: one [N][M] plane of
// scratch), W [N][M], RMS [K], and the float32 tables of the transform
// (G [K][Mh][N], 1/W [Mh][N]); *d_bad counts points with W <= 0.
cudaError_t build_bank_device(int rows, int cols, int n_scales, const int* shear_levels, int full,
                              const std::vector<BankItem>& items, double* d_spectra,
                              double* d_tmp, double* d_w, double* d_rms, float* d_G,
                              float* d_invW, unsigned* d_bad, cudaStream_t st);

// Host float64 filter-bank construction (bank_build.cpp).
struct HostBank {
  int rows = 0, cols = 0, K = 0;
  std::vector<double> spectra;   // [K][rows][cols], natural order
  std::vector<int> idx;          // [K][3]
};
// Returns empty string on success, else an error message.
const char* build_shearlet_bank(int rows, int cols, int n_scales, const int* shear_levels,
                                int full, HostBank* out);

}  // namespace shl
