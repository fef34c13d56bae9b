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
cudaError_t launch_rows_c2r_t(int M, bool bf16, const float2* in, void* out, int N, int nsub,
                              const float2* tw, cudaStream_t st);
// In place on [nsub][Mh][N] half spectra: C2R rows -> zero |c| < thresh[s]
// -> R2C rows (the fused threshold of the denoise / IHT step).
cudaError_t launch_rows_shrink_t(int M, float2* z, const float* thresh, int N, int nsub,
                                 const float2* tw, cudaStream_t st);
cudaError_t launch_lines_fwd(int N, float2* data, int nlines, const float2* tw, cudaStream_t st);
cudaError_t launch_dec_lines(int N, const float2* X, float2* out, const float* G, const float* invW,
                             float scale, int Mh, int K, int s0, int S, const float2* tw,
                             cudaStream_t st);
cudaError_t launch_rec_lines(int N, const float2* stage, float2* acc, const float* G,
                             const float* invW, float scale, int Mh, int K, int s0, int Sc,
                             const float2* tw, cudaStream_t st);
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
cudaError_t launch_absmax(const void* coeffs, bool bf16, int nsub, int K, size_t elems,
                          const float* rms, float* out, cudaStream_t st);

// Helpers of api.cpp used by noalloc.cu.
shl_status set_error(shl_status s, const char* msg);
shl_status bank_geometry(const shl_bank* b, int* device, size_t* plane_bytes);
// shl_decompose with at most `stage_subbands_max` per-subband staging planes
// after the batch's image spectra in ws.
shl_status decompose_staged(const shl_bank* b, const float* x, int batch, void* coeffs,
                            shl_dtype dtype, int flags, void* ws, size_t ws_bytes, void* stream,
                            int stage_subbands_max);

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
