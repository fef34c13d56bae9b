// internal.h - declarations shared by the C-ABI layer and the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

namespace shl {

constexpr int TW_P = 4096;      // twiddle table length: exp(-2 pi i q / TW_P)
constexpr int LOG_TW_P = 12;

// Input handling of the row R2C pass.
enum InMode : int {
  IN_F32 = 0,      // float32 reals
  IN_BF16 = 1,     // bfloat16 reals
  IN_MASKED = 2,   // u = mask * (f_masked - f_est) + f_est, float32
};

// Column pass modes (see cols kernels).
enum ColMode : int {
  COL_FWD = 0,        // in-place forward FFT of image spectra
  COL_DEC_INV = 1,    // (X_b * G_i * scale [* invW]) -> inverse FFT -> staging
  COL_REC_ACC = 2,    // forward FFT of staged rows, * G_i, sum over i -> acc
  COL_FINAL_INV = 3,  // acc * scale [* invW] -> inverse FFT, in place
};

struct RowR2CArgs {
  const void* in;          // [nlines][M] reals (float or bf16), or f_masked
  const uint8_t* mask;     // IN_MASKED only
  const float* fest;       // IN_MASKED only
  float2* out;             // [nlines][Mh]
  const float* thresh;     // per subband (line / N), may be null
  const float2* tw;
  int nlines;
  int N;                   // lines per subband (image rows)
};

struct RowC2RArgs {
  const float2* in;        // [nlines][Mh]
  void* out;               // [nlines][M] float or bf16
  const float2* tw;
  int nlines;
};

struct ColArgs {
  float2* data;            // FWD / FINAL_INV: [B][N][Mh] in place; DEC_INV: image spectra
  float2* out;             // DEC_INV: staging [S][N][Mh]
  const float2* in;        // REC_ACC: staging rows [S][N][Mh]
  float2* acc;             // REC_ACC: accumulators [B][N][Mh]
  const float* G;          // [K][N][Mh]
  const float* invW;       // [N][Mh] or null
  const float2* tw;
  float scale;
  int Mh, K;
  int s0, S;               // subband range of the chunk (DEC_INV / REC_ACC)
  int b_lo;                // REC_ACC: first image of the chunk
};

cudaError_t launch_rows_r2c(int M, InMode mode, bool thresh, const RowR2CArgs& a,
                            cudaStream_t st);
cudaError_t launch_rows_c2r(int M, bool bf16_out, const RowC2RArgs& a, cudaStream_t st);
cudaError_t launch_cols(int N, ColMode mode, const ColArgs& a, int grid_y, cudaStream_t st);
cudaError_t launch_absmax(const void* coeffs, bool bf16, int nsub, int K, size_t elems,
                          const float* rms, float* out, cudaStream_t st);

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
