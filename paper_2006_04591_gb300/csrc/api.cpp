// api.cpp - the C ABI declared in include/shearlet.h.
//
// Validation, bank ownership and the launch sequences of the transform live
// here; all arithmetic on images and coefficients runs in the kernels of
// fast.cu (power-of-two sizes 16..2048 with real, even spectra), general.cu
// (every other size, and complex Hermitian spectra) and nn.cu / nn_tc.cu
// (the learned parts).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <cstdint>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/shearlet.h"
#include "general.h"
#include "internal.h"

struct shl_bank {
  int device = 0, N = 0, M = 0, Mh = 0, K = 0;
  std::vector<double> spectra;   // [K][N][M]
  std::vector<int> idx;          // [K][3]
  std::vector<double> rms;       // [K]
  std::vector<double> dual_w;    // [N][M]
  float* dG = nullptr;           // [K][Mh][N] half spectra, transposed
  float* dInvW = nullptr;        // [Mh][N]
  float2* dTw = nullptr;         // [TW_P]
  float* dRms = nullptr;         // [K]
  // General path (general.cu): full complex planes in natural order.
  bool general = false;          // this bank runs on general.cu (row-major half planes)
  bool cplx = false;             // complex spectra (imaginary parts kept)
  std::vector<double> spectra_im;  // [K][N][M] when cplx
  void* dGg = nullptr;           // float [K][N][Mh], or float2 [K][N][Mh] when cplx
  float* dInvWg = nullptr;       // [N][Mh]
  float2* dTab = nullptr;        // line tables of both plans
  shl::gen::LinePlan planN{}, planM{};
};

namespace {

thread_local std::string g_err;

shl_status fail(shl_status s, const std::string& msg) {
  g_err = msg;
  return s;
}
shl_status cuda_fail(cudaError_t e, const char* where) {
  return fail(SHL_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Images may live in device memory of the bank's device, in managed memory,
// or in pinned host memory mapped into the device's address space (the
// kernels then read or write it over the CPU-GPU link, which moves the
// image transfer into the first and last kernels).  Returns the address a
// kernel uses, or nullptr if `device` cannot dereference p.
template <typename T>
T* device_view(T* p, int device) {
  if (!p) return nullptr;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type == cudaMemoryTypeDevice) return at.device == device ? p : nullptr;
  if (at.type == cudaMemoryTypeManaged) return p;
  if (at.type == cudaMemoryTypeHost && at.devicePointer) return static_cast<T*>(at.devicePointer);
  return nullptr;
}

// ------------------------------------------------------- launch accounting
std::atomic<long long> g_launches{0};
std::atomic<int> g_profile{0};
struct ProfRec { const char* name; cudaEvent_t a, b; };
std::mutex g_prof_mu;
std::vector<ProfRec> g_prof;

// Brackets one library launch: counts it and, when profiling is on, records
// CUDA events before and after it on the launch stream.
struct Launch {
  const char* name;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  Launch(const char* n, cudaStream_t s) : name(n), st(s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (g_profile.load(std::memory_order_relaxed)) {
      if (cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess)
        cudaEventRecord(a, st);
    }
  }
  ~Launch() {
    if (a && b) {
      cudaEventRecord(b, st);
      std::lock_guard<std::mutex> lk(g_prof_mu);
      g_prof.push_back({name, a, b});
    }
  }
};

// Subbands per chunk.  Each chunk costs one launch per pass, and launch ramp
// and tail dominate small chunks (measured at 512 x 512, K = 49, B = 16:
// 56 MB chunks 1.53 ms per step, one 1 GB chunk 1.12 ms), so the default
// staging budget holds the whole batch at the common sizes.
int stage_subbands(const shl_bank* b) {
  static const double mb = [] {
    const char* e = std::getenv("SHL_STAGE_MB");
    double v = e ? std::atof(e) : 1024.0;
    return v > 0 ? v : 1024.0;
  }();
  const double per = double(b->N) * b->Mh * sizeof(float2);
  int s = (int)(mb * 1024.0 * 1024.0 / per);
  return s < 1 ? 1 : s;
}

// Bytes of one half-spectrum plane (transposed [Mh][N] on the power-of-two
// path, row-major [N][Mh] on the general path).
size_t plane_bytes(const shl_bank* b) { return (size_t)b->N * b->Mh * sizeof(float2); }

// Pipelined decomposition: chunk of CS subbands, NS ring slots.  Opt-in
// (SHL_PIPE=1): it keeps the staging in L2 but measured slower than the
// two-launch path at 16 x 512 x 512, K = 49 (0.74-0.99 ms against 0.53 ms;
// both passes are latency-bound at 16 warps per SM and splitting the CTAs
// between them halves each pass's parallelism).  SHL_PIPE_CS / SHL_PIPE_NS
// override the ring, SHL_PIPE_COLFRAC the share of CTAs on the column pass.
struct PipeCfg { bool on; int CS, NS; float col_frac; };
const PipeCfg& pipe_cfg() {
  static const PipeCfg c = [] {
    auto env = [](const char* k, int d, int lo) {
      const char* e = std::getenv(k);
      const int v = e ? std::atoi(e) : d;
      return v >= lo ? v : d;
    };
    PipeCfg c{env("SHL_PIPE", 0, 0) != 0, env("SHL_PIPE_CS", 8, 1), env("SHL_PIPE_NS", 3, 2),
              0.4f};
    const char* f = std::getenv("SHL_PIPE_COLFRAC");
    if (f && std::atof(f) > 0.0 && std::atof(f) < 1.0) c.col_frac = (float)std::atof(f);
    return c;
  }();
  return c;
}
bool use_pipe(const shl_bank* b) {
  return !b->general && pipe_cfg().on && shl::dec_pipe_supported(b->N, b->M);
}

// Paired-subband kernels (fused.cu): both passes of each direction in one
// cluster launch, the plane between them in L2 instead of DRAM, for the
// shapes pair_supported covers.  Opt-in with SHL_FUSED=1 (read once per
// process): at 16 x 512 x 512, K = 49 they measured 0.67 + 0.83 ms against
// 0.53 + 0.56 ms for the staged kernels, which run at higher issue
// efficiency with two CTAs per SM.
bool fused_on() {
  static const bool on = [] {
    const char* e = std::getenv("SHL_FUSED");
    return e && e[0] == '1';
  }();
  return on;
}
// Tensor-core column pass of the bfloat16-output decomposition
// (tc_dft.cu): SHL_TC_DFT=1 turns it on, read once per process.
bool tc_dft_on() {
  static const bool on = [] {
    const char* e = std::getenv("SHL_TC_DFT");
    return e && e[0] == '1';
  }();
  return on;
}
bool use_tc_dft(const shl_bank* b, shl_dtype dtype) {
  return dtype == SHL_BF16 && !b->general && tc_dft_on() && shl::dec_lines_tc_supported(b->N, b->Mh);
}
// Co-resident clusters of the paired kernels on the bank's device (0 when
// the query fails, which keeps the staged kernels).
int pair_ncl_max(const shl_bank* b) {
  DevGuard g(b->device);
  int n = 0;
  if (shl::pair_max_clusters(b->N, &n) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}
bool use_pair(const shl_bank* b) {
  return !b->general && b->device >= 0 && fused_on() && shl::pair_supported(b->N, b->M) &&
         pair_ncl_max(b) > 0;
}
// Slot of one cluster: the complex plane of a subband pair, [M][N].
size_t pair_slot_bytes(const shl_bank* b) { return (size_t)b->N * b->M * sizeof(float2); }

size_t ws_need(const shl_bank* b, int batch, shl_op op) {
  const long long sub = (long long)batch * b->K;
  const size_t X = align256((size_t)batch * plane_bytes(b));
  if ((op == SHL_OP_DECOMPOSE || op == SHL_OP_RECONSTRUCT) && use_pair(b)) {
    const int ncl = pair_ncl_max(b);
    const size_t slots = align256((size_t)ncl * pair_slot_bytes(b));
    if (op == SHL_OP_DECOMPOSE) return X + slots;
    return X + slots + align256((size_t)(ncl + batch - 1) * plane_bytes(b));
  }
  if (op == SHL_OP_DECOMPOSE && use_pipe(b)) {
    const PipeCfg& c = pipe_cfg();
    const int nchunks = (int)((sub + c.CS - 1) / c.CS);
    return X + align256((size_t)c.NS * c.CS * plane_bytes(b)) +
           align256(shl::dec_pipe_ctl_bytes(nchunks));
  }
  const long long S = std::min<long long>(stage_subbands(b), sub);
  if (op == SHL_OP_SHRINK)   // image spectra and accumulators both live to the end
    return 2 * X + align256((size_t)S * plane_bytes(b));
  return X + align256((size_t)S * plane_bytes(b));
}

void free_bank(shl_bank* b) {
  if (!b) return;
  if (b->dG) cudaFree(b->dG);
  if (b->dInvW) cudaFree(b->dInvW);
  if (b->dTw) cudaFree(b->dTw);
  if (b->dRms) cudaFree(b->dRms);
  if (b->dGg) cudaFree(b->dGg);
  if (b->dInvWg) cudaFree(b->dInvWg);
  if (b->dTab) cudaFree(b->dTab);
  delete b;
}

// exp(-2 pi i q / TW_P), q < TW_P, computed in float64 and rounded.
std::vector<float2> twiddle_table() {
  std::vector<float2> hT(shl::TW_P);
  const double PI = 3.14159265358979323846264338327950288;
  for (int q = 0; q < shl::TW_P; ++q) {
    const double a = -2.0 * PI * q / shl::TW_P;
    hT[q] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  return hT;
}

// Tables of the general path: float32 filters (complex when the bank keeps
// imaginary parts) and 1/W on the half plane [N][Mh], and the line plans of
// both axes.
shl_status upload_general(shl_bank* b) {
  const int N = b->N, M = b->M, Mh = b->Mh, K = b->K;
  const size_t plane = (size_t)N * Mh;
  std::vector<float> hW(plane), hR(K);
  for (int y = 0; y < N; ++y)
    for (int x = 0; x < Mh; ++x) hW[(size_t)y * Mh + x] = (float)(1.0 / b->dual_w[(size_t)y * M + x]);
  for (int i = 0; i < K; ++i) hR[i] = (float)b->rms[i];
  std::vector<float> hG;
  std::vector<float2> hGc;
  if (b->cplx) hGc.resize((size_t)K * plane);
  else hG.resize((size_t)K * plane);
  for (int i = 0; i < K; ++i)
    for (int y = 0; y < N; ++y)
      for (int x = 0; x < Mh; ++x) {
        const size_t d = ((size_t)i * N + y) * Mh + x, f = ((size_t)i * N + y) * M + x;
        if (b->cplx) hGc[d] = make_float2((float)b->spectra[f], (float)b->spectra_im[f]);
        else hG[d] = (float)b->spectra[f];
      }
  shl::gen::LineTables tN = shl::gen::make_line_tables(N), tM = shl::gen::make_line_tables(M);
  const size_t gbytes = b->cplx ? hGc.size() * sizeof(float2) : hG.size() * sizeof(float);
  const size_t tabs = tN.data.size() + tM.data.size();
  DevGuard g(b->device);
  if (cudaMalloc(&b->dGg, gbytes) != cudaSuccess ||
      cudaMalloc(&b->dInvWg, plane * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&b->dTab, tabs * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&b->dRms, K * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return fail(SHL_ENOMEM, "cudaMalloc failed for the filter bank");
  }
  cudaError_t e;
  const void* gsrc = b->cplx ? (const void*)hGc.data() : (const void*)hG.data();
  if ((e = cudaMemcpy(b->dGg, gsrc, gbytes, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->dInvWg, hW.data(), plane * sizeof(float), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->dTab, tN.data.data(), tN.data.size() * sizeof(float2),
                      cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->dTab + tN.data.size(), tM.data.data(), tM.data.size() * sizeof(float2),
                      cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->dRms, hR.data(), K * sizeof(float), cudaMemcpyHostToDevice)))
    return cuda_fail(e, "bank upload");
  shl::gen::place_line_tables(&tN, b->dTab);
  shl::gen::place_line_tables(&tM, b->dTab + tN.data.size());
  b->planN = tN.plan;
  b->planM = tM.plan;
  return SHL_OK;
}

shl_status upload_bank(shl_bank* b) {
  const int N = b->N, M = b->M, Mh = b->Mh, K = b->K;
  const bool host_only = b->device < 0;
  b->dual_w.assign((size_t)N * M, 0.0);
  b->rms.assign(K, 0.0);
  for (int i = 0; i < K; ++i) {
    const double* G = b->spectra.data() + (size_t)i * N * M;
    const double* Gi = b->cplx ? b->spectra_im.data() + (size_t)i * N * M : nullptr;
    double s = 0.0;
    for (size_t e = 0; e < (size_t)N * M; ++e) {
      const double m2 = G[e] * G[e] + (Gi ? Gi[e] * Gi[e] : 0.0);   // |G_i|^2
      b->dual_w[e] += m2;
      s += m2;
    }
    b->rms[i] = std::sqrt(s / (double(N) * M));
  }
  for (size_t e = 0; e < (size_t)N * M; ++e)
    if (!(b->dual_w[e] > 0.0)) return fail(SHL_EINVAL, "dual frame weights W = sum |G_i|^2 must be > 0");
  if (host_only) return SHL_OK;
  if (b->general) return upload_general(b);
  std::vector<float> hG((size_t)K * N * Mh), hW((size_t)N * Mh), hR(K);
  for (int i = 0; i < K; ++i)
    for (int y = 0; y < N; ++y)
      for (int x = 0; x < Mh; ++x)
        hG[((size_t)i * Mh + x) * N + y] = (float)b->spectra[((size_t)i * N + y) * M + x];
  for (int y = 0; y < N; ++y)
    for (int x = 0; x < Mh; ++x) hW[(size_t)x * N + y] = (float)(1.0 / b->dual_w[(size_t)y * M + x]);
  for (int i = 0; i < K; ++i) hR[i] = (float)b->rms[i];
  const std::vector<float2> hT = twiddle_table();
  DevGuard g(b->device);
  if (cudaMalloc(&b->dG, hG.size() * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&b->dInvW, hW.size() * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&b->dTw, hT.size() * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&b->dRms, hR.size() * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return fail(SHL_ENOMEM, "cudaMalloc failed for the filter bank");
  }
  cudaError_t e;
  if ((e = cudaMemcpy(b->dG, hG.data(), hG.size() * sizeof(float), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->dInvW, hW.data(), hW.size() * sizeof(float), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->dTw, hT.data(), hT.size() * sizeof(float2), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->dRms, hR.data(), hR.size() * sizeof(float), cudaMemcpyHostToDevice)))
    return cuda_fail(e, "bank upload");
  return SHL_OK;
}

// Power-of-two sizes the kernels of fast.cu cover.
bool fast_size(int rows, int cols) { return pow2_in(rows, 16, 2048) && pow2_in(cols, 16, 2048); }

shl_status check_size(int rows, int cols) {
  if (!fast_size(rows, cols))
    return fail(SHL_EUNSUPPORTED, "rows and cols must be powers of two in [16, 2048]");
  return SHL_OK;
}

shl_status check_general_size(int rows, int cols) {
  if (rows < 1 || cols < 1 || rows > shl::gen::MAX_LEN || cols > shl::gen::MAX_LEN)
    return fail(SHL_EUNSUPPORTED, "rows and cols must be in [1, 4096]");
  return SHL_OK;
}

shl_status check_common(const shl_bank* b, int batch, const void* ws, size_t ws_bytes,
                        shl_op op) {
  if (!b) return fail(SHL_EINVAL, "bank is NULL");
  if (b->device < 0) return fail(SHL_EINVAL, "bank was created host-only (device < 0)");
  if (batch < 0) return fail(SHL_EINVAL, "batch must be >= 0");
  if (batch == 0) return SHL_OK;
  if (!ws || !aligned16(ws)) return fail(SHL_EINVAL, "workspace must be a 16-byte aligned device pointer");
  if (ws_bytes < ws_need(b, batch, op))
    return fail(SHL_EINVAL, "workspace too small (see shl_workspace_size)");
  return SHL_OK;
}

cudaError_t gen_decompose(const shl_bank* b, shl::InMode mode, const float* x,
                          const unsigned char* mask, const float* fest, int batch, void* coeffs,
                          shl_dtype dtype, bool dual, void* ws, int S, cudaStream_t st);
cudaError_t gen_reconstruct(const shl_bank* b, const void* coeffs, shl_dtype dtype, int batch,
                            const float* thresh, float* x_out, void* ws, bool weights,
                            cudaStream_t st);
cudaError_t gen_shrink(const shl_bank* b, const float* x, const unsigned char* mask,
                       const float* fest, int batch, const float* thresh, float* x_out, void* ws,
                       cudaStream_t st);

shl_status decompose_impl(const shl_bank* b, shl::InMode mode, const float* x,
                          const unsigned char* mask, const float* fest, int batch, void* coeffs,
                          shl_dtype dtype, int flags, void* ws, size_t ws_bytes, void* stream,
                          int stage_override = 0) {
  shl_status s;
  if (stage_override <= 0) {
    s = check_common(b, batch, ws, ws_bytes, SHL_OP_DECOMPOSE);
  } else {
    s = check_common(b, batch, ws, SIZE_MAX, SHL_OP_DECOMPOSE);
    if (s == SHL_OK && batch > 0 &&
        ws_bytes < align256((size_t)batch * plane_bytes(b)) + (size_t)stage_override * plane_bytes(b))
      s = fail(SHL_EINVAL, "workspace too small for the requested staging depth");
  }
  if (s != SHL_OK || batch == 0) return s;
  if (!x || !coeffs || !aligned16(x) || !aligned16(coeffs))
    return fail(SHL_EINVAL, "x and coeffs must be 16-byte aligned device pointers");
  if (mode == shl::IN_MASKED && (!mask || !fest || !aligned16(fest) || !aligned16(mask)))
    return fail(SHL_EINVAL, "mask and f_est must be 16-byte aligned device pointers");
  x = device_view(x, b->device);
  if (mode == shl::IN_MASKED) {
    mask = device_view(mask, b->device);
    fest = device_view(fest, b->device);
    if (!mask || !fest) return fail(SHL_EINVAL, "mask / f_est not accessible from the bank's device");
  }
  if (!x) return fail(SHL_EINVAL, "x not accessible from the bank's device (device or mapped pinned memory)");
  if (dtype != SHL_F32 && dtype != SHL_BF16) return fail(SHL_EINVAL, "bad dtype");
  if (flags & ~SHL_DUAL_WEIGHTED) return fail(SHL_EINVAL, "unknown flags");
  DevGuard g(b->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (b->general) {
    const int S = stage_override > 0 ? stage_override : stage_subbands(b);
    cudaError_t e = gen_decompose(b, mode, x, mask, fest, batch, coeffs, dtype,
                                  (flags & SHL_DUAL_WEIGHTED) != 0, ws, S, st);
    return e ? cuda_fail(e, "general decomposition") : SHL_OK;
  }
  const int N = b->N, M = b->M, K = b->K, Mh = b->Mh;
  float2* X = static_cast<float2*>(ws);
  float2* Z = reinterpret_cast<float2*>(static_cast<char*>(ws) +
                                        align256((size_t)batch * plane_bytes(b)));
  cudaError_t e;
  {
    Launch L_("rows_r2c_image", st);
    e = shl::launch_rows_r2c_t(M, mode, false, x, mask, fest, nullptr, X, N, batch, b->dTw, st);
  }
  if (e) return cuda_fail(e, "rows_r2c_image");
  {
    Launch L_("lines_fwd_image", st);
    e = shl::launch_lines_fwd(N, X, batch * Mh, b->dTw, st);
  }
  if (e) return cuda_fail(e, "lines_fwd_image");
  const int total = batch * K;
  const size_t esz = dtype == SHL_BF16 ? 2 : 4;
  const float scale = (float)(1.0 / (double(N) * M));
  const float* invW = (flags & SHL_DUAL_WEIGHTED) ? b->dInvW : nullptr;
  if (stage_override <= 0 && use_pair(b)) {
    float2* slots = reinterpret_cast<float2*>(static_cast<char*>(ws) +
                                              align256((size_t)batch * plane_bytes(b)));
    const int ncl = shl::pair_clusters_for(pair_ncl_max(b), batch * ((K + 1) / 2));
    {
      Launch L_("pair_dec", st);
      e = shl::launch_pair_dec(N, dtype == SHL_BF16, X, b->dG, invW, coeffs, slots, ncl, scale, K,
                               batch, b->dTw, st);
    }
    if (e) return cuda_fail(e, "pair_dec");
    return SHL_OK;
  }
  if (stage_override <= 0 && use_pipe(b)) {
    const PipeCfg& c = pipe_cfg();
    unsigned* ctl = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(Z) +
                                                align256((size_t)c.NS * c.CS * plane_bytes(b)));
    {
      Launch L_("dec_pipe", st);
      e = shl::launch_dec_pipe(N, M, dtype == SHL_BF16, X, Z, coeffs, b->dG, invW, scale, K, total,
                               c.CS, c.NS, c.col_frac, ctl, b->dTw, st);
    }
    if (e) return cuda_fail(e, "dec_pipe");
    return SHL_OK;
  }
  const int S = stage_override > 0 ? stage_override : stage_subbands(b);
  const bool tc = use_tc_dft(b, dtype);
  // bfloat16 coefficients: the staged half spectra between the column and the
  // row pass are bfloat16 too (half the staging traffic; the rounding is of
  // the size of the coefficients' own)
  const bool s16 = dtype == SHL_BF16;
  for (int s0 = 0; s0 < total; s0 += S) {
    const int Sc = std::min(S, total - s0);
    if (tc) {
      Launch L_("dec_lines_tc", st);
      e = shl::launch_dec_lines_tc(N, X, Z, b->dG, invW, scale, Mh, K, s0, Sc, b->dTw, st, batch,
                                    s16);
    } else {
      Launch L_("dec_lines", st);
      e = shl::launch_dec_lines(N, X, Z, b->dG, invW, scale, Mh, K, s0, Sc, b->dTw, st, batch, s16);
    }
    if (e) return cuda_fail(e, "dec_lines");
    {
      Launch L_("rows_c2r_coeffs", st);
      e = shl::launch_rows_c2r_t(M, dtype == SHL_BF16, Z,
                                 static_cast<char*>(coeffs) + (size_t)s0 * N * M * esz, N, Sc,
                                 b->dTw, st, s16);
    }
    if (e) return cuda_fail(e, "rows_c2r_coeffs");
  }
  return SHL_OK;
}

// Reconstruction-style chunks (whole images when the staging area holds K
// subbands, else filter ranges inside one image), shared by reconstruct_impl
// and shrink_impl.
int next_chunk(int s0, int total, int S, int K) {
  if (S >= K) return std::min((S / K) * K, total - s0);
  const int img_end = (s0 / K + 1) * K;
  return std::min(S, img_end - s0);
}

// Reconstruction chunks: whole images when the staging area holds K
// subbands, otherwise filter ranges inside one image (partial sums are
// carried in the accumulator plane of that image).
shl_status reconstruct_impl(const shl_bank* b, const void* coeffs, shl_dtype dtype, int batch,
                            const float* thresh, float* x_out, void* ws, size_t ws_bytes,
                            void* stream, bool weights) {
  shl_status s = check_common(b, batch, ws, ws_bytes, SHL_OP_RECONSTRUCT);
  if (s != SHL_OK || batch == 0) return s;
  if (!coeffs || !x_out || !aligned16(coeffs) || !aligned16(x_out))
    return fail(SHL_EINVAL, "coeffs and x_out must be 16-byte aligned device pointers");
  x_out = device_view(x_out, b->device);
  if (!x_out) return fail(SHL_EINVAL, "x_out not accessible from the bank's device (device or mapped pinned memory)");
  if (thresh && (reinterpret_cast<uintptr_t>(thresh) & 3u))
    return fail(SHL_EINVAL, "thresh must be 4-byte aligned");
  if (dtype != SHL_F32 && dtype != SHL_BF16) return fail(SHL_EINVAL, "bad dtype");
  DevGuard g(b->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (b->general) {
    cudaError_t e = gen_reconstruct(b, coeffs, dtype, batch, thresh, x_out, ws, weights, st);
    return e ? cuda_fail(e, "general reconstruction") : SHL_OK;
  }
  const int N = b->N, M = b->M, K = b->K, Mh = b->Mh;
  float2* A = static_cast<float2*>(ws);
  float2* Z = reinterpret_cast<float2*>(static_cast<char*>(ws) +
                                        align256((size_t)batch * plane_bytes(b)));
  const int total = batch * K, S = stage_subbands(b);
  const size_t esz = dtype == SHL_BF16 ? 2 : 4;
  const float scale = (float)(1.0 / (double(N) * M));
  cudaError_t e;
  if (use_pair(b)) {
    const int ncl_max = pair_ncl_max(b);
    const int ncl = shl::pair_clusters_for(ncl_max, batch * ((K + 1) / 2));
    float2* parts = reinterpret_cast<float2*>(reinterpret_cast<char*>(Z) +
                                              align256((size_t)ncl_max * pair_slot_bytes(b)));
    {
      Launch L_("pair_rec", st);
      e = shl::launch_pair_rec(N, dtype == SHL_BF16, coeffs, thresh, b->dG, Z, parts, ncl, K, batch,
                               b->dTw, st);
    }
    if (e) return cuda_fail(e, "pair_rec");
    {
      Launch L_("pair_final", st);
      e = shl::launch_pair_final(N, parts, A, weights ? b->dInvW : nullptr, scale, K, batch, ncl,
                                 b->dTw, st);
    }
    if (e) return cuda_fail(e, "pair_final");
    {
      Launch L_("rows_c2r_image", st);
      e = shl::launch_rows_c2r_t(M, false, A, x_out, N, batch, b->dTw, st);
    }
    if (e) return cuda_fail(e, "rows_c2r_image");
    return SHL_OK;
  }
  for (int s0 = 0; s0 < total;) {
    const int Sc = next_chunk(s0, total, S, K);
    {
      Launch L_("rows_r2c_coeffs", st);
      e = shl::launch_rows_r2c_t(M, dtype == SHL_BF16 ? shl::IN_BF16 : shl::IN_F32,
                                 thresh != nullptr,
                                 static_cast<const char*>(coeffs) + (size_t)s0 * N * M * esz,
                                 nullptr, nullptr, thresh ? thresh + s0 : nullptr, Z, N, Sc,
                                 b->dTw, st);
    }
    if (e) return cuda_fail(e, "rows_r2c_coeffs");
    {
      Launch L_("rec_lines", st);
      e = shl::launch_rec_lines(N, Z, A, b->dG, weights ? b->dInvW : nullptr, scale, Mh, K, s0,
                                Sc, b->dTw, st, batch);
    }
    if (e) return cuda_fail(e, "rec_lines");
    s0 += Sc;
  }
  {
    Launch L_("rows_c2r_image", st);
    e = shl::launch_rows_c2r_t(M, false, A, x_out, N, batch, b->dTw, st);
  }
  if (e) return cuda_fail(e, "rows_c2r_image");
  return SHL_OK;
}

shl_status shrink_impl(const shl_bank* b, const float* x, const unsigned char* mask,
                       const float* fest, int batch, const float* thresh, float* x_out, void* ws,
                       size_t ws_bytes, void* stream) {
  shl_status s = check_common(b, batch, ws, ws_bytes, SHL_OP_SHRINK);
  if (s != SHL_OK || batch == 0) return s;
  if (!x || !x_out || !thresh || !aligned16(x) || !aligned16(x_out))
    return fail(SHL_EINVAL, "x, thresh and x_out must be device pointers (x, x_out 16-byte aligned)");
  if (reinterpret_cast<uintptr_t>(thresh) & 3u) return fail(SHL_EINVAL, "thresh must be 4-byte aligned");
  if (mask && (!fest || !aligned16(fest) || !aligned16(mask)))
    return fail(SHL_EINVAL, "mask and f_est must be 16-byte aligned device pointers");
  x = device_view(x, b->device);
  x_out = device_view(x_out, b->device);
  if (mask) {
    mask = device_view(mask, b->device);
    fest = device_view(fest, b->device);
    if (!mask || !fest) return fail(SHL_EINVAL, "mask / f_est not accessible from the bank's device");
  }
  if (!x || !x_out) return fail(SHL_EINVAL, "x / x_out not accessible from the bank's device");
  DevGuard g(b->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (b->general) {
    cudaError_t e = gen_shrink(b, x, mask, fest, batch, thresh, x_out, ws, st);
    return e ? cuda_fail(e, "general shrink") : SHL_OK;
  }
  const int N = b->N, M = b->M, K = b->K, Mh = b->Mh;
  const size_t img = align256((size_t)batch * plane_bytes(b));
  float2* X = static_cast<float2*>(ws);
  float2* A = reinterpret_cast<float2*>(static_cast<char*>(ws) + img);
  float2* Z = reinterpret_cast<float2*>(static_cast<char*>(ws) + 2 * img);
  const float scale = (float)(1.0 / (double(N) * M));
  cudaError_t e;
  {
    Launch L_("rows_r2c_image", st);
    e = shl::launch_rows_r2c_t(M, mask ? shl::IN_MASKED : shl::IN_F32, false, x, mask, fest,
                               nullptr, X, N, batch, b->dTw, st);
  }
  if (e) return cuda_fail(e, "rows_r2c_image");
  {
    Launch L_("lines_fwd_image", st);
    e = shl::launch_lines_fwd(N, X, batch * Mh, b->dTw, st);
  }
  if (e) return cuda_fail(e, "lines_fwd_image");
  const int total = batch * K, S = stage_subbands(b);
  for (int s0 = 0; s0 < total;) {
    const int Sc = next_chunk(s0, total, S, K);
    {
      Launch L_("dec_lines", st);
      e = shl::launch_dec_lines(N, X, Z, b->dG, nullptr, scale, Mh, K, s0, Sc, b->dTw, st,
                                   batch);
    }
    if (e) return cuda_fail(e, "dec_lines");
    {
      Launch L_("rows_shrink", st);
      e = shl::launch_rows_shrink_t(M, Z, thresh + s0, N, Sc, b->dTw, st);
    }
    if (e) return cuda_fail(e, "rows_shrink");
    {
      Launch L_("rec_lines", st);
      e = shl::launch_rec_lines(N, Z, A, b->dG, b->dInvW, scale, Mh, K, s0, Sc, b->dTw, st,
                                  batch);
    }
    if (e) return cuda_fail(e, "rec_lines");
    s0 += Sc;
  }
  {
    Launch L_("rows_c2r_image", st);
    e = shl::launch_rows_c2r_t(M, false, A, x_out, N, batch, b->dTw, st);
  }
  if (e) return cuda_fail(e, "rows_c2r_image");
  return SHL_OK;
}

// ------------------------------------------------------- general path
// Launch sequences of general.cu: row-major half-spectrum planes [N][Mh]
// (N * Mh * 8 bytes, as on the power-of-two path).  Same chunking as the
// power-of-two path.
cudaError_t gen_image_spectra(const shl_bank* b, shl::InMode mode, const float* x,
                              const unsigned char* mask, const float* fest, int batch, float2* X,
                              cudaStream_t st) {
  namespace G = shl::gen;
  const int N = b->N, Mh = b->Mh;
  cudaError_t e;
  {
    Launch L_("gen_rows_fwd_image", st);
    e = G::launch_rows_fwd(b->planM, mode == shl::IN_MASKED ? G::RIN_MASKED : G::RIN_F32, x, mask,
                           fest, nullptr, X, N, batch, st);
  }
  if (e) return e;
  for (int b0 = 0; b0 < batch; b0 += 65535) {
    Launch L_("gen_cols_fwd_image", st);
    e = G::launch_cols_fwd(b->planN, X + (size_t)b0 * N * Mh, Mh, std::min(65535, batch - b0), st);
    if (e) return e;
  }
  return cudaSuccess;
}

cudaError_t gen_decompose(const shl_bank* b, shl::InMode mode, const float* x,
                          const unsigned char* mask, const float* fest, int batch, void* coeffs,
                          shl_dtype dtype, bool dual, void* ws, int S, cudaStream_t st) {
  namespace G = shl::gen;
  const int N = b->N, M = b->M, K = b->K;
  float2* X = static_cast<float2*>(ws);
  float2* Z = reinterpret_cast<float2*>(static_cast<char*>(ws) +
                                        align256((size_t)batch * plane_bytes(b)));
  cudaError_t e = gen_image_spectra(b, mode, x, mask, fest, batch, X, st);
  if (e) return e;
  const int total = batch * K;
  const size_t esz = dtype == SHL_BF16 ? 2 : 4;
  const float scale = (float)(1.0 / (double(N) * M));
  S = std::min(S, 65535);
  for (int s0 = 0; s0 < total; s0 += S) {
    const int Sc = std::min(S, total - s0);
    {
      Launch L_("gen_cols_dec", st);
      e = G::launch_cols_dec(b->planN, X, Z, b->dGg, b->cplx, dual ? b->dInvWg : nullptr, b->Mh,
                             K, s0, Sc, st);
    }
    if (e) return e;
    {
      Launch L_("gen_rows_inv_coeffs", st);
      e = G::launch_rows_inv(b->planM, Z, static_cast<char*>(coeffs) + (size_t)s0 * N * M * esz,
                             dtype == SHL_BF16, scale, N, Sc, st);
    }
    if (e) return e;
  }
  return cudaSuccess;
}

cudaError_t gen_reconstruct(const shl_bank* b, const void* coeffs, shl_dtype dtype, int batch,
                            const float* thresh, float* x_out, void* ws, bool weights,
                            cudaStream_t st) {
  namespace G = shl::gen;
  const int N = b->N, M = b->M, K = b->K;
  float2* A = static_cast<float2*>(ws);
  float2* Z = reinterpret_cast<float2*>(static_cast<char*>(ws) +
                                        align256((size_t)batch * plane_bytes(b)));
  const int total = batch * K, S = stage_subbands(b);
  const size_t esz = dtype == SHL_BF16 ? 2 : 4;
  cudaError_t e;
  for (int s0 = 0; s0 < total;) {
    const int Sc = next_chunk(s0, total, S, K);
    {
      Launch L_("gen_rows_fwd_coeffs", st);
      e = G::launch_rows_fwd(b->planM, dtype == SHL_BF16 ? G::RIN_BF16 : G::RIN_F32,
                             static_cast<const char*>(coeffs) + (size_t)s0 * N * M * esz, nullptr,
                             nullptr, thresh ? thresh + s0 : nullptr, Z, N, Sc, st);
    }
    if (e) return e;
    {
      Launch L_("gen_cols_rec", st);
      e = G::launch_cols_rec(b->planN, Z, A, b->dGg, b->cplx, weights ? b->dInvWg : nullptr,
                             b->Mh, K, s0, Sc, st);
    }
    if (e) return e;
    s0 += Sc;
  }
  Launch L_("gen_rows_inv_image", st);
  return G::launch_rows_inv(b->planM, A, x_out, false, (float)(1.0 / (double(N) * M)), N, batch,
                            st);
}

cudaError_t gen_shrink(const shl_bank* b, const float* x, const unsigned char* mask,
                       const float* fest, int batch, const float* thresh, float* x_out, void* ws,
                       cudaStream_t st) {
  namespace G = shl::gen;
  const int N = b->N, M = b->M, K = b->K;
  const size_t img = align256((size_t)batch * plane_bytes(b));
  float2* X = static_cast<float2*>(ws);
  float2* A = reinterpret_cast<float2*>(static_cast<char*>(ws) + img);
  float2* Z = reinterpret_cast<float2*>(static_cast<char*>(ws) + 2 * img);
  const float scale = (float)(1.0 / (double(N) * M));
  cudaError_t e = gen_image_spectra(b, mask ? shl::IN_MASKED : shl::IN_F32, x, mask, fest, batch,
                                    X, st);
  if (e) return e;
  const int total = batch * K, S = stage_subbands(b);
  for (int s0 = 0; s0 < total;) {
    const int Sc = next_chunk(s0, total, S, K);
    {
      Launch L_("gen_cols_dec", st);
      e = G::launch_cols_dec(b->planN, X, Z, b->dGg, b->cplx, nullptr, b->Mh, K, s0, Sc, st);
    }
    if (e) return e;
    {
      Launch L_("gen_rows_shrink", st);
      e = G::launch_rows_shrink(b->planM, Z, thresh + s0, scale, N, Sc, st);
    }
    if (e) return e;
    {
      Launch L_("gen_cols_rec", st);
      e = G::launch_cols_rec(b->planN, Z, A, b->dGg, b->cplx, b->dInvWg, b->Mh, K, s0, Sc, st);
    }
    if (e) return e;
    s0 += Sc;
  }
  Launch L_("gen_rows_inv_image", st);
  return G::launch_rows_inv(b->planM, A, x_out, false, scale, N, batch, st);
}

}  // namespace

namespace shl {
shl_status set_error(shl_status s, const char* msg) { return fail(s, msg); }

shl_status bank_geometry(const shl_bank* b, int* device, size_t* plane) {
  if (!b) return fail(SHL_EINVAL, "bank is NULL");
  *device = b->device;
  *plane = plane_bytes(b);
  return SHL_OK;
}

shl_status decompose_staged(const shl_bank* b, const float* x, int batch, void* coeffs,
                            shl_dtype dtype, int flags, void* ws, size_t ws_bytes, void* stream,
                            int stage_subbands_max) {
  return decompose_impl(b, IN_F32, x, nullptr, nullptr, batch, coeffs, dtype, flags, ws, ws_bytes,
                        stream, stage_subbands_max);
}
}  // namespace shl

extern "C" {

int shl_abi_version(void) { return SHL_ABI_VERSION; }

const char* shl_status_str(shl_status s) {
  switch (s) {
    case SHL_OK: return "ok";
    case SHL_EINVAL: return "invalid argument";
    case SHL_ENOMEM: return "out of memory";
    case SHL_ECUDA: return "CUDA error";
    case SHL_EUNSUPPORTED: return "unsupported";
    case SHL_ETIMEOUT: return "device wait timed out";
    case SHL_EDEVICE: return "device reported an error";
  }
  return "unknown status";
}

const char* shl_last_error_detail(void) { return g_err.c_str(); }

}  // extern "C"

namespace {
// Validates spectra in natural order: finite, and even (real spectra) or
// Hermitian (complex): G(-k) = conj(G(k)), within 1e-9 of the largest
// magnitude, so that real images give real coefficients.
shl_status check_spectra(int N, int M, int K, const double* re, const double* im) {
  for (int i = 0; i < K; ++i) {
    const double* R = re + (size_t)i * N * M;
    const double* I = im ? im + (size_t)i * N * M : nullptr;
    double mx = 0.0, asym = 0.0;
    for (int y = 0; y < N; ++y)
      for (int x = 0; x < M; ++x) {
        const size_t e = (size_t)y * M + x, f = (size_t)((N - y) % N) * M + (M - x) % M;
        const double a = R[e], ai = I ? I[e] : 0.0;
        if (!std::isfinite(a) || !std::isfinite(ai)) return fail(SHL_EINVAL, "spectra must be finite");
        mx = std::max(mx, std::hypot(a, ai));
        asym = std::max(asym, std::hypot(a - R[f], I ? ai + I[f] : 0.0));
      }
    if (asym > 1e-9 * mx)
      return fail(SHL_EINVAL, "spectrum " + std::to_string(i) +
                                  (I ? " is not Hermitian: G(-k) != conj(G(k))"
                                     : " is not even: G(-k) != G(k)"));
  }
  return SHL_OK;
}

shl_status make_bank(int N, int M, int K, std::vector<double>&& re, std::vector<double>&& im,
                     std::vector<int>&& idx, bool general, int device, shl_bank** out) {
  shl_bank* b = new shl_bank();
  b->device = device; b->N = N; b->M = M; b->Mh = M / 2 + 1; b->K = K;
  b->general = general;
  b->cplx = !im.empty();
  b->spectra = std::move(re);
  b->spectra_im = std::move(im);
  b->idx = std::move(idx);
  b->idx.resize((size_t)K * 3, 0);
  shl_status s = upload_bank(b);
  if (s != SHL_OK) { free_bank(b); return s; }
  *out = b;
  return SHL_OK;
}
}  // namespace

extern "C" {

shl_status shl_bank_create_from_spectra(int rows, int cols, int K, const double* spectra,
                                        const int* idx, int device, shl_bank** out) {
  if (!out) return fail(SHL_EINVAL, "out is NULL");
  *out = nullptr;
  shl_status s = check_general_size(rows, cols);
  if (s != SHL_OK) return s;
  if (K < 1 || K > 4096 || !spectra) return fail(SHL_EINVAL, "need 1 <= K <= 4096 and spectra");
  if ((s = check_spectra(rows, cols, K, spectra, nullptr)) != SHL_OK) return s;
  std::vector<int> ix(idx ? idx : nullptr, idx ? idx + 3 * (size_t)K : nullptr);
  return make_bank(rows, cols, K, std::vector<double>(spectra, spectra + (size_t)K * rows * cols),
                   {}, std::move(ix), !fast_size(rows, cols), device, out);
}

shl_status shl_bank_create_general(int rows, int cols, int K, const double* spectra_re,
                                   const double* spectra_im, const int* idx, int device,
                                   shl_bank** out) {
  if (!out) return fail(SHL_EINVAL, "out is NULL");
  *out = nullptr;
  shl_status s = check_general_size(rows, cols);
  if (s != SHL_OK) return s;
  if (K < 1 || K > 4096 || !spectra_re) return fail(SHL_EINVAL, "need 1 <= K <= 4096 and spectra");
  if ((s = check_spectra(rows, cols, K, spectra_re, spectra_im)) != SHL_OK) return s;
  const size_t n = (size_t)K * rows * cols;
  std::vector<int> ix(idx ? idx : nullptr, idx ? idx + 3 * (size_t)K : nullptr);
  return make_bank(rows, cols, K, std::vector<double>(spectra_re, spectra_re + n),
                   spectra_im ? std::vector<double>(spectra_im, spectra_im + n)
                              : std::vector<double>(),
                   std::move(ix), true, device, out);
}

shl_status shl_bank_create(int rows, int cols, int n_scales, const int* shear_levels, int full,
                           int device, shl_bank** out) {
  if (!out) return fail(SHL_EINVAL, "out is NULL");
  *out = nullptr;
  shl_status s = check_general_size(rows, cols);
  if (s != SHL_OK) return s;
  shl::HostBank hb;
  const char* msg = shl::build_shearlet_bank(rows, cols, n_scales, shear_levels, full, &hb);
  if (msg && *msg) return fail(SHL_EINVAL, msg);
  return make_bank(rows, cols, hb.K, std::move(hb.spectra), {}, std::move(hb.idx),
                   !fast_size(rows, cols), device, out);
}

shl_status shl_bank_create_gpu(int rows, int cols, int n_scales, const int* shear_levels,
                               int full, int device, shl_bank** out) {
  if (!out) return fail(SHL_EINVAL, "out is NULL");
  *out = nullptr;
  shl_status s = check_size(rows, cols);
  if (s != SHL_OK)
    return fail(SHL_EUNSUPPORTED, "shl_bank_create_gpu builds power-of-two sizes in [16, 2048]; "
                                  "shl_bank_create builds the others on the host");
  if (device < 0) return fail(SHL_EINVAL, "shl_bank_create_gpu needs a device >= 0");
  std::vector<shl::BankItem> items;
  const char* err = shl::bank_items(n_scales, shear_levels, full, &items);
  if (*err) return fail(SHL_EINVAL, err);
  const int N = rows, M = cols, Mh = M / 2 + 1, K = (int)items.size();
  const size_t plane = (size_t)N * M;
  DevGuard g(device);
  shl_bank* b = new shl_bank;
  b->device = device; b->N = N; b->M = M; b->Mh = Mh; b->K = K;
  b->idx.assign((size_t)K * 3, 0);
  for (int i = 0; i < K; ++i) {
    b->idx[3 * i] = items[i].cone;
    b->idx[3 * i + 1] = items[i].scale;
    b->idx[3 * i + 2] = items[i].k;
  }
  double *dS = nullptr, *dT = nullptr, *dW = nullptr, *dR = nullptr;
  unsigned* dBad = nullptr;
  auto cleanup = [&]() {
    if (dS) cudaFree(dS);
    if (dT) cudaFree(dT);
    if (dW) cudaFree(dW);
    if (dR) cudaFree(dR);
    if (dBad) cudaFree(dBad);
  };
  if (cudaMalloc(&dS, sizeof(double) * K * plane) || cudaMalloc(&dT, sizeof(double) * plane) ||
      cudaMalloc(&dW, sizeof(double) * plane) || cudaMalloc(&dR, sizeof(double) * K) ||
      cudaMalloc(&dBad, sizeof(unsigned)) ||
      cudaMalloc(&b->dG, sizeof(float) * (size_t)K * Mh * N) ||
      cudaMalloc(&b->dInvW, sizeof(float) * (size_t)Mh * N) ||
      cudaMalloc(&b->dTw, sizeof(float2) * shl::TW_P) ||
      cudaMalloc(&b->dRms, sizeof(float) * K)) {
    cudaGetLastError();
    cleanup();
    free_bank(b);
    return fail(SHL_ENOMEM, "cudaMalloc failed for the filter bank");
  }
  cudaError_t e = shl::build_bank_device(rows, cols, n_scales, shear_levels, full, items, dS, dT, dW,
                                         dR, b->dG, b->dInvW, dBad, nullptr);
  unsigned bad = 0;
  b->spectra.resize((size_t)K * plane);
  b->dual_w.resize(plane);
  b->rms.resize(K);
  if (!e) e = cudaMemcpy(&bad, dBad, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (!e) e = cudaMemcpy(b->rms.data(), dR, sizeof(double) * K, cudaMemcpyDeviceToHost);
  if (!e) e = cudaMemcpy(b->dual_w.data(), dW, sizeof(double) * plane, cudaMemcpyDeviceToHost);
  if (!e)
    e = cudaMemcpy(b->spectra.data(), dS, sizeof(double) * K * plane, cudaMemcpyDeviceToHost);
  const std::vector<float2> hT = twiddle_table();
  std::vector<float> hR(K);
  for (int i = 0; i < K; ++i) hR[i] = (float)b->rms[i];
  if (!e) e = cudaMemcpy(b->dTw, hT.data(), sizeof(float2) * hT.size(), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(b->dRms, hR.data(), sizeof(float) * K, cudaMemcpyHostToDevice);
  cleanup();
  if (e) {
    free_bank(b);
    return cuda_fail(e, "shl_bank_create_gpu");
  }
  if (bad) {
    free_bank(b);
    return fail(SHL_EINVAL, "dual frame weights W = sum G_i^2 must be > 0");
  }
  *out = b;
  return SHL_OK;
}

shl_status shl_bank_destroy(shl_bank* bank) {
  if (!bank) return SHL_OK;
  if (bank->device < 0) { free_bank(bank); return SHL_OK; }
  DevGuard g(bank->device);
  free_bank(bank);
  return SHL_OK;
}

shl_status shl_bank_query(const shl_bank* b, int* K, int* rows, int* cols) {
  if (!b) return fail(SHL_EINVAL, "bank is NULL");
  if (K) *K = b->K;
  if (rows) *rows = b->N;
  if (cols) *cols = b->M;
  return SHL_OK;
}

shl_status shl_bank_copy_info(const shl_bank* b, int* idx, double* rms, double* spectra,
                              double* dual_w) {
  if (!b) return fail(SHL_EINVAL, "bank is NULL");
  if (idx) std::memcpy(idx, b->idx.data(), b->idx.size() * sizeof(int));
  if (rms) std::memcpy(rms, b->rms.data(), b->rms.size() * sizeof(double));
  if (spectra) std::memcpy(spectra, b->spectra.data(), b->spectra.size() * sizeof(double));
  if (dual_w) std::memcpy(dual_w, b->dual_w.data(), b->dual_w.size() * sizeof(double));
  return SHL_OK;
}

shl_status shl_bank_path(const shl_bank* b, int* general) {
  if (!b || !general) return fail(SHL_EINVAL, "bank and general must be non-NULL");
  *general = b->general ? 1 : 0;
  return SHL_OK;
}

shl_status shl_bank_copy_spectra_imag(const shl_bank* b, double* imag) {
  if (!b || !imag) return fail(SHL_EINVAL, "bank and imag must be non-NULL");
  const size_t n = (size_t)b->K * b->N * b->M;
  if (b->cplx) std::memcpy(imag, b->spectra_im.data(), n * sizeof(double));
  else std::memset(imag, 0, n * sizeof(double));
  return SHL_OK;
}

shl_status shl_workspace_size(const shl_bank* b, shl_op op, int batch, size_t* bytes) {
  if (!b || !bytes) return fail(SHL_EINVAL, "bank and bytes must be non-NULL");
  if (batch < 0) return fail(SHL_EINVAL, "batch must be >= 0");
  if (op != SHL_OP_DECOMPOSE && op != SHL_OP_RECONSTRUCT && op != SHL_OP_SHRINK)
    return fail(SHL_EINVAL, "bad op");
  *bytes = batch == 0 ? 0 : ws_need(b, batch, op);
  return SHL_OK;
}

shl_status shl_decompose(const shl_bank* b, const float* x, int batch, void* coeffs,
                         shl_dtype dtype, int flags, void* ws, size_t ws_bytes, void* stream) {
  return decompose_impl(b, shl::IN_F32, x, nullptr, nullptr, batch, coeffs, dtype, flags, ws,
                        ws_bytes, stream);
}

shl_status shl_decompose_masked(const shl_bank* b, const float* f_masked,
                                const unsigned char* mask, const float* f_est, int batch,
                                void* coeffs, shl_dtype dtype, void* ws, size_t ws_bytes,
                                void* stream) {
  return decompose_impl(b, shl::IN_MASKED, f_masked, mask, f_est, batch, coeffs, dtype, 0, ws,
                        ws_bytes, stream);
}

shl_status shl_reconstruct(const shl_bank* b, const void* coeffs, shl_dtype dtype, int batch,
                           const float* thresh, float* x_out, void* ws, size_t ws_bytes,
                           void* stream) {
  return reconstruct_impl(b, coeffs, dtype, batch, thresh, x_out, ws, ws_bytes, stream, true);
}

shl_status shl_adjoint(const shl_bank* b, const void* coeffs, shl_dtype dtype, int batch,
                       const float* thresh, float* x_out, void* ws, size_t ws_bytes,
                       void* stream) {
  return reconstruct_impl(b, coeffs, dtype, batch, thresh, x_out, ws, ws_bytes, stream, false);
}

shl_status shl_shrink(const shl_bank* b, const float* x, const unsigned char* mask,
                      const float* f_est, int batch, const float* thresh, float* x_out, void* ws,
                      size_t ws_bytes, void* stream) {
  return shrink_impl(b, x, mask, f_est, batch, thresh, x_out, ws, ws_bytes, stream);
}

shl_status shl_subband_absmax(const shl_bank* b, const void* coeffs, shl_dtype dtype, int batch,
                              int by_rms, float* out, void* stream) {
  if (!b) return fail(SHL_EINVAL, "bank is NULL");
  if (batch < 0) return fail(SHL_EINVAL, "batch must be >= 0");
  if (batch == 0) return SHL_OK;
  if (b->device < 0) return fail(SHL_EINVAL, "bank was created host-only (device < 0)");
  if (!coeffs || !out || !aligned16(coeffs)) return fail(SHL_EINVAL, "bad coeffs / out pointer");
  DevGuard g(b->device);
  cudaError_t e;
  {
    Launch L_("absmax", static_cast<cudaStream_t>(stream));
    e = shl::launch_absmax(coeffs, dtype == SHL_BF16, batch * b->K, b->K, (size_t)b->N * b->M,
                           by_rms ? b->dRms : nullptr, out, static_cast<cudaStream_t>(stream));
  }
  if (e) return cuda_fail(e, "absmax");
  return SHL_OK;
}

shl_status shl_iht_thresholds(const shl_bank* b, const float* absmax_by_rms, int batch,
                              int iterations, double delta_min, float* out, void* stream) {
  if (!b) return fail(SHL_EINVAL, "bank is NULL");
  if (batch < 0 || iterations < 0) return fail(SHL_EINVAL, "batch and iterations must be >= 0");
  if (batch == 0 || iterations == 0) return SHL_OK;
  if (!(delta_min > 0.0)) return fail(SHL_EINVAL, "delta_min must be > 0");
  if (b->device < 0) return fail(SHL_EINVAL, "bank was created host-only (device < 0)");
  if (!absmax_by_rms || !out) return fail(SHL_EINVAL, "bad absmax / out pointer");
  DevGuard g(b->device);
  cudaError_t e;
  {
    Launch L_("iht_schedule", static_cast<cudaStream_t>(stream));
    e = shl::launch_iht_schedule(absmax_by_rms, b->dRms, b->K, batch, iterations, delta_min, out,
                                 static_cast<cudaStream_t>(stream));
  }
  if (e) return cuda_fail(e, "iht_schedule");
  return SHL_OK;
}

long long shl_launch_count(void) { return g_launches.load(); }

shl_status shl_profile_enable(int on) {
  g_profile.store(on ? 1 : 0);
  return SHL_OK;
}

shl_status shl_profile_read(char* buf, size_t len) {
  std::vector<ProfRec> recs;
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    recs.swap(g_prof);
  }
  std::map<std::string, std::pair<long long, double>> agg;
  cudaError_t err = cudaSuccess;
  for (auto& r : recs) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess && err == cudaSuccess) err = e;
    auto& slot = agg[r.name];
    slot.first += 1;
    slot.second += ms;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  std::string js = "{";
  bool first = true;
  for (auto& kv : agg) {
    char tmp[160];
    std::snprintf(tmp, sizeof tmp, "%s\"%s\": {\"launches\": %lld, \"ms\": %.6f}",
                  first ? "" : ", ", kv.first.c_str(), kv.second.first, kv.second.second);
    js += tmp;
    first = false;
  }
  js += "}";
  if (buf && len) {
    std::strncpy(buf, js.c_str(), len - 1);
    buf[len - 1] = 0;
  }
  if (err != cudaSuccess) return cuda_fail(err, "shl_profile_read");
  if (js.size() + 1 > len) return fail(SHL_EINVAL, "buffer too small for the profile summary");
  return SHL_OK;
}

shl_status shl_check_status(int device, unsigned* word) {
  if (!word) return fail(SHL_EINVAL, "word is NULL");
  DevGuard g(device);
  cudaError_t e = cudaDeviceSynchronize();
  if (!e) e = shl::read_check_word(word);
  unsigned w2 = 0;
  if (!e) e = shl::read_check_word_tc(&w2);
  if (!e) *word |= w2;
  if (e) return cuda_fail(e, "shl_check_status");
  return SHL_OK;
}

int shl_checked_build(void) {
#ifdef SHL_CHECKED
  return 1;
#else
  return 0;
#endif
}

shl_status shl_sync(void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e) return cuda_fail(e, "shl_sync");
  // the wait flag lives on the stream's device: read and clear it there
  int dev = -1;
  if ((e = cudaStreamGetDevice(st, &dev))) return cuda_fail(e, "shl_sync");
  DevGuard g(dev);
  unsigned flag = 0, dft = 0;
  if ((e = shl::read_pipe_error(&flag))) return cuda_fail(e, "shl_sync");
  if ((e = shl::read_dft_error(&dft))) return cuda_fail(e, "shl_sync");
  if (dft)
    return fail(SHL_ETIMEOUT, "tensor-core column pass: a wait for its MMAs ran out; the "
                             "coefficients of that call are incomplete");
  if (flag & 1u)
    return fail(SHL_ETIMEOUT, "pipelined decomposition: a wait between its passes ran out; the "
                             "coefficients of that call are incomplete");
  if (flag)
    return fail(SHL_ETIMEOUT, "a row pass gave up waiting for a bulk copy of its input tile; the "
                             "results of that call are incomplete");
  return SHL_OK;
}

}  // extern "C"
