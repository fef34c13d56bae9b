// noalloc.cu - a decomposition entry point that allocates nothing.
//
// shl_decompose needs a device workspace from its caller.  Some callers have
// no way to provide one: a host framework may own every byte of device
// memory and expose no allocator to plug-ins, a latency-critical loop may not
// afford cudaMalloc (it can synchronise the whole device), and a service
// running at its memory budget must not fail with out-of-memory at call
// time.  For them, shl_decompose_noalloc uses a scratch array compiled into
// this library instead: SHL_NOALLOC_SCRATCH_BYTES of device memory that every
// GPU holds, once loaded, until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace {

constexpr size_t kScratchBytes = SHL_NOALLOC_SCRATCH_BYTES;

// Scratch of shl_decompose_noalloc: image spectra, then per-subband staging.
// Every call uses it from the start; nothing in it has to begin at zero.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on `device`, looked up once per device
// with that device current (the host-side symbol is not a device address).
shl_status scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices)
    return shl::set_error(SHL_EINVAL, "device index out of range for the fixed scratch");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[device]) {
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaError_t e = cudaSuccess;
    if (prev != device) e = cudaSetDevice(device);
    void* p = nullptr;
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return shl::set_error(SHL_ECUDA, cudaGetErrorString(e));
    }
    g_scratch_ptr[device] = p;
  }
  *out = g_scratch_ptr[device];
  return SHL_OK;
}

}  // namespace

extern "C" shl_status shl_decompose_noalloc(const shl_bank* bank, const float* x, int batch,
                                            void* coeffs, shl_dtype dtype, int flags,
                                            void* stream) {
  int device = 0;
  size_t plane = 0;
  shl_status s = shl::bank_geometry(bank, &device, &plane);
  if (s != SHL_OK) return s;
  if (batch < 0) return shl::set_error(SHL_EINVAL, "batch must be >= 0");
  if (batch == 0) return SHL_OK;
  if (device < 0) return shl::set_error(SHL_EINVAL, "bank was created host-only (device < 0)");
  const size_t spectra = ((size_t)batch * plane + 255) & ~size_t(255);
  if (spectra + plane > kScratchBytes)
    return shl::set_error(SHL_EINVAL,
                          "batch too large for shl_decompose_noalloc: it needs (batch + 1) "
                          "half-spectrum planes within its fixed scratch; use shl_decompose");
  const int stage = (int)((kScratchBytes - spectra) / plane);
  void* ws = nullptr;
  s = scratch_address(device, &ws);
  if (s != SHL_OK) return s;
  return shl::decompose_staged(bank, x, batch, coeffs, dtype, flags, ws, kScratchBytes, stream,
                               stage);
}
