// ray.cu - parallel-beam ray transform (the forward operator of the
// learned primal-dual reconstruction of Sec. 4.4) and its exact transpose.
//
//   k_ray_forward  one thread per ray (image, angle, bin): Joseph's method,
//                  one linear-interpolation sample per pixel row (or column).
//   k_ray_adjoint  one thread per pixel: for each angle, the 2-3 bins whose
//                  rays sample this pixel's row (column) near it, with the
//                  forward's own weights.
//
// Sampling of angle a: the ray of bin d meets row (column) t of the image at
// the fractional pixel coordinate u = A_a d + B_a t + C_a along that row
// (column); the image is interpolated between pixels floor(u) and
// floor(u) + 1 with weights 1 - frac(u) and frac(u), and the samples are
// summed with weight w_a = h / |cos phi| (h / |sin phi|).  Both kernels
// evaluate u with the same float32 expression, so the adjoint applies
// exactly the forward's weights.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/shearlet_ray.h"
#include "internal.h"

namespace {

struct AngleParam {
  float A, B, C, w;   // u = A d + B t + C; sample weight w
  int by_rows;        // 1: sample t is a pixel row (|cos phi| >= |sin phi|)
  int pad[3];
};

__device__ __forceinline__ float sample_u(const AngleParam& q, int d, int t) {
  return fmaf(q.A, (float)d, fmaf(q.B, (float)t, q.C));
}

__global__ void __launch_bounds__(256) k_ray_forward(const float* __restrict__ img,
                                                     float* __restrict__ sino,
                                                     const AngleParam* __restrict__ prm, int n,
                                                     int A, int D) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y;
  if (d >= D) return;
  const AngleParam q = prm[a];
  const float* f = img + (size_t)blockIdx.z * n * n;
  float acc = 0.f;
  for (int t = 0; t < n; ++t) {
    const float u = sample_u(q, d, t);
    const float fk = floorf(u);
    if (fk < -1.f || fk > (float)(n - 1)) continue;   // both neighbours outside
    const int k0 = (int)fk;
    const float w1 = u - fk, w0 = 1.f - w1;
    float v0 = 0.f, v1 = 0.f;
    if (q.by_rows) {
      if (k0 >= 0) v0 = __ldg(f + (size_t)t * n + k0);
      if (k0 + 1 < n) v1 = __ldg(f + (size_t)t * n + k0 + 1);
    } else {
      if (k0 >= 0) v0 = __ldg(f + (size_t)k0 * n + t);
      if (k0 + 1 < n) v1 = __ldg(f + (size_t)(k0 + 1) * n + t);
    }
    acc = fmaf(w0, v0, fmaf(w1, v1, acc));
  }
  sino[((size_t)blockIdx.z * A + a) * D + d] = acc * q.w;
}

__global__ void __launch_bounds__(256) k_ray_adjoint(const float* __restrict__ sino,
                                                     float* __restrict__ img,
                                                     const AngleParam* __restrict__ prm, int n,
                                                     int A, int D) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= n) return;
  const float* p = sino + (size_t)blockIdx.z * A * D;
  float acc = 0.f;
  for (int a = 0; a < A; ++a) {
    const AngleParam q = prm[a];
    const int t = q.by_rows ? i : j, k = q.by_rows ? j : i;
    // bins whose u at sample t lies in (k - 1, k + 1): d near (k - B t - C) / A
    const float dc = ((float)k - fmaf(q.B, (float)t, q.C)) / q.A;
    const float half = 1.f / fabsf(q.A);
    const int lo = max(0, (int)floorf(dc - half) - 1);
    const int hi = min(D - 1, (int)ceilf(dc + half) + 1);
    float sa = 0.f;
    for (int d = lo; d <= hi; ++d) {
      const float u = sample_u(q, d, t);
      const float fk = floorf(u);
      const float w1 = u - fk;
      const int k0 = (int)fk;
      if (k0 == k) sa = fmaf(1.f - w1, __ldg(p + (size_t)a * D + d), sa);
      else if (k0 + 1 == k) sa = fmaf(w1, __ldg(p + (size_t)a * D + d), sa);
    }
    acc = fmaf(sa, q.w, acc);
  }
  img[((size_t)blockIdx.z * n + i) * n + j] = acc;
}

bool aligned4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

}  // namespace

struct shl_ray {
  int device = 0, n = 0, A = 0, D = 0;
  AngleParam* dPrm = nullptr;
};

extern "C" {

shl_status shl_ray_create(int n, int n_angles, int n_det, int device, shl_ray** out) {
  if (!out) return shl::set_error(SHL_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 2 || n > 4096 || n_angles < 1 || n_angles > 4096 || n_det < 1 || n_det > 16384)
    return shl::set_error(SHL_EINVAL, "need 2 <= n <= 4096, 1 <= n_angles <= 4096, 1 <= n_det <= 16384");
  if (device < 0) return shl::set_error(SHL_EINVAL, "device must be >= 0");
  const double PI = 3.14159265358979323846264338327950288, S = std::sqrt(2.0);
  const double h = 2.0 / n, ds = 2.0 * S / n_det;
  std::vector<AngleParam> prm(n_angles);
  for (int a = 0; a < n_angles; ++a) {
    const double phi = PI * a / n_angles, c = std::cos(phi), s = std::sin(phi);
    AngleParam& q = prm[a];
    q = AngleParam{};
    q.by_rows = std::fabs(c) >= std::fabs(s);
    // row mode:    u = (s_d - y_t sin) / (h cos) + 1/h - 1/2
    // column mode: u = (s_d - x_t cos) / (h sin) + 1/h - 1/2
    // with s_d = -S + (d + 1/2) ds and x_t = y_t = -1 + (t + 1/2) h
    const double den = q.by_rows ? h * c : h * s, other = q.by_rows ? s : c;
    q.A = (float)(ds / den);
    q.B = (float)(-h * other / den);
    q.C = (float)((-S + 0.5 * ds + other * (1.0 - 0.5 * h)) / den + 1.0 / h - 0.5);
    q.w = (float)(h / std::fabs(q.by_rows ? c : s));
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);
  shl_ray* op = new shl_ray;
  op->device = device; op->n = n; op->A = n_angles; op->D = n_det;
  cudaError_t e = cudaMalloc(&op->dPrm, sizeof(AngleParam) * n_angles);
  if (!e) e = cudaMemcpy(op->dPrm, prm.data(), sizeof(AngleParam) * n_angles, cudaMemcpyHostToDevice);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  if (e) {
    if (op->dPrm) cudaFree(op->dPrm);
    delete op;
    cudaGetLastError();
    return shl::set_error(e == cudaErrorMemoryAllocation ? SHL_ENOMEM : SHL_ECUDA,
                          cudaGetErrorString(e));
  }
  *out = op;
  return SHL_OK;
}

shl_status shl_ray_destroy(shl_ray* op) {
  if (!op) return SHL_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != op->device) cudaSetDevice(op->device);
  cudaFree(op->dPrm);
  if (prev >= 0 && prev != op->device) cudaSetDevice(prev);
  delete op;
  return SHL_OK;
}

shl_status shl_ray_query(const shl_ray* op, int* n, int* n_angles, int* n_det) {
  if (!op) return shl::set_error(SHL_EINVAL, "operator is NULL");
  if (n) *n = op->n;
  if (n_angles) *n_angles = op->A;
  if (n_det) *n_det = op->D;
  return SHL_OK;
}

shl_status shl_ray_forward(const shl_ray* op, const float* img, int batch, float* sino,
                           void* stream) {
  if (!op) return shl::set_error(SHL_EINVAL, "operator is NULL");
  if (batch < 0) return shl::set_error(SHL_EINVAL, "batch must be >= 0");
  if (batch == 0) return SHL_OK;
  if (!img || !sino || !aligned4(img) || !aligned4(sino))
    return shl::set_error(SHL_EINVAL, "img and sino must be 4-byte aligned device pointers");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != op->device) cudaSetDevice(op->device);
  cudaError_t e = cudaSuccess;
  for (int b0 = 0; b0 < batch && !e; b0 += 65535) {
    const int nb = std::min(65535, batch - b0);
    k_ray_forward<<<dim3((op->D + 255) / 256, op->A, nb), 256, 0,
                    static_cast<cudaStream_t>(stream)>>>(img + (size_t)b0 * op->n * op->n,
                                                         sino + (size_t)b0 * op->A * op->D,
                                                         op->dPrm, op->n, op->A, op->D);
    e = cudaGetLastError();
  }
  if (prev >= 0 && prev != op->device) cudaSetDevice(prev);
  return e ? shl::set_error(SHL_ECUDA, cudaGetErrorString(e)) : SHL_OK;
}

shl_status shl_ray_adjoint(const shl_ray* op, const float* sino, int batch, float* img,
                           void* stream) {
  if (!op) return shl::set_error(SHL_EINVAL, "operator is NULL");
  if (batch < 0) return shl::set_error(SHL_EINVAL, "batch must be >= 0");
  if (batch == 0) return SHL_OK;
  if (!img || !sino || !aligned4(img) || !aligned4(sino))
    return shl::set_error(SHL_EINVAL, "img and sino must be 4-byte aligned device pointers");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != op->device) cudaSetDevice(op->device);
  cudaError_t e = cudaSuccess;
  for (int b0 = 0; b0 < batch && !e; b0 += 65535) {
    const int nb = std::min(65535, batch - b0);
    k_ray_adjoint<<<dim3((op->n + 255) / 256, op->n, nb), 256, 0,
                    static_cast<cudaStream_t>(stream)>>>(sino + (size_t)b0 * op->A * op->D,
                                                         img + (size_t)b0 * op->n * op->n,
                                                         op->dPrm, op->n, op->A, op->D);
    e = cudaGetLastError();
  }
  if (prev >= 0 && prev != op->device) cudaSetDevice(prev);
  return e ? shl::set_error(SHL_ECUDA, cudaGetErrorString(e)) : SHL_OK;
}

}  // extern "C"
