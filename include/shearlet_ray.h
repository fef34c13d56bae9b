/*
 * shearlet_ray.h - C ABI of the parallel-beam ray transform of libshearlet
 * (the forward operator of the learned primal-dual reconstruction of
 * Sec. 4.4 of arXiv 2006.04591: R f(s, phi) = integral of f along the line
 * x cos(phi) + y sin(phi) = s).
 *
 * Geometry: an image f[i][j] (row i = y, column j = x) of n x n float32
 * pixels covers the square [-1, 1]^2 (pixel side h = 2/n, centre of pixel
 * (i, j) at (-1 + (j + 1/2) h, -1 + (i + 1/2) h)).  Angles phi_a = pi a / A,
 * a = 0..A-1; detector bins s_d = -sqrt(2) + (d + 1/2) 2 sqrt(2) / D,
 * d = 0..D-1.  Sinograms are float32 p[a][d].
 *
 * Discretisation: Joseph's method.  At angles with |cos phi| >= |sin phi|
 * the ray is sampled once per pixel row (once per column otherwise), the
 * image is interpolated linearly between the two pixels of that row
 * (column) that bracket the ray, zero outside, and the samples are summed
 * with the path length h / |cos phi| (h / |sin phi|).  shl_ray_adjoint
 * applies the transpose of exactly these weights (the same float32
 * arithmetic per weight), so <R x, y> = <x, R^T y> up to the rounding of the
 * sums.
 *
 * Conventions as in shearlet.h: shl_status return values, thread-local
 * shl_last_error_detail(), every launch on `stream` (a cudaStream_t as
 * void*), no synchronisation.  Images and sinograms are device (or managed)
 * float32 arrays on the operator's device, 4-byte aligned, caller-owned and
 * not aliased; the calls allocate nothing.
 */
#ifndef SHEARLET_RAY_H
#define SHEARLET_RAY_H

#include "shearlet.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct shl_ray shl_ray;

/*
 * shl_ray_create - the operator for n x n images, n_angles angles and n_det
 * detector bins on `device`: per-angle parameters of the sampling computed
 * in float64 and uploaded.  2 <= n <= 4096, 1 <= n_angles <= 4096,
 * 1 <= n_det <= 16384, else SHL_EINVAL; SHL_ENOMEM, SHL_ECUDA.
 */
shl_status shl_ray_create(int n, int n_angles, int n_det, int device, shl_ray** out);
shl_status shl_ray_destroy(shl_ray* op);
shl_status shl_ray_query(const shl_ray* op, int* n, int* n_angles, int* n_det);

/*
 * shl_ray_forward - sino[b] = R img[b] for b < batch.
 *   img  device float32 [batch][n][n];  sino device float32 [batch][A][D].
 */
shl_status shl_ray_forward(const shl_ray* op, const float* img, int batch, float* sino,
                           void* stream);

/*
 * shl_ray_adjoint - img[b] = R^T sino[b] (back-projection with the
 * transposed weights of shl_ray_forward).
 */
shl_status shl_ray_adjoint(const shl_ray* op, const float* sino, int batch, float* img,
                           void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SHEARLET_RAY_H */
