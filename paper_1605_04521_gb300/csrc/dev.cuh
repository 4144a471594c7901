// Device helpers shared by the library's CUDA translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace oras {

// complex helpers (interleaved re, im)
template <typename R> struct CT { R re, im; };

// Local-factor arena tiles: each TB x TB complex tile is two planes of TB*TB reals (real part,
// then imaginary part).  Tiles on or below the block diagonal (I >= J) store their planes
// row-major, tiles above it column-major, so that in the trailing update C_IJ -= L_Ik U_kJ both
// operands are contiguous along the contraction index k (K-major for the tensor cores), the
// forward substitution streams rows of L and the backward substitution streams columns of U.
__device__ __forceinline__ bool tile_rowmajor(int64_t I, int64_t J) { return I >= J; }
__device__ __forceinline__ int64_t tile_elem(bool rm, int64_t i, int64_t j) {
  return rm ? i * TB + j : j * TB + i;
}
constexpr int64_t TILE_PLANE = (int64_t)TB * TB;

__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cplx cscale(cplx a, double s) { return {a.re * s, a.im * s}; }
__device__ __forceinline__ cplx cconj(cplx a) { return {a.re, -a.im}; }

// Geometry of one tetrahedron from its sorted vertices: barycentric gradients gl[4][3], volume.
__device__ __forceinline__ void tet_geometry(const double* __restrict__ xyz, const int32_t* v,
                                             double gl[4][3], double& vol) {
  double p0[3], J[3][3];
  for (int d = 0; d < 3; ++d) p0[d] = xyz[(int64_t)v[0] * 3 + d];
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d) J[d][c] = xyz[(int64_t)v[c + 1] * 3 + d] - p0[d];
  // cofactor inverse: rows of J^{-1} are grad lambda_1..3
  double C00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  double C01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  double C02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  double det = J[0][0] * C00 + J[0][1] * C01 + J[0][2] * C02;
  double id = 1.0 / det;
  double inv[3][3];
  inv[0][0] = C00 * id;
  inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
  inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
  inv[1][0] = C01 * id;
  inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
  inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
  inv[2][0] = C02 * id;
  inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
  inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
  for (int d = 0; d < 3; ++d) {
    gl[1][d] = inv[0][d];
    gl[2][d] = inv[1][d];
    gl[3][d] = inv[2][d];
    gl[0][d] = -(inv[0][d] + inv[1][d] + inv[2][d]);
  }
  vol = fabs(det) / 6.0;
}

__device__ __forceinline__ int sym10(int p, int q) {
  if (p > q) { int t = p; p = q; q = t; }
  return p * 4 - p * (p - 1) / 2 + (q - p);
}

// bounded spin helper: returns false when the limit is reached
#define ORAS_SPIN_LIMIT (1ll << 26)


}  // namespace oras
