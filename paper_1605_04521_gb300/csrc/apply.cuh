// Device body of the ORAS preconditioner apply for one subdomain (Sec. 4):
//   y = P_s R_s v ;  y = L_s^{-1} y ;  y = U_s^{-1} y ;  z += R_s^T D_s y
// over the tiled factor arena (split re/im planes; tiles on/below the block diagonal row-major,
// above it column-major).  Used by the regular apply and by the allocation-free variant, which
// differ only in where the local vector y lives and in the layout of v and z.
#pragma once

#include "dev.cuh"

namespace oras {

struct ApplyGeom {
  const int64_t* ns; const int64_t* np; const int64_t* np_off; const int64_t* ns_off;
  const int64_t* tile_off;
  const int32_t* gidx; const int32_t* sub_dofs; const uint8_t* pou;
  const void* arena;
  int weights;
};

constexpr int DPS = TB + 1;  // padded column stride of the staged diagonal tile

__device__ __forceinline__ void z_store(cplx* z, double re, double im) { *z = {re, im}; }
__device__ __forceinline__ void z_store(CT<float>* z, double re, double im) { *z = {(float)re, (float)im}; }
__device__ __forceinline__ void z_add(cplx* z, double re, double im) {
  atomicAdd(&z->re, re);
  atomicAdd(&z->im, im);
}
__device__ __forceinline__ void z_add(CT<float>* z, double re, double im) {
  atomicAdd(&z->re, (float)re);
  atomicAdd(&z->im, (float)im);
}

// y: the subdomain's local vector (shared or global memory), dg: shared [TB][DPS] staging,
// red: shared [8][TB] partial sums.  v(g) = v[g*vs + off], z(g) = z[g*zs + off].
template <typename R, typename ZT>
__device__ void apply_subdomain(const ApplyGeom& a, int s, const cplx* __restrict__ v, int64_t vs,
                                ZT* __restrict__ z, int64_t zs, int64_t off, CT<R>* y, CT<R>* dg,
                                CT<R> (*red)[TB]) {
  const int64_t ns = a.ns[s], np = a.np[s], nts = np / TB;
  const R* F = (const R*)a.arena + a.tile_off[s] * 2 * TILE_PLANE;
  const int32_t* gi = a.gidx + a.np_off[s];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int64_t q = tid; q < np; q += blockDim.x) {
    int32_t g = gi[q];
    cplx val = g >= 0 ? v[(int64_t)g * vs + off] : cplx{0.0, 0.0};
    y[q] = {R(val.re), R(val.im)};
  }
  __syncthreads();
  // ---------------- forward: L y = P R v (unit lower).  Warp w owns rows 8w..8w+7 of the strip,
  // lane l columns 2l, 2l+1 of every row-major tile: coalesced rows, lane-parallel dot products.
  for (int64_t I = 0; I < nts; ++I) {
    CT<R> acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = {R(0), R(0)};
    for (int64_t J = 0; J < I; ++J) {
      const R* T = F + (I * nts + J) * 2 * TILE_PLANE;
      const CT<R> y0 = y[J * TB + 2 * lane], y1 = y[J * TB + 2 * lane + 1];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int64_t e = (int64_t)(warp * 8 + q) * TB + 2 * lane;
        const R r0 = T[e], r1 = T[e + 1], i0 = T[TILE_PLANE + e], i1 = T[TILE_PLANE + e + 1];
        acc[q].re += r0 * y0.re - i0 * y0.im + r1 * y1.re - i1 * y1.im;
        acc[q].im += r0 * y0.im + i0 * y0.re + r1 * y1.im + i1 * y1.re;
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      for (int o = 16; o > 0; o >>= 1) {
        acc[q].re += __shfl_down_sync(0xffffffffu, acc[q].re, o);
        acc[q].im += __shfl_down_sync(0xffffffffu, acc[q].im, o);
      }
      if (lane == 0) red[0][warp * 8 + q] = acc[q];
    }
    {  // stage the diagonal tile (row-major planes) column-major in shared memory
      const R* T = F + (I * nts + I) * 2 * TILE_PLANE;
      for (int e = tid; e < TB * TB; e += blockDim.x) dg[(e % TB) * DPS + e / TB] = {T[e], T[TILE_PLANE + e]};
    }
    __syncthreads();
    if (warp == 0) {
      CT<R> u0 = y[I * TB + lane], u1 = y[I * TB + lane + 32];
      u0.re -= red[0][lane].re; u0.im -= red[0][lane].im;
      u1.re -= red[0][lane + 32].re; u1.im -= red[0][lane + 32].im;
      for (int j = 0; j < TB; ++j) {
        CT<R> src = j < 32 ? u0 : u1;
        CT<R> yj = {__shfl_sync(0xffffffffu, src.re, j & 31), __shfl_sync(0xffffffffu, src.im, j & 31)};
        if (lane > j) { CT<R> l = dg[j * DPS + lane]; u0.re -= l.re * yj.re - l.im * yj.im; u0.im -= l.re * yj.im + l.im * yj.re; }
        if (lane + 32 > j) { CT<R> l = dg[j * DPS + lane + 32]; u1.re -= l.re * yj.re - l.im * yj.im; u1.im -= l.re * yj.im + l.im * yj.re; }
      }
      y[I * TB + lane] = u0;
      y[I * TB + lane + 32] = u1;
    }
    __syncthreads();
  }
  // ---------------- backward: U y = y.  Warp w owns columns 8w..8w+7 of every column-major
  // tile of the strip, lane l rows 2l, 2l+1; partial sums are combined across warps.
  for (int64_t I = nts - 1; I >= 0; --I) {
    CT<R> a0 = {R(0), R(0)}, a1 = {R(0), R(0)};
    for (int64_t J = I + 1; J < nts; ++J) {
      const R* T = F + (I * nts + J) * 2 * TILE_PLANE;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int c = warp * 8 + q;
        const CT<R> yc = y[J * TB + c];
        const int64_t e = (int64_t)c * TB + 2 * lane;
        const R r0 = T[e], r1 = T[e + 1], i0 = T[TILE_PLANE + e], i1 = T[TILE_PLANE + e + 1];
        a0.re += r0 * yc.re - i0 * yc.im;
        a0.im += r0 * yc.im + i0 * yc.re;
        a1.re += r1 * yc.re - i1 * yc.im;
        a1.im += r1 * yc.im + i1 * yc.re;
      }
    }
    red[warp][2 * lane] = a0;
    red[warp][2 * lane + 1] = a1;
    {
      const R* T = F + (I * nts + I) * 2 * TILE_PLANE;
      for (int e = tid; e < TB * TB; e += blockDim.x) dg[(e % TB) * DPS + e / TB] = {T[e], T[TILE_PLANE + e]};
    }
    __syncthreads();
    if (warp == 0) {
      CT<R> u0 = y[I * TB + lane], u1 = y[I * TB + lane + 32];
      for (int w = 0; w < 8; ++w) {
        u0.re -= red[w][lane].re; u0.im -= red[w][lane].im;
        u1.re -= red[w][lane + 32].re; u1.im -= red[w][lane + 32].im;
      }
      for (int j = TB - 1; j >= 0; --j) {
        // y_j = acc_j / U_jj, then remove its column from the rows above
        CT<R> src = j < 32 ? u0 : u1;
        CT<R> aj = {__shfl_sync(0xffffffffu, src.re, j & 31), __shfl_sync(0xffffffffu, src.im, j & 31)};
        CT<R> d = dg[j * DPS + j];
        R dd = d.re * d.re + d.im * d.im;
        CT<R> yj = {(aj.re * d.re + aj.im * d.im) / dd, (aj.im * d.re - aj.re * d.im) / dd};
        if (lane == (j & 31)) { if (j < 32) u0 = yj; else u1 = yj; }
        if (lane < j) { CT<R> u = dg[j * DPS + lane]; u0.re -= u.re * yj.re - u.im * yj.im; u0.im -= u.re * yj.im + u.im * yj.re; }
        if (lane + 32 < j) { CT<R> u = dg[j * DPS + lane + 32]; u1.re -= u.re * yj.re - u.im * yj.im; u1.im -= u.re * yj.im + u.im * yj.re; }
      }
      y[I * TB + lane] = u0;
      y[I * TB + lane + 32] = u1;
    }
    __syncthreads();
  }
  // ---------------- scatter with the partition of unity
  const int32_t* Ns = a.sub_dofs + a.ns_off[s];
  const uint8_t* D = a.pou + a.ns_off[s];
  for (int64_t q = tid; q < ns; q += blockDim.x) {
    CT<R> val = y[q];
    ZT* dst = z + (int64_t)Ns[q] * zs + off;
    if (a.weights == ORAS_WEIGHTS_POU) {
      if (D[q]) z_store(dst, (double)val.re, (double)val.im);
    } else {
      z_add(dst, (double)val.re, (double)val.im);
    }
  }
  __syncthreads();
}

}  // namespace oras
