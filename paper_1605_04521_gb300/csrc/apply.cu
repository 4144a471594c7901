// ORAS preconditioner apply (Sec. 4):  z = sum_s R_s^T D_s A_s^{-1} R_s v
// with A_s^{-1} = U_s^{-1} L_s^{-1} P_s from the batched LU.  One thread block per subdomain:
//   gather   y = P_s R_s v          (gidx = N_s[perm], FP64 -> factor precision)
//   forward  y = L_s^{-1} y         (row strips of TB x TB tiles, unit lower)
//   backward y = U_s^{-1} y
//   scatter  z[N_s[i]] = y[i] where D_s(i) = 1 (Boolean partition of unity: every global DOF
//            is written by exactly one subdomain, no atomics), or += y[i] for OAS (no D_s).
// The local vector y lives in shared memory when it fits, else in a global scratch slice.
#include "dev.cuh"

namespace oras {

struct ApplyArgs {
  int nsub;
  const int64_t* ns; const int64_t* np; const int64_t* np_off; const int64_t* ns_off;
  const int64_t* tile_off;
  const int32_t* gidx; const int32_t* sub_dofs; const uint8_t* pou;
  const void* arena;
  int weights;          // ORAS_WEIGHTS_POU or ORAS_WEIGHTS_NONE
  int k, r;             // number of RHS in v/z ([N][k] layout) and the column processed
  void* yglob;          // fallback storage [sum np]
  int y_in_smem;
};

template <typename R> __device__ __forceinline__ CT<R> fma_c(CT<R> acc, CT<R> a, CT<R> b) {
  acc.re += a.re * b.re - a.im * b.im;
  acc.im += a.re * b.im + a.im * b.re;
  return acc;
}

template <typename ZT> __device__ __forceinline__ void store_z(ZT* z, int64_t idx, double re, double im);
template <> __device__ __forceinline__ void store_z<cplx>(cplx* z, int64_t idx, double re, double im) {
  z[idx] = {re, im};
}
template <> __device__ __forceinline__ void store_z<CT<float>>(CT<float>* z, int64_t idx, double re, double im) {
  z[idx] = {(float)re, (float)im};
}
template <typename ZT> __device__ __forceinline__ void add_z(ZT* z, int64_t idx, double re, double im);
template <> __device__ __forceinline__ void add_z<cplx>(cplx* z, int64_t idx, double re, double im) {
  atomicAdd(&z[idx].re, re);
  atomicAdd(&z[idx].im, im);
}
template <> __device__ __forceinline__ void add_z<CT<float>>(CT<float>* z, int64_t idx, double re, double im) {
  atomicAdd(&z[idx].re, (float)re);
  atomicAdd(&z[idx].im, (float)im);
}

template <typename R, typename ZT>
__global__ void __launch_bounds__(256) k_apply(ApplyArgs a, const cplx* __restrict__ v, ZT* __restrict__ z) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ CT<R> red[4][TB];
  const int s = blockIdx.x;
  const int64_t ns = a.ns[s], np = a.np[s], nts = np / TB;
  CT<R>* y = a.y_in_smem ? (CT<R>*)smem_raw : (CT<R>*)a.yglob + a.np_off[s];
  const CT<R>* F = (const CT<R>*)a.arena + a.tile_off[s] * (int64_t)TB * TB;
  const int32_t* gi = a.gidx + a.np_off[s];
  const int tid = threadIdx.x, cg = tid >> 6, i = tid & 63, lane = tid & 31, warp = tid >> 5;
  const int K = a.k, r = a.r;
  for (int64_t q = tid; q < np; q += blockDim.x) {
    int32_t g = gi[q];
    cplx val = g >= 0 ? v[(int64_t)g * K + r] : cplx{0.0, 0.0};
    y[q] = {R(val.re), R(val.im)};
  }
  __syncthreads();
  // ---------------- forward: L y = P R v (unit lower)
  for (int64_t I = 0; I < nts; ++I) {
    CT<R> acc = {R(0), R(0)};
    for (int64_t J = 0; J < I; ++J) {
      const CT<R>* T = F + (I * nts + J) * (int64_t)TB * TB;
      const CT<R>* yJ = y + J * TB;
#pragma unroll
      for (int jj = 0; jj < TB; jj += 4) acc = fma_c(acc, T[(jj + cg) * TB + i], yJ[jj + cg]);
    }
    red[cg][i] = acc;
    __syncthreads();
    if (warp == 0) {
      const CT<R>* T = F + (I * nts + I) * (int64_t)TB * TB;
      CT<R> y0 = y[I * TB + lane], y1 = y[I * TB + lane + 32];
      for (int c = 0; c < 4; ++c) {
        y0.re -= red[c][lane].re; y0.im -= red[c][lane].im;
        y1.re -= red[c][lane + 32].re; y1.im -= red[c][lane + 32].im;
      }
      for (int j = 0; j < TB; ++j) {
        CT<R> src = j < 32 ? y0 : y1;
        CT<R> yj = {__shfl_sync(0xffffffffu, src.re, j & 31), __shfl_sync(0xffffffffu, src.im, j & 31)};
        if (lane > j) { CT<R> l = T[j * TB + lane]; y0.re -= l.re * yj.re - l.im * yj.im; y0.im -= l.re * yj.im + l.im * yj.re; }
        if (lane + 32 > j) { CT<R> l = T[j * TB + lane + 32]; y1.re -= l.re * yj.re - l.im * yj.im; y1.im -= l.re * yj.im + l.im * yj.re; }
      }
      y[I * TB + lane] = y0;
      y[I * TB + lane + 32] = y1;
    }
    __syncthreads();
  }
  // ---------------- backward: U y = y
  for (int64_t I = nts - 1; I >= 0; --I) {
    CT<R> acc = {R(0), R(0)};
    for (int64_t J = I + 1; J < nts; ++J) {
      const CT<R>* T = F + (I * nts + J) * (int64_t)TB * TB;
      const CT<R>* yJ = y + J * TB;
#pragma unroll
      for (int jj = 0; jj < TB; jj += 4) acc = fma_c(acc, T[(jj + cg) * TB + i], yJ[jj + cg]);
    }
    red[cg][i] = acc;
    __syncthreads();
    if (warp == 0) {
      const CT<R>* T = F + (I * nts + I) * (int64_t)TB * TB;
      CT<R> y0 = y[I * TB + lane], y1 = y[I * TB + lane + 32];
      for (int c = 0; c < 4; ++c) {
        y0.re -= red[c][lane].re; y0.im -= red[c][lane].im;
        y1.re -= red[c][lane + 32].re; y1.im -= red[c][lane + 32].im;
      }
      for (int j = TB - 1; j >= 0; --j) {
        // y_j = acc_j / U_jj, then remove its column from the rows above
        CT<R> src = j < 32 ? y0 : y1;
        CT<R> aj = {__shfl_sync(0xffffffffu, src.re, j & 31), __shfl_sync(0xffffffffu, src.im, j & 31)};
        CT<R> d = T[j * TB + j];
        R dd = d.re * d.re + d.im * d.im;
        CT<R> yj = {(aj.re * d.re + aj.im * d.im) / dd, (aj.im * d.re - aj.re * d.im) / dd};
        if (lane == (j & 31)) { if (j < 32) y0 = yj; else y1 = yj; }
        if (lane < j) { CT<R> u = T[j * TB + lane]; y0.re -= u.re * yj.re - u.im * yj.im; y0.im -= u.re * yj.im + u.im * yj.re; }
        if (lane + 32 < j) { CT<R> u = T[j * TB + lane + 32]; y1.re -= u.re * yj.re - u.im * yj.im; y1.im -= u.re * yj.im + u.im * yj.re; }
      }
      y[I * TB + lane] = y0;
      y[I * TB + lane + 32] = y1;
    }
    __syncthreads();
  }
  // ---------------- scatter with the partition of unity
  const int32_t* Ns = a.sub_dofs + a.ns_off[s];
  const uint8_t* D = a.pou + a.ns_off[s];
  for (int64_t q = tid; q < ns; q += blockDim.x) {
    CT<R> val = y[q];
    int64_t idx = (int64_t)Ns[q] * K + r;
    if (a.weights == ORAS_WEIGHTS_POU) {
      if (D[q]) store_z<ZT>(z, idx, (double)val.re, (double)val.im);
    } else {
      add_z<ZT>(z, idx, (double)val.re, (double)val.im);
    }
  }
}

template <typename R, typename ZT>
static int apply_t(const oras_handle* h, const cplx* v, ZT* z, int k) {
  const auto& m = h->mesh;
  const auto& d = h->dev;
  ApplyArgs a;
  a.nsub = m.nsub;
  a.ns = d.sub_ns; a.np = d.sub_np; a.np_off = d.sub_np_off; a.ns_off = d.sub_ns_off;
  a.tile_off = d.sub_tile_off;
  a.gidx = d.gidx; a.sub_dofs = d.sub_dofs; a.pou = d.sub_pou;
  a.arena = d.arena;
  a.weights = h->opt.weights;
  a.k = k;
  a.yglob = d.ybuf;
  size_t ybytes = (size_t)m.max_np * sizeof(CT<R>);
  a.y_in_smem = ybytes <= 200 * 1024;
  size_t smem = a.y_in_smem ? ybytes : 0;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_apply<R, ZT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (a.weights != ORAS_WEIGHTS_POU) cudaMemsetAsync(z, 0, sizeof(ZT) * m.ndof * k, d.stream);
  for (int r = 0; r < k; ++r) {
    a.r = r;
    k_apply<R, ZT><<<m.nsub, 256, smem, d.stream>>>(a, v, z);
  }
  count_launches(k);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// z (FP64 complex [N][k]) = M^{-1} v
int launch_apply_f64out(const oras_handle* h, const cplx* v, cplx* z, int k) {
  return h->dev.factor_bits == 64 ? apply_t<double, cplx>(h, v, z, k) : apply_t<float, cplx>(h, v, z, k);
}
// z (FP32 complex [N][k]) = M^{-1} v, FP32 factors only
int launch_apply_f32out(const oras_handle* h, const cplx* v, void* z, int k) {
  return apply_t<float, CT<float>>(h, v, (CT<float>*)z, k);
}

size_t apply_yglob_bytes(const oras_handle* h) {
  size_t el = h->dev.factor_bits == 64 ? sizeof(CT<double>) : sizeof(CT<float>);
  size_t ybytes = (size_t)h->mesh.max_np * el;
  if (ybytes <= 200 * 1024) return 0;
  int64_t total = 0;
  for (int s = 0; s < h->mesh.nsub; ++s) total += h->mesh.sub_np[s];
  return (size_t)total * el;
}

}  // namespace oras
