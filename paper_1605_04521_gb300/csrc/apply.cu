// ORAS preconditioner apply (Sec. 4):  z = sum_s R_s^T D_s A_s^{-1} R_s v
// with A_s^{-1} = U_s^{-1} L_s^{-1} P_s from the batched LU.  One cluster of two CTAs per
// subdomain (body in apply.cuh); the local vector lives in shared memory when it fits next to
// the tile ring, else in a global scratch slice.  With the Boolean partition of unity every
// global DOF is written by exactly one subdomain (no atomics); OAS (no D_s) accumulates with
// atomics.
#include "apply.cuh"

namespace oras {

template <typename R, typename ZT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(APPLY_THREADS)
    k_apply(ApplyGeom a, int k, int r, void* yglob, const cplx* __restrict__ v, ZT* __restrict__ z) {
  apply_cluster<R, ZT>(a, blockIdx.x / 2, v, k, z, k, r, (CT<R>*)yglob);
}

constexpr size_t SMEM_LIMIT = 227 * 1024 - 256;  // opt-in dynamic shared memory per block, with margin

// Ring depth and dynamic shared memory; y in shared memory when `allow_smem_y` and it fits.
template <typename R>
static void apply_config(const oras_handle* h, bool allow_smem_y, int* S, size_t* smem, bool* y_smem) {
  const int64_t ystrips = (h->mesh.max_np / TB + 1) / 2;
  if (allow_smem_y)
    for (int q = 8; q >= 2; --q)
      if (ApplySmem<R>::total(q, ystrips) <= SMEM_LIMIT) {
        *S = q;
        *smem = ApplySmem<R>::total(q, ystrips);
        *y_smem = true;
        return;
      }
  int q = 8;
  while (q > 2 && ApplySmem<R>::total(q, 0) > SMEM_LIMIT) --q;
  *S = q;
  *smem = ApplySmem<R>::total(q, 0);
  *y_smem = false;
}

ApplyGeom apply_geom(const oras_handle* h) {
  const auto& d = h->dev;
  ApplyGeom a;
  a.ns = d.sub_ns; a.np = d.sub_np; a.np_off = d.sub_np_off; a.ns_off = d.sub_ns_off;
  a.tile_off = d.sub_tile_off; a.inv_off = d.sub_inv_off;
  a.gidx = d.gidx; a.sub_dofs = d.sub_dofs; a.pou = d.sub_pou;
  a.arena = d.arena; a.dinv = d.dinv;
  a.weights = h->opt.weights;
  a.stages = 2;
  a.status = d.status;
  return a;
}

template <typename R, typename ZT>
static int apply_t(const oras_handle* h, const cplx* v, ZT* z, int k) {
  const auto& m = h->mesh;
  const auto& d = h->dev;
  ApplyGeom a = apply_geom(h);
  size_t smem;
  bool y_smem;
  apply_config<R>(h, true, &a.stages, &smem, &y_smem);
  cudaFuncSetAttribute(k_apply<R, ZT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (a.weights != ORAS_WEIGHTS_POU) cudaMemsetAsync(z, 0, sizeof(ZT) * m.ndof * k, d.stream);
  for (int r = 0; r < k; ++r)
    k_apply<R, ZT><<<2 * m.nsub, APPLY_THREADS, smem, d.stream>>>(a, k, r, y_smem ? nullptr : d.ybuf, v, z);
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
  int S;
  size_t smem;
  bool y_smem;
  if (h->dev.factor_bits == 64) apply_config<double>(h, true, &S, &smem, &y_smem);
  else apply_config<float>(h, true, &S, &smem, &y_smem);
  if (y_smem) return 0;
  size_t el = h->dev.factor_bits == 64 ? sizeof(CT<double>) : sizeof(CT<float>);
  int64_t total = 0;
  for (int s = 0; s < h->mesh.nsub; ++s) total += h->mesh.sub_np[s];
  return (size_t)total * el;
}

// Shared-memory configuration for the allocation-free variant (local vectors in global memory).
void apply_noalloc_config(const oras_handle* h, int* S, size_t* smem) {
  bool y_smem;
  if (h->dev.factor_bits == 64) apply_config<double>(h, false, S, smem, &y_smem);
  else apply_config<float>(h, false, S, smem, &y_smem);
}

}  // namespace oras
