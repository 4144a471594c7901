// ORAS preconditioner apply (Sec. 4):  z = sum_s R_s^T D_s A_s^{-1} R_s v
// with A_s^{-1} = U_s^{-1} L_s^{-1} P_s from the batched LU.  One thread block per subdomain
// (body in apply.cuh); the local vector lives in shared memory when it fits, else in a global
// scratch slice.  With the Boolean partition of unity every global DOF is written by exactly
// one subdomain (no atomics); OAS (no D_s) accumulates with atomics.
#include "apply.cuh"

namespace oras {

template <typename R, typename ZT>
__global__ void __launch_bounds__(256) k_apply(ApplyGeom a, int k, int r, void* yglob, int y_in_smem,
                                               const cplx* __restrict__ v, ZT* __restrict__ z) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ CT<R> red[8][TB];
  CT<R>* dg = (CT<R>*)smem_raw;                  // [TB][DPS]
  CT<R>* y = y_in_smem ? dg + TB * DPS : (CT<R>*)yglob + a.np_off[blockIdx.x];
  apply_subdomain<R, ZT>(a, blockIdx.x, v, k, z, k, r, y, dg, red);
}

static ApplyGeom geom(const oras_handle* h) {
  const auto& d = h->dev;
  ApplyGeom a;
  a.ns = d.sub_ns; a.np = d.sub_np; a.np_off = d.sub_np_off; a.ns_off = d.sub_ns_off;
  a.tile_off = d.sub_tile_off;
  a.gidx = d.gidx; a.sub_dofs = d.sub_dofs; a.pou = d.sub_pou;
  a.arena = d.arena;
  a.weights = h->opt.weights;
  return a;
}

template <typename R>
static bool y_fits(const oras_handle* h, size_t* smem) {
  size_t dgb = (size_t)TB * DPS * sizeof(CT<R>);
  size_t yb = (size_t)h->mesh.max_np * sizeof(CT<R>);
  bool fit = dgb + yb <= 200 * 1024;
  *smem = fit ? dgb + yb : dgb;
  return fit;
}

template <typename R, typename ZT>
static int apply_t(const oras_handle* h, const cplx* v, ZT* z, int k) {
  const auto& m = h->mesh;
  const auto& d = h->dev;
  ApplyGeom a = geom(h);
  size_t smem;
  int in_smem = y_fits<R>(h, &smem) ? 1 : 0;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_apply<R, ZT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (a.weights != ORAS_WEIGHTS_POU) cudaMemsetAsync(z, 0, sizeof(ZT) * m.ndof * k, d.stream);
  for (int r = 0; r < k; ++r)
    k_apply<R, ZT><<<m.nsub, 256, smem, d.stream>>>(a, k, r, d.ybuf, in_smem, v, z);
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
  size_t smem;
  bool fit = h->dev.factor_bits == 64 ? y_fits<double>(h, &smem) : y_fits<float>(h, &smem);
  if (fit) return 0;
  size_t el = h->dev.factor_bits == 64 ? sizeof(CT<double>) : sizeof(CT<float>);
  int64_t total = 0;
  for (int s = 0; s < h->mesh.nsub; ++s) total += h->mesh.sub_np[s];
  return (size_t)total * el;
}

}  // namespace oras
