// Allocation-free variant of the preconditioner apply (z = M^{-1} v), for callers that must not
// allocate device memory.  It runs the same per-subdomain body as the regular apply (apply.cuh),
// but keeps every subdomain's local vector in a fixed, file-scope device array instead of shared
// memory or a library-allocated buffer, and reads v and writes z in the caller's N x k
// column-major layout directly, so no staging buffer is needed either.
#include <mutex>
#include <string>

#include "apply.cuh"

namespace oras {

// Fixed scratch: one local vector per subdomain (sum of padded orders x one complex entry in the
// factor precision).  Every GPU that loads this library holds it until the process exits.
constexpr size_t NOALLOC_SCRATCH_BYTES = 16u << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

template <typename R>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(APPLY_THREADS)
    k_apply_noalloc(ApplyGeom a, int64_t n, int k, void* scratch, const cplx* __restrict__ v,
                    cplx* __restrict__ z) {
  // columns one after the other: the scratch slices are reused.  After a bounded wait gave up
  // (in either CTA: apply_cluster returns the same value in both), the cluster stops, so no
  // barrier of the ring is initialised again while a copy might still complete on it.
  for (int r = 0; r < k; ++r)
    if (apply_cluster<R, cplx, 1, 2>(a, blockIdx.x / 2, v, 1, z, 1, (int64_t)r * n, 1, (CT<R>*)scratch)) break;
}

ApplyGeom apply_geom(const oras_handle* h);
void apply_noalloc_config(const oras_handle* h, int* S, size_t* smem);

}  // namespace oras

using namespace oras;

extern "C" int oras_precond_noalloc(oras_handle* h, const oras_complex* v, oras_complex* z, int32_t k) {
  if (!h) return ORAS_ERR_INVALID_ARG;
  if (!v || !z || k < 1 || k > MAX_RHS) { h->err = "oras_precond_noalloc: bad k or NULL vector"; return ORAS_ERR_INVALID_ARG; }
  const auto& m = h->mesh;
  const auto& d = h->dev;
  // the size check needs only the host set-up (subdomain orders, factor precision)
  const size_t el = h->opt.factor_bits == 64 ? sizeof(CT<double>) : sizeof(CT<float>);
  int64_t total_np = 0;
  for (int s = 0; s < m.nsub; ++s) total_np += m.sub_np[s];
  const size_t need = (size_t)total_np * el;
  if (need > NOALLOC_SCRATCH_BYTES) {
    h->err = "oras_precond_noalloc: the local vectors need " + std::to_string(need) +
             " bytes of scratch, more than the fixed " + std::to_string(NOALLOC_SCRATCH_BYTES) + " bytes";
    return ORAS_ERR_INVALID_ARG;
  }
  if (!h->factored) { h->err = "oras_precond_noalloc: call oras_factor first"; return ORAS_ERR_STATE; }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    h->err = "oras_precond_noalloc: no usable current device";
    return ORAS_ERR_CUDA;
  }
  if (dev != d.device) {
    h->err = "oras_precond_noalloc: the current device is not the handle's device";
    return ORAS_ERR_INVALID_ARG;
  }
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      // First call on this device: resolve the device address of the fixed array.
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        h->err = std::string("oras_precond_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return ORAS_ERR_CUDA;
      }
      g_noalloc_ptr[dev] = p;
    }
    scratch = g_noalloc_ptr[dev];
  }
  ApplyGeom a = apply_geom(h);
  size_t smem = 0;
  apply_noalloc_config(h, &a.stages, &smem);
  if (a.weights != ORAS_WEIGHTS_POU) {
    e = cudaMemsetAsync(z, 0, sizeof(cplx) * (size_t)m.ndof * k, d.stream);
    if (e != cudaSuccess) { h->err = std::string("oras_precond_noalloc: ") + cudaGetErrorString(e); return ORAS_ERR_CUDA; }
  }
  if (d.factor_bits == 64) {
    allow_max_smem((const void*)k_apply_noalloc<double>);
    k_apply_noalloc<double><<<2 * m.nsub, APPLY_THREADS, smem, d.stream>>>(a, m.ndof, k, scratch, (const cplx*)v,
                                                                           (cplx*)z);
  } else {
    allow_max_smem((const void*)k_apply_noalloc<float>);
    k_apply_noalloc<float><<<2 * m.nsub, APPLY_THREADS, smem, d.stream>>>(a, m.ndof, k, scratch, (const cplx*)v,
                                                                         (cplx*)z);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) { h->err = std::string("oras_precond_noalloc: launch: ") + cudaGetErrorString(e); return ORAS_ERR_CUDA; }
  count_launches(1);
  return ORAS_OK;
}
