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

// ------------------------------------------------------------------ PTX helpers (sm_90+)
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok) : "r"(smem_u32(b)), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_test_cluster(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok) : "r"(smem_u32(b)), "r"(parity) : "memory");
  return ok != 0;
}
// Default limit of a bounded device wait (oras_options.wait_ms = 0): 2 s of %globaltimer.
constexpr uint64_t WAIT_NS_DEFAULT = 2000000000ull;

// Waits for the phase with the given parity; gives up after limit_ns of %globaltimer (or 2^26
// polls) and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, bool cluster_scope = false,
                                          uint64_t limit_ns = WAIT_NS_DEFAULT) {
  if (cluster_scope ? mbar_test_cluster(b, parity) : mbar_test(b, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (long long it = 0; it < ORAS_SPIN_LIMIT; ++it) {
    if (cluster_scope ? mbar_test_cluster(b, parity) : mbar_test(b, parity)) return true;
    if ((it & 255) == 0 && globaltimer() - t0 > limit_ns) return false;
  }
  return false;
}
// A counter in shared memory written by one thread and polled by another of the same CTA.
__device__ __forceinline__ void st_release_cta(int* p, int v) {
  asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_cta(const int* p) {
  int v;
  asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}
// Bounded wait until *p >= need (limit_ns of %globaltimer), false on timeout.
__device__ __forceinline__ bool wait_counter(const int* p, int need, uint64_t limit_ns = WAIT_NS_DEFAULT) {
  if (ld_acquire_cta(p) >= need) return true;
  const uint64_t t0 = globaltimer();
  for (long long it = 0; it < ORAS_SPIN_LIMIT; ++it) {
    if (ld_acquire_cta(p) >= need) return true;
    if ((it & 255) == 0 && globaltimer() - t0 > limit_ns) return false;
  }
  return false;
}
// Limit of the waits for a CTA's own bulk copies still in flight before it exits: never below
// the default, so a short user limit cannot let a CTA leave while copies land in its memory.
__device__ __forceinline__ uint64_t drain_limit(uint64_t limit_ns) {
  return limit_ns > WAIT_NS_DEFAULT ? limit_ns : WAIT_NS_DEFAULT;
}
// st.shared::cluster of one 32-bit word into a partner CTA's shared memory.
__device__ __forceinline__ void st_remote_u32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
// Orders this thread's generic-proxy global writes before later async-proxy (bulk copy) reads.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
// 1-D bulk copy global -> shared, completion counted on an mbarrier of this CTA.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t map_to_rank(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_remote(uint32_t addr, float a, float b) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(a), "f"(b) : "memory");
}
__device__ __forceinline__ void st_remote(uint32_t addr, double a, double b) {
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(addr), "d"(a), "d"(b) : "memory");
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t addr) {
  asm volatile("fence.acq_rel.cluster;\n\tmbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(addr)
               : "memory");
}
__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}


}  // namespace oras
