// Allocation-free variant of the preconditioner apply (z = M^{-1} v), for callers that must not
// allocate device memory.  It runs the same gather / forward / backward / scatter as the regular
// apply, but keeps every subdomain's local vector in a fixed, file-scope device array instead of
// shared memory or a library-allocated buffer, and reads v and writes z in the caller's N x k
// column-major layout directly, so no staging buffer is needed either.
#include <mutex>
#include <string>

#include "dev.cuh"

namespace oras {

// Fixed scratch: one local vector per subdomain (sum of padded orders x one complex entry in the
// factor precision).  Every GPU that loads this library holds it until the process exits.
constexpr size_t NOALLOC_SCRATCH_BYTES = 16u << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

struct NoAllocArgs {
  const int64_t* ns; const int64_t* np; const int64_t* np_off; const int64_t* ns_off;
  const int64_t* tile_off;
  const int32_t* gidx; const int32_t* sub_dofs; const uint8_t* pou;
  const void* arena;
  int weights;
  int64_t n;            // global DOFs (column length of v and z)
  int k;                // columns
  void* scratch;        // device address of g_noalloc_scratch on this device
};

template <typename R>
__global__ void __launch_bounds__(256) k_apply_noalloc(NoAllocArgs a, const cplx* __restrict__ v,
                                                       cplx* __restrict__ z) {
  __shared__ CT<R> red[4][TB];
  const int s = blockIdx.x;
  const int64_t ns = a.ns[s], np = a.np[s], nts = np / TB;
  CT<R>* y = (CT<R>*)a.scratch + a.np_off[s];
  const CT<R>* F = (const CT<R>*)a.arena + a.tile_off[s] * (int64_t)TB * TB;
  const int32_t* gi = a.gidx + a.np_off[s];
  const int32_t* Ns = a.sub_dofs + a.ns_off[s];
  const uint8_t* D = a.pou + a.ns_off[s];
  const int tid = threadIdx.x, cg = tid >> 6, i = tid & 63, lane = tid & 31, warp = tid >> 5;
  for (int r = 0; r < a.k; ++r) {
    const cplx* vr = v + (int64_t)r * a.n;
    // gather: every entry of this subdomain's slice is written before it is read
    for (int64_t q = tid; q < np; q += blockDim.x) {
      int32_t g = gi[q];
      cplx val = g >= 0 ? vr[g] : cplx{0.0, 0.0};
      y[q] = {R(val.re), R(val.im)};
    }
    __syncthreads();
    for (int64_t I = 0; I < nts; ++I) {  // forward, unit lower
      CT<R> acc = {R(0), R(0)};
      for (int64_t J = 0; J < I; ++J) {
        const CT<R>* T = F + (I * nts + J) * (int64_t)TB * TB;
        const CT<R>* yJ = y + J * TB;
#pragma unroll 4
        for (int jj = 0; jj < TB; jj += 4) {
          CT<R> l = T[(jj + cg) * TB + i], yy = yJ[jj + cg];
          acc.re += l.re * yy.re - l.im * yy.im;
          acc.im += l.re * yy.im + l.im * yy.re;
        }
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
    for (int64_t I = nts - 1; I >= 0; --I) {  // backward, upper
      CT<R> acc = {R(0), R(0)};
      for (int64_t J = I + 1; J < nts; ++J) {
        const CT<R>* T = F + (I * nts + J) * (int64_t)TB * TB;
        const CT<R>* yJ = y + J * TB;
#pragma unroll 4
        for (int jj = 0; jj < TB; jj += 4) {
          CT<R> u = T[(jj + cg) * TB + i], yy = yJ[jj + cg];
          acc.re += u.re * yy.re - u.im * yy.im;
          acc.im += u.re * yy.im + u.im * yy.re;
        }
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
    cplx* zr = z + (int64_t)r * a.n;
    for (int64_t q = tid; q < ns; q += blockDim.x) {
      CT<R> val = y[q];
      if (a.weights == ORAS_WEIGHTS_POU) {
        if (D[q]) zr[Ns[q]] = {(double)val.re, (double)val.im};
      } else {
        atomicAdd(&zr[Ns[q]].re, (double)val.re);
        atomicAdd(&zr[Ns[q]].im, (double)val.im);
      }
    }
    __syncthreads();  // the slice is reused by the next column
  }
}

}  // namespace oras

using namespace oras;

extern "C" int oras_precond_noalloc(oras_handle* h, const oras_complex* v, oras_complex* z, int32_t k) {
  if (!h) return ORAS_ERR_INVALID_ARG;
  if (!h->factored) { h->err = "oras_precond_noalloc: call oras_factor first"; return ORAS_ERR_STATE; }
  if (!v || !z || k < 1 || k > MAX_RHS) { h->err = "oras_precond_noalloc: bad k or NULL vector"; return ORAS_ERR_INVALID_ARG; }
  const auto& m = h->mesh;
  const auto& d = h->dev;
  const size_t el = d.factor_bits == 64 ? sizeof(CT<double>) : sizeof(CT<float>);
  int64_t total_np = 0;
  for (int s = 0; s < m.nsub; ++s) total_np += m.sub_np[s];
  const size_t need = (size_t)total_np * el;
  if (need > NOALLOC_SCRATCH_BYTES) {
    h->err = "oras_precond_noalloc: the local vectors need " + std::to_string(need) +
             " bytes of scratch, more than the fixed " + std::to_string(NOALLOC_SCRATCH_BYTES) + " bytes";
    return ORAS_ERR_INVALID_ARG;
  }
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
  NoAllocArgs a;
  a.ns = d.sub_ns; a.np = d.sub_np; a.np_off = d.sub_np_off; a.ns_off = d.sub_ns_off;
  a.tile_off = d.sub_tile_off;
  a.gidx = d.gidx; a.sub_dofs = d.sub_dofs; a.pou = d.sub_pou;
  a.arena = d.arena;
  a.weights = h->opt.weights;
  a.n = m.ndof;
  a.k = k;
  a.scratch = scratch;
  if (a.weights != ORAS_WEIGHTS_POU) {
    e = cudaMemsetAsync(z, 0, sizeof(cplx) * (size_t)m.ndof * k, d.stream);
    if (e != cudaSuccess) { h->err = std::string("oras_precond_noalloc: ") + cudaGetErrorString(e); return ORAS_ERR_CUDA; }
  }
  if (d.factor_bits == 64)
    k_apply_noalloc<double><<<m.nsub, 256, 0, d.stream>>>(a, (const cplx*)v, (cplx*)z);
  else
    k_apply_noalloc<float><<<m.nsub, 256, 0, d.stream>>>(a, (const cplx*)v, (cplx*)z);
  e = cudaGetLastError();
  if (e != cudaSuccess) { h->err = std::string("oras_precond_noalloc: launch: ") + cudaGetErrorString(e); return ORAS_ERR_CUDA; }
  count_launches(1);
  return ORAS_OK;
}
