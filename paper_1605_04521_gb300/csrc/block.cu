// FP64 kernels of block flexible GMRES (Sec. 6: Block GMRES for the several right-hand sides of
// one system).  A block of p right-hand sides is an [N][p] array (the p entries of a row
// adjacent), the same layout as the pseudo-block vectors.  The p x p products of the block
// Arnoldi process -- Gram matrices V_i^H W and W^H W, and W -= V_i H or W C^{-1} -- are formed
// here in FP64; the small dense algebra (Cholesky of the Gram matrices, the block Hessenberg
// least-squares problem) runs on the host.  Reductions are fixed two-stage sums (block partials,
// then a fixed-order sum over blocks), so results do not depend on scheduling.
#include <algorithm>

#include "dev.cuh"

namespace oras {

template <typename XT> __device__ __forceinline__ cplx ld_block(const XT* p, int64_t i);
template <> __device__ __forceinline__ cplx ld_block<cplx>(const cplx* p, int64_t i) { return p[i]; }
template <> __device__ __forceinline__ cplx ld_block<CT<float>>(const CT<float>* p, int64_t i) {
  const CT<float> v = p[i];
  return {(double)v.re, (double)v.im};
}

constexpr int BLK_BLOCKS = 304;     // 2 x 152 SMs
constexpr int BLK_THREADS = 256;
constexpr int BLK_ROWS = 16;        // rows of both blocks staged in shared memory at a time

// partials[b][r][c] = sum over the rows of block b of conj(A[n][r]) B[n][c]  (p <= 64)
__global__ void __launch_bounds__(BLK_THREADS) k_block_gram(int64_t n, int p, const cplx* __restrict__ A,
                                                            const cplx* __restrict__ B, cplx* __restrict__ partials) {
  __shared__ cplx sa[BLK_ROWS][MAX_RHS], sb[BLK_ROWS][MAX_RHS];
  constexpr int PAIRS = MAX_RHS * MAX_RHS / BLK_THREADS;  // pairs per thread at p = 64
  cplx acc[PAIRS];
#pragma unroll
  for (int q = 0; q < PAIRS; ++q) acc[q] = {0.0, 0.0};
  const int pp = p * p;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per, r1 = r0 + per < n ? r0 + per : n;
  for (int64_t base = r0; base < r1; base += BLK_ROWS) {
    const int rows = (int)(r1 - base < BLK_ROWS ? r1 - base : BLK_ROWS);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * p; e += blockDim.x) {
      const int rr = e / p, cc = e % p;
      sa[rr][cc] = A[(base + rr) * p + cc];
      sb[rr][cc] = B[(base + rr) * p + cc];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PAIRS; ++q) {
      const int pr = threadIdx.x + q * BLK_THREADS;
      if (pr >= pp) break;
      const int r = pr / p, c = pr % p;
      cplx t = acc[q];
      for (int rr = 0; rr < rows; ++rr) {
        const cplx a = sa[rr][r], b = sb[rr][c];
        t.re += a.re * b.re + a.im * b.im;
        t.im += a.re * b.im - a.im * b.re;
      }
      acc[q] = t;
    }
  }
#pragma unroll
  for (int q = 0; q < PAIRS; ++q) {
    const int pr = threadIdx.x + q * BLK_THREADS;
    if (pr >= pp) break;
    partials[(int64_t)blockIdx.x * pp + pr] = acc[q];
  }
}

// out[r][c] = fixed-order sum over the blocks of partials[b][r][c]
__global__ void k_block_sum(int p, const cplx* __restrict__ partials, cplx* __restrict__ out) {
  const int pp = p * p;
  for (int pr = blockIdx.x * blockDim.x + threadIdx.x; pr < pp; pr += gridDim.x * blockDim.x) {
    cplx t = {0.0, 0.0};
#pragma unroll 16
    for (int b = 0; b < BLK_BLOCKS; ++b) t = cadd(t, partials[(int64_t)b * pp + pr]);  // loads hoisted
    out[pr] = t;
  }
}

// Y[n][c] = beta * Y[n][c] + alpha * sum_r X[n][r] C[r][c]   (C: p x p row-major, alpha/beta real)
template <typename XT>
__global__ void __launch_bounds__(BLK_THREADS) k_block_mul(int64_t n, int p, const XT* __restrict__ X,
                                                           const cplx* __restrict__ C, double alpha, double beta,
                                                           cplx* __restrict__ Y) {
  const int64_t total = n * p;  // C (at most 64 KB) is read through the read-only cache
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / p;
    const int c = (int)(e % p);
    cplx t = {0.0, 0.0};
    for (int r = 0; r < p; ++r) {
      const double2 wv = __ldg(reinterpret_cast<const double2*>(C) + r * p + c);
      const cplx x = ld_block<XT>(X, row * p + r), w = {wv.x, wv.y};
      t.re += x.re * w.re - x.im * w.im;
      t.im += x.re * w.im + x.im * w.re;
    }
    const cplx y0 = beta == 0.0 ? cplx{0.0, 0.0} : Y[e];
    Y[e] = {beta * y0.re + alpha * t.re, beta * y0.im + alpha * t.im};
  }
}

int blk_blocks() { return BLK_BLOCKS; }

// G = A^H B  (p x p, device)  through block partials `part` ([BLK_BLOCKS][p][p])
void launch_block_gram(const oras_handle* h, int p, const cplx* A, const cplx* B, cplx* part, cplx* G) {
  k_block_gram<<<BLK_BLOCKS, BLK_THREADS, 0, h->dev.stream>>>(h->mesh.ndof, p, A, B, part);
  k_block_sum<<<(p * p + 255) / 256, 256, 0, h->dev.stream>>>(p, part, G);
  count_launches(2);
}

// Y = beta Y + alpha X C with X complex FP64 or FP32 ([N][p]), C p x p on the device
void launch_block_mul_f64(const oras_handle* h, int p, const cplx* X, const cplx* C, double alpha, double beta,
                          cplx* Y) {
  const int64_t total = h->mesh.ndof * p;
  const unsigned blocks = (unsigned)std::min<int64_t>((total + BLK_THREADS - 1) / BLK_THREADS, 8 * BLK_BLOCKS);
  k_block_mul<cplx><<<blocks, BLK_THREADS, 0, h->dev.stream>>>(h->mesh.ndof, p, X, C, alpha, beta, Y);
  count_launches(1);
}
void launch_block_mul_f32(const oras_handle* h, int p, const void* X, const cplx* C, double alpha, double beta,
                          cplx* Y) {
  const int64_t total = h->mesh.ndof * p;
  const unsigned blocks = (unsigned)std::min<int64_t>((total + BLK_THREADS - 1) / BLK_THREADS, 8 * BLK_BLOCKS);
  k_block_mul<CT<float>><<<blocks, BLK_THREADS, 0, h->dev.stream>>>(h->mesh.ndof, p, (const CT<float>*)X, C, alpha,
                                                                   beta, Y);
  count_launches(1);
}

}  // namespace oras
