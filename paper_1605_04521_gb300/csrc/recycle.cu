// FP64 kernels of GCRO-DR (Sec. 6: recycling a Krylov subspace across the imaging loop's
// sequence of systems).  Its vectors are single columns of N complex values, stored one after the
// other ([column][N]): the Arnoldi basis V, the recycled pair U, C (A M^{-1} U = C, C^H C = I) and
// the work vectors.  The products with a few columns -- X^H w, w -= X t and Y = X M with small
// M -- stream the columns once.  Reductions are fixed two-stage sums (block partials, then a
// fixed-order sum over the blocks), so results do not depend on scheduling.
#include "dev.cuh"

namespace oras {

constexpr int RC_BLOCKS = 304;   // 2 x 152 SMs
constexpr int RC_THREADS = 256;
constexpr int RC_MAXQ = 16;      // columns per pass of the dot kernel (more go in further passes)

// partials[b][q] = sum over the rows of block b of conj(X_q[n]) w[n], q < nq <= RC_MAXQ: per
// thread, then a shuffle tree per warp, then the warps in order
__global__ void __launch_bounds__(RC_THREADS) k_rc_dots(int64_t n, int nq, const cplx* __restrict__ X, int64_t ldx,
                                                        const cplx* __restrict__ w, cplx* __restrict__ partials) {
  __shared__ cplx sh[RC_THREADS / 32][RC_MAXQ];
  cplx acc[RC_MAXQ];
#pragma unroll
  for (int q = 0; q < RC_MAXQ; ++q) acc[q] = {0.0, 0.0};
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per, r1 = r0 + per < n ? r0 + per : n;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += RC_THREADS) {
    const cplx wv = w[i];
#pragma unroll
    for (int q = 0; q < RC_MAXQ; ++q)
      if (q < nq) {
        const cplx x = X[q * ldx + i];
        acc[q].re += x.re * wv.re + x.im * wv.im;
        acc[q].im += x.re * wv.im - x.im * wv.re;
      }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < RC_MAXQ; ++q) {
    cplx t = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      t.re += __shfl_xor_sync(0xffffffffu, t.re, o);
      t.im += __shfl_xor_sync(0xffffffffu, t.im, o);
    }
    if (lane == 0) sh[warp][q] = t;
  }
  __syncthreads();
  if (threadIdx.x < nq) {
    cplx t = sh[0][threadIdx.x];
    for (int v = 1; v < RC_THREADS / 32; ++v) t = cadd(t, sh[v][threadIdx.x]);
    partials[(int64_t)blockIdx.x * RC_MAXQ + threadIdx.x] = t;
  }
}

// out[q] = fixed-order sum over the blocks of partials[b][q]
__global__ void k_rc_sum(int nq, const cplx* __restrict__ partials, cplx* __restrict__ out) {
  const int q = threadIdx.x;
  if (q >= nq) return;
  cplx t = {0.0, 0.0};
  for (int b = 0; b < RC_BLOCKS; ++b) t = cadd(t, partials[(int64_t)b * RC_MAXQ + q]);
  out[q] = t;
}

// Y_c[n] = beta * Y_c[n] + alpha * sum_q X_q[n] M[q][c]  (M: nq x nc row-major on the device)
__global__ void __launch_bounds__(RC_THREADS) k_rc_lincomb(int64_t n, int nq, int nc, const cplx* __restrict__ X,
                                                           int64_t ldx, const cplx* __restrict__ M, double alpha,
                                                           double beta, cplx* __restrict__ Y, int64_t ldy) {
  const int64_t total = n * nc;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / n);
    const int64_t i = e % n;
    cplx t = {0.0, 0.0};
    for (int q = 0; q < nq; ++q) {
      const cplx x = X[q * ldx + i];
      const double2 m = __ldg(reinterpret_cast<const double2*>(M) + q * nc + c);
      t.re += x.re * m.x - x.im * m.y;
      t.im += x.re * m.y + x.im * m.x;
    }
    cplx& y = Y[c * ldy + i];
    const cplx y0 = beta == 0.0 ? cplx{0.0, 0.0} : y;
    y = {beta * y0.re + alpha * t.re, beta * y0.im + alpha * t.im};
  }
}

// out[n] = s * x[n] (s real)
__global__ void k_rc_scale(int64_t n, const cplx* __restrict__ x, double s, cplx* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = {s * x[i].re, s * x[i].im};
}

// out[n] = x[n] (complex FP32 to FP64, exact)
__global__ void k_rc_widen(int64_t n, const CT<float>* __restrict__ x, cplx* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = {(double)x[i].re, (double)x[i].im};
}

static unsigned rc_grid(int64_t work) {
  const int64_t b = (work + RC_THREADS - 1) / RC_THREADS;
  return (unsigned)(b < 8 * RC_BLOCKS ? (b > 0 ? b : 1) : 8 * RC_BLOCKS);
}

int rc_max_q() { return RC_MAXQ; }
size_t rc_partials_elems() { return (size_t)RC_BLOCKS * RC_MAXQ; }

// out[0..nq) = X^H w over the columns X_0..X_{nq-1} (ldx apart); partials: rc_partials_elems()
void launch_rc_dots(cudaStream_t st, int64_t n, int nq, const cplx* X, int64_t ldx, const cplx* w, cplx* partials,
                    cplx* out) {
  for (int q0 = 0; q0 < nq; q0 += RC_MAXQ) {
    const int nb = nq - q0 < RC_MAXQ ? nq - q0 : RC_MAXQ;
    k_rc_dots<<<RC_BLOCKS, RC_THREADS, 0, st>>>(n, nb, X + q0 * ldx, ldx, w, partials);
    k_rc_sum<<<1, 32, 0, st>>>(nb, partials, out + q0);
    count_launches(2);
  }
}

// Y = beta Y + alpha X M (nc columns of Y, ldy apart; M nq x nc row-major on the device)
void launch_rc_lincomb(cudaStream_t st, int64_t n, int nq, int nc, const cplx* X, int64_t ldx, const cplx* M,
                       double beta, cplx* Y, int64_t ldy, double alpha) {
  k_rc_lincomb<<<rc_grid(n * nc), RC_THREADS, 0, st>>>(n, nq, nc, X, ldx, M, alpha, beta, Y, ldy);
  count_launches(1);
}

void launch_rc_widen(cudaStream_t st, int64_t n, const void* x, cplx* out) {
  k_rc_widen<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, (const CT<float>*)x, out);
  count_launches(1);
}

void launch_rc_scale(cudaStream_t st, int64_t n, const cplx* x, double s, cplx* out) {
  k_rc_scale<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x, s, out);
  count_launches(1);
}

}  // namespace oras
