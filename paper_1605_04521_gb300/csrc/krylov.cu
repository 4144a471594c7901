// FP64 Krylov kernels of the right-preconditioned FGMRES(m) (Sec. 5): complex CSR SpMV,
// modified Gram-Schmidt Arnoldi with fused (axpy + next dot) passes, complex Givens rotations
// on the device, the small triangular solve and the solution update.  Multi-vectors are
// stored [N][k] (the k right-hand sides of a pseudo-block solve adjacent in memory).
// Every reduction is a fixed two-stage sum (block partials, then a fixed-order sum), so the
// results do not depend on scheduling.
#include "dev.cuh"

namespace oras {

constexpr int RED_BLOCKS = 304;   // 2 x 152 SMs
constexpr int RED_THREADS = 256;

template <typename XT> __device__ __forceinline__ cplx ld_c(const XT* p, int64_t i);
template <> __device__ __forceinline__ cplx ld_c<cplx>(const cplx* p, int64_t i) { return p[i]; }
template <> __device__ __forceinline__ cplx ld_c<CT<float>>(const CT<float>* p, int64_t i) {
  CT<float> v = p[i];
  return {(double)v.re, (double)v.im};
}

// y = A x  (x: [N][k] in XT, y: [N][k] FP64).  One warp per row, up to 8 RHS per pass.
template <typename XT>
__global__ void k_spmv(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ cols,
                       const cplx* __restrict__ vals, const XT* __restrict__ x, cplx* __restrict__ y,
                       int k, int r0, int kc) {
  int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  cplx acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = {0.0, 0.0};
  for (int64_t p = rowptr[row] + lane; p < rowptr[row + 1]; p += 32) {
    cplx a = vals[p];
    int64_t c = cols[p];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < kc) acc[q] = cadd(acc[q], cmul(a, ld_c<XT>(x, c * k + r0 + q)));
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (q >= kc) break;
    for (int o = 16; o > 0; o >>= 1) {
      acc[q].re += __shfl_down_sync(0xffffffffu, acc[q].re, o);
      acc[q].im += __shfl_down_sync(0xffffffffu, acc[q].im, o);
    }
    if (lane == 0) y[row * k + r0 + q] = acc[q];
  }
}

// ------------------------------------------------------------------ FP32-pipe SpMV, FP64 accuracy
// GB300 executes FP64 on a narrow pipe (about 1/64 of the FP32 rate), which caps the FP64 CSR
// SpMV far below the HBM bound.  The Arnoldi SpMV multiplies the FP64 matrix by preconditioned
// vectors that are exactly FP32 (z = M^-1 v with FP32 factors), so it is done on the FP32 pipes
// with error-free transformations: A = A_hi + A_lo with A_hi = fl32(A) and A_lo = fl32(A - A_hi)
// (the same 16 bytes per entry as FP64 complex), each product A_hi x split exactly into
// p + e by one FMA (two-product), each running sum kept as an unevaluated pair hi + lo with the
// rounding error of every addition recovered exactly (two-sum, Knuth).  The result carries
// about 2^-48 relative error per entry, the accuracy class of FP64, and is stored in FP64.

// hi + lo += a * x with a = a_hi + a_lo
__device__ __forceinline__ void df_mac(float& hi, float& lo, float a_hi, float a_lo, float x) {
  const float p = a_hi * x;
  const float ep = fmaf(a_hi, x, -p);           // a_hi * x - p, exactly
  const float t = hi + p;
  const float bp = t - hi;
  const float es = (hi - (t - bp)) + (p - bp);   // hi + p - t, exactly
  hi = t;
  lo += (ep + es) + a_lo * x;
}
// (h1 + l1) += (h2 + l2)
__device__ __forceinline__ void df_add(float& h1, float& l1, float h2, float l2) {
  const float t = h1 + h2;
  const float bp = t - h1;
  const float es = (h1 - (t - bp)) + (h2 - bp);
  h1 = t;
  l1 += es + l2;
}

// Exact float -> double by bit construction on the integer pipes (the conversion instruction runs
// on the FP64 pipe, which GB300 keeps narrow).  Subnormal floats become zero.
__device__ __forceinline__ double f2d_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t ex = (u >> 23) & 0xFFu;
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  if (ex == 0) return __longlong_as_double((long long)sign);
  const uint64_t e64 = ex == 0xFFu ? 0x7FFull : (uint64_t)ex + 896u;  // rebias 127 -> 1023
  return __longlong_as_double((long long)(sign | (e64 << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29)));
}

// vals_df[p] = {re_hi, im_hi, re_lo, im_lo}
__global__ void k_split_vals(int64_t nnz, const cplx* __restrict__ vals, float4* __restrict__ out) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nnz) return;
  const cplx v = vals[p];
  const float rh = (float)v.re, ih = (float)v.im;
  out[p] = make_float4(rh, ih, (float)(v.re - (double)rh), (float)(v.im - (double)ih));
}

// y = A x with x complex FP32 ([N][k]), y FP64 ([N][k]).  SPMV_LPR lanes per row (32 / SPMV_LPR
// rows per warp); KC right-hand sides per pass (kc <= KC of them live).  The kernel is bound by the
// latency of its dependent loads (column index, then the gathered x), so each lane issues the
// (value, column) loads of SPMV_UNR of its entries at once, then their x gathers, then the
// arithmetic: SPMV_UNR entries in flight per lane.
constexpr int SPMV_LPR = 8;
constexpr int SPMV_UNR = 4;

template <int KC>
__global__ void __launch_bounds__(256) k_spmv_df(int64_t n, const int64_t* __restrict__ rowptr,
                                                 const int32_t* __restrict__ cols, const float4* __restrict__ vals,
                                                 const CT<float>* __restrict__ x, cplx* __restrict__ y, int k,
                                                 int r0, int kc) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / SPMV_LPR;
  const int sl = threadIdx.x % SPMV_LPR;
  const bool live = row < n;
  float rh[KC], rl[KC], ih[KC], il[KC];
#pragma unroll
  for (int q = 0; q < KC; ++q) rh[q] = rl[q] = ih[q] = il[q] = 0.0f;
  if (live) {
    const int64_t p1 = rowptr[row + 1];
    for (int64_t p = rowptr[row] + sl; p < p1; p += SPMV_LPR * SPMV_UNR) {
      float4 a[SPMV_UNR];
      int64_t c[SPMV_UNR];
#pragma unroll
      for (int u = 0; u < SPMV_UNR; ++u) {
        const int64_t pu = p + (int64_t)u * SPMV_LPR;
        const bool in = pu < p1;
        a[u] = in ? vals[pu] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        c[u] = in ? (int64_t)cols[pu] : -1;
      }
      CT<float> xv[SPMV_UNR][KC];
#pragma unroll
      for (int u = 0; u < SPMV_UNR; ++u)
#pragma unroll
        for (int q = 0; q < KC; ++q)
          xv[u][q] = (c[u] >= 0 && q < kc) ? x[c[u] * k + r0 + q] : CT<float>{0.0f, 0.0f};
#pragma unroll
      for (int u = 0; u < SPMV_UNR; ++u)
#pragma unroll
        for (int q = 0; q < KC; ++q)
          if (q < kc) {
            df_mac(rh[q], rl[q], a[u].x, a[u].z, xv[u][q].re);    // + a_re x_re
            df_mac(rh[q], rl[q], -a[u].y, -a[u].w, xv[u][q].im);  // - a_im x_im
            df_mac(ih[q], il[q], a[u].x, a[u].z, xv[u][q].im);    // + a_re x_im
            df_mac(ih[q], il[q], a[u].y, a[u].w, xv[u][q].re);    // + a_im x_re
          }
    }
  }
#pragma unroll
  for (int q = 0; q < KC; ++q) {
    if (q >= kc) break;
#pragma unroll
    for (int o = SPMV_LPR / 2; o > 0; o >>= 1) {
      const float h2 = __shfl_down_sync(0xffffffffu, rh[q], o, SPMV_LPR), l2 = __shfl_down_sync(0xffffffffu, rl[q], o, SPMV_LPR);
      const float h3 = __shfl_down_sync(0xffffffffu, ih[q], o, SPMV_LPR), l3 = __shfl_down_sync(0xffffffffu, il[q], o, SPMV_LPR);
      df_add(rh[q], rl[q], h2, l2);
      df_add(ih[q], il[q], h3, l3);
    }
    if (live && sl == 0) y[row * k + r0 + q] = {f2d_bits(rh[q]) + f2d_bits(rl[q]), f2d_bits(ih[q]) + f2d_bits(il[q])};
  }
}

// Reductions over [N][k] multi-vectors (element e belongs to right-hand side e % k).  The grid's
// threads are cut to a multiple of k, teff = floor(T / k) k, and thread t < teff visits the
// elements t, t + teff, t + 2 teff, ...: all of one right-hand side r = t % k, so each thread
// keeps a single accumulator.  Block partial sums per right-hand side are formed in a fixed order
// (warp shuffles over the lanes of the same r when k divides 32, else a sequential sum of the
// block's per-thread values), then the fixed-order sum over blocks (sum_partials_warp): the results do
// not depend on scheduling.
__device__ __forceinline__ int64_t red_teff(int k) {
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  return T / k * k;
}

// partials[blockIdx.x][r] = sum of the per-thread values v of the block's threads with RHS r
__device__ void block_reduce_store(cplx v, int k, cplx* partials) {
  __shared__ cplx sh[RED_THREADS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * blockDim.x;
  if (32 % k == 0) {  // lane l holds RHS l % k (blockDim and 32 are multiples of k)
    for (int o = 16; o >= k; o >>= 1) {
      v.re += __shfl_xor_sync(0xffffffffu, v.re, o);
      v.im += __shfl_xor_sync(0xffffffffu, v.im, o);
    }
    if (lane < k) sh[warp * k + lane] = v;
    __syncthreads();
    if (threadIdx.x < k) {
      cplx t = {0.0, 0.0};
      for (int w = 0; w < RED_THREADS / 32; ++w) t = cadd(t, sh[w * k + threadIdx.x]);
      partials[(int64_t)blockIdx.x * k + threadIdx.x] = t;
    }
    return;
  }
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int r = threadIdx.x; r < k; r += blockDim.x) {
    cplx t = {0.0, 0.0};
    for (int q = (int)(((int64_t)r - base % k + k) % k); q < RED_THREADS; q += k) t = cadd(t, sh[q]);
    partials[(int64_t)blockIdx.x * k + r] = t;
  }
}

// Fixed-order sum of the block partials of the previous pass, by one warp: lane l loads the
// partials of blocks l, l + 32, ... at once (their loads overlap instead of each waiting for the
// previous add), adds them in that order, and a fixed xor-shuffle tree combines the lanes.  Every
// lane returns the total.
__device__ __forceinline__ cplx sum_partials_warp(const cplx* partials, int k, int r, int lane) {
  constexpr int PER = (RED_BLOCKS + 31) / 32;
  cplx v[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = lane + 32 * q;
    v[q] = b < RED_BLOCKS ? partials[(int64_t)b * k + r] : cplx{0.0, 0.0};
  }
  cplx t = v[0];
#pragma unroll
  for (int q = 1; q < PER; ++q) t = cadd(t, v[q]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    t.re += __shfl_xor_sync(0xffffffffu, t.re, o);
    t.im += __shfl_xor_sync(0xffffffffu, t.im, o);
  }
  return t;
}

// first dot of step j: partial <V_0, w>
__global__ void __launch_bounds__(RED_THREADS) k_dot(int64_t nk, int k, const cplx* __restrict__ a,
                                                     const cplx* __restrict__ b, cplx* __restrict__ partials) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, teff = red_teff(k);
  cplx acc = {0.0, 0.0};
  if (t < teff)
    for (int64_t e = t; e < nk; e += teff) {
      const cplx x = a[e], y = b[e];
      acc.re += x.re * y.re + x.im * y.im;
      acc.im += x.re * y.im - x.im * y.re;
    }
  block_reduce_store(acc, k, partials);
}

// h = sum(partials_in) (H[r][i][j] stored by block 0); w -= h V_i; then partial <V_next, w> or |w|^2.
__global__ void __launch_bounds__(RED_THREADS) k_mgs_step(int64_t nk, int k, int m, int i, int j,
                                                          const cplx* __restrict__ Vi, const cplx* __restrict__ Vn,
                                                          cplx* __restrict__ w, const cplx* __restrict__ pin,
                                                          cplx* __restrict__ pout, cplx* __restrict__ H) {
  __shared__ cplx hs[MAX_RHS];
  for (int r = threadIdx.x >> 5; r < k; r += blockDim.x >> 5) {  // one warp per right-hand side
    const cplx t = sum_partials_warp(pin, k, r, threadIdx.x & 31);
    if ((threadIdx.x & 31) == 0) {
      hs[r] = t;
      if (blockIdx.x == 0) H[((int64_t)r * (m + 1) + i) * m + j] = t;
    }
  }
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, teff = red_teff(k);
  cplx acc = {0.0, 0.0};
  if (t < teff) {
    const cplx h = hs[t % k];
    for (int64_t e = t; e < nk; e += teff) {
      const cplx v = Vi[e];
      cplx x = w[e];
      x.re -= h.re * v.re - h.im * v.im;
      x.im -= h.re * v.im + h.im * v.re;
      w[e] = x;
      if (Vn) {
        const cplx u = Vn[e];
        acc.re += u.re * x.re + u.im * x.im;
        acc.im += u.re * x.im - u.im * x.re;
      } else {
        acc.re += x.re * x.re + x.im * x.im;
      }
    }
  }
  block_reduce_store(acc, k, pout);
}

// h_{j+1,j} = ||w||; V_{j+1} = w / h (0 if h == 0); block 0 then runs the Givens update of
// every RHS: apply rotations 0..j-1 to column j of H, build rotation j, update g, res = |g_{j+1}|.
__global__ void __launch_bounds__(RED_THREADS) k_mgs_finish(int64_t nk, int k, int m, int j,
                                                            const cplx* __restrict__ w, cplx* __restrict__ Vn,
                                                            const cplx* __restrict__ pin, cplx* __restrict__ H,
                                                            double* __restrict__ cs, cplx* __restrict__ sn,
                                                            cplx* __restrict__ g, double* __restrict__ res) {
  __shared__ double hn[MAX_RHS];
  for (int r = threadIdx.x >> 5; r < k; r += blockDim.x >> 5) {  // one warp per right-hand side
    const cplx t = sum_partials_warp(pin, k, r, threadIdx.x & 31);
    if ((threadIdx.x & 31) == 0) hn[r] = sqrt(t.re);
  }
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nk; e += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(e % k);
    double h = hn[r];
    cplx x = w[e];
    Vn[e] = h > 0.0 ? cplx{x.re / h, x.im / h} : cplx{0.0, 0.0};
  }
  if (blockIdx.x != 0) return;
  for (int r = threadIdx.x; r < k; r += blockDim.x) {
    cplx* Hr = H + (int64_t)r * (m + 1) * m;
    double* c = cs + (int64_t)r * m;
    cplx* s = sn + (int64_t)r * m;
    cplx* gr = g + (int64_t)r * (m + 1);
    Hr[(int64_t)(j + 1) * m + j] = {hn[r], 0.0};
    for (int q = 0; q < j; ++q) {
      cplx a = Hr[(int64_t)q * m + j], b = Hr[(int64_t)(q + 1) * m + j];
      cplx t = cadd(cscale(a, c[q]), cmul(s[q], b));
      cplx u = csub(cscale(b, c[q]), cmul(cconj(s[q]), a));
      Hr[(int64_t)q * m + j] = t;
      Hr[(int64_t)(q + 1) * m + j] = u;
    }
    cplx a = Hr[(int64_t)j * m + j];
    double bb = hn[r];
    double aa = hypot(a.re, a.im);
    double cj;
    cplx sj;
    if (bb == 0.0) { cj = 1.0; sj = {0.0, 0.0}; }
    else if (aa == 0.0) { cj = 0.0; sj = {1.0, 0.0}; }
    else {
      double den = hypot(aa, bb);
      cj = aa / den;
      sj = {a.re / aa * bb / den, a.im / aa * bb / den};
    }
    c[j] = cj;
    s[j] = sj;
    Hr[(int64_t)j * m + j] = cadd(cscale(a, cj), cscale(sj, bb));
    Hr[(int64_t)(j + 1) * m + j] = {0.0, 0.0};
    cplx gj = gr[j];
    gr[j + 1] = cscale(cmul(cconj(sj), gj), -1.0);
    gr[j] = cscale(gj, cj);
    res[r] = hypot(gr[j + 1].re, gr[j + 1].im);
  }
}

// y = H(0:kk,0:kk)^{-1} g(0:kk) per RHS (back substitution), y = 0 for inactive RHS.
__global__ void k_hsolve(int k, int m, int kk, const cplx* __restrict__ H, const cplx* __restrict__ g,
                         const int32_t* __restrict__ active, cplx* __restrict__ y) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= k) return;
  const cplx* Hr = H + (int64_t)r * (m + 1) * m;
  cplx* yr = y + (int64_t)r * m;
  if (!active[r]) {
    for (int q = 0; q < kk; ++q) yr[q] = {0.0, 0.0};
    return;
  }
  for (int q = kk - 1; q >= 0; --q) {
    cplx t = g[(int64_t)r * (m + 1) + q];
    for (int l = q + 1; l < kk; ++l) t = csub(t, cmul(Hr[(int64_t)q * m + l], yr[l]));
    cplx d = Hr[(int64_t)q * m + q];
    double dd = d.re * d.re + d.im * d.im;
    yr[q] = dd > 0.0 ? cplx{(t.re * d.re + t.im * d.im) / dd, (t.im * d.re - t.re * d.im) / dd} : cplx{0.0, 0.0};
  }
}

// x += sum_q y_q Z_q   (Z: [m][N][k])
template <typename ZT>
__global__ void k_xupdate(int64_t nk, int k, int m, int kk, const ZT* __restrict__ Z, const cplx* __restrict__ y,
                          cplx* __restrict__ x) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nk) return;
  int r = (int)(e % k);
  cplx acc = x[e];
  for (int q = 0; q < kk; ++q) acc = cadd(acc, cmul(y[(int64_t)r * m + q], ld_c<ZT>(Z, (int64_t)q * nk + e)));
  x[e] = acc;
}

// r = b - A x (SpMV output in r already holds A x): r = b - r; partial |r|^2
__global__ void __launch_bounds__(RED_THREADS) k_residual(int64_t nk, int k, const cplx* __restrict__ b,
                                                          cplx* __restrict__ r, cplx* __restrict__ partials) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, teff = red_teff(k);
  cplx acc = {0.0, 0.0};
  if (t < teff)
    for (int64_t e = t; e < nk; e += teff) {
      const cplx v = csub(b[e], r[e]);
      r[e] = v;
      acc.re += v.re * v.re + v.im * v.im;
    }
  block_reduce_store(acc, k, partials);
}

// norms[r] = sqrt(sum partials) (single block)
__global__ void k_norms(int k, const cplx* __restrict__ partials, double* __restrict__ out) {
  for (int r = threadIdx.x >> 5; r < k; r += blockDim.x >> 5) {  // one warp per right-hand side
    const cplx t = sum_partials_warp(partials, k, r, threadIdx.x & 31);
    if ((threadIdx.x & 31) == 0) out[r] = sqrt(t.re);
  }
}

// V0 = r / beta for active RHS (0 otherwise); g = (beta, 0, ...)
__global__ void k_restart(int64_t nk, int k, int m, const cplx* __restrict__ rv, const double* __restrict__ beta,
                          const int32_t* __restrict__ active, cplx* __restrict__ V0, cplx* __restrict__ g) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nk) {
    int q = (int)(e % k);
    double b = beta[q];
    V0[e] = (active[q] && b > 0.0) ? cplx{rv[e].re / b, rv[e].im / b} : cplx{0.0, 0.0};
  }
  if (e < k) {
    for (int l = 0; l <= m; ++l) g[(int64_t)e * (m + 1) + l] = {0.0, 0.0};
    g[(int64_t)e * (m + 1)] = {active[e] ? beta[e] : 0.0, 0.0};
  }
}

// column-major host layout [k][N] <-> internal [N][k]
__global__ void k_to_internal(int64_t n, int k, const cplx* __restrict__ src, cplx* __restrict__ dst) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * k) return;
  int64_t g = e / k;
  int r = (int)(e % k);
  dst[e] = src[(int64_t)r * n + g];
}
__global__ void k_to_internal_c64(int64_t n, int k, const CT<float>* __restrict__ src, CT<float>* __restrict__ dst) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * k) return;
  dst[e] = src[(int64_t)(e % k) * n + e / k];
}
__global__ void k_to_external(int64_t n, int k, const cplx* __restrict__ src, cplx* __restrict__ dst) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * k) return;
  int64_t g = e / k;
  int r = (int)(e % k);
  dst[(int64_t)r * n + g] = src[e];
}

// ------------------------------------------------------------------ launchers
template <typename XT>
static void spmv_t(const oras_handle* h, const XT* x, cplx* y, int k) {
  const auto& m = h->mesh;
  const auto& d = h->dev;
  int64_t blocks = (m.ndof * 32 + 255) / 256;
  for (int r0 = 0; r0 < k; r0 += 8) {
    int kc = k - r0 < 8 ? k - r0 : 8;
    k_spmv<XT><<<(unsigned)blocks, 256, 0, d.stream>>>(m.ndof, d.rowptr, d.cols, d.vals, x, y, k, r0, kc);
    count_launches(1);
  }
}
void launch_spmv_f64(const oras_handle* h, const cplx* x, cplx* y, int k) { spmv_t<cplx>(h, x, y, k); }
// complex FP32 x: FP32-pipe kernel with FP64-class accuracy (k_spmv_df)
void launch_spmv_f32(const oras_handle* h, const void* x, cplx* y, int k) {
  const auto& m = h->mesh;
  const auto& d = h->dev;
  const int64_t blocks = (m.ndof * SPMV_LPR + 255) / 256;
  for (int r0 = 0; r0 < k; r0 += 8) {
    const int kc = k - r0 < 8 ? k - r0 : 8;
    const CT<float>* xx = (const CT<float>*)x;
    if (kc == 1) k_spmv_df<1><<<(unsigned)blocks, 256, 0, d.stream>>>(m.ndof, d.rowptr, d.cols, d.vals_df, xx, y, k, r0, kc);
    else if (kc == 2) k_spmv_df<2><<<(unsigned)blocks, 256, 0, d.stream>>>(m.ndof, d.rowptr, d.cols, d.vals_df, xx, y, k, r0, kc);
    else if (kc <= 4) k_spmv_df<4><<<(unsigned)blocks, 256, 0, d.stream>>>(m.ndof, d.rowptr, d.cols, d.vals_df, xx, y, k, r0, kc);
    else k_spmv_df<8><<<(unsigned)blocks, 256, 0, d.stream>>>(m.ndof, d.rowptr, d.cols, d.vals_df, xx, y, k, r0, kc);
    count_launches(1);
  }
}
void launch_split_vals(const oras_handle* h) {
  const int64_t nnz = (int64_t)h->mesh.cols.size();
  k_split_vals<<<(unsigned)((nnz + 255) / 256), 256, 0, h->dev.stream>>>(nnz, h->dev.vals, h->dev.vals_df);
  count_launches(1);
}

void launch_dot(const oras_handle* h, const cplx* a, const cplx* b, cplx* partials, int k) {
  k_dot<<<RED_BLOCKS, RED_THREADS, 0, h->dev.stream>>>(h->mesh.ndof * k, k, a, b, partials);
  count_launches(1);
}
void launch_mgs_step(const oras_handle* h, int k, int m, int i, int j, const cplx* Vi, const cplx* Vn, cplx* w,
                     const cplx* pin, cplx* pout, cplx* H) {
  k_mgs_step<<<RED_BLOCKS, RED_THREADS, 0, h->dev.stream>>>(h->mesh.ndof * k, k, m, i, j, Vi, Vn, w, pin, pout, H);
  count_launches(1);
}
void launch_mgs_finish(const oras_handle* h, int k, int m, int j, const cplx* w, cplx* Vn, const cplx* pin,
                       cplx* H, double* cs, cplx* sn, cplx* g, double* res) {
  k_mgs_finish<<<RED_BLOCKS, RED_THREADS, 0, h->dev.stream>>>(h->mesh.ndof * k, k, m, j, w, Vn, pin, H, cs, sn, g, res);
  count_launches(1);
}
void launch_hsolve(const oras_handle* h, int k, int m, int kk, const cplx* H, const cplx* g, const int32_t* active,
                   cplx* y) {
  k_hsolve<<<1, 64, 0, h->dev.stream>>>(k, m, kk, H, g, active, y);
  count_launches(1);
}
void launch_xupdate_f64(const oras_handle* h, int k, int m, int kk, const cplx* Z, const cplx* y, cplx* x) {
  int64_t nk = h->mesh.ndof * k;
  k_xupdate<cplx><<<(unsigned)((nk + 255) / 256), 256, 0, h->dev.stream>>>(nk, k, m, kk, Z, y, x);
  count_launches(1);
}
void launch_xupdate_f32(const oras_handle* h, int k, int m, int kk, const void* Z, const cplx* y, cplx* x) {
  int64_t nk = h->mesh.ndof * k;
  k_xupdate<CT<float>><<<(unsigned)((nk + 255) / 256), 256, 0, h->dev.stream>>>(nk, k, m, kk, (const CT<float>*)Z, y, x);
  count_launches(1);
}
void launch_residual(const oras_handle* h, int k, const cplx* b, cplx* r, cplx* partials) {
  k_residual<<<RED_BLOCKS, RED_THREADS, 0, h->dev.stream>>>(h->mesh.ndof * k, k, b, r, partials);
  count_launches(1);
}
void launch_norms(const oras_handle* h, int k, const cplx* partials, double* out) {
  k_norms<<<1, 256, 0, h->dev.stream>>>(k, partials, out);
  count_launches(1);
}
void launch_restart(const oras_handle* h, int k, int m, const cplx* rv, const double* beta, const int32_t* active,
                    cplx* V0, cplx* g) {
  int64_t nk = h->mesh.ndof * k;
  k_restart<<<(unsigned)((nk + 255) / 256), 256, 0, h->dev.stream>>>(nk, k, m, rv, beta, active, V0, g);
  count_launches(1);
}
void launch_to_internal_c64(const oras_handle* h, int k, const void* src, void* dst) {
  const int64_t nk = h->mesh.ndof * k;
  k_to_internal_c64<<<(unsigned)((nk + 255) / 256), 256, 0, h->dev.stream>>>(h->mesh.ndof, k, (const CT<float>*)src,
                                                                            (CT<float>*)dst);
  count_launches(1);
}
void launch_to_internal(const oras_handle* h, int k, const cplx* src, cplx* dst) {
  int64_t nk = h->mesh.ndof * k;
  k_to_internal<<<(unsigned)((nk + 255) / 256), 256, 0, h->dev.stream>>>(h->mesh.ndof, k, src, dst);
  count_launches(1);
}
void launch_to_external(const oras_handle* h, int k, const cplx* src, cplx* dst) {
  int64_t nk = h->mesh.ndof * k;
  k_to_external<<<(unsigned)((nk + 255) / 256), 256, 0, h->dev.stream>>>(h->mesh.ndof, k, src, dst);
  count_launches(1);
}
int red_blocks() { return RED_BLOCKS; }

}  // namespace oras
