// Batched dense LU with row pivoting of the local matrices A_s (Sec. 4: the A_s^{-1} of ORAS),
// P_s A_s = L_s U_s, over the tiled arena (TB x TB complex tiles, split re/im planes, row-major
// on and below the block diagonal, column-major above it).
//
// Blocked LU: right-looking across outer panels W tile columns wide (one trailing update per
// panel), sub-panels of LU_SUB columns inside a panel, left-looking inside a sub-panel.  Every
// tile column k is processed for all subdomains at once by
//  0. bringing column k, on and below the diagonal, up to date with the sub-panel's earlier
//     steps (C_Ik -= sum_{k1 <= j < k} L_Ij U_jk, k1 the sub-panel's first step: one tile
//     column written per step, where updating all the sub-panel's remaining columns after
//     every step would rewrite each of them up to LU_SUB times);
//  1. tournament pivoting of the tall panel column: chunks of rows are reduced with partial
//     pivoting (pivot = max |Re| + |Im|, first on ties) to TB candidate rows each; candidate
//     sets are merged the same way up a tree (4-way for FP32, 2-way for FP64); the root's
//     choice is the pivot sequence of the step and its factored TB x TB block is L11\U11
//     (communication-avoiding LU, Grigori, Demmel, Xiang 2011);
//  2. the row interchanges of the step, applied to every column (one permutation of at most
//     2 TB rows);
//  3. the pivot tile row, right of column k, receives the updates it still lacks
//     (C_kJ -= sum_j L_kj U_jJ over the steps listed below);
//  4. L21 = A21 U11^{-1} below and U12 = L11^{-1} A12 along (part of) the tile row.
// Tensor-core path (FP32 factors).  At a sub-panel's start its LU_SUB columns, for every row from
// k1 down, receive the updates of the panel's earlier sub-panels in one contraction (the
// sub-panel level is left-looking too); steps 3-4 cover the pivot row inside the sub-panel
// only; after the sub-panel's last step its rows are completed right of it by a blocked
// triangular solve with the panel's L: one product brings in the panel's earlier sub-panels,
// then row by row the sub-panel's earlier rows and U_kJ = L_kk^{-1} C_kJ (the sub-panel's
// L_kk^{-1} wait in scratch tiles for this).  A pivot row thus re-reads at most LU_SUB - 1
// earlier U rows one at a time instead of up to W - 1, and the left-looking steps at most
// LU_SUB - 1 earlier L columns.
// CUDA-core path (FP64 factors, or the CUDA-core engine).  After a sub-panel's last step a mid
// update brings the panel's later columns, for every row below, up to date with the sub-panel;
// step 3 covers the pivot row inside the panel from the sub-panel's earlier steps and beyond it
// from all the panel's earlier steps; step 4 the whole row.
// After the W columns of a panel, the trailing matrix gets one update with a W-tile-deep
// contraction, C_IJ -= sum_k L_Ik U_kJ, which reads and writes every trailing tile once per
// panel instead of once per column.  Right of column k, every row not yet a pivot row is in
// one common state until then, so a row interchange never mixes rows that have received
// different updates.
// The tree merge uses "last arriver continues" counters, so no block ever waits for another.
#include <algorithm>
#include <climits>
#include <cstdio>

#include "lu.cuh"

namespace oras {

template <typename R> __device__ __forceinline__ CT<R> mulc(CT<R> a, CT<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R> __device__ __forceinline__ CT<R> subc(CT<R> a, CT<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> __device__ __forceinline__ CT<R> invc(CT<R> a) {
  R d = a.re * a.re + a.im * a.im;
  return {a.re / d, -a.im / d};
}
template <typename R> __device__ __forceinline__ R abs1(CT<R> a) { return fabs(a.re) + fabs(a.im); }

template <typename R> struct LuCfg;
template <> struct LuCfg<float> { static constexpr int CH = 256; };
template <> struct LuCfg<double> { static constexpr int CH = 128; };

constexpr int PS = TB + 1;  // padded row stride of the panel in shared memory
constexpr int LU_THREADS = 256;
constexpr int INV_THREADS = 512;  // diagonal-block inversion: 16 warps over the 2 TB columns

struct LuArgs {
  int nsub;
  int k;
  const int64_t* np;        // [nsub] padded order
  const int64_t* tile_off;  // [nsub]
  const int64_t* np_off;    // [nsub] prefix of np (perm arrays)
  int32_t* perm;            // [sum np]
  int32_t* cand;            // [nsub][slots][TB]
  int32_t* cnt;             // [nsub][slots]
  int slots;
  int32_t* pairs;           // [nsub][2*TB][2] (dst, src)
  int32_t* pairs_n;         // [nsub]
  void* diag;               // [nsub][TB*TB] factored diagonal tile (complex, column-major)
  int32_t* status;
};


template <typename R>
__device__ __forceinline__ R* tile_base(void* arena, const LuArgs& a, int s, int64_t I, int64_t J) {
  int64_t nts = a.np[s] / TB;
  return (R*)arena + (a.tile_off[s] + I * nts + J) * 2 * TILE_PLANE;
}
template <typename R>
__device__ __forceinline__ CT<R> tload(const R* t, bool rm, int64_t i, int64_t j) {
  int64_t e = tile_elem(rm, i, j);
  return {t[e], t[TILE_PLANE + e]};
}
template <typename R>
__device__ __forceinline__ void tstore(R* t, bool rm, int64_t i, int64_t j, CT<R> v) {
  int64_t e = tile_elem(rm, i, j);
  t[e] = v.re;
  t[TILE_PLANE + e] = v.im;
}

// Partial-pivoting elimination of an m x TB panel P (row stride PS) held in shared memory,
// carrying row ids.  On return rows 0..TB-1 are the chosen pivot rows in order, factored.
template <typename R>
__device__ void gepp_panel(CT<R>* P, int32_t* ids, int m, R* rv, int* ri) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int ncol = m < TB ? m : TB;
  for (int c = 0; c < ncol; ++c) {
    R best = -1;
    int bi = 0x7fffffff;
    for (int i = c + tid; i < m; i += nthr) {
      R v = abs1(P[i * PS + c]);
      if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      R ov = __shfl_down_sync(0xffffffffu, best, o);
      int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if ((tid & 31) == 0) { rv[tid >> 5] = best; ri[tid >> 5] = bi; }
    __syncthreads();
    if (tid == 0) {
      R b = rv[0];
      int i0 = ri[0];
      for (int w = 1; w < nthr / 32; ++w)
        if (rv[w] > b || (rv[w] == b && ri[w] < i0)) { b = rv[w]; i0 = ri[w]; }
      ri[0] = (b > 0) ? i0 : c;  // exactly zero column: keep the row in place
    }
    __syncthreads();
    const int p = ri[0];
    if (p != c) {
      for (int j = tid; j < TB; j += nthr) {
        CT<R> t = P[c * PS + j];
        P[c * PS + j] = P[p * PS + j];
        P[p * PS + j] = t;
      }
      if (tid == 0) { int32_t t = ids[c]; ids[c] = ids[p]; ids[p] = t; }
    }
    __syncthreads();
    CT<R> piv = P[c * PS + c];
    if (abs1(piv) > R(0)) {
      CT<R> inv = invc(piv);
      for (int i = c + 1 + tid; i < m; i += nthr) {
        CT<R> l = mulc(P[i * PS + c], inv);
        P[i * PS + c] = l;
        for (int j = c + 1; j < TB; ++j) P[i * PS + j] = subc(P[i * PS + j], mulc(l, P[c * PS + j]));
      }
    }
    __syncthreads();
  }
}

// Load panel rows `rows[0..m)` (matrix row indices, all in tile rows >= k) of tile column k.
template <typename R>
__device__ void load_rows(void* arena, const LuArgs& a, int s, const int32_t* rows, int m, CT<R>* P) {
  for (int e = threadIdx.x; e < m * TB; e += blockDim.x) {
    int i = e / TB, j = e % TB;
    int32_t r = rows[i];
    const R* t = tile_base<R>(arena, a, s, r / TB, a.k);
    P[i * PS + j] = tload<R>(t, true, r % TB, j);
  }
}

template <typename R>
__global__ void __launch_bounds__(LU_THREADS) k_lu_tournament(LuArgs a, void* arena) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int CH = LuCfg<R>::CH;
  CT<R>* P = (CT<R>*)smem_raw;                         // [CH][PS]
  int32_t* ids = (int32_t*)(P + CH * PS);              // [CH]
  R* rv = (R*)(ids + CH);                              // [32]
  int* ri = (int*)(rv + 32);                           // [32]
  __shared__ int s_old;
  const int s = blockIdx.y;
  const int64_t np = a.np[s], nts = np / TB;
  if (a.k >= nts) return;
  const int64_t R0 = (int64_t)a.k * TB;
  const int64_t rows_total = np - R0;
  const int nch = (int)((rows_total + CH - 1) / CH);
  int c = blockIdx.x;
  if (c >= nch) return;
  int64_t mrem = rows_total - (int64_t)c * CH;
  int m = (int)(mrem < CH ? mrem : CH);
  for (int i = threadIdx.x; i < m; i += blockDim.x) ids[i] = (int32_t)(R0 + (int64_t)c * CH + i);
  __syncthreads();
  load_rows<R>(arena, a, s, ids, m, P);
  __syncthreads();
  gepp_panel<R>(P, ids, m, rv, ri);
  int32_t* cand = a.cand + (int64_t)s * a.slots * TB;
  int32_t* cnt = a.cnt + (int64_t)s * a.slots;
  int level_off = 0, n_l = nch, j = c;
  if (n_l > 1)
    for (int i = threadIdx.x; i < TB; i += blockDim.x) cand[(level_off + j) * TB + i] = ids[i];
  while (n_l > 1) {
    const int n_next = (n_l + 1) >> 1;
    const int parent = j >> 1, sib = j ^ 1;
    const int next_off = level_off + n_l;
    if (sib >= n_l) {  // odd one out: pass the candidates up unchanged
      for (int i = threadIdx.x; i < TB; i += blockDim.x) cand[(next_off + parent) * TB + i] = ids[i];
      level_off = next_off; n_l = n_next; j = parent;
      continue;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_old = atomicAdd(&cnt[next_off + parent], 1);
    __syncthreads();
    if (s_old == 0) return;  // the sibling will merge
    if (threadIdx.x == 0) cnt[next_off + parent] = 0;
    __threadfence();
    const int left = j & ~1;
    for (int i = threadIdx.x; i < 2 * TB; i += blockDim.x) {
      int child = left + (i >= TB);
      ids[i] = ((volatile int32_t*)cand)[(level_off + child) * TB + (i % TB)];
    }
    __syncthreads();
    load_rows<R>(arena, a, s, ids, 2 * TB, P);
    __syncthreads();
    gepp_panel<R>(P, ids, 2 * TB, rv, ri);
    level_off = next_off; n_l = n_next; j = parent;
    if (n_l > 1)
      for (int i = threadIdx.x; i < TB; i += blockDim.x) cand[(level_off + j) * TB + i] = ids[i];
  }
  // root: ids[0..TB) are the pivot rows, P[0..TB) the factored diagonal block
  CT<R>* dg = (CT<R>*)a.diag + (int64_t)s * TB * TB;
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    int i = e % TB, jj = e / TB;
    dg[jj * TB + i] = P[i * PS + jj];
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < TB; ++i)
      if (!(abs1(P[i * PS + i]) > R(0))) {
        atomicCAS(&a.status[ST_ERR], DEV_OK, DEV_SINGULAR);
        a.status[ST_SUB] = s;
      }
  }
  // permutation of the step: position R0+i receives row ids[i]; the displaced rows of the top
  // block fill the vacated pivot positions (LAPACK interchange order).
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t posv[2 * TB], rowv[2 * TB];
    int nm = 0;
    auto row_at = [&](int32_t pos) {
      for (int q = 0; q < nm; ++q)
        if (posv[q] == pos) return rowv[q];
      return pos;
    };
    auto pos_of = [&](int32_t row) {
      for (int q = 0; q < nm; ++q)
        if (rowv[q] == row) return posv[q];
      return row;  // untouched row is still at its own position
    };
    auto set = [&](int32_t pos, int32_t row) {
      for (int q = 0; q < nm; ++q)
        if (posv[q] == pos) { rowv[q] = row; return; }
      posv[nm] = pos; rowv[nm] = row; ++nm;
    };
    for (int i = 0; i < TB; ++i) {
      int32_t tgt = (int32_t)(R0 + i);
      int32_t pr = pos_of(ids[i]);
      if (pr != tgt) {
        int32_t ra = row_at(tgt), rb = row_at(pr);
        set(tgt, rb);
        set(pr, ra);
      }
    }
    int32_t* pr = a.pairs + (int64_t)s * 2 * TB * 2;
    int np_ = 0;
    for (int q = 0; q < nm; ++q)
      if (posv[q] != rowv[q]) { pr[np_ * 2] = posv[q]; pr[np_ * 2 + 1] = rowv[q]; ++np_; }
    a.pairs_n[s] = np_;
  }
}

// ------------------------------------------------------------------ FP32 tournament, rows in registers
// Same tournament as above, with the elimination done on register-resident rows: candidate row r
// is held by threads 2r (the real parts of its 64 entries) and 2r+1 (the imaginary parts), so a
// block of 512 threads carries 256 rows at about 100 registers per thread and 16 warps per SM
// hide the latency of each column's block-wide pivot choice.  No row is moved: the chosen pivot
// row is marked and its values are broadcast through shared memory.
// Pivot choice: max |Re| + |Im| over unchosen rows (to a relative 2^-14: the key keeps the top
// 14 mantissa bits of the magnitude), ties to the lowest candidate position.
//
// Blocked elimination, 8 columns at a time (within a block the column indices are compile-time,
// so the rows stay in registers; after each block every row is rotated left by 8 so the next
// block's columns come to positions 0..7, and after the 8th rotation the rows are back in their
// original order).  Inside a block the pivots are found column by column and only the block's 8
// columns are updated; each warp's best candidate publishes its in-block values before the
// block-wide choice, so one barrier per column suffices.  At the end of the block, the columns
// right of it receive one rank-8 update from the block's 8 pivot rows, whose own values there are
// first brought up to date by a triangular correction with the block's multipliers (blocked
// right-looking LU: U12 = L11^{-1} A12, A22 -= L21 U12).  Positions >= 64 - 8*block hold columns
// eliminated in earlier blocks (multipliers) and are skipped block by block.
//
// With the two parts of a complex entry in two threads, a complex multiply-subtract
// x -= l * u becomes, in each thread, x_part -= al * Re(u) + be * Im(u) with (al, be) = (Re l,
// -Im l) for the real part and (Im l, Re l) for the imaginary part.  The block's pivot rows are
// kept column by column ([column][pivot], the 8 values of a column contiguous), so the rank-8
// update of one entry is 8 packed FP32 multiply-adds (fma.rn.f32x2) over pairs of pivots: the
// pair of partial sums is added at the end.
constexpr int RI_THREADS = 512;
constexpr int RI_ROWS = RI_THREADS / 2;
constexpr int RI_WARPS = RI_THREADS / 32;
struct RiGepp {
  alignas(16) float candr[2][RI_WARPS][8];             // each warp's best candidate's in-block values
  alignas(16) float candi[2][RI_WARPS][8];
  uint32_t wk[2][RI_WARPS];                            // each warp's best pivot key (by column parity)
  alignas(16) float Pr[TB][8];                         // the block's pivot rows: [rotated position][pivot]
  alignas(16) float Pi[TB][8];
  int order[TB];                                       // pivot rank -> candidate position
};

// Pivot key of candidate position `row` (< 256) with magnitude v >= 0: the magnitude's bits with
// the 9 lowest replaced by a validity bit and 255 - row, so the largest key has the largest
// magnitude and, among equal magnitudes, the lowest position.  0 means no candidate.
__device__ __forceinline__ uint32_t pivot_key(float v, int row) {
  return (__float_as_uint(v) & 0xFFFFFE00u) | 0x100u | (uint32_t)(255 - row);
}

__device__ __forceinline__ void gepp_ri(float (&x)[TB], bool valid, RiGepp& g, int& myrank, float& mypiv) {
  constexpr unsigned FULL = 0xffffffffu;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, row = t >> 1, part = t & 1;
  bool chosen = false;
  myrank = -1;
  mypiv = 0.0f;
  if (t < TB) g.order[t] = -1;
  __syncthreads();
#pragma unroll 1
  for (int cb = 0; cb < TB / 8; ++cb) {
    const int lim = TB - 8 * cb;  // rotated positions >= lim: columns eliminated in earlier blocks
    int my_c8 = -1;               // in-block column at which this row became a pivot in this block
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) {
      const int c = 8 * cb + c8;
      const int b = c8 & 1;
      const float xo = __shfl_xor_sync(FULL, x[c8], 1);  // the other part of this entry
      const float xre = part ? xo : x[c8], xim = part ? x[c8] : xo;
      float v = fabsf(xre) + fabsf(xim);
      if (v != v) v = 0.0f;  // a non-finite entry still lets a row be chosen
      uint32_t k = (valid && !chosen) ? pivot_key(v, row) : 0u;
      k = __reduce_max_sync(FULL, k);  // the warp's best (both parts of a row hold the same key)
      if (k != 0u && 255 - (int)(k & 0xFFu) == row) {  // the warp's candidate publishes its in-block values
        float* dst = part ? g.candi[b][warp] : g.candr[b][warp];
#pragma unroll
        for (int j = c8; j < 8; ++j) dst[j] = x[j];
      }
      if (lane == 0) g.wk[b][warp] = k;
      __syncthreads();
      const uint32_t bk = __reduce_max_sync(FULL, g.wk[b][lane & (RI_WARPS - 1)]);
      const int brow = 255 - (int)(bk & 0xFFu), bw = brow >> 4;  // rows 16w..16w+15 are warp w's
      const bool nonzero = (bk >> 9) != 0u;
      if (bk != 0u && row == brow) {
        chosen = true;
        myrank = c;
        mypiv = nonzero ? v : 0.0f;
        my_c8 = c8;
        if (part == 0) g.order[c] = row;
      }
      if (nonzero && valid && !chosen) {  // multiplier and update of the block's later columns
        const float4* cr = reinterpret_cast<const float4*>(g.candr[b][bw]);
        const float4* ci = reinterpret_cast<const float4*>(g.candi[b][bw]);
        float ur[8], ui[8];
        *reinterpret_cast<float4*>(ur) = cr[0];
        *reinterpret_cast<float4*>(ur + 4) = cr[1];
        *reinterpret_cast<float4*>(ui) = ci[0];
        *reinterpret_cast<float4*>(ui + 4) = ci[1];
        const float pr = ur[c8], pi = ui[c8];
        const float rden = __frcp_rn(pr * pr + pi * pi);
        const float lr = (xre * pr + xim * pi) * rden, li = (xim * pr - xre * pi) * rden;
        const float al = part ? li : lr, be = part ? lr : -li;
        x[c8] = al;
#pragma unroll
        for (int j = c8 + 1; j < 8; ++j) x[j] -= al * ur[j] + be * ui[j];
      } else if (!nonzero && valid && !chosen) {  // exactly zero column: no elimination
        x[c8] = 0.0f;
      }
    }
    // the block's pivot rows: in-block multipliers and U values, then the stale part right of it
    if (my_c8 >= 0) {
      float(*dst)[8] = part ? g.Pi : g.Pr;
#pragma unroll
      for (int jb = 0; jb < TB / 8; ++jb)
        if (8 * jb < lim) {
#pragma unroll
          for (int j = 8 * jb; j < 8 * jb + 8; ++j) dst[j][my_c8] = x[j];
        }
    }
    // the row's 8 negated multipliers as (al, be) parts, in pivot pairs (exchanged before any
    // divergence)
    float2 nal[4], nbe[4];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float xo = __shfl_xor_sync(FULL, x[q], 1);
      const float lr = part ? xo : x[q], li = part ? x[q] : xo;
      const float al = -(part ? li : lr), be = -(part ? lr : -li);
      if (q & 1) { nal[q >> 1].y = al; nbe[q >> 1].y = be; }
      else { nal[q >> 1].x = al; nbe[q >> 1].x = be; }
    }
    __syncthreads();
    // U12 = L11^{-1} A12: pivot row c8 right of the block minus its multipliers times the earlier ones
    if (t < lim - 8) {
      const int j = 8 + t;
      float ur[8], ui[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) { ur[q] = g.Pr[j][q]; ui[q] = g.Pi[j][q]; }
#pragma unroll
      for (int c8 = 1; c8 < 8; ++c8) {
#pragma unroll
        for (int q = 0; q < c8; ++q) {
          const float lr = g.Pr[q][c8], li = g.Pi[q][c8];  // multiplier of pivot c8 in column q
          ur[c8] -= lr * ur[q] - li * ui[q];
          ui[c8] -= lr * ui[q] + li * ur[q];
        }
      }
#pragma unroll
      for (int q = 1; q < 8; ++q) { g.Pr[j][q] = ur[q]; g.Pi[j][q] = ui[q]; }
    }
    __syncthreads();
    if (my_c8 >= 0) {  // the block's pivot rows take their corrected values
      const float(*src)[8] = part ? g.Pi : g.Pr;
#pragma unroll
      for (int jb = 1; jb < TB / 8; ++jb)
        if (8 * jb < lim) {
#pragma unroll
          for (int j = 8 * jb; j < 8 * jb + 8; ++j) x[j] = src[j][my_c8];
        }
    } else if (valid && !chosen) {  // A22 -= L21 U12: rank-8 update right of the block
#pragma unroll
      for (int jb = 1; jb < TB / 8; ++jb)
        if (8 * jb < lim) {
#pragma unroll
          for (int j = 8 * jb; j < 8 * jb + 8; ++j) {
            const float4* ur = reinterpret_cast<const float4*>(g.Pr[j]);
            const float4* ui = reinterpret_cast<const float4*>(g.Pi[j]);
            const float4 u0 = ur[0], u1 = ur[1], w0 = ui[0], w1 = ui[1];
            float2 acc = make_float2(x[j], 0.0f);
            acc = __ffma2_rn(nal[0], make_float2(u0.x, u0.y), acc);
            acc = __ffma2_rn(nal[1], make_float2(u0.z, u0.w), acc);
            acc = __ffma2_rn(nal[2], make_float2(u1.x, u1.y), acc);
            acc = __ffma2_rn(nal[3], make_float2(u1.z, u1.w), acc);
            acc = __ffma2_rn(nbe[0], make_float2(w0.x, w0.y), acc);
            acc = __ffma2_rn(nbe[1], make_float2(w0.z, w0.w), acc);
            acc = __ffma2_rn(nbe[2], make_float2(w1.x, w1.y), acc);
            acc = __ffma2_rn(nbe[3], make_float2(w1.z, w1.w), acc);
            x[j] = acc.x + acc.y;
          }
        }
    }
    // rotate left by 8: the next block's columns move to positions 0..7
    float tr[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) tr[j] = x[j];
#pragma unroll
    for (int j = 0; j < TB - 8; ++j) x[j] = x[j + 8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[TB - 8 + j] = tr[j];
  }
}

__device__ __forceinline__ void flag_bad(const LuArgs& a, int s, int code) {
  if (atomicCAS(&a.status[ST_ERR], DEV_OK, DEV_BADINDEX) == DEV_OK) {
    a.status[ST_DETAIL] = code;
    a.status[ST_SUB] = s;
  }
}

// ids[order] when order names a candidate position holding a row of the panel, else a flagged
// fallback (the first panel row) so that no later access leaves the matrix.
__device__ __forceinline__ int32_t pick_checked(const LuArgs& a, int s, const int32_t* ids, int order, int64_t R0,
                                                int64_t np, int code) {
  if (order >= 0 && order < RI_ROWS) {
    const int32_t r = ids[order];
    if (r >= R0 && r < np) return r;
  }
  flag_bad(a, s, code);
  return (int32_t)R0;
}

// one part (0: real, 1: imaginary) of matrix row `row` in tile column k
__device__ __forceinline__ void load_part_regs(void* arena, const LuArgs& a, int s, int32_t row, int part,
                                               float (&x)[TB]) {
  const float* T = tile_base<float>(arena, a, s, row / TB, a.k) + part * TILE_PLANE + (row % TB) * TB;
#pragma unroll
  for (int j = 0; j < TB; j += 4) {
    const float4 v = *(const float4*)(T + j);
    x[j] = v.x; x[j + 1] = v.y; x[j + 2] = v.z; x[j + 3] = v.w;
  }
}

__global__ void __launch_bounds__(RI_THREADS, 1) k_lu_tournament_ri(LuArgs a, void* arena) {
  constexpr int CH = RI_ROWS;  // one candidate row per thread pair
  static_assert(CH == LuCfg<float>::CH, "chunk rows");
  __shared__ RiGepp g;
  __shared__ int32_t ids[CH];
  __shared__ int32_t nids[TB];
  __shared__ int s_old;
  const int s = blockIdx.y, t = threadIdx.x, row = t >> 1, part = t & 1;
  const int64_t np = a.np[s], nts = np / TB;
  if (a.k >= nts) return;
  const int64_t R0 = (int64_t)a.k * TB;
  const int64_t rows_total = np - R0;
  const int nch = (int)((rows_total + CH - 1) / CH);
  int c = blockIdx.x;
  if (c >= nch) return;
  int64_t mrem = rows_total - (int64_t)c * CH;
  const int m = (int)(mrem < CH ? mrem : CH);
  float x[TB];
  int myrank;
  float mypiv;
  if (t < CH) ids[t] = t < m ? (int32_t)(R0 + (int64_t)c * CH + t) : -1;
  bool okrow = row < m;
  if (okrow) load_part_regs(arena, a, s, (int32_t)(R0 + (int64_t)c * CH + row), part, x);
  __syncthreads();
  int32_t* cand = a.cand + (int64_t)s * a.slots * TB;
  int32_t* cnt = a.cnt + (int64_t)s * a.slots;
  int level_off = 0, n_l = nch, j = c, code = 1;
  // leaf elimination, then one merge per level while this block arrives last at its parent
  for (;;) {
    gepp_ri(x, okrow, g, myrank, mypiv);
    if (t < TB) nids[t] = pick_checked(a, s, ids, g.order[t], R0, np, code);
    __syncthreads();
    if (n_l > 1 && t < TB) cand[(level_off + j) * TB + t] = nids[t];
    bool merge = false;
    while (n_l > 1) {  // 4-way tree: the last of up to four siblings to arrive merges them
      const int n_next = (n_l + 3) >> 2;
      const int parent = j >> 2, first = parent << 2;
      const int nsib = n_l - first < 4 ? n_l - first : 4;
      const int next_off = level_off + n_l;
      if (nsib == 1) {  // only child: pass the candidates up unchanged
        if (t < TB) cand[(next_off + parent) * TB + t] = nids[t];
        level_off = next_off; n_l = n_next; j = parent;
        continue;
      }
      __threadfence();
      __syncthreads();
      if (t == 0) s_old = atomicAdd(&cnt[next_off + parent], 1);
      __syncthreads();
      if (s_old != nsib - 1) return;  // a sibling still to arrive will merge
      if (t == 0) cnt[next_off + parent] = 0;
      __threadfence();
      if (t < CH) ids[t] = t < nsib * TB ? ((volatile int32_t*)cand)[(level_off + first + t / TB) * TB + (t % TB)] : -1;
      __syncthreads();
      okrow = row < nsib * TB && ids[row] >= R0 && ids[row] < np;
      if (part == 0 && row < nsib * TB && !okrow) flag_bad(a, s, 2);
      if (okrow) load_part_regs(arena, a, s, ids[row], part, x);
      level_off = next_off; n_l = n_next; j = parent;
      code = 3;
      merge = true;
      break;
    }
    if (!merge) break;  // this block holds the root's result
  }
  // root: the chosen rows, in pivot order, are L11\U11 of the step
  float* dg = reinterpret_cast<float*>((CT<float>*)a.diag + (int64_t)s * TB * TB);
  if (myrank >= 0) {
#pragma unroll
    for (int q = 0; q < TB; ++q) dg[2 * (q * TB + myrank) + part] = x[q];
    if (part == 0 && !(mypiv > 0.0f)) {
      atomicCAS(&a.status[ST_ERR], DEV_OK, DEV_SINGULAR);
      a.status[ST_SUB] = s;
    }
  }
  __syncthreads();
  if (t == 0) {
    int32_t posv[2 * TB], rowv[2 * TB];
    int nm = 0;
    auto row_at = [&](int32_t pos) {
      for (int q = 0; q < nm; ++q)
        if (posv[q] == pos) return rowv[q];
      return pos;
    };
    auto pos_of = [&](int32_t r) {
      for (int q = 0; q < nm; ++q)
        if (rowv[q] == r) return posv[q];
      return r;
    };
    auto set = [&](int32_t pos, int32_t r) {
      for (int q = 0; q < nm; ++q)
        if (posv[q] == pos) { rowv[q] = r; return; }
      posv[nm] = pos; rowv[nm] = r; ++nm;
    };
    for (int i = 0; i < TB; ++i) {
      int32_t tgt = (int32_t)(R0 + i);
      int32_t pr = pos_of(nids[i]);
      if (pr != tgt) {
        int32_t ra = row_at(tgt), rb = row_at(pr);
        set(tgt, rb);
        set(pr, ra);
      }
    }
    int32_t* pp = a.pairs + (int64_t)s * 2 * TB * 2;
    int np_ = 0;
    for (int q = 0; q < nm; ++q)
      if (posv[q] != rowv[q]) { pp[np_ * 2] = posv[q]; pp[np_ * 2 + 1] = rowv[q]; ++np_; }
    a.pairs_n[s] = np_;
  }
}

// Apply the step's row permutation to every column of the matrix and to perm.
template <typename R>
__global__ void k_lu_swap(LuArgs a, void* arena) {
  extern __shared__ unsigned char smem_raw[];
  CT<R>* buf = (CT<R>*)smem_raw;  // [2*TB][TB]
  const int s = blockIdx.y;
  const int64_t nts = a.np[s] / TB;
  if (a.k >= nts) return;
  const int J = blockIdx.x;
  if (J > nts) return;
  const int n = a.pairs_n[s];
  if (n == 0) return;
  const int32_t* pr = a.pairs + (int64_t)s * 2 * TB * 2;
  if (J == nts) {  // perm vector
    int32_t* perm = a.perm + a.np_off[s];
    __shared__ int32_t pv[2 * TB];
    for (int q = threadIdx.x; q < n; q += blockDim.x) pv[q] = perm[pr[q * 2 + 1]];
    __syncthreads();
    for (int q = threadIdx.x; q < n; q += blockDim.x) perm[pr[q * 2]] = pv[q];
    return;
  }
  for (int e = threadIdx.x; e < n * TB; e += blockDim.x) {
    int q = e / TB, j = e % TB;
    int32_t src = pr[q * 2 + 1];
    int64_t I = src / TB;
    buf[q * TB + j] = tload<R>(tile_base<R>(arena, a, s, I, J), tile_rowmajor(I, J), src % TB, j);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * TB; e += blockDim.x) {
    int q = e / TB, j = e % TB;
    int32_t dst = pr[q * 2];
    int64_t I = dst / TB;
    tstore<R>(tile_base<R>(arena, a, s, I, J), tile_rowmajor(I, J), dst % TB, j, buf[q * TB + j]);
  }
}

// blockIdx.x == 0: write the factored diagonal tile; 1..nrem: L tiles below; nrem+1..2 nrem: U tiles.
template <typename R>
__global__ void __launch_bounds__(TB) k_lu_trsm(LuArgs a, void* arena) {
  extern __shared__ unsigned char smem_raw[];
  CT<R>* D = (CT<R>*)smem_raw;       // [TB][PS] diagonal, column-major with padding
  CT<R>* X = D + TB * PS;            // [TB][PS] work tile, column-major with padding
  const int s = blockIdx.y;
  const int64_t nts = a.np[s] / TB;
  const int k = a.k;
  if (k >= nts) return;
  const int nrem = (int)(nts - k - 1);
  const int b = blockIdx.x;
  if (b > 2 * nrem) return;
  const CT<R>* dg = (const CT<R>*)a.diag + (int64_t)s * TB * TB;
  const int t = threadIdx.x;
  if (b == 0) {
    R* dst = tile_base<R>(arena, a, s, k, k);
    for (int e = t; e < TB * TB; e += blockDim.x) tstore<R>(dst, true, e % TB, e / TB, dg[e]);
    return;
  }
  for (int e = t; e < TB * TB; e += blockDim.x) D[(e / TB) * PS + (e % TB)] = dg[e];
  const bool lower = b <= nrem;
  const int64_t I = lower ? k + b : k, J = lower ? k : k + (b - nrem);
  const bool rm = tile_rowmajor(I, J);
  R* tp = tile_base<R>(arena, a, s, I, J);
  for (int e = t; e < TB * TB; e += blockDim.x) {
    int i = rm ? e / TB : e % TB, j = rm ? e % TB : e / TB;  // coalesced in storage order
    X[j * PS + i] = tload<R>(tp, rm, i, j);
  }
  __syncthreads();
  if (lower) {
    // row t of X: x U = a, forward over columns
    for (int j = 0; j < TB; ++j) {
      CT<R> acc = X[j * PS + t];
      for (int l = 0; l < j; ++l) acc = subc(acc, mulc(X[l * PS + t], D[j * PS + l]));
      X[j * PS + t] = mulc(acc, invc(D[j * PS + j]));
    }
  } else {
    // column t of X: L y = a, unit lower
    for (int i = 1; i < TB; ++i) {
      CT<R> acc = X[t * PS + i];
      for (int l = 0; l < i; ++l) acc = subc(acc, mulc(D[l * PS + i], X[t * PS + l]));
      X[t * PS + i] = acc;
    }
  }
  __syncthreads();
  for (int e = t; e < TB * TB; e += blockDim.x) {
    int i = rm ? e / TB : e % TB, j = rm ? e % TB : e / TB;
    tstore<R>(tp, rm, i, j, X[j * PS + i]);
  }
}

__device__ __forceinline__ bool region_tile(const UpdArgs& u, int64_t nts, int64_t e, int64_t& I, int64_t& J) {
  for (int q = 0; q < u.nreg; ++q) {
    int64_t i0 = u.reg[q].i0, i1 = u.reg[q].i1 == INT_MAX ? nts : u.reg[q].i1;
    int64_t j0 = u.reg[q].j0, j1 = u.reg[q].j1 == INT_MAX ? nts : u.reg[q].j1;
    if (i1 > nts) i1 = nts;
    if (j1 > nts) j1 = nts;
    int64_t ni = i1 > i0 ? i1 - i0 : 0, nj = j1 > j0 ? j1 - j0 : 0;
    if (e < ni * nj) {
      I = i0 + e / nj;
      J = j0 + e % nj;
      return true;
    }
    e -= ni * nj;
  }
  return false;
}

// C_IJ -= sum_{kk in [kk0, kk1)} L_I,kk U_kk,J over the update regions.  16x16 threads, each a
// 4x4 block of complex outputs; C is read and written once per launch.
template <typename R>
__global__ void __launch_bounds__(256) k_lu_update(LuArgs a, UpdArgs u, void* arena) {
  extern __shared__ unsigned char smem_raw[];
  CT<R>* As = (CT<R>*)smem_raw;  // [TB][TB]: A(i,l) at l*TB+i
  CT<R>* Bs = As + TB * TB;      // [TB][TB]: B(l,j) at l*TB+j
  const int s = blockIdx.y;
  const int64_t nts = a.np[s] / TB;
  int64_t I, J;
  if (!region_tile(u, nts, blockIdx.x, I, J)) return;
  const int t = threadIdx.x;
  const int ty = t / 16, tx = t % 16;
  CT<R> acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = {R(0), R(0)};
  for (int kk = u.kk0; kk < u.kk1 && kk < nts; ++kk) {
    const R* L = tile_base<R>(arena, a, s, I, kk);   // I > kk: row-major planes
    const R* U = tile_base<R>(arena, a, s, kk, J);   // kk < J: column-major planes
    __syncthreads();
    for (int e = t; e < TB * TB; e += 256) {
      int hi = e / TB, lo = e % TB;                    // storage order
      As[lo * TB + hi] = {L[e], L[TILE_PLANE + e]};    // L(i=hi, l=lo)
      Bs[lo * TB + hi] = {U[e], U[TILE_PLANE + e]};    // U(l=lo, j=hi)
    }
    __syncthreads();
    for (int l = 0; l < TB; ++l) {
      CT<R> av[4], bv[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) av[p] = As[l * TB + ty * 4 + p];
#pragma unroll
      for (int q = 0; q < 4; ++q) bv[q] = Bs[l * TB + tx * 4 + q];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[p][q].re += av[p].re * bv[q].re - av[p].im * bv[q].im;
          acc[p][q].im += av[p].re * bv[q].im + av[p].im * bv[q].re;
        }
    }
  }
  R* C = tile_base<R>(arena, a, s, I, J);
  const bool rm = tile_rowmajor(I, J);
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int i = ty * 4 + p, j = tx * 4 + q;
      CT<R> c = tload<R>(C, rm, i, j);
      tstore<R>(C, rm, i, j, {c.re - acc[p][q].re, c.im - acc[p][q].im});
    }
}

__global__ void k_iota_perm(int64_t total, int32_t* perm, const int64_t* np_off, int nsub) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  int lo = 0, hi = nsub - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (np_off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  perm[i] = (int32_t)(i - np_off[lo]);
}

// gidx[i] = N_s[perm[i]] for perm[i] < n_s, else -1 (padding)
__global__ void k_gidx(int64_t total, const int32_t* perm, const int64_t* np_off, const int64_t* ns,
                       const int64_t* ns_off, const int32_t* sub_dofs, int nsub, int32_t* gidx) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  int lo = 0, hi = nsub - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (np_off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  int32_t p = perm[i];
  gidx[i] = p < ns[lo] ? sub_dofs[ns_off[lo] + p] : -1;
}

// Inverses of the diagonal blocks of the factors: Linv_I = L_II^{-1} (unit lower) stored with
// row-major planes and Uinv_I = U_II^{-1} stored with column-major planes, so that the in-block
// substitution steps of the preconditioner apply become tile matrix-vector products like the
// off-diagonal ones (block substitution with inverted diagonal blocks).
// Inverts a factored diagonal block held column-major (padded) in D: X[0] gets the columns of
// L^{-1} (unit lower), X[1] those of U^{-1}.  Tasks [task0, task1) of the 2 TB columns (L's
// columns first), one warp per column in turn; lanes own rows lane and lane + 32; column-oriented
// substitution, the pivot entry broadcast by shuffle at each step, with the reciprocals of U's
// diagonal precomputed in rd:
//   L x = e_t:  x = e_t; for l = t .. TB-2:  x_i -= L(i,l) x_l  (i > l)
//   U x = e_j:  b = e_j; for l = j .. 0:     x_l = b_l rd_l;  b_i -= U(i,l) x_l  (i < l)
template <typename R>
__device__ void invert_block(const CT<R>* D, const CT<R>* rd, CT<R>* X, int task0, int task1) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int i0 = lane, i1 = lane + 32;
  for (int task = task0 + warp; task < task1; task += nw) {
    if (task < TB) {
      const int t = task;
      CT<R> x0 = {R(i0 == t ? 1 : 0), R(0)}, x1 = {R(i1 == t ? 1 : 0), R(0)};
      for (int l = t; l < TB - 1; ++l) {
        const CT<R> own = l < 32 ? x0 : x1;
        const CT<R> xl = {__shfl_sync(0xffffffffu, own.re, l & 31), __shfl_sync(0xffffffffu, own.im, l & 31)};
        if (i0 > l) x0 = subc(x0, mulc(D[l * PS + i0], xl));
        if (i1 > l) x1 = subc(x1, mulc(D[l * PS + i1], xl));
      }
      X[t * PS + i0] = x0;
      X[t * PS + i1] = x1;
    } else {
      const int j = task - TB;
      CT<R> b0 = {R(i0 == j ? 1 : 0), R(0)}, b1 = {R(i1 == j ? 1 : 0), R(0)};
      for (int l = j; l >= 0; --l) {
        const CT<R> own = l < 32 ? b0 : b1;
        const CT<R> bl = {__shfl_sync(0xffffffffu, own.re, l & 31), __shfl_sync(0xffffffffu, own.im, l & 31)};
        const CT<R> xl = mulc(bl, rd[l]);
        if (i0 < l) b0 = subc(b0, mulc(D[l * PS + i0], xl));
        else if (i0 == l) b0 = xl;
        if (i1 < l) b1 = subc(b1, mulc(D[l * PS + i1], xl));
        else if (i1 == l) b1 = xl;
      }
      X[TB * PS + j * PS + i0] = b0;
      X[TB * PS + j * PS + i1] = b1;
    }
  }
}

// Stores L^{-1} with row-major planes at Li and U^{-1} at Ui, with row-major planes when
// u_rowmajor (the preconditioner apply) or column-major planes (the B operand of the tensor-core
// tile solves, K-major along the row index).  A null pointer skips that factor.
template <typename R>
__device__ void store_inverses(const CT<R>* X, R* Li, R* Ui, bool u_rowmajor) {
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    const int hi = e / TB, lo = e % TB;
    if (Li) {
      const CT<R> l = X[lo * PS + hi];                // Linv(i = hi, j = lo): row-major storage
      Li[e] = l.re;
      Li[TILE_PLANE + e] = l.im;
    }
    if (Ui) {
      const CT<R> u = u_rowmajor ? X[TB * PS + lo * PS + hi]   // Uinv(i = hi, j = lo)
                                 : X[TB * PS + hi * PS + lo];  // Uinv(i = lo, j = hi)
      Ui[e] = u.re;
      Ui[TILE_PLANE + e] = u.im;
    }
  }
}

// reciprocals of the diagonal of the factored block in D
template <typename R>
__device__ __forceinline__ void diag_reciprocals(const CT<R>* D, CT<R>* rd) {
  if (threadIdx.x < TB) rd[threadIdx.x] = invc(D[threadIdx.x * PS + threadIdx.x]);
}

// Inverses of the diagonal blocks of the factors: Linv_I = L_II^{-1} (unit lower) and
// Uinv_I = U_II^{-1}, both stored with row-major planes, so that the in-block substitution steps of
// the preconditioner apply become tile matrix-vector products like the off-diagonal ones (block
// substitution with inverted diagonal blocks).
template <typename R>
__global__ void __launch_bounds__(INV_THREADS) k_lu_diag_inv(LuArgs a, void* arena, void* inv, const int64_t* inv_off) {
  extern __shared__ unsigned char smem_raw[];
  CT<R>* D = (CT<R>*)smem_raw;  // [TB][PS]: D[j*PS+i] = LU(i,j)
  CT<R>* X = D + TB * PS;       // [2][TB][PS]
  CT<R>* rd = X + 2 * TB * PS;  // [TB]
  const int s = blockIdx.y;
  const int64_t nts = a.np[s] / TB;
  const int64_t I = blockIdx.x;
  if (I >= nts) return;
  const R* T = tile_base<R>(arena, a, s, I, I);
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    int i = e / TB, j = e % TB;
    D[j * PS + i] = tload<R>(T, true, i, j);
  }
  __syncthreads();
  diag_reciprocals<R>(D, rd);
  __syncthreads();
  invert_block<R>(D, rd, X, 0, 2 * TB);
  __syncthreads();
  R* Li = (R*)inv + (inv_off[s] + I) * 4 * TILE_PLANE;
  store_inverses<R>(X, Li, Li + 2 * TILE_PLANE, true);
}

// After the factorisation: the tiles above the block diagonal (U), stored with column-major planes
// while the trailing updates read them as K-major operands, are transposed in place to row-major
// planes, so that every factor tile is row-major for the preconditioner apply (the tensor-core
// apply reads every tile as a K-major operand along its column index).  One block per upper tile
// x = J (J - 1) / 2 + I (I < J) of subdomain blockIdx.y.
template <typename R>
__global__ void __launch_bounds__(256) k_lu_upper_rowmajor(LuArgs a, void* arena) {
  extern __shared__ unsigned char smem_raw[];
  R* buf = (R*)smem_raw;  // [2][TB][TB + 1]
  const int s = blockIdx.y;
  const int64_t nts = a.np[s] / TB;
  const int64_t x = blockIdx.x;
  int64_t J = (int64_t)((1.0 + sqrt(1.0 + 8.0 * (double)x)) * 0.5);
  while (J * (J - 1) / 2 > x) --J;
  while ((J + 1) * J / 2 <= x) ++J;
  const int64_t I = x - J * (J - 1) / 2;
  if (J >= nts || I >= J) return;
  R* T = tile_base<R>(arena, a, s, I, J);
  for (int e = threadIdx.x; e < 2 * TB * TB; e += blockDim.x) {
    const int p = e / (TB * TB), q = e % (TB * TB);   // plane, column-major index j * TB + i
    buf[p * TB * (TB + 1) + (q / TB) * (TB + 1) + (q % TB)] = T[e];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * TB * TB; e += blockDim.x) {
    const int p = e / (TB * TB), q = e % (TB * TB);   // row-major index i * TB + j
    T[e] = buf[p * TB * (TB + 1) + (q % TB) * (TB + 1) + (q / TB)];
  }
}

// The step's factored diagonal block (from the tournament root): written to tile (k, k) and
// inverted into the subdomain's scratch tiles for the tensor-core triangular solves: L_kk^{-1}
// into slot `slot` (kept until the sub-panel's rows are solved beyond the panel), U_kk^{-1}
// into slot LU_SUB.  Two blocks per subdomain (blockIdx.x): 0 inverts L and writes the tile,
// 1 inverts U.
template <typename R>
__global__ void __launch_bounds__(INV_THREADS) k_lu_step_inv(LuArgs a, void* arena, int64_t scratch_base, int slot) {
  extern __shared__ unsigned char smem_raw[];
  CT<R>* D = (CT<R>*)smem_raw;  // [TB][PS]
  CT<R>* X = D + TB * PS;       // [2][TB][PS]
  CT<R>* rd = X + 2 * TB * PS;  // [TB]
  const int s = blockIdx.y, half = blockIdx.x;
  const int64_t nts = a.np[s] / TB;
  const int k = a.k;
  if (k >= nts) return;
  const CT<R>* dg = (const CT<R>*)a.diag + (int64_t)s * TB * TB;  // element (e % TB, e / TB)
  R* dst = tile_base<R>(arena, a, s, k, k);
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    const CT<R> v = dg[e];
    D[(e / TB) * PS + (e % TB)] = v;
    if (half == 0) tstore<R>(dst, true, e % TB, e / TB, v);
  }
  __syncthreads();
  if (half == 1) diag_reciprocals<R>(D, rd);
  __syncthreads();
  invert_block<R>(D, rd, X, half * TB, (half + 1) * TB);
  __syncthreads();
  R* Li = (R*)arena + (scratch_base + (int64_t)LU_SCRATCH * s + slot) * 2 * TILE_PLANE;
  R* Ui = (R*)arena + (scratch_base + (int64_t)LU_SCRATCH * s + LU_SUB) * 2 * TILE_PLANE;
  store_inverses<R>(X, half == 0 ? Li : nullptr, half == 1 ? Ui : nullptr, false);
}

// number of output tiles of the update regions for the largest subdomain
static int64_t region_blocks(const UpdArgs& u, int64_t nts) {
  int64_t tot = 0;
  for (int q = 0; q < u.nreg; ++q) {
    int64_t i1 = u.reg[q].i1 == INT_MAX ? nts : std::min<int64_t>(u.reg[q].i1, nts);
    int64_t j1 = u.reg[q].j1 == INT_MAX ? nts : std::min<int64_t>(u.reg[q].j1, nts);
    int64_t ni = std::max<int64_t>(0, i1 - u.reg[q].i0), nj = std::max<int64_t>(0, j1 - u.reg[q].j0);
    tot += ni * nj;
  }
  return tot;
}


template <typename R>
static int lu_run(oras_handle* h) {
  auto& m = h->mesh;
  auto& d = h->dev;
  constexpr int CH = LuCfg<R>::CH;
  LuArgs a;
  a.nsub = m.nsub;
  a.np = d.sub_np;
  a.tile_off = d.sub_tile_off;
  a.np_off = d.sub_np_off;
  a.perm = d.perm;
  a.cand = d.lu_cand;
  a.cnt = d.lu_cnt;
  a.slots = 2 * d.lu_max_chunks + 16;
  a.pairs = d.lu_ipiv;
  a.pairs_n = d.lu_ipiv + (int64_t)m.nsub * 2 * TB * 2;
  a.diag = d.lu_diag;
  a.status = d.status;
  int64_t total = 0;
  for (int s = 0; s < m.nsub; ++s) total += m.sub_np[s];
  k_iota_perm<<<(unsigned)((total + 255) / 256), 256, 0, d.stream>>>(total, d.perm, d.sub_np_off, m.nsub);
  const int max_nts = (int)(m.max_np / TB);
  size_t smem_t = (size_t)CH * PS * sizeof(CT<R>) + CH * sizeof(int32_t) + 32 * sizeof(R) + 32 * sizeof(int);
  size_t smem_s = (size_t)2 * TB * TB * sizeof(CT<R>);
  size_t smem_r = (size_t)2 * TB * PS * sizeof(CT<R>);
  size_t smem_u = (size_t)2 * TB * TB * sizeof(CT<R>);
  allow_max_smem((const void*)k_lu_tournament<R>);
  allow_max_smem((const void*)k_lu_swap<R>);
  allow_max_smem((const void*)k_lu_trsm<R>);
  allow_max_smem((const void*)k_lu_update<R>);
  const size_t smem_i = ((size_t)3 * TB * PS + TB) * sizeof(CT<R>);
  allow_max_smem((const void*)k_lu_step_inv<R>);
  const bool tc = sizeof(R) == 4 && h->opt.lu_engine == ORAS_LU_AUTO && tc_update_available(h);
  auto update = [&](const UpdArgs& u, int cls) {
    if (tc) {
      launch_update_tc(h, u, max_nts, cls);
      return;
    }
    int64_t blocks = region_blocks(u, max_nts);
    if (blocks <= 0) return;
    int pb = prof_begin(h);
    k_lu_update<R><<<dim3((unsigned)blocks, m.nsub), 256, smem_u, d.stream>>>(a, u, d.arena);
    prof_end(h, cls, pb, 1);
    count_launches(1);
  };
  const int W = h->opt.lu_panel > 0 ? h->opt.lu_panel : 8;  // outer panel width in tile columns
  auto panel_update = [&](int kk0, int kk1, Region r) {
    UpdArgs u;
    u.kk0 = kk0;
    u.kk1 = kk1;
    u.nreg = 1;
    u.reg[0] = r;
    update(u, KC_LU_PANEL);
  };
  for (int k0 = 0; k0 < max_nts; k0 += W) {
    const int kend = k0 + W;
    for (int k = k0; k < kend && k < max_nts; ++k) {
      a.k = k;
      int64_t rows_max = m.max_np - (int64_t)k * TB;
      int nch = (int)((rows_max + CH - 1) / CH);
      int64_t nrem = max_nts - k - 1;
      const int k1 = k0 + (k - k0) / LU_SUB * LU_SUB;                    // first step of the sub-panel
      const int ks = std::min(std::min(k1 + LU_SUB, kend), max_nts);     // first step after it
      if (tc && k == k1 && k1 > k0) {
        // sub-panel start (tensor-core path): its columns, for every row from k1 down, receive
        // the updates of the panel's earlier sub-panels in one contraction
        panel_update(k0, k1, {k1, INT_MAX, k1, ks});
      }
      if (k > k1) {
        // left-looking sub-panel step: column k, on and below the diagonal, receives the updates
        // of the sub-panel's earlier steps just before its pivot search (every row there is in
        // the same state, so the row interchanges stay consistent)
        panel_update(k1, k, {k, INT_MAX, k, k + 1});
      }
      int pb = prof_begin(h);
      if (sizeof(R) == 4)
        k_lu_tournament_ri<<<dim3(nch, m.nsub), RI_THREADS, 0, d.stream>>>(a, d.arena);
      else
        k_lu_tournament<R><<<dim3(nch, m.nsub), LU_THREADS, smem_t, d.stream>>>(a, d.arena);
      prof_end(h, KC_LU_TOURNAMENT, pb, 1);
      pb = prof_begin(h);
      k_lu_swap<R><<<dim3(max_nts + 1, m.nsub), 256, smem_s, d.stream>>>(a, d.arena);
      prof_end(h, KC_LU_SWAP, pb, 1);
      // the pivot tile row right of column k: the rows below keep updates deferred, so a pivot
      // row swapped up from there receives them now.  Tensor-core path: inside the sub-panel from
      // its earlier steps (the rest of the row is solved with the sub-panel's other rows after
      // its last step).  CUDA-core path: inside the panel from the sub-panel's earlier steps
      // (earlier sub-panels reached it through their mid updates), beyond the panel from all the
      // panel's earlier steps.
      if (tc) {
        if (k > k1 && k + 1 < ks) panel_update(k1, k, {k, k + 1, k + 1, ks});
      } else if (k > k0) {
        if (k1 == k0) {
          panel_update(k0, k, {k, k + 1, k + 1, INT_MAX});
        } else {
          if (k > k1) panel_update(k1, k, {k, k + 1, k + 1, kend});
          panel_update(k0, k, {k, k + 1, kend, INT_MAX});
        }
      }
      pb = prof_begin(h);
      if (tc) {
        k_lu_step_inv<R><<<dim3(2, m.nsub), INV_THREADS, smem_i, d.stream>>>(a, d.arena, m.arena_tiles, k - k1);
        launch_trsm_tc(h, k, max_nts, true, k + 1, ks, k - k1);
        prof_end(h, KC_LU_TRSM, pb, 2);
      } else {
        k_lu_trsm<R><<<dim3((unsigned)(2 * nrem + 1), m.nsub), TB, smem_r, d.stream>>>(a, d.arena);
        prof_end(h, KC_LU_TRSM, pb, 1);
      }
      count_launches(3);
      const int kb = k + 1;
      if (kb == ks) {  // the sub-panel's last step
        if (tc && kb < max_nts) {
          // the sub-panel's rows right of it (a blocked triangular solve with the panel's L):
          // first the contributions of the panel's earlier sub-panels in one product, then row by
          // row those of the sub-panel's earlier rows and the solve with L_rr^{-1}
          if (k1 > k0) panel_update(k0, k1, {k1, kb, kb, INT_MAX});
          for (int r = k1; r < kb; ++r) {
            if (r > k1) panel_update(k1, r, {r, r + 1, kb, INT_MAX});
            pb = prof_begin(h);
            launch_trsm_tc(h, r, max_nts, false, kb, INT_MAX, r - k1);
            prof_end(h, KC_LU_TRSM, pb, 1);
          }
        }
        if (!tc && kb < kend && kb < max_nts) {
          // mid update (CUDA-core path): the panel's later columns, for every row below the
          // sub-panel, from the sub-panel's steps
          panel_update(k1, kb, {kb, INT_MAX, kb, kend});
        }
      }
    }
    UpdArgs u;  // outer update of the trailing matrix
    u.kk0 = k0;
    u.kk1 = kend;
    u.nreg = 1;
    u.reg[0] = {kend, INT_MAX, kend, INT_MAX};
    update(u, KC_LU_UPDATE);
  }
  k_gidx<<<(unsigned)((total + 255) / 256), 256, 0, d.stream>>>(total, d.perm, d.sub_np_off, d.sub_ns,
                                                              d.sub_ns_off, d.sub_dofs, m.nsub, d.gidx);
  if (max_nts > 1) {
    const size_t smem_t2 = (size_t)2 * TB * (TB + 1) * sizeof(R);
    allow_max_smem((const void*)k_lu_upper_rowmajor<R>);
    const int64_t upper = (int64_t)max_nts * (max_nts - 1) / 2;
    int pb = prof_begin(h);
    k_lu_upper_rowmajor<R><<<dim3((unsigned)upper, m.nsub), 256, smem_t2, d.stream>>>(a, d.arena);
    prof_end(h, KC_LU_SWAP, pb, 1);
    count_launches(1);
  }
  {
    allow_max_smem((const void*)k_lu_diag_inv<R>);
    int pb = prof_begin(h);
    k_lu_diag_inv<R><<<dim3(max_nts, m.nsub), INV_THREADS, smem_i, d.stream>>>(a, d.arena, d.dinv, d.sub_inv_off);
    prof_end(h, KC_LU_TRSM, pb, 1);
  }
  count_launches(3);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_lu(oras_handle* h) { return h->dev.factor_bits == 64 ? lu_run<double>(h) : lu_run<float>(h); }

int lu_max_chunks(int64_t max_np, int factor_bits) {
  int ch = factor_bits == 64 ? LuCfg<double>::CH : LuCfg<float>::CH;
  return (int)((max_np + ch - 1) / ch);
}

}  // namespace oras
