// Device body of the ORAS preconditioner apply for one subdomain (Sec. 4):
//   y = P_s R_s v ;  y = L_s^{-1} y ;  y = U_s^{-1} y ;  z += R_s^T D_s y
// Block substitution over the tiled factor arena (split re/im planes; tiles on/below the block
// diagonal row-major, above it column-major) with inverted diagonal blocks, so every step is a
// TB x TB tile times a TB-vector.
//
// A cluster of two CTAs works on one subdomain.  CTA c owns the block rows (strips) I with
// I % 2 == c: it keeps their entries of y in its shared memory and streams the tiles of the
// block columns J with J % 2 == c.  For every strip both CTAs form partial sums over their own
// block columns; the non-owner sends its 64 partial sums into the owner's shared memory
// (distributed shared memory, mbarrier with cluster-scope release/acquire) and the owner
// applies the inverted diagonal block.  Tiles stream through a ring of shared-memory stages
// filled by 1-D bulk TMA copies from one producer warp; eight consumer warps compute.
// Every wait is bounded (about 2 s); a timeout sets the device status flag and the block
// finishes without further work.
#pragma once

#include "dev.cuh"

namespace oras {

struct ApplyGeom {
  const int64_t* ns; const int64_t* np; const int64_t* np_off; const int64_t* ns_off;
  const int64_t* tile_off; const int64_t* inv_off;
  const int32_t* gidx; const int32_t* sub_dofs; const uint8_t* pou;
  const void* arena; const void* dinv;
  int weights;
  int stages;               // ring depth
  int32_t* status;
};

constexpr int APPLY_CONSUMERS = 256;            // 8 warps
constexpr int APPLY_THREADS = APPLY_CONSUMERS + 32;

__device__ __forceinline__ void z_store(cplx* z, double re, double im) { *z = {re, im}; }
__device__ __forceinline__ void z_store(CT<float>* z, double re, double im) { *z = {(float)re, (float)im}; }
__device__ __forceinline__ void z_add(cplx* z, double re, double im) {
  atomicAdd(&z->re, re);
  atomicAdd(&z->im, im);
}
__device__ __forceinline__ void z_add(CT<float>* z, double re, double im) {
  atomicAdd(&z->re, (float)re);
  atomicAdd(&z->im, (float)im);
}

template <typename R> __host__ __device__ constexpr uint32_t tile_bytes() { return (uint32_t)(2 * TB * TB * sizeof(R)); }

// Shared-memory layout of one CTA (dynamic part), given the ring depth and the number of
// owned strips kept in shared memory (0 when y lives in global memory).
template <typename R>
struct ApplySmem {
  static __host__ __device__ size_t ring_off() { return 0; }
  static __host__ __device__ size_t bar_off(int S) { return (size_t)S * tile_bytes<R>(); }
  static __host__ __device__ size_t recv_off(int S) { return bar_off(S) + (2 * S + 2) * 8; }
  static __host__ __device__ size_t red_off(int S) { return recv_off(S) + 2 * TB * sizeof(CT<R>); }
  static __host__ __device__ size_t rvec_off(int S) { return red_off(S) + 8 * TB * sizeof(CT<R>); }
  static __host__ __device__ size_t y_off(int S) { return rvec_off(S) + TB * sizeof(CT<R>); }
  static __host__ __device__ size_t total(int S, int64_t ystrips) {
    return y_off(S) + (size_t)ystrips * TB * sizeof(CT<R>);
  }
};

// Strip sequence helpers: the tiles CTA c streams for strip I (forward: J < I, backward: J > I,
// J % 2 == c), followed by the strip's inverted diagonal block when c owns the strip.
template <typename R, typename ZT>
__device__ void apply_cluster(const ApplyGeom& a, int s, const cplx* __restrict__ v, int64_t vs,
                              ZT* __restrict__ z, int64_t zs, int64_t off, CT<R>* yglob) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int S = a.stages;
  unsigned char* ring = smem_raw + ApplySmem<R>::ring_off();
  uint64_t* full = (uint64_t*)(smem_raw + ApplySmem<R>::bar_off(S));
  uint64_t* empty = full + S;
  uint64_t* msg = empty + S;                                     // [2]
  CT<R>* recv = (CT<R>*)(smem_raw + ApplySmem<R>::recv_off(S));  // [2][TB]
  CT<R>(*red)[TB] = (CT<R>(*)[TB])(smem_raw + ApplySmem<R>::red_off(S));
  CT<R>* rvec = (CT<R>*)(smem_raw + ApplySmem<R>::rvec_off(S));
  __shared__ int abort_flag;
  const int c = (int)cluster_rank();
  const int64_t ns = a.ns[s], np = a.np[s], nts = np / TB;
  const int64_t own0 = (nts + 1) / 2;                   // strips owned by CTA 0
  CT<R>* y = yglob ? yglob + a.np_off[s] + (c ? own0 * TB : 0)
                   : (CT<R>*)(smem_raw + ApplySmem<R>::y_off(S));
  const R* F = (const R*)a.arena + a.tile_off[s] * 2 * TILE_PLANE;
  const R* Dinv = (const R*)a.dinv + a.inv_off[s] * 4 * TILE_PLANE;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr uint32_t TBYTES = tile_bytes<R>();
  if (tid == 0) {
    for (int q = 0; q < S; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], APPLY_CONSUMERS / 32);
    }
    mbar_init(&msg[0], 1);
    mbar_init(&msg[1], 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  cluster_sync_all();  // the partner may signal our barriers from here on

  if (warp == APPLY_CONSUMERS / 32) {
    // ---------------- producer: one lane issues the bulk copies in consumption order
    if (lane == 0) {
      int64_t n = 0;
      auto issue = [&](const R* src) -> bool {
        const int slot = (int)(n % S);
        if (n >= S && !mbar_wait(&empty[slot], (uint32_t)(((n / S) - 1) & 1))) return false;
        mbar_expect_tx(&full[slot], TBYTES);
        bulk_g2s(ring + (size_t)slot * TBYTES, src, TBYTES, &full[slot]);
        ++n;
        return true;
      };
      bool ok = true;
      for (int64_t I = 0; I < nts && ok; ++I) {
        for (int64_t J = c; J < I && ok; J += 2) ok = issue(F + (I * nts + J) * 2 * TILE_PLANE);
        if (ok && (I & 1) == c) ok = issue(Dinv + I * 4 * TILE_PLANE);
      }
      for (int64_t I = nts - 1; I >= 0 && ok; --I) {
        for (int64_t J = I + 1 + ((I + 1 + c) & 1); J < nts && ok; J += 2) ok = issue(F + (I * nts + J) * 2 * TILE_PLANE);
        if (ok && (I & 1) == c) ok = issue(Dinv + I * 4 * TILE_PLANE + 2 * TILE_PLANE);
      }
      if (!ok) {
        atomicExch(&a.status[ST_ERR], DEV_TIMEOUT);
        abort_flag = 1;
      }
      // drain: every issued copy must land before the block may exit
      for (int64_t q = n > S ? n - S : 0; q < n; ++q) mbar_wait(&full[q % S], (uint32_t)((q / S) & 1));
    }
  } else {
    // ---------------- consumers
    const uint32_t partner = (uint32_t)(c ^ 1);
    int64_t n = 0;
    int kr = 0, ks = 0;  // messages received / sent
    bool ok = true;
    auto stage = [&](const R*& T) -> bool {
      const int slot = (int)(n % S);
      if (!mbar_wait(&full[slot], (uint32_t)((n / S) & 1))) return false;
      T = (const R*)(ring + (size_t)slot * TBYTES);
      return true;
    };
    auto release = [&]() {
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[(int)(n % S)]);
      ++n;
    };
    // gather the owned strips: y(local) = P_s R_s v
    for (int64_t q = tid; q < (c ? nts - own0 : own0) * TB; q += APPLY_CONSUMERS) {
      const int64_t I = 2 * (q / TB) + c, pos = I * TB + q % TB;
      const int32_t g = a.gidx[a.np_off[s] + pos];
      const cplx val = g >= 0 ? v[(int64_t)g * vs + off] : cplx{0.0, 0.0};
      y[q] = {R(val.re), R(val.im)};
    }
    named_sync(1, APPLY_CONSUMERS);
    for (int pass = 0; pass < 2; ++pass) {
      const bool fwd = pass == 0;
      for (int64_t it = 0; it < nts; ++it) {
        const int64_t I = fwd ? it : nts - 1 - it;
        const bool owner = (I & 1) == c;
        // partial sums over the owned block columns of strip I
        CT<R> acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = {R(0), R(0)};
        const int64_t J0 = fwd ? c : I + 1 + ((I + 1 + c) & 1), J1 = fwd ? I : nts;
        for (int64_t J = J0; J < J1; J += 2) {
          const R* T = nullptr;
          if (ok) ok = stage(T);
          if (!ok) continue;  // keep the barrier sequence uniform; no more work after a timeout
          const CT<R>* yJ = y + (J / 2) * TB;
          if (fwd) {  // row-major tile: warp rows 8w..8w+7, lane columns 2l, 2l+1
            const CT<R> y0 = yJ[2 * lane], y1 = yJ[2 * lane + 1];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int e = (warp * 8 + q) * TB + 2 * lane;
              const R r0 = T[e], r1 = T[e + 1], i0 = T[TILE_PLANE + e], i1 = T[TILE_PLANE + e + 1];
              acc[q].re += r0 * y0.re - i0 * y0.im + r1 * y1.re - i1 * y1.im;
              acc[q].im += r0 * y0.im + i0 * y0.re + r1 * y1.im + i1 * y1.re;
            }
          } else {  // column-major tile: warp columns 8w..8w+7, lane rows 2l, 2l+1
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int col = warp * 8 + q;
              const CT<R> yc = yJ[col];
              const int e = col * TB + 2 * lane;
              const R r0 = T[e], r1 = T[e + 1], i0 = T[TILE_PLANE + e], i1 = T[TILE_PLANE + e + 1];
              acc[2 * (q & 3)].re += r0 * yc.re - i0 * yc.im;   // rows 2l (even slots) and 2l+1 (odd)
              acc[2 * (q & 3)].im += r0 * yc.im + i0 * yc.re;
              acc[2 * (q & 3) + 1].re += r1 * yc.re - i1 * yc.im;
              acc[2 * (q & 3) + 1].im += r1 * yc.im + i1 * yc.re;
            }
          }
          release();
        }
        // reduce to 64 partial sums in red[0][*]
        if (fwd) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            for (int o = 16; o > 0; o >>= 1) {
              acc[q].re += __shfl_down_sync(0xffffffffu, acc[q].re, o);
              acc[q].im += __shfl_down_sync(0xffffffffu, acc[q].im, o);
            }
            if (lane == 0) red[0][warp * 8 + q] = acc[q];
          }
          named_sync(1, APPLY_CONSUMERS);
        } else {
          CT<R> p0 = {R(0), R(0)}, p1 = {R(0), R(0)};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            p0.re += acc[2 * q].re; p0.im += acc[2 * q].im;
            p1.re += acc[2 * q + 1].re; p1.im += acc[2 * q + 1].im;
          }
          red[warp][2 * lane] = p0;
          red[warp][2 * lane + 1] = p1;
          named_sync(1, APPLY_CONSUMERS);
          if (tid < TB) {
            CT<R> t = red[0][tid];
            for (int w = 1; w < 8; ++w) { t.re += red[w][tid].re; t.im += red[w][tid].im; }
            rvec[tid] = t;
          }
          named_sync(1, APPLY_CONSUMERS);
          if (tid < TB) red[0][tid] = rvec[tid];
          named_sync(1, APPLY_CONSUMERS);
        }
        if (!owner) {
          // send the partial sums to the owner's receive buffer, then signal it
          if (tid < TB) {
            const uint32_t dst = map_to_rank(&recv[(ks & 1) * TB + tid], partner);
            st_remote(dst, red[0][tid].re, red[0][tid].im);
          }
          named_sync(1, APPLY_CONSUMERS);
          if (tid == 0) mbar_arrive_remote(map_to_rank(&msg[ks & 1], partner));
          ++ks;
          continue;
        }
        // owner: r = b_I - own partial - partner partial
        if (tid == 0 && !mbar_wait(&msg[kr & 1], (uint32_t)((kr >> 1) & 1), true)) {
          atomicExch(&a.status[ST_ERR], DEV_TIMEOUT);
          abort_flag = 1;
        }
        named_sync(1, APPLY_CONSUMERS);
        if (abort_flag) ok = false;
        CT<R>* yI = y + (I / 2) * TB;
        if (tid < TB) {
          const CT<R> pr = recv[(kr & 1) * TB + tid];
          rvec[tid] = {yI[tid].re - red[0][tid].re - pr.re, yI[tid].im - red[0][tid].im - pr.im};
        }
        ++kr;
        named_sync(1, APPLY_CONSUMERS);
        // y_I = inv(diag block) r
        const R* T = nullptr;
        if (ok) ok = stage(T);
        if (!ok) {
          named_sync(1, APPLY_CONSUMERS);
          if (!fwd) named_sync(1, APPLY_CONSUMERS);
          continue;
        }
        if (fwd) {  // Linv, row-major
          const CT<R> r0v = rvec[2 * lane], r1v = rvec[2 * lane + 1];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int e = (warp * 8 + q) * TB + 2 * lane;
            const R r0 = T[e], r1 = T[e + 1], i0 = T[TILE_PLANE + e], i1 = T[TILE_PLANE + e + 1];
            CT<R> t = {r0 * r0v.re - i0 * r0v.im + r1 * r1v.re - i1 * r1v.im,
                       r0 * r0v.im + i0 * r0v.re + r1 * r1v.im + i1 * r1v.re};
            for (int o = 16; o > 0; o >>= 1) {
              t.re += __shfl_down_sync(0xffffffffu, t.re, o);
              t.im += __shfl_down_sync(0xffffffffu, t.im, o);
            }
            if (lane == 0) yI[warp * 8 + q] = t;
          }
          release();
        } else {  // Uinv, column-major
          CT<R> p0 = {R(0), R(0)}, p1 = {R(0), R(0)};
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int col = warp * 8 + q;
            const CT<R> rc = rvec[col];
            const int e = col * TB + 2 * lane;
            const R r0 = T[e], r1 = T[e + 1], i0 = T[TILE_PLANE + e], i1 = T[TILE_PLANE + e + 1];
            p0.re += r0 * rc.re - i0 * rc.im;
            p0.im += r0 * rc.im + i0 * rc.re;
            p1.re += r1 * rc.re - i1 * rc.im;
            p1.im += r1 * rc.im + i1 * rc.re;
          }
          release();
          red[warp][2 * lane] = p0;
          red[warp][2 * lane + 1] = p1;
          named_sync(1, APPLY_CONSUMERS);
          if (tid < TB) {
            CT<R> t = red[0][tid];
            for (int w = 1; w < 8; ++w) { t.re += red[w][tid].re; t.im += red[w][tid].im; }
            yI[tid] = t;
          }
        }
        named_sync(1, APPLY_CONSUMERS);
      }
    }
    if (!ok) {
      if (tid == 0) {
        atomicExch(&a.status[ST_ERR], DEV_TIMEOUT);
        abort_flag = 1;
      }
    } else {
      // scatter the owned strips with the partition of unity
      const int32_t* Ns = a.sub_dofs + a.ns_off[s];
      const uint8_t* Dp = a.pou + a.ns_off[s];
      for (int64_t q = tid; q < (c ? nts - own0 : own0) * TB; q += APPLY_CONSUMERS) {
        const int64_t pos = (2 * (q / TB) + c) * TB + q % TB;
        if (pos >= ns) continue;
        const CT<R> val = y[q];
        ZT* dst = z + (int64_t)Ns[pos] * zs + off;
        if (a.weights == ORAS_WEIGHTS_POU) {
          if (Dp[pos]) z_store(dst, (double)val.re, (double)val.im);
        } else {
          z_add(dst, (double)val.re, (double)val.im);
        }
      }
    }
  }
  __syncthreads();
  cluster_sync_all();  // the partner must not touch our shared memory after we exit
}

}  // namespace oras
