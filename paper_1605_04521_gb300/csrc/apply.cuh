// Device body of the ORAS preconditioner apply for one subdomain (Sec. 4):
//   y = P_s R_s v ;  y = L_s^{-1} y ;  y = U_s^{-1} y ;  z += R_s^T D_s y
// Block substitution over the tiled factor arena (split re/im planes, every tile row-major once the
// factorisation has finished) with inverted diagonal blocks, so every step is a TB x TB tile times a
// TB x KR block of KR right-hand sides: warp w takes rows 8w..8w+7, lane l the column pair 2l, 2l+1.  One pass over the arena serves all
// KR right-hand sides: the factor bytes are read once per group, not once per vector.
//
// A cluster of G CTAs (2, or 4 for the largest subdomains of a launch that leaves SMs idle) works
// on one subdomain.  CTA c owns the block rows (strips) I with I % G == c: it keeps their entries
// of y (shared memory, or a global slice when they do not fit) and streams the tiles of the block
// columns J with J % G == c, which are exactly its own strips.  For every strip all G CTAs form
// partial sums over their own block columns; the G - 1 non-owners send their TB x KR partial sums
// into their slots of the owner's shared memory (distributed shared memory, an mbarrier that
// counts G - 1 cluster-scope release arrivals) and the owner applies the inverted diagonal
// block.  Tiles stream through a ring of shared-memory stages filled by 1-D bulk TMA
// copies from one producer warp; eight consumer warps compute.  When y lives in global memory,
// every stage also carries the TB x KR slice y_J its tile multiplies: the producer copies it once
// the consumers have finalised strip J (a shared counter, with a proxy fence on the writer side),
// so the consumers never wait on a global load.  Every wait is bounded (ApplyGeom::wait_ns, 2 s
// by default); a timeout sets the device status flag and the block finishes without further
// work, after waiting (at least 2 s) for its own bulk copies still in flight.  apply_cluster
// returns whether any CTA of the cluster gave up, the same value in all.
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
  uint64_t wait_ns;         // limit of every bounded wait
};

constexpr int APPLY_CONSUMERS = 256;            // 8 warps
constexpr int APPLY_THREADS = APPLY_CONSUMERS + 32;
constexpr int APPLY_MAX_KR_F32 = 4;             // right-hand sides per arena pass, FP32 factors
                                                // (9 warps leave 168 registers a thread; 8 spills)
constexpr int APPLY_MAX_KR_F64 = 2;             // FP64 factors (register budget)

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

// Two adjacent plane entries as one vector load.
__device__ __forceinline__ void ld_pair(const float* p, float& a, float& b) {
  const float2 t = *reinterpret_cast<const float2*>(p);
  a = t.x; b = t.y;
}
__device__ __forceinline__ void ld_pair(const double* p, double& a, double& b) {
  const double2 t = *reinterpret_cast<const double2*>(p);
  a = t.x; b = t.y;
}

// Two adjacent complex entries (16 B for FP32, 32 B for FP64) as vector accesses.
__device__ __forceinline__ void ld_cpair(const CT<float>* p, CT<float>& a, CT<float>& b) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  a = {t.x, t.y}; b = {t.z, t.w};
}
__device__ __forceinline__ void ld_cpair(const CT<double>* p, CT<double>& a, CT<double>& b) {
  const double2 t0 = reinterpret_cast<const double2*>(p)[0], t1 = reinterpret_cast<const double2*>(p)[1];
  a = {t0.x, t0.y}; b = {t1.x, t1.y};
}
__device__ __forceinline__ void st_cpair(CT<float>* p, CT<float> a, CT<float> b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.re, a.im, b.re, b.im);
}
__device__ __forceinline__ void st_cpair(CT<double>* p, CT<double> a, CT<double> b) {
  reinterpret_cast<double2*>(p)[0] = make_double2(a.re, a.im);
  reinterpret_cast<double2*>(p)[1] = make_double2(b.re, b.im);
}

// Shared-memory layout of one CTA (dynamic part), given the ring depth, the number of
// right-hand sides per pass and the number of owned strips kept in shared memory (0 when y
// lives in global memory).  All TB x KR blocks are stored [KR][TB] (one 64-entry column per
// right-hand side), so a lane's pair of rows is contiguous for every right-hand side.
template <typename R, int KR, int G>
struct ApplySmem {
  static constexpr size_t C = sizeof(CT<R>);
  static constexpr uint32_t YB = TB * KR * sizeof(CT<R>);  // y slice staged beside a tile
  // ystrips > 0: y resident in shared memory; 0: y in global memory, staged through the ring
  static __host__ __device__ uint32_t slot(int64_t ystrips) { return tile_bytes<R>() + (ystrips ? 0u : YB); }
  static __host__ __device__ size_t bar_off(int S, int64_t ys) { return (size_t)S * slot(ys); }
  static __host__ __device__ size_t recv_off(int S, int64_t ys) { return bar_off(S, ys) + (size_t)(2 * S + 2) * 8; }
  // receive buffers: [2 (strip parity at the owner)][G - 1 (sender slot)][TB x KR]
  static __host__ __device__ size_t part_off(int S, int64_t ys) { return recv_off(S, ys) + 2 * (G - 1) * TB * KR * C; }
  static __host__ __device__ size_t rvec_off(int S, int64_t ys) { return part_off(S, ys) + TB * KR * C; }
  static __host__ __device__ size_t y_off(int S, int64_t ys) { return rvec_off(S, ys) + TB * KR * C; }
  static __host__ __device__ size_t total(int S, int64_t ys) { return y_off(S, ys) + (size_t)ys * TB * KR * C; }
};

// v and z are [N][vs] / [N][zs] complex arrays; this pass handles right-hand sides off .. off+nr-1
// (nr <= KR; the unused lanes of the last group carry zeros and are not stored).
// The first block column right of strip I among the columns J % G == c of CTA c (G a power of
// two, so the mask is the remainder also for negative differences).
template <int G>
__device__ __forceinline__ int64_t first_right(int64_t I, int c) {
  static_assert((G & (G - 1)) == 0, "G a power of two");
  return I + 1 + (((int64_t)c - (I + 1)) & (G - 1));
}

template <typename R, typename ZT, int KR, int G>
__device__ bool apply_cluster(const ApplyGeom& a, int s, const cplx* __restrict__ v, int64_t vs,
                              ZT* __restrict__ z, int64_t zs, int64_t off, int nr, CT<R>* yglob) {
  static_assert(G == 2 || G == 4, "CTAs per subdomain");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  using Sm = ApplySmem<R, KR, G>;
  const int S = a.stages;
  const bool ysm = yglob == nullptr;
  const int64_t ys = ysm ? 1 : 0;                           // layout selector (see ApplySmem)
  const uint32_t SLOT = Sm::slot(ys);
  unsigned char* ring = smem_raw;
  uint64_t* full = (uint64_t*)(smem_raw + Sm::bar_off(S, ys));
  uint64_t* empty = full + S;
  uint64_t* msg = empty + S;                                // [2]
  CT<R>* recv = (CT<R>*)(smem_raw + Sm::recv_off(S, ys));   // [2][G-1][TB*KR]
  CT<R>* part = (CT<R>*)(smem_raw + Sm::part_off(S, ys));   // [TB*KR] this CTA's partial sums
  CT<R>* rvec = (CT<R>*)(smem_raw + Sm::rvec_off(S, ys));   // [TB*KR]
  __shared__ int abort_flag;
  __shared__ int peer_abort;                                // set by another CTA of the group at the end
  __shared__ int ydone;                                     // strips of y finalised (both passes)
  const int c = (int)cluster_rank();
  const int64_t ns = a.ns[s], np = a.np[s], nts = np / TB;
  auto nown_of = [&](int r) -> int64_t { return (nts - r + G - 1) / G; };  // strips I with I % G == r
  const int64_t nown_s = nown_of(c);                    // strips owned by this CTA
  const int64_t nown = nown_s * TB;                     // owned rows
  int64_t before = 0;                                   // strips owned by the lower ranks
  for (int r = 0; r < c; ++r) before += nown_of(r);
  CT<R>* y = ysm ? (CT<R>*)(smem_raw + Sm::y_off(S, ys)) : yglob + (a.np_off[s] + before * TB) * KR;
  const R* F = (const R*)a.arena + a.tile_off[s] * 2 * TILE_PLANE;
  const R* Dinv = (const R*)a.dinv + a.inv_off[s] * 4 * TILE_PLANE;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr uint32_t TBYTES = tile_bytes<R>();
  constexpr int NV = TB * KR;               // entries of one strip of y
  if (tid == 0) {
    for (int q = 0; q < S; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], APPLY_CONSUMERS / 32);
    }
    mbar_init(&msg[0], G - 1);
    mbar_init(&msg[1], G - 1);
    abort_flag = 0;
    peer_abort = 0;
    ydone = 0;
    fence_mbar_init();
  }
  __syncthreads();
  cluster_sync_all();  // the other CTAs may signal our barriers from here on

  if (warp == APPLY_CONSUMERS / 32) {
    // ---------------- producer: one lane issues the bulk copies in consumption order
    if (lane == 0) {
      int64_t n = 0;
      int slot = 0;
      uint32_t phase = 0;  // parity of the ring round of `slot`
      // ysrc: the y slice for this tile (global y only); need: finalised strips it requires
      auto issue = [&](const R* src, const CT<R>* ysrc, int64_t need) -> bool {
        if (n >= S && !mbar_wait(&empty[slot], phase ^ 1u, false, a.wait_ns)) return false;
        unsigned char* dst = ring + (size_t)slot * SLOT;
        if (ysrc) {
          if (!wait_counter(&ydone, (int)need, a.wait_ns)) return false;
          fence_proxy_async_global();
          mbar_expect_tx(&full[slot], TBYTES + Sm::YB);
          bulk_g2s(dst + TBYTES, ysrc, Sm::YB, &full[slot]);
        } else {
          mbar_expect_tx(&full[slot], TBYTES);
        }
        bulk_g2s(dst, src, TBYTES, &full[slot]);
        ++n;
        if (++slot == S) { slot = 0; phase ^= 1u; }
        return true;
      };
      bool ok = true;
      // forward, strip by strip: the tiles of the own block columns left of the diagonal, then
      // L^{-1} of an owned strip; own strip J is the (J/G + 1)-th finalised
      for (int64_t I = 0; I < nts && ok; ++I) {
        for (int64_t J = c; J < I && ok; J += G)
          ok = issue(F + (I * nts + J) * 2 * TILE_PLANE, ysm ? nullptr : y + (J / G) * NV, J / G + 1);
        if (ok && (I % G) == c) ok = issue(Dinv + I * 4 * TILE_PLANE, nullptr, 0);
      }
      // backward, from the last strip up: the own block columns right of the diagonal, then
      // U^{-1}; the own strips are finalised again, from the last one down
      for (int64_t I = nts - 1; I >= 0 && ok; --I) {
        for (int64_t J = first_right<G>(I, c); J < nts && ok; J += G)
          ok = issue(F + (I * nts + J) * 2 * TILE_PLANE, ysm ? nullptr : y + (J / G) * NV, 2 * nown_s - J / G);
        if (ok && (I % G) == c) ok = issue(Dinv + I * 4 * TILE_PLANE + 2 * TILE_PLANE, nullptr, 0);
      }
      if (!ok) {
        atomicExch(&a.status[ST_ERR], DEV_TIMEOUT);
        abort_flag = 1;
      }
      // drain: every issued copy must land before the block may exit
      for (int64_t q = n > S ? n - S : 0; q < n; ++q)
        mbar_wait(&full[q % S], (uint32_t)((q / S) & 1), false, drain_limit(a.wait_ns));
    }
  } else {
    // ---------------- consumers
    int slot = 0;
    uint32_t phase = 0;  // parity of the ring round of `slot`
    int nfin = 0;        // strips finalised by this CTA (thread 0 publishes it in ydone)
    // receive parity of a strip = its owner's count of owned strips before it (both passes):
    // kr for this CTA's own strips, ks[o] for the strips it sends to owner o
    int kr = 0;
    int ks[G] = {};
    bool ok = true;
    // waits for the next stage; T: its tile, Y: its y slice (global y) or nullptr
    auto stage = [&](const R*& T, const CT<R>*& Y) -> bool {
      if (!mbar_wait(&full[slot], phase, false, a.wait_ns)) return false;
      T = (const R*)(ring + (size_t)slot * SLOT);
      Y = ysm ? nullptr : (const CT<R>*)(ring + (size_t)slot * SLOT + TBYTES);
      return true;
    };
    auto release = [&]() {
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[slot]);
      if (++slot == S) { slot = 0; phase ^= 1u; }
    };
    auto publish = [&]() {  // after the closing barrier of an owned strip
      ++nfin;
      if (tid == 0) st_release_cta(&ydone, nfin);
    };
    // gather the owned strips: y(local) = P_s R_s v
    for (int64_t q = tid; q < nown * KR; q += APPLY_CONSUMERS) {  // q = (strip, r, row)
      const int64_t st = q / NV;
      const int r = (int)((q % NV) / TB), i = (int)(q % TB);
      const int64_t pos = (G * st + c) * TB + i;
      const int32_t g = a.gidx[a.np_off[s] + pos];
      const cplx val = (g >= 0 && r < nr) ? v[(int64_t)g * vs + off + r] : cplx{0.0, 0.0};
      y[q] = {R(val.re), R(val.im)};
    }
    named_sync(1, APPLY_CONSUMERS);
    for (int pass = 0; pass < 2; ++pass) {
      const bool fwd = pass == 0;
      for (int64_t it = 0; it < nts; ++it) {
        const int64_t I = fwd ? it : nts - 1 - it;
        const int o = (int)(I % G);                 // owner of strip I
        const bool owner = o == c;
        // partial sums over the owned block columns of strip I
        CT<R> acc[8][KR];
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
          for (int r = 0; r < KR; ++r) acc[q][r] = {R(0), R(0)};
        const int64_t J0 = fwd ? c : first_right<G>(I, c), J1 = fwd ? I : nts;
        for (int64_t J = J0; J < J1; J += G) {
          const R* T = nullptr;
          const CT<R>* Y = nullptr;
          if (ok) ok = stage(T, Y);
          if (!ok) continue;  // keep the barrier sequence uniform; no more work after a timeout
          const CT<R>* yJ = ysm ? y + (J / G) * NV : Y;
          // row-major tile: warp rows 8w..8w+7, lane columns 2l, 2l+1
          CT<R> y0[KR], y1[KR];
#pragma unroll
          for (int r = 0; r < KR; ++r) ld_cpair(yJ + r * TB + 2 * lane, y0[r], y1[r]);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int e = (warp * 8 + q) * TB + 2 * lane;
            R r0, r1, i0, i1;
            ld_pair(T + e, r0, r1);
            ld_pair(T + TILE_PLANE + e, i0, i1);
#pragma unroll
            for (int r = 0; r < KR; ++r) {
              CT<R>& t = acc[q][r];
              t.re = fma(r0, y0[r].re, t.re); t.re = fma(-i0, y0[r].im, t.re);
              t.re = fma(r1, y1[r].re, t.re); t.re = fma(-i1, y1[r].im, t.re);
              t.im = fma(r0, y0[r].im, t.im); t.im = fma(i0, y0[r].re, t.im);
              t.im = fma(r1, y1[r].im, t.im); t.im = fma(i1, y1[r].re, t.im);
            }
          }
          release();
        }
        // reduce to the TB x KR partial sums of this CTA in part[]
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
          for (int r = 0; r < KR; ++r) {
            CT<R> t = acc[q][r];
            for (int o = 16; o > 0; o >>= 1) {
              t.re += __shfl_down_sync(0xffffffffu, t.re, o);
              t.im += __shfl_down_sync(0xffffffffu, t.im, o);
            }
            if (lane == 0) part[r * TB + warp * 8 + q] = t;
          }
        named_sync(1, APPLY_CONSUMERS);
        if (!owner) {
          // send the partial sums to this CTA's slot of the owner's receive buffer, then signal it
          const int d = ((c - o) & (G - 1)) - 1;
          int& cnt = ks[G == 2 ? 0 : o];            // G = 2: one owner besides this CTA
          const int rb = cnt & 1;
          ++cnt;
          CT<R>* rs = recv + (rb * (G - 1) + d) * NV;
          for (int q = tid; q < NV; q += APPLY_CONSUMERS) st_remote(map_to_rank(&rs[q], (uint32_t)o), part[q].re, part[q].im);
          named_sync(1, APPLY_CONSUMERS);
          if (tid == 0) mbar_arrive_remote(map_to_rank(&msg[rb], (uint32_t)o));
          continue;
        }
        // owner: r = b_I - own partial - the other CTAs' partials
        const int rb = kr & 1;
        if (tid == 0 && !mbar_wait(&msg[rb], (uint32_t)((kr >> 1) & 1), true, a.wait_ns)) {
          atomicExch(&a.status[ST_ERR], DEV_TIMEOUT);
          abort_flag = 1;
        }
        named_sync(1, APPLY_CONSUMERS);
        if (abort_flag) ok = false;
        CT<R>* yI = y + (I / G) * NV;
        for (int q = tid; q < NV; q += APPLY_CONSUMERS) {
          CT<R> t = {yI[q].re - part[q].re, yI[q].im - part[q].im};
#pragma unroll
          for (int d = 0; d < G - 1; ++d) {
            const CT<R> pr = recv[(rb * (G - 1) + d) * NV + q];
            t.re -= pr.re;
            t.im -= pr.im;
          }
          rvec[q] = t;
        }
        ++kr;
        named_sync(1, APPLY_CONSUMERS);
        // y_I = inv(diag block) r
        const R* T = nullptr;
        const CT<R>* Y = nullptr;
        if (ok) ok = stage(T, Y);
        if (!ok) {
          named_sync(1, APPLY_CONSUMERS);
          publish();
          continue;
        }
        {  // y_I = Linv_I r (forward) or Uinv_I r (backward): row-major inverse of the diagonal block
          CT<R> r0v[KR], r1v[KR];
#pragma unroll
          for (int r = 0; r < KR; ++r) ld_cpair(rvec + r * TB + 2 * lane, r0v[r], r1v[r]);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int e = (warp * 8 + q) * TB + 2 * lane;
            R r0, r1, i0, i1;
            ld_pair(T + e, r0, r1);
            ld_pair(T + TILE_PLANE + e, i0, i1);
#pragma unroll
            for (int r = 0; r < KR; ++r) {
              CT<R> t = {r0 * r0v[r].re - i0 * r0v[r].im + r1 * r1v[r].re - i1 * r1v[r].im,
                         r0 * r0v[r].im + i0 * r0v[r].re + r1 * r1v[r].im + i1 * r1v[r].re};
              for (int o = 16; o > 0; o >>= 1) {
                t.re += __shfl_down_sync(0xffffffffu, t.re, o);
                t.im += __shfl_down_sync(0xffffffffu, t.im, o);
              }
              if (lane == 0) yI[r * TB + warp * 8 + q] = t;
            }
          }
          release();
        }
        if (!ysm) fence_proxy_async_global();  // y_I is read next by bulk copies
        named_sync(1, APPLY_CONSUMERS);
        publish();
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
      for (int64_t q = tid; q < nown * KR; q += APPLY_CONSUMERS) {
        const int64_t st = q / NV;
        const int r = (int)((q % NV) / TB), i = (int)(q % TB);
        const int64_t pos = (G * st + c) * TB + i;
        if (pos >= ns || r >= nr) continue;
        const CT<R> val = y[q];
        ZT* dst = z + (int64_t)Ns[pos] * zs + off + r;
        if (a.weights == ORAS_WEIGHTS_POU) {
          if (Dp[pos]) z_store(dst, (double)val.re, (double)val.im);
        } else {
          z_add(dst, (double)val.re, (double)val.im);
        }
      }
    }
  }
  __syncthreads();
  // tell the others whether this CTA gave up; the closing cluster barrier (release/acquire)
  // makes the flag visible, so all CTAs return the same result
  if (threadIdx.x == 0 && abort_flag)
    for (int r = 0; r < G; ++r)
      if (r != c) st_remote_u32(map_to_rank(&peer_abort, (uint32_t)r), 1u);
  cluster_sync_all();  // no other CTA may touch our shared memory after we exit
  return abort_flag != 0 || peer_abort != 0;
}

}  // namespace oras
