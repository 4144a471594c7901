// ORAS preconditioner apply for many right-hand sides on the tcgen05 tensor cores (Sec. 4-5):
//   z = sum_s R_s^T D_s U_s^{-1} L_s^{-1} P_s R_s v   for KT right-hand sides per arena pass.
//
// With KT right-hand sides, each tile step of the block substitution is a 64 x 64 complex tile
// times a 64 x KT complex block: about 4 KT flops per factor byte, more than the CUDA cores can
// keep up with while the arena streams from HBM.  Here it is one real product on the tensor cores
// (kind::tf32, FP32 accumulation in tensor memory):
//   A (M = 128 x K = 64): the tile's real plane (rows 0..63) stacked on its imaginary plane
//       (rows 64..127) -- exactly the tile's storage, row-major planes, so TMA loads it as is;
//   B (N = 2 KT x K = 64): the y block, real parts of the KT columns then imaginary parts;
//   ACC = A B^T (128 x 2 KT):  rows i < 64 hold Tr Yr | Tr Yi, rows 64 + i hold Ti Yr | Ti Yi,
//   so (T Y)_re = ACC[i, r] - ACC[64 + i, KT + r],  (T Y)_im = ACC[i, KT + r] + ACC[64 + i, r].
// Both operands are K-major (contiguous along the tile's column index): every factor tile is
// row-major after the factorisation, and the y strips are kept in global memory in the 128-byte
// swizzled K-major image of the B operand, so one 1-D bulk copy stages them next to their tile.
//
// Work split and protocol as in the CUDA-core apply (apply.cuh): a cluster of two CTAs per
// subdomain (or, when the subdomains alone fill every SM, one CTA per subdomain that owns every
// strip: no partial sums to exchange, and a deeper ring); CTA c owns the strips I with I % 2 == c and streams the tiles of its own block
// columns J % 2 == c; for every strip each CTA accumulates its partial product in tensor memory;
// the non-owner sends its 64 x KT partial sums to the owner through distributed shared memory;
// the owner forms r = b_I - both partials, writes r into shared memory in the B layout, and one
// more product with the inverted diagonal block gives y_I.
//
// Warp roles (192 threads): warps 0-3 read the accumulators (warp w owns tensor-memory lanes
// 32w..32w+31) and do all vector work; warp 4 lane 0 issues the TMA and bulk copies of the ring;
// warp 5 lane 0 issues the MMAs.  Tensor memory: two strip accumulators used in turn (the MMAs of
// the next strip overlap the epilogue of the previous one) and one for the diagonal product.
// Every wait is bounded (ApplyGeom::wait_ns); after a timeout every role skips its remaining work
// but keeps the barrier sequence, so the block always finishes.
#include <cuda.h>

#include <cstring>

#include "apply.cuh"

namespace oras {

constexpr int ATC_EPI = 128;                      // epilogue threads (4 warps)
constexpr int ATC_THREADS = ATC_EPI + 64;         // + producer warp + MMA warp
constexpr uint32_t ATC_HALF = 64 * 128;           // 64 rows x 128 B: one plane of one K-chunk
constexpr uint32_t ATC_CHUNK_A = 2 * ATC_HALF;    // one K-chunk (32 columns) of a tile, both planes
constexpr uint32_t ATC_TILE = 2 * ATC_CHUNK_A;    // 32 KB

template <int KT, bool SOLO = false>
struct AtcShape {
  static_assert(KT == 8 || KT == 16 || KT == 32, "right-hand sides per pass");
  static constexpr int N = 2 * KT;                          // MMA N (multiple of 16 for M = 128)
  static constexpr uint32_t CHUNK_B = N * 128;              // one K-chunk of a y block (B layout)
  static constexpr uint32_t YB = 2 * CHUNK_B;               // a y strip: 64 rows x KT complex FP32
  static constexpr uint32_t STAGE = ATC_TILE + YB;
  static constexpr int TMEM_COLS = 3 * N <= 64 ? 64 : (3 * N <= 128 ? 128 : 256);
  static constexpr uint32_t XCH = 64 * (N + 1) * 4;         // lane exchange of the accumulators
  static constexpr uint32_t RECV = 64 * KT * 8;             // partial sums of one strip
  static __host__ __device__ size_t rb_off(int S) { return (size_t)S * STAGE; }
  static __host__ __device__ size_t xch_off(int S) { return rb_off(S) + YB; }
  static __host__ __device__ size_t recv_off(int S) { return xch_off(S) + XCH; }
  static __host__ __device__ size_t bar_off(int S) { return (recv_off(S) + (SOLO ? 0 : 2 * RECV) + 15) & ~(size_t)15; }
  // full[S], empty[S], accf[2], acce[2], rbf, dgd, msg[2], fin
  static __host__ __device__ size_t total(int S) { return bar_off(S) + (size_t)(2 * S + 9) * 8 + 1024; }
  static_assert(STAGE % 1024 == 0 && YB % 1024 == 0, "swizzle-atom alignment of the stages");
  static_assert(TMEM_COLS >= 3 * N, "tensor-memory columns");
};

// Byte offset of element (row n, column k) of a K-major operand with 128-byte swizzle, K = 64 split
// in two chunks of 32 floats: rows are 128 B, 8-row groups 1024 B apart, the 16-byte granule g of
// row n stored at g ^ (n % 8) (the layout TMA writes with CU_TENSOR_MAP_SWIZZLE_128B).
__device__ __forceinline__ uint32_t sw128_off(int n, int k, uint32_t chunk_bytes) {
  const int c = k >> 5, kk = k & 31;
  return (uint32_t)c * chunk_bytes + (uint32_t)(n >> 3) * 1024u + (uint32_t)(n & 7) * 128u +
         ((uint32_t)((kk >> 2) ^ (n & 7)) << 4) + (uint32_t)(kk & 3) * 4u;
}

__device__ __forceinline__ void atc_tma(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t atc_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | (1ull << 16) | (64ull << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major, M = 128, N.
template <int N>
__host__ __device__ constexpr uint32_t atc_idesc() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void atc_mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
      ::"r"(dtmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void atc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 16 consecutive accumulator columns of this thread's lane.
__device__ __forceinline__ void atc_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

struct AtcArgs {
  ApplyGeom g;
  int64_t dinv_tiles;       // tiles of the inverted-diagonal array (tensor map extent)
};

// Item kinds of a CTA's stream of work (atc_stream).
enum { ATC_ITEM_TILE = 0, ATC_ITEM_DIAG = 1, ATC_ITEM_COMMIT = 2 };

// The order in which CTA c loads and multiplies: f(kind, I, J, slot) for
//   ATC_ITEM_TILE   (I, J): off-diagonal tile of strip I times y_J, into the accumulator of strip `slot`;
//   ATC_ITEM_DIAG   (I)   : the inverted diagonal block of owned strip I times r_I;
//   ATC_ITEM_COMMIT (slot): strip `slot` has all its products (its accumulator may be read out).
// Strip slots number the strips in processing order (forward strips 0..nts-1, then backward from
// the last).  CTA c takes the tiles of its own block columns J % 2 == c.  Look-ahead: the strip
// that follows an owned strip I is owned by the partner, and all its tiles here but the one in
// block column I need only y values finalised earlier -- they are issued before the diagonal
// product of strip I, so the tensor cores work through them while the epilogue waits for the
// partner's partial sums of strip I; the one tile that needs y_I comes right after it.
//
// SOLO (one CTA per subdomain, every strip owned): the strip after I is again this CTA's; its tiles
// but the one in block column I are issued before the diagonal product of strip I, so they overlap
// the epilogue of strip I in the same way.
template <bool SOLO, typename F>
__device__ __forceinline__ void atc_stream(int c, int64_t nts, F&& f) {
  constexpr int ST = SOLO ? 1 : 2;  // block-column stride of this CTA
  for (int pass = 0; pass < 2; ++pass) {
    const bool fwd = pass == 0;
    for (int64_t it = 0; it < nts; ++it) {
      const int64_t I = fwd ? it : nts - 1 - it;
      const int64_t slot = (int64_t)pass * nts + it;
      if (!SOLO && (I & 1) != c) {
        if (it == 0) f(ATC_ITEM_COMMIT, I, I, slot);  // no owned strip before it: nothing to multiply
        continue;
      }
      // the owned strip: block columns J % ST == c below (forward) or above (backward) I.  Solo,
      // they were issued with the previous strip's (all but the first strip of a pass).
      if (!SOLO || it == 0) {
        if (fwd) for (int64_t J = c; J < I; J += ST) f(ATC_ITEM_TILE, I, J, slot);
        else for (int64_t J = I + ST; J < nts; J += ST) f(ATC_ITEM_TILE, I, J, slot);
        f(ATC_ITEM_COMMIT, I, I, slot);
      }
      const bool next = it + 1 < nts;
      const int64_t I1 = fwd ? I + 1 : I - 1;
      if (next) {  // the next strip: every tile but the one in block column I
        if (fwd) for (int64_t J = c; J < I; J += ST) f(ATC_ITEM_TILE, I1, J, slot + 1);
        else for (int64_t J = I + ST; J < nts; J += ST) f(ATC_ITEM_TILE, I1, J, slot + 1);
      }
      f(ATC_ITEM_DIAG, I, I, slot);
      if (next) {
        f(ATC_ITEM_TILE, I1, I, slot + 1);
        f(ATC_ITEM_COMMIT, I1, I1, slot + 1);
      }
    }
  }
}

// One pass of KT right-hand sides (columns off .. off+nr-1 of v and z) for subdomain s: a cluster
// of two CTAs, or with SOLO one CTA that owns every strip (no partial sums to exchange).
template <int KT, typename ZT, bool SOLO>
__device__ bool apply_cluster_tc(const AtcArgs& aa, const CUtensorMap* amap, const CUtensorMap* dmap, int s,
                                 const cplx* __restrict__ v, int64_t vs, ZT* __restrict__ z, int64_t zs,
                                 int64_t off, int nr, unsigned char* yglob) {
  using Sh = AtcShape<KT, SOLO>;
  constexpr int N = Sh::N;
  constexpr int ST = SOLO ? 1 : 2;  // block-column stride of this CTA
  const ApplyGeom& a = aa.g;
  extern __shared__ __align__(1024) unsigned char atc_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)atc_raw + 1023) & ~(uintptr_t)1023);
  const int S = a.stages;
  unsigned char* ring = sm;
  unsigned char* rB = sm + Sh::rb_off(S);
  float* xch = (float*)(sm + Sh::xch_off(S));
  float2* recv = (float2*)(sm + Sh::recv_off(S));          // [2][64][KT] (clusters only)
  uint64_t* full = (uint64_t*)(sm + Sh::bar_off(S));
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;                               // [2] strip accumulator ready
  uint64_t* acce = accf + 2;                                // [2] strip accumulator read out
  uint64_t* rbf = acce + 2;                                 // r written into rB
  uint64_t* dgd = rbf + 1;                                  // diagonal product done
  uint64_t* msg = dgd + 1;                                  // [2] partial sums from the partner
  uint64_t* fin = msg + 2;                                  // every MMA of this CTA done
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag, peer_abort, ydone, ep_ok;
  const int c = SOLO ? 0 : (int)cluster_rank();
  const int64_t ns = a.ns[s], np = a.np[s], nts = np / TB;
  const int64_t own0 = SOLO ? nts : (nts + 1) / 2;
  const int64_t nown_s = c ? nts - own0 : own0;
  // this CTA's strips (own strip I is number I / ST among them)
  unsigned char* ysub = yglob + ((a.np_off[s] / TB) + (c ? own0 : 0)) * (int64_t)Sh::YB;
  const int64_t toff = a.tile_off[s];
  const int64_t ioff = a.inv_off[s];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int q = 0; q < S; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&accf[q], 1);
      mbar_init(&acce[q], 1);
      mbar_init(&msg[q], 1);
    }
    mbar_init(rbf, 1);
    mbar_init(dgd, 1);
    mbar_init(fin, 1);
    abort_flag = 0;
    peer_abort = 0;
    ydone = 0;
    ep_ok = 1;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(Sh::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!SOLO) cluster_sync_all();  // the partner may signal our barriers from here on
  const uint32_t tbase = tmem_base;

  if (warp == 4) {
    // ---------------- producer: tiles (and y strips) in consumption order
    if (lane == 0) {
      int64_t n = 0;
      int slot = 0;
      uint32_t phase = 0;
      bool ok = true;
      // off-diagonal tile (I, J) with its y strip J, or an inverted diagonal block
      auto issue = [&](bool diag, int64_t I, int64_t J, int which, int64_t need) -> bool {
        if (n >= S && !mbar_wait(&empty[slot], phase ^ 1u, false, a.wait_ns)) return false;
        unsigned char* dst = ring + (size_t)slot * Sh::STAGE;
        if (!diag) {
          if (!wait_counter(&ydone, (int)need, a.wait_ns)) return false;
          fence_proxy_async_global();
          mbar_expect_tx(&full[slot], ATC_TILE + Sh::YB);
          bulk_g2s(dst + ATC_TILE, ysub + (J / ST) * (int64_t)Sh::YB, Sh::YB, &full[slot]);
          const int zt = (int)(toff + I * nts + J);
          for (int ch = 0; ch < 2; ++ch) {
            atc_tma(dst + ch * ATC_CHUNK_A, amap, 32 * ch, 0, zt, &full[slot]);
            atc_tma(dst + ch * ATC_CHUNK_A + ATC_HALF, amap, 32 * ch, 64, zt, &full[slot]);
          }
        } else {
          mbar_expect_tx(&full[slot], ATC_TILE);
          const int zt = (int)(2 * (ioff + I) + which);
          for (int ch = 0; ch < 2; ++ch) {
            atc_tma(dst + ch * ATC_CHUNK_A, dmap, 32 * ch, 0, zt, &full[slot]);
            atc_tma(dst + ch * ATC_CHUNK_A + ATC_HALF, dmap, 32 * ch, 64, zt, &full[slot]);
          }
        }
        ++n;
        if (++slot == S) { slot = 0; phase ^= 1u; }
        return true;
      };
      atc_stream<SOLO>(c, nts, [&](int kind, int64_t I, int64_t J, int64_t slot_s) {
        if (!ok || kind == ATC_ITEM_COMMIT) return;
        const bool fwd = slot_s < nts;
        if (kind == ATC_ITEM_DIAG) ok = issue(true, I, I, fwd ? 0 : 1, 0);
        else ok = issue(false, I, J, 0, fwd ? J / ST + 1 : 2 * nown_s - J / ST);
      });
      if (!ok) {
        atomicExch(&a.status[ST_ERR], DEV_TIMEOUT);
        abort_flag = 1;
      }
      // drain: every issued copy must land before the block may exit
      for (int64_t q = n > S ? n - S : 0; q < n; ++q)
        mbar_wait(&full[q % S], (uint32_t)((q / S) & 1), false, drain_limit(a.wait_ns));
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = atc_idesc<N>();
      int slot = 0;
      uint32_t phase = 0;
      int64_t owned = 0;
      bool ok = true;
      auto tile_mma = [&](uint32_t dcol, uint32_t bsaddr, bool first) {
        const uint32_t asaddr = smem_u32(ring + (size_t)slot * Sh::STAGE);
#pragma unroll
        for (int ch = 0; ch < 2; ++ch)
#pragma unroll
          for (int k8 = 0; k8 < 4; ++k8) {
            const uint64_t ad = atc_desc(asaddr + ch * ATC_CHUNK_A) + (uint64_t)((k8 * 32) >> 4);
            const uint64_t bd = atc_desc(bsaddr + ch * Sh::CHUNK_B) + (uint64_t)((k8 * 32) >> 4);
            atc_mma(tbase + dcol, ad, bd, idesc, (first && ch == 0 && k8 == 0) ? 0u : 1u);
          }
      };
      int started = 0;  // bit b: the open strip of accumulator b has had its first product
      atc_stream<SOLO>(c, nts, [&](int kind, int64_t I, int64_t J, int64_t slot_s) {
        const int b = (int)(slot_s & 1);
        if (kind == ATC_ITEM_COMMIT) {
          atc_commit(&accf[b]);  // arrives when this strip's products are in tensor memory
          started &= ~(1 << b);
          return;
        }
        if (kind == ATC_ITEM_DIAG) {
          // the inverted diagonal block times r (written into rB by the epilogue)
          if (ok && !mbar_wait(rbf, (uint32_t)(owned & 1), false, a.wait_ns)) ok = false;
          if (ok && !mbar_wait(&full[slot], phase, false, a.wait_ns)) ok = false;
          if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            tile_mma((uint32_t)(2 * N), smem_u32(rB), true);
            atc_commit(&empty[slot]);
            if (++slot == S) { slot = 0; phase ^= 1u; }
          }
          atc_commit(dgd);
          ++owned;
          return;
        }
        if (!ok) return;
        const bool first = !(started & (1 << b));
        const int64_t use = slot_s >> 1;
        if (first && use >= 1 && !mbar_wait(&acce[b], (uint32_t)((use - 1) & 1), false, a.wait_ns)) {
          ok = false;
          return;
        }
        if (!mbar_wait(&full[slot], phase, false, a.wait_ns)) { ok = false; return; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tile_mma((uint32_t)(b * N), smem_u32(ring + (size_t)slot * Sh::STAGE + ATC_TILE), first);
        started |= 1 << b;
        atc_commit(&empty[slot]);
        if (++slot == S) { slot = 0; phase ^= 1u; }
      });
      if (!ok) {
        atomicExch(&a.status[ST_ERR], DEV_TIMEOUT);
        abort_flag = 1;
      }
      atc_commit(fin);
      mbar_wait(fin, 0, false, drain_limit(a.wait_ns));  // no MMA in flight when the block exits
    }
  } else {
    // ---------------- epilogue: warps 0-3, thread t = tensor-memory lane t = accumulator row t
    const uint32_t partner = (uint32_t)(c ^ 1);
    const uint32_t lane_base = tbase + ((uint32_t)(warp * 32) << 16);
    const int i = tid;  // strip row for tid < 64
    bool ok = true;
    int64_t strips = 0, owned = 0;
    int ks = 0, kr = 0;
    float acc[N];
    // accumulator columns [col, col + N) of this lane, combined into the complex 64 x KT product
    // held by threads 0..63 (rows of the strip): out[r] = (T Y)(i, r)
    auto read_combine = [&](uint32_t col, bool have, float2* out) {
      if (have) {
#pragma unroll
        for (int q = 0; q < N; q += 16) atc_ld16(lane_base + col + q, acc + q);
      } else {
#pragma unroll
        for (int q = 0; q < N; ++q) acc[q] = 0.0f;
      }
      if (tid >= 64) {
#pragma unroll
        for (int q = 0; q < N; ++q) xch[(tid - 64) * (N + 1) + q] = acc[q];
      }
      named_sync(1, ATC_EPI);
      if (tid < 64) {
#pragma unroll
        for (int r = 0; r < KT; ++r)
          out[r] = make_float2(acc[r] - xch[i * (N + 1) + KT + r], acc[KT + r] + xch[i * (N + 1) + r]);
      }
      named_sync(1, ATC_EPI);
    };
    // a thread-0 wait whose outcome every epilogue thread takes
    auto uniform_wait = [&](uint64_t* bar, uint32_t parity, bool cluster_scope) {
      if (tid == 0) ep_ok = (ok && mbar_wait(bar, parity, cluster_scope, a.wait_ns)) ? 1 : 0;
      named_sync(1, ATC_EPI);
      const bool r = ep_ok != 0;
      named_sync(1, ATC_EPI);
      return r;
    };
    float2 d[KT];
    for (int pass = 0; pass < 2; ++pass) {
      const bool fwd = pass == 0;
      for (int64_t it = 0; it < nts; ++it) {
        const int64_t I = fwd ? it : nts - 1 - it;
        const bool owner = SOLO || (I & 1) == c;
        const int b = (int)(strips & 1);
        const int64_t use = strips >> 1;
        const int64_t J0 = fwd ? c : (SOLO ? I + 1 : I + 1 + ((I + 1 + c) & 1)), J1 = fwd ? I : nts;
        const bool have = J0 < J1;
        ok = uniform_wait(&accf[b], (uint32_t)(use & 1), false);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        read_combine((uint32_t)(b * N), ok && have, d);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (tid == 0) mbar_arrive(&acce[b]);  // the next strip on this accumulator may start
        ++strips;
        if (!owner) {
          // send the partial sums to the owner, then signal it
          if (tid < 64) {
#pragma unroll
            for (int r = 0; r < KT; ++r) {
              const uint32_t dst = map_to_rank(&recv[(ks & 1) * 64 * KT + i * KT + r], partner);
              st_remote(dst, d[r].x, d[r].y);
            }
          }
          named_sync(1, ATC_EPI);
          if (tid == 0) mbar_arrive_remote(map_to_rank(&msg[ks & 1], partner));
          ++ks;
          continue;
        }
        // owner: r = b_I - own partial - partner partial, written into rB (B layout)
        if (!SOLO) ok = uniform_wait(&msg[kr & 1], (uint32_t)((kr >> 1) & 1), true);
        unsigned char* yI = ysub + (I / ST) * (int64_t)Sh::YB;
        if (tid < 64) {
          const float2* pr = SOLO ? nullptr : recv + (kr & 1) * 64 * KT + i * KT;
          const int64_t pos = I * TB + i;
#pragma unroll
          for (int r = 0; r < KT; ++r) {
            float br = 0.0f, bi = 0.0f;
            if (fwd) {
              const int32_t g = a.gidx[a.np_off[s] + pos];
              if (g >= 0 && r < nr) {
                const cplx val = v[(int64_t)g * vs + off + r];
                br = (float)val.re;
                bi = (float)val.im;
              }
            } else {
              br = *(const float*)(yI + sw128_off(r, i, Sh::CHUNK_B));
              bi = *(const float*)(yI + sw128_off(KT + r, i, Sh::CHUNK_B));
            }
            const float2 p2 = SOLO ? make_float2(0.0f, 0.0f) : pr[r];
            *(float*)(rB + sw128_off(r, i, Sh::CHUNK_B)) = br - d[r].x - p2.x;
            *(float*)(rB + sw128_off(KT + r, i, Sh::CHUNK_B)) = bi - d[r].y - p2.y;
          }
          fence_proxy_async_smem();  // rB is read next by the tensor cores
        }
        ++kr;
        named_sync(1, ATC_EPI);
        if (tid == 0) mbar_arrive(rbf);
        // y_I = inverse of the diagonal block times r
        ok = uniform_wait(dgd, (uint32_t)(owned & 1), false);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        read_combine((uint32_t)(2 * N), ok, d);
        ++owned;
        if (tid < 64) {
#pragma unroll
          for (int r = 0; r < KT; ++r) {
            *(float*)(yI + sw128_off(r, i, Sh::CHUNK_B)) = d[r].x;
            *(float*)(yI + sw128_off(KT + r, i, Sh::CHUNK_B)) = d[r].y;
          }
          fence_proxy_async_global();  // y_I is read next by bulk copies
        }
        named_sync(1, ATC_EPI);
        if (tid == 0) st_release_cta(&ydone, (int)owned);
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
      for (int64_t q = tid; q < nown_s * TB * KT; q += ATC_EPI) {
        const int64_t st = q / (TB * KT);
        const int r = (int)((q / TB) % KT), ii = (int)(q % TB);
        const int64_t pos = (ST * st + c) * TB + ii;
        if (pos >= ns || r >= nr) continue;
        const unsigned char* yst = ysub + st * (int64_t)Sh::YB;
        const float re = *(const float*)(yst + sw128_off(r, ii, Sh::CHUNK_B));
        const float im = *(const float*)(yst + sw128_off(KT + r, ii, Sh::CHUNK_B));
        ZT* dst = z + (int64_t)Ns[pos] * zs + off + r;
        if (a.weights == ORAS_WEIGHTS_POU) {
          if (Dp[pos]) z_store(dst, (double)re, (double)im);
        } else {
          z_add(dst, (double)re, (double)im);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(Sh::TMEM_COLS));
  if (SOLO) return abort_flag != 0;
  if (threadIdx.x == 0 && abort_flag) st_remote_u32(map_to_rank(&peer_abort, (uint32_t)(c ^ 1)), 1u);
  cluster_sync_all();  // the partner must not touch our shared memory after we exit
  return abort_flag != 0 || peer_abort != 0;
}

template <int KT, typename ZT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(ATC_THREADS, 1)
    k_apply_tc(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap dmap, AtcArgs aa,
               int k, int r0, int nr, unsigned char* yglob, const cplx* __restrict__ v, ZT* __restrict__ z) {
  apply_cluster_tc<KT, ZT, false>(aa, &amap, &dmap, blockIdx.x / 2, v, k, z, k, r0, nr, yglob);
}

// One CTA per subdomain (launched when the subdomains alone fill every SM).
template <int KT, typename ZT>
__global__ void __launch_bounds__(ATC_THREADS, 1)
    k_apply_tc_solo(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap dmap, AtcArgs aa,
                    int k, int r0, int nr, unsigned char* yglob, const cplx* __restrict__ v, ZT* __restrict__ z) {
  apply_cluster_tc<KT, ZT, true>(aa, &amap, &dmap, blockIdx.x, v, k, z, k, r0, nr, yglob);
}

// ------------------------------------------------------------------ host side
typedef CUresult (*AtcEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static AtcEncodeFn atc_encode() {
  static AtcEncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (AtcEncodeFn)p;
  });
  return fn;
}

// Tensor map over an array of FP32 tiles viewed as [tiles][2 planes x 64 rows][64 floats]; boxes
// of 32 floats x 64 rows (one plane of one K-chunk), 128-byte swizzle.
static bool atc_map(void* base, int64_t tiles, CUtensorMap* map) {
  AtcEncodeFn enc = atc_encode();
  if (!enc || !base || tiles <= 0 || tiles >= (int64_t(1) << 31)) return false;
  cuuint64_t dims[3] = {64, 128, (cuuint64_t)tiles};
  cuuint64_t strides[2] = {64 * sizeof(float), 128 * 64 * sizeof(float)};
  cuuint32_t box[3] = {32, 64, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

ApplyGeom apply_geom(const oras_handle* h);
constexpr size_t ATC_SMEM_LIMIT = 227 * 1024 - 1024;  // opt-in shared memory less the static part

template <int KT, bool SOLO>
static int atc_stages() {
  for (int q = 4; q >= 2; --q)
    if (AtcShape<KT, SOLO>::total(q) <= ATC_SMEM_LIMIT) return q;
  return 0;
}

// One CTA per subdomain when the subdomains alone give every SM a CTA (no partial sums to
// exchange, so the ring has room for one more stage); else a two-CTA cluster per subdomain.
static bool atc_solo(const oras_handle* h) {
  static int sms = 0;
  if (!sms) {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0) sms = n;
    else return false;
  }
  return h->mesh.nsub >= sms;
}

// Right-hand sides per tensor-core pass for a group of `rem` columns.
static int atc_kt(int rem) { return rem > 16 ? 32 : (rem > 8 ? 16 : 8); }

// Global bytes of the y strips of a tensor-core pass of KT right-hand sides.
size_t apply_tc_ybytes(const oras_handle* h, int kt) {
  int64_t total = 0;
  for (int s = 0; s < h->mesh.nsub; ++s) total += h->mesh.sub_np[s];
  return (size_t)total * kt * 8;
}

// Tensor-core apply available for this handle (FP32 factors, tensor maps encodable, the shared
// memory of every KT fits).
bool apply_tc_available(const oras_handle* h) {
  if (h->dev.factor_bits != 32 || !h->dev.arena || !h->dev.dinv) return false;
  if (h->opt.apply_engine == ORAS_APPLY_CUDA_CORES) return false;
  if (!atc_stages<8, false>() || !atc_stages<16, false>() || !atc_stages<32, false>()) return false;
  CUtensorMap m;
  return atc_map(h->dev.arena, h->mesh.arena_tiles + (int64_t)LU_SCRATCH * h->mesh.nsub, &m);
}

template <int KT, typename ZT>
static int atc_launch(const oras_handle* h, const cplx* v, ZT* z, int k, int r0, int nr) {
  const auto& m = h->mesh;
  const auto& d = h->dev;
  CUtensorMap amap, dmap;
  const int64_t dtiles = (int64_t)(d.dinv_bytes / (2 * TB * TB * sizeof(float)));
  if (!atc_map(d.arena, m.arena_tiles + (int64_t)LU_SCRATCH * m.nsub, &amap) || !atc_map(d.dinv, dtiles, &dmap)) return -1;
  if (!d.ybuf || d.ybuf_bytes < apply_tc_ybytes(h, KT)) return -1;
  AtcArgs aa;
  aa.g = apply_geom(h);
  aa.dinv_tiles = dtiles;
  if (atc_solo(h)) {
    aa.g.stages = atc_stages<KT, true>();
    const size_t smem = AtcShape<KT, true>::total(aa.g.stages);
    allow_max_smem((const void*)k_apply_tc_solo<KT, ZT>);
    k_apply_tc_solo<KT, ZT><<<m.nsub, ATC_THREADS, smem, d.stream>>>(amap, dmap, aa, k, r0, nr,
                                                                      (unsigned char*)d.ybuf, v, z);
  } else {
    aa.g.stages = atc_stages<KT, false>();
    const size_t smem = AtcShape<KT, false>::total(aa.g.stages);
    allow_max_smem((const void*)k_apply_tc<KT, ZT>);
    k_apply_tc<KT, ZT><<<2 * m.nsub, ATC_THREADS, smem, d.stream>>>(amap, dmap, aa, k, r0, nr,
                                                                     (unsigned char*)d.ybuf, v, z);
  }
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// z = M^{-1} v for columns [r0, r0 + nr) through tensor-core passes of up to 32 columns; returns
// the number of launches, or -1.
template <typename ZT>
static int apply_tc_t(const oras_handle* h, const cplx* v, ZT* z, int k, int r0, int nr) {
  int launches = 0;
  for (int q0 = r0; q0 < r0 + nr;) {
    const int rem = r0 + nr - q0, kt = atc_kt(rem), cnt = rem < kt ? rem : kt;
    int rc;
    if (kt == 8) rc = atc_launch<8, ZT>(h, v, z, k, q0, cnt);
    else if (kt == 16) rc = atc_launch<16, ZT>(h, v, z, k, q0, cnt);
    else rc = atc_launch<32, ZT>(h, v, z, k, q0, cnt);
    if (rc) return -1;
    q0 += cnt;
    ++launches;
  }
  return launches;
}

int apply_tc_f64out(const oras_handle* h, const cplx* v, cplx* z, int k, int r0, int nr) {
  return apply_tc_t<cplx>(h, v, z, k, r0, nr);
}
int apply_tc_f32out(const oras_handle* h, const cplx* v, void* z, int k, int r0, int nr) {
  return apply_tc_t<CT<float>>(h, v, (CT<float>*)z, k, r0, nr);
}

// Launches of a tensor-core apply of nr columns.
int apply_tc_passes(int nr) {
  int n = 0;
  for (int q0 = 0; q0 < nr; ++n) {
    const int kt = atc_kt(nr - q0);
    q0 += nr - q0 < kt ? nr - q0 : kt;
  }
  return n;
}

}  // namespace oras
