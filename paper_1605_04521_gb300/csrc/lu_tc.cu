// Trailing update of the batched LU on the 5th-generation tensor cores (tcgen05, TF32 inputs,
// FP32 accumulation in tensor memory):  C_IJ -= sum_{kk in [kk0, kk1)} L_I,kk U_kk,J.
//
// Complex product as real products of the split planes (Gauss's real-split form):
//   C_re -= L_re U_re - L_im U_im ,   C_im -= L_re U_im + L_im U_re .
// L tiles (below the diagonal) store row-major planes and U tiles (above it) column-major
// planes, so both operands are K-major: an L plane is an M x K matrix with K contiguous and a
// U plane is the N x K transpose of the K x N operand.  Each CTA owns a 128 x 64*BN complex
// output block (2 x BN tiles): D_re and D_im are 128 x 64*BN FP32 accumulators in tensor memory
// (BN = 4: all 512 columns, for wide regions; BN = 1: 128 columns, for the single tile column
// that a left-looking panel step updates).  The -L_im U_im term uses the instruction's negate-B
// bit.
//
// Warp roles (128 threads): warp 0 lane 0 loads operand chunks with TMA (one tensor map over
// the whole arena, 128-byte swizzle); warp 1 lane 0 issues the MMAs and commits them to the
// stage's "empty" barrier; after the last commit all four warps read their 32 accumulator rows
// from tensor memory and subtract them from C.  Stages hold one 32-float K-chunk of all four
// operand planes (96 KB for BN = 4, two stages; 48 KB for BN = 1, four stages).  Waits are
// bounded; a timeout sets the device status flag.
#include <cuda.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "lu.cuh"

namespace oras {

constexpr int TC_THREADS = 128;
constexpr int TC_GROUP = 8;                              // default block rows per raster group (L2 reuse)
constexpr uint32_t TC_BOX_BYTES = 64 * 32 * 4;           // 64 rows x 32 floats

// Shape of one output block: BN tile columns (N = 64 BN).
template <int BN>
struct TcShape {
  static_assert(BN == 1 || BN == 4, "output block widths");
  static constexpr int STAGES = BN == 4 ? 2 : 4;
  static constexpr uint32_t STAGE_BYTES = (4 + 2 * BN) * TC_BOX_BYTES;  // A_re, A_im (2 tiles), B_re, B_im (BN)
  static constexpr uint32_t TMEM_COLS = 2 * 64 * BN;                    // D_re, D_im
  static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024;
  // stage bases stay on the 1024-byte boundary of the 128-byte swizzle atoms
  static_assert(TC_BOX_BYTES % 1024 == 0 && STAGE_BYTES % 1024 == 0, "swizzle-atom alignment");
  // dynamic (+ alignment slack) and static shared memory within the 227 KB opt-in limit
  static_assert(SMEM + 1024 <= 227 * 1024, "shared memory per CTA");
  // tcgen05.alloc takes a power of two from 32 to 512 columns
  static_assert(TMEM_COLS >= 32 && TMEM_COLS <= 512 && (TMEM_COLS & (TMEM_COLS - 1)) == 0, "TMEM columns");
  // kind::tf32 with M = 128: N a multiple of 16, at most 256
  static_assert((64 * BN) % 16 == 0 && 64 * BN <= 256, "MMA N");
};

struct TcArgs {
  const int64_t* np;
  const int64_t* tile_off;
  float* arena;
  UpdArgs u;
  int32_t* status;
  int group;                 // block rows per raster group
};

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | (1ull << 16) | (64ull << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major, M = 128, N = 64 BN.
template <int BN>
__device__ __forceinline__ uint32_t idesc_tf32(bool negate_b) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((negate_b ? 1u : 0u) << 14) | (((64u * BN) >> 3) << 17) |
         ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
      ::"r"(dtmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// Map the block index to a 2 x BN-tile output block of one region of subdomain s.  Blocks
// are ordered in groups of TC_GROUP block rows, walking down a group before moving right, so
// that CTAs running at the same time share their L (rows) and U (columns) operands in L2.
template <int BN>
__host__ __device__ __forceinline__ void region_blocks_of(const Region& r, int64_t nts, int64_t& nbi, int64_t& nbj,
                                                          int64_t& i0, int64_t& i1, int64_t& j0, int64_t& j1) {
  region_clip(r, nts, i0, i1, j0, j1);
  nbi = (i1 - i0 + 1) / 2;
  nbj = (j1 - j0 + BN - 1) / BN;
}

template <int BN>
__device__ __forceinline__ bool tc_block(const UpdArgs& u, int64_t nts, int64_t e, int group, int64_t& I0,
                                         int64_t& J0, int& ni, int& nj) {
  for (int q = 0; q < u.nreg; ++q) {
    int64_t nbi, nbj, i0, i1, j0, j1;
    region_blocks_of<BN>(u.reg[q], nts, nbi, nbj, i0, i1, j0, j1);
    if (e < nbi * nbj) {
      const int64_t gsize = (int64_t)group * nbj;
      const int64_t g = e / gsize, first = g * group;
      const int64_t gs = nbi - first < group ? nbi - first : group;
      const int64_t loc = e % gsize;
      const int64_t bi = first + loc % gs, bj = loc / gs;
      I0 = i0 + 2 * bi;
      J0 = j0 + BN * bj;
      ni = (int)((i1 - I0) < 2 ? (i1 - I0) : 2);
      nj = (int)((j1 - J0) < BN ? (j1 - J0) : BN);
      return true;
    }
    e -= nbi * nbj;
  }
  return false;
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS, 1) k_lu_update_tc(const __grid_constant__ CUtensorMap tmap, TcArgs a) {
  using S = TcShape<BN>;
  constexpr int TC_STAGES = S::STAGES;
  constexpr uint32_t TC_STAGE_BYTES = S::STAGE_BYTES;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t full[TC_STAGES], empty[TC_STAGES], done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int s = blockIdx.y;
  const int64_t nts = a.np[s] / TB;
  int64_t I0, J0;
  int ni, nj;
  if (!tc_block<BN>(a.u, nts, blockIdx.x, a.group, I0, J0, ni, nj)) return;
  int64_t kk1 = a.u.kk1 < nts ? a.u.kk1 : nts;
  const int64_t kk0 = a.u.kk0;
  if (kk1 <= kk0) return;
  const int nchunks = (int)(2 * (kk1 - kk0));
  // dynamic shared memory base rounded up to 1024 B for the swizzle atoms
  unsigned char* stages = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int q = 0; q < TC_STAGES; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    mbar_init(&done, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(S::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = tmem_base;
  const int64_t toff = a.tile_off[s];
  // operand tiles (clamped to a valid tile when the block is ragged; results discarded)
  const int64_t Ia = I0, Ib = ni > 1 ? I0 + 1 : I0;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    for (int c = 0; c < nchunks; ++c) {
      const int st = c % TC_STAGES;
      if (c >= TC_STAGES && !mbar_wait(&empty[st], (uint32_t)(((c / TC_STAGES) - 1) & 1))) {
        abort_flag = 1;
        break;
      }
      const int64_t kk = kk0 + c / 2;
      const int x = (c & 1) * 32;
      unsigned char* sb = stages + (size_t)st * TC_STAGE_BYTES;
      mbar_expect_tx(&full[st], TC_STAGE_BYTES);
      const int zA0 = (int)(toff + Ia * nts + kk), zA1 = (int)(toff + Ib * nts + kk);
      tma_load_3d(sb + 0 * TC_BOX_BYTES, &tmap, x, 0, zA0, &full[st]);    // A_re rows 0..63
      tma_load_3d(sb + 1 * TC_BOX_BYTES, &tmap, x, 0, zA1, &full[st]);    // A_re rows 64..127
      tma_load_3d(sb + 2 * TC_BOX_BYTES, &tmap, x, 64, zA0, &full[st]);   // A_im
      tma_load_3d(sb + 3 * TC_BOX_BYTES, &tmap, x, 64, zA1, &full[st]);
#pragma unroll
      for (int q = 0; q < BN; ++q) {                                      // B_re, B_im: 64 columns per tile
        const int zB = (int)(toff + kk * nts + J0 + (q < nj ? q : 0));
        tma_load_3d(sb + (4 + q) * TC_BOX_BYTES, &tmap, x, 0, zB, &full[st]);
        tma_load_3d(sb + (4 + BN + q) * TC_BOX_BYTES, &tmap, x, 64, zB, &full[st]);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    const uint32_t id_pos = idesc_tf32<BN>(false), id_neg = idesc_tf32<BN>(true);
    const uint32_t d_re = tbase, d_im = tbase + 64 * BN;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      const int st = c % TC_STAGES;
      if (!mbar_wait(&full[st], (uint32_t)((c / TC_STAGES) & 1))) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sb = smem_u32(stages + (size_t)st * TC_STAGE_BYTES);
      const uint64_t are = sdesc(sb), aim = sdesc(sb + 2 * TC_BOX_BYTES);
      const uint64_t bre = sdesc(sb + 4 * TC_BOX_BYTES), bim = sdesc(sb + (4 + BN) * TC_BOX_BYTES);
#pragma unroll
      for (int k8 = 0; k8 < 4; ++k8) {  // K = 8 TF32 = 32 B per instruction
        const uint64_t dk = (uint64_t)(k8 * 32) >> 4;
        const uint32_t first = (c == 0 && k8 == 0) ? 0u : 1u;
        mma_tf32(d_re, are + dk, bre + dk, id_pos, first);
        mma_tf32(d_re, aim + dk, bim + dk, id_neg, 1u);
        mma_tf32(d_im, are + dk, bim + dk, id_pos, first);
        mma_tf32(d_im, aim + dk, bre + dk, id_pos, 1u);
      }
      mma_commit(&empty[st]);
    }
    if (!ok) abort_flag = 1;
    mma_commit(&done);
  }
  __syncwarp();
  // ---------------- epilogue: all four warps
  const bool fin = mbar_wait(&done, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!fin || abort_flag) {
    if (tid == 0) atomicExch(&a.status[ST_ERR], DEV_TIMEOUT);
  } else {
    const int row = warp * 32 + lane;           // accumulator row = TMEM lane
    const int ti = row >> 6, li = row & 63;
    const int64_t I = I0 + ti;
#pragma unroll 1
    for (int cb = 0; cb < 2 * BN; ++cb) {        // 32-column chunks of the 64 BN complex columns
      float re[32], im[32];
      const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
      tmem_ld32(tbase + lane_off + cb * 32, re);
      tmem_ld32(tbase + lane_off + 64 * BN + cb * 32, im);
      const int tj = cb >> 1, lj0 = (cb & 1) * 32;
      const int64_t J = J0 + tj;
      if (ti >= ni || tj >= nj) continue;
      float* C = a.arena + (toff + I * nts + J) * 2 * TILE_PLANE;
      if (I >= J) {  // row-major planes: 32 contiguous floats per thread
        float4* cr = (float4*)(C + li * TB + lj0);
        float4* ci = (float4*)(C + TILE_PLANE + li * TB + lj0);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float4 x = cr[q], y = ci[q];
          x.x -= re[4 * q]; x.y -= re[4 * q + 1]; x.z -= re[4 * q + 2]; x.w -= re[4 * q + 3];
          y.x -= im[4 * q]; y.y -= im[4 * q + 1]; y.z -= im[4 * q + 2]; y.w -= im[4 * q + 3];
          cr[q] = x;
          ci[q] = y;
        }
      } else {       // column-major planes: lanes cover consecutive rows
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int64_t e = (int64_t)(lj0 + q) * TB + li;
          C[e] -= re[q];
          C[TILE_PLANE + e] -= im[q];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(S::TMEM_COLS));
}

// ------------------------------------------------------------------ triangular solves of a step
// With the step's diagonal block factored as L11 U11 and inverted into two scratch tiles
// (L11^{-1} row-major, U11^{-1} column-major), the tile solves are products:
//   below:  L_Ik = A_Ik U11^{-1}            (A_Ik row-major: M = rows of the tile, K-major)
//   right:  U_kJ^T = A_kJ^T L11^{-T}        (A_kJ column-major: its storage rows are the rows of
//                                            the transpose, K-major; the result lands in the
//                                            same storage positions)
// One item is two tiles of one side (M = 128), N = 64, K = 64, overwritten in place.  A launch
// covers the tiles below the diagonal (rows k+1 .. nts-1, when `lower`) and the tiles of row k
// in columns [ju0, ju1) (clipped to the subdomain).  The first `gl` CTAs of a subdomain take the
// lower side's items in turn (item x, x + gl, ...), the others the row's; each CTA keeps its
// side's inverse tile in shared memory and runs its items through a pipeline: warp 0 loads the
// next item's tiles with TMA while warp 1 issues the MMAs of the current one into one of two
// tensor-memory accumulators and warps 2-5 store the previous one (each reads its quarter of the
// 128 TMEM lanes).  Every wait is bounded; a timeout sets the device status flag, the roles stop,
// and the CTA waits for its own copies and MMAs in flight before it releases its memory.
struct TrsmArgs {
  const int64_t* np;
  const int64_t* tile_off;
  float* arena;
  int64_t scratch_base;   // first scratch tile: subdomain s uses scratch_base + LU_SCRATCH s + slot
  int k;
  int l_slot;             // scratch slot of L_kk^{-1} (U_kk^{-1} is in slot LU_SUB)
  int lower;              // solve the tiles below the diagonal
  int gl;                 // CTAs per subdomain on the lower side (blockIdx.x < gl); the rest take row k
  int ju0, ju1;           // columns of row k to solve
  int32_t* status;
};

constexpr int TRSM_THREADS = 192;                        // TMA, MMA, 4 epilogue warps
constexpr int TRSM_STAGES = 2;
constexpr uint32_t TRSM_A_BYTES = 8 * TC_BOX_BYTES;      // an item: [K half][A_re t0, A_re t1, A_im t0, A_im t1]
constexpr uint32_t TRSM_B_BYTES = 4 * TC_BOX_BYTES;      // the inverse: [K half][B_re, B_im]
constexpr size_t TRSM_SMEM = (size_t)TRSM_STAGES * TRSM_A_BYTES + TRSM_B_BYTES + 1024;
constexpr uint32_t TRSM_TMEM_COLS = 256;                 // two accumulators of 128 columns (D_re, D_im)
static_assert(TRSM_A_BYTES % 1024 == 0 && TRSM_B_BYTES % 1024 == 0 && TRSM_SMEM + 1024 <= 227 * 1024,
              "trsm staging");

__global__ void __launch_bounds__(TRSM_THREADS, 1) k_lu_trsm_tc(const __grid_constant__ CUtensorMap tmap, TrsmArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t bfull, full[TRSM_STAGES], empty[TRSM_STAGES], tfull[2], tempty[2];
  __shared__ uint32_t tmem_base;
  __shared__ int n_issued, n_mma;
  const int s = blockIdx.y;
  const int64_t nts = a.np[s] / TB;
  const int k = a.k;
  if (k >= nts) return;
  const bool lower = (int)blockIdx.x < a.gl;
  const int64_t first = lower ? k + 1 : a.ju0;
  const int64_t end = lower ? nts : (a.ju1 < nts ? a.ju1 : nts);
  const int64_t x = lower ? blockIdx.x : blockIdx.x - a.gl;
  const int64_t stride = lower ? a.gl : (int)gridDim.x - a.gl;
  const int64_t npairs = end > first ? (end - first + 1) / 2 : 0;
  const int nitems = x < npairs ? (int)((npairs - 1 - x) / stride + 1) : 0;
  if (nitems == 0) return;  // the same for every thread of the CTA
  const int64_t toff = a.tile_off[s];
  // arena tiles of item i (z1 == z0 when the item has one tile)
  auto item_tiles = [&](int i, int& z0, int& z1, bool& two) {
    const int64_t t0 = first + 2 * (x + (int64_t)i * stride);
    two = t0 + 1 < end;
    const int64_t t1 = two ? t0 + 1 : t0;
    z0 = (int)(lower ? toff + t0 * nts + k : toff + (int64_t)k * nts + t0);
    z1 = (int)(lower ? toff + t1 * nts + k : toff + (int64_t)k * nts + t1);
  };
  const int zB = (int)(a.scratch_base + (int64_t)LU_SCRATCH * s + (lower ? LU_SUB : a.l_slot));
  unsigned char* st = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sB = st + (size_t)TRSM_STAGES * TRSM_A_BYTES;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    mbar_init(&bfull, 1);
    for (int q = 0; q < TRSM_STAGES; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&tfull[q], 1);
      mbar_init(&tempty[q], 4);
    }
    n_issued = 0;
    n_mma = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TRSM_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = tmem_base;
  if (warp == 0) {
    // ---------------- TMA: the inverse once, then the items' tiles through the stages
    if (lane == 0) {
      mbar_expect_tx(&bfull, TRSM_B_BYTES);
      for (int h = 0; h < 2; ++h) {
        tma_load_3d(sB + (2 * h) * TC_BOX_BYTES, &tmap, 32 * h, 0, zB, &bfull);
        tma_load_3d(sB + (2 * h + 1) * TC_BOX_BYTES, &tmap, 32 * h, 64, zB, &bfull);
      }
      int n = 0;
      for (int i = 0; i < nitems; ++i) {
        const int b = i % TRSM_STAGES;
        const uint32_t round = (uint32_t)(i / TRSM_STAGES);
        if (i >= TRSM_STAGES && !mbar_wait(&empty[b], (round & 1u) ^ 1u)) {
          atomicExch(&a.status[ST_ERR], DEV_TIMEOUT);
          break;
        }
        int z0, z1;
        bool two;
        item_tiles(i, z0, z1, two);
        unsigned char* sa = st + (size_t)b * TRSM_A_BYTES;
        mbar_expect_tx(&full[b], TRSM_A_BYTES);
        for (int h = 0; h < 2; ++h) {
          unsigned char* base = sa + (size_t)(4 * h) * TC_BOX_BYTES;
          tma_load_3d(base + 0 * TC_BOX_BYTES, &tmap, 32 * h, 0, z0, &full[b]);
          tma_load_3d(base + 1 * TC_BOX_BYTES, &tmap, 32 * h, 0, z1, &full[b]);
          tma_load_3d(base + 2 * TC_BOX_BYTES, &tmap, 32 * h, 64, z0, &full[b]);
          tma_load_3d(base + 3 * TC_BOX_BYTES, &tmap, 32 * h, 64, z1, &full[b]);
        }
        n = i + 1;
      }
      n_issued = n;
    }
  } else if (warp == 1) {
    // ---------------- MMA: item i into accumulator i % 2 once the epilogue has emptied it
    if (lane == 0) {
      const uint32_t id_pos = idesc_tf32<1>(false), id_neg = idesc_tf32<1>(true);
      int n = 0;
      if (!mbar_wait(&bfull, 0)) {
        atomicExch(&a.status[ST_ERR], DEV_TIMEOUT);
      } else {
        for (int i = 0; i < nitems; ++i) {
          const int b = i % TRSM_STAGES, d = i & 1;
          if (!mbar_wait(&full[b], (uint32_t)(i / TRSM_STAGES) & 1u) ||
              (i >= 2 && !mbar_wait(&tempty[d], ((uint32_t)(i >> 1) & 1u) ^ 1u))) {
            atomicExch(&a.status[ST_ERR], DEV_TIMEOUT);
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t d_re = tbase + 128u * d, d_im = d_re + 64;
          const uint32_t sa = smem_u32(st + (size_t)b * TRSM_A_BYTES), sb = smem_u32(sB);
          for (int h = 0; h < 2; ++h) {
            const uint64_t are = sdesc(sa + 4 * h * TC_BOX_BYTES), aim = sdesc(sa + (4 * h + 2) * TC_BOX_BYTES);
            const uint64_t bre = sdesc(sb + 2 * h * TC_BOX_BYTES), bim = sdesc(sb + (2 * h + 1) * TC_BOX_BYTES);
#pragma unroll
            for (int k8 = 0; k8 < 4; ++k8) {
              const uint64_t dk = (uint64_t)(k8 * 32) >> 4;
              const uint32_t acc = (h == 0 && k8 == 0) ? 0u : 1u;
              mma_tf32(d_re, are + dk, bre + dk, id_pos, acc);
              mma_tf32(d_re, aim + dk, bim + dk, id_neg, 1u);
              mma_tf32(d_im, are + dk, bim + dk, id_pos, acc);
              mma_tf32(d_im, aim + dk, bre + dk, id_pos, 1u);
            }
          }
          mma_commit(&empty[b]);  // the stage may be refilled once these MMAs have read it
          mma_commit(&tfull[d]);  // the accumulator is complete
          n = i + 1;
        }
      }
      n_mma = n;
    }
  } else {
    // ---------------- epilogue: the rows of TMEM lane quarter q, stored over the item's tiles
    const int q = warp & 3;
    const int row = q * 32 + lane, ti = row >> 6, li = row & 63;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    for (int i = 0; i < nitems; ++i) {
      const int d = i & 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&tfull[d], (uint32_t)(i >> 1) & 1u));
      if (!ok) {
        if (lane == 0) atomicExch(&a.status[ST_ERR], DEV_TIMEOUT);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int z0, z1;
      bool two;
      item_tiles(i, z0, z1, two);
      float* T = a.arena + (size_t)(ti ? z1 : z0) * 2 * TILE_PLANE;
#pragma unroll 1
      for (int cb = 0; cb < 2; ++cb) {
        float re[32], im[32];
        tmem_ld32(tbase + lane_off + 128u * d + cb * 32, re);
        tmem_ld32(tbase + lane_off + 128u * d + 64 + cb * 32, im);
        if (ti == 1 && !two) continue;
        float4* cr = (float4*)(T + li * TB + cb * 32);
        float4* ci = (float4*)(T + TILE_PLANE + li * TB + cb * 32);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          cr[e] = make_float4(re[4 * e], re[4 * e + 1], re[4 * e + 2], re[4 * e + 3]);
          ci[e] = make_float4(im[4 * e], im[4 * e + 1], im[4 * e + 2], im[4 * e + 3]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[d]);
    }
  }
  __syncthreads();
  // After a timeout: the copies and MMAs still in flight must land before the memory goes (the
  // last phase of each stage and accumulator; earlier phases completed before it).  Without one,
  // these waits return at once.
  if (tid == 0) {
    const uint64_t lim = drain_limit(WAIT_NS_DEFAULT);
    mbar_wait(&bfull, 0, false, lim);
    for (int i = n_issued - TRSM_STAGES > 0 ? n_issued - TRSM_STAGES : 0; i < n_issued; ++i)
      mbar_wait(&full[i % TRSM_STAGES], (uint32_t)(i / TRSM_STAGES) & 1u, false, lim);
    for (int i = n_mma - 2 > 0 ? n_mma - 2 : 0; i < n_mma; ++i) mbar_wait(&tfull[i & 1], (uint32_t)(i >> 1) & 1u, false, lim);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TRSM_TMEM_COLS));
}

// ------------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

static_assert(sizeof(CUtensorMap) == sizeof(((oras_handle*)nullptr)->tc_map), "tensor map storage");

// Tensor map over the arena viewed as [tiles][2 planes x 64 rows][64 floats].
static bool make_map(const oras_handle* h, CUtensorMap* map) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const int64_t tiles = h->mesh.arena_tiles + (int64_t)LU_SCRATCH * h->mesh.nsub;
  if (tiles >= (int64_t(1) << 31)) return false;
  cuuint64_t dims[3] = {64, 128, (cuuint64_t)tiles};
  cuuint64_t strides[2] = {64 * sizeof(float), 128 * 64 * sizeof(float)};
  cuuint32_t box[3] = {32, 64, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, h->dev.arena, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool tc_update_available(oras_handle* h) {
  if (h->dev.factor_bits != 32 || !h->dev.arena) return false;
  const int64_t tiles = h->mesh.arena_tiles + (int64_t)LU_SCRATCH * h->mesh.nsub;
  if (h->tc_map_base != h->dev.arena || h->tc_map_tiles != tiles) {
    CUtensorMap map;
    h->tc_map_ok = make_map(h, &map);
    std::memcpy(h->tc_map, &map, sizeof(map));
    h->tc_map_base = h->dev.arena;
    h->tc_map_tiles = tiles;
  }
  return h->tc_map_ok;
}

// CTAs per subdomain of a tile-solve launch: about two per SM over all subdomains, split between
// the lower side and row k by their item counts, never more than the items.
static void trsm_grid(int nsub, int64_t nbl, int64_t nbu, int* gl, int* gu) {
  static int sms = 0;
  if (!sms) {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    sms = (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0) ? n : 148;
  }
  const int64_t cap = std::max<int64_t>(1, (2 * (int64_t)sms + nsub - 1) / nsub);
  int64_t l = 0, u = 0;
  if (nbl > 0) l = std::min<int64_t>(nbl, std::max<int64_t>(1, nbu > 0 ? cap * nbl / (nbl + nbu) : cap));
  if (nbu > 0) u = std::min<int64_t>(nbu, std::max<int64_t>(1, cap - l));
  *gl = (int)l;
  *gu = (int)u;
}

int launch_trsm_tc(oras_handle* h, int k, int max_nts, bool lower, int ju0, int ju1, int l_slot) {
  const auto& m = h->mesh;
  const auto& d = h->dev;
  const int64_t nbl = lower ? std::max<int64_t>(0, (max_nts - k - 1 + 1) / 2) : 0;
  const int64_t ue = std::min<int64_t>(ju1, max_nts);
  const int64_t nbu = ue > ju0 ? (ue - ju0 + 1) / 2 : 0;
  if (nbl + nbu <= 0) return 0;
  int gl = 0, gu = 0;
  trsm_grid(m.nsub, nbl, nbu, &gl, &gu);
  CUtensorMap map;
  std::memcpy(&map, h->tc_map, sizeof(map));
  TrsmArgs a;
  a.np = d.sub_np;
  a.tile_off = d.sub_tile_off;
  a.arena = (float*)d.arena;
  a.scratch_base = m.arena_tiles;
  a.k = k;
  a.l_slot = l_slot;
  a.lower = lower ? 1 : 0;
  a.gl = gl;
  a.ju0 = ju0;
  a.ju1 = ju1;
  a.status = d.status;
  allow_max_smem((const void*)k_lu_trsm_tc);
  k_lu_trsm_tc<<<dim3((unsigned)(gl + gu), m.nsub), TRSM_THREADS, TRSM_SMEM, d.stream>>>(map, a);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int BN>
static int64_t update_blocks(const UpdArgs& u, int max_nts) {
  int64_t blocks = 0;
  for (int q = 0; q < u.nreg; ++q) {
    int64_t nbi, nbj, i0, i1, j0, j1;
    region_blocks_of<BN>(u.reg[q], max_nts, nbi, nbj, i0, i1, j0, j1);
    blocks += nbi * nbj;
  }
  return blocks;
}

template <int BN>
static void launch_update_shape(oras_handle* h, const UpdArgs& u, int64_t blocks, int cls) {
  const auto& d = h->dev;
  CUtensorMap map;
  std::memcpy(&map, h->tc_map, sizeof(map));
  TcArgs a;
  a.np = d.sub_np;
  a.tile_off = d.sub_tile_off;
  a.arena = (float*)d.arena;
  a.u = u;
  a.status = d.status;
  a.group = h->opt.lu_group > 0 ? h->opt.lu_group : TC_GROUP;
  allow_max_smem((const void*)k_lu_update_tc<BN>);
  int pb = prof_begin(h);
  k_lu_update_tc<BN><<<dim3((unsigned)blocks, h->mesh.nsub), TC_THREADS, TcShape<BN>::SMEM, d.stream>>>(map, a);
  prof_end(h, cls, pb, 1);
  count_launches(1);
}

// Regions one tile column wide (the column a left-looking panel step brings up to date) take
// the 128 x 64 output blocks; wider ones the 128 x 256 blocks.
int launch_update_tc(oras_handle* h, const UpdArgs& u, int max_nts, int cls) {
  int64_t width = 0;
  for (int q = 0; q < u.nreg; ++q) {
    int64_t i0, i1, j0, j1;
    region_clip(u.reg[q], max_nts, i0, i1, j0, j1);
    if (j1 - j0 > width) width = j1 - j0;
  }
  if (width <= 1) {
    const int64_t blocks = update_blocks<1>(u, max_nts);
    if (blocks > 0) launch_update_shape<1>(h, u, blocks, cls);
  } else {
    const int64_t blocks = update_blocks<4>(u, max_nts);
    if (blocks > 0) launch_update_shape<4>(h, u, blocks, cls);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace oras
