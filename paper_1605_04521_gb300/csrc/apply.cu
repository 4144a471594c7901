// ORAS preconditioner apply (Sec. 4):  z = sum_s R_s^T D_s A_s^{-1} R_s v
// with A_s^{-1} = U_s^{-1} L_s^{-1} P_s from the batched LU.  One cluster of two CTAs per
// subdomain (body in apply.cuh); one launch serves a group of up to KR right-hand sides, so the
// factor arena is streamed once per group.  When two CTAs per subdomain leave SMs idle and the
// largest subdomains would set the apply's time (one CTA streams at a rate set by the bytes its
// ring keeps in flight), those subdomains get clusters of four CTAs in a second launch on a side
// stream, concurrent with the two-CTA launch of the others (fork and join with events).  The local vectors live in shared memory when they fit
// next to the tile ring, else in a global scratch slice.  With the Boolean partition of unity
// every global DOF is written by exactly one subdomain (no atomics); OAS (no D_s) accumulates with
// atomics.
#include <algorithm>

#include "apply.cuh"

namespace oras {

size_t apply_yglob_bytes(const oras_handle* h, int kr);
// tensor-core passes (apply_tc.cu)
bool apply_tc_available(const oras_handle* h);
size_t apply_tc_ybytes(const oras_handle* h, int kt);
int apply_tc_f64out(const oras_handle* h, const cplx* v, cplx* z, int k, int r0, int nr);
int apply_tc_f32out(const oras_handle* h, const cplx* v, void* z, int k, int r0, int nr);
int apply_tc_passes(int nr);

// Columns from which a call takes the tensor-core passes (FP32 factors, ORAS_APPLY_AUTO).
constexpr int APPLY_TC_MIN_K = 8;

static bool use_tc(const oras_handle* h, int k) {
  return k >= APPLY_TC_MIN_K && h->opt.factor_bits == 32 && h->opt.apply_engine != ORAS_APPLY_CUDA_CORES;
}

// subs: the subdomain of each cluster (nullptr: cluster q takes subdomain q)
template <typename R, typename ZT, int KR>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(APPLY_THREADS, 1)
    k_apply(ApplyGeom a, const int32_t* subs, int k, int r0, int nr, void* yglob, const cplx* __restrict__ v,
            ZT* __restrict__ z) {
  const int q = blockIdx.x / 2;
  apply_cluster<R, ZT, KR, 2>(a, subs ? subs[q] : q, v, k, z, k, r0, nr, (CT<R>*)yglob);
}

template <typename R, typename ZT, int KR>
__global__ void __cluster_dims__(4, 1, 1) __launch_bounds__(APPLY_THREADS, 1)
    k_apply4(ApplyGeom a, const int32_t* subs, int k, int r0, int nr, void* yglob, const cplx* __restrict__ v,
             ZT* __restrict__ z) {
  apply_cluster<R, ZT, KR, 4>(a, subs[blockIdx.x / 4], v, k, z, k, r0, nr, (CT<R>*)yglob);
}

constexpr size_t SMEM_LIMIT = 227 * 1024 - 2048;  // opt-in shared memory per block less the static part
constexpr size_t SMEM_PAIR = 112 * 1024;          // dynamic shared memory that lets two CTAs share an SM
constexpr int APPLY_PAIR_STAGES = 3;              // ring depth of such a CTA

// Ring depth and dynamic shared memory for KR right-hand sides per pass and G CTAs per subdomain,
// for subdomains of padded order up to max_np; y in shared memory when `allow_smem_y` and it fits
// next to a ring of at least 2 stages.  `paired`: the launch has more CTAs than SMs (they run in
// waves); then, for one right-hand side per pass (a CTA's registers leave room for a second one
// only there) and if a 3-stage ring and y fit in SMEM_PAIR, two CTAs share each SM, so one
// CTA's gather, scatter and ring fill overlap the other's stream.
template <typename R, int KR, int G>
static void apply_config(int64_t max_np, bool allow_smem_y, int* S, size_t* smem, bool* y_smem, bool paired = false) {
  using Sm = ApplySmem<R, KR, G>;
  const int64_t ystrips = (max_np / TB + G - 1) / G;
  if (paired && KR == 1 && allow_smem_y && Sm::total(APPLY_PAIR_STAGES, ystrips) <= SMEM_PAIR) {
    *S = APPLY_PAIR_STAGES;
    *smem = Sm::total(APPLY_PAIR_STAGES, ystrips);
    *y_smem = true;
    return;
  }
  if (allow_smem_y)
    for (int q = 8; q >= 2; --q)
      if (Sm::total(q, ystrips) <= SMEM_LIMIT) {
        *S = q;
        *smem = Sm::total(q, ystrips);
        *y_smem = true;
        return;
      }
  int q = 8;
  while (q > 2 && Sm::total(q, 0) > SMEM_LIMIT) --q;
  *S = q;
  *smem = Sm::total(q, 0);
  *y_smem = false;
}

// The 2-CTA launch of an apply pass has more CTAs than the SMs hold (one per SM otherwise).
static bool apply_paired(const oras_handle* h) {
  return h->dev.num_sms > 0 && 2 * (int64_t)(h->mesh.nsub - h->dev.apply_n4) > h->dev.num_sms;
}

ApplyGeom apply_geom(const oras_handle* h) {
  const auto& d = h->dev;
  ApplyGeom a;
  a.ns = d.sub_ns; a.np = d.sub_np; a.np_off = d.sub_np_off; a.ns_off = d.sub_ns_off;
  a.tile_off = d.sub_tile_off; a.inv_off = d.sub_inv_off;
  a.gidx = d.gidx; a.sub_dofs = d.sub_dofs; a.pou = d.sub_pou;
  a.arena = d.arena; a.dinv = d.dinv;
  a.weights = h->opt.weights;
  a.stages = 2;
  a.status = d.status;
  a.wait_ns = wait_limit_ns(h);
  return a;
}

// Right-hand sides per pass for the next group of `rem` (fewest passes, then the smallest KR).
static int group_kr(int rem, int maxkr) {
  int kr = 1;
  while (kr < maxkr && kr < rem) kr *= 2;
  return kr;
}

// Largest padded order among the subdomains that take G CTAs (0: none).
static int64_t group_max_np(const oras_handle* h, int G) {
  const auto& d = h->dev;
  if (d.apply_n4 == 0) return G == 2 ? h->mesh.max_np : 0;
  return G == 4 ? d.apply_np4 : d.apply_np2;
}

template <typename R, typename ZT, int KR>
static int apply_group(const oras_handle* h, const cplx* v, ZT* z, int k, int r0, int nr) {
  const auto& m = h->mesh;
  const auto& d = h->dev;
  const int n4 = d.apply_n4;
  void* yb = nullptr;
  ApplyGeom a2 = apply_geom(h), a4 = apply_geom(h);
  size_t smem2 = 0, smem4 = 0;
  bool ys2 = true, ys4 = true;
  if (m.nsub > n4) apply_config<R, KR, 2>(group_max_np(h, 2), true, &a2.stages, &smem2, &ys2, apply_paired(h));
  if (n4 > 0) apply_config<R, KR, 4>(group_max_np(h, 4), true, &a4.stages, &smem4, &ys4);
  if (!ys2 || !ys4) {
    if (!d.ybuf || d.ybuf_bytes < apply_yglob_bytes(h, KR)) return -1;
    yb = d.ybuf;
  }
  allow_max_smem((const void*)k_apply<R, ZT, KR>);
  if (n4 == 0) {  // one launch, two CTAs per subdomain
    k_apply<R, ZT, KR><<<2 * m.nsub, APPLY_THREADS, smem2, d.stream>>>(a2, nullptr, k, r0, nr, ys2 ? nullptr : yb, v, z);
    return 0;
  }
  // the largest subdomains (the first n4 of apply_subs) on the side stream, four CTAs each
  allow_max_smem((const void*)k_apply4<R, ZT, KR>);
  if (cudaEventRecord(h->apply_fork, d.stream) != cudaSuccess ||
      cudaStreamWaitEvent(h->apply_side, h->apply_fork, 0) != cudaSuccess)
    return -1;
  k_apply4<R, ZT, KR><<<4 * n4, APPLY_THREADS, smem4, h->apply_side>>>(a4, d.apply_subs, k, r0, nr,
                                                                       ys4 ? nullptr : yb, v, z);
  if (m.nsub > n4)
    k_apply<R, ZT, KR><<<2 * (m.nsub - n4), APPLY_THREADS, smem2, d.stream>>>(a2, d.apply_subs + n4, k, r0, nr,
                                                                             ys2 ? nullptr : yb, v, z);
  if (cudaEventRecord(h->apply_join, h->apply_side) != cudaSuccess ||
      cudaStreamWaitEvent(d.stream, h->apply_join, 0) != cudaSuccess)
    return -1;
  return 0;
}

template <typename R, typename ZT>
static int apply_t(const oras_handle* h, const cplx* v, ZT* z, int k) {
  const auto& m = h->mesh;
  const auto& d = h->dev;
  if (h->opt.weights != ORAS_WEIGHTS_POU) cudaMemsetAsync(z, 0, sizeof(ZT) * m.ndof * k, d.stream);
  if constexpr (sizeof(R) == 4) {
    if (use_tc(h, k) && apply_tc_available(h)) {
      int n;
      if constexpr (sizeof(ZT) == sizeof(cplx)) n = apply_tc_f64out(h, v, (cplx*)z, k, 0, k);
      else n = apply_tc_f32out(h, v, (void*)z, k, 0, k);
      if (n < 0) return -1;
      count_launches(0);
      return cudaGetLastError() == cudaSuccess ? 0 : -1;
    }
  }
  const int maxkr = sizeof(R) == 4 ? APPLY_MAX_KR_F32 : APPLY_MAX_KR_F64;
  int launches = 0, rc = 0;
  for (int r0 = 0; r0 < k && rc == 0;) {
    const int kr = group_kr(k - r0, maxkr), nr = std::min(kr, k - r0);
    if (kr == 1) rc = apply_group<R, ZT, 1>(h, v, z, k, r0, nr);
    else if (kr == 2) rc = apply_group<R, ZT, 2>(h, v, z, k, r0, nr);
    else if constexpr (sizeof(R) == 4) rc = apply_group<R, ZT, 4>(h, v, z, k, r0, nr);
    r0 += nr;
    launches += h->dev.apply_n4 > 0 ? 2 : 1;
  }
  count_launches(launches);
  if (rc) return rc;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// z (FP64 complex [N][k]) = M^{-1} v
int launch_apply_f64out(const oras_handle* h, const cplx* v, cplx* z, int k) {
  return h->dev.factor_bits == 64 ? apply_t<double, cplx>(h, v, z, k) : apply_t<float, cplx>(h, v, z, k);
}
// z (FP32 complex [N][k]) = M^{-1} v, FP32 factors only
int launch_apply_f32out(const oras_handle* h, const cplx* v, void* z, int k) {
  return apply_t<float, CT<float>>(h, v, (CT<float>*)z, k);
}

// Number of arena passes for k right-hand sides (each pass is one launch, or two when the largest
// subdomains take four CTAs).
int apply_passes(const oras_handle* h, int k) {
  if (use_tc(h, k) && apply_tc_available(h)) return apply_tc_passes(k);
  const int maxkr = h->dev.factor_bits == 64 ? APPLY_MAX_KR_F64 : APPLY_MAX_KR_F32;
  int n = 0;
  for (int r0 = 0; r0 < k; ++n) r0 += std::min(group_kr(k - r0, maxkr), k - r0);
  return n;
}

template <typename R, int KR>
static size_t yglob_bytes_kr(const oras_handle* h) {
  int S;
  size_t smem;
  bool y_smem = true, y4 = true;
  if (h->mesh.nsub > h->dev.apply_n4)
    apply_config<R, KR, 2>(group_max_np(h, 2), true, &S, &smem, &y_smem, apply_paired(h));
  if (h->dev.apply_n4 > 0) apply_config<R, KR, 4>(group_max_np(h, 4), true, &S, &smem, &y4);
  if (y_smem && y4) return 0;
  int64_t total = 0;
  for (int s = 0; s < h->mesh.nsub; ++s) total += h->mesh.sub_np[s];
  return (size_t)total * KR * sizeof(CT<R>);
}

// Global scratch for the local vectors when a group of kr right-hand sides runs (0: shared memory).
size_t apply_yglob_bytes(const oras_handle* h, int kr) {
  if (h->opt.factor_bits == 64) return kr <= 1 ? yglob_bytes_kr<double, 1>(h) : yglob_bytes_kr<double, 2>(h);
  if (kr <= 1) return yglob_bytes_kr<float, 1>(h);
  if (kr == 2) return yglob_bytes_kr<float, 2>(h);
  return yglob_bytes_kr<float, 4>(h);
}

// Largest scratch any group of a k-vector apply needs (the tensor-core passes keep their y strips
// in global memory: at most 32 columns per pass, complex FP32).
size_t apply_yglob_bytes_for(const oras_handle* h, int k) {
  const int maxkr = h->opt.factor_bits == 64 ? APPLY_MAX_KR_F64 : APPLY_MAX_KR_F32;
  size_t b = 0;
  if (use_tc(h, k)) b = apply_tc_ybytes(h, k > 16 ? 32 : (k > 8 ? 16 : 8));
  for (int r0 = 0; r0 < k;) {
    const int kr = group_kr(k - r0, maxkr);
    b = std::max(b, apply_yglob_bytes(h, kr));
    r0 += std::min(kr, k - r0);
  }
  return b;
}

// Shared-memory configuration for the allocation-free variant (local vectors in global memory).
void apply_noalloc_config(const oras_handle* h, int* S, size_t* smem) {
  bool y_smem;
  if (h->dev.factor_bits == 64) apply_config<double, 1, 2>(h->mesh.max_np, false, S, smem, &y_smem);
  else apply_config<float, 1, 2>(h->mesh.max_np, false, S, smem, &y_smem);
}

// Which subdomains take four CTAs: with one CTA per SM, a subdomain's apply time is about its
// factor bytes over the CTAs streaming it.  When two CTAs per subdomain fit on the SMs in one
// wave, the largest subdomains get four CTAs while the SMs last, as many as lower the largest
// remaining time (bytes / CTAs), and no more.  Fills `order` (the subdomains, four-CTA ones
// first, each part by decreasing size) and returns how many take four CTAs.
int plan_apply_groups(const oras_handle* h, int num_sms, std::vector<int32_t>& order) {
  const auto& m = h->mesh;
  order.resize(m.nsub);
  for (int s = 0; s < m.nsub; ++s) order[s] = s;
  std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return m.sub_np[x] > m.sub_np[y]; });
  if (m.nsub < 1 || 2 * (int64_t)m.nsub > num_sms) return 0;
  auto cost = [&](int n4) {  // the largest (np^2 / CTAs) over the subdomains
    double c = 0.0;
    if (n4 > 0) c = (double)m.sub_np[order[0]] * m.sub_np[order[0]] / 4.0;
    if (n4 < m.nsub) c = std::max(c, (double)m.sub_np[order[n4]] * m.sub_np[order[n4]] / 2.0);
    return c;
  };
  int best = 0;
  for (int n4 = 1; n4 <= m.nsub && 2 * (int64_t)(m.nsub + n4) <= num_sms; ++n4)
    if (cost(n4) < 0.9 * cost(best)) best = n4;
  return best;
}

}  // namespace oras
