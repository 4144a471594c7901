// C ABI of the ORAS-FGMRES solver: handle lifecycle, device upload, numeric set-up (element
// matrices, A, A_s, batched LU) and the right-preconditioned FGMRES(m) driver (Sec. 4-5).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <map>
#include <mutex>

#include "internal.h"

namespace oras {
// kernels (assemble.cu, lu.cu, apply.cu, krylov.cu)
int launch_element(const oras_handle* h, double k0);
int launch_faces(const oras_handle* h);
int launch_global_rows(const oras_handle* h, double k0);
int launch_local_rows(const oras_handle* h, double k0);
int launch_dipole(const oras_handle* h, const double* x0, const double* dir, cplx* b, int* found);
void launch_mask_fixed(const oras_handle* h, cplx* v, int k);
int launch_port(const oras_handle* h, const double* o, const double* u, const double* v, double beta, int load,
                const double* qs, const double* qw, int nq, const uint8_t* inport, cplx* pface, double* nface,
                cplx* out, double* norm_d);
int launch_port_dots(const oras_handle* h, int64_t nd, const int32_t* dofs, const cplx* p, const cplx* x, int k,
                     const double* norm_d, cplx* S);
int launch_plane(const oras_handle* h, const double* dvec, const oras_complex* pvec, double k0,
                 const double* qs, const double* qw, int nq, cplx* bface, cplx* b);
int launch_lu(oras_handle* h);
int lu_max_chunks(int64_t max_np, int factor_bits);
int launch_apply_f64out(const oras_handle* h, const cplx* v, cplx* z, int k);
int launch_apply_f32out(const oras_handle* h, const cplx* v, void* z, int k);
size_t apply_yglob_bytes_for(const oras_handle* h, int k);
int apply_passes(const oras_handle* h, int k);
int plan_apply_groups(const oras_handle* h, int num_sms, std::vector<int32_t>& order);
void launch_spmv_f64(const oras_handle* h, const cplx* x, cplx* y, int k);
void launch_spmv_f32(const oras_handle* h, const void* x, cplx* y, int k);
void launch_split_vals(const oras_handle* h);
void launch_to_internal_c64(const oras_handle* h, int k, const void* src, void* dst);
void launch_dot(const oras_handle* h, const cplx* a, const cplx* b, cplx* partials, int k);
void launch_mgs_step(const oras_handle* h, int k, int m, int i, int j, const cplx* Vi, const cplx* Vn, cplx* w,
                     const cplx* pin, cplx* pout, cplx* H);
void launch_mgs_finish(const oras_handle* h, int k, int m, int j, const cplx* w, cplx* Vn, const cplx* pin,
                       cplx* H, double* cs, cplx* sn, cplx* g, double* res);
void launch_hsolve(const oras_handle* h, int k, int m, int kk, const cplx* H, const cplx* g, const int32_t* active,
                   cplx* y);
void launch_xupdate_f64(const oras_handle* h, int k, int m, int kk, const cplx* Z, const cplx* y, cplx* x);
void launch_xupdate_f32(const oras_handle* h, int k, int m, int kk, const void* Z, const cplx* y, cplx* x);
void launch_residual(const oras_handle* h, int k, const cplx* b, cplx* r, cplx* partials);
void launch_norms(const oras_handle* h, int k, const cplx* partials, double* out);
void launch_restart(const oras_handle* h, int k, int m, const cplx* rv, const double* beta, const int32_t* active,
                    cplx* V0, cplx* g);
void launch_to_internal(const oras_handle* h, int k, const cplx* src, cplx* dst);
void launch_to_external(const oras_handle* h, int k, const cplx* src, cplx* dst);
int red_blocks();
int launch_wait_selftest(const oras_handle* h);
// shared with the block FGMRES driver (block_fgmres.cpp)
int ensure_ws(oras_handle* h, int k, int m);
int precond_to_z(oras_handle* h, const cplx* v, int k, int j);
void spmv_z(oras_handle* h, int k, int j, cplx* y);
int status_code(oras_handle* h, const int32_t* st);
int fgmres_block(oras_handle* h, int p, double tol, oras_info* info);
int gcrodr_solve(oras_handle* h, double tol, oras_info* info);
}  // namespace oras

using namespace oras;

static thread_local std::string g_err;
static std::atomic<int64_t> g_launches{0};

namespace oras {
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

uint64_t wait_limit_ns(const oras_handle* h) {
  return h->opt.wait_ms > 0 ? (uint64_t)h->opt.wait_ms * 1000000ull : 2000000000ull;
}

int prof_begin(const oras_handle* h) {
  if (!h->timing) return -1;
  if (h->ev_used == h->evpool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    h->evpool.push_back(e);
  }
  int i = (int)h->ev_used++;
  cudaEventRecord(h->evpool[i], h->dev.stream);
  return i;
}

void prof_end(const oras_handle* h, int cls, int begin, int launches) {
  if (begin < 0) return;
  int e = prof_begin(h);
  h->marks.insert(h->marks.end(), {cls, begin, e, launches});
}
}  // namespace oras

// Resolve the recorded event pairs into per-class totals (one synchronisation).
static void prof_resolve(oras_handle* h) {
  if (!h->timing || h->ev_used == 0) return;
  cudaEventSynchronize(h->evpool[h->ev_used - 1]);
  for (size_t q = 0; q + 3 < h->marks.size(); q += 4) {
    float ms = 0;
    cudaEventElapsedTime(&ms, h->evpool[h->marks[q + 1]], h->evpool[h->marks[q + 2]]);
    h->cls_ms[h->marks[q]] += ms;
    h->cls_n[h->marks[q]] += h->marks[q + 3];
  }
  h->marks.clear();
  h->ev_used = 0;
}

static void prof_clear(oras_handle* h) {
  for (int c = 0; c < KC_COUNT; ++c) h->cls_ms[c] = h->cls_n[c] = 0;
  h->marks.clear();
  h->ev_used = 0;
}

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) {                                                                       \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                                 \
      return e_ == cudaErrorMemoryAllocation ? ORAS_ERR_OUT_OF_MEMORY : ORAS_ERR_CUDA;              \
    }                                                                                              \
  } while (0)

// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the handle's stream): a
// free does not synchronise the device, so handles on other streams keep running.  Freed memory
// stays in the device's pool for the next handle (pool_malloc).
template <typename T>
static cudaError_t dalloc_s(T*& p, size_t n, cudaStream_t s) {
  if (p) { cudaFreeAsync(p, s); p = nullptr; }
  if (n == 0) n = 1;
  return pool_malloc((void**)&p, n * sizeof(T), s);
}
template <typename T>
static void dfree_s(T*& p, cudaStream_t s) {
  if (p) cudaFreeAsync((void*)p, s);
  p = nullptr;
}
#define dalloc(p, n) dalloc_s(p, n, d.stream)
template <typename T>
static cudaError_t dput(T*& p, const std::vector<T>& v, cudaStream_t s) {
  cudaError_t e = dalloc_s(p, v.size(), s);
  if (e != cudaSuccess) return e;
  if (!v.empty()) e = cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
  return e;
}

static void dfree_all(Device& d) {
  void* ptrs[] = {d.xyz, d.st, d.dofmap, d.tinc_ptr, d.tinc, d.if_tet0, d.if_lf0, d.if_tet1, d.if_dofs, d.if_beta, d.fixed,
                  d.finc_ptr, d.finc, d.rowptr, d.cols, d.sub_ns, d.sub_np, d.sub_ns_off, d.sub_tile_off,
                  d.sub_dofs, d.sub_pou, d.member, d.cm, d.ck, d.cs, d.fl, d.tc, d.ta, d.tm, d.eps, d.mu,
                  d.elem, d.fmat, d.vals, d.vals_df, d.arena, d.perm, d.gidx, d.sub_np_off, d.lu_cand, d.lu_cnt,
                  d.lu_ipiv, d.lu_diag, d.dinv, d.sub_inv_off, d.status, d.V, d.Zf, d.Zd, d.w, d.xk, d.bk, d.tmp, d.H, d.gcs, d.gsn,
                  d.g, d.red, d.scal, d.ybuf, d.io, d.apply_subs};
  for (void* p : ptrs)
    if (p) cudaFreeAsync(p, d.stream);
  cudaStreamSynchronize(d.stream);  // the frees have run: the memory is back in the pool
  d = Device();
}

// Small pinned host buffer for scalars read back during a solve, one per host thread, kept until
// the process exits (freeing pinned memory may synchronise the device).
static double* pinned_scratch() {
  thread_local double* p = nullptr;
  if (!p && cudaMallocHost((void**)&p, PINNED_SCRATCH_DOUBLES * sizeof(double)) != cudaSuccess) p = nullptr;
  return p;
}

// The apply's side stream and its fork/join events (once per handle).  Creating a stream takes
// device memory outside the stream-ordered pool, which may hold nearly all of it under a serving
// load: on failure the pool's unused memory is returned to the driver and the creation retried
// once.  Returns false (nothing left behind, no error pending) when that fails too.
static bool make_apply_side(oras_handle* h) {
  if (h->apply_side) return true;
  for (int attempt = 0; attempt < 2; ++attempt) {
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
        cudaEventCreateWithFlags(&e0, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) == cudaSuccess) {
      h->apply_side = st;
      h->apply_fork = e0;
      h->apply_join = e1;
      return true;
    }
    if (e0) cudaEventDestroy(e0);
    if (st) cudaStreamDestroy(st);
    cudaGetLastError();
    if (attempt == 0) {
      cudaStreamSynchronize(h->dev.stream);
      pool_trim(h->dev.device);
    }
  }
  return false;
}

static int upload(oras_handle* h) {
  auto& m = h->mesh;
  auto& d = h->dev;
  auto& T = h->tab;
  cudaStream_t s = d.stream;
  CK(cudaGetDevice(&d.device));
  CK(dput(d.xyz, m.xyz, s));
  CK(dput(d.st, m.st, s));
  CK(dput(d.dofmap, m.dofmap, s));
  CK(dput(d.tinc_ptr, m.tinc_ptr, s));
  CK(dput(d.tinc, m.tinc, s));
  CK(dput(d.if_tet0, m.if_tet0, s));
  CK(dput(d.if_lf0, m.if_lf0, s));
  CK(dput(d.if_tet1, m.if_tet1, s));
  CK(dput(d.if_dofs, m.if_dofs, s));
  if (!m.if_beta.empty()) CK(dput(d.if_beta, m.if_beta, s));
  if (!m.fixed.empty()) CK(dput(d.fixed, m.fixed, s));
  CK(dput(d.finc_ptr, m.finc_ptr, s));
  CK(dput(d.finc, m.finc, s));
  CK(dput(d.rowptr, m.rowptr, s));
  CK(dput(d.cols, m.cols, s));
  CK(dput(d.sub_ns, m.sub_ns, s));
  CK(dput(d.sub_np, m.sub_np, s));
  CK(dput(d.sub_ns_off, m.sub_ns_off, s));
  CK(dput(d.sub_tile_off, m.sub_tile_off, s));
  CK(dput(d.sub_dofs, m.sub_dofs, s));
  CK(dput(d.sub_pou, m.sub_pou, s));
  CK(dput(d.member, m.member, s));
  std::vector<int64_t> npoff(m.nsub + 1, 0);
  for (int q = 0; q < m.nsub; ++q) npoff[q + 1] = npoff[q] + m.sub_np[q];
  CK(dput(d.sub_np_off, npoff, s));
  {  // the apply's work split (which subdomains take four CTAs)
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, d.device));
    d.num_sms = nsm;
    std::vector<int32_t> order;
    d.apply_n4 = plan_apply_groups(h, nsm, order);
    // the split is an optimisation: without its side stream the apply keeps two CTAs each
    if (d.apply_n4 > 0 && !make_apply_side(h)) d.apply_n4 = 0;
    if (d.apply_n4 > 0) {
      CK(dput(d.apply_subs, order, s));
      d.apply_np4 = m.sub_np[order[0]];
      d.apply_np2 = d.apply_n4 < m.nsub ? m.sub_np[order[d.apply_n4]] : 0;
    }
  }
  CK(dput(d.cm, T.cm, s));
  CK(dput(d.ck, T.ck, s));
  CK(dput(d.cs, T.cs, s));
  std::vector<int32_t> fl(T.fl.begin(), T.fl.end()), ta(T.ta.begin(), T.ta.end()), tm(T.tm.begin(), T.tm.end());
  CK(dput(d.fl, fl, s));
  CK(dput(d.tc, T.tc, s));
  CK(dput(d.ta, ta, s));
  CK(dput(d.tm, tm, s));
  CK(dalloc(d.eps, m.nt));
  CK(dalloc(d.elem, (size_t)m.nt * m.nl * m.nl));
  CK(dalloc(d.fmat, (size_t)std::max<int64_t>(1, m.nif) * m.nfl * m.nfl));
  CK(dalloc(d.vals, m.cols.size()));
  CK(dalloc(d.vals_df, m.cols.size()));
  CK(dalloc(d.perm, npoff[m.nsub]));
  CK(dalloc(d.gidx, npoff[m.nsub]));
  CK(dalloc(d.status, 8));
  d.host_pinned = pinned_scratch();
  if (!d.host_pinned) { h->err = "pinned host scratch allocation failed"; return ORAS_ERR_OUT_OF_MEMORY; }
  d.uploaded = true;
  return ORAS_OK;
}

// Global scratch for the apply's local vectors when k right-hand sides go through it.
static int ensure_ybuf(oras_handle* h, int k) {
  auto& d = h->dev;
  const size_t yb = apply_yglob_bytes_for(h, k);
  if (yb <= d.ybuf_bytes) return ORAS_OK;
  dfree_s(d.ybuf, d.stream);
  d.ybuf_bytes = 0;
  CK(pool_malloc(&d.ybuf, yb, d.stream));
  d.ybuf_bytes = yb;
  return ORAS_OK;
}

static int alloc_factor_space(oras_handle* h, int bits) {
  auto& m = h->mesh;
  auto& d = h->dev;
  size_t el = bits == 64 ? 16 : 8;
  // the factor tiles, then LU_SCRATCH scratch tiles per subdomain (inverted diagonal blocks)
  size_t bytes = (size_t)(m.arena_tiles + (int64_t)LU_SCRATCH * m.nsub) * TB * TB * el;
  if (d.arena && d.factor_bits == bits && d.arena_bytes == bytes) return ORAS_OK;
  dfree_s(d.arena, d.stream);
  cudaError_t e = pool_malloc(&d.arena, bytes, d.stream);
  if (e != cudaSuccess) {
    h->err = "local-factor arena of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e);
    d.arena = nullptr;
    return e == cudaErrorMemoryAllocation ? ORAS_ERR_OUT_OF_MEMORY : ORAS_ERR_CUDA;
  }
  d.arena_bytes = bytes;
  d.factor_bits = bits;
  d.lu_max_chunks = lu_max_chunks(m.max_np, bits);
  int slots = 2 * d.lu_max_chunks + 16;
  CK(dalloc(d.lu_cand, (size_t)m.nsub * slots * TB));
  CK(dalloc(d.lu_cnt, (size_t)m.nsub * slots));
  CK(cudaMemsetAsync(d.lu_cnt, 0, (size_t)m.nsub * slots * sizeof(int32_t), d.stream));
  CK(dalloc(d.lu_ipiv, (size_t)m.nsub * (2 * TB * 2 + 1)));
  dfree_s(d.lu_diag, d.stream);
  CK(pool_malloc(&d.lu_diag, (size_t)m.nsub * TB * TB * el, d.stream));
  {
    std::vector<int64_t> inv_off(m.nsub + 1, 0);
    for (int q = 0; q < m.nsub; ++q) inv_off[q + 1] = inv_off[q] + m.sub_np[q] / TB;
    CK(dput(d.sub_inv_off, inv_off, d.stream));
    dfree_s(d.dinv, d.stream);
    d.dinv_bytes = (size_t)inv_off[m.nsub] * 2 * TB * TB * el;
    CK(pool_malloc(&d.dinv, d.dinv_bytes, d.stream));
  }
  dfree_s(d.ybuf, d.stream);
  d.ybuf_bytes = 0;
  return ensure_ybuf(h, 1);
}



// Device bytes that oras_factor plus an oras_solve of k right-hand sides allocate for this
// handle (the sizes of upload, alloc_factor_space, ensure_ybuf, ensure_ws and ensure_io), plus the
// stream-ordered pool's rounding (2 MiB per allocation).
int64_t footprint_bytes(const oras_handle* h, int k) {
  const auto& m = h->mesh;
  const auto& T = h->tab;
  const int bits = h->opt.factor_bits;
  const size_t el = bits == 64 ? 16 : 8;
  const int64_t N = m.ndof, mm = std::max(h->opt.restart, 1);
  auto vb = [](const auto& v) { return (int64_t)(v.size() * sizeof(v[0])); };
  int64_t total_np = 0, blocks = 0;
  for (int s = 0; s < m.nsub; ++s) {
    total_np += m.sub_np[s];
    blocks += m.sub_np[s] / TB;
  }
  int64_t b = 0;
  int nalloc = 0;
  auto add = [&](int64_t x) { b += std::max<int64_t>(x, 1); ++nalloc; };
  // upload
  for (int64_t x : {vb(m.xyz), vb(m.st), vb(m.dofmap), vb(m.tinc_ptr), vb(m.tinc), vb(m.if_tet0), vb(m.if_lf0),
                    vb(m.if_tet1), vb(m.if_dofs), vb(m.if_beta), vb(m.fixed), vb(m.finc_ptr), vb(m.finc), vb(m.rowptr), vb(m.cols),
                    vb(m.sub_ns), vb(m.sub_np), vb(m.sub_ns_off), vb(m.sub_tile_off), vb(m.sub_dofs),
                    vb(m.sub_pou), vb(m.member), (int64_t)(m.nsub + 1) * 8, vb(T.cm), vb(T.ck), vb(T.cs),
                    (int64_t)T.fl.size() * 4, vb(T.tc), (int64_t)T.ta.size() * 4, (int64_t)T.tm.size() * 4})
    add(x);
  add(m.nt * 16);                                                   // eps
  add(m.nt * 16);                                                   // mu (when given)
  add(m.nt * m.nl * m.nl * 16);                                     // element matrices
  add(std::max<int64_t>(1, m.nif) * m.nfl * m.nfl * 8);            // face matrices
  add((int64_t)m.cols.size() * 16);                                 // values of A
  add((int64_t)m.cols.size() * 16);                                 // values of A as FP32 pairs
  add(total_np * 4);                                                // perm
  add(total_np * 4);                                                // gidx
  add(8 * 4);                                                       // status
  // factor space
  const int slots = 2 * lu_max_chunks(m.max_np, bits) + 16;
  add((m.arena_tiles + (int64_t)LU_SCRATCH * m.nsub) * TB * TB * (int64_t)el);
  add((int64_t)m.nsub * slots * TB * 4);
  add((int64_t)m.nsub * slots * 4);
  add((int64_t)m.nsub * (2 * TB * 2 + 1) * 4);
  add((int64_t)m.nsub * TB * TB * (int64_t)el);
  add((int64_t)(m.nsub + 1) * 8);
  add(blocks * 2 * TB * TB * (int64_t)el);                          // inverted diagonal blocks
  add((int64_t)apply_yglob_bytes_for(h, std::max(k, 1)));
  add((int64_t)m.nsub * 4);                                         // apply work split
  // Krylov workspace and I/O staging
  const int64_t nk = N * std::max(k, 1), kk = std::max(k, 1);
  add(nk * (mm + 1) * 16);                                          // V
  add(nk * mm * (bits == 64 ? 16 : 8));                             // Z
  for (int q = 0; q < 4; ++q) add(nk * 16);                         // w, xk, bk, tmp
  add(kk * (mm + 1) * mm * 16);                                     // H
  add(kk * mm * 8);
  add(kk * mm * 16);
  add(kk * (mm + 1) * 16);
  add((int64_t)2 * red_blocks() * kk * 2 * 8);
  add((kk * 8 + kk * mm * 2 + 64) * 8);
  add(nk * 16);                                                     // io
  return b + (int64_t)nalloc * (2 << 20);
}

static int sync_status(oras_handle* h);

// Element matrices, A, local matrices and batched LU from the materials already on the device.
static int factor_device(oras_handle* h) {
  auto& d = h->dev;
  const double k0 = h->k0;
  CK(cudaMemsetAsync(d.status, 0, 8 * sizeof(int32_t), d.stream));
  {
    int b = prof_begin(h);
    if (launch_element(h, k0) || launch_faces(h)) CK(cudaGetLastError());
    prof_end(h, KC_ELEMENT, b, 2);
  }
  {
    int b = prof_begin(h);
    if (launch_global_rows(h, k0)) CK(cudaGetLastError());
    launch_split_vals(h);
    prof_end(h, KC_GLOBAL_ROWS, b, 2);
  }
  {
    int b = prof_begin(h);
    CK(cudaMemsetAsync(d.arena, 0, d.arena_bytes, d.stream));
    if (launch_local_rows(h, k0)) CK(cudaGetLastError());
    prof_end(h, KC_LOCAL_ROWS, b, 1);
  }
  if (launch_lu(h)) CK(cudaGetLastError());
  prof_resolve(h);
  return sync_status(h);
}


// Return code for the device status flags st[8] (read back from Device::status).
int oras::status_code(oras_handle* h, const int32_t* st) {
  if (st[ST_ERR] == DEV_SINGULAR) {
    h->err = "local matrix of subdomain " + std::to_string(st[ST_SUB]) + " has a zero pivot column";
    return ORAS_ERR_SINGULAR_LOCAL;
  }
  if (st[ST_ERR] == DEV_BADINDEX) {
    h->err = "internal index check failed in a device kernel (code " + std::to_string(st[ST_DETAIL]) +
             ", subdomain " + std::to_string(st[ST_SUB]) + ")";
    return ORAS_ERR_CUDA;
  }
  if (st[ST_ERR] == DEV_TIMEOUT) {
    h->err = "a bounded device wait gave up";
    return ORAS_ERR_DEVICE_TIMEOUT;
  }
  return ORAS_OK;
}

static int sync_status(oras_handle* h) {
  auto& d = h->dev;
  int32_t* st = (int32_t*)(d.host_pinned + PINNED_STATUS_OFF);
  CK(cudaMemcpyAsync(st, d.status, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, d.stream));
  CK(cudaStreamSynchronize(d.stream));
  return status_code(h, st);
}

extern "C" {

int32_t oras_abi_version(void) { return 3; }

const char* oras_last_error(const oras_handle* h) { return h ? h->err.c_str() : g_err.c_str(); }

int oras_create(const oras_problem* p, const oras_options* o, oras_handle** out) {
  if (!out) { g_err = "oras_create: out is NULL"; return ORAS_ERR_INVALID_ARG; }
  *out = nullptr;
  oras_handle* h = new (std::nothrow) oras_handle();
  if (!h) { g_err = "oras_create: host allocation failed"; return ORAS_ERR_OUT_OF_MEMORY; }
  if (o) h->opt = *o;
  if (h->opt.restart <= 0) h->opt.restart = 50;
  if (h->opt.max_iter <= 0) h->opt.max_iter = 5000;
  if (h->opt.factor_bits == 0) h->opt.factor_bits = 32;
  if (h->opt.factor_bits != 32 && h->opt.factor_bits != 64) {
    g_err = "oras_create: factor_bits must be 32 or 64";
    delete h;
    return ORAS_ERR_INVALID_ARG;
  }
  if (h->opt.weights != ORAS_WEIGHTS_POU && h->opt.weights != ORAS_WEIGHTS_NONE) {
    g_err = "oras_create: unknown weights";
    delete h;
    return ORAS_ERR_INVALID_ARG;
  }
  if (h->opt.transmission != ORAS_TRANSMISSION_IMPEDANCE && h->opt.transmission != ORAS_TRANSMISSION_DIRICHLET) {
    g_err = "oras_create: unknown transmission condition";
    delete h;
    return ORAS_ERR_INVALID_ARG;
  }
  if (h->opt.recycle < 0 || h->opt.recycle >= h->opt.restart) {
    g_err = "oras_create: recycle must be in [0, restart)";
    delete h;
    return ORAS_ERR_INVALID_ARG;
  }
  int rc;
  try {
    rc = host_setup(p, h->opt.overlap_kind, h->mesh, g_err);
    if (rc == ORAS_OK) h->tab = make_tables(p->r);
  } catch (const std::bad_alloc&) {
    g_err = "oras_create: host allocation failed";
    rc = ORAS_ERR_OUT_OF_MEMORY;
  } catch (const std::exception& e) {
    g_err = std::string("oras_create: ") + e.what();
    rc = ORAS_ERR_INVALID_ARG;
  }
  if (rc != ORAS_OK) { delete h; return rc; }
  *out = h;
  return ORAS_OK;
}

int oras_set_stream(oras_handle* h, void* stream) {
  if (!h) return ORAS_ERR_INVALID_ARG;
  h->dev.stream = (cudaStream_t)stream;
  return ORAS_OK;
}

int oras_set_timing(oras_handle* h, int32_t on) {
  if (!h) return ORAS_ERR_INVALID_ARG;
  h->timing = on != 0;
  return ORAS_OK;
}

int oras_timings(const oras_handle* h, double* t, int32_t n) {
  if (!h || !t) return ORAS_ERR_INVALID_ARG;
  for (int c = 0; c < KC_COUNT; ++c) {
    if (2 * c < n) t[2 * c] = h->cls_ms[c];
    if (2 * c + 1 < n) t[2 * c + 1] = h->cls_n[c];
  }
  return ORAS_OK;
}

int oras_reset_timings(oras_handle* h) {
  if (!h) return ORAS_ERR_INVALID_ARG;
  prof_clear(h);
  return ORAS_OK;
}

int64_t oras_launch_count(void) { return g_launches.load(); }

int oras_factor(oras_handle* h, const oras_complex* eps_r, const oras_complex* mu_r, double k0, int32_t mem) {
  if (!h || !eps_r) { if (h) h->err = "oras_factor: eps_r is NULL"; return ORAS_ERR_INVALID_ARG; }
  if (!(k0 > 0.0)) { h->err = "oras_factor: k0 must be positive"; return ORAS_ERR_INVALID_ARG; }
  auto& m = h->mesh;
  auto& d = h->dev;
  if (!d.uploaded) {
    int rc = upload(h);
    if (rc) return rc;
  }
  int rc = alloc_factor_space(h, h->opt.factor_bits);
  if (rc) return rc;
  cudaMemcpyKind kind = mem == ORAS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(d.eps, eps_r, sizeof(cplx) * m.nt, kind, d.stream));
  if (mu_r) {
    if (!d.mu) CK(dalloc(d.mu, m.nt));
    CK(cudaMemcpyAsync(d.mu, mu_r, sizeof(cplx) * m.nt, kind, d.stream));
  } else if (d.mu) {
    dfree_s(d.mu, d.stream);
  }
  h->k0 = k0;
  rc = factor_device(h);
  if (rc) return rc;
  h->factored = true;
  return ORAS_OK;
}

// Autotuner of the LU panel width: each candidate factorises the handle's current problem once
// (CUDA events on the handle's stream); the fastest is kept in the handle's options and cached
// for the process under the problem's shape, so later handles of the same shape reuse it.
static std::mutex g_tune_mu;
static std::map<std::vector<int64_t>, std::pair<int, int>> g_tune_cache;  // shape -> (panel, group)

int oras_autotune(oras_handle* h, int32_t* panel, double* ms, int32_t nms) {
  if (!h) return ORAS_ERR_INVALID_ARG;
  if (!h->factored) { h->err = "oras_autotune: call oras_factor first"; return ORAS_ERR_STATE; }
  static const int widths[] = {4, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192};
  static const int groups[] = {16, 32, 64};  // after the widths, which run with the default group 8
  constexpr int NW = sizeof(widths) / sizeof(widths[0]), NG = sizeof(groups) / sizeof(groups[0]);
  std::vector<int64_t> key = {h->opt.factor_bits, h->opt.lu_engine, h->mesh.nsub};
  key.insert(key.end(), h->mesh.sub_np.begin(), h->mesh.sub_np.end());
  std::pair<int, int> best(-1, -1);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) best = it->second;
  }
  for (int q = 0; q < nms && ms; ++q) ms[q] = -1.0;
  if (best.first < 0) {
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const oras_options keep = h->opt;
    double tbest = 1e300;
    auto time_one = [&](int w, int g, int slot) -> int {
      h->opt.lu_panel = w;
      h->opt.lu_group = g;
      cudaEventRecord(e0, h->dev.stream);
      int rc = factor_device(h);
      cudaEventRecord(e1, h->dev.stream);
      cudaEventSynchronize(e1);
      float t = 0.0f;
      cudaEventElapsedTime(&t, e0, e1);
      if (rc) return rc;
      if (ms && slot < nms) ms[slot] = t;
      if (t < tbest) { tbest = t; best = {w, g}; }
      return ORAS_OK;
    };
    int rc = ORAS_OK;
    for (int c = 0; c < NW && rc == ORAS_OK; ++c) rc = time_one(widths[c], 8, c);
    const int w = best.first;
    for (int c = 0; c < NG && rc == ORAS_OK; ++c) rc = time_one(w, groups[c], NW + c);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
      h->opt = keep;
      return rc;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
  }
  h->opt.lu_panel = best.first;
  h->opt.lu_group = best.second;
  if (panel) *panel = best.first;
  return factor_device(h);  // leave the factors of the chosen shape
}

int32_t oras_lu_group(const oras_handle* h) { return h ? h->opt.lu_group : -1; }


int oras_setup(const oras_problem* p, const oras_options* o, oras_handle** out) {
  int rc = oras_create(p, o, out);
  if (rc) return rc;
  rc = oras_factor(*out, p->eps_r, p->mu_r, p->k0, ORAS_MEM_HOST);
  if (rc) {
    g_err = (*out)->err;
    oras_destroy(*out);
    *out = nullptr;
  }
  return rc;
}

void oras_destroy(oras_handle* h) {
  if (!h) return;
  for (auto e : h->evpool) cudaEventDestroy(e);
  for (auto g : h->step_graph)
    if (g) cudaGraphExecDestroy(g);
  if (h->apply_side) {
    cudaStreamSynchronize(h->apply_side);
    cudaStreamDestroy(h->apply_side);
  }
  if (h->apply_fork) cudaEventDestroy(h->apply_fork);
  if (h->apply_join) cudaEventDestroy(h->apply_join);
  if (h->dev.uploaded) {
    cudaStreamSynchronize(h->dev.stream);
    if (h->rc_U) cudaFreeAsync(h->rc_U, h->dev.stream);
    dfree_all(h->dev);
  } else if (h->rc_U) {
    cudaFree(h->rc_U);
  }
  delete h;
}

int oras_wait_selftest(oras_handle* h, int32_t* detail) {
  if (!h) return ORAS_ERR_INVALID_ARG;
  if (!h->dev.uploaded) { h->err = "oras_wait_selftest: call oras_factor first"; return ORAS_ERR_STATE; }
  auto& d = h->dev;
  CK(cudaMemsetAsync(d.status, 0, 8 * sizeof(int32_t), d.stream));
  if (launch_wait_selftest(h)) CK(cudaGetLastError());
  int32_t* st = (int32_t*)(d.host_pinned + PINNED_STATUS_OFF);
  CK(cudaMemcpyAsync(st, d.status, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, d.stream));
  CK(cudaStreamSynchronize(d.stream));
  if (detail) *detail = st[ST_DETAIL];
  const int rc = status_code(h, st);
  CK(cudaMemsetAsync(d.status, 0, 8 * sizeof(int32_t), d.stream));  // the handle stays usable
  return rc;
}

int oras_release_memory(int32_t device) {
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return ORAS_ERR_CUDA;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = pool_trim(device);
  cudaSetDevice(prev);
  if (e == cudaErrorInvalidDevice) return ORAS_ERR_INVALID_ARG;
  return e == cudaSuccess ? ORAS_OK : ORAS_ERR_CUDA;
}

int oras_footprint(const oras_handle* h, int32_t k, int64_t* bytes) {
  if (!h || !bytes || k < 1 || k > MAX_RHS) return ORAS_ERR_INVALID_ARG;
  *bytes = footprint_bytes(h, k);
  return ORAS_OK;
}

int64_t oras_ndof(const oras_handle* h) { return h ? h->mesh.ndof : -1; }
int32_t oras_nlocal(const oras_handle* h) { return h ? h->mesh.nl : -1; }
int32_t oras_nsub(const oras_handle* h) { return h ? h->mesh.nsub : -1; }
int64_t oras_nnz(const oras_handle* h) { return h ? (int64_t)h->mesh.cols.size() : -1; }
int64_t oras_arena_bytes(const oras_handle* h) { return h ? (int64_t)h->dev.arena_bytes : -1; }

int oras_constrained_dofs(const oras_handle* h, uint8_t* out) {
  if (!h || !out) return ORAS_ERR_INVALID_ARG;
  if (h->mesh.fixed.empty()) std::memset(out, 0, (size_t)h->mesh.ndof);
  else std::memcpy(out, h->mesh.fixed.data(), (size_t)h->mesh.ndof);
  return ORAS_OK;
}

int oras_dofmap(const oras_handle* h, int32_t* out) {
  if (!h || !out) return ORAS_ERR_INVALID_ARG;
  std::memcpy(out, h->mesh.dofmap.data(), h->mesh.dofmap.size() * sizeof(int32_t));
  return ORAS_OK;
}

int oras_partition(const oras_handle* h, int32_t* out) {
  if (!h || !out) return ORAS_ERR_INVALID_ARG;
  std::memcpy(out, h->mesh.part.data(), h->mesh.part.size() * sizeof(int32_t));
  return ORAS_OK;
}

int oras_subdomain_size(const oras_handle* h, int32_t s, int64_t* ndof, int64_t* ntet, int64_t* npad) {
  if (!h || s < 0 || s >= h->mesh.nsub) return ORAS_ERR_INVALID_ARG;
  if (ndof) *ndof = h->mesh.sub_ns[s];
  if (ntet) *ntet = h->mesh.sub_nt_off[s + 1] - h->mesh.sub_nt_off[s];
  if (npad) *npad = h->mesh.sub_np[s];
  return ORAS_OK;
}

int oras_subdomain(const oras_handle* h, int32_t s, int32_t* dofs, uint8_t* pou, int32_t* tets) {
  if (!h || s < 0 || s >= h->mesh.nsub) return ORAS_ERR_INVALID_ARG;
  const auto& m = h->mesh;
  int64_t o = m.sub_ns_off[s], n = m.sub_ns[s];
  if (dofs) std::memcpy(dofs, m.sub_dofs.data() + o, n * sizeof(int32_t));
  if (pou) std::memcpy(pou, m.sub_pou.data() + o, n);
  if (tets) {
    int64_t t0 = m.sub_nt_off[s], t1 = m.sub_nt_off[s + 1];
    std::memcpy(tets, m.sub_tets.data() + t0, (t1 - t0) * sizeof(int32_t));
  }
  return ORAS_OK;
}

int oras_element_matrices(oras_handle* h, const int32_t* tets, int64_t count, oras_complex* out) {
  if (!h || (!tets && count) || (!out && count)) return ORAS_ERR_INVALID_ARG;
  if (!h->factored) { h->err = "oras_element_matrices: call oras_factor first"; return ORAS_ERR_STATE; }
  const auto& m = h->mesh;
  size_t per = (size_t)m.nl * m.nl;
  for (int64_t q = 0; q < count; ++q) {
    if (tets[q] < 0 || tets[q] >= m.nt) { h->err = "oras_element_matrices: tet out of range"; return ORAS_ERR_INVALID_ARG; }
    CK(cudaMemcpyAsync(out + q * per, h->dev.elem + (size_t)tets[q] * per, per * sizeof(cplx),
                       cudaMemcpyDeviceToHost, h->dev.stream));
  }
  CK(cudaStreamSynchronize(h->dev.stream));
  return ORAS_OK;
}

int oras_global_csr(oras_handle* h, int64_t* rowptr, int32_t* cols, oras_complex* vals) {
  if (!h) return ORAS_ERR_INVALID_ARG;
  const auto& m = h->mesh;
  if (rowptr) std::memcpy(rowptr, m.rowptr.data(), m.rowptr.size() * sizeof(int64_t));
  if (cols) std::memcpy(cols, m.cols.data(), m.cols.size() * sizeof(int32_t));
  if (vals) {
    if (!h->factored) { h->err = "oras_global_csr: call oras_factor first"; return ORAS_ERR_STATE; }
    CK(cudaMemcpyAsync(vals, h->dev.vals, m.cols.size() * sizeof(cplx), cudaMemcpyDeviceToHost, h->dev.stream));
    CK(cudaStreamSynchronize(h->dev.stream));
  }
  return ORAS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ Krylov workspace
int oras::ensure_ws(oras_handle* h, int k, int m) {
  auto& d = h->dev;
  const int64_t N = h->mesh.ndof;
  if (int rc = ensure_ybuf(h, k)) return rc;
  if (d.ws_k >= k && d.ws_m >= m && d.V) return ORAS_OK;
  int kk = std::max(k, d.ws_k), mm = std::max(m, d.ws_m);
  size_t nk = (size_t)N * kk;
  CK(dalloc(d.V, nk * (mm + 1)));
  if (d.factor_bits == 64) {
    CK(dalloc(d.Zd, nk * mm));
  } else {
    dfree_s(d.Zf, d.stream);
    CK(pool_malloc((void**)&d.Zf, nk * mm * 2 * sizeof(float), d.stream));
  }
  CK(dalloc(d.w, nk));
  CK(dalloc(d.xk, nk));
  CK(dalloc(d.bk, nk));
  CK(dalloc(d.tmp, nk));
  CK(dalloc(d.H, (size_t)kk * (mm + 1) * mm));
  CK(dalloc(d.gcs, (size_t)kk * mm));
  CK(dalloc(d.gsn, (size_t)kk * mm));
  CK(dalloc(d.g, (size_t)kk * (mm + 1)));
  CK(dalloc(d.red, (size_t)2 * red_blocks() * kk * 2));
  CK(dalloc(d.scal, (size_t)kk * 8 + (size_t)kk * mm * 2 + 64));
  d.ws_k = kk;
  d.ws_m = mm;
  return ORAS_OK;
}

static int ensure_io(oras_handle* h, size_t elems) {
  auto& d = h->dev;
  if (d.io_elems >= elems && d.io) return ORAS_OK;
  CK(dalloc(d.io, elems));
  d.io_elems = elems;
  return ORAS_OK;
}

// Copy an N x k column-major input (host or device) into the internal [N][k] buffer dst.
static int load_input(oras_handle* h, const oras_complex* src, int k, int mem, cplx* dst) {
  auto& d = h->dev;
  const int64_t N = h->mesh.ndof;
  int rc = ensure_io(h, (size_t)N * k);
  if (rc) return rc;
  CK(cudaMemcpyAsync(d.io, src, sizeof(cplx) * N * k,
                     mem == ORAS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, d.stream));
  launch_to_internal(h, k, d.io, dst);
  return ORAS_OK;
}

static int store_output(oras_handle* h, const cplx* src, int k, int mem, oras_complex* dst) {
  auto& d = h->dev;
  const int64_t N = h->mesh.ndof;
  int rc = ensure_io(h, (size_t)N * k);
  if (rc) return rc;
  launch_to_external(h, k, src, d.io);
  CK(cudaMemcpyAsync(dst, d.io, sizeof(cplx) * N * k,
                     mem == ORAS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, d.stream));
  if (mem != ORAS_MEM_DEVICE) CK(cudaStreamSynchronize(d.stream));
  return ORAS_OK;
}

int oras::precond_to_z(oras_handle* h, const cplx* v, int k, int j) {
  auto& d = h->dev;
  size_t nk = (size_t)h->mesh.ndof * k;
  int rc = d.factor_bits == 64 ? launch_apply_f64out(h, v, d.Zd + nk * j, k)
                               : launch_apply_f32out(h, v, (char*)d.Zf + nk * j * 2 * sizeof(float), k);
  if (rc) h->err = "preconditioner apply launch failed";
  return rc ? ORAS_ERR_CUDA : ORAS_OK;
}

void oras::spmv_z(oras_handle* h, int k, int j, cplx* y) {
  auto& d = h->dev;
  size_t nk = (size_t)h->mesh.ndof * k;
  if (d.factor_bits == 64) launch_spmv_f64(h, d.Zd + nk * j, y, k);
  else launch_spmv_f32(h, (char*)d.Zf + nk * j * 2 * sizeof(float), y, k);
}

// Drops every captured Arnoldi step and sizes the cache for restart length m.
static void reset_step_graphs(oras_handle* h, int m) {
  for (auto g : h->step_graph)
    if (g) cudaGraphExecDestroy(g);
  h->step_graph.assign(m, nullptr);
  h->step_seen.assign(m, 0);
  h->step_kernels.assign(m, 0);
}

// Runs Arnoldi step j through `body` (which launches its kernels on the handle's stream): directly
// on its first use, captured into an executable graph on its second, replayed from then on.  A
// capture that fails falls back to direct launches.
template <typename Body>
static int run_step(oras_handle* h, int j, int k, int m, Body&& body) {
  auto& d = h->dev;
  const void* Z = d.factor_bits == 64 ? (const void*)d.Zd : (const void*)d.Zf;
  if (h->graph_stream != d.stream || h->graph_k != k || h->graph_m != m || h->graph_V != d.V || h->graph_Z != Z ||
      h->graph_arena != d.arena || h->graph_ybuf != d.ybuf || (int)h->step_graph.size() != m) {
    reset_step_graphs(h, m);
    h->graph_stream = d.stream;
    h->graph_k = k;
    h->graph_m = m;
    h->graph_V = d.V;
    h->graph_Z = Z;
    h->graph_arena = d.arena;
    h->graph_ybuf = d.ybuf;
  }
  if (h->step_graph[j]) {
    if (cudaGraphLaunch(h->step_graph[j], d.stream) != cudaSuccess) return ORAS_ERR_CUDA;
    count_launches(h->step_kernels[j]);
    return ORAS_OK;
  }
  if (h->step_seen[j] == 0) {
    ++h->step_seen[j];
    return body();
  }
  // second use: capture (the captured launches do not run), instantiate, then launch
  const int64_t l0 = g_launches.load();
  if (cudaStreamBeginCapture(d.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return body();
  const int rc = body();
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(d.stream, &graph);
  const int kernels = (int)(g_launches.load() - l0);
  count_launches(-kernels);  // captured, not yet run
  cudaGraphExec_t exec = nullptr;
  if (rc == ORAS_OK && e == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
    h->step_graph[j] = exec;
    h->step_kernels[j] = kernels;
  }
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();  // a failed capture leaves its error here; the step runs below either way
  if (h->step_graph[j]) {
    if (cudaGraphLaunch(h->step_graph[j], d.stream) != cudaSuccess) return ORAS_ERR_CUDA;
    count_launches(kernels);
    return ORAS_OK;
  }
  return body();
}

// FGMRES(m) on internal [N][k] vectors: b = d.bk, solution in d.xk.
static int fgmres(oras_handle* h, int k, double tol, oras_info* info) {
  auto& d = h->dev;
  const int64_t N = h->mesh.ndof;
  const int m = h->opt.restart, max_iter = h->opt.max_iter;
  int rc = ensure_ws(h, k, m);
  if (rc) return rc;
  const size_t nk = (size_t)N * k;
  cplx* pA = (cplx*)d.red;
  cplx* pB = pA + (size_t)red_blocks() * k;
  double* beta_d = d.scal;                     // [k]
  double* res_d = d.scal + k;                  // [k]
  int32_t* active_d = (int32_t*)(d.scal + 2 * k);
  cplx* y_d = (cplx*)(d.scal + 3 * k + 8);     // [k][m]
  double* hp = d.host_pinned;                  // [0,k): norms; [k,2k): res
  std::vector<double> bnorm(k), relres(k);
  std::vector<int32_t> active(k, 1), iters(k, 0), cycles(k, 0), conv(k, 0);
  int32_t* st_h = (int32_t*)(hp + PINNED_STATUS_OFF);  // device status flags, read with every step
  CK(cudaMemsetAsync(d.status, 0, 8 * sizeof(int32_t), d.stream));
  // ||b||
  CK(cudaMemsetAsync(d.xk, 0, nk * sizeof(cplx), d.stream));
  CK(cudaMemsetAsync(d.tmp, 0, nk * sizeof(cplx), d.stream));
  launch_residual(h, k, d.bk, d.tmp, pA);
  launch_norms(h, k, pA, beta_d);
  CK(cudaMemcpyAsync(hp, beta_d, k * sizeof(double), cudaMemcpyDeviceToHost, d.stream));
  CK(cudaStreamSynchronize(d.stream));
  for (int r = 0; r < k; ++r) {
    bnorm[r] = hp[r];
    if (!(bnorm[r] > 0.0)) { active[r] = 0; conv[r] = 1; relres[r] = 0.0; }
  }
  bool first = true;
  while (true) {
    if (!first) {
      // true residual r = b - A x
      int pb = prof_begin(h);
      launch_spmv_f64(h, d.xk, d.tmp, k);
      prof_end(h, KC_SPMV64, pb, (k + 7) / 8);
      launch_residual(h, k, d.bk, d.tmp, pA);
      launch_norms(h, k, pA, beta_d);
      CK(cudaMemcpyAsync(hp, beta_d, k * sizeof(double), cudaMemcpyDeviceToHost, d.stream));
      CK(cudaStreamSynchronize(d.stream));
    }
    first = false;
    bool any = false;
    for (int r = 0; r < k; ++r) {
      if (!(bnorm[r] > 0.0)) continue;
      relres[r] = hp[r] / bnorm[r];
      if (relres[r] <= tol) { active[r] = 0; conv[r] = 1; }
      else if (iters[r] >= max_iter) active[r] = 0;
      else active[r] = 1;
      any |= active[r] != 0;
    }
    if (!any) break;
    CK(cudaMemcpyAsync(active_d, active.data(), k * sizeof(int32_t), cudaMemcpyHostToDevice, d.stream));
    launch_restart(h, k, m, d.tmp, beta_d, active_d, d.V, d.g);
    int kk = 0;
    const bool graphs = h->opt.graphs && d.stream != nullptr && !h->timing;
    for (int j = 0; j < m; ++j) {
      cplx* Vj = d.V + nk * j;
      cplx* Vn = d.V + nk * (j + 1);
      // z_j = M^-1 v_j ; w = A z_j ; modified Gram-Schmidt against v_0..v_j ; Givens
      auto step = [&]() -> int {
        int pb = prof_begin(h);
        if (precond_to_z(h, Vj, k, j)) return ORAS_ERR_CUDA;
        prof_end(h, KC_APPLY, pb, apply_passes(h, k));
        pb = prof_begin(h);
        spmv_z(h, k, j, d.w);
        prof_end(h, d.factor_bits == 64 ? KC_SPMV64 : KC_SPMV, pb, (k + 7) / 8);
        pb = prof_begin(h);
        launch_dot(h, d.V, d.w, pA, k);
        cplx* pin = pA;
        cplx* pout = pB;
        for (int i = 0; i <= j; ++i) {
          launch_mgs_step(h, k, m, i, j, d.V + nk * i, i < j ? d.V + nk * (i + 1) : nullptr, d.w, pin, pout, d.H);
          std::swap(pin, pout);
        }
        launch_mgs_finish(h, k, m, j, d.w, Vn, pin, d.H, d.gcs, d.gsn, d.g, res_d);
        prof_end(h, KC_ORTH, pb, j + 3);
        return ORAS_OK;
      };
      if ((graphs ? run_step(h, j, k, m, step) : step()) != ORAS_OK) return ORAS_ERR_CUDA;
      kk = j + 1;
      for (int r = 0; r < k; ++r)
        if (active[r]) ++iters[r];
      CK(cudaMemcpyAsync(hp + k, res_d, k * sizeof(double), cudaMemcpyDeviceToHost, d.stream));
      CK(cudaMemcpyAsync(st_h, d.status, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, d.stream));
      CK(cudaStreamSynchronize(d.stream));
      // a bounded wait that gave up in this step's apply: the step's vectors are not valid
      if (int sc = status_code(h, st_h)) return sc;
      bool more = false;
      for (int r = 0; r < k; ++r)
        if (active[r] && hp[k + r] / bnorm[r] > tol && iters[r] < max_iter) more = true;
      if (!more) break;
    }
    launch_hsolve(h, k, m, kk, d.H, d.g, active_d, y_d);
    if (d.factor_bits == 64) launch_xupdate_f64(h, k, m, kk, d.Zd, y_d, d.xk);
    else launch_xupdate_f32(h, k, m, kk, d.Zf, y_d, d.xk);
    for (int r = 0; r < k; ++r)
      if (active[r]) ++cycles[r];
    CK(cudaGetLastError());
  }
  prof_resolve(h);
  bool all = true;
  for (int r = 0; r < k; ++r) {
    if (info) {
      info[r].iterations = iters[r];
      info[r].restarts = cycles[r];
      info[r].converged = conv[r];
      info[r].relres = relres[r];
      info[r].pad = 0;
    }
    all &= conv[r] != 0;
  }
  return all ? ORAS_OK : ORAS_NOT_CONVERGED;
}

extern "C" {

int oras_solve(oras_handle* h, const oras_complex* rhs, int32_t k, double tol, oras_complex* x, oras_info* info,
               int32_t mem) {
  if (!h) return ORAS_ERR_INVALID_ARG;
  if (!h->factored) { h->err = "oras_solve: call oras_factor first"; return ORAS_ERR_STATE; }
  if (k < 1 || k > MAX_RHS || !rhs || !x || !(tol > 0.0)) { h->err = "oras_solve: bad k, tol or NULL vector"; return ORAS_ERR_INVALID_ARG; }
  int rc = ensure_ws(h, k, h->opt.restart);
  if (rc) return rc;
  rc = load_input(h, rhs, k, mem, h->dev.bk);
  if (rc) return rc;
  launch_mask_fixed(h, h->dev.bk, k);  // metallic faces: zero right-hand side on constrained unknowns
  if (h->opt.block && k > 1) {
    rc = fgmres_block(h, k, tol, info);
    prof_resolve(h);
  } else if (h->opt.recycle > 0 && k == 1) {
    rc = gcrodr_solve(h, tol, info);
    prof_resolve(h);
  } else {
    rc = fgmres(h, k, tol, info);
  }
  if (rc < 0) return rc;
  int rc2 = store_output(h, h->dev.xk, k, mem, x);
  if (rc2) return rc2;
  return rc;
}

int oras_matvec(oras_handle* h, const oras_complex* x, oras_complex* y, int32_t k, int32_t mem) {
  if (!h || !x || !y || k < 1 || k > MAX_RHS) return ORAS_ERR_INVALID_ARG;
  if (!h->factored) { h->err = "oras_matvec: call oras_factor first"; return ORAS_ERR_STATE; }
  int rc = ensure_ws(h, k, h->opt.restart);
  if (rc) return rc;
  rc = load_input(h, x, k, mem, h->dev.bk);
  if (rc) return rc;
  launch_spmv_f64(h, h->dev.bk, h->dev.tmp, k);
  return store_output(h, h->dev.tmp, k, mem, y);
}

int oras_matvec_c64(oras_handle* h, const void* x, oras_complex* y, int32_t k, int32_t mem) {
  if (!h || !x || !y || k < 1 || k > MAX_RHS) return ORAS_ERR_INVALID_ARG;
  if (!h->factored) { h->err = "oras_matvec_c64: call oras_factor first"; return ORAS_ERR_STATE; }
  int rc = ensure_ws(h, k, h->opt.restart);
  if (rc) return rc;
  rc = ensure_io(h, (size_t)h->mesh.ndof * k);
  if (rc) return rc;
  auto& d = h->dev;
  const size_t bytes = (size_t)h->mesh.ndof * k * 2 * sizeof(float);
  // staging: the first half of io holds the column-major copy, the internal [N][k] copy goes to w
  CK(cudaMemcpyAsync(d.io, x, bytes, mem == ORAS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     d.stream));
  launch_to_internal_c64(h, k, d.io, d.w);
  launch_spmv_f32(h, d.w, d.tmp, k);
  return store_output(h, d.tmp, k, mem, y);
}

int oras_precond(oras_handle* h, const oras_complex* v, oras_complex* z, int32_t k, int32_t mem) {
  if (!h || !v || !z || k < 1 || k > MAX_RHS) return ORAS_ERR_INVALID_ARG;
  if (!h->factored) { h->err = "oras_precond: call oras_factor first"; return ORAS_ERR_STATE; }
  int rc = ensure_ws(h, k, h->opt.restart);
  if (rc) return rc;
  rc = load_input(h, v, k, mem, h->dev.bk);
  if (rc) return rc;
  CK(cudaMemsetAsync(h->dev.status, 0, 8 * sizeof(int32_t), h->dev.stream));
  const int pb = prof_begin(h);
  if (launch_apply_f64out(h, h->dev.bk, h->dev.tmp, k)) {
    h->err = "oras_precond: apply launch failed";
    return ORAS_ERR_CUDA;
  }
  prof_end(h, KC_APPLY, pb, apply_passes(h, k));
  rc = store_output(h, h->dev.tmp, k, mem, z);
  prof_resolve(h);
  if (rc) return rc;
  return sync_status(h);  // a bounded wait that gave up inside the apply
}

int oras_rhs_dipole(oras_handle* h, const double* x0, const double* dir, oras_complex* b, int32_t mem) {
  if (!h || !x0 || !dir || !b) return ORAS_ERR_INVALID_ARG;
  if (!h->dev.uploaded) { h->err = "oras_rhs_dipole: call oras_factor first"; return ORAS_ERR_STATE; }
  auto& d = h->dev;
  int rc = ensure_ws(h, 1, h->opt.restart);
  if (rc) return rc;
  int* found = (int*)(d.scal + 4);
  if (launch_dipole(h, x0, dir, d.tmp, found)) CK(cudaGetLastError());
  launch_mask_fixed(h, d.tmp, 1);
  int hf = 0;
  CK(cudaMemcpyAsync(&hf, found, sizeof(int), cudaMemcpyDeviceToHost, d.stream));
  CK(cudaStreamSynchronize(d.stream));
  if (hf == 0x7fffffff) { h->err = "oras_rhs_dipole: source point lies in no tetrahedron"; return ORAS_ERR_INVALID_ARG; }
  CK(cudaMemcpyAsync(b, d.tmp, sizeof(cplx) * h->mesh.ndof,
                     mem == ORAS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, d.stream));
  CK(cudaStreamSynchronize(d.stream));
  return ORAS_OK;
}

// Gauss-Legendre nodes/weights on [0, 1] by Newton's method on the Legendre recurrence.
static void gauss_legendre01(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int q = 2; q <= n; ++q) {
        double p2 = ((2.0 * q - 1.0) * z * p1 - (q - 1.0) * p0) / q;
        p0 = p1;
        p1 = p2;
      }
      double pn = n == 1 ? z : p1, pm = n == 1 ? 1.0 : p0;
      dp = n * (z * pn - pm) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

int oras_rhs_plane_wave(oras_handle* h, const double* dvec, const oras_complex* pvec, oras_complex* b, int32_t mem) {
  if (!h || !dvec || !pvec || !b) return ORAS_ERR_INVALID_ARG;
  if (!h->factored) { h->err = "oras_rhs_plane_wave: call oras_factor first"; return ORAS_ERR_STATE; }
  auto& d = h->dev;
  int rc = ensure_ws(h, 1, h->opt.restart);
  if (rc) return rc;
  const int nq = 12;
  double qs[16], qw[16];
  gauss_legendre01(nq, qs, qw);
  cplx* bface = nullptr;
  CK(dalloc(bface, (size_t)std::max<int64_t>(1, h->mesh.nif) * h->mesh.nfl));
  rc = launch_plane(h, dvec, pvec, h->k0, qs, qw, nq, bface, d.tmp);
  launch_mask_fixed(h, d.tmp, 1);
  cudaError_t e = cudaMemcpyAsync(b, d.tmp, sizeof(cplx) * h->mesh.ndof,
                                  mem == ORAS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, d.stream);
  cudaFreeAsync(bface, d.stream);
  cudaStreamSynchronize(d.stream);
  if (rc || e != cudaSuccess) { h->err = "oras_rhs_plane_wave: launch failed"; return ORAS_ERR_CUDA; }
  return ORAS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ waveguide ports
namespace {
struct PortSel {
  std::vector<uint8_t> inport;   // [nif]
  std::vector<int32_t> dofs;     // sorted unique degrees of freedom of the port's faces
};

// the outer faces whose centroid lies in the port rectangle (the decision in FP64 on the host,
// vertices in ascending id order)
int select_port(oras_handle* h, const oras_port* P, PortSel& out) {
  const auto& m = h->mesh;
  const double* o = P->origin;
  const double* u = P->u;
  const double* v = P->v;
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2], vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  const double uv = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
  if (!(uu > 0.0) || !(vv > 0.0) || !(std::fabs(uv) <= 1e-12 * std::sqrt(uu * vv)) || !(P->beta > 0.0)) {
    h->err = "port: u and v must be nonzero and orthogonal, beta > 0";
    return ORAS_ERR_INVALID_ARG;
  }
  double n[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
  const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  for (double& c : n) c /= nn;
  const double tol = 1e-9 * (std::sqrt(uu) + std::sqrt(vv));
  static const int FACES[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
  out.inport.assign(m.nif, 0);
  out.dofs.clear();
  for (int64_t i = 0; i < m.nif; ++i) {
    if (m.if_tet1[i] >= 0) continue;
    const int64_t t = m.if_tet0[i];
    const int lf = m.if_lf0[i];
    double c[3];
    for (int dd = 0; dd < 3; ++dd) {
      const double x0 = m.xyz[(int64_t)m.st[t * 4 + FACES[lf][0]] * 3 + dd];
      const double x1 = m.xyz[(int64_t)m.st[t * 4 + FACES[lf][1]] * 3 + dd];
      const double x2 = m.xyz[(int64_t)m.st[t * 4 + FACES[lf][2]] * 3 + dd];
      c[dd] = ((x0 + x1) + x2) / 3.0;
    }
    const double d[3] = {c[0] - o[0], c[1] - o[1], c[2] - o[2]};
    const double s = (d[0] * u[0] + d[1] * u[1] + d[2] * u[2]) / uu;
    const double tt = (d[0] * v[0] + d[1] * v[1] + d[2] * v[2]) / vv;
    const double dn = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
    if (std::fabs(dn) <= tol && s >= 0.0 && s <= 1.0 && tt >= 0.0 && tt <= 1.0) {
      out.inport[i] = 1;
      for (int af = 0; af < m.nfl; ++af) out.dofs.push_back(m.if_dofs[i * m.nfl + af]);
    }
  }
  if (out.dofs.empty()) {
    h->err = "port: no outer face lies in the port rectangle";
    return ORAS_ERR_INVALID_ARG;
  }
  std::sort(out.dofs.begin(), out.dofs.end());
  out.dofs.erase(std::unique(out.dofs.begin(), out.dofs.end()), out.dofs.end());
  return ORAS_OK;
}

// device scratch of the port integrals
struct PortBufs {
  uint8_t* inport = nullptr;
  cplx* pface = nullptr;
  double* nface = nullptr;
  double* norm = nullptr;
  int32_t* dofs = nullptr;
  cplx* S = nullptr;
  cudaStream_t s = nullptr;
  ~PortBufs() {
    for (void* p : {(void*)inport, (void*)pface, (void*)nface, (void*)norm, (void*)dofs, (void*)S})
      if (p) cudaFreeAsync(p, s);
  }
};

// p (load = 0) or the port load b (load = 1) into out (device [N]), norm into bufs.norm
int port_integrals(oras_handle* h, const oras_port* P, int load, PortSel& sel, PortBufs& B, cplx* out) {
  auto& m = h->mesh;
  auto& d = h->dev;
  int rc = select_port(h, P, sel);
  if (rc) return rc;
  B.s = d.stream;
  if (!B.inport) {
    CK(dalloc(B.inport, (size_t)m.nif));
    CK(dalloc(B.pface, (size_t)m.nif * m.nfl));
    CK(dalloc(B.nface, (size_t)m.nif));
    CK(dalloc(B.norm, (size_t)1));
  }
  CK(cudaMemcpyAsync(B.inport, sel.inport.data(), (size_t)m.nif, cudaMemcpyHostToDevice, d.stream));
  const int nq = 12;
  double qs[16], qw[16];
  gauss_legendre01(nq, qs, qw);
  if (launch_port(h, P->origin, P->u, P->v, P->beta, load, qs, qw, nq, B.inport, B.pface, B.nface, out, B.norm)) {
    h->err = "port: launch failed";
    return ORAS_ERR_CUDA;
  }
  if (load) launch_mask_fixed(h, out, 1);
  return ORAS_OK;
}
}  // namespace

extern "C" {

int oras_port_vector(oras_handle* h, const oras_port* port, oras_complex* p, double* norm, int32_t mem) {
  if (!h || !port || !p) return ORAS_ERR_INVALID_ARG;
  if (!h->factored) { h->err = "oras_port_vector: call oras_factor first"; return ORAS_ERR_STATE; }
  auto& d = h->dev;
  int rc = ensure_ws(h, 1, h->opt.restart);
  if (rc) return rc;
  PortSel sel;
  PortBufs B;
  rc = port_integrals(h, port, 0, sel, B, d.tmp);
  if (rc) return rc;
  double hn = 0.0;
  CK(cudaMemcpyAsync(&hn, B.norm, sizeof(double), cudaMemcpyDeviceToHost, d.stream));
  CK(cudaMemcpyAsync(p, d.tmp, sizeof(cplx) * h->mesh.ndof,
                     mem == ORAS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, d.stream));
  CK(cudaStreamSynchronize(d.stream));
  if (norm) *norm = hn;
  return ORAS_OK;
}

int oras_rhs_port(oras_handle* h, const oras_port* port, oras_complex* b, int32_t mem) {
  if (!h || !port || !b) return ORAS_ERR_INVALID_ARG;
  if (!h->factored) { h->err = "oras_rhs_port: call oras_factor first"; return ORAS_ERR_STATE; }
  auto& d = h->dev;
  int rc = ensure_ws(h, 1, h->opt.restart);
  if (rc) return rc;
  PortSel sel;
  PortBufs B;
  rc = port_integrals(h, port, 1, sel, B, d.tmp);
  if (rc) return rc;
  CK(cudaMemcpyAsync(b, d.tmp, sizeof(cplx) * h->mesh.ndof,
                     mem == ORAS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, d.stream));
  CK(cudaStreamSynchronize(d.stream));
  return ORAS_OK;
}

int oras_s_matrix(oras_handle* h, int32_t nports, const oras_port* ports, const oras_complex* x, int32_t k,
                  oras_complex* S, int32_t mem) {
  if (!h || !ports || !x || !S || nports < 1 || k < 1 || k > MAX_RHS) return ORAS_ERR_INVALID_ARG;
  if (!h->factored) { h->err = "oras_s_matrix: call oras_factor first"; return ORAS_ERR_STATE; }
  auto& d = h->dev;
  int rc = ensure_ws(h, k, h->opt.restart);
  if (rc) return rc;
  rc = load_input(h, x, k, mem, d.bk);  // [N][k] internal layout
  if (rc) return rc;
  PortBufs B;
  B.s = d.stream;
  CK(dalloc(B.S, (size_t)nports * k));
  for (int i = 0; i < nports; ++i) {
    PortSel sel;
    rc = port_integrals(h, &ports[i], 0, sel, B, d.tmp);
    if (rc) return rc;
    if (B.dofs) cudaFreeAsync(B.dofs, d.stream);
    B.dofs = nullptr;
    CK(dalloc(B.dofs, sel.dofs.size()));
    CK(cudaMemcpyAsync(B.dofs, sel.dofs.data(), sel.dofs.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                       d.stream));
    if (launch_port_dots(h, (int64_t)sel.dofs.size(), B.dofs, d.tmp, d.bk, k, B.norm, B.S + (int64_t)i * k)) {
      h->err = "oras_s_matrix: launch failed";
      return ORAS_ERR_CUDA;
    }
    CK(cudaStreamSynchronize(d.stream));  // the host port selection of the next port reuses the buffers
  }
  CK(cudaMemcpyAsync(S, B.S, sizeof(cplx) * nports * k, cudaMemcpyDeviceToHost, d.stream));
  CK(cudaStreamSynchronize(d.stream));
  return ORAS_OK;
}

double oras_s_error(const oras_complex* S, const oras_complex* S_ref, int64_t n) {
  if (!S || !S_ref || n < 1) return -1.0;
  double num = 0.0, den = 0.0;
  for (int64_t q = 0; q < n; ++q) {
    const double dr = S[q].re - S_ref[q].re, di = S[q].im - S_ref[q].im;
    num += dr * dr + di * di;
    den += S_ref[q].re * S_ref[q].re + S_ref[q].im * S_ref[q].im;
  }
  return den > 0.0 ? std::sqrt(num / den) : -1.0;
}

}  // extern "C"
