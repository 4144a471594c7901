// Internal declarations of the ORAS-FGMRES library (not part of the C ABI).
#pragma once

#include <cstdint>
#include <mutex>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/oras.h"

namespace oras {

constexpr int TB = 64;            // tile order of the local-factor arena (TB x TB complex)
constexpr int LU_SUB = 8;         // sub-panel width (tile columns) of the LU's left-looking steps
// scratch tiles per subdomain after the factor tiles: the inverted unit-lower diagonal blocks
// L_kk^{-1} of a sub-panel's steps (slots 0 .. LU_SUB-1) and U_kk^{-1} of the current step
constexpr int LU_SCRATCH = LU_SUB + 1;
constexpr int MAX_NFL = 15;       // face-local DOFs r(r+2) for r <= 3
constexpr int MAX_NL = 45;        // tet-local DOFs for r <= 3
constexpr int MAX_RHS = 64;
constexpr int PINNED_SCRATCH_DOUBLES = 4096;
constexpr int PINNED_STATUS_OFF = 2048;   // pinned scratch: doubles [2048, 2052) hold the status flags

struct cplx { double re, im; };

// device status flags (Device::status): [0] error code, [1] detail, [2] subdomain
enum { ST_ERR = 0, ST_DETAIL = 1, ST_SUB = 2 };
enum { DEV_OK = 0, DEV_SINGULAR = 1, DEV_TIMEOUT = 2, DEV_BADINDEX = 3 };


// ------------------------------------------------------------------ local DOF convention
struct LocalDof {
  char kind;      // 'e', 'f', 'v'
  int ent, q;     // local entity index and index inside the entity
  int i, j;       // Whitney edge (local vertices, i < j)
  int k[4];       // exponents of lambda^k
};
std::vector<LocalDof> local_dofs(int r);
int n_local(int r);
int n_face_local(int r);                       // r(r+2)
// tet-local indices of the face-local DOFs of local face lf (intrinsic face order:
// edges (a,b), (a,c), (b,c), then the face's own DOFs)
std::vector<int> face_local_dofs(int r, int lf);

// Exact integration tables of the element and face matrices (see tables.cpp).
struct Tables {
  int r = 0, nl = 0, nfl = 0;
  std::vector<double> cm;   // [nl][nl][10]   mass, unique Gram pairs p <= q
  std::vector<double> ck;   // [nl][nl][21]   stiffness, unique pairs of the 6 cross products
  std::vector<double> cs;   // [4][nfl][nfl][10] face tangential mass per local face
  std::vector<int> fl;      // [4][nfl] tet-local index of each face-local DOF
  // basis-value term table: DOF a = sum_t c * lambda^alpha * grad(lambda_m), 2 terms each
  std::vector<double> tc;   // [nl][2]
  std::vector<int> ta;      // [nl][2][4]
  std::vector<int> tm;      // [nl][2]
};
Tables make_tables(int r);

// ------------------------------------------------------------------ host integer set-up
struct HostMesh {
  int r = 0, nl = 0, nfl = 0;
  int64_t nv = 0, nt = 0, ne = 0, nf = 0, ndof = 0;
  int nsub = 0, overlap = 0, overlap_kind = 0;
  std::vector<double> xyz;        // [nv][3]
  std::vector<int32_t> st;        // [nt][4] sorted vertex ids
  std::vector<int32_t> tet_faces; // [nt][4]
  std::vector<int32_t> face_tets; // [nf][2]
  std::vector<int32_t> dofmap;    // [nt][nl]
  std::vector<int32_t> part;      // [nt]
  // global row incidence: (t*nl + a) for every tet t carrying DOF g, ascending t
  std::vector<int64_t> tinc_ptr;  // [ndof+1]
  std::vector<int32_t> tinc;
  // impedance faces (outer boundary + every interface face of some subdomain)
  int64_t nif = 0;
  std::vector<int32_t> if_face, if_tet0, if_lf0, if_tet1;  // tet1 = -1 on the outer boundary
  std::vector<int32_t> if_dofs;   // [nif][nfl] global DOFs, intrinsic face order
  std::vector<double> if_beta;    // [nif] caller's beta of outer faces (empty: derived per factor)
  std::vector<uint8_t> fixed;     // [ndof] 1: constrained by a metallic face (empty: none)
  int64_t nfixed = 0;
  std::vector<int64_t> finc_ptr;  // [ndof+1]
  std::vector<int32_t> finc;      // slot*nfl + a_f
  // CSR pattern of A
  std::vector<int64_t> rowptr;    // [ndof+1]
  std::vector<int32_t> cols;
  int max_row_nnz = 0;
  // subdomains
  std::vector<int64_t> sub_ns, sub_np, sub_ns_off, sub_tile_off, sub_nt_off;
  std::vector<int32_t> sub_dofs;  // concatenated N_s
  std::vector<uint8_t> sub_pou;   // concatenated D_s
  std::vector<int32_t> sub_tets;  // concatenated Omega_s^delta
  std::vector<uint32_t> member;   // [nsub][words] tet membership bitmaps
  int64_t member_words = 0;
  int64_t arena_tiles = 0;
  int64_t max_np = 0;
};

// Returns ORAS_OK or an error code with `err` filled.
int host_setup(const oras_problem* p, int overlap_kind, HostMesh& m, std::string& err);

// ------------------------------------------------------------------ device state
template <typename T> struct DBuf {
  T* p = nullptr;
  size_t n = 0;
};

struct Device {
  bool uploaded = false;
  int device = -1;
  cudaStream_t stream = nullptr;
  // mesh
  double* xyz = nullptr;
  int32_t* st = nullptr;
  int32_t* dofmap = nullptr;
  int64_t* tinc_ptr = nullptr;
  int32_t* tinc = nullptr;
  int32_t* if_tet0 = nullptr; int32_t* if_lf0 = nullptr; int32_t* if_tet1 = nullptr;
  int32_t* if_dofs = nullptr;
  double* if_beta = nullptr;                    // [nif] or nullptr (beta derived from the materials)
  uint8_t* fixed = nullptr;                     // [ndof] constrained degrees of freedom, or nullptr
  int64_t* finc_ptr = nullptr;
  int32_t* finc = nullptr;
  int64_t* rowptr = nullptr;
  int32_t* cols = nullptr;
  int64_t* sub_ns = nullptr; int64_t* sub_np = nullptr; int64_t* sub_ns_off = nullptr;
  int64_t* sub_tile_off = nullptr;
  int32_t* sub_dofs = nullptr;
  uint8_t* sub_pou = nullptr;
  uint32_t* member = nullptr;
  // tables
  double* cm = nullptr; double* ck = nullptr; double* cs = nullptr; int32_t* fl = nullptr;
  double* tc = nullptr; int32_t* ta = nullptr; int32_t* tm = nullptr;
  // numeric
  cplx* eps = nullptr; cplx* mu = nullptr;      // [nt]
  cplx* elem = nullptr;                         // [nt][nl][nl]
  double* fmat = nullptr;                       // [nif][nfl][nfl]
  cplx* vals = nullptr;                         // [nnz]
  float4* vals_df = nullptr;                    // [nnz] A = hi + lo in FP32 pairs (FP32-pipe SpMV)
  void* arena = nullptr;                        // tiles, complex float or double
  size_t arena_bytes = 0;
  int factor_bits = 0;
  int32_t* perm = nullptr;                      // [sum np] row permutation of P A = L U
  int32_t* gidx = nullptr;                      // [sum np] N_s[perm[i]] or -1
  int64_t* sub_np_off = nullptr;                // prefix of np (device)
  // LU workspace
  int32_t* lu_cand = nullptr;                   // tournament candidates
  int32_t* lu_cnt = nullptr;                    // tournament arrival counters
  int32_t* lu_ipiv = nullptr;                   // [nsub][TB] interchanges of the current step
  void* lu_diag = nullptr;                      // [nsub] factored diagonal tile of the step
  void* dinv = nullptr;                         // inverted diagonal blocks, 2 tiles per block row
  size_t dinv_bytes = 0;
  int64_t* sub_inv_off = nullptr;               // [nsub] prefix of block rows (device)
  int32_t* status = nullptr;                    // device error flags [8]
  int lu_max_chunks = 0;
  // Krylov workspace
  int ws_k = 0, ws_m = 0;
  cplx* V = nullptr;                            // [(m+1)][N][k]
  float* Zf = nullptr;                          // [m][N][k] complex FP32 (factor_bits 32)
  cplx* Zd = nullptr;                           // [m][N][k] complex FP64 (factor_bits 64)
  cplx* w = nullptr; cplx* xk = nullptr; cplx* bk = nullptr; cplx* tmp = nullptr;  // [N][k]
  cplx* H = nullptr;                            // [k][(m+1)][m]
  double* gcs = nullptr; cplx* gsn = nullptr;   // Givens [k][m]
  cplx* g = nullptr;                            // [k][m+1]
  double* red = nullptr;                        // reduction partials
  double* scal = nullptr;                       // small scalars [k][8]
  void* ybuf = nullptr;                         // apply: per-subdomain local vectors
  size_t ybuf_bytes = 0;
  // apply work split: the first apply_n4 subdomains of apply_subs take clusters of four CTAs
  // (largest padded order apply_np4), the rest two (apply_np2); apply_n4 == 0: two CTAs each
  int32_t* apply_subs = nullptr;
  int apply_n4 = 0;
  int num_sms = 0;                              // SMs of the handle's device
  int64_t apply_np4 = 0, apply_np2 = 0;
  cplx* io = nullptr;                           // staging for host I/O [N][k] col-major
  size_t io_elems = 0;
  double* host_pinned = nullptr;                // small pinned host scalars (per host thread)
};

// ------------------------------------------------------------------ instrumentation
// Kernel classes timed with CUDA event pairs on the handle's stream when timing is on.
enum KClass { KC_ELEMENT = 0, KC_GLOBAL_ROWS, KC_LOCAL_ROWS, KC_LU_TOURNAMENT, KC_LU_SWAP, KC_LU_TRSM,
              KC_LU_UPDATE, KC_APPLY, KC_SPMV, KC_ORTH, KC_OTHER, KC_SPMV64, KC_LU_PANEL, KC_COUNT };
int prof_begin(const oras_handle* h);                 // -1 when timing is off
void prof_end(const oras_handle* h, int cls, int begin, int launches);
void count_launches(int n);                           // process-wide launch counter
// Limit of the bounded device waits of a handle's kernels (oras_options.wait_ms; 0 -> 2 s).
uint64_t wait_limit_ns(const oras_handle* h);

// Stream-ordered allocation from the current device's default memory pool.  The pool keeps
// memory freed by cudaFreeAsync for reuse (release threshold unlimited, set once per device), so
// a set-up after a destroy does not map the pages again.  If an allocation fails for lack of
// memory, the pool's unused memory is returned to the driver and the allocation retried once.
inline cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t s) {
  static std::mutex mu;
  static std::set<int> done;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!done.count(dev) && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess) done.insert(dev);
    }
  }
  cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e != cudaErrorMemoryAllocation) return e;
  cudaGetLastError();
  if (!pool && cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return e;
  cudaMemPoolTrimTo(pool, 0);
  return cudaMallocAsync(p, bytes, s);
}

// Returns the unused memory of a device's default pool to the driver.
inline cudaError_t pool_trim(int dev) {
  cudaMemPool_t pool = nullptr;
  cudaError_t e = cudaDeviceGetDefaultMemPool(&pool, dev);
  return e == cudaSuccess ? cudaMemPoolTrimTo(pool, 0) : e;
}

// Raises a kernel's dynamic shared-memory limit to the device's opt-in maximum, once per
// (device, kernel).  A fixed maximum (instead of the size of the next launch) keeps launches of
// the same kernel from different host threads from lowering each other's limit.
inline void allow_max_smem(const void* fn) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({dev, fn})) return;
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  cudaFuncGetAttributes(&fa, fn);
  if (optin > (int)fa.sharedSizeBytes &&
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes) == cudaSuccess)
    done.insert({dev, fn});
}

}  // namespace oras

struct oras_handle {
  oras::HostMesh mesh;
  oras::Tables tab;
  oras::Device dev;
  oras_options opt{};
  std::string err;
  bool factored = false;
  double k0 = 0.0;
  bool timing = false;
  double timings[16] = {0};
  mutable std::vector<cudaEvent_t> evpool;
  mutable size_t ev_used = 0;
  mutable std::vector<int> marks;                    // (class, begin event, end event, launches)*
  double cls_ms[oras::KC_COUNT] = {0};
  double cls_n[oras::KC_COUNT] = {0};
  // tcgen05 operand tensor map over this handle's factor arena (a CUtensorMap, 128 bytes),
  // rebuilt when the arena moves; per handle, so concurrent handles never share one
  alignas(64) unsigned char tc_map[128] = {0};
  const void* tc_map_base = nullptr;
  int64_t tc_map_tiles = 0;
  bool tc_map_ok = false;
  // captured Arnoldi steps (oras_options.graphs): one executable graph per inner index j, valid
  // for the stream, k, restart length and workspace it was captured with
  std::vector<cudaGraphExec_t> step_graph;
  std::vector<int> step_seen;                // direct executions of step j since the cache was built
  std::vector<int> step_kernels;             // kernels in graph j (launch accounting)
  cudaStream_t graph_stream = nullptr;
  int graph_k = 0, graph_m = 0;
  const void* graph_V = nullptr;
  const void* graph_Z = nullptr;
  const void* graph_arena = nullptr;
  const void* graph_ybuf = nullptr;
  // the apply's side stream (four-CTA launch, concurrent with the two-CTA launch) and its
  // fork and join events; created with the upload when some subdomains take four CTAs
  cudaStream_t apply_side = nullptr;
  cudaEvent_t apply_fork = nullptr, apply_join = nullptr;
  // GCRO-DR (oras_options.recycle): the deflation subspace U kept for the next solve
  oras::cplx* rc_U = nullptr;
  int rc_k = 0;
  int64_t rc_n = 0;
};
