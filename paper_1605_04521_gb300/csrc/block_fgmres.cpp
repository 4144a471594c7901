// Block flexible GMRES(m) (Sec. 6 names Block GMRES for the several right-hand sides of one
// system; the paper prints no algorithm).  The p right-hand sides form one block: x0 = 0; the
// block residual R = Q S by CholQR2; for each block step j, Z_j = M^{-1} V_j (the ORAS apply of
// the p columns together), W = A Z_j, block modified Gram-Schmidt against V_0..V_j (H_ij =
// V_i^H W, W -= V_i H_ij), V_{j+1} H_{j+1,j} = W by CholQR2; the least-squares problem
// min || E1 S - Hbar Y ||_F is kept triangular by Householder reflections applied block column by
// block column, which gives every column's residual estimate after every step.  A cycle ends when
// every estimate is <= tol (or after m block steps); then x += Z Y, the true FP64 residuals are
// formed, and the method restarts if some column is above tol.  Large vectors stay on the GPU
// (block.cu, the apply and the SpMV); the p x p Cholesky factors and the small least-squares
// problem are on the host.
#include <algorithm>
#include <cmath>
#include <complex>
#include <string>
#include <vector>

#include "internal.h"

namespace oras {

using zc = std::complex<double>;

// kernels and helpers of the other translation units
void launch_block_gram(const oras_handle* h, int p, const cplx* A, const cplx* B, cplx* part, cplx* G);
void launch_block_mul_f64(const oras_handle* h, int p, const cplx* X, const cplx* C, double alpha, double beta,
                          cplx* Y);
void launch_block_mul_f32(const oras_handle* h, int p, const void* X, const cplx* C, double alpha, double beta,
                          cplx* Y);
int blk_blocks();
int ensure_ws(oras_handle* h, int k, int m);
int precond_to_z(oras_handle* h, const cplx* v, int k, int j);
void spmv_z(oras_handle* h, int k, int j, cplx* y);
int status_code(oras_handle* h, const int32_t* st);
void launch_spmv_f64(const oras_handle* h, const cplx* x, cplx* y, int k);
void launch_residual(const oras_handle* h, int k, const cplx* b, cplx* r, cplx* partials);
void launch_norms(const oras_handle* h, int k, const cplx* partials, double* out);

namespace {

// Upper Cholesky factor C (row-major p x p) of the Hermitian positive definite G = C^H C; false if
// a pivot is not positive (the block is numerically rank deficient).
bool cholesky_upper(const std::vector<zc>& G, int p, std::vector<zc>& C) {
  C.assign((size_t)p * p, zc(0.0));
  for (int i = 0; i < p; ++i) {
    double d = G[(size_t)i * p + i].real();
    for (int q = 0; q < i; ++q) d -= std::norm(C[(size_t)q * p + i]);
    if (!(d > 0.0)) return false;
    const double cii = std::sqrt(d);
    C[(size_t)i * p + i] = cii;
    for (int j = i + 1; j < p; ++j) {
      zc s = G[(size_t)i * p + j];
      for (int q = 0; q < i; ++q) s -= std::conj(C[(size_t)q * p + i]) * C[(size_t)q * p + j];
      C[(size_t)i * p + j] = s / cii;
    }
  }
  return true;
}

// Inverse of an upper triangular row-major p x p matrix.
std::vector<zc> inverse_upper(const std::vector<zc>& C, int p) {
  std::vector<zc> X((size_t)p * p, zc(0.0));
  for (int j = 0; j < p; ++j) {  // column j of C^{-1}: C x = e_j
    for (int i = j; i >= 0; --i) {
      zc s = i == j ? zc(1.0) : zc(0.0);
      for (int q = i + 1; q <= j; ++q) s -= C[(size_t)i * p + q] * X[(size_t)q * p + j];
      X[(size_t)i * p + j] = s / C[(size_t)i * p + i];
    }
  }
  return X;
}

std::vector<zc> matmul(const std::vector<zc>& A, const std::vector<zc>& B, int p) {
  std::vector<zc> C((size_t)p * p, zc(0.0));
  for (int i = 0; i < p; ++i)
    for (int q = 0; q < p; ++q)
      for (int j = 0; j < p; ++j) C[(size_t)i * p + j] += A[(size_t)i * p + q] * B[(size_t)q * p + j];
  return C;
}

// One Householder reflection I - tau v v^H acting on rows [row0, row0 + v.size()).
struct Reflector {
  int64_t row0;
  std::vector<zc> v;
  double tau;
  void apply(zc* col) const {  // col: the whole column (indexed by global row)
    zc s(0.0);
    for (size_t q = 0; q < v.size(); ++q) s += std::conj(v[q]) * col[row0 + q];
    s *= tau;
    for (size_t q = 0; q < v.size(); ++q) col[row0 + q] -= v[q] * s;
  }
};

// Reflector mapping x (rows [row0, row0 + len) of col) to (alpha, 0, ..., 0); writes alpha.
Reflector make_reflector(zc* col, int64_t row0, int64_t len) {
  Reflector r;
  r.row0 = row0;
  r.v.assign(col + row0, col + row0 + len);
  double nrm2 = 0.0;
  for (auto& z : r.v) nrm2 += std::norm(z);
  const double nrm = std::sqrt(nrm2);
  if (nrm == 0.0) { r.tau = 0.0; return r; }
  const zc x0 = r.v[0];
  const zc ph = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : zc(1.0);
  r.v[0] = x0 + ph * nrm;
  double vn2 = 0.0;
  for (auto& z : r.v) vn2 += std::norm(z);
  r.tau = vn2 > 0.0 ? 2.0 / vn2 : 0.0;
  col[row0] = -ph * nrm;
  for (int64_t q = 1; q < len; ++q) col[row0 + q] = 0.0;
  return r;
}

}  // namespace

// Block FGMRES on the internal [N][p] vectors: b = d.bk, solution in d.xk.  Returns ORAS_OK,
// ORAS_NOT_CONVERGED (also when a block became numerically rank deficient: x is the last iterate)
// or an error.
int fgmres_block(oras_handle* h, int p, double tol, oras_info* info) {
  auto& d = h->dev;
  const int64_t N = h->mesh.ndof;
  const int m = h->opt.restart, max_iter = h->opt.max_iter;
  int rc = ensure_ws(h, p, m);
  if (rc) return rc;
  const size_t nk = (size_t)N * p;
  const size_t pp = (size_t)p * p;
  cplx* part = nullptr;   // [blocks][p][p] Gram partials
  cplx* dmat = nullptr;   // p x p device matrices: [0] Gram / factor, [1 + i] H_ij of the step
  if (pool_malloc((void**)&part, sizeof(cplx) * pp * blk_blocks(), d.stream) != cudaSuccess ||
      pool_malloc((void**)&dmat, sizeof(cplx) * pp * (m + 2), d.stream) != cudaSuccess) {
    if (part) cudaFreeAsync(part, d.stream);
    h->err = "block FGMRES workspace allocation failed";
    return ORAS_ERR_OUT_OF_MEMORY;
  }
  struct Free {
    cudaStream_t s; cplx* a; cplx* b;
    ~Free() { cudaFreeAsync(a, s); cudaFreeAsync(b, s); }
  } free_ws{d.stream, part, dmat};
  cplx* pA = (cplx*)d.red;
  double* beta_d = d.scal;
  double* hp = d.host_pinned;
  int32_t* st_h = (int32_t*)(hp + PINNED_STATUS_OFF);
  auto cuda_err = [&](cudaError_t e) {
    h->err = std::string("block FGMRES: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? ORAS_ERR_OUT_OF_MEMORY : ORAS_ERR_CUDA;
  };
#define BCK(call)                          \
  do {                                     \
    cudaError_t e_ = (call);               \
    if (e_ != cudaSuccess) return cuda_err(e_); \
  } while (0)
  std::vector<zc> hbuf(pp);
  auto to_host = [&](const cplx* dsrc, std::vector<zc>& out) -> int {
    out.resize(pp);
    BCK(cudaMemcpyAsync(out.data(), dsrc, sizeof(cplx) * pp, cudaMemcpyDeviceToHost, d.stream));
    BCK(cudaStreamSynchronize(d.stream));
    return ORAS_OK;
  };
  auto to_dev = [&](const std::vector<zc>& src, cplx* ddst) -> int {
    BCK(cudaMemcpyAsync(ddst, src.data(), sizeof(cplx) * pp, cudaMemcpyHostToDevice, d.stream));
    return ORAS_OK;
  };
  // Q C = X (CholQR2) with Q written to `out` (may not alias X): returns false on breakdown
  auto cholqr2 = [&](const cplx* X, cplx* out, std::vector<zc>& C, int& err) -> bool {
    std::vector<zc> G, C1, C2;
    launch_block_gram(h, p, X, X, part, dmat);
    if ((err = to_host(dmat, G))) return false;
    if (!cholesky_upper(G, p, C1)) return false;
    if ((err = to_dev(inverse_upper(C1, p), dmat))) return false;
    launch_block_mul_f64(h, p, X, dmat, 1.0, 0.0, out);
    launch_block_gram(h, p, out, out, part, dmat);
    if ((err = to_host(dmat, G))) return false;
    if (!cholesky_upper(G, p, C2)) return false;
    if ((err = to_dev(inverse_upper(C2, p), dmat))) return false;
    launch_block_mul_f64(h, p, out, dmat, 1.0, 0.0, d.tmp);  // second pass into tmp, then back
    BCK(cudaMemcpyAsync(out, d.tmp, sizeof(cplx) * nk, cudaMemcpyDeviceToDevice, d.stream));
    C = matmul(C2, C1, p);
    return true;
  };
  // ||b|| per column, R = b
  BCK(cudaMemsetAsync(d.status, 0, 8 * sizeof(int32_t), d.stream));
  BCK(cudaMemsetAsync(d.xk, 0, nk * sizeof(cplx), d.stream));
  BCK(cudaMemsetAsync(d.tmp, 0, nk * sizeof(cplx), d.stream));
  launch_residual(h, p, d.bk, d.tmp, pA);
  launch_norms(h, p, pA, beta_d);
  BCK(cudaMemcpyAsync(hp, beta_d, p * sizeof(double), cudaMemcpyDeviceToHost, d.stream));
  BCK(cudaStreamSynchronize(d.stream));
  std::vector<double> bnorm(p), relres(p);
  for (int c = 0; c < p; ++c) bnorm[c] = hp[c] > 0.0 ? hp[c] : 1.0;
  int it = 0, cycles = 0;
  bool converged = false, breakdown = false;
  const int64_t rows = (int64_t)(m + 1) * p;
  while (true) {
    // true residual R = b - A x (d.tmp) and its column norms
    if (it > 0) {
      launch_spmv_f64(h, d.xk, d.tmp, p);
      launch_residual(h, p, d.bk, d.tmp, pA);
      launch_norms(h, p, pA, beta_d);
      BCK(cudaMemcpyAsync(hp, beta_d, p * sizeof(double), cudaMemcpyDeviceToHost, d.stream));
      BCK(cudaStreamSynchronize(d.stream));
    }
    bool all = true;
    for (int c = 0; c < p; ++c) {
      relres[c] = hp[c] / bnorm[c];
      all &= relres[c] <= tol;
    }
    if (all) { converged = true; break; }
    if (it >= max_iter || breakdown) break;
    // V_0 S = R
    std::vector<zc> S;
    int err = 0;
    if (!cholqr2(d.tmp, d.V, S, err)) {
      if (err) return err;
      breakdown = true;
      h->err = "block FGMRES: the residual block is numerically rank deficient";
      break;
    }
    // transformed right-hand side G = Q^H E1 S, stored column by column ((m+1)p rows each)
    std::vector<zc> Gt((size_t)p * rows, zc(0.0));
    for (int r = 0; r < p; ++r)
      for (int c = 0; c < p; ++c) Gt[(size_t)c * rows + r] = S[(size_t)r * p + c];
    std::vector<std::vector<zc>> Hcols;   // block column j: p columns of (j+2)p rows (triangularised)
    std::vector<std::vector<Reflector>> refl;
    int k = 0;
    for (int j = 0; j < m; ++j) {
      cplx* Vj = d.V + nk * j;
      cplx* Vn = d.V + nk * (j + 1);
      int pb = prof_begin(h);
      if (precond_to_z(h, Vj, p, j)) return ORAS_ERR_CUDA;
      prof_end(h, KC_APPLY, pb, 1);
      pb = prof_begin(h);
      spmv_z(h, p, j, d.w);
      prof_end(h, d.factor_bits == 64 ? KC_SPMV64 : KC_SPMV, pb, (p + 7) / 8);
      pb = prof_begin(h);
      std::vector<zc> col((size_t)p * (j + 2) * p, zc(0.0));  // [c][row], rows (j+2)p
      const int64_t cr = (int64_t)(j + 2) * p;
      for (int i = 0; i <= j; ++i) {
        cplx* Hi = dmat + pp * (1 + i);
        launch_block_gram(h, p, d.V + nk * i, d.w, part, Hi);
        launch_block_mul_f64(h, p, d.V + nk * i, Hi, -1.0, 1.0, d.w);
      }
      BCK(cudaMemcpyAsync(st_h, d.status, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, d.stream));
      std::vector<zc> Hall(pp * (j + 1));
      BCK(cudaMemcpyAsync(Hall.data(), dmat + pp, sizeof(cplx) * pp * (j + 1), cudaMemcpyDeviceToHost, d.stream));
      BCK(cudaStreamSynchronize(d.stream));
      if (int sc = status_code(h, st_h)) return sc;
      for (int i = 0; i <= j; ++i)
        for (int r = 0; r < p; ++r)
          for (int c = 0; c < p; ++c) col[(size_t)c * cr + (int64_t)i * p + r] = Hall[pp * i + (size_t)r * p + c];
      std::vector<zc> Hn;
      if (!cholqr2(d.w, Vn, Hn, err)) {
        if (err) return err;
        breakdown = true;
        h->err = "block FGMRES: a new Krylov block is numerically rank deficient";
        break;
      }
      prof_end(h, KC_ORTH, pb, 2 * (j + 1) + 4);
      for (int r = 0; r < p; ++r)
        for (int c = 0; c < p; ++c) col[(size_t)c * cr + (int64_t)(j + 1) * p + r] = Hn[(size_t)r * p + c];
      // previous reflections, then p new ones on rows [jp + c, (j+2)p)
      for (auto& rs : refl)
        for (auto& rf : rs)
          for (int c = 0; c < p; ++c) rf.apply(&col[(size_t)c * cr]);
      std::vector<Reflector> nr;
      for (int c = 0; c < p; ++c) {
        Reflector rf = make_reflector(&col[(size_t)c * cr], (int64_t)j * p + c, 2 * p - c);
        for (int c2 = c + 1; c2 < p; ++c2) rf.apply(&col[(size_t)c2 * cr]);
        for (int c2 = 0; c2 < p; ++c2) rf.apply(&Gt[(size_t)c2 * rows]);
        nr.push_back(std::move(rf));
      }
      refl.push_back(std::move(nr));
      Hcols.push_back(std::move(col));
      ++it;
      k = j + 1;
      bool done = true;
      for (int c = 0; c < p; ++c) {
        double e2 = 0.0;
        for (int r = 0; r < p; ++r) e2 += std::norm(Gt[(size_t)c * rows + (int64_t)k * p + r]);
        done &= std::sqrt(e2) / bnorm[c] <= tol;
      }
      if (done || it >= max_iter) break;
    }
    if (k == 0) break;
    // Y = R^{-1} G (block upper triangular kp x kp), x += sum_i Z_i Y_i
    const int64_t kp = (int64_t)k * p;
    std::vector<zc> Y((size_t)kp * p, zc(0.0));  // [row][c]
    for (int c = 0; c < p; ++c)
      for (int64_t r = kp - 1; r >= 0; --r) {
        zc s = Gt[(size_t)c * rows + r];
        for (int64_t q = r + 1; q < kp; ++q) {
          const int64_t bj = q / p, qc = q % p;
          s -= Hcols[bj][(size_t)qc * ((bj + 2) * p) + r] * Y[(size_t)q * p + c];
        }
        const int64_t bj = r / p, rc2 = r % p;
        const zc diag = Hcols[bj][(size_t)rc2 * ((bj + 2) * p) + r];
        Y[(size_t)r * p + c] = std::abs(diag) > 0.0 ? s / diag : zc(0.0);
      }
    for (int i = 0; i < k; ++i) {
      std::vector<zc> Yi(Y.begin() + (size_t)i * pp, Y.begin() + (size_t)(i + 1) * pp);
      if (int e = to_dev(Yi, dmat)) return e;
      if (d.factor_bits == 64) launch_block_mul_f64(h, p, d.Zd + nk * i, dmat, 1.0, 1.0, d.xk);
      else launch_block_mul_f32(h, p, (const char*)d.Zf + nk * i * 2 * sizeof(float), dmat, 1.0, 1.0, d.xk);
    }
    ++cycles;
    BCK(cudaGetLastError());
  }
#undef BCK
  for (int c = 0; c < p; ++c) {
    if (!info) break;
    info[c].iterations = it;
    info[c].restarts = cycles;
    info[c].converged = relres[c] <= tol ? 1 : 0;
    info[c].relres = relres[c];
    info[c].pad = 0;
  }
  return converged ? ORAS_OK : ORAS_NOT_CONVERGED;
}

}  // namespace oras
