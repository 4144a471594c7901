// GCRO-DR(m, k): GMRES with deflated restarting and a subspace recycled across a sequence of
// systems (Sec. 6 names recycling, GCRO-DR in particular, for the imaging loop's slowly varying
// systems; the paper prints no algorithm).  The method of Parks, de Sturler, Mackey, Johnson and
// Maiti (SIAM J. Sci. Comput. 28, 2006), on the right-preconditioned operator A_hat = A M^{-1}
// (x = M^{-1} y), one right-hand side:
//
// * the handle keeps U (N x k) from the previous solve; a solve first forms C from A_hat U by a
//   QR factorisation (A_hat U = C, C^H C = I, U <- U R^{-1});
// * a cycle projects the residual off C (x += U_x C^H r, r -= C C^H r), runs up to m - k Arnoldi
//   steps with (I - C C^H) A_hat (the first cycle without C: m steps of GMRES), re-solving the
//   small least-squares problem min || c - G z || after every step and stopping once its
//   estimate reaches tol; x += [U_x D, Z] z (D = diag(1 / ||u_i||), see below);
// * U and C are refreshed from the harmonic Ritz vectors of the cycle with the k smallest
//   harmonic Ritz values (first cycle: (H + |h|^2 H^{-H} e_m e_m^T) z = theta z; later:
//   G^H G z = theta G^H W^H V_hat z), P -> G P = Q R, C = W_hat Q, U = V_hat P R^{-1};
// * a cycle ends with the true residual r = b - A x.
//
// The iterate is kept flexibly, as in the FGMRES of oras_solve: every preconditioned vector
// Z_j = M^{-1} V_j is stored, U_x = M^{-1} U (with A U_x = C) is carried beside U, and x is
// accumulated from them (x += U_x C^H r, x += [U_x D, Z] z), so the Krylov relations hold in FP64
// even when M^{-1} is applied with FP32 factors; true residuals are b - A x (no apply).  U (the
// preconditioned space) defines the harmonic Ritz problems and is what a later system recycles:
// U_x = M_new^{-1} U, C from A U_x.
// Vectors live on the GPU as single columns (recycle.cu); the new Arnoldi vector is projected
// against [C, V] together by classical Gram-Schmidt with one reorthogonalisation (two dot passes),
// where the oracle takes modified Gram-Schmidt: both leave the basis orthonormal to rounding.
// W^H V_hat uses C^H V = 0 and V^H V = I from that orthonormality.  The small dense algebra
// (least squares, QR, eigenproblems; dense.cpp) is on the host in FP64.
#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <string>
#include <vector>

#include "internal.h"

namespace oras {

using zc = std::complex<double>;

bool dense_eig(int n, const std::vector<zc>& A, std::vector<zc>& w, std::vector<zc>& V);
void dense_qr(int p, int q, const std::vector<zc>& M, std::vector<zc>& Q, std::vector<zc>& R);
double dense_lstsq(int p, int q, const std::vector<zc>& G, const std::vector<zc>& c, std::vector<zc>& z);
bool dense_solve(int n, std::vector<zc> A, std::vector<zc> B, int nr, std::vector<zc>& X);
int rc_max_q();
size_t rc_partials_elems();
void launch_rc_dots(cudaStream_t st, int64_t n, int nq, const cplx* X, int64_t ldx, const cplx* w, cplx* partials,
                    cplx* out);
void launch_rc_lincomb(cudaStream_t st, int64_t n, int nq, int nc, const cplx* X, int64_t ldx, const cplx* M,
                       double beta, cplx* Y, int64_t ldy, double alpha = 1.0);
void launch_rc_scale(cudaStream_t st, int64_t n, const cplx* x, double s, cplx* out);
void launch_rc_widen(cudaStream_t st, int64_t n, const void* x, cplx* out);
int launch_apply_f64out(const oras_handle* h, const cplx* v, cplx* z, int k);
int launch_apply_f32out(const oras_handle* h, const cplx* v, void* z, int k);
void launch_spmv_f64(const oras_handle* h, const cplx* x, cplx* y, int k);
void launch_spmv_f32(const oras_handle* h, const void* x, cplx* y, int k);
int apply_passes(const oras_handle* h, int k);
int status_code(oras_handle* h, const int32_t* st);

namespace {

// indices of the k eigenvalues of smallest modulus (ties by index)
std::vector<int> smallest(const std::vector<zc>& theta, int k) {
  std::vector<int> idx(theta.size());
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return std::abs(theta[a]) < std::abs(theta[b]); });
  idx.resize(k);
  return idx;
}

struct Dev {
  cplx* p = nullptr;
  cudaStream_t s = nullptr;
  ~Dev() {
    if (p) cudaFreeAsync(p, s);
  }
};

}  // namespace

#define RK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      h->err = std::string("gcrodr: ") + #call + ": " + cudaGetErrorString(e_);       \
      return e_ == cudaErrorMemoryAllocation ? ORAS_ERR_OUT_OF_MEMORY : ORAS_ERR_CUDA; \
    }                                                                                 \
  } while (0)

// Solves A x = b (b = d.bk, x -> d.xk) for one right-hand side; info[0] gets the products with
// A_hat = A M^{-1} (Arnoldi steps and the k products that rebuild C from a recycled U), the
// cycles and the true relative residual.
int gcrodr_solve(oras_handle* h, double tol, oras_info* info) {
  auto& d = h->dev;
  const int64_t N = h->mesh.ndof;
  const int m = std::max(h->opt.restart, 2);
  const int kdef = std::min(h->opt.recycle, m - 1);
  const int max_mv = h->opt.max_iter > 0 ? h->opt.max_iter : 5000;
  cudaStream_t st = d.stream;
  // device columns: W = [C (kdef) | V (m + 1)], U, Unew, Cnew, Ux, Uxnew (kdef each), Z (m), x,
  // r, w, z
  const int ncol = kdef + (m + 1) + 5 * kdef + m + 4;
  Dev buf, part, small;
  buf.s = part.s = small.s = st;
  RK(cudaMallocAsync((void**)&buf.p, sizeof(cplx) * (size_t)N * ncol, st));
  RK(cudaMallocAsync((void**)&part.p, sizeof(cplx) * rc_partials_elems(), st));
  const size_t nsmall = (size_t)(kdef + m + 2) * std::max(kdef, 1) + 2 * (size_t)(kdef + m + 2) + 1;
  RK(cudaMallocAsync((void**)&small.p, sizeof(cplx) * nsmall, st));
  cplx* W = buf.p;
  cplx* V = W + (size_t)kdef * N;
  cplx* U = V + (size_t)(m + 1) * N;
  cplx* Unew = U + (size_t)kdef * N;
  cplx* Cnew = Unew + (size_t)kdef * N;
  cplx* Ux = Cnew + (size_t)kdef * N;
  cplx* Uxnew = Ux + (size_t)kdef * N;
  cplx* Z = Uxnew + (size_t)kdef * N;
  cplx* x = Z + (size_t)m * N;
  cplx* r = x + N;
  cplx* w = r + N;
  cplx* z = w + N;
  cplx* dM = small.p;                                  // small coefficient matrices
  cplx* dots = small.p + (size_t)(kdef + m + 2) * std::max(kdef, 1);
  std::vector<cplx> hbuf(2 * (kdef + m + 2) + 1);
  int32_t st_h[8];
  auto put_small = [&](const std::vector<zc>& M) -> int {
    RK(cudaMemcpyAsync(dM, M.data(), sizeof(cplx) * M.size(), cudaMemcpyHostToDevice, st));
    return ORAS_OK;
  };
  auto get_dots = [&](int nq, std::vector<zc>& out) -> int {
    RK(cudaMemcpyAsync(hbuf.data(), dots, sizeof(cplx) * nq, cudaMemcpyDeviceToHost, st));
    RK(cudaStreamSynchronize(st));
    out.resize(nq);
    for (int q = 0; q < nq; ++q) out[q] = zc(hbuf[q].re, hbuf[q].im);
    return ORAS_OK;
  };
  auto norm_of = [&](const cplx* v, double& out) -> int {
    launch_rc_dots(st, N, 1, v, N, v, part.p, dots);
    std::vector<zc> t;
    if (int rc = get_dots(1, t)) return rc;
    out = std::sqrt(std::max(t[0].real(), 0.0));
    return ORAS_OK;
  };
  // zv = M^{-1} v, out = A zv.  With FP32 factors M^{-1} v is FP32-valued: the apply writes it
  // in FP32, the SpMV takes the FP32-pipe error-free kernel (FP64-class result), and zv is its
  // exact FP64 copy
  const bool f32 = d.factor_bits == 32;
  auto op = [&](const cplx* v, cplx* zv, cplx* out) -> int {
    int pb = prof_begin(h);
    const int arc = f32 ? launch_apply_f32out(h, v, (void*)z, 1) : launch_apply_f64out(h, v, zv, 1);
    if (arc) { h->err = "gcrodr: apply launch failed"; return ORAS_ERR_CUDA; }
    prof_end(h, KC_APPLY, pb, apply_passes(h, 1));
    pb = prof_begin(h);
    if (f32) {
      launch_spmv_f32(h, (const void*)z, out, 1);
      launch_rc_widen(st, N, (const void*)z, zv);
    } else {
      launch_spmv_f64(h, zv, out, 1);
    }
    prof_end(h, f32 ? KC_SPMV : KC_SPMV64, pb, f32 ? 2 : 1);
    return ORAS_OK;
  };
  // Y = beta Y + X coef (coef host, nq)
  auto add_comb = [&](const cplx* X, int nq, const std::vector<zc>& coef, double beta, cplx* Y) -> int {
    if (nq == 0) return ORAS_OK;
    if (int rc = put_small(coef)) return rc;
    launch_rc_lincomb(st, N, nq, 1, X, N, dM, beta, Y, N);
    return ORAS_OK;
  };
  RK(cudaMemsetAsync(d.status, 0, 8 * sizeof(int32_t), st));
  RK(cudaMemsetAsync(x, 0, sizeof(cplx) * N, st));
  double bnorm = 0.0;
  if (int rc = norm_of(d.bk, bnorm)) return rc;
  int mv = 0, cycles = 0;
  bool conv = false;
  double relres = 0.0;
  if (bnorm == 0.0) {
    RK(cudaMemsetAsync(d.xk, 0, sizeof(cplx) * N, st));
    if (info) { info[0] = oras_info{}; info[0].converged = 1; }
    return ORAS_OK;
  }
  int kk = 0;  // columns of C and U in use
  if (kdef > 0 && h->rc_k == kdef && h->rc_U && h->rc_n == N) {
    // recycled U: U_x = M^{-1} U, C = A U_x by QR (classical Gram-Schmidt, reorthogonalised),
    // U <- U R^{-1}, U_x <- U_x R^{-1}
    RK(cudaMemcpyAsync(U, h->rc_U, sizeof(cplx) * N * kdef, cudaMemcpyDeviceToDevice, st));
    std::vector<zc> R((size_t)kdef * kdef, zc(0.0));
    for (int c = 0; c < kdef; ++c) {
      cplx* a = W + (size_t)c * N;
      if (int rc = op(U + (size_t)c * N, Ux + (size_t)c * N, a)) return rc;
      ++mv;
      for (int pass = 0; pass < 2 && c > 0; ++pass) {
        launch_rc_dots(st, N, c, W, N, a, part.p, dots);
        std::vector<zc> t;
        if (int rc = get_dots(c, t)) return rc;
        std::vector<zc> neg(c);
        for (int q = 0; q < c; ++q) {
          R[(size_t)q * kdef + c] += t[q];
          neg[q] = -t[q];
        }
        if (int rc = add_comb(W, c, neg, 1.0, a)) return rc;
      }
      double nr = 0.0;
      if (int rc = norm_of(a, nr)) return rc;
      if (!(nr > 0.0)) { h->err = "gcrodr: recycled subspace is rank deficient"; return ORAS_NOT_CONVERGED; }
      R[(size_t)c * kdef + c] = nr;
      launch_rc_scale(st, N, a, 1.0 / nr, a);
    }
    // U <- U R^{-1}
    std::vector<zc> Id((size_t)kdef * kdef, zc(0.0)), Rinv;
    for (int i = 0; i < kdef; ++i) Id[(size_t)i * kdef + i] = 1.0;
    if (!dense_solve(kdef, R, Id, kdef, Rinv)) { h->err = "gcrodr: singular R"; return ORAS_NOT_CONVERGED; }
    if (int rc = put_small(Rinv)) return rc;
    launch_rc_lincomb(st, N, kdef, kdef, U, N, dM, 0.0, Unew, N);
    launch_rc_lincomb(st, N, kdef, kdef, Ux, N, dM, 0.0, Uxnew, N);
    std::swap(U, Unew);
    std::swap(Ux, Uxnew);
    kk = kdef;
  }
  RK(cudaMemcpyAsync(r, d.bk, sizeof(cplx) * N, cudaMemcpyDeviceToDevice, st));
  for (;;) {
    if (kk) {  // x += U_x C^H r, r -= C C^H r
      launch_rc_dots(st, N, kk, W, N, r, part.p, dots);
      std::vector<zc> t;
      if (int rc = get_dots(kk, t)) return rc;
      if (int rc = add_comb(Ux, kk, t, 1.0, x)) return rc;
      std::vector<zc> neg(kk);
      for (int q = 0; q < kk; ++q) neg[q] = -t[q];
      if (int rc = add_comb(W, kk, neg, 1.0, r)) return rc;
    }
    double rn = 0.0;
    if (int rc = norm_of(r, rn)) return rc;
    relres = rn / bnorm;
    if (relres <= tol || mv >= max_mv) break;
    // ---- one cycle
    const int steps = std::min(kk ? m - kk : m, max_mv - mv);
    cplx* Wc = kk ? W : V;  // [C, V] as one block of columns
    std::vector<zc> G((size_t)(kk + steps + 1) * (kk + steps), zc(0.0));
    const int gq = kk + steps;  // row stride of G
    auto g = [&](int i, int j) -> zc& { return G[(size_t)i * gq + j]; };
    std::vector<double> unorm(kk);
    for (int i = 0; i < kk; ++i) {
      if (int rc = norm_of(U + (size_t)i * N, unorm[i])) return rc;
      g(i, i) = 1.0 / unorm[i];
    }
    launch_rc_scale(st, N, r, 1.0 / rn, V);
    std::vector<zc> cvec(kk + steps + 1, zc(0.0)), zs;
    cvec[kk] = rn;
    // least squares min || c - G z || kept by Givens rotations as the columns arrive: G is upper
    // Hessenberg (its leading k x k block is diagonal), so column kk + j needs the rotations of the
    // earlier columns and one new rotation; |rotated c[kk + j + 1]| is the residual estimate
    std::vector<zc> Rg((size_t)(kk + steps) * (kk + steps), zc(0.0)), gr(cvec), rs(kk + steps);
    std::vector<double> rc_(kk + steps);
    const int rq = kk + steps;  // row stride of Rg
    for (int i = 0; i < kk; ++i) Rg[(size_t)i * rq + i] = g(i, i);
    int nst = 0;
    for (int j = 0; j < steps; ++j) {
      cplx* vj = V + (size_t)j * N;
      if (int rc = op(vj, Z + (size_t)j * N, w)) return rc;
      ++mv;
      int pb = prof_begin(h);
      const int nq = kk + j + 1;
      // w -= [C, V_0..V_j] ([C, V]^H w), twice (coefficients stay on the device), then ||w||
      cplx* d1 = dots;
      cplx* d2 = dots + nq;
      cplx* dn = dots + 2 * nq;
      launch_rc_dots(st, N, nq, Wc, N, w, part.p, d1);
      launch_rc_lincomb(st, N, nq, 1, Wc, N, d1, 1.0, w, N, -1.0);
      launch_rc_dots(st, N, nq, Wc, N, w, part.p, d2);
      launch_rc_lincomb(st, N, nq, 1, Wc, N, d2, 1.0, w, N, -1.0);
      launch_rc_dots(st, N, 1, w, N, w, part.p, dn);
      RK(cudaMemcpyAsync(hbuf.data(), dots, sizeof(cplx) * (2 * nq + 1), cudaMemcpyDeviceToHost, st));
      RK(cudaMemcpyAsync(st_h, d.status, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      RK(cudaStreamSynchronize(st));
      if (int sc = status_code(h, st_h)) return sc;
      const double hn = std::sqrt(std::max(hbuf[2 * nq].re, 0.0));
      for (int q = 0; q < nq; ++q)
        g(q, kk + j) = zc(hbuf[q].re + hbuf[nq + q].re, hbuf[q].im + hbuf[nq + q].im);
      g(kk + j + 1, kk + j) = hn;
      if (hn > 0.0) launch_rc_scale(st, N, w, 1.0 / hn, V + (size_t)(j + 1) * N);
      prof_end(h, KC_ORTH, pb, 4 * ((nq + rc_max_q() - 1) / rc_max_q()) + 5);
      nst = j + 1;
      // the new column through the earlier rotations, then its own rotation
      const int cj = kk + j;
      std::vector<zc> col(cj + 2);
      for (int i = 0; i <= cj + 1; ++i) col[i] = g(i, cj);
      for (int i = kk; i < cj; ++i) {
        const zc x = col[i], y_ = col[i + 1];
        col[i] = rc_[i] * x + rs[i] * y_;
        col[i + 1] = -std::conj(rs[i]) * x + rc_[i] * y_;
      }
      {
        const zc a = col[cj], b = col[cj + 1];
        const double r = std::hypot(std::abs(a), std::abs(b));
        double c;
        zc s;
        if (r == 0.0) { c = 1.0; s = 0.0; }
        else if (std::abs(a) == 0.0) { c = 0.0; s = std::conj(b) / std::abs(b); }
        else { c = std::abs(a) / r; s = (a / std::abs(a)) * std::conj(b) / r; }
        rc_[cj] = c;
        rs[cj] = s;
        col[cj] = c * a + s * b;
        const zc x = gr[cj], y_ = gr[cj + 1];
        gr[cj] = c * x + s * y_;
        gr[cj + 1] = -std::conj(s) * x + c * y_;
      }
      for (int i = 0; i <= cj; ++i) Rg[(size_t)i * rq + cj] = col[i];
      const double est = std::abs(gr[cj + 1]) / bnorm;
      if (est <= tol || hn == 0.0) break;
    }
    {  // z from the triangular factor
      const int q = kk + nst;
      zs.assign(q, zc(0.0));
      for (int i = q - 1; i >= 0; --i) {
        zc s = gr[i];
        for (int c = i + 1; c < q; ++c) s -= Rg[(size_t)i * rq + c] * zs[c];
        zs[i] = s / Rg[(size_t)i * rq + i];
      }
    }
    ++cycles;
    const int p = kk + nst + 1, q = kk + nst;
    std::vector<zc> Gc((size_t)p * q);
    for (int i = 0; i < p; ++i)
      for (int c = 0; c < q; ++c) Gc[(size_t)i * q + c] = g(i, c);
    // x += [U_x D, Z] z
    {
      std::vector<zc> zu(kk), zv(zs.begin() + kk, zs.begin() + q);
      for (int i = 0; i < kk; ++i) zu[i] = zs[i] / unorm[i];
      if (int rc = add_comb(Ux, kk, zu, 1.0, x)) return rc;
      RK(cudaStreamSynchronize(st));  // the coefficient buffer is rewritten next
      if (int rc = add_comb(Z, nst, zv, 1.0, x)) return rc;
    }
    // deflation space from the cycle
    const int knew = kk ? kk : (kdef > 0 && nst >= kdef ? kdef : 0);
    if (knew > 0) {
      std::vector<zc> theta, EV;
      int nz;  // rows of P
      if (!kk) {  // harmonic Ritz vectors of the GMRES cycle
        nz = nst;
        std::vector<zc> H((size_t)nst * nst);
        for (int i = 0; i < nst; ++i)
          for (int c = 0; c < nst; ++c) H[(size_t)i * nst + c] = g(i, c);
        const zc hnext = g(nst, nst - 1);
        std::vector<zc> Hh((size_t)nst * nst), em(nst, zc(0.0)), f;
        em[nst - 1] = 1.0;
        for (int i = 0; i < nst; ++i)
          for (int c = 0; c < nst; ++c) Hh[(size_t)i * nst + c] = std::conj(H[(size_t)c * nst + i]);
        if (!dense_solve(nst, Hh, em, 1, f)) { h->err = "gcrodr: singular H"; return ORAS_NOT_CONVERGED; }
        for (int i = 0; i < nst; ++i)
          for (int c = 0; c < nst; ++c)
            Hh[(size_t)i * nst + c] = H[(size_t)i * nst + c] + (c == nst - 1 ? std::norm(hnext) * f[i] : zc(0.0));
        if (!dense_eig(nst, Hh, theta, EV)) { h->err = "gcrodr: eigenproblem did not converge"; return ORAS_NOT_CONVERGED; }
      } else {  // G^H G z = theta G^H (W^H V_hat) z
        nz = q;
        std::vector<zc> WhV((size_t)p * q, zc(0.0));
        for (int c = 0; c < kk; ++c) {  // [C, V]^H u_c / ||u_c||
          launch_rc_dots(st, N, p, W, N, U + (size_t)c * N, part.p, dots);
          std::vector<zc> t;
          if (int rc = get_dots(p, t)) return rc;
          for (int i = 0; i < p; ++i) WhV[(size_t)i * q + c] = t[i] / unorm[c];
        }
        for (int c = 0; c < nst; ++c) WhV[(size_t)(kk + c) * q + kk + c] = 1.0;  // V^H V = I, C^H V = 0
        std::vector<zc> A((size_t)q * q, zc(0.0)), B((size_t)q * q, zc(0.0)), M;
        for (int i = 0; i < q; ++i)
          for (int c = 0; c < q; ++c)
            for (int l = 0; l < p; ++l) {
              A[(size_t)i * q + c] += std::conj(Gc[(size_t)l * q + i]) * Gc[(size_t)l * q + c];
              B[(size_t)i * q + c] += std::conj(Gc[(size_t)l * q + i]) * WhV[(size_t)l * q + c];
            }
        if (!dense_solve(q, B, A, q, M)) { h->err = "gcrodr: singular G^H W^H V"; return ORAS_NOT_CONVERGED; }
        if (!dense_eig(q, M, theta, EV)) { h->err = "gcrodr: eigenproblem did not converge"; return ORAS_NOT_CONVERGED; }
      }
      const std::vector<int> sel = smallest(theta, knew);
      std::vector<zc> P((size_t)nz * knew);
      for (int i = 0; i < nz; ++i)
        for (int c = 0; c < knew; ++c) P[(size_t)i * knew + c] = EV[(size_t)i * nz + sel[c]];
      // G P = Q R
      const int pr = kk ? p : nst + 1;
      std::vector<zc> GP((size_t)pr * knew, zc(0.0)), Qm, Rm;
      for (int i = 0; i < pr; ++i)
        for (int c = 0; c < knew; ++c)
          for (int l = 0; l < nz; ++l) GP[(size_t)i * knew + c] += Gc[(size_t)i * q + l] * P[(size_t)l * knew + c];
      dense_qr(pr, knew, GP, Qm, Rm);
      std::vector<zc> Id((size_t)knew * knew, zc(0.0)), Rinv;
      for (int i = 0; i < knew; ++i) Id[(size_t)i * knew + i] = 1.0;
      if (!dense_solve(knew, Rm, Id, knew, Rinv)) { h->err = "gcrodr: singular R"; return ORAS_NOT_CONVERGED; }
      // PR = P R^{-1}; U_new = [U D, V] PR, U_x,new = [U_x D, Z] PR; C_new = [C, V] Q
      std::vector<zc> PR((size_t)nz * knew, zc(0.0));
      for (int i = 0; i < nz; ++i)
        for (int c = 0; c < knew; ++c)
          for (int l = 0; l < knew; ++l) PR[(size_t)i * knew + c] += P[(size_t)i * knew + l] * Rinv[(size_t)l * knew + c];
      if (kk) {
        std::vector<zc> top((size_t)kk * knew), bot(PR.begin() + (size_t)kk * knew, PR.end());
        for (int i = 0; i < kk; ++i)
          for (int c = 0; c < knew; ++c) top[(size_t)i * knew + c] = PR[(size_t)i * knew + c] / unorm[i];
        if (int rc = put_small(top)) return rc;
        launch_rc_lincomb(st, N, kk, knew, U, N, dM, 0.0, Unew, N);
        launch_rc_lincomb(st, N, kk, knew, Ux, N, dM, 0.0, Uxnew, N);
        RK(cudaStreamSynchronize(st));  // dM is rewritten next
        if (int rc = put_small(bot)) return rc;
        launch_rc_lincomb(st, N, nst, knew, V, N, dM, 1.0, Unew, N);
        launch_rc_lincomb(st, N, nst, knew, Z, N, dM, 1.0, Uxnew, N);
      } else {
        if (int rc = put_small(PR)) return rc;
        launch_rc_lincomb(st, N, nst, knew, V, N, dM, 0.0, Unew, N);
        launch_rc_lincomb(st, N, nst, knew, Z, N, dM, 0.0, Uxnew, N);
      }
      RK(cudaStreamSynchronize(st));
      if (int rc = put_small(Qm)) return rc;
      launch_rc_lincomb(st, N, pr, knew, Wc, N, dM, 0.0, Cnew, N);
      RK(cudaMemcpyAsync(W, Cnew, sizeof(cplx) * N * knew, cudaMemcpyDeviceToDevice, st));
      std::swap(U, Unew);
      std::swap(Ux, Uxnew);
      kk = knew;
    }
    // true residual r = b - A x
    {
      int pb = prof_begin(h);
      launch_spmv_f64(h, x, w, 1);
      prof_end(h, KC_SPMV64, pb, 1);
    }
    std::vector<zc> one = {zc(-1.0)};
    RK(cudaMemcpyAsync(r, d.bk, sizeof(cplx) * N, cudaMemcpyDeviceToDevice, st));
    if (int rc = add_comb(w, 1, one, 1.0, r)) return rc;
    RK(cudaStreamSynchronize(st));
  }
  conv = relres <= tol;
  // keep U for the next system; x = M^{-1} y
  if (kdef > 0 && kk == kdef) {
    if (!h->rc_U || h->rc_n != N || h->rc_k != kdef) {
      if (h->rc_U) cudaFreeAsync(h->rc_U, st);
      h->rc_U = nullptr;
      RK(cudaMallocAsync((void**)&h->rc_U, sizeof(cplx) * N * kdef, st));
      h->rc_n = N;
      h->rc_k = kdef;
    }
    RK(cudaMemcpyAsync(h->rc_U, U, sizeof(cplx) * N * kdef, cudaMemcpyDeviceToDevice, st));
  }
  RK(cudaMemcpyAsync(d.xk, x, sizeof(cplx) * N, cudaMemcpyDeviceToDevice, st));
  // the true residual of the returned x
  RK(cudaMemcpyAsync(r, d.bk, sizeof(cplx) * N, cudaMemcpyDeviceToDevice, st));
  launch_spmv_f64(h, d.xk, w, 1);
  {
    std::vector<zc> one = {zc(-1.0)};
    if (int rc = add_comb(w, 1, one, 1.0, r)) return rc;
  }
  double rn = 0.0;
  if (int rc = norm_of(r, rn)) return rc;
  relres = rn / bnorm;
  conv = relres <= tol;
  if (info) {
    info[0].iterations = mv;
    info[0].restarts = cycles;
    info[0].converged = conv ? 1 : 0;
    info[0].relres = relres;
    info[0].pad = 0;
  }
  return conv ? ORAS_OK : ORAS_NOT_CONVERGED;
}

}  // namespace oras

extern "C" int oras_recycle_reset(oras_handle* h) {
  if (!h) return ORAS_ERR_INVALID_ARG;
  if (h->rc_U) cudaFreeAsync(h->rc_U, h->dev.stream);
  h->rc_U = nullptr;
  h->rc_k = 0;
  h->rc_n = 0;
  return ORAS_OK;
}
