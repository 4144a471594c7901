// Small dense complex linear algebra on the host for the recycling solver (GCRO-DR, Sec. 6): its
// least-squares problems, QR factorisations and harmonic Ritz eigenproblems are (m+k)-sized,
// m + k <= a few hundred.  Row-major storage throughout.
//
// Eigen-decomposition: the textbook QR algorithm (Golub & Van Loan, Matrix Computations, ch. 7):
// Householder reduction to upper Hessenberg form, shifted QR steps with Givens rotations and the
// Wilkinson shift on the active unreduced block (deflation when a subdiagonal entry is below
// eps (|h_ii| + |h_i+1,i+1|), an exceptional shift every 10 steps without deflation), the Schur
// vectors accumulated; eigenvectors by back substitution with the triangular Schur factor.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <vector>

#include "../../include/oras.h"

namespace oras {

using zc = std::complex<double>;
constexpr double DEPS = 2.220446049250313e-16;

// A = Q T Q^H: T upper triangular (in place of A), Q unitary.  Returns false if the QR steps did
// not converge within 60 n steps.
bool schur(int n, std::vector<zc>& H, std::vector<zc>& Q) {
  Q.assign((size_t)n * n, zc(0.0));
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  auto h = [&](int i, int j) -> zc& { return H[(size_t)i * n + j]; };
  auto q = [&](int i, int j) -> zc& { return Q[(size_t)i * n + j]; };
  // Householder reduction to Hessenberg form
  std::vector<zc> v(n);
  for (int k = 0; k + 2 < n; ++k) {
    double xn = 0.0;
    for (int i = k + 1; i < n; ++i) xn += std::norm(h(i, k));
    xn = std::sqrt(xn);
    if (xn == 0.0) continue;
    const zc x0 = h(k + 1, k);
    const zc ph = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : zc(1.0);
    const zc alpha = -ph * xn;
    double vn = 0.0;
    for (int i = k + 1; i < n; ++i) {
      v[i] = h(i, k) - (i == k + 1 ? alpha : zc(0.0));
      vn += std::norm(v[i]);
    }
    vn = std::sqrt(vn);
    if (vn == 0.0) continue;
    for (int i = k + 1; i < n; ++i) v[i] /= vn;
    // H <- (I - 2 v v^H) H (I - 2 v v^H); Q <- Q (I - 2 v v^H)
    for (int j = 0; j < n; ++j) {
      zc s = 0.0;
      for (int i = k + 1; i < n; ++i) s += std::conj(v[i]) * h(i, j);
      for (int i = k + 1; i < n; ++i) h(i, j) -= 2.0 * v[i] * s;
    }
    for (int i = 0; i < n; ++i) {
      zc s = 0.0;
      for (int j = k + 1; j < n; ++j) s += h(i, j) * v[j];
      for (int j = k + 1; j < n; ++j) h(i, j) -= 2.0 * s * std::conj(v[j]);
      zc t = 0.0;
      for (int j = k + 1; j < n; ++j) t += q(i, j) * v[j];
      for (int j = k + 1; j < n; ++j) q(i, j) -= 2.0 * t * std::conj(v[j]);
    }
    for (int i = k + 2; i < n; ++i) h(i, k) = 0.0;
  }
  // shifted QR steps
  int hi = n - 1, iter = 0, total = 0;
  std::vector<double> cs(n);
  std::vector<zc> sn(n);
  while (hi > 0) {
    int l = hi;
    while (l > 0 && std::abs(h(l, l - 1)) > DEPS * (std::abs(h(l - 1, l - 1)) + std::abs(h(l, l)))) --l;
    if (l > 0) h(l, l - 1) = 0.0;
    if (l == hi) {  // h(hi, hi) has converged
      --hi;
      iter = 0;
      continue;
    }
    if (++total > 60 * n) return false;
    ++iter;
    zc mu;
    if (iter % 10 == 0) {  // exceptional shift
      mu = h(hi, hi) + 0.75 * std::abs(h(hi, hi - 1));
    } else {  // Wilkinson: the eigenvalue of the trailing 2 x 2 block closer to h(hi, hi)
      const zc a = h(hi - 1, hi - 1), b = h(hi - 1, hi), c = h(hi, hi - 1), d = h(hi, hi);
      const zc tr = a + d, det = a * d - b * c;
      const zc disc = std::sqrt(tr * tr * 0.25 - det);
      const zc m1 = tr * 0.5 + disc, m2 = tr * 0.5 - disc;
      mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
    }
    for (int i = l; i <= hi; ++i) h(i, i) -= mu;
    // H - mu I = R by Givens rotations G_i (rows i, i+1), then R G^H and back + mu I
    for (int i = l; i < hi; ++i) {
      const zc a = h(i, i), b = h(i + 1, i);
      const double r = std::hypot(std::abs(a), std::abs(b));
      double c;
      zc s;
      if (r == 0.0) {
        c = 1.0;
        s = 0.0;
      } else if (std::abs(a) == 0.0) {
        c = 0.0;
        s = std::conj(b) / std::abs(b);
      } else {
        c = std::abs(a) / r;
        s = (a / std::abs(a)) * std::conj(b) / r;
      }
      cs[i] = c;
      sn[i] = s;
      for (int j = i; j < n; ++j) {
        const zc x = h(i, j), y = h(i + 1, j);
        h(i, j) = c * x + s * y;
        h(i + 1, j) = -std::conj(s) * x + c * y;
      }
    }
    for (int i = l; i < hi; ++i) {
      const double c = cs[i];
      const zc s = sn[i];
      const int pmax = std::min(i + 2, hi);
      for (int p = 0; p <= pmax; ++p) {
        const zc x = h(p, i), y = h(p, i + 1);
        h(p, i) = x * c + y * std::conj(s);
        h(p, i + 1) = -x * s + y * c;
      }
      for (int p = 0; p < n; ++p) {
        const zc x = q(p, i), y = q(p, i + 1);
        q(p, i) = x * c + y * std::conj(s);
        q(p, i + 1) = -x * s + y * c;
      }
    }
    for (int i = l; i <= hi; ++i) h(i, i) += mu;
  }
  for (int i = 1; i < n; ++i)
    for (int j = 0; j < i; ++j) h(i, j) = 0.0;
  return true;
}

// Eigenvalues w[n] and unit eigenvectors (columns of V, row-major n x n) of A (row-major n x n).
bool dense_eig(int n, const std::vector<zc>& A, std::vector<zc>& w, std::vector<zc>& V) {
  std::vector<zc> T(A), Q;
  if (!schur(n, T, Q)) return false;
  double tn = 0.0;
  for (const zc& x : T) tn = std::max(tn, std::abs(x));
  const double small = DEPS * std::max(tn, 1e-300);
  w.resize(n);
  V.assign((size_t)n * n, zc(0.0));
  std::vector<zc> y(n);
  for (int j = 0; j < n; ++j) {
    const zc lam = T[(size_t)j * n + j];
    w[j] = lam;
    std::fill(y.begin(), y.end(), zc(0.0));
    y[j] = 1.0;
    for (int i = j - 1; i >= 0; --i) {
      zc s = 0.0;
      for (int p = i + 1; p <= j; ++p) s += T[(size_t)i * n + p] * y[p];
      zc den = T[(size_t)i * n + i] - lam;
      if (std::abs(den) < small) den = small;
      y[i] = -s / den;
    }
    double nrm = 0.0;
    for (int i = 0; i < n; ++i) {
      zc s = 0.0;
      for (int p = 0; p <= j; ++p) s += Q[(size_t)i * n + p] * y[p];
      V[(size_t)i * n + j] = s;
      nrm += std::norm(s);
    }
    nrm = std::sqrt(nrm);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + j] /= nrm;
  }
  return true;
}

// Reduced QR of M (p x q, p >= q): M = Q R, Q p x q with orthonormal columns, R q x q upper
// triangular (Householder).
void dense_qr(int p, int q, const std::vector<zc>& M, std::vector<zc>& Q, std::vector<zc>& R) {
  std::vector<zc> A(M);
  std::vector<std::vector<zc>> vs(q);
  for (int k = 0; k < q; ++k) {
    double xn = 0.0;
    for (int i = k; i < p; ++i) xn += std::norm(A[(size_t)i * q + k]);
    xn = std::sqrt(xn);
    std::vector<zc> v(p, zc(0.0));
    if (xn > 0.0) {
      const zc x0 = A[(size_t)k * q + k];
      const zc ph = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : zc(1.0);
      double vn = 0.0;
      for (int i = k; i < p; ++i) {
        v[i] = A[(size_t)i * q + k] + (i == k ? ph * xn : zc(0.0));
        vn += std::norm(v[i]);
      }
      vn = std::sqrt(vn);
      for (int i = k; i < p; ++i) v[i] /= vn;
      for (int j = k; j < q; ++j) {
        zc s = 0.0;
        for (int i = k; i < p; ++i) s += std::conj(v[i]) * A[(size_t)i * q + j];
        for (int i = k; i < p; ++i) A[(size_t)i * q + j] -= 2.0 * v[i] * s;
      }
    }
    vs[k] = std::move(v);
  }
  R.assign((size_t)q * q, zc(0.0));
  for (int i = 0; i < q; ++i)
    for (int j = i; j < q; ++j) R[(size_t)i * q + j] = A[(size_t)i * q + j];
  // Q = H_0 H_1 ... H_{q-1} [I; 0]
  Q.assign((size_t)p * q, zc(0.0));
  for (int i = 0; i < q; ++i) Q[(size_t)i * q + i] = 1.0;
  for (int k = q - 1; k >= 0; --k) {
    const std::vector<zc>& v = vs[k];
    for (int j = 0; j < q; ++j) {
      zc s = 0.0;
      for (int i = k; i < p; ++i) s += std::conj(v[i]) * Q[(size_t)i * q + j];
      for (int i = k; i < p; ++i) Q[(size_t)i * q + j] -= 2.0 * v[i] * s;
    }
  }
}

// min || c - G z || for G p x q (p >= q, full column rank): z[q]; returns the residual norm.
double dense_lstsq(int p, int q, const std::vector<zc>& G, const std::vector<zc>& c, std::vector<zc>& z) {
  std::vector<zc> Q, R;
  dense_qr(p, q, G, Q, R);
  std::vector<zc> t(q, zc(0.0));
  for (int j = 0; j < q; ++j)
    for (int i = 0; i < p; ++i) t[j] += std::conj(Q[(size_t)i * q + j]) * c[i];
  z.assign(q, zc(0.0));
  for (int i = q - 1; i >= 0; --i) {
    zc s = t[i];
    for (int j = i + 1; j < q; ++j) s -= R[(size_t)i * q + j] * z[j];
    z[i] = s / R[(size_t)i * q + i];
  }
  double rn = 0.0;
  for (int i = 0; i < p; ++i) {
    zc s = c[i];
    for (int j = 0; j < q; ++j) s -= G[(size_t)i * q + j] * z[j];
    rn += std::norm(s);
  }
  return std::sqrt(rn);
}

// X = A^{-1} B (A n x n, B n x nr, row-major), LU with partial pivoting; false if singular.
bool dense_solve(int n, std::vector<zc> A, std::vector<zc> B, int nr, std::vector<zc>& X) {
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::abs(A[(size_t)i * n + k]) > std::abs(A[(size_t)p * n + k])) p = i;
    if (std::abs(A[(size_t)p * n + k]) == 0.0) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
      for (int j = 0; j < nr; ++j) std::swap(B[(size_t)k * nr + j], B[(size_t)p * nr + j]);
    }
    for (int i = k + 1; i < n; ++i) {
      const zc l = A[(size_t)i * n + k] / A[(size_t)k * n + k];
      A[(size_t)i * n + k] = l;
      for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
      for (int j = 0; j < nr; ++j) B[(size_t)i * nr + j] -= l * B[(size_t)k * nr + j];
    }
  }
  X.assign((size_t)n * nr, zc(0.0));
  for (int j = 0; j < nr; ++j)
    for (int i = n - 1; i >= 0; --i) {
      zc s = B[(size_t)i * nr + j];
      for (int q = i + 1; q < n; ++q) s -= A[(size_t)i * n + q] * X[(size_t)q * nr + j];
      X[(size_t)i * nr + j] = s / A[(size_t)i * n + i];
    }
  return true;
}

}  // namespace oras

extern "C" int oras_dense_eig(int32_t n, const oras_complex* A, oras_complex* w, oras_complex* V) {
  if (n < 1 || !A || !w) return ORAS_ERR_INVALID_ARG;
  std::vector<oras::zc> M((size_t)n * n), ev, vec;
  for (size_t i = 0; i < M.size(); ++i) M[i] = oras::zc(A[i].re, A[i].im);
  if (!oras::dense_eig(n, M, ev, vec)) return ORAS_NOT_CONVERGED;
  for (int i = 0; i < n; ++i) w[i] = {ev[i].real(), ev[i].imag()};
  if (V)
    for (size_t i = 0; i < vec.size(); ++i) V[i] = {vec[i].real(), vec[i].imag()};
  return ORAS_OK;
}
