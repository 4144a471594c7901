// Element matrices (Sec. 2-3), global CSR values, dense local matrices A_s (Sec. 4) and
// right-hand sides, on the GPU in FP64.
#include <cstdio>

#include "dev.cuh"

namespace oras {

// ------------------------------------------------------------------ element matrices
// A_T[a][b] = mu_r^{-1} |T| sum_u ck[a][b][u] H_u  -  k0^2 eps_r |T| sum_u cm[a][b][u] G_u
// G_u: unique entries of G_pq = grad l_p . grad l_q; H_u: unique entries of the Gram matrix of the
// six cross products grad l_p x grad l_m (p < m), H = G_pq G_mn - G_pn G_mq.
constexpr int EL_TETS = 4;

__global__ void k_element(int64_t nt, int nl, const double* __restrict__ xyz,
                          const int32_t* __restrict__ st, const cplx* __restrict__ eps,
                          const cplx* __restrict__ mu, double k0sq, const double* __restrict__ cm,
                          const double* __restrict__ ck, cplx* __restrict__ out) {
  __shared__ double sg[EL_TETS][10], sh[EL_TETS][21], svol[EL_TETS];
  __shared__ cplx smu[EL_TETS], seps[EL_TETS];
  const int64_t t0 = (int64_t)blockIdx.x * EL_TETS;
  if (threadIdx.x < EL_TETS && t0 + threadIdx.x < nt) {
    int64_t t = t0 + threadIdx.x;
    int32_t v[4];
    for (int q = 0; q < 4; ++q) v[q] = st[t * 4 + q];
    double gl[4][3], vol;
    tet_geometry(xyz, v, gl, vol);
    double G[4][4];
    for (int p = 0; p < 4; ++p)
      for (int q = 0; q < 4; ++q) G[p][q] = gl[p][0] * gl[q][0] + gl[p][1] * gl[q][1] + gl[p][2] * gl[q][2];
    for (int p = 0; p < 4; ++p)
      for (int q = p; q < 4; ++q) sg[threadIdx.x][sym10(p, q)] = G[p][q];
    const int E[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    int idx = 0;
    for (int u = 0; u < 6; ++u)
      for (int w = u; w < 6; ++w) {
        int p = E[u][0], m = E[u][1], q = E[w][0], n = E[w][1];
        sh[threadIdx.x][idx++] = G[p][q] * G[m][n] - G[p][n] * G[m][q];
      }
    svol[threadIdx.x] = vol;
    cplx mm = mu ? mu[t] : cplx{1.0, 0.0};
    double den = mm.re * mm.re + mm.im * mm.im;
    smu[threadIdx.x] = {mm.re / den, -mm.im / den};  // 1 / mu_r
    seps[threadIdx.x] = eps[t];
  }
  __syncthreads();
  const int per = nl * nl;
  for (int e = threadIdx.x; e < EL_TETS * per; e += blockDim.x) {
    int lt = e / per, ab = e % per;
    int64_t t = t0 + lt;
    if (t >= nt) break;
    const double* cmr = cm + (int64_t)ab * 10;
    const double* ckr = ck + (int64_t)ab * 21;
    double m = 0.0, k = 0.0;
#pragma unroll
    for (int u = 0; u < 10; ++u) m += cmr[u] * sg[lt][u];
#pragma unroll
    for (int u = 0; u < 21; ++u) k += ckr[u] * sh[lt][u];
    m *= svol[lt];
    k *= svol[lt];
    cplx iv = smu[lt], ep = seps[lt];
    out[t * per + ab] = {iv.re * k - k0sq * ep.re * m, iv.im * k - k0sq * ep.im * m};
  }
}

// ------------------------------------------------------------------ face matrices
// S_f[a][b] = int_f (w_a x n).(w_b x n) = |f| sum_u cs[lf][a][b][u] GT_u with the tangential Gram
// matrix GT_pq = G_pq - G_po G_qo / G_oo (n = grad l_o / |grad l_o|) and |f| = 3 |T| |grad l_o|.
__global__ void k_faces(int64_t nif, int nfl, const double* __restrict__ xyz,
                        const int32_t* __restrict__ st, const int32_t* __restrict__ tet0,
                        const int32_t* __restrict__ lf0, const double* __restrict__ cs,
                        double* __restrict__ out) {
  int64_t f = blockIdx.x;
  if (f >= nif) return;
  __shared__ double gt[10];
  __shared__ double sarea;
  __shared__ int slf;
  if (threadIdx.x == 0) {
    int64_t t = tet0[f];
    int lf = lf0[f];
    const int OPP[4] = {3, 2, 1, 0};
    int o = OPP[lf];
    int32_t v[4];
    for (int q = 0; q < 4; ++q) v[q] = st[t * 4 + q];
    double gl[4][3], vol;
    tet_geometry(xyz, v, gl, vol);
    double G[4][4];
    for (int p = 0; p < 4; ++p)
      for (int q = 0; q < 4; ++q) G[p][q] = gl[p][0] * gl[q][0] + gl[p][1] * gl[q][1] + gl[p][2] * gl[q][2];
    for (int p = 0; p < 4; ++p)
      for (int q = p; q < 4; ++q) gt[sym10(p, q)] = G[p][q] - G[p][o] * G[q][o] / G[o][o];
    sarea = 3.0 * vol * sqrt(G[o][o]);
    slf = lf;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nfl * nfl; e += blockDim.x) {
    const double* c = cs + ((int64_t)slf * nfl * nfl + e) * 10;
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < 10; ++u) s += c[u] * gt[u];
    out[f * nfl * nfl + e] = sarea * s;
  }
}

// ------------------------------------------------------------------ row assembly
// One warp per matrix row.  Contributions are summed in a fixed order (tets ascending, then
// impedance faces ascending) into FP64 accumulators indexed by the row's CSR pattern, so the
// result is deterministic.  GLOBAL: the row of A (outer faces only).  LOCAL: the row of A_s for
// subdomain s -- only tets of Omega_s^delta, outer faces of those tets, and faces with exactly
// one tet in Omega_s^delta (impedance transmission, omega~ of the inside tet) -- written to the
// dense tiled arena (column-major TB x TB tiles).
struct RowArgs {
  int nl, nfl;
  double k0;
  const int32_t* dofmap;
  const int64_t* tinc_ptr; const int32_t* tinc;
  const int64_t* finc_ptr; const int32_t* finc;
  const int32_t* if_tet0; const int32_t* if_tet1; const int32_t* if_dofs;
  const int64_t* rowptr; const int32_t* cols;
  const cplx* elem; const double* fmat;
  const cplx* eps; const cplx* mu;
  const double* if_beta;     // [nif] caller's beta of outer faces, or nullptr (derived)
  const uint8_t* fixed;      // [ndof] constrained by a metallic face (identity row and column), or nullptr
  const uint32_t* member; int64_t member_words;
  int dirichlet;             // local rows: 1 = rows of the global matrix (RAS), 0 = ORAS local problem
};

__device__ __forceinline__ int bsearch32(const int32_t* a, int n, int32_t key) {
  int lo = 0, hi = n - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int32_t v = a[mid];
    if (v == key) return mid;
    if (v < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

__device__ __forceinline__ double omega_t(const RowArgs& A, int64_t t) {
  double mr = A.mu ? A.mu[t].re : 1.0;
  return A.k0 * sqrt(mr * A.eps[t].re);
}

__device__ __forceinline__ bool is_member(const RowArgs& A, int s, int64_t t) {
  return (A.member[(int64_t)s * A.member_words + (t >> 5)] >> (t & 31)) & 1u;
}

template <bool LOCAL>
__device__ void accumulate_row(const RowArgs& A, int64_t g, int s, cplx* acc, int rn,
                               const int32_t* rc) {
  const int lane = threadIdx.x & 31;
  for (int p = lane; p < rn; p += 32) acc[p] = {0.0, 0.0};
  __syncwarp();
  for (int64_t q = A.tinc_ptr[g]; q < A.tinc_ptr[g + 1]; ++q) {
    int32_t e = A.tinc[q];
    int64_t t = e / A.nl;
    int a = e - (int)t * A.nl;
    if (LOCAL && !is_member(A, s, t)) continue;
    const cplx* er = A.elem + (t * A.nl + a) * A.nl;
    for (int b = lane; b < A.nl; b += 32) {
      int p = bsearch32(rc, rn, A.dofmap[t * A.nl + b]);
      if (p >= 0) acc[p] = cadd(acc[p], er[b]);
    }
    __syncwarp();
  }
  for (int64_t q = A.finc_ptr[g]; q < A.finc_ptr[g + 1]; ++q) {
    int32_t e = A.finc[q];
    int64_t slot = e / A.nfl;
    int af = e - (int)slot * A.nfl;
    int64_t t0 = A.if_tet0[slot], t1 = A.if_tet1[slot];
    int64_t tin;
    if (t1 < 0) {
      if (LOCAL && !is_member(A, s, t0)) continue;
      tin = t0;
    } else {
      if (!LOCAL) continue;
      bool m0 = is_member(A, s, t0), m1 = is_member(A, s, t1);
      if (m0 == m1) continue;
      tin = m0 ? t0 : t1;
    }
    // outer faces: the caller's beta when given; interfaces: omega~ of the inside tet
    double w = (t1 < 0 && A.if_beta) ? A.if_beta[slot] : omega_t(A, tin);
    const double* fr = A.fmat + (slot * A.nfl + af) * A.nfl;
    for (int bf = lane; bf < A.nfl; bf += 32) {
      int p = bsearch32(rc, rn, A.if_dofs[slot * A.nfl + bf]);
      if (p >= 0) acc[p].im += w * fr[bf];
    }
    __syncwarp();
  }
}

constexpr int ROW_WARPS = 8;

__global__ void k_global_rows(RowArgs A, int64_t ndof, int maxnnz, cplx* __restrict__ vals) {
  extern __shared__ cplx sacc[];
  const int w = threadIdx.x >> 5;
  int64_t g = (int64_t)blockIdx.x * ROW_WARPS + w;
  if (g >= ndof) return;
  cplx* acc = sacc + w * maxnnz;
  int64_t r0 = A.rowptr[g];
  int rn = (int)(A.rowptr[g + 1] - r0);
  accumulate_row<false>(A, g, 0, acc, rn, A.cols + r0);
  if (A.fixed) {  // metallic faces: identity rows and columns of the constrained unknowns
    const bool gf = A.fixed[g] != 0;
    for (int p = threadIdx.x & 31; p < rn; p += 32) {
      const int32_t c = A.cols[r0 + p];
      vals[r0 + p] = (gf || A.fixed[c]) ? cplx{c == g ? 1.0 : 0.0, 0.0} : acc[p];
    }
    return;
  }
  for (int p = threadIdx.x & 31; p < rn; p += 32) vals[r0 + p] = acc[p];
}

template <typename R>
__global__ void k_local_rows(RowArgs A, int nsub, int64_t total_rows, const int64_t* __restrict__ np_off,
                             const int64_t* __restrict__ sub_ns, const int64_t* __restrict__ sub_np,
                             const int64_t* __restrict__ ns_off, const int64_t* __restrict__ tile_off,
                             const int32_t* __restrict__ sub_dofs, int maxnnz, void* __restrict__ arena) {
  extern __shared__ cplx sacc[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t row = (int64_t)blockIdx.x * ROW_WARPS + w;
  if (row >= total_rows) return;
  int lo = 0, hi = nsub - 1;
  while (lo < hi) {  // last s with np_off[s] <= row
    int mid = (lo + hi + 1) >> 1;
    if (np_off[mid] <= row) lo = mid; else hi = mid - 1;
  }
  const int s = lo;
  const int64_t li = row - np_off[s];
  const int64_t ns = sub_ns[s], np = sub_np[s], nts = np / TB;
  R* base = (R*)arena + tile_off[s] * 2 * TILE_PLANE;
  auto put = [&](int64_t i, int64_t j, R re, R im) {
    const int64_t I = i / TB, J = j / TB;
    R* t = base + (I * nts + J) * 2 * TILE_PLANE;
    const int64_t e = tile_elem(tile_rowmajor(I, J), i % TB, j % TB);
    t[e] = re;
    t[TILE_PLANE + e] = im;
  };
  if (li >= ns) {  // padding row: identity
    if (lane == 0) put(li, li, R(1), R(0));
    return;
  }
  const int32_t* Ns = sub_dofs + ns_off[s];
  const int64_t g = Ns[li];
  if (A.fixed && A.fixed[g]) {  // constrained by a metallic face: identity row (the arena is cleared)
    if (lane == 0) put(li, li, R(1), R(0));
    return;
  }
  cplx* acc = sacc + w * maxnnz;
  int64_t r0 = A.rowptr[g];
  int rn = (int)(A.rowptr[g + 1] - r0);
  const int32_t* rc = A.cols + r0;
  if (A.dirichlet) accumulate_row<false>(A, g, s, acc, rn, rc);  // R_s A R_s^T: the global row
  else accumulate_row<true>(A, g, s, acc, rn, rc);
  for (int p = lane; p < rn; p += 32) {
    if (A.fixed && A.fixed[rc[p]]) continue;  // constrained column: zero
    int lj = bsearch32(Ns, (int)ns, rc[p]);
    if (lj >= 0) put(li, lj, R(acc[p].re), R(acc[p].im));
  }
}

// ------------------------------------------------------------------ right-hand sides
__device__ __forceinline__ void basis_value(int a, const double* lam, const double gl[4][3],
                                            const double* tc, const int32_t* ta, const int32_t* tm,
                                            double out[3]) {
  out[0] = out[1] = out[2] = 0.0;
  for (int q = 0; q < 2; ++q) {
    double mono = tc[a * 2 + q];
    for (int v = 0; v < 4; ++v)
      for (int e = 0; e < ta[(a * 2 + q) * 4 + v]; ++e) mono *= lam[v];
    int m = tm[a * 2 + q];
    out[0] += mono * gl[m][0];
    out[1] += mono * gl[m][1];
    out[2] += mono * gl[m][2];
  }
}

__global__ void k_locate(int64_t nt, const double* __restrict__ xyz, const int32_t* __restrict__ st,
                         double x0, double x1, double x2, int* __restrict__ found) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  int32_t v[4];
  for (int q = 0; q < 4; ++q) v[q] = st[t * 4 + q];
  double gl[4][3], vol;
  tet_geometry(xyz, v, gl, vol);
  double d[3] = {x0 - xyz[(int64_t)v[0] * 3], x1 - xyz[(int64_t)v[0] * 3 + 1], x2 - xyz[(int64_t)v[0] * 3 + 2]};
  double l1 = gl[1][0] * d[0] + gl[1][1] * d[1] + gl[1][2] * d[2];
  double l2 = gl[2][0] * d[0] + gl[2][1] * d[1] + gl[2][2] * d[2];
  double l3 = gl[3][0] * d[0] + gl[3][1] * d[1] + gl[3][2] * d[2];
  double l0 = 1.0 - l1 - l2 - l3;
  const double tol = -1e-12;
  if (l0 >= tol && l1 >= tol && l2 >= tol && l3 >= tol) atomicMin(found, (int)t);
}

__global__ void k_dipole(int nl, const double* __restrict__ xyz, const int32_t* __restrict__ st,
                         const int32_t* __restrict__ dofmap, const int* __restrict__ found,
                         double x0, double x1, double x2, double d0, double d1, double d2,
                         const double* tc, const int32_t* ta, const int32_t* tm, cplx* __restrict__ b) {
  int t = *found;
  if (t == 0x7fffffff) return;
  int a = threadIdx.x;
  if (a >= nl) return;
  int32_t v[4];
  for (int q = 0; q < 4; ++q) v[q] = st[(int64_t)t * 4 + q];
  double gl[4][3], vol;
  tet_geometry(xyz, v, gl, vol);
  double d[3] = {x0 - xyz[(int64_t)v[0] * 3], x1 - xyz[(int64_t)v[0] * 3 + 1], x2 - xyz[(int64_t)v[0] * 3 + 2]};
  double lam[4];
  for (int q = 1; q < 4; ++q) lam[q] = gl[q][0] * d[0] + gl[q][1] * d[1] + gl[q][2] * d[2];
  lam[0] = 1.0 - lam[1] - lam[2] - lam[3];
  double w[3];
  basis_value(a, lam, gl, tc, ta, tm, w);
  b[dofmap[(int64_t)t * nl + a]] = {w[0] * d0 + w[1] * d1 + w[2] * d2, 0.0};
}

struct PlaneArgs {
  double d[3];
  cplx p[3];
  double k0;
  int nq;
  double qs[16], qw[16];  // Gauss-Legendre on [0,1]
};

// per outer face: b_face[slot][af] = int_f g . w_af, collapsed Gauss-Legendre product rule
__global__ void k_plane_faces(int64_t nif, int nfl, const double* __restrict__ xyz,
                              const int32_t* __restrict__ st, const int32_t* __restrict__ tet0,
                              const int32_t* __restrict__ lf0, const int32_t* __restrict__ tet1,
                              const int32_t* __restrict__ fl, const cplx* __restrict__ eps,
                              const cplx* __restrict__ mu, const double* __restrict__ if_beta,
                              const double* tc, const int32_t* ta, const int32_t* tm, PlaneArgs P,
                              cplx* __restrict__ bface) {
  int64_t f = blockIdx.x;
  int af = threadIdx.x;
  if (f >= nif || af >= nfl) return;
  if (tet1[f] >= 0) { bface[f * nfl + af] = {0.0, 0.0}; return; }
  const int FACES[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
  const int OPP[4] = {3, 2, 1, 0};
  int64_t t = tet0[f];
  int lf = lf0[f], o = OPP[lf];
  int32_t v[4];
  for (int q = 0; q < 4; ++q) v[q] = st[t * 4 + q];
  double gl[4][3], vol;
  tet_geometry(xyz, v, gl, vol);
  double go = sqrt(gl[o][0] * gl[o][0] + gl[o][1] * gl[o][1] + gl[o][2] * gl[o][2]);
  double n[3] = {-gl[o][0] / go, -gl[o][1] / go, -gl[o][2] / go};
  double area = 3.0 * vol * go;
  cplx e = eps[t];
  cplx m = mu ? mu[t] : cplx{1.0, 0.0};
  // gamma = k0 sqrt(mu eps), principal root
  cplx me = cmul(m, e);
  double mod = sqrt(me.re * me.re + me.im * me.im);
  double sr = sqrt(0.5 * (mod + me.re));
  double si = copysign(sqrt(fmax(0.0, 0.5 * (mod - me.re))), me.im);
  cplx gam = {P.k0 * sr, P.k0 * si};
  double beta = if_beta ? if_beta[f] : P.k0 * sqrt(m.re * e.re);
  double mden = m.re * m.re + m.im * m.im;
  cplx imu = {m.re / mden, -m.im / mden};
  // d x p
  cplx dxp[3] = {
      {P.d[1] * P.p[2].re - P.d[2] * P.p[1].re, P.d[1] * P.p[2].im - P.d[2] * P.p[1].im},
      {P.d[2] * P.p[0].re - P.d[0] * P.p[2].re, P.d[2] * P.p[0].im - P.d[0] * P.p[2].im},
      {P.d[0] * P.p[1].re - P.d[1] * P.p[0].re, P.d[0] * P.p[1].im - P.d[1] * P.p[0].im}};
  const int a = fl[lf * nfl + af];
  cplx acc = {0.0, 0.0};
  for (int i = 0; i < P.nq; ++i)
    for (int j = 0; j < P.nq; ++j) {
      double u = P.qs[i], vv = P.qs[j] * (1.0 - P.qs[i]);
      double wq = P.qw[i] * P.qw[j] * (1.0 - P.qs[i]);
      double lam[4] = {0, 0, 0, 0};
      lam[FACES[lf][0]] = 1.0 - u - vv;
      lam[FACES[lf][1]] = u;
      lam[FACES[lf][2]] = vv;
      double x[3];
      for (int dd = 0; dd < 3; ++dd)
        x[dd] = lam[0] * xyz[(int64_t)v[0] * 3 + dd] + lam[1] * xyz[(int64_t)v[1] * 3 + dd] +
                lam[2] * xyz[(int64_t)v[2] * 3 + dd] + lam[3] * xyz[(int64_t)v[3] * 3 + dd];
      double dx = P.d[0] * x[0] + P.d[1] * x[1] + P.d[2] * x[2];
      // phase = exp(-i gamma d.x)
      cplx arg = {gam.im * dx, -gam.re * dx};
      double ex = exp(arg.re);
      cplx ph = {ex * cos(arg.im), ex * sin(arg.im)};
      cplx E[3], C[3], gv[3];
      cplx mig = {gam.im, -gam.re};  // -i gamma
      for (int dd = 0; dd < 3; ++dd) {
        E[dd] = cmul(ph, P.p[dd]);
        C[dd] = cmul(cmul(mig, ph), dxp[dd]);
      }
      // g = mu^{-1} (C x n) + i beta (E - (E.n) n)
      cplx En = {E[0].re * n[0] + E[1].re * n[1] + E[2].re * n[2], E[0].im * n[0] + E[1].im * n[1] + E[2].im * n[2]};
      cplx Cxn[3] = {{C[1].re * n[2] - C[2].re * n[1], C[1].im * n[2] - C[2].im * n[1]},
                     {C[2].re * n[0] - C[0].re * n[2], C[2].im * n[0] - C[0].im * n[2]},
                     {C[0].re * n[1] - C[1].re * n[0], C[0].im * n[1] - C[1].im * n[0]}};
      for (int dd = 0; dd < 3; ++dd) {
        cplx et = {E[dd].re - En.re * n[dd], E[dd].im - En.im * n[dd]};
        cplx ib = {-beta * et.im, beta * et.re};
        gv[dd] = cadd(cmul(imu, Cxn[dd]), ib);
      }
      double wv[3];
      basis_value(a, lam, gl, tc, ta, tm, wv);
      acc.re += wq * (gv[0].re * wv[0] + gv[1].re * wv[1] + gv[2].re * wv[2]);
      acc.im += wq * (gv[0].im * wv[0] + gv[1].im * wv[1] + gv[2].im * wv[2]);
    }
  bface[f * nfl + af] = {2.0 * area * acc.re, 2.0 * area * acc.im};
}

// b[g] = sum over outer-face entries of g (ascending slots)
__global__ void k_gather_faces(int64_t ndof, int nfl, const int64_t* __restrict__ finc_ptr,
                               const int32_t* __restrict__ finc, const cplx* __restrict__ bface,
                               cplx* __restrict__ b) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ndof) return;
  cplx s = {0.0, 0.0};
  for (int64_t q = finc_ptr[g]; q < finc_ptr[g + 1]; ++q) s = cadd(s, bface[finc[q]]);
  b[g] = s;
}

// v[g][r] = 0 for the constrained degrees of freedom ([N][k] layout)
__global__ void k_mask_fixed(int64_t ndof, int k, const uint8_t* __restrict__ fixed, cplx* __restrict__ v) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ndof * k) return;
  if (fixed[e / k]) v[e] = {0.0, 0.0};
}

// ------------------------------------------------------------------ waveguide ports (Sec. 2, Sec. 5.1)
struct PortArgs {
  double o[3], u[3], vhat[3];
  double inv_uu;          // 1 / |u|^2
  double beta;
  int load;               // 0: p_a = int w_a . E0;  1: b_a = int i beta (1 + 1/mu) E0 . w_a
  int nq;
  double qs[16], qw[16];  // Gauss-Legendre on [0, 1]
};

// per impedance face f in the port (inport[f]): pface[f][af] = int_f c_f E0 . w_af and
// nface[f] = int_f |E0|^2, collapsed Gauss-Legendre product rule; zero for the other faces
__global__ void k_port_faces(int64_t nif, int nfl, const double* __restrict__ xyz, const int32_t* __restrict__ st,
                             const int32_t* __restrict__ tet0, const int32_t* __restrict__ lf0,
                             const uint8_t* __restrict__ inport, const int32_t* __restrict__ fl,
                             const cplx* __restrict__ mu, const double* tc, const int32_t* ta, const int32_t* tm,
                             PortArgs P, cplx* __restrict__ pface, double* __restrict__ nface) {
  const int64_t f = blockIdx.x;
  const int af = threadIdx.x;
  if (f >= nif || af >= nfl) return;
  if (!inport[f]) {
    pface[f * nfl + af] = {0.0, 0.0};
    if (af == 0) nface[f] = 0.0;
    return;
  }
  const int FACES[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
  const int OPP[4] = {3, 2, 1, 0};
  const int64_t t = tet0[f];
  const int lf = lf0[f], o = OPP[lf];
  int32_t v[4];
  for (int q = 0; q < 4; ++q) v[q] = st[t * 4 + q];
  double gl[4][3], vol;
  tet_geometry(xyz, v, gl, vol);
  const double go = sqrt(gl[o][0] * gl[o][0] + gl[o][1] * gl[o][1] + gl[o][2] * gl[o][2]);
  const double area = 3.0 * vol * go;
  const double pi = 3.14159265358979323846;
  const int a = fl[lf * nfl + af];
  double acc = 0.0, accn = 0.0;
  for (int i = 0; i < P.nq; ++i)
    for (int j = 0; j < P.nq; ++j) {
      const double uu = P.qs[i], vv = P.qs[j] * (1.0 - P.qs[i]);
      const double wq = P.qw[i] * P.qw[j] * (1.0 - P.qs[i]);
      double lam[4] = {0, 0, 0, 0};
      lam[FACES[lf][0]] = 1.0 - uu - vv;
      lam[FACES[lf][1]] = uu;
      lam[FACES[lf][2]] = vv;
      double x[3];
      for (int dd = 0; dd < 3; ++dd)
        x[dd] = lam[0] * xyz[(int64_t)v[0] * 3 + dd] + lam[1] * xyz[(int64_t)v[1] * 3 + dd] +
                lam[2] * xyz[(int64_t)v[2] * 3 + dd] + lam[3] * xyz[(int64_t)v[3] * 3 + dd];
      const double s = ((x[0] - P.o[0]) * P.u[0] + (x[1] - P.o[1]) * P.u[1] + (x[2] - P.o[2]) * P.u[2]) * P.inv_uu;
      const double amp = sin(pi * s);
      double wv[3];
      basis_value(a, lam, gl, tc, ta, tm, wv);
      acc += wq * amp * (P.vhat[0] * wv[0] + P.vhat[1] * wv[1] + P.vhat[2] * wv[2]);
      accn += wq * amp * amp;
    }
  cplx c = {1.0, 0.0};
  if (P.load) {  // i beta (1 + 1/mu)
    const cplx m = mu ? mu[t] : cplx{1.0, 0.0};
    const double den = m.re * m.re + m.im * m.im;
    const cplx f1 = {1.0 + m.re / den, -m.im / den};
    c = {-P.beta * f1.im, P.beta * f1.re};
  }
  pface[f * nfl + af] = {2.0 * area * acc * c.re, 2.0 * area * acc * c.im};
  if (af == 0) nface[f] = 2.0 * area * accn;
}

// out = sum of x[0..n) in a fixed order (one block of 256 threads: strided partial sums, then a tree)
__global__ void k_sum_fixed(int64_t n, const double* __restrict__ x, double* __restrict__ out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 256) s += x[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// S[j] = sum over the port's degrees of freedom d of conj(x[d][j]) p[d] / norm, one block per
// column j, fixed-order partial sums and tree
__global__ void k_port_dots(int64_t nd, const int32_t* __restrict__ dofs, const cplx* __restrict__ p,
                            const cplx* __restrict__ x, int k, const double* __restrict__ norm,
                            cplx* __restrict__ S) {
  __shared__ double sr[256], si[256];
  const int j = blockIdx.x;
  double ar = 0.0, ai = 0.0;
  for (int64_t q = threadIdx.x; q < nd; q += 256) {
    const int32_t d = dofs[q];
    const cplx xv = x[(int64_t)d * k + j], pv = p[d];
    ar += xv.re * pv.re + xv.im * pv.im;  // conj(x) p
    ai += xv.re * pv.im - xv.im * pv.re;
  }
  sr[threadIdx.x] = ar;
  si[threadIdx.x] = ai;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sr[threadIdx.x] += sr[threadIdx.x + w];
      si[threadIdx.x] += si[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) S[j] = {sr[0] / *norm, si[0] / *norm};
}

// ------------------------------------------------------------------ launchers
int launch_element(const oras_handle* h, double k0) {
  const auto& m = h->mesh;
  const auto& d = h->dev;
  int64_t blocks = (m.nt + EL_TETS - 1) / EL_TETS;
  k_element<<<(unsigned)blocks, 256, 0, d.stream>>>(m.nt, m.nl, d.xyz, d.st, d.eps, d.mu, k0 * k0,
                                                    d.cm, d.ck, d.elem);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_faces(const oras_handle* h) {
  const auto& m = h->mesh;
  const auto& d = h->dev;
  if (m.nif == 0) return 0;
  k_faces<<<(unsigned)m.nif, 256, 0, d.stream>>>(m.nif, m.nfl, d.xyz, d.st, d.if_tet0, d.if_lf0, d.cs,
                                                 d.fmat);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

static RowArgs row_args(const oras_handle* h, double k0) {
  const auto& m = h->mesh;
  const auto& d = h->dev;
  RowArgs A;
  A.nl = m.nl; A.nfl = m.nfl; A.k0 = k0;
  A.dofmap = d.dofmap; A.tinc_ptr = d.tinc_ptr; A.tinc = d.tinc;
  A.finc_ptr = d.finc_ptr; A.finc = d.finc;
  A.if_tet0 = d.if_tet0; A.if_tet1 = d.if_tet1; A.if_dofs = d.if_dofs;
  A.rowptr = d.rowptr; A.cols = d.cols;
  A.elem = d.elem; A.fmat = d.fmat; A.eps = d.eps; A.mu = d.mu;
  A.if_beta = d.if_beta;
  A.fixed = d.fixed;
  A.member = d.member; A.member_words = m.member_words;
  A.dirichlet = h->opt.transmission == ORAS_TRANSMISSION_DIRICHLET ? 1 : 0;
  return A;
}

int launch_global_rows(const oras_handle* h, double k0) {
  const auto& m = h->mesh;
  RowArgs A = row_args(h, k0);
  size_t smem = (size_t)ROW_WARPS * m.max_row_nnz * sizeof(cplx);
  if (smem > 48 * 1024)
    allow_max_smem((const void*)k_global_rows);
  int64_t blocks = (m.ndof + ROW_WARPS - 1) / ROW_WARPS;
  k_global_rows<<<(unsigned)blocks, ROW_WARPS * 32, smem, h->dev.stream>>>(A, m.ndof, m.max_row_nnz,
                                                                          h->dev.vals);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <typename R>
static int launch_local_rows_t(const oras_handle* h, double k0) {
  const auto& m = h->mesh;
  const auto& d = h->dev;
  RowArgs A = row_args(h, k0);
  int64_t total = 0;
  for (int s = 0; s < m.nsub; ++s) total += m.sub_np[s];
  size_t smem = (size_t)ROW_WARPS * m.max_row_nnz * sizeof(cplx);
  if (smem > 48 * 1024)
    allow_max_smem((const void*)k_local_rows<R>);
  int64_t blocks = (total + ROW_WARPS - 1) / ROW_WARPS;
  k_local_rows<R><<<(unsigned)blocks, ROW_WARPS * 32, smem, d.stream>>>(
      A, m.nsub, total, d.sub_np_off, d.sub_ns, d.sub_np, d.sub_ns_off, d.sub_tile_off, d.sub_dofs,
      m.max_row_nnz, d.arena);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_local_rows(const oras_handle* h, double k0) {
  return h->dev.factor_bits == 64 ? launch_local_rows_t<double>(h, k0) : launch_local_rows_t<float>(h, k0);
}

int launch_dipole(const oras_handle* h, const double* x0, const double* dir, cplx* b, int* found) {
  const auto& m = h->mesh;
  const auto& d = h->dev;
  int init = 0x7fffffff;
  cudaMemcpyAsync(found, &init, sizeof(int), cudaMemcpyHostToDevice, d.stream);
  cudaMemsetAsync(b, 0, sizeof(cplx) * m.ndof, d.stream);
  k_locate<<<(unsigned)((m.nt + 255) / 256), 256, 0, d.stream>>>(m.nt, d.xyz, d.st, x0[0], x0[1], x0[2], found);
  count_launches(1);
  k_dipole<<<1, 64, 0, d.stream>>>(m.nl, d.xyz, d.st, d.dofmap, found, x0[0], x0[1], x0[2], dir[0],
                                   dir[1], dir[2], d.tc, d.ta, d.tm, b);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_plane(const oras_handle* h, const double* dvec, const oras_complex* pvec, double k0,
                 const double* qs, const double* qw, int nq, cplx* bface, cplx* b) {
  const auto& m = h->mesh;
  const auto& d = h->dev;
  PlaneArgs P;
  for (int i = 0; i < 3; ++i) {
    P.d[i] = dvec[i];
    P.p[i] = {pvec[i].re, pvec[i].im};
  }
  P.k0 = k0;
  P.nq = nq;
  for (int i = 0; i < nq; ++i) { P.qs[i] = qs[i]; P.qw[i] = qw[i]; }
  if (m.nif > 0)
    k_plane_faces<<<(unsigned)m.nif, 32, 0, d.stream>>>(m.nif, m.nfl, d.xyz, d.st, d.if_tet0, d.if_lf0,
                                                        d.if_tet1, d.fl, d.eps, d.mu, d.if_beta, d.tc, d.ta,
                                                        d.tm, P, bface);
  count_launches(1);
  k_gather_faces<<<(unsigned)((m.ndof + 255) / 256), 256, 0, d.stream>>>(m.ndof, m.nfl, d.finc_ptr, d.finc,
                                                                        bface, b);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

void launch_mask_fixed(const oras_handle* h, cplx* v, int k) {
  const auto& m = h->mesh;
  if (!h->dev.fixed) return;
  const int64_t n = m.ndof * k;
  k_mask_fixed<<<(unsigned)((n + 255) / 256), 256, 0, h->dev.stream>>>(m.ndof, k, h->dev.fixed, v);
  count_launches(1);
}

// p (or the load b) of one port into out [N], its norm into *norm_d (device); inport: [nif]
// device flags of the port's faces; pface/nface: device scratch [nif * nfl] / [nif]
int launch_port(const oras_handle* h, const double* o, const double* u, const double* v, double beta, int load,
                const double* qs, const double* qw, int nq, const uint8_t* inport, cplx* pface, double* nface,
                cplx* out, double* norm_d) {
  const auto& m = h->mesh;
  const auto& d = h->dev;
  PortArgs P;
  double uu = 0.0, vv = 0.0;
  for (int i = 0; i < 3; ++i) {
    P.o[i] = o[i];
    P.u[i] = u[i];
    uu += u[i] * u[i];
    vv += v[i] * v[i];
  }
  for (int i = 0; i < 3; ++i) P.vhat[i] = v[i] / std::sqrt(vv);
  P.inv_uu = 1.0 / uu;
  P.beta = beta;
  P.load = load;
  P.nq = nq;
  for (int i = 0; i < nq; ++i) { P.qs[i] = qs[i]; P.qw[i] = qw[i]; }
  k_port_faces<<<(unsigned)m.nif, 32, 0, d.stream>>>(m.nif, m.nfl, d.xyz, d.st, d.if_tet0, d.if_lf0, inport, d.fl,
                                                     d.mu, d.tc, d.ta, d.tm, P, pface, nface);
  k_gather_faces<<<(unsigned)((m.ndof + 255) / 256), 256, 0, d.stream>>>(m.ndof, m.nfl, d.finc_ptr, d.finc,
                                                                        pface, out);
  k_sum_fixed<<<1, 256, 0, d.stream>>>(m.nif, nface, norm_d);
  count_launches(3);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_port_dots(const oras_handle* h, int64_t nd, const int32_t* dofs, const cplx* p, const cplx* x, int k,
                     const double* norm_d, cplx* S) {
  k_port_dots<<<(unsigned)k, 256, 0, h->dev.stream>>>(nd, dofs, p, x, k, norm_d, S);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace oras
