// Local DOF convention and exact-integration tables for the element kernels.
//
// Sec. 3 defines the generators  w^{k,e} = lambda^k w^e,  w^e = lambda_i grad l_j - lambda_j grad l_i,
// |k| = r - 1.  The independent subset used here (the paper defers the choice):
//   edge (a,b):   every k supported on {a,b}                                   (r per edge)
//   face (a,b,c): Whitney edges (a,b) and (a,c), k on the face with k_opp >= 1  (r(r-1) per face)
//   volume:       Whitney edges (0,1),(0,2),(0,3) with k = the two other vertices (r = 3)
// Exponent tuples are listed in ascending lexicographic order over the entity's vertices.
//
// Each generator is two terms c * lambda^alpha * grad(lambda_m); curl(f grad g) = grad f x grad g
// turns its curl into terms c' * lambda^beta * (grad l_p x grad l_m).  Products are integrated
// exactly:  int_T lambda^alpha = 6|T| alpha!/(|alpha|+3)!,  int_f lambda^alpha = 2|f| alpha!/(|alpha|+2)!.
// The tables below hold the rational coefficients that multiply the per-element geometric
// factors (Gram matrix G of the barycentric gradients, and the Gram matrix of their cross products).
#include <algorithm>
#include <array>
#include <stdexcept>

#include "internal.h"

namespace oras {

static const int EDGES[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
static const int FACES[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
static const int OPP[4] = {3, 2, 1, 0};

int n_local(int r) { return 6 * r + 4 * r * (r - 1) + r * (r - 1) * (r - 2) / 2; }
int n_face_local(int r) { return 3 * r + r * (r - 1); }

// exponent tuples of total weight w on the vertices `sup` (ascending), ascending lexicographic
static void tuples(const std::vector<int>& sup, int w, size_t pos, std::vector<int>& cur,
                   std::vector<std::vector<int>>& out) {
  if (pos + 1 == sup.size()) {
    cur[pos] = w;
    out.push_back(cur);
    return;
  }
  for (int e = 0; e <= w; ++e) {
    cur[pos] = e;
    tuples(sup, w - e, pos + 1, cur, out);
  }
}

static std::vector<std::array<int, 4>> exps(const std::vector<int>& sup, int w) {
  std::vector<std::vector<int>> t;
  std::vector<int> cur(sup.size());
  tuples(sup, w, 0, cur, t);
  std::vector<std::array<int, 4>> out;
  for (auto& v : t) {
    std::array<int, 4> k{0, 0, 0, 0};
    for (size_t q = 0; q < sup.size(); ++q) k[sup[q]] = v[q];
    out.push_back(k);
  }
  return out;
}

std::vector<LocalDof> local_dofs(int r) {
  if (r < 1 || r > 3) throw std::invalid_argument("r");
  std::vector<LocalDof> d;
  for (int e = 0; e < 6; ++e) {
    int a = EDGES[e][0], b = EDGES[e][1], q = 0;
    for (auto& k : exps({a, b}, r - 1)) d.push_back({'e', e, q++, a, b, {k[0], k[1], k[2], k[3]}});
  }
  if (r >= 2) {
    for (int f = 0; f < 4; ++f) {
      int a = FACES[f][0], b = FACES[f][1], c = FACES[f][2], q = 0;
      const int pairs[2][3] = {{a, b, c}, {a, c, b}};
      for (auto& pr : pairs) {
        for (auto& k : exps({a, b, c}, r - 1))
          if (k[pr[2]] >= 1) d.push_back({'f', f, q++, pr[0], pr[1], {k[0], k[1], k[2], k[3]}});
      }
    }
  }
  if (r == 3) {
    const int ed[3][2] = {{0, 1}, {0, 2}, {0, 3}};
    for (int q = 0; q < 3; ++q) {
      LocalDof x{'v', 0, q, ed[q][0], ed[q][1], {1, 1, 1, 1}};
      x.k[ed[q][0]] = 0;
      x.k[ed[q][1]] = 0;
      d.push_back(x);
    }
  }
  if ((int)d.size() != n_local(r)) throw std::logic_error("local dof count");
  return d;
}

std::vector<int> face_local_dofs(int r, int lf) {
  int a = FACES[lf][0], b = FACES[lf][1], c = FACES[lf][2];
  auto edge_index = [](int u, int v) {
    for (int e = 0; e < 6; ++e)
      if (EDGES[e][0] == u && EDGES[e][1] == v) return e;
    return -1;
  };
  std::vector<int> out;
  const int fe[3][2] = {{a, b}, {a, c}, {b, c}};
  for (auto& e : fe)
    for (int q = 0; q < r; ++q) out.push_back(edge_index(e[0], e[1]) * r + q);
  for (int q = 0; q < r * (r - 1); ++q) out.push_back(6 * r + lf * r * (r - 1) + q);
  return out;
}

static double fact(int n) {
  double f = 1;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

struct Term { double c; int al[4]; int m; };
struct CurlTerm { double c; int be[4]; int pair; };  // pair index of (p<m) cross product

static int pair_index(int p, int m) {
  for (int e = 0; e < 6; ++e)
    if (EDGES[e][0] == p && EDGES[e][1] == m) return e;
  return -1;
}
static int sym10(int p, int q) {  // unique (p <= q) index of a symmetric 4x4
  if (p > q) std::swap(p, q);
  static const int idx[4][4] = {{0, 1, 2, 3}, {1, 4, 5, 6}, {2, 5, 7, 8}, {3, 6, 8, 9}};
  return idx[p][q];
}
static int sym21(int u, int v) {  // unique (u <= v) index of a symmetric 6x6
  if (u > v) std::swap(u, v);
  return u * 6 - u * (u - 1) / 2 + (v - u);
}

static std::vector<Term> terms(const LocalDof& d) {
  Term t1{1.0, {d.k[0], d.k[1], d.k[2], d.k[3]}, d.j};
  t1.al[d.i] += 1;
  Term t2{-1.0, {d.k[0], d.k[1], d.k[2], d.k[3]}, d.i};
  t2.al[d.j] += 1;
  return {t1, t2};
}

static std::vector<CurlTerm> curl_terms(const LocalDof& d) {
  std::vector<CurlTerm> out;
  for (auto& t : terms(d)) {
    for (int p = 0; p < 4; ++p) {
      if (t.al[p] == 0 || p == t.m) continue;  // grad l_p x grad l_p = 0
      CurlTerm c{t.c * t.al[p], {t.al[0], t.al[1], t.al[2], t.al[3]}, 0};
      c.be[p] -= 1;
      int a = p, b = t.m;
      if (a > b) { std::swap(a, b); c.c = -c.c; }
      c.pair = pair_index(a, b);
      out.push_back(c);
    }
  }
  return out;
}

static double vol_int(const int* al) {  // int_T lambda^al / |T|
  int s = al[0] + al[1] + al[2] + al[3];
  return 6.0 * fact(al[0]) * fact(al[1]) * fact(al[2]) * fact(al[3]) / fact(s + 3);
}

Tables make_tables(int r) {
  Tables T;
  T.r = r;
  auto d = local_dofs(r);
  int nl = (int)d.size(), nfl = n_face_local(r);
  T.nl = nl;
  T.nfl = nfl;
  T.cm.assign((size_t)nl * nl * 10, 0.0);
  T.ck.assign((size_t)nl * nl * 21, 0.0);
  std::vector<std::vector<Term>> tt(nl);
  std::vector<std::vector<CurlTerm>> ct(nl);
  for (int a = 0; a < nl; ++a) {
    tt[a] = terms(d[a]);
    ct[a] = curl_terms(d[a]);
  }
  for (int a = 0; a < nl; ++a)
    for (int b = 0; b < nl; ++b) {
      for (auto& x : tt[a])
        for (auto& y : tt[b]) {
          int al[4];
          for (int v = 0; v < 4; ++v) al[v] = x.al[v] + y.al[v];
          T.cm[((size_t)a * nl + b) * 10 + sym10(x.m, y.m)] += x.c * y.c * vol_int(al);
        }
      for (auto& x : ct[a])
        for (auto& y : ct[b]) {
          int be[4];
          for (int v = 0; v < 4; ++v) be[v] = x.be[v] + y.be[v];
          T.ck[((size_t)a * nl + b) * 21 + sym21(x.pair, y.pair)] += x.c * y.c * vol_int(be);
        }
    }
  T.cs.assign((size_t)4 * nfl * nfl * 10, 0.0);
  T.fl.assign((size_t)4 * nfl, 0);
  for (int lf = 0; lf < 4; ++lf) {
    auto fld = face_local_dofs(r, lf);
    int o = OPP[lf];
    for (int af = 0; af < nfl; ++af) T.fl[lf * nfl + af] = fld[af];
    for (int af = 0; af < nfl; ++af)
      for (int bf = 0; bf < nfl; ++bf) {
        for (auto& x : tt[fld[af]])
          for (auto& y : tt[fld[bf]]) {
            int al[4];
            for (int v = 0; v < 4; ++v) al[v] = x.al[v] + y.al[v];
            if (al[o] != 0) continue;  // lambda_o vanishes on the face
            int s = 0;
            double num = 1;
            for (int v = 0; v < 4; ++v)
              if (v != o) { s += al[v]; num *= fact(al[v]); }
            double fi = 2.0 * num / fact(s + 2);  // int_f lambda^al / |f|
            T.cs[(((size_t)lf * nfl + af) * nfl + bf) * 10 + sym10(x.m, y.m)] += x.c * y.c * fi;
          }
      }
  }
  T.tc.assign((size_t)nl * 2, 0.0);
  T.ta.assign((size_t)nl * 8, 0);
  T.tm.assign((size_t)nl * 2, 0);
  for (int a = 0; a < nl; ++a)
    for (int q = 0; q < 2; ++q) {
      T.tc[a * 2 + q] = tt[a][q].c;
      T.tm[a * 2 + q] = tt[a][q].m;
      for (int v = 0; v < 4; ++v) T.ta[(a * 2 + q) * 4 + v] = tt[a][q].al[v];
    }
  return T;
}

}  // namespace oras
