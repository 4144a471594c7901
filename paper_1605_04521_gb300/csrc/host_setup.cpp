// Host integer set-up: topology, DOF numbering (Sec. 3), partition, overlap, restriction sets
// N_s and partition of unity D_s (Sec. 4), impedance-face lists and the CSR pattern of A.
//
// Readings where the paper is silent (it names R_s, D_s, Omega_s but not their construction):
//  * partition: recursive coordinate bisection of tetrahedron centroids
//    c = (((v0 + v1) + v2) + v3) * 0.25 over the sorted vertices; axis = largest centroid extent
//    (ties -> x, y, z); order by (coordinate, tet id); child 0 takes floor(m * p0 / p) tets with
//    p0 = floor(p / 2) parts; ids depth-first, child 0 first;
//  * overlap: `overlap` layers, each adds every tetrahedron sharing a vertex (or, with
//    ORAS_OVERLAP_FACE, a face) with the current set;
//  * N_s: every DOF on an entity of a tetrahedron of Omega_s^delta, ascending;
//  * D_s: a DOF belongs to the subdomain of the lowest-index tetrahedron carrying it.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace oras {

static const int EDGES[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
static const int FACES[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};

static inline bool member_of(const HostMesh& m, int s, int64_t t) {
  return (m.member[(size_t)s * m.member_words + (t >> 5)] >> (t & 31)) & 1u;
}

static void rcb(const HostMesh& m, int nsub, std::vector<int32_t>& part) {
  const int64_t T = m.nt;
  std::vector<double> cen((size_t)T * 3);
  for (int64_t t = 0; t < T; ++t) {
    const int32_t* v = &m.st[t * 4];
    for (int d = 0; d < 3; ++d)
      cen[t * 3 + d] = (((m.xyz[v[0] * 3 + d] + m.xyz[v[1] * 3 + d]) + m.xyz[v[2] * 3 + d]) +
                        m.xyz[v[3] * 3 + d]) * 0.25;
  }
  part.assign(T, 0);
  struct Seg { std::vector<int32_t> ids; int base, p; };
  std::vector<Seg> stack;
  {
    Seg s;
    s.ids.resize(T);
    std::iota(s.ids.begin(), s.ids.end(), 0);
    s.base = 0;
    s.p = nsub;
    stack.push_back(std::move(s));
  }
  while (!stack.empty()) {
    Seg s = std::move(stack.back());
    stack.pop_back();
    if (s.p == 1) {
      for (auto id : s.ids) part[id] = s.base;
      continue;
    }
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) { lo[d] = INFINITY; hi[d] = -INFINITY; }
    for (auto id : s.ids)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], cen[(size_t)id * 3 + d]);
        hi[d] = std::max(hi[d], cen[(size_t)id * 3 + d]);
      }
    int axis = 0;
    double best = hi[0] - lo[0];
    for (int d = 1; d < 3; ++d)
      if (hi[d] - lo[d] > best) { best = hi[d] - lo[d]; axis = d; }
    std::sort(s.ids.begin(), s.ids.end(), [&](int32_t a, int32_t b) {
      double ca = cen[(size_t)a * 3 + axis], cb = cen[(size_t)b * 3 + axis];
      if (ca < cb) return true;
      if (cb < ca) return false;
      return a < b;
    });
    int p0 = s.p / 2;
    int64_t h = ((int64_t)s.ids.size() * p0) / s.p;
    Seg c0, c1;
    c0.ids.assign(s.ids.begin(), s.ids.begin() + h);
    c1.ids.assign(s.ids.begin() + h, s.ids.end());
    c0.base = s.base;
    c0.p = p0;
    c1.base = s.base + p0;
    c1.p = s.p - p0;
    stack.push_back(std::move(c1));
    stack.push_back(std::move(c0));
  }
}

int host_setup(const oras_problem* p, int overlap_kind, HostMesh& m, std::string& err) {
  if (!p || !p->xyz || !p->tets || p->nv <= 0 || p->nt <= 0) {
    err = "oras_create: NULL or empty mesh";
    return ORAS_ERR_INVALID_ARG;
  }
  if (p->r < 1 || p->r > 3) { err = "oras_create: degree r must be 1, 2 or 3"; return ORAS_ERR_INVALID_ARG; }
  if (p->nsub < 1 || p->nsub > p->nt) { err = "oras_create: nsub must be in [1, nt]"; return ORAS_ERR_INVALID_ARG; }
  if (p->overlap < 0) { err = "oras_create: overlap must be >= 0"; return ORAS_ERR_INVALID_ARG; }
  if (p->nv >= (int64_t(1) << 21)) { err = "oras_create: more than 2^21 vertices"; return ORAS_ERR_UNSUPPORTED; }
  if (p->nt >= (int64_t(1) << 31) / 64) { err = "oras_create: too many tetrahedra"; return ORAS_ERR_UNSUPPORTED; }
  m.r = p->r;
  m.nl = n_local(p->r);
  m.nfl = n_face_local(p->r);
  m.nv = p->nv;
  m.nt = p->nt;
  m.nsub = p->nsub;
  m.overlap = p->overlap;
  m.overlap_kind = overlap_kind;
  const int64_t nv = m.nv, T = m.nt;
  const int r = m.r, nl = m.nl, nfl = m.nfl;
  m.xyz.assign(p->xyz, p->xyz + nv * 3);
  m.st.resize(T * 4);
  for (int64_t t = 0; t < T; ++t) {
    int32_t v[4];
    for (int q = 0; q < 4; ++q) {
      v[q] = p->tets[t * 4 + q];
      if (v[q] < 0 || v[q] >= nv) { err = "oras_create: vertex id out of range in tet " + std::to_string(t); return ORAS_ERR_BAD_MESH; }
    }
    std::sort(v, v + 4);
    for (int q = 0; q < 3; ++q)
      if (v[q] == v[q + 1]) { err = "oras_create: repeated vertex in tet " + std::to_string(t); return ORAS_ERR_BAD_MESH; }
    double J[3][3];
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) J[d][c] = m.xyz[v[c + 1] * 3 + d] - m.xyz[v[0] * 3 + d];
    double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                 J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                 J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    if (!(std::fabs(det) > 0.0)) { err = "oras_create: zero-volume tet " + std::to_string(t); return ORAS_ERR_BAD_MESH; }
    for (int q = 0; q < 4; ++q) m.st[t * 4 + q] = v[q];
  }
  // ---------------- edges and faces (sorted keys)
  std::vector<uint64_t> ek(T * 6);
  for (int64_t t = 0; t < T; ++t)
    for (int e = 0; e < 6; ++e)
      ek[t * 6 + e] = (uint64_t)m.st[t * 4 + EDGES[e][0]] * nv + m.st[t * 4 + EDGES[e][1]];
  std::vector<uint64_t> ue(ek);
  std::sort(ue.begin(), ue.end());
  ue.erase(std::unique(ue.begin(), ue.end()), ue.end());
  m.ne = (int64_t)ue.size();
  std::vector<int32_t> tet_edges(T * 6);
  for (int64_t i = 0; i < T * 6; ++i)
    tet_edges[i] = (int32_t)(std::lower_bound(ue.begin(), ue.end(), ek[i]) - ue.begin());
  std::vector<uint64_t> fk(T * 4);
  for (int64_t t = 0; t < T; ++t)
    for (int f = 0; f < 4; ++f)
      fk[t * 4 + f] = ((uint64_t)m.st[t * 4 + FACES[f][0]] * nv + m.st[t * 4 + FACES[f][1]]) * nv +
                      m.st[t * 4 + FACES[f][2]];
  std::vector<uint64_t> uf(fk);
  std::sort(uf.begin(), uf.end());
  uf.erase(std::unique(uf.begin(), uf.end()), uf.end());
  m.nf = (int64_t)uf.size();
  m.tet_faces.resize(T * 4);
  m.face_tets.assign(m.nf * 2, -1);
  for (int64_t t = 0; t < T; ++t)
    for (int f = 0; f < 4; ++f) {
      int32_t id = (int32_t)(std::lower_bound(uf.begin(), uf.end(), fk[t * 4 + f]) - uf.begin());
      m.tet_faces[t * 4 + f] = id;
      if (m.face_tets[id * 2] < 0) m.face_tets[id * 2] = (int32_t)t;
      else if (m.face_tets[id * 2 + 1] < 0) m.face_tets[id * 2 + 1] = (int32_t)t;
      else { err = "oras_create: a face is shared by more than two tets"; return ORAS_ERR_BAD_MESH; }
    }
  // ---------------- DOF numbering
  const int ned = r, nfd = r * (r - 1), nvd = r * (r - 1) * (r - 2) / 2;
  int64_t ndof = m.ne * ned + m.nf * nfd + T * nvd;
  if (ndof >= (int64_t(1) << 31) - 1) { err = "oras_create: more than 2^31-1 DOFs"; return ORAS_ERR_UNSUPPORTED; }
  m.ndof = ndof;
  auto dofs = local_dofs(r);
  m.dofmap.resize(T * nl);
  for (int64_t t = 0; t < T; ++t)
    for (int a = 0; a < nl; ++a) {
      const LocalDof& d = dofs[a];
      int64_t g;
      if (d.kind == 'e') g = (int64_t)tet_edges[t * 6 + d.ent] * ned + d.q;
      else if (d.kind == 'f') g = m.ne * ned + (int64_t)m.tet_faces[t * 4 + d.ent] * nfd + d.q;
      else g = m.ne * ned + m.nf * nfd + t * nvd + d.q;
      m.dofmap[t * nl + a] = (int32_t)g;
    }
  // ---------------- row incidence (counting sort, ascending tet then local index)
  m.tinc_ptr.assign(ndof + 1, 0);
  for (int64_t i = 0; i < T * nl; ++i) m.tinc_ptr[m.dofmap[i] + 1]++;
  for (int64_t g = 0; g < ndof; ++g) m.tinc_ptr[g + 1] += m.tinc_ptr[g];
  m.tinc.resize(T * nl);
  {
    std::vector<int64_t> pos(m.tinc_ptr.begin(), m.tinc_ptr.end() - 1);
    for (int64_t t = 0; t < T; ++t)
      for (int a = 0; a < nl; ++a) m.tinc[pos[m.dofmap[t * nl + a]]++] = (int32_t)(t * nl + a);
  }
  // ---------------- partition
  if (p->part) {
    m.part.assign(p->part, p->part + T);
    for (int64_t t = 0; t < T; ++t)
      if (m.part[t] < 0 || m.part[t] >= m.nsub) { err = "oras_create: part entry out of range"; return ORAS_ERR_BAD_MESH; }
  } else {
    rcb(m, m.nsub, m.part);
  }
  // ---------------- overlap and membership
  m.member_words = (T + 31) / 32;
  m.member.assign((size_t)m.nsub * m.member_words, 0u);
  {
    std::vector<uint8_t> tmark(T), vmark(nv);
    for (int s = 0; s < m.nsub; ++s) {
      for (int64_t t = 0; t < T; ++t) tmark[t] = m.part[t] == s;
      for (int layer = 0; layer < m.overlap; ++layer) {
        if (overlap_kind == ORAS_OVERLAP_FACE) {
          std::vector<uint8_t> next(tmark);
          for (int64_t t = 0; t < T; ++t)
            if (tmark[t])
              for (int f = 0; f < 4; ++f) {
                int32_t fid = m.tet_faces[t * 4 + f];
                for (int q = 0; q < 2; ++q) {
                  int32_t o = m.face_tets[fid * 2 + q];
                  if (o >= 0) next[o] = 1;
                }
              }
          tmark.swap(next);
        } else {
          std::fill(vmark.begin(), vmark.end(), 0);
          for (int64_t t = 0; t < T; ++t)
            if (tmark[t])
              for (int q = 0; q < 4; ++q) vmark[m.st[t * 4 + q]] = 1;
          for (int64_t t = 0; t < T; ++t) {
            const int32_t* v = &m.st[t * 4];
            tmark[t] = vmark[v[0]] | vmark[v[1]] | vmark[v[2]] | vmark[v[3]];
          }
        }
      }
      for (int64_t t = 0; t < T; ++t)
        if (tmark[t]) m.member[(size_t)s * m.member_words + (t >> 5)] |= 1u << (t & 31);
    }
  }
  // ---------------- owners (lowest tet carrying the DOF) and N_s / D_s
  std::vector<int32_t> owner(ndof, -1);
  for (int64_t t = 0; t < T; ++t)
    for (int a = 0; a < nl; ++a) {
      int32_t g = m.dofmap[t * nl + a];
      if (owner[g] < 0) owner[g] = m.part[t];
    }
  m.sub_ns.resize(m.nsub);
  m.sub_np.resize(m.nsub);
  m.sub_ns_off.resize(m.nsub + 1);
  m.sub_nt_off.resize(m.nsub + 1);
  m.sub_tile_off.resize(m.nsub + 1);
  m.sub_ns_off[0] = 0;
  m.sub_nt_off[0] = 0;
  m.sub_tile_off[0] = 0;
  m.sub_dofs.clear();
  m.sub_pou.clear();
  m.sub_tets.clear();
  m.max_np = 0;
  std::vector<uint8_t> iface_mark(m.nf, 0);
  std::vector<int32_t> buf;
  for (int s = 0; s < m.nsub; ++s) {
    buf.clear();
    int64_t nts = 0;
    for (int64_t t = 0; t < T; ++t) {
      if (!member_of(m, s, t)) continue;
      m.sub_tets.push_back((int32_t)t);
      ++nts;
      for (int a = 0; a < nl; ++a) buf.push_back(m.dofmap[t * nl + a]);
      for (int f = 0; f < 4; ++f) {
        int32_t fid = m.tet_faces[t * 4 + f];
        int32_t o = m.face_tets[fid * 2] == t ? m.face_tets[fid * 2 + 1] : m.face_tets[fid * 2];
        if (o >= 0 && !member_of(m, s, o)) iface_mark[fid] = 1;
      }
    }
    std::sort(buf.begin(), buf.end());
    buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
    int64_t ns = (int64_t)buf.size();
    m.sub_ns[s] = ns;
    m.sub_np[s] = (ns + TB - 1) / TB * TB;
    m.max_np = std::max(m.max_np, m.sub_np[s]);
    for (auto g : buf) {
      m.sub_dofs.push_back(g);
      m.sub_pou.push_back(owner[g] == s ? 1 : 0);
    }
    m.sub_ns_off[s + 1] = m.sub_ns_off[s] + ns;
    m.sub_nt_off[s + 1] = m.sub_nt_off[s] + nts;
    int64_t tt = m.sub_np[s] / TB;
    m.sub_tile_off[s + 1] = m.sub_tile_off[s] + tt * tt;
  }
  m.arena_tiles = m.sub_tile_off[m.nsub];
  // ---------------- impedance faces: outer boundary + interface faces of some subdomain
  m.if_face.clear(); m.if_tet0.clear(); m.if_lf0.clear(); m.if_tet1.clear();
  for (int64_t f = 0; f < m.nf; ++f) {
    bool outer = m.face_tets[f * 2 + 1] < 0;
    if (!outer && !iface_mark[f]) continue;
    int32_t t0 = m.face_tets[f * 2];
    int lf = 0;
    while (m.tet_faces[t0 * 4 + lf] != f) ++lf;
    m.if_face.push_back((int32_t)f);
    m.if_tet0.push_back(t0);
    m.if_lf0.push_back(lf);
    m.if_tet1.push_back(m.face_tets[f * 2 + 1]);
  }
  m.nif = (int64_t)m.if_face.size();
  m.if_dofs.resize(m.nif * nfl);
  std::vector<std::vector<int>> fld(4);
  for (int lf = 0; lf < 4; ++lf) fld[lf] = face_local_dofs(r, lf);
  for (int64_t i = 0; i < m.nif; ++i)
    for (int af = 0; af < nfl; ++af)
      m.if_dofs[i * nfl + af] = m.dofmap[(int64_t)m.if_tet0[i] * nl + fld[m.if_lf0[i]][af]];
  m.finc_ptr.assign(ndof + 1, 0);
  for (int64_t i = 0; i < m.nif * nfl; ++i) m.finc_ptr[m.if_dofs[i] + 1]++;
  for (int64_t g = 0; g < ndof; ++g) m.finc_ptr[g + 1] += m.finc_ptr[g];
  m.finc.resize(m.nif * nfl);
  {
    std::vector<int64_t> pos(m.finc_ptr.begin(), m.finc_ptr.end() - 1);
    for (int64_t i = 0; i < m.nif; ++i)
      for (int af = 0; af < nfl; ++af) m.finc[pos[m.if_dofs[i * nfl + af]]++] = (int32_t)(i * nfl + af);
  }
  // ---------------- CSR pattern: union of the DOFs of the tets carrying each row
  m.rowptr.assign(ndof + 1, 0);
  std::vector<std::vector<int32_t>> rows;
  const int64_t CH = 1 << 16;
  std::vector<int32_t> colbuf;
  m.cols.clear();
  m.max_row_nnz = 0;
  std::vector<int32_t> row;
  for (int64_t g = 0; g < ndof; ++g) {
    row.clear();
    for (int64_t q = m.tinc_ptr[g]; q < m.tinc_ptr[g + 1]; ++q) {
      int64_t t = m.tinc[q] / nl;
      for (int b = 0; b < nl; ++b) row.push_back(m.dofmap[t * nl + b]);
    }
    std::sort(row.begin(), row.end());
    row.erase(std::unique(row.begin(), row.end()), row.end());
    m.cols.insert(m.cols.end(), row.begin(), row.end());
    m.rowptr[g + 1] = (int64_t)m.cols.size();
    m.max_row_nnz = std::max<int>(m.max_row_nnz, (int)row.size());
  }
  (void)CH;
  return ORAS_OK;
}

}  // namespace oras
