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
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <exception>
#include <mutex>
#include <numeric>
#include <system_error>
#include <thread>

#include "internal.h"

namespace oras {

// Number of workers parallel_for(n, grain, ...) uses (at most min(hardware_concurrency(), 16));
// per-worker buffers are sized with it.
static int workers_for(int64_t n, int64_t grain) {
  unsigned hw = std::thread::hardware_concurrency();
  int64_t nw = std::min<int64_t>(hw ? hw : 1, 16);
  return (int)std::max<int64_t>(1, std::min<int64_t>(nw, (n + grain - 1) / grain));
}

// Runs fn(i, worker) for i in [0, n), worker in [0, workers_for(n, grain)), chunks of `grain`
// taken from a shared counter.  Every i writes only its own outputs, so results do not depend on
// the thread count or the schedule.  An exception in any worker is rethrown here after all
// workers joined.
template <typename F>
static void parallel_for(int64_t n, int64_t grain, F fn) {
  const int nw = workers_for(n, grain);
  if (nw <= 1) {
    for (int64_t i = 0; i < n; ++i) fn(i, 0);
    return;
  }
  std::atomic<int64_t> next(0);
  std::exception_ptr err;
  std::mutex err_mu;
  auto work = [&](int w) {
    try {
      for (;;) {
        const int64_t i0 = next.fetch_add(grain);
        if (i0 >= n) return;
        const int64_t i1 = std::min(n, i0 + grain);
        for (int64_t i = i0; i < i1; ++i) fn(i, w);
      }
    } catch (...) {  // keep the first error for the caller; no further chunks are taken
      std::lock_guard<std::mutex> lk(err_mu);
      if (!err) err = std::current_exception();
      next.store(n);
    }
  };
  std::vector<std::thread> th;
  for (int w = 1; w < nw; ++w) {
    try {
      th.emplace_back(work, w);
    } catch (const std::system_error&) {  // no more threads: the started ones take the rest
      break;
    }
  }
  work(0);
  for (auto& x : th) x.join();
  if (err) std::rethrow_exception(err);
}

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
    int p0 = s.p / 2;
    int64_t h = ((int64_t)s.ids.size() * p0) / s.p;
    // the first h tets in (coordinate, id) order: a strict total order, so the selected set is
    // the same as after a full sort (the order inside each child is not used)
    std::nth_element(s.ids.begin(), s.ids.begin() + h, s.ids.end(), [&](int32_t a, int32_t b) {
      double ca = cen[(size_t)a * 3 + axis], cb = cen[(size_t)b * 3 + axis];
      if (ca < cb) return true;
      if (cb < ca) return false;
      return a < b;
    });
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
  parallel_for(T * 6, 1 << 14, [&](int64_t i, int) {
    tet_edges[i] = (int32_t)(std::lower_bound(ue.begin(), ue.end(), ek[i]) - ue.begin());
  });
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
  parallel_for(T * 4, 1 << 14, [&](int64_t i, int) {
    m.tet_faces[i] = (int32_t)(std::lower_bound(uf.begin(), uf.end(), fk[i]) - uf.begin());
  });
  for (int64_t t = 0; t < T; ++t)
    for (int f = 0; f < 4; ++f) {
      const int32_t id = m.tet_faces[t * 4 + f];
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
  // Omega_s^delta grown layer by layer from the tets of part s: a layer adds every tet sharing a
  // vertex (or a face) with the current set.  Only the tets added by the previous layer can
  // bring new neighbours, so each layer walks that frontier through the vertex -> tet (or face)
  // adjacency instead of sweeping the whole mesh.
  m.member_words = (T + 31) / 32;
  m.member.assign((size_t)m.nsub * m.member_words, 0u);
  std::vector<std::vector<int32_t>> omega(m.nsub);  // Omega_s^delta, ascending
  {
    std::vector<int64_t> part_ptr(m.nsub + 1, 0);
    for (int64_t t = 0; t < T; ++t) part_ptr[m.part[t] + 1]++;
    for (int s = 0; s < m.nsub; ++s) part_ptr[s + 1] += part_ptr[s];
    std::vector<int32_t> part_tets(T);
    {
      std::vector<int64_t> pos(part_ptr.begin(), part_ptr.end() - 1);
      for (int64_t t = 0; t < T; ++t) part_tets[pos[m.part[t]]++] = (int32_t)t;
    }
    std::vector<int64_t> v2t_ptr(nv + 1, 0);
    std::vector<int32_t> v2t;
    if (m.overlap > 0 && overlap_kind != ORAS_OVERLAP_FACE) {
      for (int64_t i = 0; i < T * 4; ++i) v2t_ptr[m.st[i] + 1]++;
      for (int64_t v = 0; v < nv; ++v) v2t_ptr[v + 1] += v2t_ptr[v];
      v2t.resize(T * 4);
      std::vector<int64_t> pos(v2t_ptr.begin(), v2t_ptr.end() - 1);
      for (int64_t i = 0; i < T * 4; ++i) v2t[pos[m.st[i]]++] = (int32_t)(i / 4);
    }
    const int nw = workers_for(m.nsub, 1);
    std::vector<std::vector<int32_t>> tstamp(nw), vstamp(nw);
    parallel_for(m.nsub, 1, [&](int64_t s64, int w) {
      const int s = (int)s64;
      auto& ts = tstamp[w];
      auto& vs = vstamp[w];
      if (ts.empty()) ts.assign(T, -1);
      if (vs.empty() && !v2t.empty()) vs.assign(nv, -1);
      std::vector<int32_t>& list = omega[s];
      list.assign(part_tets.begin() + part_ptr[s], part_tets.begin() + part_ptr[s + 1]);
      for (int32_t t : list) ts[t] = s;
      size_t begin = 0;
      for (int layer = 0; layer < m.overlap; ++layer) {
        const size_t end = list.size();
        for (size_t i = begin; i < end; ++i) {
          const int32_t t = list[i];
          if (overlap_kind == ORAS_OVERLAP_FACE) {
            for (int f = 0; f < 4; ++f) {
              const int32_t fid = m.tet_faces[(int64_t)t * 4 + f];
              for (int q = 0; q < 2; ++q) {
                const int32_t o = m.face_tets[(int64_t)fid * 2 + q];
                if (o >= 0 && ts[o] != s) { ts[o] = s; list.push_back(o); }
              }
            }
          } else {
            for (int q = 0; q < 4; ++q) {
              const int32_t v = m.st[(int64_t)t * 4 + q];
              if (vs[v] == s) continue;
              vs[v] = s;
              for (int64_t k = v2t_ptr[v]; k < v2t_ptr[v + 1]; ++k) {
                const int32_t o = v2t[k];
                if (ts[o] != s) { ts[o] = s; list.push_back(o); }
              }
            }
          }
        }
        begin = end;
      }
      std::sort(list.begin(), list.end());
      uint32_t* row = m.member.data() + (size_t)s * m.member_words;
      for (int32_t t : list) row[t >> 5] |= 1u << (t & 31);
    });
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
  // N_s of every subdomain (ascending DOFs of the tets of Omega_s^delta), in parallel
  std::vector<std::vector<int32_t>> ndofs(m.nsub);
  {
    const int nw = workers_for(m.nsub, 1);
    std::vector<std::vector<int32_t>> stamp(nw);
    parallel_for(m.nsub, 1, [&](int64_t s64, int w) {
      const int s = (int)s64;
      auto& st = stamp[w];
      if (st.empty()) st.assign(ndof, -1);
      auto& buf = ndofs[s];
      for (int32_t t : omega[s])
        for (int a = 0; a < nl; ++a) {
          const int32_t g = m.dofmap[(int64_t)t * nl + a];
          if (st[g] != s) { st[g] = s; buf.push_back(g); }
        }
      std::sort(buf.begin(), buf.end());
    });
  }
  for (int s = 0; s < m.nsub; ++s) {
    const int64_t nts = (int64_t)omega[s].size();
    for (int32_t t : omega[s]) {
      m.sub_tets.push_back(t);
      for (int f = 0; f < 4; ++f) {
        int32_t fid = m.tet_faces[(int64_t)t * 4 + f];
        int32_t o = m.face_tets[fid * 2] == t ? m.face_tets[fid * 2 + 1] : m.face_tets[fid * 2];
        if (o >= 0 && !member_of(m, s, o)) iface_mark[fid] = 1;
      }
    }
    const std::vector<int32_t>& buf = ndofs[s];
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
    std::vector<int32_t>().swap(ndofs[s]);
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
  // caller's impedance coefficients: face (t, q) of the caller is the one opposite the caller's
  // vertex tets[4t+q]; the sorted local face lf is opposite the sorted vertex 3 - lf
  // the caller's face index q of the face (t, sorted local face lf)
  auto caller_face = [&](int64_t t, int lf) {
    const int32_t vo = m.st[t * 4 + (3 - lf)];
    int q = 0;
    while (q < 4 && p->tets[t * 4 + q] != vo) ++q;
    return q;
  };
  // metallic faces (Sec. 2 eq. metallicbc): every entry 0 or 1, 1 only on outer faces
  std::vector<uint8_t> metal_if(m.nif, 0);
  m.fixed.clear();
  m.nfixed = 0;
  if (p->face_kind) {
    for (int64_t t = 0; t < m.nt; ++t)
      for (int lf = 0; lf < 4; ++lf) {
        const int q = caller_face(t, lf);
        const uint8_t kd = q < 4 ? p->face_kind[t * 4 + q] : 0;
        if (kd > 1) {
          err = "oras_create: face_kind of face " + std::to_string(q) + " of tetrahedron " + std::to_string(t) +
                " is neither 0 (impedance) nor 1 (metallic)";
          return ORAS_ERR_INVALID_ARG;
        }
        if (kd == 1 && m.face_tets[(int64_t)m.tet_faces[t * 4 + lf] * 2 + 1] >= 0) {
          err = "oras_create: face " + std::to_string(q) + " of tetrahedron " + std::to_string(t) +
                " is metallic but interior";
          return ORAS_ERR_INVALID_ARG;
        }
      }
    for (int64_t i = 0; i < m.nif; ++i)
      if (m.if_tet1[i] < 0) {
        const int q = caller_face(m.if_tet0[i], m.if_lf0[i]);
        metal_if[i] = q < 4 && p->face_kind[(int64_t)m.if_tet0[i] * 4 + q] == 1;
      }
  }
  m.if_beta.clear();
  if (p->beta_face) {
    m.if_beta.assign(m.nif, 0.0);
    for (int64_t i = 0; i < m.nif; ++i) {
      if (m.if_tet1[i] >= 0) continue;
      if (metal_if[i]) {  // not read: the face's degrees of freedom are constrained
        m.if_beta[i] = 1.0;
        continue;
      }
      const int64_t t = m.if_tet0[i];
      const int q = caller_face(t, m.if_lf0[i]);
      const double b = q < 4 ? p->beta_face[t * 4 + q] : NAN;
      if (!(std::isfinite(b) && b > 0.0)) {
        err = "oras_create: beta_face of the outer face " + std::to_string(q) + " of tetrahedron " +
              std::to_string(t) + " is not finite and positive";
        return ORAS_ERR_INVALID_ARG;
      }
      m.if_beta[i] = b;
    }
  }
  m.if_dofs.resize(m.nif * nfl);
  std::vector<std::vector<int>> fld(4);
  for (int lf = 0; lf < 4; ++lf) fld[lf] = face_local_dofs(r, lf);
  for (int64_t i = 0; i < m.nif; ++i)
    for (int af = 0; af < nfl; ++af)
      m.if_dofs[i * nfl + af] = m.dofmap[(int64_t)m.if_tet0[i] * nl + fld[m.if_lf0[i]][af]];
  // constrained degrees of freedom: those of the edges and of the face of every metallic face
  // (the face-local degrees of freedom: the only ones with a tangential trace on the face)
  if (p->face_kind) {
    m.fixed.assign(ndof, 0);
    for (int64_t i = 0; i < m.nif; ++i)
      if (metal_if[i])
        for (int af = 0; af < nfl; ++af) m.fixed[m.if_dofs[i * nfl + af]] = 1;
    for (int64_t g = 0; g < ndof; ++g) m.nfixed += m.fixed[g];
    if (m.nfixed == 0) m.fixed.clear();
  }
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
  // All DOFs of one entity (edge, face, volume) are carried by the same tets, so they share
  // one column set: it is built once per entity, in parallel over entities, in two passes
  // (count the distinct columns with a per-worker stamp array, then fill and sort).
  m.rowptr.assign(ndof + 1, 0);
  {
    const int64_t n_e = m.ne, n_f = nfd ? m.nf : 0, n_v = nvd ? T : 0;
    const int64_t ngroups = n_e + n_f + n_v;
    auto group = [&](int64_t q, int64_t& g0, int64_t& len) {
      if (q < n_e) { g0 = q * ned; len = ned; }
      else if (q < n_e + n_f) { g0 = m.ne * ned + (q - n_e) * nfd; len = nfd; }
      else { g0 = m.ne * ned + m.nf * nfd + (q - n_e - n_f) * nvd; len = nvd; }
    };
    const int64_t grain = 2048;
    const int nw = workers_for(ngroups, grain);
    std::vector<std::vector<int32_t>> stamp(nw);
    auto each_col = [&](int64_t g, int w, auto&& emit) {
      auto& st = stamp[w];
      if (st.empty()) st.assign(ndof, -1);
      for (int64_t q = m.tinc_ptr[g]; q < m.tinc_ptr[g + 1]; ++q) {
        const int64_t t = m.tinc[q] / nl;
        for (int b = 0; b < nl; ++b) {
          const int32_t c = m.dofmap[t * nl + b];
          if (st[c] != (int32_t)g) { st[c] = (int32_t)g; emit(c); }
        }
      }
    };
    parallel_for(ngroups, grain, [&](int64_t q, int w) {
      int64_t g0, len;
      group(q, g0, len);
      int64_t n = 0;
      each_col(g0, w, [&](int32_t) { ++n; });
      for (int64_t g = g0; g < g0 + len; ++g) m.rowptr[g + 1] = n;
    });
    // a row stamped in the counting pass must count again in the filling pass
    for (auto& st : stamp) std::fill(st.begin(), st.end(), -1);
    int max_nnz = 0;
    for (int64_t g = 0; g < ndof; ++g) {
      max_nnz = std::max<int>(max_nnz, (int)m.rowptr[g + 1]);
      m.rowptr[g + 1] += m.rowptr[g];
    }
    m.max_row_nnz = max_nnz;
    m.cols.resize(m.rowptr[ndof]);
    parallel_for(ngroups, grain, [&](int64_t q, int w) {
      int64_t g0, len;
      group(q, g0, len);
      int32_t* out = m.cols.data() + m.rowptr[g0];
      int64_t n = 0;
      each_col(g0, w, [&](int32_t c) { out[n++] = c; });
      std::sort(out, out + n);
      for (int64_t g = g0 + 1; g < g0 + len; ++g) std::memcpy(m.cols.data() + m.rowptr[g], out, n * sizeof(int32_t));
    });
  }
  return ORAS_OK;
}

}  // namespace oras
