// Element partitions for partitioned runs (not part of the paper's method, which runs on one
// processor): the operator of Eq. euler3 couples an element only to its face neighbours, so a
// partition computes its own elements' rows of R(u) and J v from its own elements plus a
// one-element halo, and everything else of the Krylov step (Sec. 2.2) is vector arithmetic
// and inner products over the own rows.
#include "partition.h"

#include <algorithm>
#include <array>
#include <unordered_map>

namespace pcexp {

namespace {

using Key = std::array<int64_t, 3>;

struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t h = (uint64_t)k[0] * 0x9E3779B97F4A7C15ull;
    h ^= (uint64_t)k[1] + 0x632BE59BD9B4E019ull + (h << 6) + (h >> 2);
    h ^= (uint64_t)k[2] + 0x85157AF5ull + (h << 6) + (h >> 2);
    return (size_t)h;
  }
};

// local face f of an element: the vertices f+1, ..., f+D (mod D+1), as in the face list
inline int face_vertex(int D, int f, int k) { return (f + 1 + k) % (D + 1); }

int64_t master_of(const pcexp_mesh& m, int64_t v) { return m.vert_master ? m.vert_master[v] : v; }

// sorted vertices of local face f of e: periodic masters (what faces match on) or the element's
// own vertices (what boundary tags are looked up by)
Key face_key(const pcexp_mesh& m, int64_t e, int f, bool masters = true) {
  const int D = m.dim;
  Key k{-1, -1, -1};
  for (int i = 0; i < D; ++i) {
    const int64_t v = m.elem_vert[(int64_t)(D + 1) * e + face_vertex(D, f, i)];
    k[i] = masters ? master_of(m, v) : v;
  }
  std::sort(k.begin(), k.begin() + D);
  return k;
}

void centroid(const pcexp_mesh& m, int64_t e, double* c) {
  const int D = m.dim;
  for (int d = 0; d < D; ++d) c[d] = 0;
  for (int i = 0; i <= D; ++i) {
    const int64_t v = m.elem_vert[(int64_t)(D + 1) * e + i];
    for (int d = 0; d < D; ++d) c[d] += m.coords[(int64_t)D * v + d];
  }
  for (int d = 0; d < D; ++d) c[d] /= (D + 1);
}

void bisect(const std::vector<double>& cen, int D, std::vector<int64_t>& ids, size_t lo, size_t hi, int n_parts,
            int first, int32_t* part) {
  if (n_parts <= 1 || hi - lo <= 1) {
    for (size_t i = lo; i < hi; ++i) part[ids[i]] = first;
    return;
  }
  double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
  for (size_t i = lo; i < hi; ++i)
    for (int d = 0; d < D; ++d) {
      mn[d] = std::min(mn[d], cen[(size_t)D * ids[i] + d]);
      mx[d] = std::max(mx[d], cen[(size_t)D * ids[i] + d]);
    }
  int ax = 0;
  for (int d = 1; d < D; ++d)
    if (mx[d] - mn[d] > mx[ax] - mn[ax]) ax = d;
  const int n1 = n_parts / 2;
  const size_t cut = lo + (size_t)((double)(hi - lo) * n1 / n_parts + 0.5);
  auto less = [&](int64_t a, int64_t b) {
    const double ca = cen[(size_t)D * a + ax], cb = cen[(size_t)D * b + ax];
    return ca < cb || (ca == cb && a < b);
  };
  std::nth_element(ids.begin() + lo, ids.begin() + cut, ids.begin() + hi, less);
  bisect(cen, D, ids, lo, cut, n1, first, part);
  bisect(cen, D, ids, cut, hi, n_parts - n1, first + n1, part);
}

}  // namespace

void rcb_partition(const pcexp_mesh& m, int n_parts, int32_t* part) {
  const int D = m.dim;
  std::vector<double> cen((size_t)D * m.n_elem);
  for (int64_t e = 0; e < m.n_elem; ++e) centroid(m, e, &cen[(size_t)D * e]);
  std::vector<int64_t> ids((size_t)m.n_elem);
  for (int64_t e = 0; e < m.n_elem; ++e) ids[(size_t)e] = e;
  bisect(cen, D, ids, 0, ids.size(), n_parts, 0, part);
}

int face_neighbours(const pcexp_mesh& m, std::vector<int64_t>& nbr, std::string& msg) {
  const int NF = m.dim + 1;
  nbr.assign((size_t)m.n_elem * NF, -1);
  std::vector<std::pair<Key, int64_t>> all((size_t)m.n_elem * NF);
  for (int64_t e = 0; e < m.n_elem; ++e)
    for (int f = 0; f < NF; ++f) all[(size_t)e * NF + f] = {face_key(m, e, f), e * NF + f};
  std::sort(all.begin(), all.end());
  for (size_t i = 0; i < all.size();) {
    size_t j = i + 1;
    while (j < all.size() && all[j].first == all[i].first) ++j;
    if (j - i > 2) {
      msg = "face shared by more than two elements";
      return PCEXP_ERR_MESH;
    }
    if (j - i == 2) {
      nbr[(size_t)all[i].second] = all[i + 1].second / NF;
      nbr[(size_t)all[i + 1].second] = all[i].second / NF;
    }
    i = j;
  }
  return PCEXP_OK;
}

void build_halo(const pcexp_mesh& m, const std::vector<int64_t>& nbr, const int32_t* part, int k, Halo& h) {
  const int NF = m.dim + 1;
  h.elems.clear();
  std::vector<int64_t> ghost;
  for (int64_t e = 0; e < m.n_elem; ++e) {
    if (part[e] != k) continue;
    h.elems.push_back(e);
    for (int f = 0; f < NF; ++f) {
      const int64_t n = nbr[(size_t)e * NF + f];
      if (n >= 0 && part[n] != k) ghost.push_back(n);
    }
  }
  h.n_owned = (int64_t)h.elems.size();
  std::sort(ghost.begin(), ghost.end());
  ghost.erase(std::unique(ghost.begin(), ghost.end()), ghost.end());
  h.elems.insert(h.elems.end(), ghost.begin(), ghost.end());
}

int build_submesh(const pcexp_mesh& m, const Halo& h, Submesh& s, std::string& msg) {
  const int D = m.dim, NF = D + 1;
  s.dim = D;
  s.periodic = m.vert_master != nullptr;
  s.coords.clear();
  s.elem_vert.clear();
  s.vert_master.clear();
  s.bface_vert.clear();
  s.bface_tag.clear();
  // local vertices: those of the elements, then (periodic meshes) their masters
  std::unordered_map<int64_t, int32_t> loc;
  std::vector<int64_t> glob;
  auto local_of = [&](int64_t g) -> int32_t {
    auto it = loc.find(g);
    if (it != loc.end()) return it->second;
    const int32_t l = (int32_t)glob.size();
    loc.emplace(g, l);
    glob.push_back(g);
    return l;
  };
  for (int64_t e : h.elems)
    for (int i = 0; i <= D; ++i) s.elem_vert.push_back(local_of(m.elem_vert[(int64_t)(D + 1) * e + i]));
  if (s.periodic)
    for (size_t i = 0; i < glob.size(); ++i) local_of(master_of(m, glob[i]));  // glob grows only by masters
  for (int64_t g : glob)
    for (int d = 0; d < D; ++d) s.coords.push_back(m.coords[(int64_t)D * g + d]);
  if (s.periodic)
    for (int64_t g : glob) s.vert_master.push_back(loc.at(master_of(m, g)));
  // faces of the local elements: how many local elements share each
  struct Use {
    int count;
    int64_t le;
    int f;
    bool tagged;
  };
  std::unordered_map<Key, Use, KeyHash> faces;   // on master vertices
  std::unordered_map<Key, Key, KeyHash> by_own;   // the element's own face vertices -> master key
  faces.reserve(h.elems.size() * NF);
  by_own.reserve(h.elems.size() * NF);
  for (size_t le = 0; le < h.elems.size(); ++le)
    for (int f = 0; f < NF; ++f) {
      const Key k = face_key(m, h.elems[le], f);
      by_own.emplace(face_key(m, h.elems[le], f, false), k);
      auto it = faces.find(k);
      if (it == faces.end()) faces.emplace(k, Use{1, (int64_t)le, f, false});
      else ++it->second.count;
    }
  // tagged boundary faces of the local elements (tags are looked up by an element's own face
  // vertices)
  for (int64_t i = 0; i < m.n_bface; ++i) {
    Key k{-1, -1, -1};
    for (int d = 0; d < D; ++d) k[d] = m.bface_vert[(int64_t)D * i + d];
    std::sort(k.begin(), k.begin() + D);
    auto ob = by_own.find(k);
    if (ob == by_own.end()) continue;
    auto it = faces.find(ob->second);
    it->second.tagged = true;
    for (int d = 0; d < D; ++d) {
      auto lv = loc.find(m.bface_vert[(int64_t)D * i + d]);
      if (lv == loc.end()) {
        msg = "boundary face vertex is not a vertex of its element";
        return PCEXP_ERR_MESH;
      }
      s.bface_vert.push_back(lv->second);
    }
    s.bface_tag.push_back(m.bface_tag ? m.bface_tag[i] : 0);
  }
  // the outer faces of the halo: symmetry planes, on the element's own face vertices
  std::vector<std::pair<int64_t, int>> outer;
  for (const auto& kv : faces)
    if (kv.second.count == 1 && !kv.second.tagged) {
      if (kv.second.le < h.n_owned) {
        msg = "face of an owned element with no partner and no tag";
        return PCEXP_ERR_MESH;
      }
      outer.push_back({kv.second.le, kv.second.f});
    }
  std::sort(outer.begin(), outer.end());  // deterministic order
  for (const auto& of : outer) {
    const Key k = face_key(m, h.elems[(size_t)of.first], of.second, false);
    for (int d = 0; d < D; ++d) s.bface_vert.push_back(loc.at(k[d]));
    s.bface_tag.push_back(PCEXP_BC_SYMMETRY);
  }
  return PCEXP_OK;
}

pcexp_mesh Submesh::view() const {
  pcexp_mesh v{};
  v.dim = dim;
  v.n_vert = (int64_t)coords.size() / dim;
  v.coords = coords.data();
  v.n_elem = (int64_t)elem_vert.size() / (dim + 1);
  v.elem_vert = elem_vert.data();
  v.vert_master = periodic ? vert_master.data() : nullptr;
  v.n_bface = (int64_t)bface_tag.size();
  v.bface_vert = bface_vert.data();
  v.bface_tag = bface_tag.data();
  return v;
}

}  // namespace pcexp
