// Skeleton E_h = E_h^I u E_h^B (Sec. 2.1): faces numbered in lexicographic order of their
// sorted vertex ids, each with its (at most two) element slots; affine geometry per element.
#include "mesh.h"

#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <unordered_map>
#include <unordered_set>

namespace hdg {

bool build_skeleton(int dim, int64_t nv, int64_t ne, const double* vert, const int32_t* ev, Skeleton& sk,
                    std::string& err) {
  if (dim != 2 && dim != 3) { err = "dim must be 2 or 3"; return false; }
  if (ne <= 0 || nv <= dim) { err = "empty mesh"; return false; }
  if (ne > (int64_t)1 << 28) { err = "too many elements"; return false; }
  const int nc = dim + 1;
  sk.dim = dim; sk.ne = ne;
  sk.elem.assign(ev, ev + ne * nc);
  for (int64_t e = 0; e < ne; ++e) {
    int32_t* v = &sk.elem[e * nc];
    std::sort(v, v + nc);
    for (int i = 0; i < nc; ++i)
      if (v[i] < 0 || v[i] >= nv) { err = "vertex id out of range in element " + std::to_string(e); return false; }
    for (int i = 1; i < nc; ++i)
      if (v[i] == v[i - 1]) { err = "repeated vertex in element " + std::to_string(e); return false; }
  }
  // (face key, slot) records sorted by key then slot
  struct Rec { std::array<int32_t, 3> key; int64_t slot; };
  std::vector<Rec> recs((size_t)ne * nc);
  for (int64_t e = 0; e < ne; ++e)
    for (int j = 0; j < nc; ++j) {
      Rec r; r.key = {-1, -1, -1}; int c = 0;
      for (int i = 0; i < nc; ++i) if (i != j) r.key[c++] = sk.elem[e * nc + i];
      r.slot = e * nc + j;
      recs[e * nc + j] = r;
    }
  std::sort(recs.begin(), recs.end(), [](const Rec& a, const Rec& b) {
    return a.key != b.key ? a.key < b.key : a.slot < b.slot;
  });
  sk.elem_face.assign((size_t)ne * nc, -1);
  sk.face_slot.clear(); sk.face_bnd.clear(); sk.bnd_faces.clear();
  size_t i = 0;
  while (i < recs.size()) {
    size_t j = i + 1;
    while (j < recs.size() && recs[j].key == recs[i].key) ++j;
    if (j - i > 2) { err = "face shared by more than two elements"; return false; }
    int32_t f = (int32_t)sk.face_slot.size() / 2;
    sk.face_slot.push_back((int32_t)recs[i].slot);
    sk.face_slot.push_back(j - i == 2 ? (int32_t)recs[i + 1].slot : -1);
    for (size_t q = i; q < j; ++q) sk.elem_face[recs[q].slot] = f;
    if (j - i == 1) { sk.face_bnd.push_back((int32_t)sk.bnd_faces.size()); sk.bnd_faces.push_back(f); }
    else sk.face_bnd.push_back(-1);
    i = j;
  }
  sk.nf = (int64_t)sk.face_slot.size() / 2;
  sk.nb = (int64_t)sk.bnd_faces.size();
  // geometry
  sk.geo.assign((size_t)ne * GEO_STRIDE, 0.0);
  for (int64_t e = 0; e < ne; ++e) {
    double X[4][3] = {};
    for (int a = 0; a < nc; ++a)
      for (int r = 0; r < dim; ++r) X[a][r] = vert[(int64_t)sk.elem[e * nc + a] * dim + r];
    double J[3][3] = {}, Ji[3][3] = {};
    for (int r = 0; r < dim; ++r)
      for (int q = 0; q < dim; ++q) J[q][r] = X[r + 1][q] - X[0][q];   // column r = X_r - X_0
    double det, scale = 0.0;
    for (int a = 1; a < nc; ++a)
      for (int q = 0; q < dim; ++q) scale = std::max(scale, std::fabs(X[a][q] - X[0][q]));
    if (dim == 2) {
      det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      Ji[0][0] = J[1][1] / det; Ji[0][1] = -J[0][1] / det;
      Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
    } else {
      det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
            J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
      Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
      Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
      Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
      Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
      Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
      Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
      Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
      Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
      Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    }
    if (!(std::fabs(det) > 1e-13 * std::pow(scale, dim))) { err = "degenerate element " + std::to_string(e); return false; }
    double* g = &sk.geo[e * GEO_STRIDE];
    g[0] = std::fabs(det);
    for (int r = 0; r < dim; ++r)
      for (int q = 0; q < dim; ++q) g[1 + r * dim + q] = Ji[r][q];
    for (int f = 0; f < nc; ++f) {
      int fv[3], c = 0;
      for (int a = 0; a < nc; ++a) if (a != f) fv[c++] = a;
      double n[3] = {}, jf;
      if (dim == 2) {
        double tx = X[fv[1]][0] - X[fv[0]][0], ty = X[fv[1]][1] - X[fv[0]][1];
        jf = std::sqrt(tx * tx + ty * ty);
        n[0] = ty / jf; n[1] = -tx / jf;
      } else {
        double a[3], b[3];
        for (int q = 0; q < 3; ++q) { a[q] = X[fv[1]][q] - X[fv[0]][q]; b[q] = X[fv[2]][q] - X[fv[0]][q]; }
        n[0] = a[1] * b[2] - a[2] * b[1]; n[1] = a[2] * b[0] - a[0] * b[2]; n[2] = a[0] * b[1] - a[1] * b[0];
        jf = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int q = 0; q < 3; ++q) n[q] /= jf;
      }
      double s = 0.0;
      for (int q = 0; q < dim; ++q) s += n[q] * (X[f][q] - X[fv[0]][q]);
      if (s > 0) for (int q = 0; q < dim; ++q) n[q] = -n[q];
      g[geo_jf(dim) + f] = jf;
      for (int q = 0; q < dim; ++q) g[geo_n(dim) + f * dim + q] = n[q];
    }
  }
  return true;
}

namespace {
struct Key3 {
  std::array<int64_t, 3> v;
  bool operator==(const Key3& o) const { return v == o.v; }
};
struct Key3Hash {
  size_t operator()(const Key3& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int64_t x : k.v) { h ^= (uint64_t)x + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2); }
    return (size_t)h;
  }
};
}  // namespace

bool build_trace_nodes(const Skeleton& sk, int k, bool all_faces, int64_t& n_free, std::vector<int32_t>& face_node,
                       std::string& err) {
  const int dim = sk.dim, nc = dim + 1, fv = dim;   // a face has dim vertices
  if (k < 1 || k > 4) { err = "trace degree must be 1..4"; return false; }
  const int Nf = dim == 2 ? k + 1 : (k + 1) * (k + 2) / 2;
  auto face_verts = [&](int64_t f, int64_t* out) {
    const int32_t slot = sk.face_slot[2 * f];
    const int64_t e = slot / nc;
    const int j = slot % nc;
    int c = 0;
    for (int i = 0; i < nc; ++i) if (i != j) out[c++] = sk.elem[e * nc + i];
  };
  // node weights of a face in lexicographic order
  std::vector<std::array<int, 3>> bs;
  for (int b0 = 0; b0 <= k; ++b0)
    if (fv == 2) bs.push_back({b0, k - b0, 0});
    else for (int b1 = 0; b0 + b1 <= k; ++b1) bs.push_back({b0, b1, k - b0 - b1});
  // sub-simplices of boundary faces (EDG: nodes supported there are fixed)
  std::unordered_set<Key3, Key3Hash> bsub;
  if (all_faces)
    for (int64_t f = 0; f < sk.nf; ++f) {
      if (sk.face_bnd[f] < 0) continue;
      int64_t v[3];
      face_verts(f, v);
      for (int mask = 1; mask < (1 << fv); ++mask) {
        Key3 key{{-1, -1, -1}};
        int c = 0;
        for (int i = 0; i < fv; ++i) if (mask & (1 << i)) key.v[c++] = v[i];
        bsub.insert(key);
      }
    }
  std::unordered_map<Key3, int64_t, Key3Hash> id;
  std::vector<uint8_t> fixed;
  std::vector<int64_t> node_of((size_t)sk.nf * Nf, -1);
  for (int64_t f = 0; f < sk.nf; ++f) {
    if (!all_faces && sk.face_bnd[f] >= 0) continue;
    int64_t v[3];
    face_verts(f, v);
    for (int a = 0; a < Nf; ++a) {
      Key3 key{{-1, -1, -1}}, support{{-1, -1, -1}};
      int c = 0;
      for (int i = 0; i < fv; ++i)
        if (bs[a][i] > 0) { key.v[c] = v[i] * (k + 1) + bs[a][i]; support.v[c] = v[i]; ++c; }
      auto it = id.find(key);
      if (it == id.end()) {
        it = id.emplace(key, (int64_t)fixed.size()).first;
        fixed.push_back(all_faces && bsub.count(support) ? 1 : 0);
      }
      node_of[(size_t)f * Nf + a] = it->second;
    }
  }
  std::vector<int64_t> free_pos(fixed.size(), -1);
  n_free = 0;
  for (size_t i = 0; i < fixed.size(); ++i) if (!fixed[i]) free_pos[i] = n_free++;
  if (n_free > INT32_MAX) { err = "too many trace nodes"; return false; }
  face_node.assign((size_t)sk.nf * Nf, -1);
  for (size_t t = 0; t < node_of.size(); ++t)
    if (node_of[t] >= 0) face_node[t] = (int32_t)free_pos[node_of[t]];
  return true;
}

}  // namespace hdg
