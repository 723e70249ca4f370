// Mesh skeleton and affine geometry (host side), Sec. 2.1.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace hdg {

// Per-element geometry record, GEO_STRIDE doubles:
//   [0]                    |det J|
//   [1 .. 1+d*d)           J^{-1} row-major: Jinv[r][j] = d xi_r / d x_j
//   [1+d*d .. +d+1)        face Jacobians J_F (edge length / twice the face area)
//   [.. +(d+1)*d)          outward unit normals n_f, face-major
constexpr int GEO_STRIDE = 32;
inline int geo_jf(int d) { return 1 + d * d; }
inline int geo_n(int d) { return 1 + d * d + d + 1; }

struct Skeleton {
  int dim = 0;
  int64_t ne = 0, nf = 0, nb = 0;
  std::vector<int32_t> elem;       // [ne][d+1] ascending vertex ids
  std::vector<int32_t> elem_face;  // [ne][d+1] face of local face j
  std::vector<int32_t> face_slot;  // [nf][2] slot e*(d+1)+j (lower element first), -1 if none
  std::vector<int32_t> face_bnd;   // [nf] boundary index or -1
  std::vector<int64_t> bnd_faces;  // [nb] face ids of boundary faces, ascending
  std::vector<double> geo;         // [ne][GEO_STRIDE]
};

// Builds the skeleton; returns false and sets err on invalid input.
bool build_skeleton(int dim, int64_t nv, int64_t ne, const double* vert, const int32_t* ev, Skeleton& sk,
                    std::string& err);

// Continuous traces on a face subset (Sec. 2.2): all faces (EDG) or the interior faces (IEDG).
// The unknowns are the degree-k equispaced nodes of those faces, shared between faces by the
// vertices of the smallest sub-simplex containing the node and its integer barycentric
// weights there, and numbered by first appearance over the faces in face order, lexicographic
// (b_0, ..) within a face. EDG fixes the nodes that lie on the boundary. face_node [nf][Nf]:
// the free node of each face node, -1 for a fixed node or a face outside the subset.
bool build_trace_nodes(const Skeleton& sk, int k, bool all_faces, int64_t& n_free, std::vector<int32_t>& face_node,
                       std::string& err);

}  // namespace hdg
