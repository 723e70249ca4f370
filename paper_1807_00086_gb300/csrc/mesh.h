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

}  // namespace hdg
