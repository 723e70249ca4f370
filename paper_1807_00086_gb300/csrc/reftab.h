// Reference-element tables of the library (host side). Written independently of the
// CPU oracle; both follow the basis and quadrature conventions stated in include/hdg.h.
#pragma once
#include <vector>

namespace hdg {

int n_modes(int dim, int k);  // C(k+dim, dim)

// Gauss-Jacobi rule for weight (1-x)^a (1+x)^b on [-1, 1], n points.
void gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& w);
// Collapsed product rule with n points per direction on the unit simplex of dimension dim
// (dim = 1: [0,1]); pts is [nq][dim], weights sum to the simplex measure.
void simplex_rule(int dim, int n, std::vector<double>& pts, std::vector<double>& w);
// Orthonormal Dubiner basis of degree k at points pts [np][dim] of the unit simplex:
// val [np][Nb], grad [np][Nb][dim] (grad may be null).
void dubiner(int dim, int k, const double* pts, int np, double* val, double* grad);

struct RefTables {
  int dim = 0, k = 0, Np = 0, Nf = 0, nqv = 0, nqf = 0;
  std::vector<double> Dr;    // [dim][Np][Np]     Dr[r][i][l] = int d_r phi_l phi_i
  std::vector<double> Ff;    // [dim+1][Np][Nf]   int_face phi_i(xi_f(eta)) mu_m(eta) d eta
  std::vector<double> Ef;    // [dim+1][Np][Np]   Ff Ff^T
  std::vector<double> Trs;   // [dim][dim][Np][Np] Dr Ds^T
  std::vector<double> DFrf;  // [dim][dim+1][Np][Nf] Dr Ff
  std::vector<double> Pfg;   // [dim+1][dim+1][Nf][Nf] Ff^T Fg
  std::vector<double> qv_pts, qv_w, qv_phi;  // volume rule: [nqv][dim], [nqv], [nqv][Np]
  std::vector<double> qf_pts, qf_w, qf_mu;   // face rule:   [nqf][dim-1], [nqf], [nqf][Nf]
};

RefTables build_tables(int dim, int k);
// Tables of a volume degree kv whose faces carry traces of degree kf >= kv (variable-degree
// meshes): Np = Np(kv), Nf = Nf(kf); the rules take max(kv, kf) + 2 points per direction.
// build_tables(dim, k) == build_tables_pair(dim, k, k).
RefTables build_tables_pair(int dim, int kv, int kf);
// total degree of each face mode of degree kf, in the face basis order
std::vector<int> face_mode_degrees(int dim, int kf);

// Tables of the local post-processing into P_{k+1} (psi: orthonormal degree-(k+1) basis,
// phi: degree k; volume rule of k + 3 points per direction, exact for both products):
//   K1[r][s][i][l] = int d_r psi_i d_s psi_l      [dim][dim][Np1][Np1]
//   E1[r][i][l]    = int d_r psi_i phi_l          [dim][Np1][Np]
// psi_0 = phi_0 (the same constant); build_post_tables checks it.
struct PostTables {
  int dim = 0, k = 0, Np = 0, Np1 = 0;
  std::vector<double> K1, E1;
};
PostTables build_post_tables(int dim, int k);

// Values at the degree-k equispaced nodes of the reference face of a dim-simplex (integer
// barycentric weights (b_0, .., b_{dim-1}) summing to k, in lexicographic order; reference
// coordinates (b_1, .., b_{dim-1}) / k) -> coefficients in the orthonormal face basis:
// [Nf][Nf] row-major, the L2 projection of each nodal Lagrange function (built from monomials,
// so the collapsed-coordinate basis is never evaluated at its singular vertex).
std::vector<double> face_nodal_to_modal(int dim, int k);

}  // namespace hdg
