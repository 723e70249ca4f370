// Reference-element tables (host). Quadrature: collapsed Gauss-Jacobi (Stroud) rules;
// basis: orthonormal Dubiner/PKDO polynomials on the unit simplex, modes ordered
// lexicographically in (i, j[, l]). These realise the discrete spaces of Sec. 2.2.
#include "reftab.h"

#include <array>
#include <cmath>
#include <stdexcept>

namespace hdg {

int n_modes(int dim, int k) {
  int r = 1;
  for (int i = 1; i <= dim; ++i) r = r * (k + i) / i;
  return r;
}

// P_n^{(a,b)}(x) and its derivative by the three-term recurrence.
static void jacobi_p(int n, double a, double b, double x, double& p, double& dp) {
  if (n < 0) { p = 0; dp = 0; return; }
  double p0 = 1.0, p1 = 0.5 * ((a + b + 2.0) * x + (a - b));
  double d0 = 0.0, d1 = 0.5 * (a + b + 2.0);
  if (n == 0) { p = p0; dp = d0; return; }
  for (int m = 2; m <= n; ++m) {
    double c = 2.0 * m + a + b;
    double A1 = 2.0 * m * (m + a + b) * (c - 2.0);
    double A2 = (c - 1.0) * (c * (c - 2.0) * x + a * a - b * b);
    double A3 = 2.0 * (m + a - 1.0) * (m + b - 1.0) * c;
    double A2d = (c - 1.0) * c * (c - 2.0);
    double p2 = (A2 * p1 - A3 * p0) / A1;
    double d2 = (A2 * d1 + A2d * p1 - A3 * d0) / A1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  p = p1; dp = d1;
}

static double jac(int n, double a, double b, double x) { double p, d; jacobi_p(n, a, b, x, p, d); return p; }
static double djac(int n, double a, double b, double x) { double p, d; jacobi_p(n, a, b, x, p, d); return d; }

void gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0); w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    // Chebyshev-like start, then Newton with deflation against the roots found so far.
    double z = -std::cos(pi * (i + 0.75 + 0.5 * a) / (n + 0.5 * (a + b + 1.0)));
    if (i > 0 && z <= x[i - 1]) z = x[i - 1] + 1e-3;
    for (int it = 0; it < 100; ++it) {
      double p, dp; jacobi_p(n, a, b, z, p, dp);
      double s = 0.0;
      for (int j = 0; j < i; ++j) s += 1.0 / (z - x[j]);
      double dz = p / (dp - s * p);
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
  double lg = std::lgamma(n + a + 1.0) + std::lgamma(n + b + 1.0) - std::lgamma(n + a + b + 1.0) - std::lgamma(n + 1.0);
  double c = std::exp(lg) * std::pow(2.0, a + b + 1.0);
  for (int i = 0; i < n; ++i) {
    double dp = djac(n, a, b, x[i]);
    w[i] = c / ((1.0 - x[i] * x[i]) * dp * dp);
  }
}

void simplex_rule(int dim, int n, std::vector<double>& pts, std::vector<double>& w) {
  std::vector<double> xa, wa, xb, wb, xc, wc;
  gauss_jacobi(n, 0, 0, xa, wa);
  pts.clear(); w.clear();
  if (dim == 1) {
    for (int i = 0; i < n; ++i) { pts.push_back(0.5 * (xa[i] + 1.0)); w.push_back(0.5 * wa[i]); }
    return;
  }
  gauss_jacobi(n, 1, 0, xb, wb);
  if (dim == 2) {
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double y = 0.5 * (1.0 + xb[j]);
        double x = 0.5 * (1.0 + xa[i]) * (1.0 - y);
        pts.push_back(x); pts.push_back(y);
        w.push_back(wa[i] * wb[j] / 8.0);
      }
    return;
  }
  gauss_jacobi(n, 2, 0, xc, wc);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int l = 0; l < n; ++l) {
        double z = 0.5 * (1.0 + xc[l]);
        double y = 0.5 * (1.0 + xb[j]) * (1.0 - z);
        double x = 0.5 * (1.0 + xa[i]) * (1.0 - y - z);
        pts.push_back(x); pts.push_back(y); pts.push_back(z);
        w.push_back(wa[i] * wb[j] * wc[l] / 64.0);
      }
}

void dubiner(int dim, int k, const double* pts, int np, double* val, double* grad) {
  const int Nb = n_modes(dim, k);
  for (int q = 0; q < np; ++q) {
    const double* P = pts + (size_t)q * dim;
    double* V = val + (size_t)q * Nb;
    double* G = grad ? grad + (size_t)q * Nb * dim : nullptr;
    int mode = 0;
    if (dim == 1) {
      double s = 2.0 * P[0] - 1.0;
      for (int i = 0; i <= k; ++i, ++mode) {
        double c = std::sqrt(2.0 * i + 1.0);
        V[mode] = c * jac(i, 0, 0, s);
        if (G) G[mode] = 2.0 * c * djac(i, 0, 0, s);
      }
    } else if (dim == 2) {
      double x = P[0], y = P[1];
      double om = 1.0 - y;                 // (1 - b)/2 with b = 2y - 1
      double a = 2.0 * x / om - 1.0, b = 2.0 * y - 1.0;
      for (int i = 0; i <= k; ++i)
        for (int j = 0; i + j <= k; ++j, ++mode) {
          double c = std::sqrt(2.0 * (2 * i + 1) * (i + j + 1));
          double Pa = jac(i, 0, 0, a), dPa = djac(i, 0, 0, a);
          double f1 = Pa * std::pow(om, i);
          double f1x = i > 0 ? 2.0 * dPa * std::pow(om, i - 1) : 0.0;
          double f1y = i > 0 ? std::pow(om, i - 1) * (dPa * (a + 1.0) - i * Pa) : 0.0;
          double f2 = jac(j, 2 * i + 1, 0, b), f2y = 2.0 * djac(j, 2 * i + 1, 0, b);
          V[mode] = c * f1 * f2;
          if (G) { G[mode * 2 + 0] = c * f1x * f2; G[mode * 2 + 1] = c * (f1y * f2 + f1 * f2y); }
        }
    } else {
      double x = P[0], y = P[1], z = P[2];
      double w1 = 1.0 - y - z, w2 = 1.0 - z;
      double a = 2.0 * x / w1 - 1.0, b = 2.0 * y / w2 - 1.0, cc = 2.0 * z - 1.0;
      for (int i = 0; i <= k; ++i)
        for (int j = 0; i + j <= k; ++j)
          for (int l = 0; i + j + l <= k; ++l, ++mode) {
            double c = std::sqrt((2.0 * i + 1) * (2.0 * i + 2 * j + 2) * (2.0 * i + 2 * j + 2 * l + 3));
            double Pa = jac(i, 0, 0, a), dPa = djac(i, 0, 0, a);
            double f1 = Pa * std::pow(w1, i);
            double f1x = i > 0 ? 2.0 * dPa * std::pow(w1, i - 1) : 0.0;
            double f1yz = i > 0 ? std::pow(w1, i - 1) * (dPa * (a + 1.0) - i * Pa) : 0.0;
            double Pb = jac(j, 2 * i + 1, 0, b), dPb = djac(j, 2 * i + 1, 0, b);
            double f2 = Pb * std::pow(w2, j);
            double f2y = j > 0 ? 2.0 * dPb * std::pow(w2, j - 1) : 0.0;
            double f2z = j > 0 ? std::pow(w2, j - 1) * (dPb * (b + 1.0) - j * Pb) : 0.0;
            double f3 = jac(l, 2 * i + 2 * j + 2, 0, cc), f3z = 2.0 * djac(l, 2 * i + 2 * j + 2, 0, cc);
            V[mode] = c * f1 * f2 * f3;
            if (G) {
              G[mode * 3 + 0] = c * f1x * f2 * f3;
              G[mode * 3 + 1] = c * (f1yz * f2 * f3 + f1 * f2y * f3);
              G[mode * 3 + 2] = c * (f1yz * f2 * f3 + f1 * f2z * f3 + f1 * f2 * f3z);
            }
          }
    }
  }
}

std::vector<int> face_mode_degrees(int dim, int kf) {
  std::vector<int> d;
  if (dim == 2) {
    for (int i = 0; i <= kf; ++i) d.push_back(i);
  } else {
    for (int i = 0; i <= kf; ++i)
      for (int j = 0; i + j <= kf; ++j) d.push_back(i + j);
  }
  return d;
}

RefTables build_tables(int dim, int k) { return build_tables_pair(dim, k, k); }

RefTables build_tables_pair(int dim, int k, int kf) {
  if (dim < 2 || dim > 3 || k < 1 || k > 4 || kf < k || kf > 4)
    throw std::invalid_argument("dim must be 2/3 and 1 <= k <= kf <= 4");
  RefTables T;
  T.dim = dim; T.k = k;
  const int Np = T.Np = n_modes(dim, k);
  const int Nf = T.Nf = n_modes(dim - 1, kf);
  const int nfc = dim + 1;
  const int kq = kf;   // kf >= k: rules exact for the face products of degree k + kf
  // volume rule and derivative matrices
  simplex_rule(dim, kq + 2, T.qv_pts, T.qv_w);
  const int nqv = T.nqv = (int)T.qv_w.size();
  T.qv_phi.resize((size_t)nqv * Np);
  std::vector<double> grad((size_t)nqv * Np * dim);
  dubiner(dim, k, T.qv_pts.data(), nqv, T.qv_phi.data(), grad.data());
  T.Dr.assign((size_t)dim * Np * Np, 0.0);
  for (int r = 0; r < dim; ++r)
    for (int i = 0; i < Np; ++i)
      for (int l = 0; l < Np; ++l) {
        double s = 0.0;
        for (int q = 0; q < nqv; ++q) s += T.qv_w[q] * grad[((size_t)q * Np + l) * dim + r] * T.qv_phi[(size_t)q * Np + i];
        T.Dr[((size_t)r * Np + i) * Np + l] = s;
      }
  // face rule and face-trace coupling: local face j has the reference vertices {0..d}\{j}
  simplex_rule(dim - 1, kq + 2, T.qf_pts, T.qf_w);
  const int nqf = T.nqf = (int)T.qf_w.size();
  T.qf_mu.resize((size_t)nqf * Nf);
  dubiner(dim - 1, kf, T.qf_pts.data(), nqf, T.qf_mu.data(), nullptr);
  T.Ff.assign((size_t)nfc * Np * Nf, 0.0);
  std::vector<double> vref((size_t)(dim + 1) * dim, 0.0);  // reference vertices
  for (int r = 0; r < dim; ++r) vref[(size_t)(r + 1) * dim + r] = 1.0;
  std::vector<double> xi((size_t)nqf * dim), phi((size_t)nqf * Np);
  for (int f = 0; f < nfc; ++f) {
    int fv[3], c = 0;
    for (int v = 0; v <= dim; ++v) if (v != f) fv[c++] = v;
    for (int q = 0; q < nqf; ++q)
      for (int r = 0; r < dim; ++r) {
        double s = vref[(size_t)fv[0] * dim + r];
        for (int e = 1; e < dim; ++e) s += T.qf_pts[(size_t)q * (dim - 1) + e - 1] * (vref[(size_t)fv[e] * dim + r] - vref[(size_t)fv[0] * dim + r]);
        xi[(size_t)q * dim + r] = s;
      }
    dubiner(dim, k, xi.data(), nqf, phi.data(), nullptr);
    for (int i = 0; i < Np; ++i)
      for (int mm = 0; mm < Nf; ++mm) {
        double s = 0.0;
        for (int q = 0; q < nqf; ++q) s += T.qf_w[q] * phi[(size_t)q * Np + i] * T.qf_mu[(size_t)q * Nf + mm];
        T.Ff[((size_t)f * Np + i) * Nf + mm] = s;
      }
  }
  // derived products
  T.Ef.assign((size_t)nfc * Np * Np, 0.0);
  for (int f = 0; f < nfc; ++f)
    for (int i = 0; i < Np; ++i)
      for (int l = 0; l < Np; ++l) {
        double s = 0.0;
        for (int mm = 0; mm < Nf; ++mm) s += T.Ff[((size_t)f * Np + i) * Nf + mm] * T.Ff[((size_t)f * Np + l) * Nf + mm];
        T.Ef[((size_t)f * Np + i) * Np + l] = s;
      }
  T.Trs.assign((size_t)dim * dim * Np * Np, 0.0);
  for (int r = 0; r < dim; ++r)
    for (int s2 = 0; s2 < dim; ++s2)
      for (int i = 0; i < Np; ++i)
        for (int l = 0; l < Np; ++l) {
          double s = 0.0;
          for (int q = 0; q < Np; ++q) s += T.Dr[((size_t)r * Np + i) * Np + q] * T.Dr[((size_t)s2 * Np + l) * Np + q];
          T.Trs[(((size_t)r * dim + s2) * Np + i) * Np + l] = s;
        }
  T.DFrf.assign((size_t)dim * nfc * Np * Nf, 0.0);
  for (int r = 0; r < dim; ++r)
    for (int f = 0; f < nfc; ++f)
      for (int i = 0; i < Np; ++i)
        for (int mm = 0; mm < Nf; ++mm) {
          double s = 0.0;
          for (int q = 0; q < Np; ++q) s += T.Dr[((size_t)r * Np + i) * Np + q] * T.Ff[((size_t)f * Np + q) * Nf + mm];
          T.DFrf[(((size_t)r * nfc + f) * Np + i) * Nf + mm] = s;
        }
  T.Pfg.assign((size_t)nfc * nfc * Nf * Nf, 0.0);
  for (int f = 0; f < nfc; ++f)
    for (int g = 0; g < nfc; ++g)
      for (int a = 0; a < Nf; ++a)
        for (int b = 0; b < Nf; ++b) {
          double s = 0.0;
          for (int i = 0; i < Np; ++i) s += T.Ff[((size_t)f * Np + i) * Nf + a] * T.Ff[((size_t)g * Np + i) * Nf + b];
          T.Pfg[(((size_t)f * nfc + g) * Nf + a) * Nf + b] = s;
        }
  return T;
}

PostTables build_post_tables(int dim, int k) {
  if (dim < 2 || dim > 3 || k < 1 || k > 4) throw std::invalid_argument("dim must be 2/3 and 1 <= k <= 4");
  PostTables T;
  T.dim = dim; T.k = k;
  const int Np = T.Np = n_modes(dim, k), Np1 = T.Np1 = n_modes(dim, k + 1);
  std::vector<double> pts, w;
  simplex_rule(dim, k + 3, pts, w);
  const int nq = (int)w.size();
  std::vector<double> phi((size_t)nq * Np), psi((size_t)nq * Np1), dpsi((size_t)nq * Np1 * dim);
  dubiner(dim, k, pts.data(), nq, phi.data(), nullptr);
  dubiner(dim, k + 1, pts.data(), nq, psi.data(), dpsi.data());
  double c00 = 0.0;
  for (int q = 0; q < nq; ++q) c00 += w[q] * psi[(size_t)q * Np1] * phi[(size_t)q * Np];
  if (std::fabs(c00 - 1.0) > 1e-12) throw std::logic_error("constant modes of degrees k and k+1 differ");
  T.K1.assign((size_t)dim * dim * Np1 * Np1, 0.0);
  for (int r = 0; r < dim; ++r)
    for (int s2 = 0; s2 < dim; ++s2)
      for (int i = 0; i < Np1; ++i)
        for (int l = 0; l < Np1; ++l) {
          double s = 0.0;
          for (int q = 0; q < nq; ++q)
            s += w[q] * dpsi[((size_t)q * Np1 + i) * dim + r] * dpsi[((size_t)q * Np1 + l) * dim + s2];
          T.K1[(((size_t)r * dim + s2) * Np1 + i) * Np1 + l] = s;
        }
  T.E1.assign((size_t)dim * Np1 * Np, 0.0);
  for (int r = 0; r < dim; ++r)
    for (int i = 0; i < Np1; ++i)
      for (int l = 0; l < Np; ++l) {
        double s = 0.0;
        for (int q = 0; q < nq; ++q) s += w[q] * dpsi[((size_t)q * Np1 + i) * dim + r] * phi[(size_t)q * Np + l];
        T.E1[((size_t)r * Np1 + i) * Np + l] = s;
      }
  return T;
}

std::vector<double> face_nodal_to_modal(int dim, int k) {
  if (dim < 2 || dim > 3 || k < 1 || k > 4) throw std::invalid_argument("dim must be 2/3 and 1 <= k <= 4");
  const int fd = dim - 1, nf = n_modes(fd, k);
  // nodes and monomial exponents, both in lexicographic order
  std::vector<std::array<int, 2>> nodes, expo;
  for (int b0 = 0; b0 <= k; ++b0)
    if (fd == 1) nodes.push_back({k - b0, 0});
    else for (int b1 = 0; b0 + b1 <= k; ++b1) nodes.push_back({b1, k - b0 - b1});
  for (int i = 0; i <= k; ++i)
    for (int j = 0; (fd == 2 ? i + j : j) <= (fd == 2 ? k : 0); ++j) expo.push_back({i, j});
  auto mono = [&](const double* x, int m) {
    double v = std::pow(x[0], expo[m][0]);
    if (fd == 2) v *= std::pow(x[1], expo[m][1]);
    return v;
  };
  // W[a][m] = x_a^m at the nodes; invert by Gauss-Jordan with partial pivoting
  std::vector<double> W((size_t)nf * nf), Wi((size_t)nf * nf, 0.0);
  for (int a = 0; a < nf; ++a) {
    const double x[2] = {nodes[a][0] / (double)k, nodes[a][1] / (double)k};
    for (int m = 0; m < nf; ++m) W[(size_t)a * nf + m] = mono(x, m);
    Wi[(size_t)a * nf + a] = 1.0;
  }
  for (int c = 0; c < nf; ++c) {
    int piv = c;
    for (int r = c + 1; r < nf; ++r)
      if (std::fabs(W[(size_t)r * nf + c]) > std::fabs(W[(size_t)piv * nf + c])) piv = r;
    for (int j = 0; j < nf; ++j) {
      std::swap(W[(size_t)c * nf + j], W[(size_t)piv * nf + j]);
      std::swap(Wi[(size_t)c * nf + j], Wi[(size_t)piv * nf + j]);
    }
    const double d = W[(size_t)c * nf + c];
    if (std::fabs(d) < 1e-14) throw std::logic_error("face nodes are not unisolvent");
    for (int j = 0; j < nf; ++j) { W[(size_t)c * nf + j] /= d; Wi[(size_t)c * nf + j] /= d; }
    for (int r = 0; r < nf; ++r) {
      if (r == c) continue;
      const double f = W[(size_t)r * nf + c];
      if (f == 0.0) continue;
      for (int j = 0; j < nf; ++j) { W[(size_t)r * nf + j] -= f * W[(size_t)c * nf + j]; Wi[(size_t)r * nf + j] -= f * Wi[(size_t)c * nf + j]; }
    }
  }
  // Lagrange functions at a face rule, projected on the orthonormal basis
  std::vector<double> pts, w;
  simplex_rule(fd, k + 2, pts, w);
  const int nq = (int)w.size();
  std::vector<double> U((size_t)nq * nf);
  dubiner(fd, k, pts.data(), nq, U.data(), nullptr);
  std::vector<double> out((size_t)nf * nf, 0.0);
  for (int q = 0; q < nq; ++q) {
    std::vector<double> mq(nf);
    for (int m = 0; m < nf; ++m) mq[m] = mono(&pts[(size_t)q * fd], m);
    for (int a = 0; a < nf; ++a) {
      double ell = 0.0;   // ell_a(x_q) = sum_m x_q^m (W^{-1})[m][a]
      for (int m = 0; m < nf; ++m) ell += mq[m] * Wi[(size_t)m * nf + a];
      for (int mm = 0; mm < nf; ++mm) out[(size_t)mm * nf + a] += w[q] * U[(size_t)q * nf + mm] * ell;
    }
  }
  return out;
}

}  // namespace hdg
