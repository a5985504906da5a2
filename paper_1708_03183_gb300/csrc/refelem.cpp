// Reference-element matrices of the nodal P_p basis used by the CUDA executor.
//
// Basis: Lagrange functions on the equispaced points (i/p, j/p) of the reference triangle
// (0,0), (1,0), (0,1), j outer, i inner.  Computed here with floating-point quadrature:
// the Vandermonde matrix of the monomials r^a s^b at the nodes is inverted by Gauss-Jordan
// elimination with partial pivoting; the mass matrix uses a collapsed (Duffy) Gauss-Legendre
// rule on the triangle, exact for the degree-2p integrand; face integrals use Gauss-Legendre
// on [0, 1].  Face f runs from local vertex f to local vertex f+1 (mod 3).
//
// Nodal strong form: the volume terms need only the differentiation matrices Dr, Ds
// (Dr[i][j] = d phi_j / dr at node i): the divergence / gradient of a degree-p field is
// represented exactly at the nodes, so the inverse mass matrix cancels.  The facet terms need
// Lift_f = M^-1 E_f, E_f[i][k] = int_0^1 phi_i(face f, t) phi_{face node k}(face f, t) dt.
#include <cmath>
#include <string>
#include <vector>

#include "internal.h"

namespace slt {

namespace {

// Gauss-Legendre points and weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      // p1 = P_n(z), p0 = P_{n-1}(z)
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = pk;
    }
    double dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

std::vector<double> invert(std::vector<double> A, int n) {
  std::vector<double> I(n * n, 0.0);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) fail(SLT_ERR_ARG, "singular reference matrix");
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(A[c * n + k], A[piv * n + k]);
        std::swap(I[c * n + k], I[piv * n + k]);
      }
    double d = A[c * n + c];
    for (int k = 0; k < n; ++k) { A[c * n + k] /= d; I[c * n + k] /= d; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = A[r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) { A[r * n + k] -= f * A[c * n + k]; I[r * n + k] -= f * I[c * n + k]; }
    }
  }
  return I;
}

double ipow(double x, int k) {
  double r = 1.0;
  for (int i = 0; i < k; ++i) r *= x;
  return r;
}

}  // namespace

std::vector<double> RefElem::eval(double r, double s) const {
  int nm = (int)mono.size() / 2;
  std::vector<double> phi(Np, 0.0);
  for (int m = 0; m < nm; ++m) {
    double t = ipow(r, mono[2 * m]) * ipow(s, mono[2 * m + 1]);
    for (int j = 0; j < Np; ++j) phi[j] += Vinv[m * Np + j] * t;
  }
  return phi;
}

RefElem make_refelem(int p) {
  if (p < 1 || p > 4) fail(SLT_ERR_ARG, "degree must be in 1..4");
  RefElem R;
  R.p = p;
  R.Np = (p + 1) * (p + 2) / 2;
  R.Nfp = p + 1;
  const int Np = R.Np, Nfp = R.Nfp;
  for (int j = 0; j <= p; ++j)
    for (int i = 0; i <= p - j; ++i) {
      R.nodes.push_back(double(i) / p);
      R.nodes.push_back(double(j) / p);
    }
  for (int d = 0; d <= p; ++d)
    for (int a = 0; a <= d; ++a) {
      R.mono.push_back(a);
      R.mono.push_back(d - a);
    }
  // V[i][m] = monomial m at node i; basis coefficients C = V^-1 (V C = I)
  std::vector<double> V(Np * Np);
  for (int i = 0; i < Np; ++i)
    for (int m = 0; m < Np; ++m)
      V[i * Np + m] = ipow(R.nodes[2 * i], R.mono[2 * m]) * ipow(R.nodes[2 * i + 1], R.mono[2 * m + 1]);
  R.Vinv = invert(V, Np);
  // derivative matrices at the nodes
  R.Dr.assign(Np * Np, 0.0);
  R.Ds.assign(Np * Np, 0.0);
  for (int i = 0; i < Np; ++i) {
    double r = R.nodes[2 * i], s = R.nodes[2 * i + 1];
    for (int m = 0; m < Np; ++m) {
      int a = R.mono[2 * m], b = R.mono[2 * m + 1];
      double dr = a ? a * ipow(r, a - 1) * ipow(s, b) : 0.0;
      double ds = b ? b * ipow(r, a) * ipow(s, b - 1) : 0.0;
      for (int j = 0; j < Np; ++j) {
        R.Dr[i * Np + j] += R.Vinv[m * Np + j] * dr;
        R.Ds[i * Np + j] += R.Vinv[m * Np + j] * ds;
      }
    }
  }
  // mass matrix by a collapsed Gauss-Legendre rule: r = (1+x)(1-y)/4, s = (1+y)/2
  std::vector<double> gx, gw;
  gauss_legendre(p + 2, gx, gw);
  std::vector<double> M(Np * Np, 0.0);
  for (int a = 0; a < p + 2; ++a)
    for (int b = 0; b < p + 2; ++b) {
      double r = (1.0 + gx[a]) * (1.0 - gx[b]) / 4.0, s = (1.0 + gx[b]) / 2.0;
      double w = gw[a] * gw[b] * (1.0 - gx[b]) / 8.0;
      std::vector<double> phi = R.eval(r, s);
      for (int i = 0; i < Np; ++i)
        for (int j = 0; j < Np; ++j) M[i * Np + j] += w * phi[i] * phi[j];
    }
  R.Minv = invert(M, Np);
  // face nodes: face 0 (k, 0), face 1 (p-k, k), face 2 (0, p-k), k = 0..p
  auto nidx = [p](int i, int j) { return j * (p + 1) - j * (j - 1) / 2 + i; };
  R.fnode.resize(3 * Nfp);
  for (int k = 0; k <= p; ++k) {
    R.fnode[0 * Nfp + k] = nidx(k, 0);
    R.fnode[1 * Nfp + k] = nidx(p - k, k);
    R.fnode[2 * Nfp + k] = nidx(0, p - k);
  }
  // face matrices E_f and lifts M^-1 E_f
  static const double org[3][2] = {{0, 0}, {1, 0}, {0, 1}};
  static const double dir[3][2] = {{1, 0}, {-1, 1}, {0, -1}};
  R.Lift.assign(3 * Np * Nfp, 0.0);
  for (int f = 0; f < 3; ++f) {
    std::vector<double> E(Np * Nfp, 0.0);
    for (int q = 0; q < p + 2; ++q) {
      double t = 0.5 * (gx[q] + 1.0), w = 0.5 * gw[q];
      std::vector<double> phi = R.eval(org[f][0] + t * dir[f][0], org[f][1] + t * dir[f][1]);
      for (int i = 0; i < Np; ++i)
        for (int k = 0; k < Nfp; ++k) E[i * Nfp + k] += w * phi[i] * phi[R.fnode[f * Nfp + k]];
    }
    for (int i = 0; i < Np; ++i)
      for (int k = 0; k < Nfp; ++k) {
        double acc = 0.0;
        for (int l = 0; l < Np; ++l) acc += R.Minv[i * Np + l] * E[l * Nfp + k];
        R.Lift[(f * Np + i) * Nfp + k] = acc;
      }
  }
  return R;
}

}  // namespace slt
