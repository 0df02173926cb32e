// Reference-simplex integrals of the P2 velocity / P1 pressure bases
// (Sec. 2.3), computed exactly on the host.
//
// Every basis function is a polynomial in the barycentric coordinates
// lam_0..lam_d of the reference simplex (lam_0 = 1 - sum xi, lam_i = xi_i).
// Products of such polynomials are integrated with the closed form
//     int_ref lam_0^a0 ... lam_d^ad dxi = a0! ... ad! / (a0 + ... + ad + d)!
// so the tables carry no quadrature error.  A derivative d/dxi_i of a
// barycentric polynomial is d/dlam_i - d/dlam_0 (chain rule).
#include <cmath>
#include <map>
#include <array>
#include <vector>
#include <cstring>
#include "common.cuh"

namespace scvs {
namespace {

using Mono = std::array<int, 4>;
using Poly = std::map<Mono, double>;

Poly lam(int i) { Mono m{0, 0, 0, 0}; m[i] = 1; return Poly{{m, 1.0}}; }
Poly constant(double c) { return Poly{{Mono{0, 0, 0, 0}, c}}; }

Poly add(const Poly &a, const Poly &b, double sb = 1.0) {
  Poly r = a;
  for (auto &kv : b) r[kv.first] += sb * kv.second;
  return r;
}
Poly mul(const Poly &a, const Poly &b) {
  Poly r;
  for (auto &x : a)
    for (auto &y : b) {
      Mono m;
      for (int i = 0; i < 4; ++i) m[i] = x.first[i] + y.first[i];
      r[m] += x.second * y.second;
    }
  return r;
}
Poly scale(const Poly &a, double s) { Poly r; for (auto &kv : a) r[kv.first] = s * kv.second; return r; }
Poly dlam(const Poly &a, int v) {
  Poly r;
  for (auto &kv : a) {
    if (kv.first[v] == 0) continue;
    Mono m = kv.first;
    double c = kv.second * m[v];
    m[v] -= 1;
    r[m] += c;
  }
  return r;
}
// d/dxi_i (i = 0..d-1) of a polynomial in lam_0..lam_d
Poly dxi(const Poly &a, int i) { return add(dlam(a, i + 1), dlam(a, 0), -1.0); }

double fact(int n) { double f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; }
double integrate(const Poly &a, int dim) {
  double s = 0;
  for (auto &kv : a) {
    int tot = 0;
    double num = 1;
    for (int i = 0; i <= dim; ++i) { tot += kv.first[i]; num *= fact(kv.first[i]); }
    s += kv.second * num / fact(tot + dim);
  }
  return s;
}

void bases(int dim, std::vector<Poly> &p2, std::vector<Poly> &p1) {
  static const int E2[3][2] = {{0, 1}, {1, 2}, {2, 0}};
  static const int E3[6][2] = {{0, 1}, {1, 2}, {2, 0}, {0, 3}, {1, 3}, {2, 3}};
  p2.clear(); p1.clear();
  for (int a = 0; a <= dim; ++a) {
    p2.push_back(add(scale(mul(lam(a), lam(a)), 2.0), lam(a), -1.0));  // lam(2 lam - 1)
    p1.push_back(lam(a));
  }
  int ne = dim == 2 ? 3 : 6;
  for (int e = 0; e < ne; ++e) {
    int a = dim == 2 ? E2[e][0] : E3[e][0];
    int b = dim == 2 ? E2[e][1] : E3[e][1];
    p2.push_back(scale(mul(lam(a), lam(b)), 4.0));
  }
}

double evaluate(const Poly &a, const double *lam) {
  double s = 0;
  for (auto &kv : a) {
    double t = kv.second;
    for (int i = 0; i < 4; ++i)
      for (int q = 0; q < kv.first[i]; ++q) t *= lam[i];
    s += t;
  }
  return s;
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_n
// (three-term recurrence), started from the Tricomi-type estimate
// cos(pi (i - 1/4) / (n + 1/2)).
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

}  // namespace

// Quadrature of curved (isoparametric) elements: the collapsed (Duffy)
// product Gauss-Legendre rule with n points per direction on the reference
// simplex (triangle: xi = u, eta = v (1 - u), weight (1 - u); tet: zeta = t (1
// - u)(1 - v), weight (1 - u)^2 (1 - v)), with the P2 basis, its reference
// gradients and the P1 basis at every point.
void quad_tables(int dim, int n, QuadTables *out) {
  std::vector<double> g, wg;
  gauss_legendre(n, g, wg);
  for (int i = 0; i < n; ++i) { g[i] = 0.5 * (g[i] + 1.0); wg[i] *= 0.5; }
  std::vector<Poly> p2, p1;
  bases(dim, p2, p1);
  const int nl = (int)p2.size(), nv = (int)p1.size();
  std::vector<std::vector<Poly>> d2(nl);
  for (int a = 0; a < nl; ++a)
    for (int i = 0; i < dim; ++i) d2[a].push_back(dxi(p2[a], i));
  out->dim = dim;
  out->nq = 0;
  const int n3 = dim == 3 ? n : 1;
  for (int iu = 0; iu < n; ++iu)
    for (int iv = 0; iv < n; ++iv)
      for (int it = 0; it < n3; ++it) {
        const double u = g[iu], v = g[iv], t = dim == 3 ? g[it] : 0.0;
        double xi[3] = {u, v * (1.0 - u), dim == 3 ? t * (1.0 - u) * (1.0 - v) : 0.0};
        double w = wg[iu] * wg[iv] * (dim == 3 ? wg[it] * (1.0 - u) * (1.0 - u) * (1.0 - v) : (1.0 - u));
        double lm[4] = {1.0 - xi[0] - xi[1] - xi[2], xi[0], xi[1], xi[2]};
        const int q = out->nq++;
        out->w[q] = w;
        for (int a = 0; a < nl; ++a) {
          out->phi[q][a] = evaluate(p2[a], lm);
          for (int i = 0; i < dim; ++i) out->dphi[q][a][i] = evaluate(d2[a][i], lm);
        }
        for (int b = 0; b < nv; ++b) out->psi[q][b] = evaluate(p1[b], lm);
      }
}

// Mass matrix M[a][b] = int phi_a phi_b dGamma of one isoparametric P2 face
// (fdim = 1: segment, nodes (end, end, middle); fdim = 2: triangle in face VTK
// order) with node coordinates X [nfl][dim]: the face map x(xi) = sum_a x_a
// phi_a(xi), surface Jacobian |dx/dxi| or |dx/dxi_1 x dx/dxi_2|, and the
// collapsed Gauss-Legendre rule with n points per direction.
void face_mass_iso(int fdim, int dim, int n, const double *X, double *M) {
  std::vector<double> g, wg;
  gauss_legendre(n, g, wg);
  for (int i = 0; i < n; ++i) { g[i] = 0.5 * (g[i] + 1.0); wg[i] *= 0.5; }
  const int nfl = fdim == 1 ? 3 : 6;
  for (int i = 0; i < nfl * nfl; ++i) M[i] = 0.0;
  static const int FE[3][2] = {{0, 1}, {1, 2}, {2, 0}};
  const double dl[3][2] = {{-1.0, -1.0}, {1.0, 0.0}, {0.0, 1.0}};  // grad of lam_0..2 (triangle)
  const int nj = fdim == 1 ? 1 : n;
  for (int iu = 0; iu < n; ++iu)
    for (int iv = 0; iv < nj; ++iv) {
      double phi[6], dphi[6][2] = {{0}};
      double w;
      if (fdim == 1) {
        const double t = g[iu], l0 = 1.0 - t, l1 = t;
        w = wg[iu];
        phi[0] = l0 * (2 * l0 - 1); phi[1] = l1 * (2 * l1 - 1); phi[2] = 4 * l0 * l1;
        dphi[0][0] = -(4 * l0 - 1); dphi[1][0] = 4 * l1 - 1; dphi[2][0] = 4 * (l0 - l1);
      } else {
        const double u = g[iu], v = g[iv] * (1.0 - u);
        w = wg[iu] * wg[iv] * (1.0 - u);
        const double lm[3] = {1.0 - u - v, u, v};
        for (int a = 0; a < 3; ++a) {
          phi[a] = lm[a] * (2 * lm[a] - 1);
          for (int i = 0; i < 2; ++i) dphi[a][i] = (4 * lm[a] - 1) * dl[a][i];
        }
        for (int e = 0; e < 3; ++e) {
          const int a = FE[e][0], b = FE[e][1];
          phi[3 + e] = 4 * lm[a] * lm[b];
          for (int i = 0; i < 2; ++i) dphi[3 + e][i] = 4 * (lm[a] * dl[b][i] + lm[b] * dl[a][i]);
        }
      }
      double T[2][3] = {{0}};
      for (int i = 0; i < fdim; ++i)
        for (int r = 0; r < dim; ++r)
          for (int a = 0; a < nfl; ++a) T[i][r] += X[a * dim + r] * dphi[a][i];
      double js;
      if (fdim == 1) {
        js = 0;
        for (int r = 0; r < dim; ++r) js += T[0][r] * T[0][r];
        js = std::sqrt(js);
      } else {
        const double cx = T[0][1] * T[1][2] - T[0][2] * T[1][1];
        const double cy = T[0][2] * T[1][0] - T[0][0] * T[1][2];
        const double cz = T[0][0] * T[1][1] - T[0][1] * T[1][0];
        js = std::sqrt(cx * cx + cy * cy + cz * cz);
      }
      for (int a = 0; a < nfl; ++a)
        for (int b = 0; b < nfl; ++b) M[a * nfl + b] += w * js * phi[a] * phi[b];
    }
}

void reference_tables(int dim, RefTables *t) {
  std::memset(t, 0, sizeof(*t));
  std::vector<Poly> p2, p1;
  bases(dim, p2, p1);
  const int nl = (int)p2.size(), nv = (int)p1.size();
  std::vector<std::vector<Poly>> d2(nl), d1(nv);
  for (int a = 0; a < nl; ++a)
    for (int i = 0; i < dim; ++i) d2[a].push_back(dxi(p2[a], i));
  for (int a = 0; a < nv; ++a)
    for (int i = 0; i < dim; ++i) d1[a].push_back(dxi(p1[a], i));
  for (int a = 0; a < nl; ++a)
    for (int b = 0; b < nl; ++b) {
      t->mref[a][b] = integrate(mul(p2[a], p2[b]), dim);
      int p = 0;
      for (int i = 0; i < dim; ++i)
        for (int j = i; j < dim; ++j, ++p) {
          double v = integrate(mul(d2[a][i], d2[b][j]), dim);
          if (i != j) v += integrate(mul(d2[a][j], d2[b][i]), dim);
          t->ksym[p][a][b] = v;
        }
    }
  for (int i = 0; i < dim; ++i)
    for (int a = 0; a < nl; ++a)
      for (int b = 0; b < nv; ++b) t->eref[i][a][b] = integrate(mul(d2[a][i], p1[b]), dim);
  for (int a = 0; a < nv; ++a)
    for (int b = 0; b < nv; ++b) {
      t->m1[a][b] = integrate(mul(p1[a], p1[b]), dim);
      int p = 0;
      for (int i = 0; i < dim; ++i)
        for (int j = i; j < dim; ++j, ++p) {
          double v = integrate(mul(d1[a][i], d1[b][j]), dim);
          if (i != j) v += integrate(mul(d1[a][j], d1[b][i]), dim);
          t->k1sym[p][a][b] = v;
        }
    }
}

}  // namespace scvs
