// Reference-simplex integrals of the P2 velocity / P1 pressure bases
// (Sec. 2.3), computed exactly on the host.
//
// Every basis function is a polynomial in the barycentric coordinates
// lam_0..lam_d of the reference simplex (lam_0 = 1 - sum xi, lam_i = xi_i).
// Products of such polynomials are integrated with the closed form
//     int_ref lam_0^a0 ... lam_d^ad dxi = a0! ... ad! / (a0 + ... + ad + d)!
// so the tables carry no quadrature error.  A derivative d/dxi_i of a
// barycentric polynomial is d/dlam_i - d/dlam_0 (chain rule).
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

}  // namespace

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
