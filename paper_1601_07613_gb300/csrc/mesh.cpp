// Host side of the library: quadrature and basis tables, mesh ingest and
// geometry, the edge coloring of Sec. 3.1 and the reordering of Sec. 5.
//
// Everything here runs once per mesh on the host (the paper's "mesh
// preprocessing stage", Sec. 5); the per-step work is in kernels_tri.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>
#include <stdexcept>

#include "dgc_internal.h"

namespace dgc {

// ---------------------------------------------------------------------------
// Jacobi polynomials and Gauss-Jacobi rules
// ---------------------------------------------------------------------------

// P_n^{(a,b)}(x) by the three-term recurrence in n.
static double jacobi(int n, double a, double b, double x) {
  if (n == 0) return 1.0;
  double pm = 1.0, p = 0.5 * ((a - b) + (a + b + 2.0) * x);
  for (int k = 2; k <= n; ++k) {
    double s = 2.0 * k + a + b;
    double c1 = 2.0 * k * (k + a + b) * (s - 2.0);
    double c2 = (s - 1.0) * (s * (s - 2.0) * x + a * a - b * b);
    double c3 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * s;
    double pn = (c2 * p - c3 * pm) / c1;
    pm = p;
    p = pn;
  }
  return p;
}

// d/dx P_n^{(a,b)} = (n+a+b+1)/2 P_{n-1}^{(a+1,b+1)}.
static double djacobi(int n, double a, double b, double x) {
  return n == 0 ? 0.0 : 0.5 * (n + a + b + 1.0) * jacobi(n - 1, a + 1.0, b + 1.0, x);
}

// Newton iteration with polynomial deflation from Chebyshev starting points;
// weights from the Christoffel formula for beta = 0.
void gauss_jacobi(int n, double alpha, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    double r = -std::cos((2.0 * k + 1.0) * pi / (2.0 * n));
    if (k > 0) r = 0.5 * (r + x[k - 1]);
    for (int it = 0; it < 100; ++it) {
      double s = 0.0;
      for (int i = 0; i < k; ++i) s += 1.0 / (r - x[i]);
      double P = jacobi(n, alpha, 0.0, r), dP = djacobi(n, alpha, 0.0, r);
      double delta = -P / (dP - s * P);
      r += delta;
      if (std::fabs(delta) < 1e-16) break;
    }
    x[k] = r;
  }
  std::sort(x, x + n);
  double cst = std::exp((alpha + 1.0) * std::log(2.0) + std::lgamma(n + alpha + 1.0) +
                        std::lgamma(n + 1.0) - std::lgamma(n + alpha + 1.0) - std::lgamma(n + 1.0));
  for (int i = 0; i < n; ++i) {
    double d = djacobi(n, alpha, 0.0, x[i]);
    w[i] = cst / ((1.0 - x[i] * x[i]) * d * d);
  }
}

// ---------------------------------------------------------------------------
// Orthonormal modal basis (the v_ij of Eq. 2): Dubiner polynomials in
// collapsed coordinates, normalised numerically on the reference element.
// Ordering: total degree d = 0..p, first index from d down to 0.
// ---------------------------------------------------------------------------

static int npoly(int dim, int p, bool quad = false) {
  if (quad) return (p + 1) * (p + 1);
  return dim == 2 ? (p + 1) * (p + 2) / 2 : (p + 1) * (p + 2) * (p + 3) / 6;
}

// Unnormalised quadrilateral modes psi_{a,b} = P_a(2r-1) P_b(2s-1) on the
// square [0,1]^2, mode a (p+1) + b, with their gradients.
static void quad_raw(int p, double r, double s, double* phi, double* dr, double* ds) {
  double Pr[16], Ps[16], dPr[16], dPs[16];
  for (int k = 0; k <= p; ++k) {
    Pr[k] = jacobi(k, 0, 0, 2.0 * r - 1.0);
    Ps[k] = jacobi(k, 0, 0, 2.0 * s - 1.0);
    dPr[k] = 2.0 * djacobi(k, 0, 0, 2.0 * r - 1.0);
    dPs[k] = 2.0 * djacobi(k, 0, 0, 2.0 * s - 1.0);
  }
  for (int a = 0; a <= p; ++a)
    for (int b = 0; b <= p; ++b) {
      const int j = a * (p + 1) + b;
      phi[j] = Pr[a] * Ps[b];
      if (dr) {
        dr[j] = dPr[a] * Ps[b];
        ds[j] = Pr[a] * dPs[b];
      }
    }
}

// Square rule: n x n Gauss-Legendre points on [0,1]^2, weights summing to 1.
static void quad_rule(int n, std::vector<double>& r, std::vector<double>& s, std::vector<double>& w) {
  std::vector<double> xg(n), wg(n);
  gauss_jacobi(n, 0.0, xg.data(), wg.data());
  r.clear();
  s.clear();
  w.clear();
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      r.push_back(0.5 * (1.0 + xg[i]));
      s.push_back(0.5 * (1.0 + xg[k]));
      w.push_back(0.25 * wg[i] * wg[k]);
    }
}

// Unnormalised triangle modes psi_{k,l} = P_k(a) (1-s)^k P_l^{(2k+1,0)}(b),
// a = 2r/(1-s) - 1, b = 2s - 1, with gradients by the chain rule.
static void tri_raw(int p, double r, double s, double* phi, double* dr, double* ds) {
  double om = 1.0 - s;
  double a = om > 0.0 ? 2.0 * r / om - 1.0 : -1.0;
  double b = 2.0 * s - 1.0;
  int j = 0;
  for (int d = 0; d <= p; ++d)
    for (int k = d; k >= 0; --k) {
      int l = d - k;
      double Pk = jacobi(k, 0, 0, a), dPk = djacobi(k, 0, 0, a);
      double Pl = jacobi(l, 2.0 * k + 1.0, 0, b), dPl = djacobi(l, 2.0 * k + 1.0, 0, b);
      double omk = std::pow(om, k), omk1 = k > 0 ? std::pow(om, k - 1) : 0.0;
      phi[j] = Pk * omk * Pl;
      if (dr) {
        dr[j] = k > 0 ? 2.0 * dPk * omk1 * Pl : 0.0;
        ds[j] = (k > 0 ? (dPk * (1.0 + a) - k * Pk) * omk1 * Pl : 0.0) + 2.0 * Pk * omk * dPl;
      }
      ++j;
    }
}

// Unnormalised tetrahedron modes
// psi_{i,j,k} = P_i(a) ((1-b)/2)^i P_j^{(2i+1,0)}(b) ((1-c)/2)^{i+j} P_k^{(2i+2j+2,0)}(c),
// a = 2r/(1-s-t) - 1, b = 2s/(1-t) - 1, c = 2t - 1; gradients by the chain rule.
static void tet_raw(int p, double r, double s, double t, double* phi, double* g) {
  double u = 1.0 - s - t, v = 1.0 - t;
  double a = u > 0.0 ? 2.0 * r / u - 1.0 : -1.0;
  double b = v > 0.0 ? 2.0 * s / v - 1.0 : -1.0;
  double c = 2.0 * t - 1.0;
  // partial derivatives of (a, b, c) w.r.t. (r, s, t)
  double da[3] = {u > 0 ? 2.0 / u : 0.0, u > 0 ? 2.0 * r / (u * u) : 0.0, u > 0 ? 2.0 * r / (u * u) : 0.0};
  double db[3] = {0.0, v > 0 ? 2.0 / v : 0.0, v > 0 ? 2.0 * s / (v * v) : 0.0};
  double dc[3] = {0.0, 0.0, 2.0};
  int n = 0;
  for (int d = 0; d <= p; ++d)
    for (int i = d; i >= 0; --i)
      for (int j = d - i; j >= 0; --j) {
        int k = d - i - j;
        double A = jacobi(i, 0, 0, a), dA = djacobi(i, 0, 0, a);
        double hb = 0.5 * (1.0 - b), hc = 0.5 * (1.0 - c);
        double B0 = std::pow(hb, i), B1 = jacobi(j, 2.0 * i + 1.0, 0, b);
        double dB = (i > 0 ? -0.5 * i * std::pow(hb, i - 1) : 0.0) * B1 + B0 * djacobi(j, 2.0 * i + 1.0, 0, b);
        double Bv = B0 * B1;
        double C0 = std::pow(hc, i + j), C1 = jacobi(k, 2.0 * i + 2.0 * j + 2.0, 0, c);
        double dC = (i + j > 0 ? -0.5 * (i + j) * std::pow(hc, i + j - 1) : 0.0) * C1 +
                    C0 * djacobi(k, 2.0 * i + 2.0 * j + 2.0, 0, c);
        double Cv = C0 * C1;
        phi[n] = A * Bv * Cv;
        if (g) {
          int np = npoly(3, p);
          for (int x = 0; x < 3; ++x)
            g[x * np + n] = dA * da[x] * Bv * Cv + A * dB * db[x] * Cv + A * Bv * dC * dc[x];
        }
        ++n;
      }
}

// Triangle rule: Gauss-Legendre (n) x Gauss-Jacobi(1,0) (n), collapsed.
static void tri_rule(int n, std::vector<double>& r, std::vector<double>& s, std::vector<double>& w) {
  std::vector<double> xg(n), wg(n), xj(n), wj(n);
  gauss_jacobi(n, 0.0, xg.data(), wg.data());
  gauss_jacobi(n, 1.0, xj.data(), wj.data());
  r.clear();
  s.clear();
  w.clear();
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      r.push_back(0.25 * (1.0 + xg[k]) * (1.0 - xj[i]));
      s.push_back(0.5 * (1.0 + xj[i]));
      w.push_back(0.125 * wg[k] * wj[i]);
    }
}

static void tet_rule(int n, std::vector<double>& r, std::vector<double>& s, std::vector<double>& t,
                     std::vector<double>& w) {
  std::vector<double> xa(n), wa(n), xb(n), wb(n), xc(n), wc(n);
  gauss_jacobi(n, 0.0, xa.data(), wa.data());
  gauss_jacobi(n, 1.0, xb.data(), wb.data());
  gauss_jacobi(n, 2.0, xc.data(), wc.data());
  r.clear();
  s.clear();
  t.clear();
  w.clear();
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        t.push_back(0.5 * (1.0 + xc[i]));
        s.push_back(0.25 * (1.0 + xb[j]) * (1.0 - xc[i]));
        r.push_back(0.125 * (1.0 + xa[k]) * (1.0 - xb[j]) * (1.0 - xc[i]));
        w.push_back(wa[k] * wb[j] * wc[i] / 64.0);
      }
}

// normalisation constants, cached per (dim, p, quad)
static std::vector<double> norms(int dim, int p, bool quad) {
  int np = npoly(dim, p, quad);
  std::vector<double> acc(np, 0.0), phi(np);
  std::vector<double> r, s, t, w;
  if (quad) {
    quad_rule(p + 2, r, s, w);
    for (size_t q = 0; q < w.size(); ++q) {
      quad_raw(p, r[q], s[q], phi.data(), nullptr, nullptr);
      for (int j = 0; j < np; ++j) acc[j] += w[q] * phi[j] * phi[j];
    }
  } else if (dim == 2) {
    tri_rule(p + 2, r, s, w);
    for (size_t q = 0; q < w.size(); ++q) {
      tri_raw(p, r[q], s[q], phi.data(), nullptr, nullptr);
      for (int j = 0; j < np; ++j) acc[j] += w[q] * phi[j] * phi[j];
    }
  } else {
    tet_rule(p + 2, r, s, t, w);
    for (size_t q = 0; q < w.size(); ++q) {
      tet_raw(p, r[q], s[q], t[q], phi.data(), nullptr);
      for (int j = 0; j < np; ++j) acc[j] += w[q] * phi[j] * phi[j];
    }
  }
  for (int j = 0; j < np; ++j) acc[j] = 1.0 / std::sqrt(acc[j]);
  return acc;
}

void basis_eval(int dim, int p, const double* x, double* phi, double* grad, bool quad) {
  static thread_local int cdim = -1, cp = -1, cq = -1;
  static thread_local std::vector<double> N;
  if (cdim != dim || cp != p || cq != (int)quad) {
    N = norms(dim, p, quad);
    cdim = dim;
    cp = p;
    cq = (int)quad;
  }
  int np = npoly(dim, p, quad);
  if (quad) {
    quad_raw(p, x[0], x[1], phi, grad, grad ? grad + np : nullptr);
  } else if (dim == 2) {
    tri_raw(p, x[0], x[1], phi, grad, grad ? grad + np : nullptr);
  } else {
    tet_raw(p, x[0], x[1], x[2], phi, grad);
  }
  for (int j = 0; j < np; ++j) {
    phi[j] *= N[j];
    if (grad)
      for (int a = 0; a < dim; ++a) grad[a * np + j] *= N[j];
  }
}

// reference vertices of the simplices and of the square
static const double kTriV[3][2] = {{0, 0}, {1, 0}, {0, 1}};
static const double kQuadV[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
static const double kTetV[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

// local face vertices: triangle edge q = (q, q+1); tetrahedron face q = the
// three vertices other than q, ascending
static void face_vertices(int dim, int q, int* fv) {
  if (dim == 2) {
    fv[0] = q;
    fv[1] = (q + 1) % 3;
    return;
  }
  int n = 0;
  for (int k = 0; k < 4; ++k)
    if (k != q) fv[n++] = k;
}

RefTables make_tables(int dim, int p, bool quad) {
  if (dim != 2 && dim != 3) throw std::runtime_error("dim");
  if (quad && dim != 2) throw std::runtime_error("quad");
  RefTables T;
  T.dim = dim;
  T.p = p;
  T.quad = quad;
  T.np = npoly(dim, p, quad);
  T.nfaces = quad ? 4 : dim + 1;
  std::vector<double> fa, fb;
  if (dim == 2) {
    if (quad) quad_rule(p + 1, T.vr, T.vs, T.vw);
    else tri_rule(p + 1, T.vr, T.vs, T.vw);
    T.vt.assign(T.vr.size(), 0.0);
    int n = 2 * p + 1;
    std::vector<double> x(n), w(n);
    gauss_jacobi(n, 0.0, x.data(), w.data());
    for (int i = 0; i < n; ++i) {
      fa.push_back(0.5 * (1.0 + x[i]));
      fb.push_back(0.0);
      T.fw.push_back(0.5 * w[i]);
      T.ft.push_back(fa.back());
    }
  } else {
    tet_rule(p + 2, T.vr, T.vs, T.vt, T.vw);
    std::vector<double> w;
    tri_rule(p + 2, fa, fb, w);
    for (double v : w) T.fw.push_back(2.0 * v);
  }
  T.nqv = (int)T.vw.size();
  T.nqf = (int)T.fw.size();
  T.phiV.resize((size_t)T.nqv * T.np);
  T.dphiV.resize((size_t)dim * T.nqv * T.np);
  std::vector<double> phi(T.np), g((size_t)dim * T.np);
  for (int q = 0; q < T.nqv; ++q) {
    double x[3] = {T.vr[q], T.vs[q], T.vt[q]};
    basis_eval(dim, p, x, phi.data(), g.data(), quad);
    for (int j = 0; j < T.np; ++j) {
      T.phiV[(size_t)q * T.np + j] = phi[j];
      for (int a = 0; a < dim; ++a) T.dphiV[((size_t)a * T.nqv + q) * T.np + j] = g[a * T.np + j];
    }
  }
  T.phiF.resize((size_t)T.nfaces * T.nqf * T.np);
  if (quad) {
    for (int f = 0; f < 4; ++f)
      for (int q = 0; q < T.nqf; ++q) {
        const double* V0 = kQuadV[f];
        const double* V1 = kQuadV[(f + 1) % 4];
        double x[3] = {V0[0] + fa[q] * (V1[0] - V0[0]), V0[1] + fa[q] * (V1[1] - V0[1]), 0.0};
        basis_eval(2, p, x, phi.data(), nullptr, true);
        for (int j = 0; j < T.np; ++j) T.phiF[((size_t)f * T.nqf + q) * T.np + j] = phi[j];
      }
    // the 1-D factors: phi_{a(p+1)}(x, 0) = l_a(x) l_0(0) with l_0 = 1
    T.eleg.resize((size_t)T.nqf * (p + 1));
    T.lend0.resize(p + 1);
    T.lend1.resize(p + 1);
    for (int k = 0; k <= p; ++k) {
      const double c = std::sqrt(2.0 * k + 1.0);
      for (int q = 0; q < T.nqf; ++q) T.eleg[(size_t)q * (p + 1) + k] = c * jacobi(k, 0, 0, 2.0 * fa[q] - 1.0);
      T.lend0[k] = c * jacobi(k, 0, 0, -1.0);
      T.lend1[k] = c * jacobi(k, 0, 0, 1.0);
    }
    std::vector<double> xg(p + 1), wg(p + 1);
    gauss_jacobi(p + 1, 0.0, xg.data(), wg.data());
    T.vleg.resize((size_t)(p + 1) * (p + 1));
    T.vdleg.resize((size_t)(p + 1) * (p + 1));
    T.vw1.resize(p + 1);
    for (int i = 0; i <= p; ++i) {
      T.vw1[i] = 0.5 * wg[i];
      for (int k = 0; k <= p; ++k) {
        const double c = std::sqrt(2.0 * k + 1.0);
        T.vleg[(size_t)i * (p + 1) + k] = c * jacobi(k, 0, 0, xg[i]);
        T.vdleg[(size_t)i * (p + 1) + k] = 2.0 * c * djacobi(k, 0, 0, xg[i]);
      }
    }
    return T;
  }
  for (int f = 0; f < T.nfaces; ++f) {
    int fv[3];
    face_vertices(dim, f, fv);
    for (int q = 0; q < T.nqf; ++q) {
      double x[3] = {0, 0, 0};
      for (int a = 0; a < dim; ++a) {
        const double* V0 = dim == 2 ? kTriV[fv[0]] : kTetV[fv[0]];
        const double* V1 = dim == 2 ? kTriV[fv[1]] : kTetV[fv[1]];
        x[a] = V0[a] + fa[q] * (V1[a] - V0[a]);
        if (dim == 3) x[a] += fb[q] * (kTetV[fv[2]][a] - V0[a]);
      }
      basis_eval(dim, p, x, phi.data(), nullptr);
      for (int j = 0; j < T.np; ++j) T.phiF[((size_t)f * T.nqf + q) * T.np + j] = phi[j];
    }
  }
  if (dim == 2) {
    T.phiX.resize((size_t)3 * T.np);
    for (int v = 0; v < 3; ++v) {
      double x[3] = {kTriV[v][0], kTriV[v][1], 0.0};
      basis_eval(dim, p, x, phi.data(), nullptr);
      for (int j = 0; j < T.np; ++j) T.phiX[(size_t)v * T.np + j] = phi[j];
    }
    T.phiH.resize((size_t)3 * 2 * T.nqf * T.np);
    for (int f = 0; f < 3; ++f)
      for (int h = 0; h < 2; ++h)
        for (int q = 0; q < T.nqf; ++q) {
          const double t = 0.5 * (h + fa[q]);
          const double* V0 = kTriV[f];
          const double* V1 = kTriV[(f + 1) % 3];
          double x[3] = {V0[0] + t * (V1[0] - V0[0]), V0[1] + t * (V1[1] - V0[1]), 0.0};
          basis_eval(dim, p, x, phi.data(), nullptr);
          for (int j = 0; j < T.np; ++j) T.phiH[(((size_t)f * 2 + h) * T.nqf + q) * T.np + j] = phi[j];
        }
  }
  return T;
}

// Face points in the face's own parameters (s, t): reconstructed from the
// table's first face (vertex order a0 < a1 < a2, point = a0 + s(a1-a0) + t(a2-a0)).
const int kFacePerms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

std::vector<double> tet_face_orient_tables(const RefTables& T) {
  // barycentric coordinates of the face points (lambda_0 = 1 - s - t, s, t)
  std::vector<double> fa, fb, w;
  tri_rule(T.p + 2, fa, fb, w);
  std::vector<double> out((size_t)4 * 6 * T.nqf * T.np);
  std::vector<double> phi(T.np);
  for (int f = 0; f < 4; ++f) {
    int fv[3];
    face_vertices(3, f, fv);
    for (int o = 0; o < 6; ++o)
      for (int q = 0; q < T.nqf; ++q) {
        const double lam[3] = {1.0 - fa[q] - fb[q], fa[q], fb[q]};
        // vertex i of this face carries the weight of vertex perm[i] of the other side's face
        double x[3] = {0, 0, 0};
        for (int i = 0; i < 3; ++i)
          for (int a = 0; a < 3; ++a) x[a] += lam[kFacePerms[o][i]] * kTetV[fv[i]][a];
        basis_eval(3, T.p, x, phi.data(), nullptr);
        for (int j = 0; j < T.np; ++j) out[(((size_t)f * 6 + o) * T.nqf + q) * T.np + j] = phi[j];
      }
  }
  return out;
}

// ---------------------------------------------------------------------------
// Mesh ingest: edge table (Sec. 5, "an edge points to the two elements that
// share it") with open-addressing hashing of sorted vertex keys.
// ---------------------------------------------------------------------------

namespace {
struct KeyTable {
  std::vector<uint64_t> keys;
  std::vector<int64_t> vals;
  uint64_t mask = 0;
  explicit KeyTable(int64_t n) {
    uint64_t cap = 16;
    while (cap < (uint64_t)n * 2) cap <<= 1;
    keys.assign(cap, ~0ull);
    vals.assign(cap, -1);
    mask = cap - 1;
  }
  static uint64_t mix(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
  }
  // returns the stored value, or inserts v and returns -1
  int64_t find_or_insert(uint64_t k, int64_t v) {
    uint64_t h = mix(k) & mask;
    while (true) {
      if (keys[h] == ~0ull) {
        keys[h] = k;
        vals[h] = v;
        return -1;
      }
      if (keys[h] == k) return vals[h];
      h = (h + 1) & mask;
    }
  }
};
}  // namespace

// faces of element e: 3 (triangle, also one of a hybrid mesh), 4 (quadrilateral
// or tetrahedron)
static int elem_faces(const Mesh& m, int64_t e) {
  if (!m.quad) return m.nfpe;
  return m.ev[(size_t)e * 4 + 3] < 0 ? 3 : 4;
}

// local face q of element e: edge (v_q, v_{q+1}) of a triangle or quadrilateral,
// the face opposite v_q of a tetrahedron
static void elem_face_vertices(const Mesh& m, int64_t e, int q, int* fv) {
  if (m.dim == 2) {
    fv[0] = q;
    fv[1] = (q + 1) % elem_faces(m, e);
    return;
  }
  face_vertices(3, q, fv);
}

// detJ and the inverse Jacobian of element e from its unwrapped coordinates.
// A quadrilateral maps the square's corners (0,0), (1,0), (1,1), (0,1) to
// v0..v3 through v0, v1 and v3 (affine: exact for parallelograms); it must turn
// counterclockwise at every corner, and one that is not a parallelogram is
// counted in m.nonaffine and marked in m.bil (its map is bilinear; detJ and
// J^-1 here are those of the corner v0 only, used for nothing but the sign
// check).  A triangle of a hybrid mesh is affine.
static void element_jacobian(Mesh& m, int64_t e) {
  const int dim = m.dim;
  const double* X = &m.X[(size_t)e * m.nvpe * dim];
  double* Ji = &m.Jinv[(size_t)e * dim * dim];
  double det;
  if (dim == 2) {
    const bool q4 = m.quad && elem_faces(m, e) == 4;
    const int v2 = q4 ? 3 : 2;  // the vertex at reference (0, 1)
    double a = X[2] - X[0], b = X[2 * v2] - X[0], c = X[3] - X[1], d = X[2 * v2 + 1] - X[1];
    if (q4) {
      double scale = 0.0, off = 0.0;
      for (int k = 0; k < 4; ++k) {
        const double* A = X + 2 * k;
        const double* B = X + 2 * ((k + 1) % 4);
        const double* P = X + 2 * ((k + 3) % 4);
        const double cr = (B[0] - A[0]) * (P[1] - A[1]) - (B[1] - A[1]) * (P[0] - A[0]);
        if (!(cr > 0.0)) throw Error{DGC_ERR_MESH, "quadrilateral that is not convex and counterclockwise"};
        scale = std::max(scale, std::fabs(B[0] - A[0]) + std::fabs(B[1] - A[1]));
      }
      for (int k = 0; k < 2; ++k) off = std::max(off, std::fabs(X[k] + X[4 + k] - X[2 + k] - X[6 + k]));
      if (off > 1e-12 * scale) {
        m.nonaffine++;
        if (m.bil.size() != (size_t)m.ne) m.bil.assign(m.ne, 0);
        m.bil[e] = 1;
      }
    }
    det = a * d - b * c;
    Ji[0] = d / det;
    Ji[1] = -b / det;
    Ji[2] = -c / det;
    Ji[3] = a / det;
  } else {
    double J[3][3];
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < 3; ++k) J[a][k] = X[(k + 1) * 3 + a] - X[a];
    det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
          J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
          J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    // inverse by cofactors: Ji[k][a] = cof(a,k)/det
    for (int k = 0; k < 3; ++k)
      for (int a = 0; a < 3; ++a) {
        int r0 = (a + 1) % 3, r1 = (a + 2) % 3, c0 = (k + 1) % 3, c1 = (k + 2) % 3;
        Ji[k * 3 + a] = (J[r0][c0] * J[r1][c1] - J[r0][c1] * J[r1][c0]) / det;
      }
  }
  if (!(det > 0.0)) throw Error{DGC_ERR_MESH, "element with non-positive Jacobian (check orientation)"};
  m.detJ[e] = det;
}

// Outward unit normal and measure of local face q of element e (from its
// unwrapped coordinates).
static double face_normal(const Mesh& m, int64_t e, int q, double* n) {
  const int dim = m.dim;
  const double* X = &m.X[(size_t)e * m.nvpe * dim];
  int fv[3];
  elem_face_vertices(m, e, q, fv);
  double meas;
  n[0] = n[1] = n[2] = 0.0;
  if (dim == 2) {
    // CCW element: outward normal of edge v_q -> v_{q+1} is (dy, -dx)/|d|
    double dx = X[fv[1] * 2] - X[fv[0] * 2], dy = X[fv[1] * 2 + 1] - X[fv[0] * 2 + 1];
    meas = std::hypot(dx, dy);
    n[0] = dy / meas;
    n[1] = -dx / meas;
  } else {
    double u[3], v[3], w[3];
    for (int a = 0; a < 3; ++a) {
      u[a] = X[fv[1] * 3 + a] - X[fv[0] * 3 + a];
      v[a] = X[fv[2] * 3 + a] - X[fv[0] * 3 + a];
      w[a] = X[q * 3 + a] - X[fv[0] * 3 + a];  // towards the opposite vertex
    }
    n[0] = u[1] * v[2] - u[2] * v[1];
    n[1] = u[2] * v[0] - u[0] * v[2];
    n[2] = u[0] * v[1] - u[1] * v[0];
    double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    meas = 0.5 * nn;
    double sgn = (n[0] * w[0] + n[1] * w[1] + n[2] * w[2]) > 0.0 ? -1.0 : 1.0;
    for (int a = 0; a < 3; ++a) n[a] *= sgn / nn;
  }
  return meas;
}

// Face geometry from the left element (normal, measure: on a hanging side the
// left element is the fine one, so the measure is the half edge's), and the
// inradius dim |element| / |boundary| from each element's own faces.
static void side_geometry(Mesh& m) {
  const int dim = m.dim;
  m.snormal.assign((size_t)m.ns * dim, 0.0);
  m.smeas.assign(m.ns, 0.0);
  for (int64_t s = 0; s < m.ns; ++s) {
    double n[3];
    m.smeas[s] = face_normal(m, m.sl[s], m.sql[s], n);
    for (int a = 0; a < dim; ++a) m.snormal[(size_t)s * dim + a] = n[a];
  }
  m.inradius.resize(m.ne);
  for (int64_t e = 0; e < m.ne; ++e) {
    double bnd = 0.0, n[3];
    for (int q = 0; q < elem_faces(m, e); ++q) bnd += face_normal(m, e, q, n);
    const bool q4 = m.quad && elem_faces(m, e) == 4;
    double vol = m.detJ[e] / (q4 ? 1.0 : dim == 2 ? 2.0 : 6.0);
    if (q4 && !m.bil.empty() && m.bil[e]) {  // a general quadrilateral: its area (shoelace)
      const double* X = &m.X[(size_t)e * 8];
      double a = 0.0;
      for (int k = 0; k < 4; ++k) a += X[2 * k] * X[2 * ((k + 1) % 4) + 1] - X[2 * ((k + 1) % 4)] * X[2 * k + 1];
      vol = 0.5 * a;
    }
    m.inradius[e] = dim * vol / bnd;
  }
}

Mesh* build_mesh(int dim, int p, int64_t nv, const double* xyz, int64_t ne, const int32_t* ev,
                 const double* periodic_len, bool quad) {
  if (dim != 2 && dim != 3) throw Error{DGC_ERR_ARG, "dim must be 2 or 3"};
  if (quad && dim != 2) throw Error{DGC_ERR_ARG, "quadrilateral meshes are two-dimensional"};
  if (dim == 2 && (p < 1 || p > 3)) throw Error{DGC_ERR_UNSUPPORTED, quad ? "quadrilaterals support p = 1..3" : "triangles support p = 1..3"};
  if (dim == 3 && (p < 1 || p > 2)) throw Error{DGC_ERR_UNSUPPORTED, "tetrahedra support p = 1..2"};
  if (nv <= 0 || ne <= 0 || !xyz || !ev) throw Error{DGC_ERR_ARG, "empty mesh or null arrays"};
  if (ne > (1LL << 30) || nv > (1LL << 30)) throw Error{DGC_ERR_ARG, "mesh too large"};
  if (dim == 3 && nv >= (1LL << 21)) throw Error{DGC_ERR_UNSUPPORTED, "tetrahedral meshes need < 2^21 vertices"};
  auto m = std::make_unique<Mesh>();
  m->dim = dim;
  m->p = p;
  m->M = dim + 2;
  m->quad = quad;
  m->nvpe = m->nfpe = quad ? 4 : dim + 1;
  m->nv = nv;
  m->ne = ne;
  m->periodic = periodic_len != nullptr;
  for (int a = 0; a < dim; ++a) {
    m->L[a] = periodic_len ? periodic_len[a] : 0.0;
    if (periodic_len && !(m->L[a] > 0.0)) throw Error{DGC_ERR_ARG, "period lengths must be positive"};
  }
  const int nvpe = m->nvpe;
  m->ev.assign(ev, ev + ne * nvpe);
  m->X.resize((size_t)ne * nvpe * dim);
  m->detJ.resize(ne);
  m->Jinv.resize((size_t)ne * dim * dim);
  m->inradius.resize(ne);
  for (int64_t e = 0; e < ne; ++e) {
    double* X = &m->X[(size_t)e * nvpe * dim];
    for (int k = 0; k < nvpe; ++k) {
      int32_t v = ev[e * nvpe + k];
      if (quad && k == 3 && v == -1) {  // a triangle of a hybrid mesh
        for (int a = 0; a < dim; ++a) X[k * dim + a] = X[a];
        continue;
      }
      if (v < 0 || v >= nv) throw Error{DGC_ERR_MESH, "vertex id out of range"};
      for (int a = 0; a < dim; ++a) {
        double x = xyz[(size_t)v * dim + a];
        if (m->periodic && k > 0) x += m->L[a] * std::nearbyint((X[a] - x) / m->L[a]);
        X[k * dim + a] = x;
      }
    }
    element_jacobian(*m, e);
  }
  // edge/face table, numbered by first appearance
  KeyTable kt(ne * m->nfpe);
  const int nfpe = m->nfpe;
  m->face_of.assign((size_t)ne * nfpe, -1);
  m->sl.reserve(ne * nfpe / 2 + 16);
  for (int64_t e = 0; e < ne; ++e)
    for (int q = 0; q < elem_faces(*m, e); ++q) {
      int fv[3];
      elem_face_vertices(*m, e, q, fv);
      uint64_t g[3] = {0, 0, 0};
      for (int i = 0; i < dim; ++i) g[i] = (uint64_t)ev[e * nvpe + fv[i]];
      std::sort(g, g + dim);
      uint64_t key = dim == 2 ? (g[0] << 32 | g[1]) : (g[0] << 42 | g[1] << 21 | g[2]);
      int64_t s = kt.find_or_insert(key, (int64_t)m->sl.size());
      if (s < 0) {
        m->face_of[(size_t)e * nfpe + q] = (int32_t)m->sl.size();
        m->sl.push_back((int32_t)e);
        m->sql.push_back((int8_t)q);
        m->sr.push_back(-1);
        m->sqr.push_back(-1);
      } else {
        if (m->sr[s] >= 0 || m->sl[s] == e) throw Error{DGC_ERR_MESH, "face shared by more than two elements"};
        m->sr[s] = (int32_t)e;
        m->sqr[s] = (int8_t)q;
        m->face_of[(size_t)e * nfpe + q] = (int32_t)s;
      }
    }
  m->ns = (int64_t)m->sl.size();
  side_geometry(*m);
  m->tab = make_tables(dim, p, quad);
  m->np = m->tab.np;
  for (int64_t e = 0; quad && e < m->ne && !m->hybrid; ++e) m->hybrid = elem_faces(*m, e) == 3;
  if (quad && m->nonaffine > 0) m->hybrid = true;  // general quadrilaterals: the table-driven kernels
  if (m->hybrid) m->tab_tri = make_tables(2, p, false);
  return m.release();
}

// ---------------------------------------------------------------------------
// Coloring (Sec. 3.1).  Protocol (reading of "randomly" and of the order in
// which conflicts are visited): xorshift64 draws, pick(n) = (draw >> 32) % n;
// greedy pass over the edges in order; FIFO of conflicts; a swap candidate is
// a colored face of left(e) then right(e), other than e and the previous
// edge, whose color is unique among the other faces of those two elements;
// a revisited edge (or no candidate) triggers the loop break.
// ---------------------------------------------------------------------------

namespace {
struct Xorshift64 {
  uint64_t s;
  uint32_t pick(uint32_t n) {
    s ^= s << 13;
    s ^= s >> 7;
    s ^= s << 17;
    return (uint32_t)((s >> 32) % n);
  }
};

struct Colorer {
  const Mesh& m;
  int nc;
  std::vector<int8_t>& col;
  Colorer(const Mesh& mm, int n, std::vector<int8_t>& c) : m(mm), nc(n), col(c) {}
  const int32_t* faces(int32_t e) const { return &m.face_of[(size_t)e * m.nfpe]; }
  // bitmask of colors on faces of l(k), r(k) other than k
  uint32_t used(int64_t k) const {
    uint32_t u = 0;
    for (int32_t el : {m.sl[k], m.sr[k]}) {
      if (el < 0) continue;
      const int32_t* f = faces(el);
      for (int q = 0; q < m.nfpe; ++q)
        if (f[q] >= 0 && f[q] != k && col[f[q]] > 0) u |= 1u << col[f[q]];
    }
    return u;
  }
  int avail(int64_t k, int* out) const {
    uint32_t u = used(k);
    int n = 0;
    for (int c = 1; c <= nc; ++c)
      if (!(u & (1u << c))) out[n++] = c;
    return n;
  }
};
}  // namespace

ColorStats color_faces(Mesh& m, uint64_t seed, int64_t max_swaps) {
  const int nc = m.nfpe;  // 3 colors for triangles, 4 for quadrilateral (and hybrid) meshes and tetrahedra
  ColorStats st;
  std::vector<int8_t> col(m.ns, -1);
  Colorer C(m, nc, col);
  Xorshift64 rng{seed ? seed : 0x9E3779B97F4A7C15ull};
  if (max_swaps <= 0) max_swaps = 1000 * m.ns;
  std::vector<int64_t> ring(m.ns + 1);
  int64_t head = 0, tail = 0, count = 0;
  const int64_t cap = m.ns + 1;
  auto push = [&](int64_t k) {
    ring[tail] = k;
    tail = tail + 1 == cap ? 0 : tail + 1;
    ++count;
  };
  int av[kMaxColors + 1];
  for (int64_t k = 0; k < m.ns; ++k) {
    int n = C.avail(k, av);
    if (n) col[k] = (int8_t)av[rng.pick(n)];
    else push(k);
  }
  st.greedy_conflicts = count;
  std::vector<int64_t> seen(m.ns, -1);
  int64_t chain = 0, work = 0;
  while (count > 0) {
    int64_t e = ring[head];
    head = head + 1 == cap ? 0 : head + 1;
    --count;
    if (col[e] >= 0) continue;
    seen[e] = ++chain;
    int64_t prev = -1;
    for (;;) {
      int n = C.avail(e, av);
      if (n) {
        col[e] = (int8_t)av[rng.pick(n)];
        break;
      }
      int32_t el[2] = {m.sl[e], m.sr[e]};
      int tally[kMaxColors + 1] = {0};
      for (int32_t x : el) {
        if (x < 0) continue;
        const int32_t* f = C.faces(x);
        for (int q = 0; q < m.nfpe; ++q)
          if (f[q] >= 0 && f[q] != e && col[f[q]] > 0) ++tally[col[f[q]]];
      }
      int64_t cand[2 * 4];
      int ncand = 0;
      for (int32_t x : el) {
        if (x < 0) continue;
        const int32_t* f = C.faces(x);
        for (int q = 0; q < m.nfpe; ++q) {
          int64_t g = f[q];
          if (g >= 0 && g != e && g != prev && col[g] > 0 && tally[col[g]] == 1) cand[ncand++] = g;
        }
      }
      if (ncand) {
        int64_t g = cand[rng.pick(ncand)];
        if (seen[g] != chain) {
          if (++work > max_swaps) throw Error{DGC_ERR_COLORING_LIMIT, "conflict resolution exceeded max_swaps"};
          col[e] = col[g];
          col[g] = -1;
          prev = e;
          e = g;
          seen[g] = chain;
          ++st.swaps;
          continue;
        }
      }
      // loop break: smallest color present on both sides; e takes it and the
      // two faces that carried it become conflicts
      if (++work > max_swaps) throw Error{DGC_ERR_COLORING_LIMIT, "conflict resolution exceeded max_swaps"};
      int64_t fa = -1, fb = -1;
      int cs = 0;
      if (el[1] >= 0) {
        const int32_t* f0 = C.faces(el[0]);
        const int32_t* f1 = C.faces(el[1]);
        for (int c = 1; c <= nc && !cs; ++c) {
          int64_t a = -1, b = -1;
          for (int q = 0; q < m.nfpe; ++q) {
            if (f0[q] >= 0 && f0[q] != e && col[f0[q]] == c) a = f0[q];
            if (f1[q] >= 0 && f1[q] != e && col[f1[q]] == c) b = f1[q];
          }
          if (a >= 0 && b >= 0) {
            cs = c;
            fa = a;
            fb = b;
          }
        }
      }
      if (cs) {
        col[e] = (int8_t)cs;
        col[fa] = -1;
        col[fb] = -1;
        push(fa);
        push(fb);
        ++st.breaks;
      } else {
        push(e);  // no shared color (another conflict touches e): retry later
        ++st.deferrals;
      }
      break;
    }
  }
  m.color.swap(col);
  m.ncolors = nc;
  // every element has one face of each color, except a hybrid mesh's triangles
  // (three faces, four colors)
  m.perfect = !m.hybrid;
  m.dirty = true;
  return st;
}

int color_faces_naive(Mesh& m) {
  std::vector<int8_t> col(m.ns, -1);
  Colorer C(m, kMaxColors, col);
  int maxc = 0;
  for (int64_t k = 0; k < m.ns; ++k) {
    uint32_t u = C.used(k);
    int c = 1;
    while (u & (1u << c)) ++c;
    if (c > kMaxColors) throw Error{DGC_ERR_COLORING_LIMIT, "naive coloring needs too many colors"};
    col[k] = (int8_t)c;
    maxc = std::max(maxc, c);
  }
  m.color.swap(col);
  m.ncolors = maxc;
  m.perfect = (maxc == m.nfpe);
  m.dirty = true;
  return maxc;
}

// ---------------------------------------------------------------------------
// Reordering (Sec. 5): color-major edges (stable), color-1 renumbering of
// elements (left of the k-th color-1 edge -> k, rights of interior color-1
// edges -> N1, N1+1, ... in the same order; elements no color-1 edge reaches
// follow in original order), then ascending new left element within each
// color >= 2 (ties by original id).  With renumber = false the elements keep
// their ids; with reorder_left = false colors >= 2 keep original edge order.
// ---------------------------------------------------------------------------
void reorder(Mesh& m, bool renumber, bool reorder_left) {
  const int nc = m.ncolors;
  m.color_off.assign(nc + 1, 0);
  for (int64_t k = 0; k < m.ns; ++k) m.color_off[m.color[k]]++;
  std::partial_sum(m.color_off.begin(), m.color_off.end(), m.color_off.begin());
  std::vector<int32_t> order(m.ns);
  {
    std::vector<int32_t> next(m.color_off.begin(), m.color_off.end() - 1);
    for (int64_t k = 0; k < m.ns; ++k) order[next[m.color[k] - 1]++] = (int32_t)k;
  }
  std::vector<int32_t>& en = m.elem_new_of_old;
  en.assign(m.ne, -1);
  if (renumber) {
    int32_t id = 0, n1 = m.color_off[1];
    for (int32_t i = 0; i < n1; ++i) {
      int32_t l = m.sl[order[i]];
      if (en[l] < 0) en[l] = id++;
    }
    for (int32_t i = 0; i < n1; ++i) {
      int32_t r = m.sr[order[i]];
      if (r >= 0 && en[r] < 0) en[r] = id++;
    }
    m.reached = id;
    for (int64_t e = 0; e < m.ne; ++e)
      if (en[e] < 0) en[e] = id++;
  } else {
    std::iota(en.begin(), en.end(), 0);
    m.reached = -1;
  }
  if (reorder_left) {
    for (int c = 2; c <= nc; ++c)
      std::sort(order.begin() + m.color_off[c - 1], order.begin() + m.color_off[c],
                [&](int32_t a, int32_t b) {
                  int32_t la = en[m.sl[a]], lb = en[m.sl[b]];
                  return la != lb ? la < lb : a < b;
                });
  }
  m.side_old_of_new = order;
  m.side_new_of_old.assign(m.ns, 0);
  for (int64_t i = 0; i < m.ns; ++i) m.side_new_of_old[order[i]] = (int32_t)i;
  m.dirty = true;
}

// ---------------------------------------------------------------------------
// Nonconforming refinement and its 6-color map (Sec. 3.2).  One level of
// quadrisection of the flagged triangles of a mesh colored by the map: a
// conforming mesh colored with three colors, or a mesh refined before.
// Triangle (v0, v1, v2) with edge midpoints m01, m12, m20 is replaced, in
// place, by the children [v0, m01, m20], [m01, v1, m12], [m20, m12, v2] and
// [m01, m12, m20].  Corner child k holds the halves of the parent's local edges
// that meet at v_k, on its own local edges of the same index.  Edge colors:
//  - the half of a parent edge of color c next to the edge's endpoint with the
//    smaller vertex id is the first child (m = 1), the other the second
//    (m = 2); child m gets ((c + 3m - 4) mod 6) + 1, i.e. c or c + 3.  (Reading:
//    the paper counts children counterclockwise per element; two refined
//    neighbours run along their common edge in opposite directions, so the
//    count is fixed once, by the global vertex order, for both sides.)
//  - an interior edge takes the color of the parent edge it is parallel to;
//  - edges of unrefined neighbours keep their colors.
// Further levels (reading: the paper says the map extends and gives no rule):
// an element of level L has colors 1..K, K = 3 * 2^L, and its split edges'
// halves take c and c + K, the palette doubling again, so a child's three
// edges stay distinct modulo K.  A flagged element may not be finer than a
// neighbour (adjacent elements differ by at most one level); a flagged element
// that is the coarse side of hanging halves keeps that edge's midpoint vertex,
// each half joins the fine neighbour and the child that now holds it (its color
// kept), and the parallel interior edge takes the parent color, the half's
// color taken modulo K.
// Side order: the base sides in order (one side, or its two halves, first
// child first), then three interior sides per refined element, in element
// order.  A half whose other neighbour is not refined is a hanging side: the
// fine child is its left element, the coarse element its right one, and shalf
// records which half of the coarse element's local edge it covers (0: the half
// next to the coarse edge's first vertex).
// ---------------------------------------------------------------------------
void refine(Mesh& m, const std::vector<uint8_t>& flag) {
  const int64_t ne0 = m.ne, ns0 = m.ns;
  auto lev = [&](int64_t e) { return m.level.empty() ? 0 : (int)m.level[e]; };
  auto hanging = [&](int64_t s) { return !m.shalf.empty() && m.shalf[s] >= 0; };
  for (int64_t s = 0; s < ns0; ++s)
    if (hanging(s) && flag[m.sl[s]])
      throw Error{DGC_ERR_ARG, "refinement: an element finer than its neighbour (refine the coarser one first)"};
  int maxlev = 0;
  for (int64_t e = 0; e < ne0; ++e) {
    if (flag[e] && 3 << (lev(e) + 1) > kMaxColors)
      throw Error{DGC_ERR_UNSUPPORTED, "refinement: at most two levels (12 colors)"};
    maxlev = std::max(maxlev, lev(e) + (flag[e] ? 1 : 0));
  }
  std::vector<int64_t> first(ne0);
  int64_t ne = 0;
  for (int64_t e = 0; e < ne0; ++e) {
    first[e] = ne;
    ne += flag[e] ? 4 : 1;
  }
  if (ne > (1LL << 30)) throw Error{DGC_ERR_ARG, "refined mesh too large"};
  std::vector<int32_t> mid(ns0, -1);  // midpoint vertex of each split base edge
  int64_t nv = m.nv;
  for (int64_t s = 0; s < ns0; ++s)
    if (!hanging(s) && (flag[m.sl[s]] || (m.sr[s] >= 0 && flag[m.sr[s]]))) mid[s] = (int32_t)nv++;
  if (nv > (1LL << 30)) throw Error{DGC_ERR_ARG, "refined mesh too large"};
  // the midpoint vertex of local edge k of element e: a new one, or on an edge
  // already split (e the coarse side of its hanging halves) the vertex the
  // halves share, the end of the fine element's edge that is not e's
  auto midpoint = [&](int64_t e, int k) -> int32_t {
    const int32_t s = m.face_of[(size_t)e * 3 + k];
    if (!hanging(s)) return mid[s];
    const int32_t A = m.ev[(size_t)e * 3 + k], B = m.ev[(size_t)e * 3 + (k + 1) % 3];
    const int32_t f = m.sl[s], x = m.ev[(size_t)f * 3 + m.sql[s]], y = m.ev[(size_t)f * 3 + (m.sql[s] + 1) % 3];
    return x != A && x != B ? x : y;
  };

  std::vector<double> X((size_t)ne * 6);
  std::vector<int32_t> ev((size_t)ne * 3);
  std::vector<int8_t> level((size_t)ne);
  for (int64_t e = 0; e < ne0; ++e) {
    const double* P = &m.X[(size_t)e * 6];
    const int32_t* v = &m.ev[(size_t)e * 3];
    const int64_t n = first[e];
    if (!flag[e]) {
      std::copy_n(P, 6, &X[(size_t)n * 6]);
      std::copy_n(v, 3, &ev[(size_t)n * 3]);
      level[n] = (int8_t)lev(e);
      continue;
    }
    double Q[3][2];
    int32_t mv[3];
    for (int k = 0; k < 3; ++k) {
      const int k1 = (k + 1) % 3;
      for (int a = 0; a < 2; ++a) Q[k][a] = 0.5 * (P[k * 2 + a] + P[k1 * 2 + a]);
      mv[k] = midpoint(e, k);
    }
    const int32_t cv[4][3] = {{v[0], mv[0], mv[2]}, {mv[0], v[1], mv[1]}, {mv[2], mv[1], v[2]}, {mv[0], mv[1], mv[2]}};
    const double* cx[4][3] = {{P, Q[0], Q[2]}, {Q[0], P + 2, Q[1]}, {Q[2], Q[1], P + 4}, {Q[0], Q[1], Q[2]}};
    for (int c = 0; c < 4; ++c) {
      level[n + c] = (int8_t)(lev(e) + 1);
      for (int k = 0; k < 3; ++k) {
        ev[(size_t)(n + c) * 3 + k] = cv[c][k];
        for (int a = 0; a < 2; ++a) X[((size_t)(n + c) * 3 + k) * 2 + a] = cx[c][k][a];
      }
    }
  }

  std::vector<int32_t> sl, sr, csrc;
  std::vector<int8_t> sql, sqr, half, col, crule;
  const size_t cap = (size_t)ns0 * 2 + (size_t)(ne - ne0);
  sl.reserve(cap), sr.reserve(cap), sql.reserve(cap), sqr.reserve(cap), half.reserve(cap), col.reserve(cap);
  csrc.reserve(cap), crule.reserve(cap);
  int32_t src = 0;
  int8_t rule = 0;
  auto add = [&](int64_t l, int64_t r, int ql, int qr, int h, int c) {
    sl.push_back((int32_t)l);
    sr.push_back((int32_t)r);
    sql.push_back((int8_t)ql);
    sqr.push_back((int8_t)qr);
    half.push_back((int8_t)h);
    col.push_back((int8_t)c);
    csrc.push_back(src);
    crule.push_back(rule);
  };
  for (int64_t s = 0; s < ns0; ++s) {
    const int32_t l = m.sl[s], r = m.sr[s];
    const int ql = m.sql[s], qr = m.sqr[s], c = m.color[s];
    src = (int32_t)s;
    rule = 0;
    if (hanging(s)) {
      // l fine, r coarse: the half stays hanging, or joins l and the corner
      // child of r that holds it (half 0 lies at v_qr: child qr; half 1 at
      // v_qr+1: child qr + 1), on that child's local edge qr
      if (!flag[r]) add(first[l], first[r], ql, qr, m.shalf[s], c);
      else add(first[l], first[r] + (m.shalf[s] == 0 ? qr : (qr + 1) % 3), ql, qr, -1, c);
      continue;
    }
    const bool Rl = flag[l] != 0, Rr = r >= 0 && flag[r] != 0;
    if (!Rl && !Rr) {
      add(first[l], r >= 0 ? first[r] : -1, ql, r >= 0 ? qr : -1, -1, c);
      continue;
    }
    // the palette of the side's level (both elements of a conforming side have it)
    const int L = lev(l), K = 3 << L;
    // l runs along the edge from a to b, r (if any) from b to a
    const int32_t a = m.ev[(size_t)l * 3 + ql], b = m.ev[(size_t)l * 3 + (ql + 1) % 3];
    for (int child = 1; child <= 2; ++child) {
      const int32_t P = child == 1 ? std::min(a, b) : std::max(a, b);  // endpoint the half touches
      const int cc = c + (child - 1) * K;  // ((c + 3m - 4) mod 6) + 1 at level 0
      rule = (int8_t)(child | L << 4);
      const int64_t lc = first[l] + (P == a ? ql : (ql + 1) % 3);
      if (r < 0) {
        add(lc, -1, ql, -1, -1, cc);
        continue;
      }
      const int64_t rc = first[r] + (P == b ? qr : (qr + 1) % 3);
      if (Rl && Rr) add(lc, rc, ql, qr, -1, cc);
      else if (Rl) add(lc, first[r], ql, qr, P == b ? 0 : 1, cc);
      else add(rc, first[l], qr, ql, P == a ? 0 : 1, cc);
    }
  }
  for (int64_t e = 0; e < ne0; ++e) {
    if (!flag[e]) continue;
    const int64_t n = first[e];
    const int L = lev(e), K = 3 << L;
    int c[3];  // the parent colors (a split edge's half, taken modulo K)
    for (int k = 0; k < 3; ++k) c[k] = (m.color[m.face_of[(size_t)e * 3 + k]] - 1) % K + 1;
    src = (int32_t)e;
    rule = (int8_t)((3 + 1) | L << 4);
    add(n + 0, n + 3, 1, 2, -1, c[1]);  // m01-m20, parallel to parent edge 1
    rule = (int8_t)((3 + 2) | L << 4);
    add(n + 1, n + 3, 2, 0, -1, c[2]);  // m12-m01, parallel to parent edge 2
    rule = (int8_t)((3 + 0) | L << 4);
    add(n + 2, n + 3, 0, 1, -1, c[0]);  // m20-m12, parallel to parent edge 0
  }
  const int64_t ns = (int64_t)sl.size();
  std::vector<int32_t> face_of((size_t)ne * 3, -1);
  for (int64_t s = 0; s < ns; ++s) {
    int32_t& fl = face_of[(size_t)sl[s] * 3 + sql[s]];
    if (fl >= 0) throw Error{DGC_ERR_MESH, "refinement: local edge listed twice"};
    fl = (int32_t)s;
    if (sr[s] >= 0) {
      int32_t& fr = face_of[(size_t)sr[s] * 3 + sqr[s]];
      if (fr < 0) fr = (int32_t)s;
      else if (half[s] < 0) throw Error{DGC_ERR_MESH, "refinement: local edge listed twice"};
    }
  }
  for (int32_t f : face_of)
    if (f < 0) throw Error{DGC_ERR_MESH, "refinement: element edge without a side"};

  if (m.refined) m.base_stack.push_back(std::move(m.base));
  m.base = Mesh::Base();
  Mesh::Base& b = m.base;
  b.nv = m.nv;
  b.ne = m.ne;
  b.ns = m.ns;
  b.ncolors = m.ncolors;
  b.flag = flag;
  b.elem_new_of_old = m.elem_new_of_old;
  b.color_src.swap(csrc);
  b.color_rule.swap(crule);
  m.ne = ne;
  m.nv = nv;
  m.ns = ns;
  m.X.swap(X);
  m.ev.swap(ev);
  m.sl.swap(sl);
  m.sr.swap(sr);
  m.sql.swap(sql);
  m.sqr.swap(sqr);
  m.shalf.swap(half);
  m.color.swap(col);
  m.face_of.swap(face_of);
  m.level.swap(level);
  b.X.swap(X);
  b.ev.swap(ev);
  b.sl.swap(sl);
  b.sr.swap(sr);
  b.sql.swap(sql);
  b.sqr.swap(sqr);
  b.shalf.swap(half);
  b.color.swap(col);
  b.face_of.swap(face_of);
  b.level.swap(level);
  m.detJ.assign(ne, 0.0);
  m.Jinv.assign((size_t)ne * 4, 0.0);
  for (int64_t e = 0; e < ne; ++e) element_jacobian(m, e);
  side_geometry(m);
  m.refined = true;
  m.ncolors = 3 << std::max(1, maxlev);  // 6 even when nothing was refined
  m.perfect = false;
  // the refined region's colors fill less than one wave of blocks: one wave per
  // color, grid-stride (DGC_OPT_PERSISTENT; results identical)
  m.persistent = true;
  reorder(m, true, true);
  m.dirty = true;
}

// Coarsening (Sec. 3.2): the four children of each refined element merge back
// into the parent, and a parent edge takes the color of the child edge parallel
// to it -- the middle child's edge (k + 1) mod 3 is parallel to parent edge k.
// A parent edge whose neighbour stayed coarse is also read off its halves
// (colors c and c + K, K = 3 * 2^L at the parents' level L: the parent's is the
// one <= K).  The colors so derived from the refined mesh alone are checked
// against the coloring before refinement, and the mesh before the last
// refinement is restored (with its own refinement, if it had one).
void coarsen(Mesh& m) {
  const Mesh::Base& b = m.base;
  auto bhang = [&](int64_t s) { return !b.shalf.empty() && b.shalf[s] >= 0; };
  const int64_t ne0 = b.ne, ns0 = b.ns;
  std::vector<int64_t> first(ne0);
  for (int64_t e = 0, n = 0; e < ne0; ++e) {
    first[e] = n;
    n += b.flag[e] ? 4 : 1;
  }
  std::vector<int8_t> col(ns0, 0);
  auto set = [&](int64_t s, int c) {
    if (col[s] != 0 && col[s] != c) throw Error{DGC_ERR_MESH, "coarsening: children disagree on a parent color"};
    col[s] = (int8_t)c;
  };
  int64_t pos = 0;  // refined sides: the base sides in order (one, or two halves), then interior sides
  for (int64_t s = 0; s < ns0; ++s) {
    const int32_t l = b.sl[s], r = b.sr[s];
    const bool split = !bhang(s) && (b.flag[l] || (r >= 0 && b.flag[r]));
    if (!split) {
      set(s, m.color[pos++]);
      continue;
    }
    const int c1 = m.color[pos], c2 = m.color[pos + 1], K = 3 << (b.level.empty() ? 0 : b.level[l]);
    pos += 2;
    if (std::min(c1, c2) < 1 || std::min(c1, c2) > K || std::max(c1, c2) != std::min(c1, c2) + K)
      throw Error{DGC_ERR_MESH, "coarsening: the halves of a split edge are not colored c and c + K"};
    set(s, std::min(c1, c2));
    for (int32_t x : {l, r}) {
      if (x < 0 || !b.flag[x]) continue;
      const int k = x == l ? b.sql[s] : b.sqr[s];
      const int32_t side = m.face_of[(size_t)(first[x] + 3) * 3 + (k + 1) % 3];
      set(s, m.color[side]);
    }
  }
  for (int64_t s = 0; s < ns0; ++s)
    if (col[s] != b.color[s]) throw Error{DGC_ERR_MESH, "coarsening did not recover the coloring before refinement"};
  m.nv = b.nv;
  m.ne = b.ne;
  m.ns = b.ns;
  m.X = b.X;
  m.ev = b.ev;
  m.sl = b.sl;
  m.sr = b.sr;
  m.sql = b.sql;
  m.sqr = b.sqr;
  m.face_of = b.face_of;
  m.color.swap(col);
  m.shalf = b.shalf;
  m.level = b.level;
  m.ncolors = b.ncolors;
  m.perfect = b.shalf.empty();
  m.refined = !m.base_stack.empty();
  m.persistent = m.refined;  // a conforming mesh again: one block per tile
  if (m.refined) {
    m.base = std::move(m.base_stack.back());
    m.base_stack.pop_back();
  } else {
    m.base = Mesh::Base();
  }
  m.detJ.assign(m.ne, 0.0);
  m.Jinv.assign((size_t)m.ne * 4, 0.0);
  for (int64_t e = 0; e < m.ne; ++e) element_jacobian(m, e);
  side_geometry(m);
  reorder(m, true, true);
  m.dirty = true;
}

// ---------------------------------------------------------------------------
// Volume points and L2 projection (initial states)
// ---------------------------------------------------------------------------
// an element's reference tables: a triangle of a hybrid mesh has its own
static const RefTables& elem_tab(const Mesh& m, int64_t e) {
  return m.hybrid && elem_faces(m, e) == 3 ? m.tab_tri : m.tab;
}

// a general quadrilateral's bilinear map of the square's corners to v0..v3 at
// (r, s), its point x and Jacobian J[a * 2 + k] = d x_a / d r_k
void bilinear_map(const double* X, double r, double s, double* x, double* J) {
  const double w[4] = {(1 - r) * (1 - s), r * (1 - s), r * s, (1 - r) * s};
  const double wr[4] = {-(1 - s), 1 - s, s, -s}, ws[4] = {-(1 - r), -r, r, 1 - r};
  for (int a = 0; a < 2; ++a) {
    double v = 0.0, vr = 0.0, vs = 0.0;
    for (int k = 0; k < 4; ++k) {
      v += w[k] * X[k * 2 + a];
      vr += wr[k] * X[k * 2 + a];
      vs += ws[k] * X[k * 2 + a];
    }
    if (x) x[a] = v;
    if (J) J[a * 2] = vr, J[a * 2 + 1] = vs;
  }
}

// the inverse of a general quadrilateral's mass matrix M_ij = sum_q w_q detJ_q
// phi_i phi_j over the volume rule (row-major, np x np), by Gauss-Jordan
// elimination with partial pivoting (M is symmetric positive definite)
std::vector<double> bilinear_mass_inverse(const Mesh& m, int64_t e) {
  const RefTables& T = m.tab;
  const int n = T.np;
  std::vector<double> A((size_t)n * n, 0.0), I((size_t)n * n, 0.0);
  const double* X = &m.X[(size_t)e * 8];
  for (int q = 0; q < T.nqv; ++q) {
    double J[4];
    bilinear_map(X, T.vr[q], T.vs[q], nullptr, J);
    const double det = J[0] * J[3] - J[1] * J[2];
    const double* ph = &T.phiV[(size_t)q * n];
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) A[(size_t)i * n + j] += T.vw[q] * det * ph[i] * ph[j];
  }
  for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int i = c + 1; i < n; ++i)
      if (std::fabs(A[(size_t)i * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = i;
    for (int j = 0; j < n; ++j) {
      std::swap(A[(size_t)c * n + j], A[(size_t)piv * n + j]);
      std::swap(I[(size_t)c * n + j], I[(size_t)piv * n + j]);
    }
    const double d = A[(size_t)c * n + c];
    for (int j = 0; j < n; ++j) A[(size_t)c * n + j] /= d, I[(size_t)c * n + j] /= d;
    for (int i = 0; i < n; ++i) {
      if (i == c) continue;
      const double f = A[(size_t)i * n + c];
      for (int j = 0; j < n; ++j) A[(size_t)i * n + j] -= f * A[(size_t)c * n + j], I[(size_t)i * n + j] -= f * I[(size_t)c * n + j];
    }
  }
  return I;
}

void vol_points(const Mesh& m, double* xyz) {
  for (int64_t e = 0; e < m.ne; ++e) {
    const RefTables& T = elem_tab(m, e);
    const bool q4 = m.quad && elem_faces(m, e) == 4;
    const int kv[3] = {1, q4 ? 3 : 2, 3};  // the vertices at the reference axes' ends
    const double* X = &m.X[(size_t)e * m.nvpe * m.dim];
    const bool bil = !m.bil.empty() && m.bil[e];
    for (int q = 0; q < T.nqv; ++q) {
      double rs[3] = {T.vr[q], T.vs[q], T.vt[q]};
      for (int a = 0; a < m.dim; ++a) {
        double v = X[a];
        for (int k = 0; k < m.dim; ++k) v += (X[kv[k] * m.dim + a] - X[a]) * rs[k];
        xyz[((size_t)e * T.nqv + q) * m.dim + a] = v;
      }
      if (bil) bilinear_map(X, rs[0], rs[1], &xyz[((size_t)e * T.nqv + q) * 2], nullptr);
    }
  }
}

void project(const Mesh& m, const double* vals, double* c) {
  const int M = m.M, np = m.np;  // the state's stride (hybrid: the quadrilaterals' count)
  for (int64_t e = 0; e < m.ne; ++e) {
    const RefTables& T = elem_tab(m, e);
    const bool bil = !m.bil.empty() && m.bil[e];
    double* ce = c + (size_t)e * M * np;
    std::fill(ce, ce + M * np, 0.0);
    for (int q = 0; q < T.nqv; ++q) {
      double wq = T.vw[q];
      if (bil) {
        double J[4];
        bilinear_map(&m.X[(size_t)e * 8], T.vr[q], T.vs[q], nullptr, J);
        wq *= J[0] * J[3] - J[1] * J[2];
      }
      for (int k = 0; k < M; ++k) {
        double v = wq * vals[((size_t)e * T.nqv + q) * M + k];
        for (int j = 0; j < T.np; ++j) ce[k * np + j] += v * T.phiV[(size_t)q * T.np + j];
      }
    }
    if (bil) {  // the L2 projection on a general quadrilateral: c = M^-1 (sum w detJ u phi)
      const std::vector<double> Mi = bilinear_mass_inverse(m, e);
      std::vector<double> b(ce, ce + M * np);
      for (int k = 0; k < M; ++k)
        for (int i = 0; i < np; ++i) {
          double v = 0.0;
          for (int j = 0; j < np; ++j) v += Mi[(size_t)i * np + j] * b[k * np + j];
          ce[k * np + i] = v;
        }
    }
  }
}

}  // namespace dgc
