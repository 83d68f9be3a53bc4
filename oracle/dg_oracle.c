/*
 * dg_oracle.c -- plain, slow, FP64 CPU oracle for the colored DG right-hand side.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
 * baseline load this file's library.  The product path (the CUDA library under
 * paper_1601_07613_gb300/) never links, loads or calls it, and it shares no code,
 * header, table or constant generator with that path.
 *
 * What it computes, and where the paper defines it (Giuliani & Krivodonova,
 * "Edge coloring in unstructured CFD codes"):
 *
 *   - the modal DG semi-discretisation of the conservation law (Eq. 1) as in
 *     Eq. 2: volume integral of F(U).grad(v_j) minus, over the element's faces,
 *     the integral of v_j times the numerical flux F(U_i, U_nb).n  (Sec. 1);
 *     written element by element, exactly as Eq. 2 is stated -- no edge loop,
 *     no coloring, no scatter, so it is structurally independent of the
 *     colored edge kernels it checks;
 *   - the connectivity graph / edge table with left and right elements
 *     (Sec. 2, Sec. 5 "an edge points to the two elements that share it");
 *   - the modified greedy coloring, the conflict resolution by swaps and the
 *     loop breaking of Sec. 3.1;
 *   - the color-major edge order, the color-1 element renumbering and the
 *     left-ascending order of the remaining colors of Sec. 5 (Tables 5, 6);
 *   - quadrilateral and hybrid triangle/quadrilateral meshes, colored with
 *     C = {1, 2, 3, 4} (Sec. 3.1, Table 2), and Eq. 2 on parallelogram
 *     quadrilaterals;
 *   - the boundary conditions and the limiter of the double Mach reflection
 *     run of Sec. 5 (Table 7): slip walls, prescribed states, a moving planar
 *     shock, and a Barth-Jespersen limiter after every RK stage (readings: the
 *     paper takes both from [giuliani]).
 *
 * The same file builds three ways (oracle/__init__.py): FP64 (the tests'
 * oracle), long double (the extended build: the same steps with a wider
 * significand, the reference an FP64 evaluation's rounding is measured
 * against), and FP64 with OpenMP over the elements of a right-hand side (the
 * CPU baseline; every element's arithmetic is unchanged).
 *
 * The paper leaves the DG ingredients to its reference [giuliani]; the readings
 * used here (orthonormal Dubiner basis, Gauss rules, local Lax-Friedrichs flux,
 * the CFL rule, SSP-RK3, the RNG and tie-break protocol of the coloring) are
 * stated beside each function.  Parity pins for each function live in tests/.
 */
#include <float.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <tgmath.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Arithmetic type.  The default build computes in FP64; the extended build
 * (-DORC_REAL="long double": the x87 80-bit format on x86-64, IEEE binary128 on
 * aarch64) evaluates the same steps with a wider significand, as a reference
 * for how close an FP64 evaluation of Eq. 2 comes to the exact result of the
 * same inputs.  <tgmath.h> makes sqrt, fabs, pow, fmax and round follow the
 * argument type. */
#ifndef ORC_REAL
#define ORC_REAL double
#endif
typedef ORC_REAL real;

/* size of the arithmetic type and its significand bits (53 for FP64) */
int orc_real_bytes(void) { return (int)sizeof(real); }
int orc_real_mant_dig(void) { return sizeof(real) == sizeof(double) ? DBL_MANT_DIG : LDBL_MANT_DIG; }

#define ORC_MAXP 8
#define ORC_MAXNP 165 /* (p+1)(p+2)(p+3)/6 at p = 8 */
#define ORC_MAXM 5
#define ORC_MAXBCS 8

static char orc_err[256];
const char *orc_last_error(void) { return orc_err; }
static int fail(const char *msg) {
  snprintf(orc_err, sizeof orc_err, "%s", msg);
  return -1;
}

/* ======================================================================= */
/* 1-D Gauss rules                                                          */
/* ======================================================================= */

/* Jacobi polynomial P_n^{(a,0)}(x) and its derivative, by the classical
 * three-term recurrence in n (beta = 0). */
static void jacobi_a0(int n, real a, real x, real *P, real *dP) {
  real p0 = 1.0, p1, d0 = 0.0, d1;
  if (n == 0) {
    *P = 1.0;
    *dP = 0.0;
    return;
  }
  p1 = 0.5 * ((a + 2.0) * x + a);
  d1 = 0.5 * (a + 2.0);
  for (int k = 2; k <= n; ++k) {
    real c = 2.0 * k + a; /* 2k + a + b with b = 0 */
    real A = 2.0 * k * (k + a) * (c - 2.0);
    real B = (c - 1.0) * (c * (c - 2.0) * x + a * a);
    real C = 2.0 * (k + a - 1.0) * (k - 1.0) * c;
    real p2 = (B * p1 - C * p0) / A;
    real d2 = ((c - 1.0) * c * (c - 2.0) * p1 + B * d1 - C * d0) / A;
    p0 = p1;
    p1 = p2;
    d0 = d1;
    d1 = d2;
  }
  *P = p1;
  *dP = d1;
}

/* n-point Gauss-Jacobi rule for the weight (1-x)^a on [-1, 1] (a = 0 is
 * Gauss-Legendre).  Roots are bracketed by sign changes on a fine grid, then
 * polished by Newton; weights from the classical formula
 *   w_i = 2^(a+1) * G(n+a+1) G(n+1) / (G(n+a+1) n!) / ((1-x_i^2) P_n'(x_i)^2)
 * which for integer a in {0,1,2} reduces to 2^(a+1) / ((1-x^2) P'^2). */
/* the root search stops when a step is below 1e-17 in FP64 and below the
 * same multiple of the unit roundoff in a wider type */
#define ORC_ROOT_TOL \
  ((real)1e-17 * (sizeof(real) == sizeof(double) ? (real)1 : (real)(LDBL_EPSILON / DBL_EPSILON)))

int orc_gauss_jacobi(int n, real a, real *x, real *w) {
  if (n < 1 || n > 64) return fail("gauss_jacobi: n out of range");
  int found = 0;
  const int grid = 200000;
  real xa = -1.0, Pa, dPa;
  jacobi_a0(n, a, xa, &Pa, &dPa);
  for (int g = 1; g <= grid && found < n; ++g) {
    real xb = -1.0 + 2.0 * g / grid, Pb, dPb;
    jacobi_a0(n, a, xb, &Pb, &dPb);
    if (Pa == 0.0) {
      x[found++] = xa;
    } else if (Pa * Pb < 0.0) {
      real lo = xa, hi = xb, r = 0.5 * (xa + xb);
      for (int it = 0; it < 200; ++it) { /* safeguarded Newton */
        real P, dP;
        jacobi_a0(n, a, r, &P, &dP);
        if ((P < 0.0) == (Pa < 0.0)) lo = r; else hi = r;
        real rn = r - P / dP;
        if (!(rn > lo && rn < hi)) rn = 0.5 * (lo + hi);
        if (fabs(rn - r) < ORC_ROOT_TOL) { r = rn; break; }
        r = rn;
      }
      x[found++] = r;
    }
    xa = xb;
    Pa = Pb;
  }
  if (found != n) return fail("gauss_jacobi: root count mismatch");
  for (int i = 0; i < n; ++i) {
    real P, dP;
    jacobi_a0(n, a, x[i], &P, &dP);
    w[i] = pow(2.0, a + 1.0) / ((1.0 - x[i] * x[i]) * dP * dP);
  }
  return 0;
}

int orc_gauss_legendre(int n, real *x, real *w) { return orc_gauss_jacobi(n, 0.0, x, w); }

/* ======================================================================= */
/* Reference-element rules (collapsed "Duffy" products)                    */
/* ======================================================================= */

/* Triangle {r,s >= 0, r+s <= 1}: n Gauss-Legendre points in xi times n
 * Gauss-Jacobi(1,0) points in eta; r = (1+xi)(1-eta)/4, s = (1+eta)/2,
 * w = w_xi w_eta / 8.  Exact for total degree 2n-1.  Point index = i*n + k
 * (i over eta, k over xi). */
int orc_tri_rule(int n, real *r, real *s, real *w) {
  real xg[64], wg[64], xj[64], wj[64];
  if (orc_gauss_jacobi(n, 0.0, xg, wg) || orc_gauss_jacobi(n, 1.0, xj, wj)) return -1;
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      r[i * n + k] = 0.25 * (1.0 + xg[k]) * (1.0 - xj[i]);
      s[i * n + k] = 0.5 * (1.0 + xj[i]);
      w[i * n + k] = wg[k] * wj[i] / 8.0;
    }
  return 0;
}

/* Tetrahedron {r,s,t >= 0, r+s+t <= 1}: Gauss-Legendre x Gauss-Jacobi(1,0) x
 * Gauss-Jacobi(2,0), n points each; exact for total degree 2n-1. */
int orc_tet_rule(int n, real *r, real *s, real *t, real *w) {
  real xa[64], wa[64], xb[64], wb[64], xc[64], wc[64];
  if (orc_gauss_jacobi(n, 0.0, xa, wa) || orc_gauss_jacobi(n, 1.0, xb, wb) ||
      orc_gauss_jacobi(n, 2.0, xc, wc))
    return -1;
  int q = 0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k, ++q) {
        real a = xa[k], b = xb[j], c = xc[i];
        t[q] = 0.5 * (1.0 + c);
        s[q] = 0.25 * (1.0 + b) * (1.0 - c);
        r[q] = 0.125 * (1.0 + a) * (1.0 - b) * (1.0 - c);
        w[q] = wa[k] * wb[j] * wc[i] / 64.0;
      }
  return 0;
}

/* ======================================================================= */
/* Orthonormal modal basis (the v_ij of Eq. 2)                              */
/* ======================================================================= */
/* Reading: Dubiner's orthogonal polynomials on the reference simplex,
 * normalised to unit L2 norm on the reference element.  Ordering by total
 * degree d = 0..p; within a degree the first index runs from d down to 0.
 *
 * Triangle: phi_{k,l}(r,s) = N_kl Q_k(r,s) P_l^{(2k+1,0)}(2s-1),
 *   Q_k = (1-s)^k P_k(2r/(1-s) - 1), evaluated without division through
 *   (n+1) Q_{n+1} = (2n+1)(2r-1+s) Q_n - n (1-s)^2 Q_{n-1}, Q_0 = 1,
 *   Q_1 = 2r - 1 + s;  N_kl^2 = 2 (2k+1)(k+l+1) (closed form of the Jacobi
 *   norms; pinned numerically by the orthonormality test). */

static int npoly_tri(int p) { return (p + 1) * (p + 2) / 2; }
static int npoly_tet(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

/* Q_n, dQ/dr, dQ/ds for n = 0..p of the homogeneous Legendre recurrence in
 * the variable (2r - 1 + s) with "scale" (1 - s); used by both simplices. */
static void hleg(int p, real u, real du_dr, real du_ds, real v, real dv_ds,
                 real *Q, real *Qr, real *Qs) {
  /* Q_n = v^n P_n(u / v); recurrence (n+1)Q_{n+1} = (2n+1) u Q_n - n v^2 Q_{n-1} */
  Q[0] = 1.0;
  Qr[0] = 0.0;
  Qs[0] = 0.0;
  if (p >= 1) {
    Q[1] = u;
    Qr[1] = du_dr;
    Qs[1] = du_ds;
  }
  for (int n = 1; n < p; ++n) {
    Q[n + 1] = ((2 * n + 1) * u * Q[n] - n * v * v * Q[n - 1]) / (n + 1);
    Qr[n + 1] = ((2 * n + 1) * (du_dr * Q[n] + u * Qr[n]) - n * v * v * Qr[n - 1]) / (n + 1);
    Qs[n + 1] = ((2 * n + 1) * (du_ds * Q[n] + u * Qs[n]) -
                 n * (2.0 * v * dv_ds * Q[n - 1] + v * v * Qs[n - 1])) / (n + 1);
  }
}

int orc_basis_tri(int p, real r, real s, real *phi, real *dr, real *ds) {
  if (p < 0 || p > ORC_MAXP) return fail("basis_tri: p out of range");
  real Q[ORC_MAXP + 1], Qr[ORC_MAXP + 1], Qs[ORC_MAXP + 1];
  hleg(p, 2.0 * r - 1.0 + s, 2.0, 1.0, 1.0 - s, -1.0, Q, Qr, Qs);
  int j = 0;
  for (int d = 0; d <= p; ++d)
    for (int k = d; k >= 0; --k) {
      int l = d - k;
      real J, dJ;
      jacobi_a0(l, 2.0 * k + 1.0, 2.0 * s - 1.0, &J, &dJ);
      real N = sqrt((real)(2 * (2 * k + 1) * (k + l + 1)));
      phi[j] = N * Q[k] * J;
      if (dr) dr[j] = N * Qr[k] * J;
      if (ds) ds[j] = N * (Qs[k] * J + Q[k] * 2.0 * dJ);
      ++j;
    }
  return j;
}

/* Tetrahedron: phi_{i,j,k} = N Q_i R_ij P_k^{(2i+2j+2,0)}(2t-1),
 *   Q_i  = (1-s-t)^i P_i(2r/(1-s-t) - 1),
 *   R_ij = (1-t)^j P_j^{(2i+1,0)}(2s/(1-t) - 1)   (homogeneous Jacobi, below),
 *   N^2  = 2 (2i+1)(i+j+1)(2i+2j+2k+3)  (closed form of the three Jacobi norms
 *          in collapsed coordinates; pinned numerically by orthonormality).
 * Ordering: d = 0..p, i = d..0, j = d-i..0, k = d-i-j. */
/* homogeneous Jacobi H_n = v^n P_n^{(a,0)}(u/v) with partial derivatives */
static void hjac(int p, real a, real u, real ur, real us, real ut, real v, real vs,
                 real vt, real *H, real *Hr, real *Hs, real *Ht) {
  H[0] = 1.0;
  Hr[0] = Hs[0] = Ht[0] = 0.0;
  if (p >= 1) {
    /* P_1 = ((a+2) x + a)/2  ->  H_1 = ((a+2) u + a v)/2 */
    H[1] = 0.5 * ((a + 2.0) * u + a * v);
    Hr[1] = 0.5 * ((a + 2.0) * ur);
    Hs[1] = 0.5 * ((a + 2.0) * us + a * vs);
    Ht[1] = 0.5 * ((a + 2.0) * ut + a * vt);
  }
  for (int n = 2; n <= p; ++n) {
    real c = 2.0 * n + a;
    real A = 2.0 * n * (n + a) * (c - 2.0);
    real B1 = (c - 1.0) * c * (c - 2.0); /* multiplies x P_{n-1} -> u H_{n-1} */
    real B0 = (c - 1.0) * a * a;         /* multiplies P_{n-1}   -> v H_{n-1} */
    real C = 2.0 * (n + a - 1.0) * (n - 1.0) * c; /* multiplies P_{n-2} -> v^2 H_{n-2} */
    H[n] = (B1 * u * H[n - 1] + B0 * v * H[n - 1] - C * v * v * H[n - 2]) / A;
    Hr[n] = (B1 * (ur * H[n - 1] + u * Hr[n - 1]) + B0 * v * Hr[n - 1] - C * v * v * Hr[n - 2]) / A;
    Hs[n] = (B1 * (us * H[n - 1] + u * Hs[n - 1]) + B0 * (vs * H[n - 1] + v * Hs[n - 1]) -
             C * (2.0 * v * vs * H[n - 2] + v * v * Hs[n - 2])) / A;
    Ht[n] = (B1 * (ut * H[n - 1] + u * Ht[n - 1]) + B0 * (vt * H[n - 1] + v * Ht[n - 1]) -
             C * (2.0 * v * vt * H[n - 2] + v * v * Ht[n - 2])) / A;
  }
}

int orc_basis_tet(int p, real r, real s, real t, real *phi, real *dr, real *ds,
                  real *dt) {
  if (p < 0 || p > ORC_MAXP) return fail("basis_tet: p out of range");
  /* Q_i: homogeneous Legendre in u = 2r - 1 + s + t, v = 1 - s - t */
  real Q[ORC_MAXP + 1], Qr[ORC_MAXP + 1], Qs[ORC_MAXP + 1], Qt[ORC_MAXP + 1];
  hjac(p, 0.0, 2.0 * r - 1.0 + s + t, 2.0, 1.0, 1.0, 1.0 - s - t, -1.0, -1.0, Q, Qr, Qs, Qt);
  int n = 0;
  for (int d = 0; d <= p; ++d)
    for (int i = d; i >= 0; --i) {
      /* R_ij: homogeneous Jacobi(2i+1,0) in u = 2s - 1 + t, v = 1 - t */
      real R[ORC_MAXP + 1], Rr[ORC_MAXP + 1], Rs[ORC_MAXP + 1], Rt[ORC_MAXP + 1];
      hjac(d - i, 2.0 * i + 1.0, 2.0 * s - 1.0 + t, 0.0, 2.0, 1.0, 1.0 - t, 0.0, -1.0, R, Rr, Rs, Rt);
      for (int j = d - i; j >= 0; --j) {
        int k = d - i - j;
        real J, dJ;
        jacobi_a0(k, 2.0 * i + 2.0 * j + 2.0, 2.0 * t - 1.0, &J, &dJ);
        real N = sqrt((real)(2 * (2 * i + 1) * (i + j + 1) * (2 * i + 2 * j + 2 * k + 3)));
        real a = Q[i] * R[j];
        phi[n] = N * a * J;
        if (dr) dr[n] = N * (Qr[i] * R[j]) * J;
        if (ds) ds[n] = N * (Qs[i] * R[j] + Q[i] * Rs[j]) * J;
        if (dt) dt[n] = N * ((Qt[i] * R[j] + Q[i] * Rt[j]) * J + a * 2.0 * dJ);
        ++n;
      }
    }
  return n;
}

/* Quadrilateral (reading: the paper colors quadrilateral meshes but leaves
 * their DG space to [giuliani]): the tensor-product Legendre space Q_p on the
 * reference square [0,1]^2, phi_{a,b}(r, s) = l_a(r) l_b(s), where
 * l_n(x) = sqrt(2n+1) P_n(2x-1) is orthonormal on [0, 1]; mode j = a (p+1) + b,
 * so mode 0 is the constant.  P_n from Bonnet's recurrence
 * (n+1) P_{n+1}(t) = (2n+1) t P_n(t) - n P_{n-1}(t), derivatives from
 * P'_{n+1} = P'_{n-1} + (2n+1) P_n. */
static void legendre01(int p, real x, real *l, real *dl) {
  real t = 2.0 * x - 1.0, P[ORC_MAXP + 2], D[ORC_MAXP + 2];
  P[0] = 1.0;
  D[0] = 0.0;
  P[1] = t;
  D[1] = 1.0;
  for (int n = 1; n < p; ++n) {
    P[n + 1] = ((2 * n + 1) * t * P[n] - n * P[n - 1]) / (n + 1);
    D[n + 1] = D[n - 1] + (2 * n + 1) * P[n];
  }
  for (int n = 0; n <= p; ++n) {
    real c = sqrt((real)(2 * n + 1));
    l[n] = c * P[n];
    if (dl) dl[n] = 2.0 * c * D[n]; /* dt/dx = 2 */
  }
}

static int npoly_quad(int p) { return (p + 1) * (p + 1); }

int orc_basis_quad(int p, real r, real s, real *phi, real *dr, real *ds) {
  if (p < 0 || p > ORC_MAXP) return fail("basis_quad: p out of range");
  real lr[ORC_MAXP + 2], dlr[ORC_MAXP + 2], ls[ORC_MAXP + 2], dls[ORC_MAXP + 2];
  legendre01(p, r, lr, dlr);
  legendre01(p, s, ls, dls);
  for (int a = 0; a <= p; ++a)
    for (int b = 0; b <= p; ++b) {
      int j = a * (p + 1) + b;
      phi[j] = lr[a] * ls[b];
      if (dr) dr[j] = dlr[a] * ls[b];
      if (ds) ds[j] = lr[a] * dls[b];
    }
  return 0;
}

/* Square [0,1]^2: n x n Gauss-Legendre points, point i n + k at
 * (x_i, x_k); weights sum to 1. */
int orc_quad_rule(int n, real *r, real *s, real *w) {
  real x[64], wg[64];
  if (n < 1 || n > 64) return fail("quad_rule: n out of range");
  if (orc_gauss_legendre(n, x, wg)) return -1;
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      r[i * n + k] = 0.5 * (1.0 + x[i]);
      s[i * n + k] = 0.5 * (1.0 + x[k]);
      w[i * n + k] = 0.25 * wg[i] * wg[k];
    }
  return 0;
}

/* ======================================================================= */
/* Mesh: edge/face table (Sec. 2 connectivity graph, Sec. 5 edge table)     */
/* ======================================================================= */
/* Reading of the edge table: a face key is the sorted tuple of its global
 * vertex ids; faces are numbered in order of first appearance when elements
 * 0..E-1 and their local faces 0..F-1 are scanned; the left element is the
 * first to list the face, the right the second (-1 on a boundary).
 * Local face q of a triangle (v0,v1,v2) is (v_q, v_{q+1 mod 3}), of a
 * quadrilateral (v0,v1,v2,v3) (v_q, v_{q+1 mod 4}); local face q of a
 * tetrahedron is the face opposite vertex q.  Periodic meshes share
 * vertex ids across the period; each element's coordinates are unwrapped to
 * lie within half a period of its vertex 0. */

typedef struct {
  int dim, nvpe, nfpe;
  /* quadrilateral meshes: nvpe = nfpe = 4; a triangle of a hybrid mesh lists
   * -1 as its fourth vertex and has faces 0..2 only.  nonaffine counts the
   * quadrilaterals that are not parallelograms (bil[e] = 1): their map is
   * bilinear and their mass matrix is not diagonal. */
  int quad;
  int64_t nonaffine;
  int8_t *bil;    /* ne, quadrilateral meshes: 1 for a bilinear (non-parallelogram) element */
  int64_t nv, ne, ns;
  real L[3];
  int periodic;
  real *X;      /* ne * nvpe * dim unwrapped vertex coordinates */
  int32_t *ev;    /* ne * nvpe */
  int32_t *sl, *sr;
  int8_t *sql, *sqr;
  int32_t *es;    /* ne * nfpe: side of each local face */
  int32_t *enb;   /* ne * nfpe: neighbour element (-1 on boundary) */
  /* geometry, FP64 */
  real *detJ;   /* ne */
  real *Jinv;   /* ne * dim * dim, row k = grad of reference coordinate k */
  /* nonconforming meshes only (orc_refine), NULL otherwise */
  int32_t *es2;   /* ne * nfpe: second side on a split edge of a coarse element, -1 if none */
  int8_t *shalf;  /* per side: half of the right element's edge a hanging side covers, or -1 */
  int8_t *col;    /* per side: color from the map of Sec. 3.2 */
  int8_t *lev;    /* per element: refinement level (NULL: every element level 0) */
  /* boundary conditions and limiter (orc_set_bc, orc_set_limiter); all zero by
   * default: every boundary face transmissive, no limiter */
  int8_t *bck;    /* per side: ORC_BC_* kind of a boundary side (r = -1) */
  int8_t *bcs;    /* per side: state index of an ORC_BC_STATE side */
  real bcst[ORC_MAXBCS][ORC_MAXM];
  real shock[3];  /* ORC_BC_SHOCK: state shock_st[0] where x < shock[0] + shock[1] y + shock[2] t */
  int8_t shock_st[2];
  real time;      /* the time the boundary states are taken at */
  int limit;      /* 1: the limiter after every RK stage */
} orc_mesh;

static void face_verts(int dim, int q, int *fv) {
  if (dim == 2) {
    fv[0] = q;
    fv[1] = (q + 1) % 3;
  } else {
    int n = 0;
    for (int k = 0; k < 4; ++k)
      if (k != q) fv[n++] = k;
  }
}

/* faces of element e: 4 for a quadrilateral, 3 for a triangle (also one of a
 * hybrid mesh), 4 for a tetrahedron */
static int elem_nfaces(const orc_mesh *m, int64_t e) {
  if (!m->quad) return m->nfpe;
  return m->ev[e * 4 + 3] < 0 ? 3 : 4;
}

static void face_verts_e(const orc_mesh *m, int64_t e, int q, int *fv) {
  if (m->dim == 2) {
    fv[0] = q;
    fv[1] = (q + 1) % elem_nfaces(m, e);
  } else {
    face_verts(3, q, fv);
  }
}

static int npoly_m(const orc_mesh *m, int p) {
  return m->quad ? npoly_quad(p) : (m->dim == 2 ? npoly_tri(p) : npoly_tet(p));
}

typedef struct {
  int32_t k[3];
  int64_t idx;
} fkey;

static int fkey_cmp(const void *a, const void *b) {
  const fkey *x = (const fkey *)a, *y = (const fkey *)b;
  for (int i = 0; i < 3; ++i)
    if (x->k[i] != y->k[i]) return x->k[i] < y->k[i] ? -1 : 1;
  return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static void sort3(int32_t *k, int n) {
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (k[j] < k[i]) {
        int32_t t = k[i];
        k[i] = k[j];
        k[j] = t;
      }
}

static real det_and_inv(int dim, const real *J, real *Ji) {
  /* J column-major by reference direction: J[a*dim + k] = d x_a / d r_k */
  if (dim == 2) {
    real a = J[0], b = J[1], c = J[2], d = J[3]; /* [[a b],[c d]] */
    real det = a * d - b * c;
    Ji[0] = d / det;
    Ji[1] = -b / det;
    Ji[2] = -c / det;
    Ji[3] = a / det;
    return det;
  }
  real a = J[0], b = J[1], c = J[2], d = J[3], e = J[4], f = J[5], g = J[6], h = J[7], i = J[8];
  real det = a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g);
  Ji[0] = (e * i - f * h) / det;
  Ji[1] = (c * h - b * i) / det;
  Ji[2] = (b * f - c * e) / det;
  Ji[3] = (f * g - d * i) / det;
  Ji[4] = (a * i - c * g) / det;
  Ji[5] = (c * d - a * f) / det;
  Ji[6] = (d * h - e * g) / det;
  Ji[7] = (b * g - a * h) / det;
  Ji[8] = (a * e - b * d) / det;
  return det;
}

void orc_mesh_free(void *h);

/* detJ and J^-1 of element e from its unwrapped coordinates; -1 if detJ <= 0.
 * Simplices map the reference vertices (0,..), (1,0,..), (0,1,..), .. to
 * v0, v1, v2, ..; a quadrilateral maps the square's corners (0,0), (1,0),
 * (1,1), (0,1) to v0..v3, affinely through v0, v1, v3 (exact when it is a
 * parallelogram, v2 = v1 + v3 - v0; otherwise counted in m->nonaffine).  A
 * quadrilateral must also turn counterclockwise at every corner. */
static int elem_geometry(orc_mesh *m, int64_t e) {
  int dim = m->dim;
  real J[9];
  const real *X = m->X + e * m->nvpe * dim;
  int nf = elem_nfaces(m, e);
  int kv[3] = {1, (m->quad && nf == 4) ? 3 : 2, 3};
  for (int a = 0; a < dim; ++a)
    for (int k = 0; k < dim; ++k) J[a * dim + k] = X[kv[k] * dim + a] - X[a];
  real det = det_and_inv(dim, J, m->Jinv + e * dim * dim);
  m->detJ[e] = det;
  if (m->quad && nf == 4) {
    real scale = 0.0, off = 0.0;
    for (int c = 0; c < 4; ++c) {
      const real *A = X + c * 2, *B = X + ((c + 1) % 4) * 2, *Cc = X + ((c + 3) % 4) * 2;
      real cr = (B[0] - A[0]) * (Cc[1] - A[1]) - (B[1] - A[1]) * (Cc[0] - A[0]);
      if (!(cr > 0.0)) return -1;
      scale = fmax(scale, fabs(B[0] - A[0]) + fabs(B[1] - A[1]));
    }
    for (int a = 0; a < 2; ++a) off = fmax(off, fabs(X[a] + X[4 + a] - X[2 + a] - X[6 + a]));
    if (off > 1e-12 * scale) {
      m->nonaffine++;
      m->bil[e] = 1;
    }
  }
  return det > 0.0 ? 0 : -1;
}

static void *mesh_new(int dim, int quad, int64_t nv, const real *xyz, int64_t ne, const int32_t *ev,
                      const real *L) {
  if (dim != 2 && dim != 3) return fail("mesh: dim must be 2 or 3"), (void *)0;
  if (ne <= 0 || nv <= 0 || ne > (1LL << 30) || nv > (1LL << 30))
    return fail("mesh: element or vertex count out of range"), (void *)0;
  orc_mesh *m = (orc_mesh *)calloc(1, sizeof *m);
  m->dim = dim;
  m->quad = quad;
  m->nvpe = quad ? 4 : dim + 1;
  m->nfpe = quad ? 4 : dim + 1;
  m->nv = nv;
  m->ne = ne;
  m->periodic = L != NULL;
  for (int a = 0; a < dim; ++a) m->L[a] = L ? L[a] : 0.0;
  int nvpe = m->nvpe, nfpe = m->nfpe;
  m->ev = (int32_t *)malloc(sizeof(int32_t) * ne * nvpe);
  memcpy(m->ev, ev, sizeof(int32_t) * ne * nvpe);
  m->X = (real *)malloc(sizeof(real) * ne * nvpe * dim);
  m->detJ = (real *)malloc(sizeof(real) * ne);
  m->Jinv = (real *)malloc(sizeof(real) * ne * dim * dim);
  m->bil = (int8_t *)calloc(ne, 1);
  for (int64_t e = 0; e < ne; ++e) {
    for (int k = 0; k < nvpe; ++k) {
      int32_t v = ev[e * nvpe + k];
      if (quad && k == 3 && v == -1) {  /* triangle of a hybrid mesh */
        for (int a = 0; a < dim; ++a) m->X[(e * nvpe + k) * dim + a] = m->X[(e * nvpe) * dim + a];
        continue;
      }
      if (v < 0 || v >= nv) {
        orc_mesh_free(m);
        return fail("mesh: vertex id out of range"), (void *)0;
      }
      for (int a = 0; a < dim; ++a) {
        real x = xyz[(int64_t)v * dim + a];
        if (m->periodic && k > 0) {
          real x0 = m->X[(e * nvpe) * dim + a];
          x += m->L[a] * round((x0 - x) / m->L[a]);
        }
        m->X[(e * nvpe + k) * dim + a] = x;
      }
    }
    if (elem_geometry(m, e)) {
      orc_mesh_free(m);
      return fail("mesh: element with non-positive Jacobian"), (void *)0;
    }
  }
  /* face table by sorting keys (slot e * nfpe + q; a hybrid mesh's triangles
   * have no slot 3) */
  int64_t nent = ne * nfpe, nkeys = 0;
  fkey *keys = (fkey *)malloc(sizeof(fkey) * nent);
  for (int64_t e = 0; e < ne; ++e)
    for (int q = 0; q < elem_nfaces(m, e); ++q) {
      int fv[3];
      face_verts_e(m, e, q, fv);
      fkey *k = keys + nkeys++;
      k->k[2] = -1;
      for (int i = 0; i < dim; ++i) k->k[i] = ev[e * nvpe + fv[i]];
      sort3(k->k, dim);
      k->idx = e * nfpe + q;
    }
  qsort(keys, nkeys, sizeof(fkey), fkey_cmp);
  int64_t *partner = (int64_t *)malloc(sizeof(int64_t) * nent);
  char *first = (char *)calloc(nent, 1);
  int bad = 0;
  for (int64_t i = 0; i < nkeys;) {
    int64_t j = i + 1;
    while (j < nkeys && memcmp(keys[j].k, keys[i].k, sizeof keys[i].k) == 0) ++j;
    if (j - i > 2) bad = 1;
    if (j - i == 2 && keys[i].idx / nfpe == keys[i + 1].idx / nfpe) bad = 1;
    first[keys[i].idx] = 1;
    partner[keys[i].idx] = (j - i == 2) ? keys[i + 1].idx : -1;
    if (j - i == 2) partner[keys[i + 1].idx] = keys[i].idx;
    i = j;
  }
  free(keys);
  if (bad) {
    free(partner);
    free(first);
    orc_mesh_free(m);
    return fail("mesh: face shared by more than two elements"), (void *)0;
  }
  m->es = (int32_t *)malloc(sizeof(int32_t) * nent);
  m->enb = (int32_t *)malloc(sizeof(int32_t) * nent);
  m->sl = (int32_t *)malloc(sizeof(int32_t) * nent);
  m->sr = (int32_t *)malloc(sizeof(int32_t) * nent);
  m->sql = (int8_t *)malloc(nent);
  m->sqr = (int8_t *)malloc(nent);
  for (int64_t i = 0; i < nent; ++i) m->es[i] = m->enb[i] = -1;
  int64_t ns = 0;
  for (int64_t i = 0; i < nent; ++i) {
    if (!first[i]) continue;
    int64_t s = ns++;
    m->sl[s] = (int32_t)(i / nfpe);
    m->sql[s] = (int8_t)(i % nfpe);
    m->es[i] = (int32_t)s;
    if (partner[i] >= 0) {
      int64_t o = partner[i];
      m->sr[s] = (int32_t)(o / nfpe);
      m->sqr[s] = (int8_t)(o % nfpe);
      m->es[o] = (int32_t)s;
      m->enb[i] = (int32_t)(o / nfpe);
      m->enb[o] = (int32_t)(i / nfpe);
    } else {
      m->sr[s] = -1;
      m->sqr[s] = -1;
      m->enb[i] = -1;
    }
  }
  m->ns = ns;
  free(partner);
  free(first);
  return m;
}

void *orc_mesh_new(int dim, int64_t nv, const real *xyz, int64_t ne, const int32_t *ev,
                   const real *L) {
  return mesh_new(dim, 0, nv, xyz, ne, ev, L);
}

/* quadrilateral or hybrid mesh: ev is [ne][4], -1 as the fourth id of a triangle */
void *orc_mesh_new_quad(int64_t nv, const real *xyz, int64_t ne, const int32_t *ev, const real *L) {
  return mesh_new(2, 1, nv, xyz, ne, ev, L);
}

int orc_mesh_is_quad(void *h) { return ((orc_mesh *)h)->quad; }
int64_t orc_mesh_nonaffine(void *h) { return ((orc_mesh *)h)->nonaffine; }

void orc_mesh_free(void *h) {
  orc_mesh *m = (orc_mesh *)h;
  if (!m) return;
  free(m->X);
  free(m->ev);
  free(m->sl);
  free(m->sr);
  free(m->sql);
  free(m->sqr);
  free(m->es);
  free(m->enb);
  free(m->detJ);
  free(m->Jinv);
  free(m->bil);
  free(m->es2);
  free(m->shalf);
  free(m->col);
  free(m->lev);
  free(m->bck);
  free(m->bcs);
  free(m);
}

int64_t orc_mesh_nsides(void *h) { return ((orc_mesh *)h)->ns; }

void orc_mesh_sides(void *h, int32_t *l, int32_t *r, int8_t *ql, int8_t *qr) {
  orc_mesh *m = (orc_mesh *)h;
  memcpy(l, m->sl, sizeof(int32_t) * m->ns);
  memcpy(r, m->sr, sizeof(int32_t) * m->ns);
  memcpy(ql, m->sql, m->ns);
  memcpy(qr, m->sqr, m->ns);
}

void orc_mesh_detj(void *h, real *detJ) {
  orc_mesh *m = (orc_mesh *)h;
  memcpy(detJ, m->detJ, sizeof(real) * m->ne);
}

/* ======================================================================= */
/* Coloring (Sec. 3.1)                                                       */
/* ======================================================================= */
/* Reading of "randomly": xorshift64 (Marsaglia 2003), state = seed or
 * 0x9E3779B97F4A7C15 when seed = 0; one draw is x ^= x<<13, x ^= x>>7,
 * x ^= x<<17; pick(n) = (draw >> 32) mod n, drawn even when n = 1. */
typedef struct {
  uint64_t x;
} orc_rng;
static uint64_t rng_draw(orc_rng *g) {
  uint64_t x = g->x;
  x ^= x << 13;
  x ^= x >> 7;
  x ^= x << 17;
  g->x = x;
  return x;
}
static int rng_pick(orc_rng *g, int n) { return (int)((rng_draw(g) >> 32) % (uint64_t)n); }

/* colors (1..nc) that no other face of left(k) or right(k) carries, ascending */
static int avail_colors(const orc_mesh *m, const int8_t *col, int nc, int64_t k, int *out) {
  int used[16] = {0};
  int32_t el[2] = {m->sl[k], m->sr[k]};
  for (int side = 0; side < 2; ++side) {
    if (el[side] < 0) continue;
    for (int q = 0; q < m->nfpe; ++q) {
      int32_t f = m->es[(int64_t)el[side] * m->nfpe + q];
      if (f >= 0 && f != k && col[f] > 0) used[col[f]] = 1;
    }
  }
  int n = 0;
  for (int c = 1; c <= nc; ++c)
    if (!used[c]) out[n++] = c;
  return n;
}

/* stats[0] = conflicts left by the greedy pass, [1] = swaps, [2] = loop breaks,
 * [3] = deferrals.  Returns 0, or 1 when the swap cap was exceeded. */
int orc_color(void *h, int nc, uint64_t seed, int64_t max_swaps, int8_t *col, int64_t *stats) {
  orc_mesh *m = (orc_mesh *)h;
  int64_t ns = m->ns;
  if (nc < m->nfpe || nc > 15) return fail("color: bad color count");
  if (max_swaps <= 0) max_swaps = 1000 * ns;
  orc_rng g = {seed ? seed : 0x9E3779B97F4A7C15ull};
  for (int64_t k = 0; k < ns; ++k) col[k] = -1;
  /* FIFO of uncolored faces as a ring buffer; it never holds a face twice */
  int64_t cap = ns + 1, head = 0, tail = 0, qlen = 0;
  int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * cap);
  int64_t *stamp = (int64_t *)malloc(sizeof(int64_t) * ns);
  for (int64_t k = 0; k < ns; ++k) stamp[k] = -1;
  int av[16];
  /* modified greedy: a random nonconflicting color from C, or -1 */
  for (int64_t k = 0; k < ns; ++k) {
    int n = avail_colors(m, col, nc, k, av);
    if (n == 0) {
      queue[tail] = k;
      tail = (tail + 1) % cap;
      ++qlen;
    } else {
      col[k] = (int8_t)av[rng_pick(&g, n)];
    }
  }
  stats[0] = qlen;
  stats[1] = stats[2] = stats[3] = 0;
  int64_t work = 0, chain = 0;
  int rc = 0;
  while (qlen > 0) {
    int64_t e = queue[head];
    head = (head + 1) % cap;
    --qlen;
    if (col[e] >= 0) continue;
    ++chain;
    stamp[e] = chain;
    int64_t prev = -1;
    for (;;) {
      int n = avail_colors(m, col, nc, e, av);
      if (n > 0) {
        col[e] = (int8_t)av[rng_pick(&g, n)];
        break;
      }
      /* candidate swaps that do not raise the conflict count: faces f of
       * left(e) then right(e), in local order, f != e, f != prev, colored,
       * whose color occurs once among all faces of left(e), right(e) but e */
      int64_t cand[16];
      int nca = 0;
      int cnt[16] = {0};
      int32_t el[2] = {m->sl[e], m->sr[e]};
      for (int side = 0; side < 2; ++side)
        for (int q = 0; q < m->nfpe; ++q) {
          int32_t f = m->es[(int64_t)el[side] * m->nfpe + q];
          if (f >= 0 && f != e && col[f] > 0) cnt[col[f]]++;
        }
      for (int side = 0; side < 2; ++side)
        for (int q = 0; q < m->nfpe; ++q) {
          int32_t f = m->es[(int64_t)el[side] * m->nfpe + q];
          if (f < 0 || f == e || f == prev || col[f] <= 0) continue;
          if (cnt[col[f]] == 1) cand[nca++] = f;
        }
      if (nca > 0) {
        int64_t f = cand[rng_pick(&g, nca)];
        if (stamp[f] != chain) {
          if (++work > max_swaps) { rc = 1; goto done; }
          col[e] = col[f];
          col[f] = -1;
          prev = e;
          e = f;
          stamp[f] = chain;
          stats[1]++;
          continue;
        }
      }
      /* loop break: the smallest color carried by a face a of left(e) and a
       * face b of right(e); e takes it, a and b become conflicts (Sec. 3.1) */
      if (++work > max_swaps) { rc = 1; goto done; }
      int32_t fa = -1, fb = -1;
      for (int c = 1; c <= nc && fa < 0; ++c) {
        int32_t a = -1, b = -1;
        for (int q = 0; q < m->nfpe; ++q) {
          int32_t f = m->es[(int64_t)el[0] * m->nfpe + q];
          if (f >= 0 && f != e && col[f] == c) a = f;
          if (el[1] >= 0) {
            int32_t f2 = m->es[(int64_t)el[1] * m->nfpe + q];
            if (f2 >= 0 && f2 != e && col[f2] == c) b = f2;
          }
        }
        if (a >= 0 && b >= 0) {
          fa = a;
          fb = b;
          col[e] = (int8_t)c;
        }
      }
      if (fa >= 0) {
        col[fa] = -1;
        col[fb] = -1;
        queue[tail] = fa;
        tail = (tail + 1) % cap;
        queue[tail] = fb;
        tail = (tail + 1) % cap;
        qlen += 2;
        stats[2]++;
      } else {
        /* reading: no color is shared by the two sides (possible only when
         * another conflict touches e); defer e to the back of the queue */
        queue[tail] = e;
        tail = (tail + 1) % cap;
        qlen += 1;
        stats[3]++;
      }
      break;
    }
  }
done:
  free(queue);
  free(stamp);
  if (rc) return fail("color: swap cap exceeded"), 1;
  return 0;
}

/* Naive greedy (Sec. 1): the first color not used by the faces of left and
 * right; needs up to 5 colors on triangles, 7 on tetrahedra. */
int orc_color_naive(void *h, int8_t *col) {
  orc_mesh *m = (orc_mesh *)h;
  int maxc = 0;
  for (int64_t k = 0; k < m->ns; ++k) col[k] = -1;
  for (int64_t k = 0; k < m->ns; ++k) {
    int av[16];
    if (avail_colors(m, col, 15, k, av) == 0) return fail("naive: more than 15 colors");
    col[k] = (int8_t)av[0];
    if (av[0] > maxc) maxc = av[0];
  }
  return maxc;
}

/* ======================================================================= */
/* Reordering (Sec. 5, Tables 5 and 6)                                      */
/* ======================================================================= */
/* Edges stable-sorted by color.  The k-th color-1 edge's left element becomes
 * element k; the right elements of the interior color-1 edges follow, from
 * N1 on, in the same order (= N1 + k on a closed mesh); elements reached by
 * no color-1 edge are appended in original order (reading).  Within each
 * color >= 2 edges are sorted by new left id, ties by original id. */
static const int32_t *g_newl; /* qsort context */
static int edge_cmp_left(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  if (g_newl[x] != g_newl[y]) return g_newl[x] < g_newl[y] ? -1 : 1;
  return x < y ? -1 : (x > y);
}

int orc_reorder(void *h, int nc, const int8_t *col, int32_t *elem_new_of_old,
                int32_t *side_new_of_old, int32_t *offsets) {
  orc_mesh *m = (orc_mesh *)h;
  int64_t ns = m->ns, ne = m->ne;
  for (int c = 0; c <= nc; ++c) offsets[c] = 0;
  for (int64_t k = 0; k < ns; ++k) {
    if (col[k] < 1 || col[k] > nc) return fail("reorder: uncolored edge");
    offsets[col[k]]++;
  }
  for (int c = 1; c <= nc; ++c) offsets[c] += offsets[c - 1];
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * ns);
  int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (nc + 1));
  for (int c = 0; c <= nc; ++c) fill[c] = offsets[c > 0 ? c - 1 : 0];
  for (int c = 1; c <= nc; ++c) fill[c] = offsets[c - 1];
  for (int64_t k = 0; k < ns; ++k) order[fill[col[k]]++] = (int32_t)k; /* stable */
  for (int64_t e = 0; e < ne; ++e) elem_new_of_old[e] = -1;
  int32_t next = 0, n1 = offsets[1];
  for (int32_t i = 0; i < n1; ++i) {
    int32_t l = m->sl[order[i]];
    if (elem_new_of_old[l] < 0) elem_new_of_old[l] = next++;
  }
  for (int32_t i = 0; i < n1; ++i) {
    int32_t r = m->sr[order[i]];
    if (r >= 0 && elem_new_of_old[r] < 0) elem_new_of_old[r] = next++;
  }
  for (int64_t e = 0; e < ne; ++e)
    if (elem_new_of_old[e] < 0) elem_new_of_old[e] = next++;
  int32_t *newl = (int32_t *)malloc(sizeof(int32_t) * ns);
  for (int64_t k = 0; k < ns; ++k) newl[k] = elem_new_of_old[m->sl[k]];
  g_newl = newl;
  for (int c = 2; c <= nc; ++c)
    qsort(order + offsets[c - 1], offsets[c] - offsets[c - 1], sizeof(int32_t), edge_cmp_left);
  for (int32_t i = 0; i < ns; ++i) side_new_of_old[order[i]] = i;
  free(order);
  free(fill);
  free(newl);
  return 0;
}

/* ======================================================================= */
/* Nonconforming refinement and its 6-color map (Sec. 3.2)                  */
/* ======================================================================= */
/* One level of isotropic refinement of the flagged triangles of a triangle
 * mesh whose edges carry a valid coloring: a conforming mesh colored 1..3, or
 * a mesh this function refined before.  A flagged triangle (v0, v1, v2)
 * is split through the midpoints m_k of its edges k = (v_k, v_k+1) into the
 * corner triangles (v0, m0, m2), (m0, v1, m1), (m2, m1, v2) and the middle
 * triangle (m0, m1, m2), numbered in place of the parent in that order.  The
 * midpoint of a split edge is a new vertex; ids nv, nv+1, ... follow the order
 * of the split edges.
 *
 * Colors (Sec. 3.2): the two halves m = 1, 2 of a split edge of color c get
 * ((c + 3m - 4) mod 6) + 1, that is c and c + 3; an edge inside a refined
 * triangle takes the color of the parent edge it is parallel to (the edge
 * joining the midpoints of parent edges a and b is parallel to the third one);
 * the other edges keep their colors.
 * Further levels (the paper says the map extends to several levels and gives no
 * rule; reading): elements of level L carry colors 1..K, K = 3 * 2^L, the map
 * doubles the palette again, halves c and c + K, so a level-L+1 child's edges
 * are distinct modulo K as its parent's are, and the mesh uses 3 * 2^Lmax
 * colors.  The elements refined must have no coarser neighbour (adjacent
 * elements differ by at most one level, as the paper assumes); an element that
 * is the coarse side of hanging halves may be refined: its split edge keeps its
 * midpoint vertex, each half becomes a conforming side with its color, and the
 * parent color of that edge, for the parallel interior edge, is the smaller of
 * its halves' colors (c against c + K).
 * Readings:
 *  - half m = 1 is the one touching the endpoint of the parent edge with the
 *    smaller vertex id.  The paper counts the halves counterclockwise per
 *    element; two refined neighbours would count in opposite directions, so the
 *    count is fixed by the global vertex order instead.
 *  - Sides are listed as: each parent side in order (itself, or its halves with
 *    m = 1 first), then for each refined triangle in element order its three
 *    interior edges, with the corner children 0, 1, 2 as left elements and the
 *    middle child as the right one.
 *  - A half whose other neighbour is not refined is a hanging side: the fine
 *    child is its left element and the coarse neighbour its right one.  shalf
 *    gives which half of the coarse element's local edge it covers: 0 for the
 *    half at the edge's first vertex, 1 for the other.
 * Children and local edges are found by matching vertex ids, not from a fixed
 * table.  Returns a new mesh (orc_mesh_free), or NULL. */

/* local edge q of element e of mesh m joining vertices x and y, or -1 */
static int find_edge(const orc_mesh *m, int64_t e, int32_t x, int32_t y) {
  for (int q = 0; q < 3; ++q) {
    int32_t a = m->ev[e * 3 + q], b = m->ev[e * 3 + (q + 1) % 3];
    if ((a == x && b == y) || (a == y && b == x)) return q;
  }
  return -1;
}

/* the midpoint vertex of local edge k of base element e: a new one (mid[] of
 * its side), or, on an edge already split into two hanging halves (e their
 * coarse element), the vertex the halves share */
static int32_t edge_midpoint(const orc_mesh *b, const int32_t *mid, int64_t e, int k) {
  const int32_t s = b->es[e * 3 + k];
  if (!b->es2 || b->es2[e * 3 + k] < 0) return mid[s];
  const int32_t A = b->ev[e * 3 + k], B = b->ev[e * 3 + (k + 1) % 3];
  const int32_t l = b->sl[s];
  const int32_t x = b->ev[l * 3 + b->sql[s]], y = b->ev[l * 3 + (b->sql[s] + 1) % 3];
  return (x != A && x != B) ? x : y;
}

/* the color of parent edge k of base element e: its side's color, or the
 * smaller of its two halves' colors on a split edge */
static int parent_color(const orc_mesh *b, const int8_t *col, int64_t e, int k) {
  int c = col[b->es[e * 3 + k]];
  if (b->es2 && b->es2[e * 3 + k] >= 0 && col[b->es2[e * 3 + k]] < c) c = col[b->es2[e * 3 + k]];
  return c;
}

void *orc_refine(void *h, const int8_t *col, const uint8_t *flag) {
  const orc_mesh *b = (const orc_mesh *)h;
  if (b->dim != 2 || b->quad) return fail("refine: triangles only"), (void *)0;
  int64_t ne0 = b->ne, ns0 = b->ns, ne = 0, nv = b->nv, nref = 0;
  /* adjacent elements differ by at most one level: no flagged element may be
   * the fine side of a hanging side */
  if (b->shalf)
    for (int64_t s = 0; s < ns0; ++s)
      if (b->shalf[s] >= 0 && flag[b->sl[s]]) return fail("refine: an element finer than its neighbour"), (void *)0;
  int64_t *first = (int64_t *)malloc(sizeof(int64_t) * ne0);
  for (int64_t e = 0; e < ne0; ++e) {
    first[e] = ne;
    ne += flag[e] ? 4 : 1;
    nref += flag[e] ? 1 : 0;
  }
  int32_t *mid = (int32_t *)malloc(sizeof(int32_t) * ns0);
  for (int64_t s = 0; s < ns0; ++s) {
    int32_t l = b->sl[s], r = b->sr[s];
    int hang = b->shalf && b->shalf[s] >= 0;
    mid[s] = (!hang && (flag[l] || (r >= 0 && flag[r]))) ? (int32_t)nv++ : -1;
  }
  orc_mesh *m = (orc_mesh *)calloc(1, sizeof *m);
  m->dim = 2;
  m->nvpe = m->nfpe = 3;
  m->nv = nv;
  m->ne = ne;
  m->periodic = b->periodic;
  m->L[0] = b->L[0];
  m->L[1] = b->L[1];
  m->ev = (int32_t *)malloc(sizeof(int32_t) * ne * 3);
  m->X = (real *)malloc(sizeof(real) * ne * 6);
  m->detJ = (real *)malloc(sizeof(real) * ne);
  m->Jinv = (real *)malloc(sizeof(real) * ne * 4);
  m->lev = (int8_t *)malloc(ne);
  int bad = 0;
  for (int64_t e = 0; e < ne0; ++e) {
    const int32_t *v = b->ev + e * 3;
    const real *P = b->X + e * 6;
    const int le = b->lev ? b->lev[e] : 0;
    int64_t n = first[e];
    if (!flag[e]) {
      memcpy(m->ev + n * 3, v, sizeof(int32_t) * 3);
      memcpy(m->X + n * 6, P, sizeof(real) * 6);
      m->lev[n] = (int8_t)le;
      continue;
    }
    int32_t mv[3];
    real Q[3][2];
    for (int k = 0; k < 3; ++k) {
      mv[k] = edge_midpoint(b, mid, e, k);
      for (int a = 0; a < 2; ++a) Q[k][a] = 0.5 * (P[k * 2 + a] + P[((k + 1) % 3) * 2 + a]);
    }
    /* children as (vertex id, coordinates) */
    int32_t cid[4][3] = {{v[0], mv[0], mv[2]}, {mv[0], v[1], mv[1]}, {mv[2], mv[1], v[2]}, {mv[0], mv[1], mv[2]}};
    const real *cx[4][3] = {{P, Q[0], Q[2]}, {Q[0], P + 2, Q[1]}, {Q[2], Q[1], P + 4}, {Q[0], Q[1], Q[2]}};
    for (int c = 0; c < 4; ++c) {
      m->lev[n + c] = (int8_t)(le + 1);
      for (int k = 0; k < 3; ++k) {
        m->ev[(n + c) * 3 + k] = cid[c][k];
        m->X[((n + c) * 3 + k) * 2 + 0] = cx[c][k][0];
        m->X[((n + c) * 3 + k) * 2 + 1] = cx[c][k][1];
      }
    }
  }
  int64_t cap = 2 * ns0 + 3 * nref, ns = 0;
  m->sl = (int32_t *)malloc(sizeof(int32_t) * cap);
  m->sr = (int32_t *)malloc(sizeof(int32_t) * cap);
  m->sql = (int8_t *)malloc(cap);
  m->sqr = (int8_t *)malloc(cap);
  m->shalf = (int8_t *)malloc(cap);
  m->col = (int8_t *)malloc(cap);
#define ADD_SIDE(L_, R_, QL_, QR_, H_, C_)                                        \
  do {                                                                           \
    m->sl[ns] = (int32_t)(L_);                                                   \
    m->sr[ns] = (int32_t)(R_);                                                   \
    m->sql[ns] = (int8_t)(QL_);                                                  \
    m->sqr[ns] = (int8_t)(QR_);                                                  \
    m->shalf[ns] = (int8_t)(H_);                                                 \
    m->col[ns] = (int8_t)(C_);                                                   \
    ++ns;                                                                        \
  } while (0)
  for (int64_t s = 0; s < ns0; ++s) {
    int32_t l = b->sl[s], r = b->sr[s];
    int c = col[s];
    if (b->shalf && b->shalf[s] >= 0) {
      /* a hanging half (l fine, r coarse): it stays hanging, or, when the
       * coarse element is refined, joins l and the child of r that holds it */
      if (!flag[r]) {
        ADD_SIDE(first[l], first[r], b->sql[s], b->sqr[s], b->shalf[s], c);
        continue;
      }
      int32_t x = b->ev[l * 3 + b->sql[s]], y = b->ev[l * 3 + (b->sql[s] + 1) % 3];
      int64_t fr = -1;
      int qr = -1;
      for (int k = 0; k < 4; ++k)
        if ((qr = find_edge(m, first[r] + k, x, y)) >= 0) {
          fr = first[r] + k;
          break;
        }
      if (fr < 0) bad = 1;
      ADD_SIDE(first[l], fr, b->sql[s], qr, -1, c);
      continue;
    }
    int Rl = flag[l] != 0, Rr = r >= 0 && flag[r] != 0;
    if (!Rl && !Rr) {
      ADD_SIDE(first[l], r >= 0 ? first[r] : -1, b->sql[s], r >= 0 ? b->sqr[s] : -1, -1, c);
      continue;
    }
    /* the palette of the side's level (a conforming side joins two elements of one level) */
    const int lv = b->lev ? b->lev[l] : 0;
    if (r >= 0 && b->lev && b->lev[r] != lv) bad = 1;
    const int K = 3 << lv;
    int32_t va = b->ev[l * 3 + b->sql[s]], vb = b->ev[l * 3 + (b->sql[s] + 1) % 3];
    for (int half = 1; half <= 2; ++half) {
      int32_t Pv = (half == 1) == (va < vb) ? va : vb; /* endpoint this half touches */
      int cm = c + (half - 1) * K; /* ((c + 3m - 4) mod 6) + 1 at level 0 */
      /* the fine element(s) holding the half (Pv, mid) and their local edge */
      int64_t fl = -1, fr = -1;
      int ql = -1, qr = -1;
      for (int k = 0; k < 4 && Rl; ++k)
        if ((ql = find_edge(m, first[l] + k, Pv, mid[s])) >= 0) {
          fl = first[l] + k;
          break;
        }
      for (int k = 0; k < 4 && Rr; ++k)
        if ((qr = find_edge(m, first[r] + k, Pv, mid[s])) >= 0) {
          fr = first[r] + k;
          break;
        }
      if ((Rl && fl < 0) || (Rr && fr < 0)) bad = 1;
      if (r < 0) {
        ADD_SIDE(fl, -1, ql, -1, -1, cm);
      } else if (Rl && Rr) {
        ADD_SIDE(fl, fr, ql, qr, -1, cm);
      } else if (Rl) { /* coarse right neighbour */
        int qc = b->sqr[s];
        ADD_SIDE(fl, first[r], ql, qc, b->ev[r * 3 + qc] == Pv ? 0 : 1, cm);
      } else { /* coarse left element: the fine child becomes the left one */
        int qc = b->sql[s];
        ADD_SIDE(fr, first[l], qr, qc, b->ev[l * 3 + qc] == Pv ? 0 : 1, cm);
      }
    }
  }
  for (int64_t e = 0; e < ne0; ++e) {
    if (!flag[e]) continue;
    int64_t n = first[e];
    int32_t mv[3];
    for (int t = 0; t < 3; ++t) mv[t] = edge_midpoint(b, mid, e, t);
    for (int k = 0; k < 3; ++k) { /* the interior edge of corner child k: both ends are midpoints */
      int q = -1, qm = -1, ea = -1, eb = -1;
      for (int t = 0; t < 3 && q < 0; ++t) {
        int32_t x = m->ev[(n + k) * 3 + t], y = m->ev[(n + k) * 3 + (t + 1) % 3];
        int xm = x == mv[0] || x == mv[1] || x == mv[2], ym = y == mv[0] || y == mv[1] || y == mv[2];
        if (xm && ym) q = t;
      }
      if (q < 0) {
        bad = 1;
        continue;
      }
      int32_t x = m->ev[(n + k) * 3 + q], y = m->ev[(n + k) * 3 + (q + 1) % 3];
      qm = find_edge(m, n + 3, x, y);
      for (int t = 0; t < 3; ++t) {
        if (mv[t] == x || mv[t] == y) {
          if (ea < 0) ea = t;
          else eb = t;
        }
      }
      if (qm < 0 || ea < 0 || eb < 0) {
        bad = 1;
        continue;
      }
      ADD_SIDE(n + k, n + 3, q, qm, -1, parent_color(b, col, e, 3 - ea - eb));
    }
  }
#undef ADD_SIDE
  m->ns = ns;
  m->es = (int32_t *)malloc(sizeof(int32_t) * ne * 3);
  m->es2 = (int32_t *)malloc(sizeof(int32_t) * ne * 3);
  m->enb = (int32_t *)malloc(sizeof(int32_t) * ne * 3);
  for (int64_t i = 0; i < ne * 3; ++i) m->es[i] = m->es2[i] = -1;
  for (int64_t t = 0; t < ns && !bad; ++t) {
    int64_t il = (int64_t)m->sl[t] * 3 + m->sql[t];
    if (m->es[il] >= 0) bad = 1;
    m->es[il] = (int32_t)t;
    m->enb[il] = m->sr[t];
    if (m->sr[t] >= 0) {
      int64_t ir = (int64_t)m->sr[t] * 3 + m->sqr[t];
      if (m->es[ir] < 0) {
        m->es[ir] = (int32_t)t;
        m->enb[ir] = m->sl[t];
      } else if (m->shalf[t] >= 0 && m->es2[ir] < 0) {
        m->es2[ir] = (int32_t)t;
      } else {
        bad = 1;
      }
    }
  }
  for (int64_t i = 0; i < ne * 3 && !bad; ++i)
    if (m->es[i] < 0) bad = 1;
  for (int64_t e = 0; e < ne && !bad; ++e)
    if (elem_geometry(m, e)) bad = 1;
  free(first);
  free(mid);
  if (bad) {
    orc_mesh_free(m);
    return fail("refine: inconsistent refined mesh"), (void *)0;
  }
  return m;
}

/* refinement level of each element (0 on a mesh orc_refine did not make) */
void orc_mesh_levels(void *h, int8_t *lev) {
  orc_mesh *m = (orc_mesh *)h;
  for (int64_t e = 0; e < m->ne; ++e) lev[e] = m->lev ? m->lev[e] : 0;
}

int64_t orc_mesh_nelem(void *h) { return ((orc_mesh *)h)->ne; }
int64_t orc_mesh_nvert(void *h) { return ((orc_mesh *)h)->nv; }

/* element vertex ids and unwrapped coordinates */
void orc_mesh_elements(void *h, int32_t *ev, real *X) {
  orc_mesh *m = (orc_mesh *)h;
  memcpy(ev, m->ev, sizeof(int32_t) * m->ne * m->nvpe);
  memcpy(X, m->X, sizeof(real) * m->ne * m->nvpe * m->dim);
}

/* colors of a refined mesh and the hanging half of each side (-1 conforming) */
int orc_mesh_refined(void *h, int8_t *col, int8_t *half) {
  orc_mesh *m = (orc_mesh *)h;
  if (!m->col) return fail("mesh: not refined");
  memcpy(col, m->col, m->ns);
  memcpy(half, m->shalf, m->ns);
  return 0;
}

/* ======================================================================= */
/* Physics: Euler flux and local Lax-Friedrichs flux                        */
/* ======================================================================= */
/* Euler: U = (rho, rho u, rho v[, rho w], E), p = (gamma-1)(E - rho|u|^2/2).
 * Reading of "Lax-Friedrichs": local (Rusanov) at each quadrature point,
 *   F* = (F(U-).n + F(U+).n)/2 - lambda (U+ - U-)/2,
 *   lambda = max(|u-.n| + c-, |u+.n| + c+),  c = sqrt(gamma p / rho).
 * Linear advection (M = 1, F = a u) is kept for the exactness pins; there the
 * same formula is the upwind flux. */
#define ORC_GAMMA 1.4
enum { ORC_EULER = 0, ORC_ADVECTION = 1 };

static void euler_flux_n(int dim, const real *U, const real *n, real *Fn, real *lam) {
  real rho = U[0], E = U[dim + 1];
  real vel[3] = {0, 0, 0}, q2 = 0.0, un = 0.0;
  for (int a = 0; a < dim; ++a) {
    vel[a] = U[1 + a] / rho;
    q2 += vel[a] * vel[a];
    un += vel[a] * n[a];
  }
  real p = (ORC_GAMMA - 1.0) * (E - 0.5 * rho * q2);
  Fn[0] = rho * un;
  for (int a = 0; a < dim; ++a) Fn[1 + a] = U[1 + a] * un + p * n[a];
  Fn[dim + 1] = (E + p) * un;
  *lam = fabs(un) + sqrt(ORC_GAMMA * p / rho);
}

/* physical flux in direction a (for the volume term) */
static void euler_flux_dir(int dim, const real *U, int a, real *F) {
  real n[3] = {0, 0, 0}, lam;
  n[a] = 1.0;
  euler_flux_n(dim, U, n, F, &lam);
}

typedef struct {
  int kind, dim, M;
  real adv[3];
} orc_phys;

static void phys_flux_dir(const orc_phys *ph, const real *U, int a, real *F) {
  if (ph->kind == ORC_EULER) euler_flux_dir(ph->dim, U, a, F);
  else F[0] = ph->adv[a] * U[0];
}

static void num_flux(const orc_phys *ph, const real *Um, const real *Up, const real *n,
                     real *Fs) {
  if (ph->kind == ORC_EULER) {
    real Fm[ORC_MAXM], Fp[ORC_MAXM], lm, lp;
    euler_flux_n(ph->dim, Um, n, Fm, &lm);
    euler_flux_n(ph->dim, Up, n, Fp, &lp);
    real lam = lm > lp ? lm : lp;
    for (int k = 0; k < ph->M; ++k) Fs[k] = 0.5 * (Fm[k] + Fp[k]) - 0.5 * lam * (Up[k] - Um[k]);
  } else {
    real an = 0.0;
    for (int a = 0; a < ph->dim; ++a) an += ph->adv[a] * n[a];
    Fs[0] = 0.5 * an * (Um[0] + Up[0]) - 0.5 * fabs(an) * (Up[0] - Um[0]);
  }
}

/* Boundary kinds and the state U+ outside a boundary face at the physical
 * point x (readings: Sec. 5 runs the double Mach reflection of [giuliani],
 * whose boundaries are slip walls, inflow states and the moving incident
 * shock; the paper states none of them):
 *   transmissive: U+ = U-;
 *   wall (slip): U+ = U- with its normal momentum reversed, m+ = m- - 2 (m-.n) n
 *     (so the Lax-Friedrichs flux carries no mass and no energy through it);
 *   state: U+ = the face's prescribed state;
 *   shock: a planar shock whose trace moves along x: U+ = the state behind it
 *     where x < a + b y + c t, else the state ahead of it. */
enum { ORC_BC_TRANSMISSIVE = 0, ORC_BC_WALL = 1, ORC_BC_STATE = 2, ORC_BC_SHOCK = 3 };

static void bc_state(const orc_mesh *m, int32_t s, int M, const real *Um, const real *n, const real *x,
                     real *Up) {
  const int kind = m->bck ? m->bck[s] : ORC_BC_TRANSMISSIVE;
  if (kind == ORC_BC_WALL) {
    real mn = 0.0;
    for (int a = 0; a < m->dim; ++a) mn += Um[1 + a] * n[a];
    Up[0] = Um[0];
    for (int a = 0; a < m->dim; ++a) Up[1 + a] = Um[1 + a] - 2.0 * mn * n[a];
    Up[M - 1] = Um[M - 1];
  } else if (kind == ORC_BC_STATE) {
    for (int k = 0; k < M; ++k) Up[k] = m->bcst[m->bcs[s]][k];
  } else if (kind == ORC_BC_SHOCK) {
    const real xs = m->shock[0] + m->shock[1] * x[1] + m->shock[2] * m->time;
    const real *S = m->bcst[m->shock_st[x[0] < xs ? 0 : 1]];
    for (int k = 0; k < M; ++k) Up[k] = S[k];
  } else {
    for (int k = 0; k < M; ++k) Up[k] = Um[k];
  }
}

/* exported for the boundary pins: U+ of boundary side s at point x, with the
 * side's outward unit normal n (that of its element) */
int orc_boundary_state(void *h, int32_t s, const real *Um, const real *n, const real *x, real *Up) {
  const orc_mesh *m = (const orc_mesh *)h;
  if (s < 0 || s >= m->ns || m->sr[s] >= 0) return fail("boundary_state: not a boundary side");
  bc_state(m, s, m->dim + 2, Um, n, x, Up);
  return 0;
}

/* Boundary conditions of a triangle mesh: kind[s] (ORC_BC_*) for every side s
 * with r = -1 (entries of interior sides are ignored), sidx[s] the state of an
 * ORC_BC_STATE side, states [nstates][4], shock = (a, b, c) and shock_st = (the
 * states behind and ahead) of ORC_BC_SHOCK sides (either may be NULL when no
 * side is of that kind). */
int orc_set_bc(void *h, const int8_t *kind, const int8_t *sidx, int nstates, const real *states,
               const real *shock, const int8_t *shock_st) {
  orc_mesh *m = (orc_mesh *)h;
  if (m->dim != 2 || m->quad) return fail("set_bc: triangle meshes only");
  if (nstates < 0 || nstates > ORC_MAXBCS) return fail("set_bc: state count out of range");
  for (int64_t s = 0; s < m->ns; ++s) {
    if (m->sr[s] >= 0) continue;
    if (kind[s] < 0 || kind[s] > ORC_BC_SHOCK) return fail("set_bc: unknown boundary kind");
    if (kind[s] == ORC_BC_STATE && (!sidx || sidx[s] < 0 || sidx[s] >= nstates))
      return fail("set_bc: state index out of range");
    if (kind[s] == ORC_BC_SHOCK && (!shock || !shock_st || shock_st[0] < 0 || shock_st[0] >= nstates ||
                                    shock_st[1] < 0 || shock_st[1] >= nstates))
      return fail("set_bc: shock states out of range");
  }
  if (!m->bck) {
    m->bck = (int8_t *)calloc((size_t)(m->ns > 0 ? m->ns : 1), 1);
    m->bcs = (int8_t *)calloc((size_t)(m->ns > 0 ? m->ns : 1), 1);
  }
  for (int64_t s = 0; s < m->ns; ++s) {
    m->bck[s] = m->sr[s] >= 0 ? 0 : kind[s];
    m->bcs[s] = m->sr[s] >= 0 || !sidx ? 0 : sidx[s];
  }
  for (int i = 0; i < nstates; ++i)
    for (int k = 0; k < 4; ++k) m->bcst[i][k] = states[i * 4 + k];
  for (int a = 0; a < 3; ++a) m->shock[a] = shock ? shock[a] : 0.0;
  m->shock_st[0] = shock_st ? shock_st[0] : 0;
  m->shock_st[1] = shock_st ? shock_st[1] : 0;
  return 0;
}

int orc_set_time(void *h, real t) {
  ((orc_mesh *)h)->time = t;
  return 0;
}
int orc_get_time(void *h, real *t) {
  *t = ((orc_mesh *)h)->time;
  return 0;
}
int orc_set_limiter(void *h, int on) {
  orc_mesh *m = (orc_mesh *)h;
  if (on && (m->dim != 2 || m->quad)) return fail("set_limiter: triangle meshes only");
  m->limit = on != 0;
  return 0;
}

/* exported for the flux pins */
int orc_lf_flux(int dim, const real *Um, const real *Up, const real *n, real *Fs) {
  orc_phys ph = {ORC_EULER, dim, dim + 2, {0, 0, 0}};
  num_flux(&ph, Um, Up, n, Fs);
  return 0;
}

/* ======================================================================= */
/* Eq. 2, element by element                                                */
/* ======================================================================= */

static int basis_eval(const orc_mesh *m, int p, const real *x, real *phi, real *d0, real *d1,
                      real *d2) {
  if (m->quad) return orc_basis_quad(p, x[0], x[1], phi, d0, d1);
  if (m->dim == 2) return orc_basis_tri(p, x[0], x[1], phi, d0, d1);
  return orc_basis_tet(p, x[0], x[1], x[2], phi, d0, d1, d2);
}

/* Element e's own space on a hybrid triangle/quadrilateral mesh (Sec. 3.1,
 * Table 2's hybrid mesh; reading: each element carries the space of its kind,
 * P_p on a triangle and Q_p on a quadrilateral, and the state is stored with
 * the larger count Np = (p+1)^2 per variable, a triangle using the first
 * (p+1)(p+2)/2 entries).  On other meshes these are the mesh-wide ones. */
static int elem_is_quad(const orc_mesh *m, int64_t e) { return m->quad && m->ev[e * 4 + 3] >= 0; }
static int npoly_e(const orc_mesh *m, int64_t e, int p) {
  return m->quad && !elem_is_quad(m, e) ? npoly_tri(p) : npoly_m(m, p);
}
static int basis_eval_e(const orc_mesh *m, int64_t e, int p, const real *x, real *phi, real *d0, real *d1,
                        real *d2) {
  if (m->quad && !elem_is_quad(m, e)) return orc_basis_tri(p, x[0], x[1], phi, d0, d1);
  return basis_eval(m, p, x, phi, d0, d1, d2);
}

/* A quadrilateral that is not a parallelogram (reading: Sec. 1 and Table 2
 * include general quadrilaterals; [giuliani] is not available): the bilinear
 * map of the square's corners (0,0), (1,0), (1,1), (0,1) to v0..v3,
 *   x(r, s) = v0 (1-r)(1-s) + v1 r (1-s) + v2 r s + v3 (1-r) s,
 * with its Jacobian J[a*2 + k] = d x_a / d r_k (straight edges; the map is
 * linear along each edge). */
static int elem_is_bil(const orc_mesh *m, int64_t e) { return m->bil && m->bil[e]; }
static void bil_map(const real *X, real r, real s, real *x, real *J) {
  const real w[4] = {(1 - r) * (1 - s), r * (1 - s), r * s, (1 - r) * s};
  const real wr[4] = {-(1 - s), 1 - s, s, -s}, ws[4] = {-(1 - r), -r, r, 1 - r};
  for (int a = 0; a < 2; ++a) {
    real v = 0.0, vr = 0.0, vs = 0.0;
    for (int k = 0; k < 4; ++k) {
      v += w[k] * X[k * 2 + a];
      vr += wr[k] * X[k * 2 + a];
      vs += ws[k] * X[k * 2 + a];
    }
    if (x) x[a] = v;
    if (J) {
      J[a * 2] = vr;
      J[a * 2 + 1] = vs;
    }
  }
}
/* detJ and J^-1 (row k = gradient of r_k) of the bilinear map at (r, s) */
static real bil_jinv(const real *X, real r, real s, real *Ji) {
  real J[4];
  bil_map(X, r, s, NULL, J);
  const real det = J[0] * J[3] - J[1] * J[2];
  Ji[0] = J[3] / det;
  Ji[1] = -J[1] / det;
  Ji[2] = -J[2] / det;
  Ji[3] = J[0] / det;
  return det;
}

/* reference coordinates of physical point x in element e (nearest periodic
 * image of x to the element's centroid); a bilinear element's by Newton's
 * method from the affine guess (ten steps: quadratic convergence from a guess
 * within the element) */
static void ref_coords(const orc_mesh *m, int64_t e, const real *x, real *rs) {
  int dim = m->dim;
  const real *X = m->X + e * m->nvpe * dim;
  real xs[3];
  for (int a = 0; a < dim; ++a) {
    real cen = 0.0;
    for (int k = 0; k < m->nvpe; ++k) cen += X[k * dim + a];
    cen /= m->nvpe;
    xs[a] = x[a];
    if (m->periodic) xs[a] += m->L[a] * round((cen - x[a]) / m->L[a]);
  }
  const real *Ji = m->Jinv + e * dim * dim;
  for (int k = 0; k < dim; ++k) {
    real v = 0.0;
    for (int a = 0; a < dim; ++a) v += Ji[k * dim + a] * (xs[a] - X[a]);
    rs[k] = v;
  }
  if (elem_is_bil(m, e))
    for (int it = 0; it < 10; ++it) {
      real y[2], Jb[4];
      bil_map(X, rs[0], rs[1], y, NULL);
      bil_jinv(X, rs[0], rs[1], Jb);
      const real d0 = y[0] - xs[0], d1 = y[1] - xs[1];
      rs[0] -= Jb[0] * d0 + Jb[1] * d1;
      rs[1] -= Jb[2] * d0 + Jb[3] * d1;
    }
}

/* solve A x = b in place for nrhs right-hand sides (b[i * ldb + k], row i),
 * Gaussian elimination with partial pivoting; A (n x n, row-major) is destroyed */
static int dense_solve(int n, real *A, real *b, int nrhs, int ldb) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int i = c + 1; i < n; ++i)
      if (fabs(A[i * n + c]) > fabs(A[piv * n + c])) piv = i;
    if (!(fabs(A[piv * n + c]) > 0.0)) return -1;
    if (piv != c) {
      for (int j = 0; j < n; ++j) {
        real t = A[c * n + j];
        A[c * n + j] = A[piv * n + j];
        A[piv * n + j] = t;
      }
      for (int k = 0; k < nrhs; ++k) {
        real t = b[c * ldb + k];
        b[c * ldb + k] = b[piv * ldb + k];
        b[piv * ldb + k] = t;
      }
    }
    for (int i = c + 1; i < n; ++i) {
      const real f = A[i * n + c] / A[c * n + c];
      for (int j = c; j < n; ++j) A[i * n + j] -= f * A[c * n + j];
      for (int k = 0; k < nrhs; ++k) b[i * ldb + k] -= f * b[c * ldb + k];
    }
  }
  for (int c = n - 1; c >= 0; --c)
    for (int k = 0; k < nrhs; ++k) {
      real v = b[c * ldb + k];
      for (int j = c + 1; j < n; ++j) v -= A[c * n + j] * b[j * ldb + k];
      b[c * ldb + k] = v / A[c * n + c];
    }
  return 0;
}

/* a bilinear element's mass matrix M_ij = sum_q w_q detJ(x_q) phi_i phi_j over
 * the volume rule (exact: degree 2p+1 in each direction), into A[n x n] */
static void bil_mass(const orc_mesh *m, int64_t e, int p, int n, const real *vr, const real *vs, const real *vw,
                     int nvq, real *A) {
  const real *X = m->X + e * 8;
  for (int i = 0; i < n * n; ++i) A[i] = 0.0;
  for (int q = 0; q < nvq; ++q) {
    real Ji[4], x[3] = {vr[q], vs[q], 0.0}, phi[ORC_MAXNP];
    const real det = bil_jinv(X, vr[q], vs[q], Ji);
    basis_eval_e(m, e, p, x, phi, NULL, NULL, NULL);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) A[i * n + j] += vw[q] * det * phi[i] * phi[j];
  }
}

static void eval_state(const orc_mesh *m, int p, int M, int Np, const real *c, const real *rs,
                       real *U) {
  real phi[ORC_MAXNP];
  basis_eval(m, p, rs, phi, NULL, NULL, NULL);
  for (int k = 0; k < M; ++k) {
    real v = 0.0;
    for (int j = 0; j < Np; ++j) v += c[k * Np + j] * phi[j];
    U[k] = v;
  }
}

/* the state of element e (block c, stride Np per variable) at reference point rs,
 * in e's own space */
static void eval_state_e(const orc_mesh *m, int64_t e, int p, int M, int Np, const real *c, const real *rs,
                         real *U) {
  if (!(m->quad && !elem_is_quad(m, e))) {
    eval_state(m, p, M, Np, c, rs, U);
    return;
  }
  real phi[ORC_MAXNP];
  const int n = basis_eval_e(m, e, p, rs, phi, NULL, NULL, NULL);
  for (int k = 0; k < M; ++k) {
    real v = 0.0;
    for (int j = 0; j < n; ++j) v += c[k * Np + j] * phi[j];
    U[k] = v;
  }
}



/* Quadrature rules of one call, computed once.  Default sizes (reading, fixed
 * by the configurations' "7-pt edge / 16-pt area" at p = 3): triangle edges
 * 2p+1 Gauss points, triangle areas (p+1)^2; tetrahedron faces (p+2)^2,
 * volumes (p+2)^3; quadrilaterals as triangles, (p+1)^2 tensor Gauss points
 * on the square and 2p+1 on an edge.  Face points are given in the face's own parameters:
 * t in [0,1] along an edge, (sigma, tau) on a triangular face; face weights
 * sum to 1. */
typedef struct {
  int dim, nv, nf;
  real *vr, *vs, *vt, *vw;
  real *fa, *fb, *fw;
  /* quadrilateral (and hybrid) meshes: the triangle volume rule of the same
   * size, for the triangles of a hybrid mesh */
  int tnv;
  real *tvr, *tvs, *tvw;
} orc_rules;

static int default_face_n1(int dim, int p) { return dim == 2 ? 2 * p + 1 : p + 2; }
static int default_vol_n1(int dim, int p) { return dim == 2 ? p + 1 : p + 2; }

static void rules_free(orc_rules *R) {
  free(R->vr);
  free(R->vs);
  free(R->vt);
  free(R->vw);
  free(R->fa);
  free(R->fb);
  free(R->fw);
  free(R->tvr);
  free(R->tvs);
  free(R->tvw);
  memset(R, 0, sizeof *R);
}

static int rules_make(int dim, int quad, int nf1, int nv1, orc_rules *R) {
  memset(R, 0, sizeof *R);
  R->dim = dim;
  if (nf1 < 1 || nf1 > 64 || nv1 < 1 || nv1 > 64) return fail("rules: size out of range");
  R->nv = dim == 2 ? nv1 * nv1 : nv1 * nv1 * nv1;
  R->vr = (real *)malloc(sizeof(real) * R->nv);
  R->vs = (real *)malloc(sizeof(real) * R->nv);
  R->vt = (real *)calloc(R->nv, sizeof(real));
  R->vw = (real *)malloc(sizeof(real) * R->nv);
  int rc = quad ? orc_quad_rule(nv1, R->vr, R->vs, R->vw)
           : dim == 2 ? orc_tri_rule(nv1, R->vr, R->vs, R->vw)
                      : orc_tet_rule(nv1, R->vr, R->vs, R->vt, R->vw);
  if (rc) return rc;
  if (quad) {
    R->tnv = nv1 * nv1;
    R->tvr = (real *)malloc(sizeof(real) * R->tnv);
    R->tvs = (real *)malloc(sizeof(real) * R->tnv);
    R->tvw = (real *)malloc(sizeof(real) * R->tnv);
    if (orc_tri_rule(nv1, R->tvr, R->tvs, R->tvw)) return -1;
  }
  R->nf = dim == 2 ? nf1 : nf1 * nf1;
  R->fa = (real *)malloc(sizeof(real) * R->nf);
  R->fb = (real *)calloc(R->nf, sizeof(real));
  R->fw = (real *)malloc(sizeof(real) * R->nf);
  if (dim == 2) {
    real xg[64], wg[64];
    if (orc_gauss_legendre(nf1, xg, wg)) return -1;
    for (int i = 0; i < nf1; ++i) {
      R->fa[i] = 0.5 * (1.0 + xg[i]);
      R->fw[i] = 0.5 * wg[i];
    }
  } else {
    if (orc_tri_rule(nf1, R->fa, R->fb, R->fw)) return -1;
    for (int i = 0; i < R->nf; ++i) R->fw[i] *= 2.0;
  }
  return 0;
}

/* element e's volume rule */
static int vol_rule_e(const orc_rules *R, const orc_mesh *m, int64_t e, const real **vr, const real **vs,
                      const real **vt, const real **vw) {
  if (m->quad && !elem_is_quad(m, e)) {
    *vr = R->tvr, *vs = R->tvs, *vt = R->vt, *vw = R->tvw;
    return R->tnv;
  }
  *vr = R->vr, *vs = R->vs, *vt = R->vt, *vw = R->vw;
  return R->nv;
}

/* One face of element e, in physical space: its measure, its outward unit
 * normal (pointing away from the opposite vertex) and its quadrature points. */
typedef struct {
  int nq;
  real meas, n[3];
  real *x; /* nq * 3 */
  const real *w;
} orc_face;

static void face_geometry(const orc_mesh *m, int64_t e, int q, const orc_rules *R, orc_face *F) {
  int dim = m->dim;
  const real *X = m->X + e * m->nvpe * dim;
  int fv[3], nf = elem_nfaces(m, e);
  face_verts_e(m, e, q, fv);
  const real *A = X + fv[0] * dim, *B = X + fv[1] * dim;
  const real *O = dim == 2 ? X + ((q + 2) % nf) * dim : X + q * dim; /* a vertex off the face */
  real u[3] = {0, 0, 0}, v[3] = {0, 0, 0};
  for (int a = 0; a < dim; ++a) u[a] = B[a] - A[a];
  if (dim == 2) {
    F->meas = sqrt(u[0] * u[0] + u[1] * u[1]);
    F->n[0] = u[1] / F->meas;
    F->n[1] = -u[0] / F->meas;
    F->n[2] = 0.0;
  } else {
    const real *C = X + fv[2] * dim;
    for (int a = 0; a < 3; ++a) v[a] = C[a] - A[a];
    real cr[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
    real nn = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    F->meas = 0.5 * nn;
    for (int a = 0; a < 3; ++a) F->n[a] = cr[a] / nn;
  }
  real side = 0.0;
  for (int a = 0; a < dim; ++a) side += F->n[a] * (O[a] - A[a]);
  if (side > 0.0)
    for (int a = 0; a < dim; ++a) F->n[a] = -F->n[a];
  F->nq = R->nf;
  F->w = R->fw;
  for (int i = 0; i < R->nf; ++i)
    for (int a = 0; a < dim; ++a) F->x[i * 3 + a] = A[a] + R->fa[i] * u[a] + R->fb[i] * v[a];
}

/* Reading (Algorithm 1 evaluates one numerical flux per edge or face and adds
 * it to both elements): a face's quadrature points are the ones of its left
 * element's parameterisation of that face, for both elements.  On a triangle
 * edge the Gauss points are symmetric and either side gives the same points;
 * on a tetrahedral face the collapsed rule is not symmetric under a
 * permutation of the face's vertices, and a per-element choice would evaluate
 * the flux at different points on the two sides (not conservative). */
static void face_points_of_left(const orc_mesh *m, int64_t e, int32_t s, const orc_rules *R, orc_face *F) {
  int64_t l = m->sl[s];
  if (l == e) return;
  int dim = m->dim, fv[3];
  const real *X = m->X + l * m->nvpe * dim;
  face_verts_e(m, l, m->sql[s], fv);
  const real *A = X + fv[0] * dim, *B = X + fv[1] * dim, *C = dim == 3 ? X + fv[2] * dim : A;
  for (int i = 0; i < R->nf; ++i)
    for (int a = 0; a < dim; ++a)
      F->x[i * 3 + a] = A[a] + R->fa[i] * (B[a] - A[a]) + R->fb[i] * (C[a] - A[a]);
}

/* rhs[e][k][j] = d c_{e,k,j} / dt for the listed elements (all when
 * nelem < 0; then rhs is [E][M][Np], else [nelem][M][Np] in list order).
 * c is [E][M][Np] in original element order.  kind 0 = Euler, 1 = linear
 * advection with velocity adv.  nq_face1 / nq_vol1 override the 1-D point
 * counts (0 = defaults).  Boundary faces take U+ from bc_state: the
 * transmissive state U+ = U- unless orc_set_bc gave the face another kind. */
int orc_rhs(void *h, int p, int kind, const real *adv, const real *c, real *rhs,
            const int64_t *elems, int64_t nelem, int nq_face1, int nq_vol1) {
  orc_mesh *m = (orc_mesh *)h;
  int dim = m->dim;
  if (p < 0 || p > ORC_MAXP) return fail("rhs: p out of range");
  int Np = npoly_m(m, p);
  orc_phys ph = {kind, dim, kind == ORC_EULER ? dim + 2 : 1, {0, 0, 0}};
  if (m->bck && kind != ORC_EULER) return fail("rhs: boundary conditions are for the Euler system");
  if (adv)
    for (int a = 0; a < dim; ++a) ph.adv[a] = adv[a];
  int M = ph.M;
  orc_rules R;
  if (rules_make(dim, m->quad, nq_face1 > 0 ? nq_face1 : default_face_n1(dim, p),
                 nq_vol1 > 0 ? nq_vol1 : default_vol_n1(dim, p), &R)) {
    rules_free(&R);
    return -1;
  }
  int64_t count = nelem < 0 ? m->ne : nelem;
  /* elements are independent: the threaded build (-fopenmp) splits the list
   * across threads, each with its own face scratch; the arithmetic of each
   * element is the same as in the sequential build */
#ifdef _OPENMP
#pragma omp parallel
#endif
  {
  orc_face F;
  F.x = (real *)malloc(sizeof(real) * 3 * R.nf);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
  for (int64_t ii = 0; ii < count; ++ii) {
    int64_t e = nelem < 0 ? ii : elems[ii];
    const real *ce = c + e * M * Np;
    real *re = rhs + ii * M * Np;
    for (int i = 0; i < M * Np; ++i) re[i] = 0.0;
    const real *Ji = m->Jinv + e * dim * dim;
    const int Ne = npoly_e(m, e, p); /* the element's own modes (hybrid: fewer on a triangle) */
    const real *vr, *vs, *vt, *vw;
    const int nvq = vol_rule_e(&R, m, e, &vr, &vs, &vt, &vw);
    /* volume integral: sum_q w_q F(U_q) . (J^-T grad_ref phi_j); a bilinear
     * element weighs each point by its own detJ and J^-1 (and its mass matrix
     * is applied at the end), the others have the constant ones folded into
     * the mass matrix detJ I */
    const int bil = elem_is_bil(m, e);
    for (int q = 0; q < nvq; ++q) {
      real x[3] = {vr[q], vs[q], vt[q]};
      real phi[ORC_MAXNP], d[3][ORC_MAXNP], U[ORC_MAXM], Jq[4], wq = vw[q];
      if (bil) {
        wq *= bil_jinv(m->X + e * 8, vr[q], vs[q], Jq);
        Ji = Jq;
      }
      basis_eval_e(m, e, p, x, phi, d[0], d[1], d[2]);
      for (int k = 0; k < M; ++k) {
        real v = 0.0;
        for (int j = 0; j < Ne; ++j) v += ce[k * Np + j] * phi[j];
        U[k] = v;
      }
      for (int a = 0; a < dim; ++a) {
        real Fa[ORC_MAXM];
        phys_flux_dir(&ph, U, a, Fa);
        for (int j = 0; j < Ne; ++j) {
          real gx = 0.0; /* d phi_j / d x_a */
          for (int r = 0; r < dim; ++r) gx += Ji[r * dim + a] * d[r][j];
          for (int k = 0; k < M; ++k) re[k * Np + j] += wq * Fa[k] * gx;
        }
      }
    }
    /* surface integrals: - (1/detJ) sum_faces |f| sum_q w_q phi_j(x_q) F*(U_e, U_nb, n);
     * a coarse element's split edge is integrated as its two halves, each with
     * the points and length of the fine neighbour's edge (Sec. 3.2) */
    for (int sub = 0; sub < 2 * m->nfpe; ++sub) {
      int f = sub % m->nfpe;
      int32_t s = sub < m->nfpe ? m->es[e * m->nfpe + f] : (m->es2 ? m->es2[e * m->nfpe + f] : -1);
      if (s < 0) continue;
      face_geometry(m, e, f, &R, &F);  /* own outward normal and measure */
      face_points_of_left(m, e, s, &R, &F);
      int32_t nb = m->sl[s] == e ? m->sr[s] : m->sl[s];
      if (m->shalf && m->shalf[s] >= 0 && m->sr[s] == e) {
        const real *Xl = m->X + (int64_t)m->sl[s] * 6;
        int q = m->sql[s];
        real dx = Xl[((q + 1) % 3) * 2] - Xl[q * 2], dy = Xl[((q + 1) % 3) * 2 + 1] - Xl[q * 2 + 1];
        F.meas = sqrt(dx * dx + dy * dy);
      }
      real scale = elem_is_bil(m, e) ? F.meas : F.meas / m->detJ[e];
      for (int q = 0; q < F.nq; ++q) {
        real rs[3], Um[ORC_MAXM], Up[ORC_MAXM], Fs[ORC_MAXM], phi[ORC_MAXNP];
        ref_coords(m, e, F.x + 3 * q, rs);
        eval_state_e(m, e, p, M, Np, ce, rs, Um);
        if (nb >= 0) {
          real rn[3];
          ref_coords(m, nb, F.x + 3 * q, rn);
          eval_state_e(m, nb, p, M, Np, c + (int64_t)nb * M * Np, rn, Up);
        } else {
          bc_state(m, s, M, Um, F.n, F.x + 3 * q, Up);
        }
        num_flux(&ph, Um, Up, F.n, Fs);
        basis_eval_e(m, e, p, rs, phi, NULL, NULL, NULL);
        for (int j = 0; j < Ne; ++j)
          for (int k = 0; k < M; ++k) re[k * Np + j] -= scale * F.w[q] * phi[j] * Fs[k];
      }
    }
    if (bil) {
      /* dc/dt = M^-1 (volume - surface) with the element's own mass matrix */
      real *A = (real *)malloc(sizeof(real) * Ne * Ne), *b = (real *)malloc(sizeof(real) * Ne * M);
      bil_mass(m, e, p, Ne, vr, vs, vw, nvq, A);
      for (int j = 0; j < Ne; ++j)
        for (int k = 0; k < M; ++k) b[j * M + k] = re[k * Np + j];
      dense_solve(Ne, A, b, M, M);
      for (int j = 0; j < Ne; ++j)
        for (int k = 0; k < M; ++k) re[k * Np + j] = b[j * M + k];
      free(A);
      free(b);
    }
  }
  free(F.x);
  }
  rules_free(&R);
  return 0;
}

/* threads the element loop of orc_rhs uses (threaded build only); returns
 * the count in effect, 1 in the sequential build */
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ======================================================================= */
/* Limiter (reading: the paper's solver takes its limiter from [giuliani])  */
/* ======================================================================= */
/* The Barth-Jespersen limiter on the conserved variables, one variable at a
 * time.  On element e with mean u_e (its mode-0 coefficient times phi_0):
 * u_min, u_max = the least and greatest of u_e and the means of the elements
 * across its faces (both halves of a split face); d_i = u(x_i) - u_e =
 * sum_{j>=1} c_j phi_j(x_i) at the element's vertices and volume points; then
 *   alpha = min(1, min over d_i > 0 of (u_max - u_e) / d_i,
 *                  min over d_i < 0 of (u_min - u_e) / d_i)
 * and every mode j >= 1 is multiplied by alpha.  The means never change, so the
 * result does not depend on the order the elements are visited in; at p = 1 the
 * limited polynomial lies within [u_min, u_max] on the whole element (a linear
 * function takes its extremes at the vertices). */
int orc_limit(void *h, int p, real *c) {
  orc_mesh *m = (orc_mesh *)h;
  if (m->dim != 2 || m->quad) return fail("limit: triangle meshes only");
  if (p < 1 || p > ORC_MAXP) return fail("limit: p out of range");
  const int M = 4, Np = npoly_tri(p);
  orc_rules R;
  if (rules_make(2, 0, 1, default_vol_n1(2, p), &R)) {
    rules_free(&R);
    return -1;
  }
  const int npt = 3 + R.nv;
  real *phi = (real *)malloc(sizeof(real) * npt * Np), *mean = (real *)malloc(sizeof(real) * m->ne * M);
  for (int i = 0; i < npt; ++i) {
    real x[3] = {i == 1 ? 1.0 : 0.0, i == 2 ? 1.0 : 0.0, 0.0};
    if (i >= 3) x[0] = R.vr[i - 3], x[1] = R.vs[i - 3];
    basis_eval(m, p, x, phi + i * Np, NULL, NULL, NULL);
  }
  const real phi0 = phi[0];
  for (int64_t e = 0; e < m->ne; ++e)
    for (int k = 0; k < M; ++k) mean[e * M + k] = c[(e * M + k) * Np] * phi0;
  for (int64_t e = 0; e < m->ne; ++e) {
    for (int k = 0; k < M; ++k) {
      const real ue = mean[e * M + k];
      real lo = ue, hi = ue;
      for (int sub = 0; sub < 2 * m->nfpe; ++sub) {
        const int f = sub % m->nfpe;
        const int32_t s = sub < m->nfpe ? m->es[e * m->nfpe + f] : (m->es2 ? m->es2[e * m->nfpe + f] : -1);
        if (s < 0) continue;
        const int32_t nb = m->sl[s] == e ? m->sr[s] : m->sl[s];
        if (nb < 0) continue;
        const real v = mean[(int64_t)nb * M + k];
        if (v < lo) lo = v;
        if (v > hi) hi = v;
      }
      real *ce = c + (e * M + k) * Np;
      real alpha = 1.0;
      for (int i = 0; i < npt; ++i) {
        real d = 0.0;
        for (int j = 1; j < Np; ++j) d += ce[j] * phi[i * Np + j];
        if (d > 0.0 && (hi - ue) / d < alpha) alpha = (hi - ue) / d;
        if (d < 0.0 && (lo - ue) / d < alpha) alpha = (lo - ue) / d;
      }
      for (int j = 1; j < Np; ++j) ce[j] *= alpha;
    }
  }
  free(phi);
  free(mean);
  rules_free(&R);
  return 0;
}

/* ======================================================================= */
/* Time step and SSP-RK3 (readings; the paper defers the solver to [giuliani]) */
/* ======================================================================= */
/* dt = cfl * min_i r_i / ((2p+1) lambda_i); r_i = dim |element| / |boundary|
 * (the inradius), lambda_i = max over the element's volume points of |u|+c. */
int orc_dt(void *h, int p, const real *c, real cfl, real *dt_out) {
  orc_mesh *m = (orc_mesh *)h;
  int dim = m->dim, M = dim + 2, Np = npoly_m(m, p);
  orc_rules R;
  if (rules_make(dim, m->quad, 1, default_vol_n1(dim, p), &R)) {
    rules_free(&R);
    return -1;
  }
  orc_face F;
  F.x = (real *)malloc(sizeof(real) * 3 * R.nf);
  real best = INFINITY;
  for (int64_t e = 0; e < m->ne; ++e) {
    real lam = 0.0;
    const real *vr, *vs, *vt, *vw;
    const int nvq = vol_rule_e(&R, m, e, &vr, &vs, &vt, &vw);
    for (int q = 0; q < nvq; ++q) {
      real x[3] = {vr[q], vs[q], vt[q]}, U[ORC_MAXM];
      eval_state_e(m, e, p, M, Np, c + e * M * Np, x, U);
      real rho = U[0], q2 = 0.0;
      for (int a = 0; a < dim; ++a) q2 += (U[1 + a] / rho) * (U[1 + a] / rho);
      real pr = (ORC_GAMMA - 1.0) * (U[dim + 1] - 0.5 * rho * q2);
      real l = sqrt(q2) + sqrt(ORC_GAMMA * pr / rho);
      if (l > lam) lam = l;
    }
    real bnd = 0.0;
    for (int f = 0; f < elem_nfaces(m, e); ++f) {
      face_geometry(m, e, f, &R, &F);
      bnd += F.meas;
    }
    real vol = m->detJ[e] / (elem_is_quad(m, e) ? 1.0 : dim == 2 ? 2.0 : 6.0);
    if (elem_is_bil(m, e)) { /* the area, the integral of the bilinear map's detJ */
      vol = 0.0;
      for (int q = 0; q < nvq; ++q) {
        real Jq[4];
        vol += vw[q] * bil_jinv(m->X + e * 8, vr[q], vs[q], Jq);
      }
    }
    real r = dim * vol / bnd;
    real v = r / ((2 * p + 1) * lam);
    if (v < best) best = v;
  }
  free(F.x);
  rules_free(&R);
  *dt_out = cfl * best;
  return 0;
}

/* One SSP-RK3 (Shu-Osher) step, in place:
 *   u1 = u + dt L(u);  u2 = 3/4 u + 1/4 (u1 + dt L(u1));
 *   u  = 1/3 u + 2/3 (u2 + dt L(u2)),
 * with L the right-hand side of Eq. 2 for the flux kind (ORC_EULER, or
 * ORC_ADVECTION with velocity adv and one equation).  dt comes from the
 * state at the start of the step (Euler only), or is dt_in when > 0.  The
 * stages take their boundary states at t, t + dt and t + dt/2 (t the mesh's
 * time, advanced by dt), and with the limiter on (orc_set_limiter) each stage's
 * result is limited (orc_limit) before the next stage reads it. */
int orc_rk_step_kind(void *h, int p, int kind, const real *adv, real *c, real cfl, real dt_in,
                     real *dt_out) {
  orc_mesh *m = (orc_mesh *)h;
  int dim = m->dim, M = kind == ORC_EULER ? dim + 2 : 1, Np = npoly_m(m, p);
  int64_t n = m->ne * M * Np;
  real dt = dt_in;
  if (!(dt > 0.0)) {
    if (kind != ORC_EULER) return fail("rk_step: the advection form needs dt_in > 0");
    if (orc_dt(h, p, c, cfl, &dt)) return -1;
  }
  real *u1 = (real *)malloc(sizeof(real) * n), *u2 = (real *)malloc(sizeof(real) * n);
  real *L = (real *)malloc(sizeof(real) * n);
  /* stage times t, t + dt, t + dt/2 (for time-dependent boundary states); the
   * limiter, when on, after every stage */
  const real t0 = m->time;
  const int lim = m->limit && kind == ORC_EULER;
  int rc = orc_rhs(h, p, kind, adv, c, L, NULL, -1, 0, 0);
  for (int64_t i = 0; i < n && !rc; ++i) u1[i] = c[i] + dt * L[i];
  if (!rc && lim) rc = orc_limit(h, p, u1);
  m->time = t0 + dt;
  if (!rc) rc = orc_rhs(h, p, kind, adv, u1, L, NULL, -1, 0, 0);
  for (int64_t i = 0; i < n && !rc; ++i) u2[i] = 0.75 * c[i] + 0.25 * (u1[i] + dt * L[i]);
  if (!rc && lim) rc = orc_limit(h, p, u2);
  m->time = t0 + 0.5 * dt;
  if (!rc) rc = orc_rhs(h, p, kind, adv, u2, L, NULL, -1, 0, 0);
  for (int64_t i = 0; i < n && !rc; ++i) c[i] = c[i] / 3.0 + (real)2 / 3 * (u2[i] + dt * L[i]);
  if (!rc && lim) rc = orc_limit(h, p, c);
  m->time = t0 + dt;
  free(u1);
  free(u2);
  free(L);
  if (dt_out) *dt_out = dt;
  return rc;
}

/* the Euler system's step */
int orc_rk_step(void *h, int p, real *c, real cfl, real dt_in, real *dt_out) {
  return orc_rk_step_kind(h, p, ORC_EULER, NULL, c, cfl, dt_in, dt_out);
}

/* ======================================================================= */
/* State transfer between a mesh and its one-level refinement (Sec. 3.2)   */
/* ======================================================================= */
/* coarse: the mesh before refinement, fine: orc_refine(coarse, ., flag), whose
 * children of coarse element e are fine elements first(e) .. first(e) + 3 (an
 * unrefined element is one fine element).  States [E][M][Np], each element's
 * coefficients w.r.t. its own reference-orthonormal basis.
 *   dir 0, prolongation: a child's coefficients are the L2 projection of its
 *     parent's polynomial onto the child, d_j = sum_q w_q u(x_q) phi_j(rho_q)
 *     over the child's volume rule (exact: the integrand has degree 2p);
 *   dir 1, restriction: a parent's coefficients are the L2 projection of its
 *     children's piecewise polynomial, c_k = sum_children (detJ_child /
 *     detJ_parent) sum_q w_q u_child(rho_q) phi_k(r_parent(x_q)), each child
 *     integrated with its own rule.
 * Points are mapped through physical space: a child's reference point to its
 * physical point, then the parent's reference coordinates by inverting the
 * parent's affine map. */
int orc_transfer(void *hc, void *hf, const uint8_t *flag, int p, int M, int dir, const real *cin, real *cout) {
  const orc_mesh *mc = (const orc_mesh *)hc, *mf = (const orc_mesh *)hf;
  if (mc->dim != 2 || mc->quad || mf->dim != 2) return fail("transfer: triangle meshes only");
  const int Np = npoly_tri(p);
  orc_rules R;
  if (rules_make(2, 0, 1, default_vol_n1(2, p), &R)) {
    rules_free(&R);
    return -1;
  }
  int64_t n = 0;
  for (int64_t e = 0; e < mc->ne; ++e) {
    const int kids = flag[e] ? 4 : 1;
    if (n + kids > mf->ne) {
      rules_free(&R);
      return fail("transfer: the meshes do not match the flags");
    }
    if (!flag[e]) {
      const real *src = cin + (dir == 0 ? e : n) * M * Np;
      real *dst = cout + (dir == 0 ? n : e) * M * Np;
      for (int i = 0; i < M * Np; ++i) dst[i] = src[i];
      n += 1;
      continue;
    }
    const real *ce = dir == 0 ? cin + e * M * Np : NULL;
    real *pe = dir == 1 ? cout + e * M * Np : NULL;
    if (pe)
      for (int i = 0; i < M * Np; ++i) pe[i] = 0.0;
    for (int c = 0; c < 4; ++c, ++n) {
      const real *Xc = mf->X + n * 6;
      real *de = dir == 0 ? cout + n * M * Np : NULL;
      const real *dc = dir == 1 ? cin + n * M * Np : NULL;
      if (de)
        for (int i = 0; i < M * Np; ++i) de[i] = 0.0;
      const real ratio = mf->detJ[n] / mc->detJ[e];
      for (int q = 0; q < R.nv; ++q) {
        real rho[3] = {R.vr[q], R.vs[q], 0.0}, x[3], rs[3], phi[ORC_MAXNP], U[ORC_MAXM];
        for (int a = 0; a < 2; ++a) x[a] = Xc[a] + (Xc[2 + a] - Xc[a]) * rho[0] + (Xc[4 + a] - Xc[a]) * rho[1];
        ref_coords(mc, e, x, rs);
        if (dir == 0) {
          eval_state(mc, p, M, Np, ce, rs, U);  /* the parent's polynomial at the child's point */
          basis_eval(mf, p, rho, phi, NULL, NULL, NULL);
          for (int k = 0; k < M; ++k)
            for (int j = 0; j < Np; ++j) de[k * Np + j] += R.vw[q] * U[k] * phi[j];
        } else {
          eval_state(mf, p, M, Np, dc, rho, U);  /* the child's polynomial at its own point */
          basis_eval(mc, p, rs, phi, NULL, NULL, NULL);
          for (int k = 0; k < M; ++k)
            for (int j = 0; j < Np; ++j) pe[k * Np + j] += ratio * R.vw[q] * U[k] * phi[j];
        }
      }
    }
  }
  rules_free(&R);
  if (n != mf->ne) return fail("transfer: the meshes do not match the flags");
  return 0;
}

/* ======================================================================= */
/* Initial conditions: L2 projection onto the orthonormal basis             */
/* ======================================================================= */
int orc_num_vol_points(int dim, int p) {
  int n1 = default_vol_n1(dim, p);
  return dim == 2 ? n1 * n1 : n1 * n1 * n1;
}

/* physical coordinates (unwrapped per element) of the volume points of a
 * rule with n1 points per direction (0 = default), [E][Nq][dim]; optional
 * physical weights [E][Nq] and DG solution values U [E][Nq][M] of c. */
int orc_eval_points(void *h, int p, int M, const real *c, int n1, real *xyz, real *w,
                    real *U) {
  orc_mesh *m = (orc_mesh *)h;
  int dim = m->dim, Np = npoly_m(m, p);
  orc_rules R;
  if (rules_make(dim, m->quad, 1, n1 > 0 ? n1 : default_vol_n1(dim, p), &R)) {
    rules_free(&R);
    return -1;
  }
  for (int64_t e = 0; e < m->ne; ++e) {
    /* the reference axes run from v0 to v1, v2 (simplices) or v1, v3 (quadrilaterals) */
    const int kv[3] = {1, elem_is_quad(m, e) ? 3 : 2, 3};
    const real *X = m->X + e * m->nvpe * dim;
    const real *vr, *vs, *vt, *vw;
    vol_rule_e(&R, m, e, &vr, &vs, &vt, &vw);
    for (int q = 0; q < R.nv; ++q) {
      real rs[3] = {vr[q], vs[q], vt[q]}, det = m->detJ[e];
      for (int a = 0; a < dim; ++a) {
        real v = X[a];
        for (int k = 0; k < dim; ++k) v += (X[kv[k] * dim + a] - X[a]) * rs[k];
        if (xyz) xyz[(e * R.nv + q) * dim + a] = v;
      }
      if (elem_is_bil(m, e)) {
        real y[2], Jq[4];
        bil_map(X, rs[0], rs[1], y, NULL);
        det = bil_jinv(X, rs[0], rs[1], Jq);
        if (xyz)
          for (int a = 0; a < 2; ++a) xyz[(e * R.nv + q) * dim + a] = y[a];
      }
      if (w) w[e * R.nv + q] = vw[q] * det;
      if (U) eval_state_e(m, e, p, M, Np, c + e * M * Np, rs, U + (e * R.nv + q) * M);
    }
  }
  int nq = R.nv;
  rules_free(&R);
  return nq;
}

/* L2 projection: with a basis orthonormal on the reference element the
 * coefficients are c[e][k][j] = sum_q w_q U_k(x_q) phi_j(x_q) over the
 * default volume rule; vals is [E][Nq][M] at the points of orc_eval_points. */
int orc_project(void *h, int p, int M, const real *vals, real *c) {
  orc_mesh *m = (orc_mesh *)h;
  int dim = m->dim, Np = npoly_m(m, p);
  orc_rules R;
  if (rules_make(dim, m->quad, 1, default_vol_n1(dim, p), &R)) {
    rules_free(&R);
    return -1;
  }
  for (int64_t e = 0; e < m->ne; ++e) {
    real *ce = c + e * M * Np;
    for (int i = 0; i < M * Np; ++i) ce[i] = 0.0;
    const real *vr, *vs, *vt, *vw;
    vol_rule_e(&R, m, e, &vr, &vs, &vt, &vw);
    const int Ne = npoly_e(m, e, p), bil = elem_is_bil(m, e);
    for (int q = 0; q < R.nv; ++q) {
      real x[3] = {vr[q], vs[q], vt[q]}, phi[ORC_MAXNP], wq = vw[q];
      if (bil) {
        real Jq[4];
        wq *= bil_jinv(m->X + e * 8, vr[q], vs[q], Jq);
      }
      basis_eval_e(m, e, p, x, phi, NULL, NULL, NULL);
      for (int k = 0; k < M; ++k)
        for (int j = 0; j < Ne; ++j) ce[k * Np + j] += wq * vals[(e * R.nv + q) * M + k] * phi[j];
    }
    if (bil) { /* the L2 projection of a bilinear element: M c = sum w detJ u phi */
      real *A = (real *)malloc(sizeof(real) * Ne * Ne), *b = (real *)malloc(sizeof(real) * Ne * M);
      bil_mass(m, e, p, Ne, vr, vs, vw, R.nv, A);
      for (int j = 0; j < Ne; ++j)
        for (int k = 0; k < M; ++k) b[j * M + k] = ce[k * Np + j];
      dense_solve(Ne, A, b, M, M);
      for (int j = 0; j < Ne; ++j)
        for (int k = 0; k < M; ++k) ce[k * Np + j] = b[j * M + k];
      free(A);
      free(b);
    }
  }
  rules_free(&R);
  return 0;
}
