"""Pins for the oracle's quadrature rules and modal basis.

Each check ties the oracle to something other than itself: a library routine
(numpy / scipy Gauss rules), a closed form (monomial integrals over the
reference simplex), or a property any correct orthonormal modal basis has
(orthonormality via exact monomial integration, polynomial degree per mode,
derivatives against finite differences).
"""

from math import factorial

import numpy as np
import pytest
import scipy.special as sp


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 12, 30])
def test_gauss_legendre_matches_numpy(oracle_mod, n):
    x, w = oracle_mod.gauss_jacobi(n, 0.0)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, xr, atol=1e-14)
    np.testing.assert_allclose(w, wr, atol=1e-14)


@pytest.mark.parametrize("a", [1.0, 2.0])
@pytest.mark.parametrize("n", [1, 2, 4, 7, 16])
def test_gauss_jacobi_matches_scipy(oracle_mod, n, a):
    x, w = oracle_mod.gauss_jacobi(n, a)
    xr, wr = sp.roots_jacobi(n, a, 0.0)
    np.testing.assert_allclose(x, xr, atol=1e-13)
    np.testing.assert_allclose(w, wr, rtol=1e-12)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6])
def test_tri_rule_exact_monomials(oracle_mod, n):
    """int_T r^a s^b = a! b! / (a+b+2)! for a+b <= 2n-1 (collapsed Gauss rule)."""
    r, s, w = oracle_mod.tri_rule(n)
    for a in range(2 * n):
        for b in range(2 * n - a):
            exact = factorial(a) * factorial(b) / factorial(a + b + 2)
            assert abs(np.sum(w * r ** a * s ** b) - exact) < 1e-15 + 1e-13 * exact


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_tet_rule_exact_monomials(oracle_mod, n):
    r, s, t, w = oracle_mod.tet_rule(n)
    for a in range(2 * n):
        for b in range(2 * n - a):
            for c in range(2 * n - a - b):
                exact = factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 3)
                assert abs(np.sum(w * r ** a * s ** b * t ** c) - exact) < 1e-15 + 1e-13 * exact


def test_config_rule_sizes(oracle_mod):
    """p = 3 triangles: 7-point edge rule and 16-point area rule (configuration 2)."""
    p = 3
    x, _ = oracle_mod.gauss_jacobi(2 * p + 1, 0.0)
    r, _, _ = oracle_mod.tri_rule(p + 1)
    assert x.size == 7 and r.size == 16


def _monomials_2d(deg, r, s):
    cols, exps = [], []
    for d in range(deg + 1):
        for a in range(d + 1):
            cols.append(r ** (d - a) * s ** a)
            exps.append((d - a, a))
    return np.stack(cols, axis=1), exps


def _monomials_3d(deg, r, s, t):
    cols, exps = [], []
    for d in range(deg + 1):
        for a in range(d + 1):
            for b in range(d - a + 1):
                c = d - a - b
                cols.append(r ** a * s ** b * t ** c)
                exps.append((a, b, c))
    return np.stack(cols, axis=1), exps


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4, 5])
def test_tri_basis_orthonormal_by_exact_monomial_integration(oracle_mod, p):
    """Fit each phi_j exactly by monomials (it must be a polynomial of degree <= p),
    then integrate phi_i phi_j in closed form: the Gram matrix must be I."""
    rng = np.random.default_rng(p)
    u = rng.uniform(size=(400, 2))
    r = np.minimum(u[:, 0], u[:, 1])
    s = np.abs(u[:, 0] - u[:, 1])
    phi, _, _ = oracle_mod.basis_tri(p, r, s)
    V, exps = _monomials_2d(p, r, s)
    coef, *_ = np.linalg.lstsq(V, phi, rcond=None)
    assert np.abs(V @ coef - phi).max() < 1e-10  # a polynomial of degree <= p
    n = len(exps)
    Mmat = np.zeros((n, n))
    for i, (a1, b1) in enumerate(exps):
        for j, (a2, b2) in enumerate(exps):
            a, b = a1 + a2, b1 + b2
            Mmat[i, j] = factorial(a) * factorial(b) / factorial(a + b + 2)
    G = coef.T @ Mmat @ coef
    np.testing.assert_allclose(G, np.eye(G.shape[0]), atol=1e-10)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_tri_basis_hierarchical_degrees(oracle_mod, p):
    """phi_j with index in degree block d has total degree exactly d, and the
    first (d+1)(d+2)/2 functions span all polynomials of degree <= d."""
    rng = np.random.default_rng(10 + p)
    u = rng.uniform(size=(300, 2))
    r = np.minimum(u[:, 0], u[:, 1])
    s = np.abs(u[:, 0] - u[:, 1])
    phi, _, _ = oracle_mod.basis_tri(p, r, s)
    j = 0
    for d in range(p + 1):
        nd = (d + 1) * (d + 2) // 2
        V, _ = _monomials_2d(d, r, s)
        # the span of phi_0..phi_{nd-1} equals the monomials of degree <= d
        assert np.linalg.matrix_rank(phi[:, :nd], tol=1e-9) == nd
        coef, *_ = np.linalg.lstsq(V, phi[:, j:nd], rcond=None)
        assert np.abs(V @ coef - phi[:, j:nd]).max() < 1e-10
        if d > 0:
            Vl, _ = _monomials_2d(d - 1, r, s)
            coef, *_ = np.linalg.lstsq(Vl, phi[:, j:nd], rcond=None)
            assert np.abs(Vl @ coef - phi[:, j:nd]).max() > 1e-3  # genuinely degree d
        j = nd
    np.testing.assert_allclose(phi[:, 0], np.sqrt(2.0), rtol=1e-15)


@pytest.mark.parametrize("p", [1, 3, 5])
def test_tri_basis_gradients_finite_difference(oracle_mod, p):
    rng = np.random.default_rng(20 + p)
    r = rng.uniform(0.05, 0.45, 25)
    s = rng.uniform(0.05, 0.45, 25)
    h = 1e-6
    _, dr, ds = oracle_mod.basis_tri(p, r, s)
    fd_r = (oracle_mod.basis_tri(p, r + h, s)[0] - oracle_mod.basis_tri(p, r - h, s)[0]) / (2 * h)
    fd_s = (oracle_mod.basis_tri(p, r, s + h)[0] - oracle_mod.basis_tri(p, r, s - h)[0]) / (2 * h)
    np.testing.assert_allclose(dr, fd_r, atol=1e-6 * (1 + np.abs(dr).max()))
    np.testing.assert_allclose(ds, fd_s, atol=1e-6 * (1 + np.abs(ds).max()))


@pytest.mark.parametrize("p", [0, 1, 2, 3])
def test_tet_basis_orthonormal_by_exact_monomial_integration(oracle_mod, p):
    rng = np.random.default_rng(30 + p)
    u = np.sort(rng.uniform(size=(600, 3)), axis=1)
    r, s, t = u[:, 0], u[:, 1] - u[:, 0], u[:, 2] - u[:, 1]
    phi, _, _, _ = oracle_mod.basis_tet(p, r, s, t)
    V, exps = _monomials_3d(p, r, s, t)
    coef, *_ = np.linalg.lstsq(V, phi, rcond=None)
    assert np.abs(V @ coef - phi).max() < 1e-9
    n = len(exps)
    Mmat = np.zeros((n, n))
    for i, e1 in enumerate(exps):
        for j, e2 in enumerate(exps):
            a, b, c = (e1[k] + e2[k] for k in range(3))
            Mmat[i, j] = factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 3)
    G = coef.T @ Mmat @ coef
    np.testing.assert_allclose(G, np.eye(G.shape[0]), atol=1e-9)
    np.testing.assert_allclose(phi[:, 0], np.sqrt(6.0), rtol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_tet_basis_gradients_finite_difference(oracle_mod, p):
    rng = np.random.default_rng(40 + p)
    r, s, t = (rng.uniform(0.05, 0.3, 15) for _ in range(3))
    h = 1e-6
    _, dr, ds, dt = oracle_mod.basis_tet(p, r, s, t)
    B = lambda a, b, c: oracle_mod.basis_tet(p, a, b, c)[0]
    for g, fd in ((dr, (B(r + h, s, t) - B(r - h, s, t)) / (2 * h)),
                  (ds, (B(r, s + h, t) - B(r, s - h, t)) / (2 * h)),
                  (dt, (B(r, s, t + h) - B(r, s, t - h)) / (2 * h))):
        np.testing.assert_allclose(g, fd, atol=1e-6 * (1 + np.abs(g).max()))
