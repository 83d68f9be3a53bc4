"""Pins for the oracle's right-hand side (Eq. 2), flux, CFL rule and SSP-RK3.

* freestream preservation: a constant state has a zero right-hand side;
* conservation: on a periodic mesh the face contributions cancel, so the total
  of the mean modes does not change;
* linear advection, a closed form: for F = a u and a global polynomial u of
  degree p (no jumps), Eq. 2 reproduces exactly -a.grad(u), a polynomial of
  degree p-1 the basis represents;
* brute force: for linear advection every integrand is a polynomial the default
  rules integrate exactly, so 30-point rules give the same result;
* L2 stability: with the upwind flux the discrete energy cannot grow;
* hand-computed Euler flux values and the conservation property of the
  Lax-Friedrichs flux;
* design order p+1 of the whole scheme on the isentropic vortex.
"""

import numpy as np
import pytest

from paper_1601_07613_gb300 import workloads as W


def _const_state(ne, np_, dim):
    ub = np.array([1.1, 0.3, -0.2, 2.6]) if dim == 2 else np.array([1.1, 0.3, -0.2, 0.15, 2.6])
    c = np.zeros((ne, dim + 2, np_))
    c[:, :, 0] = ub / (np.sqrt(2.0) if dim == 2 else np.sqrt(6.0))
    return c, ub


@pytest.mark.parametrize("p", [0, 1, 2, 3])
@pytest.mark.parametrize("kind", ["periodic", "open"])
def test_freestream_tri(oracle_mod, p, kind):
    mi = (W.periodic_square_tri(12, jitter=0.2, seed=5) if kind == "periodic"
          else W.open_square_tri(12, jitter=0.2, seed=5))
    m = oracle_mod.OracleMesh.from_input(mi)
    c, ub = _const_state(m.ne, oracle_mod.npoly(2, p), 2)
    rhs = m.rhs(p, c)
    # scale-normalised: |rhs| detJ / (perimeter max|F|) (rhs scales as |F| / h)
    h = 1.0 / 12
    fmax = 3.0  # max |F| component of the state above
    assert np.abs(rhs).max() * (0.5 * h * h) / (3.4 * h * fmax) < 1e-13


@pytest.mark.parametrize("p", [1, 2])
def test_freestream_tet(oracle_mod, p):
    m = oracle_mod.OracleMesh.from_input(W.periodic_cube_tet(3))
    c, _ = _const_state(m.ne, oracle_mod.npoly(3, p), 3)
    assert np.abs(m.rhs(p, c)).max() < 1e-12


@pytest.mark.parametrize("p", [1, 3])
def test_conservation_periodic(oracle_mod, p):
    m = oracle_mod.OracleMesh.from_input(W.periodic_square_tri(10, jitter=0.2, seed=6))
    c = W.random_state(m.ne, 4, oracle_mod.npoly(2, p), seed=p, amp=2e-2)
    rhs = m.rhs(p, c)
    detj = m.detj()
    total = (detj[:, None] * rhs[:, :, 0]).sum(axis=0)
    scale = (detj[:, None] * np.abs(rhs[:, :, 0])).sum(axis=0)
    assert np.all(np.abs(total) < 1e-13 * scale)


def _poly2(deg, coef, x, y):
    v = np.zeros_like(x)
    gx = np.zeros_like(x)
    gy = np.zeros_like(x)
    k = 0
    for d in range(deg + 1):
        for a in range(d + 1):
            b = d - a
            v += coef[k] * x ** a * y ** b
            if a:
                gx += coef[k] * a * x ** (a - 1) * y ** b
            if b:
                gy += coef[k] * b * x ** a * y ** (b - 1)
            k += 1
    return v, gx, gy


@pytest.mark.parametrize("p", [1, 2, 3])
def test_linear_advection_global_polynomial_closed_form(oracle_mod, p):
    """u continuous polynomial of degree p => d u_h/dt = -a.grad u exactly."""
    m = oracle_mod.OracleMesh.from_input(W.open_square_tri(6, jitter=0.2, seed=7))
    a = np.array([0.7, -1.3])
    coef = np.random.default_rng(p).uniform(-1, 1, size=(p + 1) * (p + 2) // 2)
    xyz, _, _ = m.eval_points(p, M=1)
    u, _, _ = _poly2(p, coef, xyz[..., 0], xyz[..., 1])
    c = m.project(p, u[..., None])
    rhs = m.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a)
    # evaluate the result at independent points and compare with -a.grad u
    xyz2, _, U = m.eval_points(p, c=rhs, n1=p + 3)
    _, gx, gy = _poly2(p, coef, xyz2[..., 0], xyz2[..., 1])
    np.testing.assert_allclose(U[..., 0], -(a[0] * gx + a[1] * gy), atol=1e-11)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_linear_advection_brute_force_quadrature(oracle_mod, p):
    """Discontinuous data, linear flux: default rules equal 30-point rules."""
    m = oracle_mod.OracleMesh.from_input(W.periodic_square_tri(5, jitter=0.2, seed=8))
    c = np.random.default_rng(p).uniform(-1, 1, size=(m.ne, 1, oracle_mod.npoly(2, p)))
    a = np.array([0.4, 0.9])
    r0 = m.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a)
    r1 = m.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a, nq_face1=30, nq_vol1=30)
    np.testing.assert_allclose(r0, r1, atol=1e-12 * np.abs(r1).max())


def test_euler_brute_force_quadrature_converges(oracle_mod):
    """Euler integrands are rational: the default rules differ from 30-point
    rules by a small quadrature error, which drops when the rules are refined."""
    m = oracle_mod.OracleMesh.from_input(W.periodic_square_tri(6, jitter=0.2, seed=9))
    for p in (1, 2, 3):
        c = W.random_state(m.ne, 4, oracle_mod.npoly(2, p), seed=p, amp=2e-3)
        r1 = m.rhs(p, c, nq_face1=30, nq_vol1=30)
        e0 = np.linalg.norm(m.rhs(p, c) - r1) / np.linalg.norm(r1)
        e1 = np.linalg.norm(m.rhs(p, c, nq_face1=2 * p + 3, nq_vol1=p + 2) - r1) / np.linalg.norm(r1)
        assert e0 < 1e-3 and e1 < e0


def test_linear_advection_energy_stable(oracle_mod):
    """Upwind DG: d/dt ||u_h||^2 = -sum_f |a.n| int [u]^2 <= 0 (periodic)."""
    m = oracle_mod.OracleMesh.from_input(W.periodic_square_tri(8, jitter=0.2, seed=10))
    c = np.random.default_rng(3).uniform(-1, 1, size=(m.ne, 1, 6))
    rhs = m.rhs(2, c, kind=oracle_mod.ADVECTION, adv=np.array([1.0, 0.5]))
    rate = np.sum(m.detj()[:, None, None] * c * rhs)
    assert rate < -1e-3


def test_euler_flux_hand_values(oracle_mod):
    # rest state rho=1, E=2.5 -> p = 1, F.n = (0, p n, 0)
    U = np.array([1.0, 0.0, 0.0, 2.5])
    np.testing.assert_allclose(oracle_mod.lf_flux(2, U, U, np.array([1.0, 0.0])), [0, 1, 0, 0],
                               atol=1e-15)
    # u = 0.5, v = -0.2, p = 0.4 (3 - 0.5*1.2*0.29) = 1.1304, u.n = 0.14 with n = (0.6, 0.8)
    U = np.array([1.2, 0.6, -0.24, 3.0])
    Fn = oracle_mod.lf_flux(2, U, U, np.array([0.6, 0.8]))
    np.testing.assert_allclose(Fn, [0.168, 0.084 + 0.67824, -0.0336 + 0.90432, 4.1304 * 0.14],
                               rtol=1e-13)


def test_lf_flux_conservative_and_dissipative(oracle_mod):
    rng = np.random.default_rng(11)
    for _ in range(20):
        a = np.array([1.0, 0.2, -0.1, 2.5]) + rng.uniform(-0.1, 0.1, 4)
        b = np.array([0.9, -0.1, 0.3, 2.2]) + rng.uniform(-0.1, 0.1, 4)
        th = rng.uniform(0, 2 * np.pi)
        n = np.array([np.cos(th), np.sin(th)])
        f1 = oracle_mod.lf_flux(2, a, b, n)
        f2 = oracle_mod.lf_flux(2, b, a, -n)
        np.testing.assert_allclose(f1, -f2, atol=1e-14)
        # dissipation is a positive multiple (at least the fastest wave) of the jump
        avg = 0.5 * (oracle_mod.lf_flux(2, a, a, n) + oracle_mod.lf_flux(2, b, b, n))
        lam = (avg - f1) / (0.5 * (b - a))
        assert np.allclose(lam, lam[0]) and lam[0] > 1.0


def test_cfl_dt_constant_state(oracle_mod):
    """dt = cfl r / ((2p+1) lambda) with r the inradius and lambda = |u| + c."""
    m = oracle_mod.OracleMesh.from_input(W.periodic_square_tri(4))
    c, ub = _const_state(m.ne, 3, 2)
    rho, u, v, E = ub[0], ub[1] / ub[0], ub[2] / ub[0], ub[3]
    p_ = 0.4 * (E - 0.5 * rho * (u * u + v * v))
    lam = np.hypot(u, v) + np.sqrt(1.4 * p_ / rho)
    h = 0.25
    r = 2 * (0.5 * h * h) / (h * (2 + np.sqrt(2)))  # right isosceles triangle inradius
    assert abs(m.dt(1, c, 0.3) - 0.3 * r / (3 * lam)) < 1e-15


def _vortex_error(oracle_mod, n, p, T, cfl):
    m = oracle_mod.OracleMesh.from_input(W.periodic_square_tri(n))
    xyz, _, _ = m.eval_points(p)
    c = m.project(p, W.vortex_field(xyz[..., 0], xyz[..., 1], 0.0))
    dt0 = m.dt(p, c, cfl)
    steps = int(np.ceil(T / dt0))
    dt = T / steps
    for _ in range(steps):
        c, _ = m.rk_step(p, c, cfl, dt=dt)
    xyz2, w, U = m.eval_points(p, c=c, n1=p + 3)
    ex = W.vortex_field(xyz2[..., 0], xyz2[..., 1], T)
    return np.sqrt(np.sum(w[..., None] * (U - ex) ** 2))


@pytest.mark.parametrize("p,ns", [(1, (32, 64)), (2, (16, 32))])
def test_design_order_vortex(oracle_mod, p, ns):
    e = [_vortex_error(oracle_mod, n, p, 0.02, 0.3) for n in ns]
    order = np.log(e[0] / e[1]) / np.log(ns[1] / ns[0])
    assert order > p + 0.6, (e, order)


@pytest.mark.parametrize("p", [1, 2])
def test_conservation_periodic_tet(oracle_mod, p):
    """Face contributions cancel on a closed tetrahedral mesh: one flux per
    face, evaluated at one set of points for both elements."""
    m = oracle_mod.OracleMesh.from_input(W.periodic_cube_tet(4))
    c = W.random_state(m.ne, 5, oracle_mod.npoly(3, p), seed=p, amp=2e-2,
                       mean=(0.5, 0.05, -0.04, 0.03, 1.3))
    rhs = m.rhs(p, c)
    detj = m.detj()
    total = (detj[:, None] * rhs[:, :, 0]).sum(axis=0)
    scale = (detj[:, None] * np.abs(rhs[:, :, 0])).sum(axis=0)
    assert np.all(np.abs(total) < 1e-13 * scale)


@pytest.mark.parametrize("p", [1, 2])
def test_linear_advection_global_polynomial_closed_form_tet(oracle_mod, p):
    """3D form of the closed form: u a global polynomial of degree p on an open
    Kuhn cube => d u_h/dt = -a.grad u exactly."""
    m = oracle_mod.OracleMesh.from_input(W.open_cube_tet(3, jitter=0.15, seed=3))
    a = np.array([0.7, -1.3, 0.4])
    ncoef = (p + 1) * (p + 2) * (p + 3) // 6
    coef = np.random.default_rng(p).uniform(-1, 1, size=ncoef)

    def poly3(x, y, z):
        v, gx, gy, gz = (np.zeros_like(x) for _ in range(4))
        k = 0
        for d in range(p + 1):
            for i in range(d + 1):
                for j in range(d - i + 1):
                    l = d - i - j
                    v += coef[k] * x ** i * y ** j * z ** l
                    if i:
                        gx += coef[k] * i * x ** (i - 1) * y ** j * z ** l
                    if j:
                        gy += coef[k] * j * x ** i * y ** (j - 1) * z ** l
                    if l:
                        gz += coef[k] * l * x ** i * y ** j * z ** (l - 1)
                    k += 1
        return v, gx, gy, gz

    xyz, _, _ = m.eval_points(p, M=1)
    u = poly3(xyz[..., 0], xyz[..., 1], xyz[..., 2])[0]
    c = m.project(p, u[..., None])
    rhs = m.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a)
    xyz2, _, U = m.eval_points(p, c=rhs, n1=p + 3)
    _, gx, gy, gz = poly3(xyz2[..., 0], xyz2[..., 1], xyz2[..., 2])
    np.testing.assert_allclose(U[..., 0], -(a[0] * gx + a[1] * gy + a[2] * gz), atol=1e-11)
