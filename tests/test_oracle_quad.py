"""Pins for the oracle's quadrilateral and hybrid meshes (Sec. 3.1, Table 2) and
for Eq. 2 on parallelogram quadrilaterals with the tensor-product Legendre
space Q_p.

* the basis against the closed forms of the first Legendre polynomials, and its
  orthonormality under a rule that is exact for it;
* the square rule against the exact integrals of monomials;
* the edge table: 2 n^2 edges on an n x n periodic grid, each shared by two
  elements that run along it in opposite directions;
* the coloring: 4 colors with no element seeing a color twice, on quadrilateral
  and hybrid meshes; on a periodic grid with an even number of elements every
  element has each color once; an odd number of elements on a closed
  quadrilateral mesh cannot be 4-colored at all (each color would have to be a
  perfect matching of an odd vertex set), and the swap cap must say so;
* freestream preservation, conservation, the closed-form linear advection
  result for a global polynomial, the default rules against 30-point rules for
  a linear flux, L2 stability of the upwind flux, the CFL rule on a square, a
  90-degree rotation of the whole mesh, and the design order on the vortex.
"""

import numpy as np
import pytest

from paper_1601_07613_gb300 import workloads as W


def _legendre01(n, x):
    t = 2.0 * x - 1.0
    P = [np.ones_like(t), t, (3 * t ** 2 - 1) / 2, (5 * t ** 3 - 3 * t) / 2][n]
    dP = [np.zeros_like(t), np.ones_like(t), 3 * t, (15 * t ** 2 - 3) / 2][n]
    return np.sqrt(2 * n + 1) * P, 2 * np.sqrt(2 * n + 1) * dP


@pytest.mark.parametrize("p", [1, 2, 3])
def test_quad_basis_closed_form(oracle_mod, p):
    rng = np.random.default_rng(p)
    r, s = rng.uniform(0, 1, 7), rng.uniform(0, 1, 7)
    phi, dr, ds = oracle_mod.basis_quad(p, r, s)
    for a in range(p + 1):
        for b in range(p + 1):
            la, dla = _legendre01(a, r)
            lb, dlb = _legendre01(b, s)
            j = a * (p + 1) + b
            np.testing.assert_allclose(phi[:, j], la * lb, rtol=1e-13, atol=1e-13)
            np.testing.assert_allclose(dr[:, j], dla * lb, rtol=1e-13, atol=1e-12)
            np.testing.assert_allclose(ds[:, j], la * dlb, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_quad_basis_orthonormal(oracle_mod, p):
    r, s, w = oracle_mod.quad_rule(p + 1)
    phi, _, _ = oracle_mod.basis_quad(p, r, s)
    np.testing.assert_allclose(phi.T @ (w[:, None] * phi), np.eye((p + 1) ** 2), atol=1e-13)


@pytest.mark.parametrize("n", [1, 2, 4])
def test_quad_rule_monomials(oracle_mod, n):
    r, s, w = oracle_mod.quad_rule(n)
    assert abs(w.sum() - 1.0) < 1e-15
    for a in range(2 * n):
        for b in range(2 * n):
            assert abs(np.sum(w * r ** a * s ** b) - 1.0 / ((a + 1) * (b + 1))) < 1e-14


def test_quad_edge_table(oracle_mod):
    n = 6
    mi = W.periodic_square_quad(n, jitter=0.2, slant=0.3, seed=1)
    m = oracle_mod.OracleMesh.from_input(mi)
    assert m.ns == 2 * n * n and m.nonaffine == 0
    l, r, ql, qr = m.sides()
    assert (r >= 0).all()
    ev = mi.ev
    for k in range(m.ns):
        a = ev[l[k], ql[k]], ev[l[k], (ql[k] + 1) % 4]
        b = ev[r[k], qr[k]], ev[r[k], (qr[k] + 1) % 4]
        assert a == (b[1], b[0])
    # every element has 4 distinct sides
    cnt = np.bincount(np.concatenate([l, r]), minlength=m.ne)
    assert (cnt == 4).all()


def _check_coloring(m, col, ev):
    l, r, _, _ = m.sides()
    assert col.min() >= 1 and col.max() <= 4
    seen = {}
    for k in range(m.ns):
        for e in (l[k], r[k]):
            if e < 0:
                continue
            assert (e, col[k]) not in seen, "an element sees a color twice"
            seen[(e, col[k])] = k
    return seen


@pytest.mark.parametrize("seed", [1, 7, 99])
def test_quad_coloring_perfect_on_even_periodic_grid(oracle_mod, seed):
    mi = W.periodic_square_quad(10, "vertex", jitter=0.2, seed=seed)
    m = oracle_mod.OracleMesh.from_input(mi)
    col, _ = m.color(4, seed)
    seen = _check_coloring(m, col, mi.ev)
    assert len(seen) == 4 * m.ne  # every element has each of the 4 colors once
    assert (np.bincount(col)[1:] == m.ns // 4).all()


@pytest.mark.parametrize("kind", ["periodic", "open"])
def test_hybrid_coloring_valid(oracle_mod, kind):
    mi = W.hybrid_square(9 if kind == "open" else 10, 0.3, periodic=kind == "periodic", seed=3)
    m = oracle_mod.OracleMesh.from_input(mi)
    assert m.nonaffine == 0  # unjittered squares and their triangles: every element affine
    col, _ = m.color(4, 5)
    _check_coloring(m, col, mi.ev)
    counts = np.bincount(col)[1:]
    assert counts.min() > 0.8 * counts.mean()  # roughly balanced, as in Table 2
    # with every vertex jittered the quadrilaterals are general (bilinear maps; the
    # pins of Eq. 2 on them are in tests/test_oracle_bilinear.py)
    mj = oracle_mod.OracleMesh.from_input(W.hybrid_square(9, 0.3, periodic=kind == "periodic", jitter=0.2, seed=3))
    assert 0 < mj.nonaffine <= int((mi.ev[:, 3] >= 0).sum())


def test_odd_closed_quad_mesh_is_not_4_colorable(oracle_mod):
    m = oracle_mod.OracleMesh.from_input(W.periodic_square_quad(5))
    with pytest.raises(RuntimeError, match="swap cap"):
        m.color(4, 1, max_swaps=20000)


def _const_state(ne, p):
    ub = np.array([1.1, 0.3, -0.2, 2.6])
    c = np.zeros((ne, 4, (p + 1) ** 2))
    c[:, :, 0] = ub  # phi_0 = 1 on the unit reference square
    return c


@pytest.mark.parametrize("p", [0, 1, 2, 3])
@pytest.mark.parametrize("kind", ["periodic", "open"])
def test_quad_freestream(oracle_mod, p, kind):
    mi = (W.periodic_square_quad(8, jitter=0.2, slant=0.3, seed=5) if kind == "periodic"
          else W.open_square_quad(8, jitter=0.2, seed=5))
    m = oracle_mod.OracleMesh.from_input(mi)
    rhs = m.rhs(p, _const_state(m.ne, p))
    h = 1.0 / 8
    assert np.abs(rhs).max() * h * h / (4 * h * 3.0) < 1e-13


@pytest.mark.parametrize("p", [1, 3])
def test_quad_conservation_periodic(oracle_mod, p):
    m = oracle_mod.OracleMesh.from_input(W.periodic_square_quad(8, jitter=0.2, slant=0.3, seed=6))
    c = W.random_state(m.ne, 4, (p + 1) ** 2, seed=p, amp=2e-2)
    rhs = m.rhs(p, c)
    detj = m.detj()
    total = (detj[:, None] * rhs[:, :, 0]).sum(axis=0)
    scale = (detj[:, None] * np.abs(rhs[:, :, 0])).sum(axis=0)
    assert np.all(np.abs(total) < 1e-13 * scale)


def _poly2(deg, coef, x, y):
    v, gx, gy = np.zeros_like(x), np.zeros_like(x), np.zeros_like(x)
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
def test_quad_linear_advection_global_polynomial_closed_form(oracle_mod, p):
    """Jittered rectangles on the open square: a continuous polynomial u of
    degree p lies in Q_p, so Eq. 2 reproduces -a.grad u exactly."""
    a = np.array([0.7, -1.3])
    coef = np.random.default_rng(p).uniform(-1, 1, size=(p + 1) * (p + 2) // 2)
    m = oracle_mod.OracleMesh.from_input(W.open_square_quad(6, jitter=0.2, seed=7))
    xyz, _, _ = m.eval_points(p, M=1)
    u, _, _ = _poly2(p, coef, xyz[..., 0], xyz[..., 1])
    c = m.project(p, u[..., None])
    rhs = m.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a)
    xyz2, _, U = m.eval_points(p, c=rhs, n1=p + 3)
    _, gx, gy = _poly2(p, coef, xyz2[..., 0], xyz2[..., 1])
    np.testing.assert_allclose(U[..., 0], -(a[0] * gx + a[1] * gy), atol=1e-11)


@pytest.mark.parametrize("p", [1, 2])
def test_quad_linear_advection_slanted_closed_form(oracle_mod, p):
    """The slanted periodic mesh unrolled into an open mesh of the same
    parallelograms (wrapped vertices get copies one period away).  A linear
    u = u0 + b.x is continuous and exact on every element, and on the boundary
    the transmissive state equals the exact trace, so Eq. 2 gives -a.b in
    mode 0 and nothing else, on every element."""
    mi = W.periodic_square_quad(6, jitter=0.2, slant=0.3, seed=8)
    n = 6
    xyz = mi.xyz
    ids = {}
    pts = []
    ev = np.zeros_like(mi.ev)
    for e in range(mi.ne):
        i, j = e % n, e // n
        corner = [(i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)]
        for k, (ci, cj) in enumerate(corner):
            key = (ci, cj)
            if key not in ids:
                x, y = xyz[(cj % n) * n + (ci % n)]
                # periodic images: shift by whole periods to follow the grid
                x += np.floor(ci / n)
                y += np.floor(cj / n)
                ids[key] = len(pts)
                pts.append((x, y))
            ev[e, k] = ids[key]
    m = oracle_mod.OracleMesh(2, np.array(pts), ev)
    assert m.nonaffine == 0
    a = np.array([0.4, 0.9])
    b = np.array([1.7, -0.6])
    xyz_q, _, _ = m.eval_points(p, M=1)
    u = 0.3 + b[0] * xyz_q[..., 0] + b[1] * xyz_q[..., 1]
    c = m.project(p, u[..., None])
    rhs = m.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a)
    np.testing.assert_allclose(rhs[:, 0, 0], -(a @ b), atol=1e-12)
    np.testing.assert_allclose(rhs[:, 0, 1:], 0.0, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_quad_linear_advection_brute_force_quadrature(oracle_mod, p):
    m = oracle_mod.OracleMesh.from_input(W.periodic_square_quad(4, jitter=0.2, slant=0.3, seed=9))
    c = np.random.default_rng(p).uniform(-1, 1, size=(m.ne, 1, (p + 1) ** 2))
    a = np.array([0.4, 0.9])
    r0 = m.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a)
    r1 = m.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a, nq_face1=30, nq_vol1=30)
    np.testing.assert_allclose(r0, r1, atol=1e-12 * np.abs(r1).max())


def test_quad_linear_advection_energy_stable(oracle_mod):
    m = oracle_mod.OracleMesh.from_input(W.periodic_square_quad(6, jitter=0.2, slant=0.3, seed=10))
    c = np.random.default_rng(3).uniform(-1, 1, size=(m.ne, 1, 9))
    rhs = m.rhs(2, c, kind=oracle_mod.ADVECTION, adv=np.array([1.0, 0.5]))
    assert np.sum(m.detj()[:, None, None] * c * rhs) < -1e-3


def test_quad_cfl_dt_constant_state(oracle_mod):
    """On an h x h square the inradius rule gives r = 2 h^2 / (4 h) = h / 2."""
    m = oracle_mod.OracleMesh.from_input(W.periodic_square_quad(4))
    c = _const_state(m.ne, 1)
    rho, u, v, E = 1.1, 0.3 / 1.1, -0.2 / 1.1, 2.6
    pr = 0.4 * (E - 0.5 * rho * (u * u + v * v))
    lam = np.hypot(u, v) + np.sqrt(1.4 * pr / rho)
    assert abs(m.dt(1, c, 0.3) - 0.3 * (0.25 / 2) / (3 * lam)) < 1e-15


@pytest.mark.parametrize("p", [1, 3])
def test_quad_rotation_by_90_degrees(oracle_mod, p):
    """Rotating the periodic mesh and the state's velocity by 90 degrees about
    the centre leaves the reference-element problem unchanged: density and
    energy rates equal, momentum rates rotated."""
    mi = W.periodic_square_quad(6, jitter=0.2, slant=0.3, seed=11)
    m0 = oracle_mod.OracleMesh.from_input(mi)
    xr = np.stack([(1.0 - mi.xyz[:, 1]) % 1.0, mi.xyz[:, 0]], axis=1)
    m1 = oracle_mod.OracleMesh(2, xr, mi.ev, mi.periodic_len)
    c0 = W.random_state(m0.ne, 4, (p + 1) ** 2, seed=p, amp=2e-2)
    c1 = c0.copy()
    c1[:, 1], c1[:, 2] = -c0[:, 2], c0[:, 1]
    r0, r1 = m0.rhs(p, c0), m1.rhs(p, c1)
    scale = np.abs(r0).max()
    np.testing.assert_allclose(r1[:, 0], r0[:, 0], atol=1e-12 * scale)
    np.testing.assert_allclose(r1[:, 3], r0[:, 3], atol=1e-12 * scale)
    np.testing.assert_allclose(r1[:, 1], -r0[:, 2], atol=1e-12 * scale)
    np.testing.assert_allclose(r1[:, 2], r0[:, 1], atol=1e-12 * scale)


def _vortex_error(oracle_mod, n, p, T, cfl):
    m = oracle_mod.OracleMesh.from_input(W.periodic_square_quad(n, jitter=0.1, slant=0.2, seed=12))
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


def test_quad_design_order_vortex(oracle_mod):
    e = [_vortex_error(oracle_mod, n, 1, 0.02, 0.3) for n in (16, 32)]
    order = np.log(e[0] / e[1]) / np.log(2.0)
    assert order > 1.6, (e, order)
