"""Pins for the oracle's boundary conditions, time and limiter (dg_oracle.c
bc_state, orc_set_bc, orc_limit; the double Mach reflection run of Sec. 5,
Table 7, whose walls, inflow states, moving shock and limiter the paper takes
from [giuliani]).

Each pin is fixed by the mathematics rather than by the code:
* a slip wall reverses the normal momentum and keeps density, energy, speed
  and the tangential momentum; the Lax-Friedrichs flux through it carries no
  mass and no energy;
* uniform states that satisfy every boundary (a gas at rest in a walled box,
  a flow along walls with its own state prescribed at the ends) are steady;
* a walled box conserves mass and energy over many steps, not momentum;
* the moving shock selects the state behind it exactly where x < x_s(y, t);
* the limiter keeps every mean, keeps constant states, bounds the values at
  the vertices and volume points by the neighbouring means (and, at p = 1,
  everywhere on the element), limits no more than it must, and is idempotent.
"""

import numpy as np
import pytest

import oracle
from paper_1601_07613_gb300 import workloads as W

OM = oracle.OracleMesh
WALL, STATE, SHOCK = OM.BC_WALL, OM.BC_STATE, OM.BC_SHOCK


def _mesh(mi):
    om = OM.from_input(mi)
    l, r, ql, qr = om.sides()
    return om, l, r, ql


def _mid(mi, l, ql, b):
    v0 = mi.ev[l[b], ql[b]]
    v1 = mi.ev[l[b], (ql[b] + 1) % 3]
    return 0.5 * (mi.xyz[v0] + mi.xyz[v1])


def _uniform(om, p, U):
    xyz, _, _ = om.eval_points(p)
    return om.project(p, np.broadcast_to(U, xyz.shape[:2] + (4,)).copy())


def test_wall_state_invariants():
    mi = W.open_square_tri(4)
    om, l, r, ql = _mesh(mi)
    kind = np.where(r < 0, WALL, 0).astype(np.int8)
    om.set_bc(kind)
    s = int(np.nonzero(r < 0)[0][0])
    rng = np.random.default_rng(3)
    for _ in range(20):
        th = rng.uniform(0, 2 * np.pi)
        n = np.array([np.cos(th), np.sin(th)])
        Um = np.array([rng.uniform(0.5, 2), rng.normal(), rng.normal(), rng.uniform(5, 9)])
        Up = om.boundary_state(s, Um, n, np.zeros(2))
        m, mp = Um[1:3], Up[1:3]
        t = np.array([-n[1], n[0]])
        assert Up[0] == Um[0] and Up[3] == Um[3]
        assert np.isclose(np.linalg.norm(mp), np.linalg.norm(m), rtol=1e-15)
        assert np.isclose(mp @ n, -(m @ n), rtol=1e-14, atol=1e-15)
        assert np.isclose(mp @ t, m @ t, rtol=1e-14, atol=1e-15)
        F = oracle.lf_flux(2, Um, Up, n)
        scale = np.abs(oracle.lf_flux(2, Um, Um, n)).max()
        assert abs(F[0]) < 1e-15 * scale and abs(F[3]) < 1e-15 * scale


@pytest.mark.parametrize("p", [1, 2, 3])
def test_rest_state_in_walled_box_is_steady(p):
    mi = W.open_square_tri(6, jitter=0.2, seed=11)
    om, l, r, ql = _mesh(mi)
    om.set_bc(np.where(r < 0, WALL, 0).astype(np.int8))
    c = _uniform(om, p, np.array([1.4, 0.0, 0.0, 2.5]))
    rhs = om.rhs(p, c)
    h = 1.0 / 6
    assert np.abs(rhs).max() * h / 1.0 < 1e-13  # |F| ~ p = 1


@pytest.mark.parametrize("p", [1, 3])
def test_channel_flow_along_walls_is_steady(p):
    """Walls at y = 0 and y = 1, the flow's own state prescribed at x = 0 and
    x = 2: the uniform flow along x is an exact steady solution."""
    mi = W.open_rect_tri(8, 4, 2.0, 1.0, jitter=0.2, seed=12)
    om, l, r, ql = _mesh(mi)
    b = np.nonzero(r < 0)[0]
    mid = _mid(mi, l, ql, b)
    kind = np.zeros(om.ns, np.int8)
    horiz = (mid[:, 1] < 1e-12) | (mid[:, 1] > 1 - 1e-12)
    kind[b] = np.where(horiz, WALL, STATE)
    U = W._conserved(1.2, 0.8, 0.0, 1.5)
    om.set_bc(kind, np.zeros(om.ns, np.int8), U[None, :])
    rhs = om.rhs(p, _uniform(om, p, U))
    assert np.abs(rhs).max() * 0.25 / 3.0 < 1e-13


def test_walled_box_conserves_mass_and_energy():
    mi = W.open_square_tri(10, jitter=0.2, seed=13)
    om, l, r, ql = _mesh(mi)
    om.set_bc(np.where(r < 0, WALL, 0).astype(np.int8))
    p = 2
    xyz, _, _ = om.eval_points(p)
    U = W.vortex_field(xyz[..., 0], xyz[..., 1], beta=5.0)  # velocity ~1 crosses every wall
    c = om.project(p, U)
    detj = om.detj()
    tot = lambda c: (detj[:, None] * c[:, :, 0]).sum(0)
    t0 = tot(c)
    for _ in range(10):
        c, _ = om.rk_step(p, c, 0.3)
    t1 = tot(c)
    np.testing.assert_allclose(t1[[0, 3]], t0[[0, 3]], rtol=1e-13)
    assert np.abs(t1[1:3] - t0[1:3]).max() > 1e-6 * np.abs(t0).max()  # the walls push on the gas


def test_transmissive_kind_equals_no_boundary_conditions():
    mi = W.open_square_tri(5, jitter=0.2, seed=14)
    om, l, r, ql = _mesh(mi)
    c = W.random_state(om.ne, 4, 6, seed=2)
    a = om.rhs(2, c)
    om.set_bc(np.zeros(om.ns, np.int8))
    assert np.array_equal(om.rhs(2, c), a)


def test_shock_boundary_follows_the_shock():
    mi = W.open_rect_tri(16, 4, 4.0, 1.0)
    om, l, r, ql = _mesh(mi)
    kind, sidx = W.double_mach_boundary(mi, l, r, ql)
    S = W.double_mach_states()
    om.set_bc(kind, sidx, S, W.DMR_SHOCK, (0, 1))
    s = int(np.nonzero(kind == SHOCK)[0][0])
    a, b, cc = W.DMR_SHOCK
    n = np.array([0.0, 1.0])
    for t in (0.0, 0.01, 0.1):
        om.set_time(t)
        assert om.time() == t
        xs = a + b * 1.0 + cc * t
        for x, want in ((xs - 1e-9, 0), (xs + 1e-9, 1), (0.0, 0), (4.0, 1 if xs < 4 else 0)):
            Up = om.boundary_state(s, S[1], n, np.array([x, 1.0]))
            assert np.array_equal(Up, S[want])
            assert np.array_equal(Up, W.double_mach_field(np.array(x), np.array(1.0), t))
    # the states are those of a Mach 10 shock at rest in the shock's frame:
    # mass flux continuity across the shock moving at speed 10 along its normal
    rho0, rho1 = S[0, 0], S[1, 0]
    un = np.array([np.cos(np.pi / 6), -np.sin(np.pi / 6)])  # the shock's normal (direction of motion)
    u0 = S[0, 1:3] @ un / rho0
    assert np.isclose(rho0 * (u0 - 10.0), rho1 * (0.0 - 10.0), rtol=1e-12)


# ------------------------------------------------------------------------------------------
# Limiter
# ------------------------------------------------------------------------------------------

def _nb_bounds(om, c):
    """min / max over each element's mean and its face neighbours' means [E][4]."""
    l, r, _, _ = om.sides()
    phi0 = oracle.basis_tri(1, 0.3, 0.3)[0][0, 0]
    mean = c[:, :, 0] * phi0
    lo, hi = mean.copy(), mean.copy()
    inner = r >= 0
    for a, b in ((l[inner], r[inner]), (r[inner], l[inner])):
        np.minimum.at(lo, a, mean[b])
        np.maximum.at(hi, a, mean[b])
    return mean, lo, hi


def _values(c, p, r, s):
    phi = oracle.basis_tri(p, r, s)[0]  # [npts][Np]
    return np.einsum("emj,qj->eqm", c, phi)


@pytest.fixture(scope="module")
def rough():
    """A rough state on a jittered open mesh (vortex plus large random modes)."""
    mi = W.open_square_tri(12, jitter=0.2, seed=15)
    om = OM.from_input(mi)
    out = {}
    for p in (1, 2, 3):
        xyz, _, _ = om.eval_points(p)
        c = om.project(p, W.vortex_field(xyz[..., 0], xyz[..., 1], beta=5.0))
        c[:, :, 1:] += np.random.default_rng(p).uniform(-0.3, 0.3, c[:, :, 1:].shape)
        out[p] = c
    return om, out


@pytest.mark.parametrize("p", [1, 2, 3])
def test_limiter_keeps_means_and_constants(rough, p):
    om, cs = rough
    c = cs[p]
    lc = om.limit(p, c)
    assert np.array_equal(lc[:, :, 0], c[:, :, 0])
    assert not np.array_equal(lc, c)
    u = np.zeros_like(c)  # exactly constant: deviation modes zero
    u[:, :, 0] = np.array([1.1, 0.3, -0.2, 2.6])
    assert np.array_equal(om.limit(p, u), u)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_limiter_bounds_vertex_and_volume_values(rough, p):
    om, cs = rough
    lc = om.limit(p, cs[p])
    mean, lo, hi = _nb_bounds(om, lc)
    rv, sv, _ = oracle.tri_rule(p + 1)
    r = np.concatenate([[0.0, 1.0, 0.0], rv])
    s = np.concatenate([[0.0, 0.0, 1.0], sv])
    v = _values(lc, p, r, s)  # [E][pts][4]
    tol = 1e-13 * np.abs(mean).max()
    assert (v >= lo[:, None, :] - tol).all() and (v <= hi[:, None, :] + tol).all()


def test_limiter_p1_bounded_everywhere_and_tight(rough):
    """p = 1: dense sampling of every element stays within the bounds (a linear
    function's extremes are at the vertices), and every limited variable
    touches a bound at some vertex (alpha is as large as the bounds allow)."""
    om, cs = rough
    c = cs[1]
    lc = om.limit(1, c)
    mean, lo, hi = _nb_bounds(om, lc)
    rng = np.random.default_rng(0)
    a = rng.dirichlet(np.ones(3), 300)
    v = _values(lc, 1, a[:, 1], a[:, 2])
    tol = 1e-13 * np.abs(mean).max()
    assert (v >= lo[:, None, :] - tol).all() and (v <= hi[:, None, :] + tol).all()
    vert = _values(lc, 1, np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0]))
    limited = np.abs(lc[:, :, 1:] - c[:, :, 1:]).max(axis=2) > 0
    touch = (np.abs(vert - hi[:, None, :]) < tol) | (np.abs(vert - lo[:, None, :]) < tol)
    assert limited.sum() > 10
    assert touch.any(axis=1)[limited].all()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_limiter_is_idempotent(rough, p):
    om, cs = rough
    a = om.limit(p, cs[p])
    b = om.limit(p, a)
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-13 * np.abs(a).max())


def test_double_mach_small_run_stays_physical():
    """20 limited steps of the double Mach setup on a coarse mesh: the means
    stay finite with positive density and pressure, and the mesh's time
    advances by the steps' dt."""
    mi = W.open_rect_tri(32, 8, 4.0, 1.0, jitter=0.2, seed=16)
    om, l, r, ql = _mesh(mi)
    kind, sidx = W.double_mach_boundary(mi, l, r, ql)
    om.set_bc(kind, sidx, W.double_mach_states(), W.DMR_SHOCK, (0, 1))
    om.set_limiter(True)
    p = 1
    xyz, _, _ = om.eval_points(p)
    c = om.limit(p, om.project(p, W.double_mach_field(xyz[..., 0], xyz[..., 1])))
    t = 0.0
    for _ in range(20):
        c, dt = om.rk_step(p, c, 0.3)
        t += dt
    assert np.isclose(om.time(), t, rtol=1e-14)
    phi0 = oracle.basis_tri(1, 0.3, 0.3)[0][0, 0]
    U = c[:, :, 0] * phi0
    pr = 0.4 * (U[:, 3] - 0.5 * (U[:, 1] ** 2 + U[:, 2] ** 2) / U[:, 0])
    assert np.isfinite(c).all() and (U[:, 0] > 0).all() and (pr > 0).all()
