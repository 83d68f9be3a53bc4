"""Pins for the oracle's SSP-RK3 step and for its extended-precision and
threaded builds.

* SSP-RK3 stability polynomial: for a linear right-hand side L (the linear
  advection flux, whose Lax-Friedrichs form is the upwind flux, so Eq. 2 is
  linear in the coefficients) any three-stage, third-order Runge-Kutta step is
  exactly u + dt Lu + dt^2 L^2 u / 2 + dt^3 L^3 u / 6.  A wrong Shu-Osher weight
  or stage operand changes that polynomial.  L is applied by the oracle's
  right-hand side; the step's own stage code is what is checked.
* The extended build (long double arithmetic, the same C file) is pinned on
  its own: a significand wider than FP64's, freestream and the linear-advection
  closed form to its own precision, far below FP64's rounding, and agreement
  with the FP64 build within FP64's rounding on every element type.
* The threaded build computes every element with the same arithmetic: its
  right-hand side equals the sequential one bit for bit at any thread count.
"""

import numpy as np
import pytest

from paper_1601_07613_gb300 import workloads as W


def _rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).astype(np.float64)) /
                 np.linalg.norm(np.asarray(b).astype(np.float64)))


MESHES = {
    "open": lambda: W.open_square_tri(9, jitter=0.2, seed=21),
    "periodic": lambda: W.periodic_square_tri(8, jitter=0.2, seed=22),
}


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("name", ["open", "periodic"])
def test_rk_step_is_the_ssp_rk3_stability_polynomial(oracle_mod, name, p):
    mi = MESHES[name]()
    m = oracle_mod.OracleMesh.from_input(mi)
    a = np.array([1.0, 0.6])
    u = np.random.default_rng(p).uniform(-1, 1, size=(m.ne, 1, m.np_modes(p)))
    h = 1.0 / 9
    dt = 0.3 * h / (np.hypot(*a) * (2 * p + 1))

    def L(v):
        return m.rhs(p, v, kind=oracle_mod.ADVECTION, adv=a)

    L1 = L(u)
    L2 = L(L1)
    L3 = L(L2)
    poly = u + dt * L1 + dt ** 2 / 2 * L2 + dt ** 3 / 6 * L3
    got, dt_used = m.rk_step(p, u, 0.0, dt=dt, kind=oracle_mod.ADVECTION, adv=a)
    assert dt_used == dt
    du = got - u
    assert _rel(du, poly - u) < 1e-13
    # the test has power: each term of the polynomial is far above the tolerance
    # (a wrong weight on any stage moves the dt^2 or dt^3 coefficient)
    assert np.linalg.norm(dt ** 3 / 6 * L3) / np.linalg.norm(du) > 1e-4
    assert _rel(du, dt * L1 + dt ** 2 / 2 * L2) > 1e-4


def test_rk_step_advection_needs_dt(oracle_mod):
    m = oracle_mod.OracleMesh.from_input(MESHES["open"]())
    u = np.zeros((m.ne, 1, 3))
    with pytest.raises(RuntimeError, match="dt_in"):
        m.rk_step(1, u, 0.3, kind=oracle_mod.ADVECTION, adv=np.array([1.0, 0.0]))


def test_rk_step_euler_matches_its_stages(oracle_mod):
    """The Euler step is the same stage code with the Euler right-hand side: its
    stages, rebuilt here from three oracle right-hand sides, give the step."""
    mi = W.periodic_square_tri(7, jitter=0.2, seed=23)
    m = oracle_mod.OracleMesh.from_input(mi)
    c = W.random_state(m.ne, 4, 6, seed=4, amp=2e-2)
    got, dt = m.rk_step(2, c, 0.3)
    assert dt == m.dt(2, c, 0.3)
    u1 = c + dt * m.rhs(2, c)
    u2 = 0.75 * c + 0.25 * (u1 + dt * m.rhs(2, u1))
    u3 = c / 3.0 + 2.0 / 3.0 * (u2 + dt * m.rhs(2, u2))
    assert np.array_equal(got, u3)


# ------------------------------------------------------------------------------------------
# extended build
# ------------------------------------------------------------------------------------------

def test_extended_build_is_wider(oracle_mod):
    ext = oracle_mod.get("extended")
    assert oracle_mod.get("fp64").mant_dig == 53
    assert ext.mant_dig >= 64, ext.mant_dig  # x87 extended (64) or IEEE binary128 (113)
    assert np.finfo(ext.dtype).nmant + 1 >= ext.mant_dig


def test_extended_gauss_rules_to_own_precision(oracle_mod):
    """Closed-form Gauss-Legendre rules (n = 2: +-1/sqrt 3, weights 1; n = 3: 0,
    +-sqrt(3/5), weights 8/9, 5/9) and the Gauss-Jacobi(1,0) weight total
    int (1-x) dx = 2, met to a few units of the wider type's roundoff."""
    B = oracle_mod.get("extended")
    R = B.dtype
    eps = 2.0 ** (1 - B.mant_dig)

    def rule(n, a):
        x = np.zeros(n, R)
        w = np.zeros(n, R)
        B.check(B.L.orc_gauss_jacobi(n, a, B.ptr(x), B.ptr(w)))
        return x, w

    x, w = rule(2, 0.0)
    r3 = 1 / np.sqrt(R(3))
    assert np.abs(x - np.array([-r3, r3])).max() < 8 * eps and np.abs(w - 1).max() < 8 * eps
    x, w = rule(3, 0.0)
    r = np.sqrt(R(3) / 5)
    assert np.abs(x - np.array([-r, 0, r])).max() < 8 * eps
    assert np.abs(w - np.array([R(5) / 9, R(8) / 9, R(5) / 9])).max() < 8 * eps
    for n in (4, 7, 9):
        assert abs(rule(n, 1.0)[1].sum() - 2) < 16 * eps


@pytest.mark.parametrize("p", [1, 3])
def test_extended_freestream_far_below_fp64(oracle_mod, p):
    mi = W.periodic_square_tri(12, jitter=0.2, seed=5)
    ub = np.array([1.1, 0.3, -0.2, 2.6])
    h = 1.0 / 12
    out = {}
    for build in ("fp64", "extended"):
        m = oracle_mod.OracleMesh.from_input(mi, build=build)
        c = np.zeros((m.ne, 4, m.np_modes(p)), m.real)
        c[:, :, 0] = m.real(ub) / np.sqrt(m.real(2))
        out[build] = float(np.abs(m.rhs(p, c)).max()) * (0.5 * h * h) / (3.4 * h * 3.0)
    eps = 2.0 ** (1 - oracle_mod.get("extended").mant_dig)
    assert out["extended"] < 1e3 * eps  # 1e3 x the unit roundoff of the wider type
    assert out["extended"] < 1e-2 * out["fp64"]


@pytest.mark.parametrize("p", [1, 2, 3])
def test_extended_linear_advection_closed_form(oracle_mod, p):
    """u a global polynomial of degree p => d u_h/dt = -a.grad u exactly; in the
    extended build to its own precision (FP64 meets it to ~1e-13)."""
    m = oracle_mod.OracleMesh.from_input(W.open_square_tri(6, jitter=0.2, seed=7), build="extended")
    R = m.real
    a = np.array([0.7, -1.3], dtype=R)
    coef = np.random.default_rng(p).uniform(-1, 1, size=(p + 1) * (p + 2) // 2).astype(R)

    def poly(x, y):
        v, gx, gy = (np.zeros_like(x) for _ in range(3))
        k = 0
        for d in range(p + 1):
            for i in range(d + 1):
                j = d - i
                v += coef[k] * x ** i * y ** j
                if i:
                    gx += coef[k] * i * x ** (i - 1) * y ** j
                if j:
                    gy += coef[k] * j * x ** i * y ** (j - 1)
                k += 1
        return v, gx, gy

    xyz, _, _ = m.eval_points(p, M=1)
    c = m.project(p, poly(xyz[..., 0], xyz[..., 1])[0][..., None])
    rhs = m.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a)
    xyz2, _, U = m.eval_points(p, c=rhs, n1=p + 3)
    _, gx, gy = poly(xyz2[..., 0], xyz2[..., 1])
    err = float(np.abs(U[..., 0] + (a[0] * gx + a[1] * gy)).max())
    eps = 2.0 ** (1 - oracle_mod.get("extended").mant_dig)
    assert err < 1e5 * eps, err


@pytest.mark.parametrize("case", ["tri", "open_tri", "tet", "quad", "refined"])
def test_extended_agrees_with_fp64(oracle_mod, case):
    """Same inputs, same steps: the two builds differ by FP64 rounding only."""
    if case == "tri":
        mi, p, M = W.periodic_square_tri(14, jitter=0.2, seed=24), 3, 4
    elif case == "open_tri":
        mi, p, M = W.open_square_tri(11, jitter=0.2, seed=25), 2, 4
    elif case == "tet":
        mi, p, M = W.periodic_cube_tet(3), 2, 5
    elif case == "quad":
        mi, p, M = W.periodic_square_quad(8, jitter=0.2, slant=0.3, seed=26), 3, 4
    else:
        mi, p, M = W.periodic_square_tri(10, jitter=0.2, seed=27), 2, 4
    m64 = oracle_mod.OracleMesh.from_input(mi)
    mx = oracle_mod.OracleMesh.from_input(mi, build="extended")
    if case == "refined":
        col, _ = m64.color(3, 1601)
        m64 = m64.refine(col, np.arange(0, m64.ne, 5))
        mx = mx.refine(col, np.arange(0, mx.ne, 5))
        assert np.array_equal(m64.colors, mx.colors)
    mean = (0.5, 0.05, -0.04, 0.03, 1.3) if M == 5 else None
    kw = {"mean": mean} if mean else {}
    c = W.random_state(m64.ne, M, m64.np_modes(p), seed=7, **kw)
    r64 = m64.rhs(p, c)
    rx = mx.rhs(p, c)
    assert rx.dtype == np.longdouble
    e = _rel(r64, rx)
    assert 0.0 < e < 1e-12, e
    assert np.array_equal(m64.sides()[0], mx.sides()[0])


# ------------------------------------------------------------------------------------------
# threaded build (the CPU baseline)
# ------------------------------------------------------------------------------------------

def test_threaded_build_bit_identical(oracle_mod):
    mi = W.periodic_square_tri(20, jitter=0.2, seed=28)
    c = W.random_state(mi.ne, 4, 10, seed=8)
    ref = oracle_mod.OracleMesh.from_input(mi).rhs(3, c)
    mt = oracle_mod.OracleMesh.from_input(mi, build="threads")
    sample = np.random.default_rng(1).choice(mi.ne, 97, replace=False)
    for n in (1, 3, 4):
        assert oracle_mod.set_threads(n) == n
        assert np.array_equal(mt.rhs(3, c), ref)
        assert np.array_equal(mt.rhs(3, c, elems=sample), ref[sample])
