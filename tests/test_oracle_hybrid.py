"""Pins for the oracle's right-hand side (Eq. 2) on hybrid triangle /
quadrilateral meshes (Sec. 3.1, Table 2's hybrid mesh), each element with the
space of its kind: P_p on a triangle, Q_p on a parallelogram, the state stored
with (p+1)^2 coefficients per variable (a triangle uses the first
(p+1)(p+2)/2).

* freestream, and conservation on a periodic mesh;
* linear advection of a global polynomial of degree p (in both spaces), whose
  exact result is -a.grad(u), on an open mesh: a wrong basis, rule, Jacobian or
  face point on either kind of element, or at a mixed edge, breaks it;
* brute force: for linear advection every integrand is a polynomial the default
  rules integrate exactly, so 30-point rules give the same result;
* upwind energy stability;
* the limits: with every cell split the mesh is a triangle mesh, and with none a
  quadrilateral mesh, and the results equal those of the same meshes given as
  pure meshes.
"""

import numpy as np
import pytest

from paper_1601_07613_gb300 import workloads as W


def _hyb(n=10, frac=0.4, periodic=True, seed=3):
    return W.hybrid_square(n, frac, periodic=periodic, jitter=0.2, slant=0.3 if periodic else 0.0, seed=seed,
                           mode="parallelogram")


def _state(om, p, seed, amp=3e-3):
    npq = (p + 1) ** 2
    return W.random_state(om.ne, 4, npq, seed=seed, amp=amp)


def test_hybrid_mesh_is_affine(oracle_mod):
    om = oracle_mod.OracleMesh.from_input(_hyb())
    assert om.quad and om.nonaffine == 0
    ev, _ = om.elements()
    assert (ev[:, 3] < 0).any() and (ev[:, 3] >= 0).any()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_hybrid_freestream_and_conservation(oracle_mod, p):
    om = oracle_mod.OracleMesh.from_input(_hyb())
    c = np.zeros((om.ne, 4, (p + 1) ** 2))
    ub = np.array([1.1, 0.3, -0.2, 2.6])
    c[:, :, 0] = ub  # phi_0 = 1 on the square; on the triangle phi_0 = sqrt(2): set per kind below
    ev, _ = om.elements()
    tri = ev[:, 3] < 0
    c[tri, :, 0] = ub / np.sqrt(2.0)
    r = om.rhs(p, c)
    h = 0.1
    assert np.abs(r).max() * (0.5 * h * h) / (3.4 * h * 3.0) < 1e-13
    c = _state(om, p, seed=p)
    c[tri, :, (p + 1) * (p + 2) // 2:] = 0.0
    r = om.rhs(p, c)
    dj = om.detj()
    area = np.where(tri, 0.5, 1.0) * dj
    phi0 = np.where(tri, np.sqrt(2.0), 1.0)
    tot = (area[:, None] * phi0[:, None] * r[:, :, 0]).sum(0)
    scale = (area[:, None] * phi0[:, None] * np.abs(r[:, :, 0])).sum(0)
    assert np.all(np.abs(tot) < 1e-13 * scale)
    # a triangle's unused coefficients stay zero in the result
    assert np.all(r[tri][:, :, (p + 1) * (p + 2) // 2:] == 0.0)


def _poly(p, coef, x, y):
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


@pytest.mark.parametrize("p", [1, 2, 3])
def test_hybrid_linear_advection_closed_form(oracle_mod, p):
    om = oracle_mod.OracleMesh.from_input(_hyb(9, 0.5, periodic=False, seed=4))
    a = np.array([0.7, -1.3])
    coef = np.random.default_rng(p).uniform(-1, 1, size=(p + 1) * (p + 2) // 2)
    xyz, _, _ = om.eval_points(p, M=1)
    c = om.project(p, _poly(p, coef, xyz[..., 0], xyz[..., 1])[0][..., None])
    rhs = om.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a)
    xyz2, _, U = om.eval_points(p, c=rhs, n1=p + 3)
    _, gx, gy = _poly(p, coef, xyz2[..., 0], xyz2[..., 1])
    np.testing.assert_allclose(U[..., 0], -(a[0] * gx + a[1] * gy), atol=1e-11)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_hybrid_linear_advection_brute_force(oracle_mod, p):
    om = oracle_mod.OracleMesh.from_input(_hyb(6, 0.5, seed=5))
    c = np.random.default_rng(p).uniform(-1, 1, size=(om.ne, 1, (p + 1) ** 2))
    a = np.array([0.4, 0.9])
    r0 = om.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a)
    r1 = om.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a, nq_face1=30, nq_vol1=30)
    np.testing.assert_allclose(r0, r1, atol=1e-12 * np.abs(r1).max())


def test_hybrid_linear_advection_energy_stable(oracle_mod):
    om = oracle_mod.OracleMesh.from_input(_hyb(8, 0.5, seed=6))
    ev, _ = om.elements()
    tri = ev[:, 3] < 0
    c = np.random.default_rng(3).uniform(-1, 1, size=(om.ne, 1, 9))
    c[tri, :, 6:] = 0.0
    rhs = om.rhs(2, c, kind=oracle_mod.ADVECTION, adv=np.array([1.0, 0.5]))
    area = np.where(tri, 0.5, 1.0) * om.detj()
    assert np.sum(area[:, None, None] / np.where(tri, 0.5, 1.0)[:, None, None] * c * rhs) < -1e-3


@pytest.mark.parametrize("p", [1, 3])
def test_hybrid_limits_equal_pure_meshes(oracle_mod, p):
    """frac = 1: the triangles as a plain triangle mesh; frac = 0: the
    parallelograms as a plain quadrilateral mesh."""
    ntri = (p + 1) * (p + 2) // 2
    h = _hyb(7, 1.0, seed=7)
    assert (h.ev[:, 3] < 0).all()
    om = oracle_mod.OracleMesh.from_input(h)
    ot = oracle_mod.OracleMesh(2, h.xyz, np.ascontiguousarray(h.ev[:, :3]), h.periodic_len)
    ct = W.random_state(ot.ne, 4, ntri, seed=p)
    ch = np.zeros((om.ne, 4, (p + 1) ** 2))
    ch[:, :, :ntri] = ct
    np.testing.assert_allclose(om.rhs(p, ch)[:, :, :ntri], ot.rhs(p, ct), rtol=0, atol=1e-12 * np.abs(ot.rhs(p, ct)).max())
    q = _hyb(7, 0.0, seed=7)
    assert (q.ev[:, 3] >= 0).all()
    oq = oracle_mod.OracleMesh.from_input(q)
    oq2 = oracle_mod.OracleMesh.from_input(W.periodic_square_quad(7, "parallelogram", 0.2, 0.3, seed=7))
    cq = W.random_state(oq.ne, 4, (p + 1) ** 2, seed=p)
    assert np.array_equal(oq.rhs(p, cq), oq2.rhs(p, cq))
