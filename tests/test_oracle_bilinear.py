"""Pins for the oracle's Eq. 2 on general (bilinear) quadrilaterals: a
quadrilateral that is not a parallelogram maps the square bilinearly, so its
detJ and J^-1 vary over the element and its mass matrix
M_ij = int phi_i phi_j detJ is not diagonal; the right-hand side is
M^-1 (volume - surface).  With straight edges and the default rules (p+1
Gauss points per direction, 2p+1 on an edge) every integrand below is a
polynomial the rules integrate exactly, so:

* freestream: a constant state has a zero right-hand side (the discrete metric
  identities hold);
* the L2 projection reproduces a linear function exactly (it is bilinear on the
  square, in Q_1), checked at points the projection did not use;
* linear advection of a linear function gives -a.grad(u) exactly (open mesh);
* brute force: for linear advection the default rules equal 30-point rules;
* conservation: the integral of the right-hand side over a periodic mesh is zero
  (integrated with each element's physical weights, detJ at every point);
* on a hybrid mesh (general quadrilaterals and triangles) the same holds.
"""

import numpy as np
import pytest

from paper_1601_07613_gb300 import workloads as W


def _periodic(n=8, seed=3):
    return W.periodic_square_quad(n, "vertex", jitter=0.2, seed=seed)


def _open(n=7, seed=4):
    return W.open_square_quad(n, "vertex", jitter=0.2, seed=seed)


def test_vertex_jittered_quads_are_bilinear(oracle_mod):
    om = oracle_mod.OracleMesh.from_input(_periodic())
    assert om.quad and om.nonaffine > 0.9 * om.ne


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("mk", [_periodic, _open])
def test_bilinear_freestream(oracle_mod, p, mk):
    om = oracle_mod.OracleMesh.from_input(mk())
    c = np.zeros((om.ne, 4, (p + 1) ** 2))
    c[:, :, 0] = [1.1, 0.3, -0.2, 2.6]
    h = 1.0 / 8
    assert np.abs(om.rhs(p, c)).max() * (h * h) / (4 * h * 3.0) < 1e-13


def _lin(x, y):
    return 0.3 + 0.7 * x - 1.1 * y


@pytest.mark.parametrize("p", [1, 2, 3])
def test_bilinear_projection_reproduces_linear(oracle_mod, p):
    om = oracle_mod.OracleMesh.from_input(_open())
    xyz, _, _ = om.eval_points(p, M=1)
    c = om.project(p, _lin(xyz[..., 0], xyz[..., 1])[..., None])
    xyz2, _, U = om.eval_points(p, c=c, n1=p + 3)
    assert np.abs(U[..., 0] - _lin(xyz2[..., 0], xyz2[..., 1])).max() < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3])
def test_bilinear_linear_advection_closed_form(oracle_mod, p):
    om = oracle_mod.OracleMesh.from_input(_open())
    a = np.array([0.7, -1.3])
    xyz, _, _ = om.eval_points(p, M=1)
    c = om.project(p, _lin(xyz[..., 0], xyz[..., 1])[..., None])
    rhs = om.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a)
    _, _, U = om.eval_points(p, c=rhs, n1=p + 3)
    assert np.abs(U[..., 0] - (-(a[0] * 0.7 + a[1] * (-1.1)))).max() < 1e-11


@pytest.mark.parametrize("p", [1, 2, 3])
def test_bilinear_linear_advection_brute_force(oracle_mod, p):
    om = oracle_mod.OracleMesh.from_input(_periodic(6, seed=5))
    c = np.random.default_rng(p).uniform(-1, 1, size=(om.ne, 1, (p + 1) ** 2))
    a = np.array([0.4, 0.9])
    r0 = om.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a)
    r1 = om.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a, nq_face1=30, nq_vol1=30)
    np.testing.assert_allclose(r0, r1, atol=1e-11 * np.abs(r1).max())


@pytest.mark.parametrize("hybrid", [False, True])
def test_bilinear_conservation(oracle_mod, hybrid):
    mi = W.hybrid_square(9, 0.4, periodic=True, jitter=0.2, seed=6) if hybrid else _periodic(9, seed=6)
    om = oracle_mod.OracleMesh.from_input(mi)
    p = 2
    c = W.random_state(om.ne, 4, 9, seed=8, amp=2e-2)
    if hybrid:
        c[mi.ev[:, 3] < 0, :, 6:] = 0.0
    rhs = om.rhs(p, c)
    _, w, U = om.eval_points(p, c=rhs)
    tot = (w[..., None] * U).sum((0, 1))
    scale = (w[..., None] * np.abs(U)).sum((0, 1))
    assert np.all(np.abs(tot) < 1e-13 * scale)


def test_bilinear_hybrid_freestream_and_closed_form(oracle_mod):
    mi = W.hybrid_square(8, 0.4, periodic=False, jitter=0.2, seed=7)
    om = oracle_mod.OracleMesh.from_input(mi)
    assert om.nonaffine > 0 and (mi.ev[:, 3] < 0).any()
    p = 2
    a = np.array([0.7, -1.3])
    xyz, _, _ = om.eval_points(p, M=1)
    c = om.project(p, _lin(xyz[..., 0], xyz[..., 1])[..., None])
    rhs = om.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a)
    _, _, U = om.eval_points(p, c=rhs, n1=p + 3)
    assert np.abs(U[..., 0] - (-(a[0] * 0.7 + a[1] * (-1.1)))).max() < 1e-11
