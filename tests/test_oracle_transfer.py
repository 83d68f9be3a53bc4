"""Pins for the oracle's state transfer between a triangle mesh and its one-level
refinement (Sec. 3.2; dynamic adaptivity moves the solution between the two):

* prolongation is exact for polynomials: a global polynomial of degree p,
  L2-projected on the coarse mesh (exactly representable there), prolonged to
  the refined mesh, equals its projection computed on the refined mesh itself;
* restriction after prolongation is the identity (each child's projection of
  its parent's polynomial carries all of it);
* restriction is the L2 projection: the residual f - P(R f) of any refined state
  f is orthogonal, in the mass-weighted inner product (detJ times the dot product
  of orthonormal coefficients), to every prolonged coarse state;
* both conserve the element means' total (the integral of the solution);
* unrefined elements are copied.
"""

import numpy as np
import pytest

from paper_1601_07613_gb300 import workloads as W


def _pair(oracle_mod, kind, build="fp64"):
    mi = W.periodic_square_tri(10, jitter=0.2, seed=81) if kind == "periodic" else W.open_square_tri(9, jitter=0.2,
                                                                                                    seed=82)
    om = oracle_mod.OracleMesh.from_input(mi, build=build)
    col, _ = om.color(3, 1601)
    elems = W.elements_near(mi, (0.45, 0.55), 0.3)
    return mi, om, om.refine(col, elems), elems


def _poly(p, coef, x, y):
    v = np.zeros_like(x)
    k = 0
    for d in range(p + 1):
        for i in range(d + 1):
            v = v + coef[k] * x ** i * y ** (d - i)
            k += 1
    return v


@pytest.mark.parametrize("p", [1, 2, 3])
def test_prolongation_exact_for_polynomials(oracle_mod, p):
    """(a global polynomial is not periodic: the open mesh)"""
    mi, om, fm, _ = _pair(oracle_mod, "open")
    rng = np.random.default_rng(p)
    coef = rng.uniform(-1, 1, size=(4, (p + 1) * (p + 2) // 2))
    xc, _, _ = om.eval_points(p, M=4)
    xf, _, _ = fm.eval_points(p, M=4)
    vc = np.stack([_poly(p, coef[m], xc[..., 0], xc[..., 1]) for m in range(4)], axis=-1)
    vf = np.stack([_poly(p, coef[m], xf[..., 0], xf[..., 1]) for m in range(4)], axis=-1)
    cc = om.project(p, vc)
    cf = fm.project(p, vf)
    got = fm.prolong(p, cc)
    assert np.abs(got - cf).max() < 1e-13 * np.abs(cf).max()


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("kind", ["periodic", "open"])
def test_restriction_is_the_l2_projection(oracle_mod, kind, p):
    mi, om, fm, _ = _pair(oracle_mod, kind)
    rng = np.random.default_rng(10 + p)
    npm = (p + 1) * (p + 2) // 2
    g = rng.uniform(-1, 1, size=(om.ne, 4, npm))
    f = rng.uniform(-1, 1, size=(fm.ne, 4, npm))
    # R P = I
    assert np.abs(fm.restrict(p, fm.prolong(p, g)) - g).max() < 1e-13
    # <f - P R f, P g> = 0 in the mass-weighted inner product
    dj = fm.detj()
    res = f - fm.prolong(p, fm.restrict(p, f))
    pg = fm.prolong(p, g)
    ip = np.sum(dj[:, None, None] * res * pg)
    scale = np.sum(dj[:, None, None] * np.abs(res * pg))
    assert abs(ip) < 1e-13 * scale
    # the residual is not zero (f is not a prolonged state): the test has power
    assert np.abs(res).max() > 1e-2


@pytest.mark.parametrize("kind", ["periodic", "open"])
def test_transfer_conserves_and_copies(oracle_mod, kind):
    mi, om, fm, elems = _pair(oracle_mod, kind)
    p = 2
    rng = np.random.default_rng(3)
    g = rng.uniform(-1, 1, size=(om.ne, 4, 6))
    f = rng.uniform(-1, 1, size=(fm.ne, 4, 6))
    dc, df = om.detj(), fm.detj()
    tot = lambda d, c: (d[:, None] * c[:, :, 0]).sum(0)
    np.testing.assert_allclose(tot(df, fm.prolong(p, g)), tot(dc, g), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(tot(dc, fm.restrict(p, f)), tot(df, f), rtol=1e-13, atol=1e-13)
    # unrefined coarse elements are copied (children of refined ones take 4 slots)
    flag = np.zeros(om.ne, bool)
    flag[elems] = True
    first = np.concatenate([[0], np.cumsum(np.where(flag, 4, 1))[:-1]])
    keep = np.nonzero(~flag)[0]
    assert np.array_equal(fm.prolong(p, g)[first[keep]], g[keep])
    assert np.array_equal(fm.restrict(p, f)[keep], f[first[keep]])


def test_transfer_extended_agrees(oracle_mod):
    """The extended build's transfer agrees with the FP64 build's within FP64 rounding."""
    _, om, fm, _ = _pair(oracle_mod, "open")
    _, ox, fx, _ = _pair(oracle_mod, "open", build="extended")
    g = np.random.default_rng(4).uniform(-1, 1, size=(om.ne, 4, 10))
    a = fm.prolong(3, g)
    b = fx.prolong(3, g)
    assert np.abs(a - b.astype(np.float64)).max() < 1e-14 * np.abs(a).max()
