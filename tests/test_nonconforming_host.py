"""Nonconforming refinement and its 6-color map (Sec. 3.2): oracle pins, and the
library's refinement against the oracle's (bit-exact), on the CPU.

Pins of the oracle's map, independent of the code under test:
* the worked example of Sec. 3.2 (triangle DBA; children of BA get colors 1 and
  4; the interior edge GF, parallel to AD, gets 3), from the golden file;
* validity: no element has two edges (halves included) of one color;
* the six-refined-neighbours case, which needs all six colors;
* coarsening: the middle child carries the parent's edge colors (each on the
  edge parallel to the parent edge), so merging the children gives them back.
Pins of the oracle's right-hand side on meshes with hanging edges:
* freestream, and conservation on a periodic mesh;
* linear advection of a global polynomial of degree p, whose exact result is
  -a.grad(u): a coarse element that integrated the wrong half, length or
  points of a split edge would break it;
* refining every element gives a conforming mesh: the result equals the one of
  the same mesh built directly from its element list.
A second level (the map with its palette doubled again, 12 colors): validity,
the 2:1 refusal, the same right-hand-side pins on a two-level mesh, refining
every element twice, and the library's second level and its coarsening stack
against the oracle, bit for bit.
"""

import json
import os

import numpy as np
import pytest

from paper_1601_07613_gb300 import dgc
from paper_1601_07613_gb300 import workloads as W
from _amr import second_level

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def _colored(oracle_mod, mi, seed):
    om = oracle_mod.OracleMesh.from_input(mi)
    col, _ = om.color(3, seed)
    return om, col


def _edge_colors_per_element(m_sides, colors, ne):
    l, r, _, _ = m_sides
    per = [[] for _ in range(ne)]
    for s in range(len(l)):
        per[l[s]].append(colors[s])
        if r[s] >= 0:
            per[r[s]].append(colors[s])
    return per


def test_worked_example_sec32(oracle_mod):
    g = json.load(open(GOLDEN))["refinement_example"]
    # D = 0, B = 1, A = 2 (counterclockwise); parent edges DB, BA, AD
    xyz = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    om = oracle_mod.OracleMesh(2, xyz, np.array([[0, 1, 2]], np.int32))
    col = np.array(g["parent_colors"], np.int8)
    rm = om.refine(col, [0])
    ev, X = rm.elements()
    l, _, ql, _ = rm.sides()

    def vid(pt):
        for e in range(rm.ne):
            for k in range(3):
                if np.allclose(X[e, k], pt):
                    return ev[e, k]
        raise AssertionError(pt)

    D, B, A = 0, 1, 2
    G, F, E = vid([0.5, 0.5]), vid([0.5, 0.0]), vid([0.0, 0.5])  # midpoints of BA, DB, AD

    def color_of(x, y):
        for s in range(rm.ns):
            a, b = ev[l[s], ql[s]], ev[l[s], (ql[s] + 1) % 3]
            if {a, b} == {x, y}:
                return int(rm.colors[s])
        raise AssertionError((x, y))

    # the paper: BA's children BG, GA take 1 and 4 (B has the smaller id, so BG is
    # the first child under the global-vertex reading as well); GF, parallel to AD,
    # takes AD's color
    assert [color_of(B, G), color_of(G, A)] == g["children_of_edge2"]
    assert color_of(G, F) == g["interior_parallel_to_edge3"]
    # the other two interior edges follow the same rule: GE || DB, EF || BA
    assert color_of(G, E) == g["parent_colors"][0]
    assert color_of(E, F) == g["parent_colors"][1]
    assert rm.ne == 4 and rm.ns == 9 and (rm.hanging < 0).all()


@pytest.mark.parametrize("kind", ["periodic", "open"])
def test_refined_coloring_is_valid_and_uses_six_colors(oracle_mod, kind):
    mi = (W.periodic_square_tri(10, jitter=0.2, seed=21) if kind == "periodic"
          else W.open_square_tri(10, jitter=0.2, seed=21))
    om, col = _colored(oracle_mod, mi, 5)
    flag = np.random.default_rng(1).random(om.ne) < 0.3
    rm = om.refine(col, np.nonzero(flag)[0])
    assert rm.ne == om.ne + 3 * flag.sum()
    assert set(np.unique(rm.colors)) == {1, 2, 3, 4, 5, 6}
    for cs in _edge_colors_per_element(rm.sides(), rm.colors, rm.ne):
        assert len(cs) == len(set(cs)), cs
    # a coarse element with a hanging edge has 4..6 sides; fine ones exactly 3
    l, r, _, _ = rm.sides()
    nsides = np.bincount(np.concatenate([l, r[r >= 0]]), minlength=rm.ne)
    assert nsides.min() == 3 and nsides.max() <= 6
    hang = rm.hanging >= 0
    assert hang.any() and set(np.unique(rm.hanging[hang])) <= {0, 1}


def test_six_refined_neighbours(oracle_mod):
    mi = W.periodic_square_tri(8, jitter=0.15, seed=22)
    om, col = _colored(oracle_mod, mi, 9)
    l, r, _, _ = om.sides()
    e0 = 17
    nbrs = sorted({int(r[s]) for s in range(om.ns) if l[s] == e0} | {int(l[s]) for s in range(om.ns) if r[s] == e0})
    assert len(nbrs) == 3
    rm = om.refine(col, nbrs)
    # the coarse element is renumbered in place of itself; find it by its side count
    L, R, _, _ = rm.sides()
    cnt = np.bincount(np.concatenate([L, R[R >= 0]]), minlength=rm.ne)
    coarse = np.nonzero(cnt == 6)[0]
    assert len(coarse) == 1
    cs = [rm.colors[s] for s in range(rm.ns) if L[s] == coarse[0] or R[s] == coarse[0]]
    assert sorted(cs) == [1, 2, 3, 4, 5, 6]


def test_coarsening_recovers_parent_colors(oracle_mod):
    mi = W.periodic_square_tri(9, jitter=0.2, seed=23)
    om, col = _colored(oracle_mod, mi, 4)
    flag = np.zeros(om.ne, bool)
    flag[::4] = True
    rm = om.refine(col, np.nonzero(flag)[0])
    ev0, X0 = om.elements()
    ev, X = rm.elements()
    L, R, QL, QR = rm.sides()
    bl, br, bql, bqr = om.sides()
    first = np.cumsum(np.where(flag, 4, 1)) - np.where(flag, 4, 1)
    for e in np.nonzero(flag)[0]:
        mid = first[e] + 3
        for k in range(3):  # parent edge k and the middle child's edge parallel to it
            pk = X0[e, (k + 1) % 3] - X0[e, k]
            found = []
            for s in range(rm.ns):
                if R[s] == mid or L[s] == mid:
                    q = QR[s] if R[s] == mid else QL[s]
                    d = X[mid, (q + 1) % 3] - X[mid, q]
                    if abs(d[0] * pk[1] - d[1] * pk[0]) < 1e-12:
                        found.append(rm.colors[s])
            ps = [s for s in range(om.ns) if (bl[s] == e and bql[s] == k) or (br[s] == e and bqr[s] == k)]
            assert found == [col[ps[0]]]


def _refined_pair(oracle_mod, mi, p, seed, frac, rseed=1):
    """Library mesh and oracle mesh refined the same way (oracle colors come
    from its own coloring, equal to the library's bit for bit)."""
    om, col = _colored(oracle_mod, mi, seed)
    m = dgc.Mesh.from_input(mi, p)
    m.color(seed)
    flag = np.nonzero(np.random.default_rng(rseed).random(om.ne) < frac)[0]
    m.refine(flag)
    return m, om.refine(col, flag)


@pytest.mark.parametrize("kind,frac", [("periodic", 0.25), ("open", 0.4), ("periodic", 1.0), ("periodic", 0.0)])
def test_library_refinement_matches_oracle(oracle_mod, kind, frac):
    mi = (W.periodic_square_tri(12, jitter=0.2, seed=24) if kind == "periodic"
          else W.open_square_tri(12, jitter=0.2, seed=24))
    m, rm = _refined_pair(oracle_mod, mi, 2, 31, frac)
    for a, b in zip(dgc.dgc_get_sides(m.h), rm.sides()):
        np.testing.assert_array_equal(a, b)
    ev, X = dgc.dgc_get_elements(m.h)
    evo, Xo = rm.elements()
    np.testing.assert_array_equal(ev, evo)
    np.testing.assert_array_equal(X, Xo)
    np.testing.assert_array_equal(dgc.dgc_get_hanging(m.h), rm.hanging)
    en, sn, colL, off = dgc.dgc_get_ordering(m.h)
    np.testing.assert_array_equal(colL, rm.colors)
    en_o, sn_o, off_o = rm.reorder(rm.colors, 6)
    np.testing.assert_array_equal(en, en_o)
    np.testing.assert_array_equal(sn, sn_o)
    np.testing.assert_array_equal(off, off_o)
    assert m.info["ncolors"] == 6 and m.info["perfect"] == 0
    np.testing.assert_array_equal(dgc.dgc_mesh_info(m.h)["ne"], rm.ne)
    m.close()


def test_refine_errors():
    mi = W.periodic_square_tri(6, jitter=0.1, seed=25)
    m = dgc.Mesh.from_input(mi, 1)
    with pytest.raises(dgc.DgcError) as e:  # not colored
        m.refine([0])
    assert e.value.status == 1
    m.color(3)
    with pytest.raises(dgc.DgcError) as e:
        m.refine([m.info["ne"]])
    assert e.value.status == 1
    m.refine([0, 0, 5])  # duplicates are one element
    assert m.info["ne"] == 72 + 6
    l, r, _, _ = dgc.dgc_get_sides(m.h)
    hang = dgc.dgc_get_hanging(m.h) >= 0
    with pytest.raises(dgc.DgcError) as e:  # finer than its neighbour: 2:1 balance
        m.refine([int(l[hang][0])])
    assert e.value.status == 1
    m.refine([3])  # the middle child of element 0 (only siblings around it): level 2
    assert m.info["ncolors"] == 12
    with pytest.raises(dgc.DgcError) as e:  # a third level would need 24 colors
        m.refine([6])  # the middle grandchild
    assert e.value.status == 4
    t = dgc.Mesh.from_input(W.periodic_cube_tet(3), 1)
    t.color(1)
    with pytest.raises(dgc.DgcError) as e:
        t.refine([0])
    assert e.value.status == 4


# ---------------------------------------------------------------------------
# the oracle's right-hand side on meshes with hanging edges
# ---------------------------------------------------------------------------
def _refined_oracle(oracle_mod, mi, frac, seed=2):
    om, col = _colored(oracle_mod, mi, 7)
    flag = np.nonzero(np.random.default_rng(seed).random(om.ne) < frac)[0]
    return om.refine(col, flag)


def _const(ne, np_):
    ub = np.array([1.1, 0.3, -0.2, 2.6])
    c = np.zeros((ne, 4, np_))
    c[:, :, 0] = ub / np.sqrt(2.0)
    return c


@pytest.mark.parametrize("p", [1, 2, 3])
def test_refined_freestream(oracle_mod, p):
    rm = _refined_oracle(oracle_mod, W.periodic_square_tri(10, jitter=0.2, seed=26), 0.3)
    rhs = rm.rhs(p, _const(rm.ne, oracle_mod.npoly(2, p)))
    h = 1.0 / 20  # fine elements
    assert np.abs(rhs).max() * (0.5 * h * h) / (3.4 * h * 3.0) < 1e-13


@pytest.mark.parametrize("p", [1, 3])
def test_refined_conservation(oracle_mod, p):
    rm = _refined_oracle(oracle_mod, W.periodic_square_tri(10, jitter=0.2, seed=27), 0.35)
    c = W.random_state(rm.ne, 4, oracle_mod.npoly(2, p), seed=p, amp=2e-2)
    rhs = rm.rhs(p, c)
    detj = rm.detj()
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
def test_refined_linear_advection_closed_form(oracle_mod, p):
    """A global polynomial of degree p has no jumps across any edge, hanging or
    not, so Eq. 2 gives -a.grad(u) exactly on the nonconforming mesh too."""
    rm = _refined_oracle(oracle_mod, W.open_square_tri(7, jitter=0.2, seed=28), 0.4)
    assert (rm.hanging >= 0).sum() > 10
    a = np.array([0.7, -1.3])
    coef = np.random.default_rng(p).uniform(-1, 1, size=(p + 1) * (p + 2) // 2)
    xyz, _, _ = rm.eval_points(p, M=1)
    u, _, _ = _poly2(p, coef, xyz[..., 0], xyz[..., 1])
    c = rm.project(p, u[..., None])
    rhs = rm.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a)
    xyz2, _, U = rm.eval_points(p, c=rhs, n1=p + 3)
    _, gx, gy = _poly2(p, coef, xyz2[..., 0], xyz2[..., 1])
    np.testing.assert_allclose(U[..., 0], -(a[0] * gx + a[1] * gy), atol=1e-10)


@pytest.mark.parametrize("p", [1, 3])
def test_refined_linear_advection_brute_force(oracle_mod, p):
    """Discontinuous data across hanging edges, linear flux: the default rules
    equal 30-point rules (every integrand is a polynomial they integrate)."""
    rm = _refined_oracle(oracle_mod, W.periodic_square_tri(6, jitter=0.2, seed=29), 0.4)
    c = np.random.default_rng(p).uniform(-1, 1, size=(rm.ne, 1, oracle_mod.npoly(2, p)))
    a = np.array([0.4, 0.9])
    r0 = rm.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a)
    r1 = rm.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a, nq_face1=30, nq_vol1=30)
    np.testing.assert_allclose(r0, r1, atol=1e-12 * np.abs(r1).max())


def test_all_refined_equals_conforming_mesh(oracle_mod):
    """Refining every element leaves no hanging edge: Eq. 2 on the refined mesh
    equals Eq. 2 on the same triangles given as a plain element list."""
    mi = W.open_square_tri(6, jitter=0.2, seed=30)
    om, col = _colored(oracle_mod, mi, 3)
    rm = om.refine(col, np.arange(om.ne))
    ev, X = rm.elements()
    xyz = np.zeros((rm.nv, 2))
    xyz[ev.ravel()] = X.reshape(-1, 2)
    plain = oracle_mod.OracleMesh(2, xyz, ev)
    assert plain.ns == rm.ns and (rm.hanging < 0).all()
    c = W.random_state(rm.ne, 4, 10, seed=4, amp=2e-2)
    r0 = rm.rhs(3, c)
    r1 = plain.rhs(3, c)
    assert np.linalg.norm(r0 - r1) <= 1e-14 * np.linalg.norm(r1)


@pytest.mark.parametrize("frac", [0.3, 1.0])
def test_library_coarsening_restores_mesh_and_coloring(frac):
    """dgc_coarsen merges the children back; the parent colors it derives by the
    parallel-edge rule of Sec. 3.2 equal the coloring before refinement, and the
    mesh, its sides and its ordering come back bit for bit."""
    mi = W.periodic_square_tri(12, jitter=0.2, seed=60)
    m = dgc.Mesh.from_input(mi, 2)
    m.color(17)
    before = [dgc.dgc_get_sides(m.h), dgc.dgc_get_ordering(m.h), dgc.dgc_get_elements(m.h)]
    info = dict(m.info)
    flag = np.nonzero(np.random.default_rng(3).random(info["ne"]) < frac)[0]
    m.refine(flag)
    assert m.info["ncolors"] == 6
    m.coarsen()
    after = [dgc.dgc_get_sides(m.h), dgc.dgc_get_ordering(m.h), dgc.dgc_get_elements(m.h)]
    for a, b in zip(before, after):
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
    assert m.info == info
    assert (dgc.dgc_get_hanging(m.h) < 0).all()
    with pytest.raises(dgc.DgcError) as e:
        m.coarsen()
    assert e.value.status == 1
    m.refine(flag)  # and refine again
    assert m.info["ncolors"] == 6
    m.close()


# ---------------------------------------------------------------------------
# a second level of refinement
# ---------------------------------------------------------------------------
def _two_level(oracle_mod, mi, seed=7, frac=None, center=(0.45, 0.55), r1=0.3, r2=0.18):
    om, col = _colored(oracle_mod, mi, seed)
    e1 = W.elements_near(mi, center, r1)
    rm = om.refine(col, e1)
    e2 = second_level(rm, center, r2, r1 + 0.06)
    return om, col, e1, rm, e2, rm.refine(rm.colors, e2)


@pytest.mark.parametrize("kind", ["periodic", "open"])
def test_second_level_coloring_is_valid(oracle_mod, kind):
    mi = (W.periodic_square_tri(16, jitter=0.2, seed=61) if kind == "periodic"
          else W.open_square_tri(16, jitter=0.2, seed=61))
    om, col, e1, rm, e2, r2 = _two_level(oracle_mod, mi)
    assert len(e2) > 10 and (rm.levels[e2] == 0).any() and (rm.levels[e2] == 1).any()
    assert set(np.unique(r2.colors)) == set(range(1, 13))
    assert set(np.unique(r2.levels)) == {0, 1, 2}
    for cs in _edge_colors_per_element(r2.sides(), r2.colors, r2.ne):
        assert len(cs) == len(set(cs)), cs
    L, R, _, _ = r2.sides()
    hang = r2.hanging >= 0
    # every hanging edge joins elements one level apart; conforming edges equal levels
    assert (r2.levels[L[hang]] == r2.levels[R[hang]] + 1).all()
    conf = ~hang & (R >= 0)
    assert (r2.levels[L[conf]] == r2.levels[R[conf]]).all()
    # a level-L element's colors lie in 1..3 * 2^L (split edges of coarse ones aside)
    nsides = np.bincount(np.concatenate([L, R[R >= 0]]), minlength=r2.ne)
    for s in range(r2.ns):
        e = L[s]
        if nsides[e] == 3:
            assert r2.colors[s] <= 3 << r2.levels[e]


def test_second_level_refuses_a_finer_element(oracle_mod):
    mi = W.periodic_square_tri(10, jitter=0.2, seed=62)
    om, col = _colored(oracle_mod, mi, 3)
    rm = om.refine(col, W.elements_near(mi, (0.5, 0.5), 0.25))
    l, _, _, _ = rm.sides()
    fine = l[rm.hanging >= 0][0]
    with pytest.raises(ValueError):
        rm.refine(rm.colors, [fine])


@pytest.mark.parametrize("p", [1, 2, 3])
def test_second_level_freestream_and_conservation(oracle_mod, p):
    mi = W.periodic_square_tri(12, jitter=0.2, seed=63)
    *_, r2 = _two_level(oracle_mod, mi)
    rhs = r2.rhs(p, _const(r2.ne, oracle_mod.npoly(2, p)))
    h = 1.0 / 48  # finest elements
    assert np.abs(rhs).max() * (0.5 * h * h) / (3.4 * h * 3.0) < 1e-13
    c = W.random_state(r2.ne, 4, oracle_mod.npoly(2, p), seed=p, amp=2e-2)
    rhs = r2.rhs(p, c)
    detj = r2.detj()
    total = (detj[:, None] * rhs[:, :, 0]).sum(axis=0)
    scale = (detj[:, None] * np.abs(rhs[:, :, 0])).sum(axis=0)
    assert np.all(np.abs(total) < 1e-13 * scale)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_second_level_linear_advection_closed_form(oracle_mod, p):
    mi = W.open_square_tri(10, jitter=0.2, seed=64)
    *_, r2 = _two_level(oracle_mod, mi)
    assert ((r2.hanging >= 0) & (r2.levels[r2.sides()[0]] == 2)).sum() > 5
    a = np.array([0.7, -1.3])
    coef = np.random.default_rng(p).uniform(-1, 1, size=(p + 1) * (p + 2) // 2)
    xyz, _, _ = r2.eval_points(p, M=1)
    u, _, _ = _poly2(p, coef, xyz[..., 0], xyz[..., 1])
    c = r2.project(p, u[..., None])
    rhs = r2.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a)
    xyz2, _, U = r2.eval_points(p, c=rhs, n1=p + 3)
    _, gx, gy = _poly2(p, coef, xyz2[..., 0], xyz2[..., 1])
    np.testing.assert_allclose(U[..., 0], -(a[0] * gx + a[1] * gy), atol=1e-9)


@pytest.mark.parametrize("p", [1, 3])
def test_second_level_linear_advection_brute_force(oracle_mod, p):
    mi = W.periodic_square_tri(8, jitter=0.2, seed=65)
    *_, r2 = _two_level(oracle_mod, mi)
    c = np.random.default_rng(p).uniform(-1, 1, size=(r2.ne, 1, oracle_mod.npoly(2, p)))
    a = np.array([0.4, 0.9])
    r0 = r2.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a)
    r1 = r2.rhs(p, c, kind=oracle_mod.ADVECTION, adv=a, nq_face1=30, nq_vol1=30)
    np.testing.assert_allclose(r0, r1, atol=1e-12 * np.abs(r1).max())


def test_all_refined_twice_equals_conforming_mesh(oracle_mod):
    mi = W.open_square_tri(4, jitter=0.2, seed=66)
    om, col = _colored(oracle_mod, mi, 3)
    rm = om.refine(col, np.arange(om.ne))
    r2 = rm.refine(rm.colors, np.arange(rm.ne))
    assert (r2.hanging < 0).all() and set(np.unique(r2.levels)) == {2}
    ev, X = r2.elements()
    xyz = np.zeros((r2.nv, 2))
    xyz[ev.ravel()] = X.reshape(-1, 2)
    plain = oracle_mod.OracleMesh(2, xyz, ev)
    assert plain.ns == r2.ns
    c = W.random_state(r2.ne, 4, 10, seed=4, amp=2e-2)
    r0 = r2.rhs(3, c)
    r1 = plain.rhs(3, c)
    assert np.linalg.norm(r0 - r1) <= 1e-14 * np.linalg.norm(r1)


@pytest.mark.parametrize("kind", ["periodic", "open"])
def test_library_second_level_matches_oracle_and_coarsens_back(oracle_mod, kind):
    mi = (W.periodic_square_tri(16, jitter=0.2, seed=67) if kind == "periodic"
          else W.open_square_tri(16, jitter=0.2, seed=67))
    om, col, e1, rm, e2, r2 = _two_level(oracle_mod, mi, seed=31)
    m = dgc.Mesh.from_input(mi, 2)
    m.color(31)
    states = [(dgc.dgc_get_sides(m.h), dgc.dgc_get_ordering(m.h), dgc.dgc_get_elements(m.h), dict(m.info))]
    m.refine(e1)
    states.append((dgc.dgc_get_sides(m.h), dgc.dgc_get_ordering(m.h), dgc.dgc_get_elements(m.h), dict(m.info)))
    m.refine(e2)
    for a, b in zip(dgc.dgc_get_sides(m.h), r2.sides()):
        np.testing.assert_array_equal(a, b)
    ev, X = dgc.dgc_get_elements(m.h)
    evo, Xo = r2.elements()
    np.testing.assert_array_equal(ev, evo)
    np.testing.assert_array_equal(X, Xo)
    np.testing.assert_array_equal(dgc.dgc_get_hanging(m.h), r2.hanging)
    en, sn, colL, off = dgc.dgc_get_ordering(m.h)
    np.testing.assert_array_equal(colL, r2.colors)
    en_o, sn_o, off_o = r2.reorder(r2.colors, 12)
    np.testing.assert_array_equal(en, en_o)
    np.testing.assert_array_equal(sn, sn_o)
    np.testing.assert_array_equal(off, off_o)
    assert m.info["ncolors"] == 12 and m.info["perfect"] == 0
    for want in reversed(states):  # coarsening undoes one level at a time
        m.coarsen()
        got = (dgc.dgc_get_sides(m.h), dgc.dgc_get_ordering(m.h), dgc.dgc_get_elements(m.h))
        for a, b in zip(want[:3], got):
            for x, y in zip(a, b):
                np.testing.assert_array_equal(x, y)
        assert m.info == want[3]
    with pytest.raises(dgc.DgcError):
        m.coarsen()
    m.refine(e1)  # and both levels come back the same
    m.refine(e2)
    np.testing.assert_array_equal(dgc.dgc_get_ordering(m.h)[2], r2.colors)
    m.close()


def test_second_level_selection_helpers_agree(oracle_mod):
    """The bench's second-level selection (workloads.second_level_elements, from
    the library's sides, hanging flags and elements) picks the same elements as
    the tests' (from the oracle's levels), and the library refines them."""
    ref = W.refined_square_vortex_p2_256(n=48, radius=0.2)
    mi = ref["mesh"]
    om, col = _colored(oracle_mod, mi, 1601)
    rm = om.refine(col, ref["refine"])
    m = dgc.Mesh.from_input(mi, 2)
    m.color(1601)
    m.refine(ref["refine"])
    l, r, _, _ = dgc.dgc_get_sides(m.h)
    _, xyz = dgc.dgc_get_elements(m.h)
    got = W.second_level_elements(ref["refine"], mi.ne, l, r, dgc.dgc_get_hanging(m.h), xyz, (0.5, 0.5), 0.1, 0.23)
    want = second_level(rm, (0.5, 0.5), 0.1, 0.23)
    np.testing.assert_array_equal(got, want)
    assert len(got) > 10
    m.refine(got)
    assert m.info["ncolors"] == 12
    np.testing.assert_array_equal(dgc.dgc_get_ordering(m.h)[2], rm.refine(rm.colors, want).colors)
    m.close()
