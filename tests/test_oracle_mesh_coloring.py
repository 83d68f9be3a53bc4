"""Pins for the oracle's edge table, coloring (Sec. 3.1) and reordering (Sec. 5).

The coloring is checked against the paper's definition of a valid coloring
(no element carries two edges of one color, Sec. 1 / Sec. 3), the minimal color
counts (3 for triangles, 4 for tetrahedra, Sec. 3), the closed-mesh count of
exactly one third (quarter) of the sides per color (Table 1, spherical shells),
the conflict fraction of the greedy pass (Fig. "graphs", left) and the
structure of the renumbered connectivity (Tables 5b and 6b).
"""

import json
import os

import numpy as np
import pytest

from paper_1601_07613_gb300 import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _rows(key):
    return [v for v in GOLDEN[key].values() if isinstance(v, dict)]


def valid_coloring(l, r, ql, qr, col, ne, nfpe, nc):
    """Independent checker: every element's faces carry pairwise distinct colors in 1..nc."""
    if col.min() < 1 or col.max() > nc:
        return False
    slots = np.zeros((ne, nfpe), np.int64)
    slots[l, ql] = col
    inner = r >= 0
    slots[r[inner], qr[inner]] = col[inner]
    srt = np.sort(slots, axis=1)
    return bool(np.all(srt[:, 1:] != srt[:, :-1]))


def test_edge_table_counts_periodic(oracle_mod):
    for n in (3, 8, 17):
        m = oracle_mod.OracleMesh.from_input(W.periodic_square_tri(n))
        assert m.ne == 2 * n * n and m.ns == 3 * n * n
        l, r, ql, qr = m.sides()
        assert np.all(r >= 0) and np.all(l != r)
        # first appearance: element 0's local edges come first, in order
        assert list(l[:3]) == [0, 0, 0] and list(ql[:3]) == [0, 1, 2]
        assert np.all(np.diff(l) >= 0)  # lefts appear in scan order
        np.testing.assert_allclose(m.detj().sum() / 2.0, 1.0, rtol=1e-13)


def test_edge_table_open_boundary_identity(oracle_mod):
    """sides - 1.5 E = (number of boundary sides) / 2 (each row of Table 1 obeys it)."""
    for row in _rows("table1_open_meshes"):
        nb = 2 * (row["sides"] - 1.5 * row["elements"])
        assert nb == int(nb) and nb > 0
    for n in (4, 9):
        m = oracle_mod.OracleMesh.from_input(W.open_square_tri(n, jitter=0.2, seed=3))
        _, r, _, _ = m.sides()
        nbnd = int(np.sum(r < 0))
        assert nbnd == 4 * n
        assert m.ns - 1.5 * m.ne == nbnd / 2


def test_mesh_errors(oracle_mod):
    mi = W.periodic_square_tri(4)
    bad = mi.ev.copy()
    bad[0] = bad[0, ::-1]  # clockwise -> negative Jacobian
    with pytest.raises(ValueError):
        oracle_mod.OracleMesh(2, mi.xyz, bad, mi.periodic_len)
    ev3 = np.concatenate([mi.ev, mi.ev[:1]], axis=0)  # a face shared three times
    with pytest.raises(ValueError):
        oracle_mod.OracleMesh(2, mi.xyz, ev3, mi.periodic_len)


@pytest.mark.parametrize("seed", [1, 2, 1601, 0])
@pytest.mark.parametrize("n", [3, 5, 16, 64])
def test_coloring_valid_three_colors_closed(oracle_mod, n, seed):
    m = oracle_mod.OracleMesh.from_input(W.periodic_square_tri(n, jitter=0.2, seed=seed))
    col, st = m.color(3, seed)
    l, r, ql, qr = m.sides()
    assert valid_coloring(l, r, ql, qr, col, m.ne, 3, 3)
    # closed mesh: each element has one edge of each color -> E/2 per color
    assert list(np.bincount(col, minlength=4)[1:]) == [m.ne // 2] * 3


def test_sphere_rows_of_table1_are_exact_thirds():
    for row in _rows("table1_closed_meshes"):
        assert row["per_color"] == [row["sides"] // 3] * 3 == [row["elements"] // 2] * 3


@pytest.mark.parametrize("n", [6, 40])
def test_coloring_valid_open(oracle_mod, n):
    m = oracle_mod.OracleMesh.from_input(W.open_square_tri(n, jitter=0.2, seed=n))
    col, _ = m.color(3, 7)
    l, r, ql, qr = m.sides()
    assert valid_coloring(l, r, ql, qr, col, m.ne, 3, 3)
    counts = np.bincount(col, minlength=4)[1:]
    assert counts.sum() == m.ns and counts.max() - counts.min() <= 0.05 * m.ns


@pytest.mark.parametrize("n", [3, 6])
def test_coloring_tets_four_colors(oracle_mod, n):
    m = oracle_mod.OracleMesh.from_input(W.periodic_cube_tet(n))
    assert m.ne == 6 * n ** 3 and m.ns == 12 * n ** 3
    col, _ = m.color(4, 11)
    l, r, ql, qr = m.sides()
    assert valid_coloring(l, r, ql, qr, col, m.ne, 4, 4)
    assert list(np.bincount(col, minlength=5)[1:]) == [m.ne // 2] * 4


def test_greedy_conflict_fraction_band(oracle_mod):
    """Fig. 'graphs': ~11% of the sides are left uncolored by the greedy pass."""
    paper = [c / s for s, c in GOLDEN["greedy_conflicts"]["triangles"]]
    assert 0.10 < min(paper) and max(paper) < 0.12
    m = oracle_mod.OracleMesh.from_input(W.periodic_square_tri(200, jitter=0.2, seed=1601))
    _, st = m.color(3, 1601)
    frac = st["greedy_conflicts"] / m.ns
    assert 0.07 < frac < 0.15


def test_swap_cap_is_reported(oracle_mod):
    m = oracle_mod.OracleMesh.from_input(W.periodic_square_tri(32))
    with pytest.raises(RuntimeError, match="swap cap"):
        m.color(3, 5, max_swaps=1)


def test_coloring_deterministic_per_seed(oracle_mod):
    m = oracle_mod.OracleMesh.from_input(W.periodic_square_tri(20, jitter=0.2, seed=1))
    a, _ = m.color(3, 42)
    b, _ = m.color(3, 42)
    c, _ = m.color(3, 43)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_naive_greedy_needs_more_colors(oracle_mod):
    """Sec. 1: the first-available greedy coloring uses up to five colors on triangles
    (element order shuffled, as from an unstructured mesh generator)."""
    mi = W.periodic_square_tri(40, jitter=0.2, seed=2)
    ev = mi.ev[np.random.default_rng(0).permutation(mi.ne)]
    m = oracle_mod.OracleMesh(2, mi.xyz, ev, mi.periodic_len)
    col, nc = m.color_naive()
    l, r, ql, qr = m.sides()
    assert 3 < nc <= 5 and valid_coloring(l, r, ql, qr, col, m.ne, 3, nc)


@pytest.mark.parametrize("mesh", ["periodic", "open"])
def test_reorder_structure_tables_5_and_6(oracle_mod, mesh):
    mi = (W.periodic_square_tri(24, jitter=0.2, seed=4) if mesh == "periodic"
          else W.open_square_tri(24, jitter=0.2, seed=4))
    m = oracle_mod.OracleMesh.from_input(mi)
    col, _ = m.color(3, 9)
    en, sn, off = m.reorder(col, 3)
    assert sorted(en) == list(range(m.ne)) and sorted(sn) == list(range(m.ns))
    l, r, _, _ = m.sides()
    inv = np.empty(m.ns, np.int64)
    inv[sn] = np.arange(m.ns)
    L = en[l[inv]]
    R = np.where(r[inv] >= 0, en[np.maximum(r[inv], 0)], -1)
    C = col[inv]
    n1 = off[1]
    assert np.all(C[:n1] == 1) and np.all(C[off[1]:off[2]] == 2) and np.all(C[off[2]:] == 3)
    # Table 5b: the k-th color-1 edge joins elements k and N1 + k
    assert np.array_equal(L[:n1], np.arange(n1))
    inner = R[:n1] >= 0
    if mesh == "periodic":
        assert np.all(inner) and np.array_equal(R[:n1], n1 + np.arange(n1))
    else:
        assert np.array_equal(R[:n1][inner], n1 + np.arange(int(inner.sum())))
    # Table 6b: colors >= 2 have strictly ascending left elements
    for c in (2, 3):
        seg = L[off[c - 1]:off[c]]
        assert np.all(np.diff(seg) > 0)
