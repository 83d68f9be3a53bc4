"""CPU checks of the CUDA library's host side and of its C ABI (no GPU calls).

* the shared library loads and exports every function include/dgc.h declares;
* its edge table, coloring and reordering equal the oracle's bit for bit;
* its host L2 projection (own quadrature and basis tables) agrees with the
  oracle's to rounding;
* the two-pass buffer size reproduces Table 4;
* error statuses for bad meshes, the swap cap and calls out of order.
"""

import json
import os
import re

import numpy as np
import pytest

from paper_1601_07613_gb300 import dgc
from paper_1601_07613_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_values.json")))


@pytest.fixture(scope="module")
def L():
    return dgc.lib()


def header_functions():
    txt = open(os.path.join(ROOT, "include", "dgc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dgc_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_function(L):
    names = header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
        assert n in dgc.SIGNATURES, n


MESHES = [
    ("periodic3", lambda: W.periodic_square_tri(3)),
    ("periodic7j", lambda: W.periodic_square_tri(7, jitter=0.2, seed=7)),
    ("periodic64j", lambda: W.periodic_square_tri(64, jitter=0.2, seed=1601)),
    ("open9j", lambda: W.open_square_tri(9, jitter=0.2, seed=9)),
    ("open40", lambda: W.open_square_tri(40)),
    ("tet3", lambda: W.periodic_cube_tet(3)),
    ("tet5", lambda: W.periodic_cube_tet(5)),
    ("quad6p", lambda: W.periodic_square_quad(6, jitter=0.2, slant=0.3, seed=4)),
    ("quad30v", lambda: W.periodic_square_quad(30, "vertex", jitter=0.2, seed=5)),
    ("quad9open", lambda: W.open_square_quad(9, "vertex", jitter=0.2, seed=6)),
    ("hybrid12", lambda: W.hybrid_square(12, 0.3, seed=7)),
    ("hybrid11open", lambda: W.hybrid_square(11, 0.4, periodic=False, jitter=0.2, seed=8)),
]


def _ncolors(mi):
    return 4 if mi.dim == 2 and mi.ev.shape[1] == 4 else mi.dim + 1


@pytest.mark.parametrize("name,make", MESHES)
@pytest.mark.parametrize("seed", [0, 1, 1601])
def test_coloring_and_ordering_bit_exact_vs_oracle(oracle_mod, name, make, seed):
    mi = make()
    p = 1
    m = dgc.Mesh.from_input(mi, p)
    om = oracle_mod.OracleMesh.from_input(mi)
    for a, b in zip(dgc.dgc_get_sides(m.h), om.sides()):
        assert np.array_equal(a, b)
    nc, per = m.color(seed)
    col_o, _ = om.color(_ncolors(mi), seed)
    en, sn, col, off = dgc.dgc_get_ordering(m.h)
    assert nc == _ncolors(mi)
    assert np.array_equal(col, col_o)
    en_o, sn_o, off_o = om.reorder(col_o, nc)
    assert np.array_equal(en, en_o) and np.array_equal(sn, sn_o) and np.array_equal(off, off_o)
    assert list(np.diff(off)) == per
    m.close()


def test_coloring_bit_exact_large(oracle_mod):
    """The configuration-2 mesh family at a quarter of the size (262k triangles)."""
    mi = W.periodic_square_tri(362, jitter=0.2, seed=1601)
    m = dgc.Mesh.from_input(mi, 3)
    om = oracle_mod.OracleMesh.from_input(mi)
    m.color(1601)
    col_o, _ = om.color(3, 1601)
    en, sn, col, off = dgc.dgc_get_ordering(m.h)
    assert np.array_equal(col, col_o)
    en_o, sn_o, _ = om.reorder(col_o, 3)
    assert np.array_equal(en, en_o) and np.array_equal(sn, sn_o)
    assert list(np.diff(off)) == [mi.ne // 2] * 3


@pytest.mark.parametrize("p", [1, 2, 3])
def test_projection_matches_oracle(oracle_mod, p):
    mi = W.periodic_square_tri(10, jitter=0.2, seed=2)
    m = dgc.Mesh.from_input(mi, p)
    om = oracle_mod.OracleMesh.from_input(mi)
    xyz = dgc.dgc_vol_points(m.h)
    xyz_o, _, _ = om.eval_points(p)
    np.testing.assert_allclose(xyz, xyz_o, atol=1e-15)
    vals = W.vortex_field(xyz[..., 0], xyz[..., 1])
    c = dgc.dgc_project(m.h, vals)
    c_o = om.project(p, vals)
    np.testing.assert_allclose(c, c_o, atol=1e-13 * np.abs(c_o).max())


@pytest.mark.parametrize("p", [1, 2, 3])
def test_projection_matches_oracle_quad(oracle_mod, p):
    mi = W.periodic_square_quad(8, jitter=0.2, slant=0.3, seed=2)
    m = dgc.Mesh.from_input(mi, p)
    assert (m.elem, m.nonaffine) == (dgc.DGC_QUAD, 0)
    assert m.info["np"] == (p + 1) ** 2
    om = oracle_mod.OracleMesh.from_input(mi)
    xyz = dgc.dgc_vol_points(m.h)
    xyz_o, _, _ = om.eval_points(p)
    np.testing.assert_allclose(xyz, xyz_o, atol=1e-15)
    vals = W.vortex_field(xyz[..., 0], xyz[..., 1])
    c_o = om.project(p, vals)
    np.testing.assert_allclose(dgc.dgc_project(m.h, vals), c_o, atol=1e-13 * np.abs(c_o).max())
    np.testing.assert_allclose(dgc.dgc_mesh_info(m.h)["ne"], mi.ne)


@pytest.mark.parametrize("p", [1, 3])
@pytest.mark.parametrize("kind", ["quad", "hybrid"])
def test_projection_matches_oracle_bilinear(oracle_mod, p, kind):
    """General quadrilaterals: the volume points under the bilinear map and the
    L2 projection through each element's own mass matrix, as the oracle's."""
    mi = (W.periodic_square_quad(8, "vertex", 0.2, seed=3) if kind == "quad"
          else W.hybrid_square(8, 0.3, jitter=0.2, seed=3))
    m = dgc.Mesh.from_input(mi, p)
    assert m.elem == dgc.DGC_QUAD and m.nonaffine > 0
    om = oracle_mod.OracleMesh.from_input(mi)
    xyz = dgc.dgc_vol_points(m.h)
    xyz_o, _, _ = om.eval_points(p)
    np.testing.assert_allclose(xyz, xyz_o, atol=1e-15)
    vals = W.vortex_field(xyz[..., 0], xyz[..., 1])
    c_o = om.project(p, vals)
    np.testing.assert_allclose(dgc.dgc_project(m.h, vals), c_o, atol=1e-12 * np.abs(c_o).max())
    m.close()


def test_quad_mesh_statuses(L):
    """Non-convex or clockwise quadrilaterals are mesh errors; a hybrid mesh
    (of parallelograms and triangles, or with general quadrilaterals) and a mesh
    of general quadrilaterals take device calls in FP64 only, the others refused
    on the host, and cannot be refined; an odd closed quadrilateral mesh cannot
    be 4-colored."""
    mi = W.periodic_square_quad(6)
    bad = mi.ev.copy()
    bad[3] = bad[3, ::-1]
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_mesh_create_elem(dgc.DGC_QUAD, 1, mi.xyz, bad, mi.periodic_len)
    assert e.value.status == 2
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_mesh_create_elem(dgc.DGC_QUAD, 4, mi.xyz, mi.ev, mi.periodic_len)
    assert e.value.status == 4
    h = dgc.Mesh.from_input(W.hybrid_square(8, 0.3, seed=1), 2)  # unjittered squares and triangles: affine
    assert h.elem == dgc.DGC_QUAD and h.nonaffine == 0
    h.color(3)
    with pytest.raises(dgc.DgcError) as e:  # hybrid meshes: FP64 and FP32-mixed, no Kahan form
        dgc.dgc_rhs(h.h, dgc.DGC_FP32_KAHAN, 4096, 8192, 0)
    assert e.value.status == 4
    h.close()
    for gen in (lambda: W.hybrid_square(8, 0.3, jitter=0.2, seed=1),
                lambda: W.periodic_square_quad(8, "vertex", 0.2, seed=1)):
        g = gen()
        m = dgc.Mesh.from_input(g, 2)
        assert m.elem == dgc.DGC_QUAD and m.nonaffine > 0
        m.color(3)
        with pytest.raises(dgc.DgcError) as e:
            dgc.dgc_rhs(m.h, dgc.DGC_FP32_KAHAN, 4096, 8192, 0)
        assert e.value.status == 4
        with pytest.raises(dgc.DgcError) as e:
            dgc.dgc_refine(m.h, np.array([0], np.int32))
        assert e.value.status == 4
        m.close()
    m = dgc.Mesh.from_input(W.periodic_square_quad(5), 1)
    with pytest.raises(dgc.DgcError) as e:
        m.color(1, max_swaps=20000)
    assert e.value.status == 3
    m.close()


@pytest.mark.parametrize("p", [1, 2])
def test_projection_matches_oracle_tet(oracle_mod, p):
    mi = W.periodic_cube_tet(3)
    m = dgc.Mesh.from_input(mi, p)
    om = oracle_mod.OracleMesh.from_input(mi)
    xyz = dgc.dgc_vol_points(m.h)
    vals = W.vortex_tube_field(xyz[..., 0], xyz[..., 1], xyz[..., 2])
    np.testing.assert_allclose(dgc.dgc_project(m.h, vals), om.project(p, vals), atol=1e-12)


def test_table4_buffer_memory(L):
    row = GOLDEN["table4_memory_saved_gb"]
    for p, gb in zip(row["p"], row["gb"]):
        np_ = (p + 1) * (p + 2) // 2
        b = dgc.dgc_two_pass_buffer_bytes(row["sides"], np_, row["neq"], 8)
        # the table truncates to two decimals (1.4493 GB is printed as 1.44)
        assert int(b / 1e9 * 100) / 100 == gb


def test_error_statuses(L):
    mi = W.periodic_square_tri(4)
    bad = mi.ev.copy()
    bad[3] = bad[3, ::-1]
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_mesh_create(2, 1, mi.xyz, bad, mi.periodic_len)
    assert e.value.status == 2
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_mesh_create(2, 1, mi.xyz, np.concatenate([mi.ev, mi.ev[:1]]), mi.periodic_len)
    assert e.value.status == 2
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_mesh_create(2, 7, mi.xyz, mi.ev, mi.periodic_len)
    assert e.value.status == 4
    m = dgc.Mesh.from_input(W.periodic_square_tri(24), 1)
    with pytest.raises(dgc.DgcError) as e:
        m.color(5, max_swaps=1)
    assert e.value.status == 3
    # device calls before coloring fail on the host, before any device work
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_rhs(m.h, dgc.DGC_FP64, 4096, 8192, 0)
    assert e.value.status == 1
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_rhs(m.h, dgc.DGC_FP64, 4097, 8192, 0)  # misaligned
    assert e.value.status == 1
    with pytest.raises(dgc.DgcError):
        dgc.dgc_set_option(m.h, dgc.DGC_OPT_EDGES_PER_BLOCK, 7)
    m.close()


def test_naive_coloring_ablation(L):
    mi = W.periodic_square_tri(30, jitter=0.2, seed=2)
    ev = mi.ev[np.random.default_rng(0).permutation(mi.ne)]
    m = dgc.Mesh(2, 1, mi.xyz, ev, mi.periodic_len)
    nc, per = dgc.dgc_color_edges_naive(m.h, True, True)
    assert 3 < nc <= 5 and sum(per) == m.info["ns"]
    info = dgc.dgc_mesh_info(m.h)
    assert info["ncolors"] == nc and info["perfect"] == 0
    m.close()


@pytest.mark.parametrize("renumber,reorder", [(False, False), (True, False), (False, True), (True, True)])
def test_reorder_switches(L, oracle_mod, renumber, reorder):
    """The Table 7 ordering switches on an existing coloring: edges stay
    color-major (stable by original id); without renumbering elements keep their
    ids; without the left sort colors >= 2 keep original edge order; with both on
    the result equals the full Sec. 5 ordering (and the oracle's)."""
    mi = W.periodic_square_tri(14, jitter=0.2, seed=3)
    m = dgc.Mesh.from_input(mi, 1)
    m.color(5)
    en_full, sn_full, col, off = dgc.dgc_get_ordering(m.h)
    dgc.dgc_reorder(m.h, renumber, reorder)
    en, sn, col2, off2 = dgc.dgc_get_ordering(m.h)
    np.testing.assert_array_equal(col2, col)
    np.testing.assert_array_equal(off2, off)
    order = np.empty(len(sn), np.int64)
    order[sn] = np.arange(len(sn))  # original edge at each new position
    assert np.all(np.diff(col[order]) >= 0)  # color-major
    if not renumber:
        np.testing.assert_array_equal(en, np.arange(mi.ne))
    l, _, _, _ = dgc.dgc_get_sides(m.h)
    for c in range(2, len(off)):
        seg = order[off[c - 1]:off[c]]
        if reorder:
            assert np.all(np.diff(en[l[seg]]) >= 0)
        else:
            assert np.all(np.diff(seg) > 0)
    if renumber and reorder:
        np.testing.assert_array_equal(en, en_full)
        np.testing.assert_array_equal(sn, sn_full)
    m.close()


def test_buffer_sizes_are_checked_before_device_work(L):
    """The RK workspace and the two-pass buffer carry their sizes; too small is an
    argument error returned on the host, before anything is enqueued."""
    m = dgc.Mesh.from_input(W.periodic_square_tri(8), 2)
    m.color(1)
    need = dgc.dgc_workspace_size(m.h, dgc.DGC_FP32_MIXED)
    assert need >= dgc.dgc_workspace_size(m.h, dgc.DGC_FP64) - 512  # mixed keeps an FP32 record too
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_rk_step(m.h, dgc.DGC_FP32_MIXED, 4096, 0.3, 8192, 1 << 20, workspace_bytes=need - 1, stream=0)
    assert e.value.status == 1 and "workspace" in str(e.value)
    info = m.info
    nb = dgc.dgc_two_pass_buffer_bytes(info["ns"], info["np"], info["M"], 8)
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_rhs_two_pass(m.h, dgc.DGC_FP64, 4096, 8192, 1 << 20, buffer_bytes=nb - 8, stream=0)
    assert e.value.status == 1 and "buffer" in str(e.value)
    m.close()


def test_boundary_arguments_are_checked_on_the_host(L):
    """dgc_set_boundary validates kinds, state indices and the shock before any
    device work; quadrilateral meshes refuse it; the time round-trips on the
    host before the first upload; the FP32 forms refuse the limiter."""
    mi = W.open_rect_tri(8, 2, 4.0, 1.0)
    m = dgc.Mesh.from_input(mi, 1)
    m.color(1)
    l, r, ql, qr = dgc.dgc_get_sides(m.h)
    kind, sidx = W.double_mach_boundary(mi, l, r, ql)
    S = W.double_mach_states()
    dgc.dgc_set_boundary(m.h, kind, sidx, S, W.DMR_SHOCK, (0, 1))
    bad = kind.copy()
    bad[np.nonzero(r < 0)[0][0]] = 7
    for args in ((bad, sidx, S, W.DMR_SHOCK, (0, 1)),       # unknown kind
                 (kind, sidx + 5, S, W.DMR_SHOCK, (0, 1)),  # state index out of range (state faces)
                 (kind, sidx, S, None, None),               # shock faces without the shock
                 (kind, sidx, S, W.DMR_SHOCK, (0, 2))):     # shock state out of range
        with pytest.raises(dgc.DgcError) as e:
            dgc.dgc_set_boundary(m.h, *args)
        assert e.value.status == 1
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_set_boundary(m.h, kind, sidx, np.zeros((9, 4)), W.DMR_SHOCK, (0, 1))
    assert e.value.status == 1
    dgc.dgc_set_time(m.h, 0.125)
    assert dgc.dgc_get_time(m.h) == 0.125
    dgc.dgc_set_option(m.h, dgc.DGC_OPT_LIMITER, 1)  # the limiter runs in FP64 only
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_rhs(m.h, dgc.DGC_FP32_MIXED, 4096, 8192, 0)
    assert e.value.status == 4
    m.close()
    q = dgc.Mesh.from_input(W.open_square_quad(4), 1)
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_set_boundary(q.h, np.zeros(q.info["ns"], np.int8))
    assert e.value.status == 4
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_set_option(q.h, dgc.DGC_OPT_LIMITER, 1)
    assert e.value.status == 4
    q.close()

