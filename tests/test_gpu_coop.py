"""dgc_rhs as one cooperative launch (DGC_OPT_COOPERATIVE): the phases of
Algorithm 1 separated by grid-wide barriers instead of kernel boundaries.  Per
element the arithmetic and its order are those of the separate launches, so
the right-hand side must equal theirs bit for bit (FP64 and FP32-mixed), on
closed conforming meshes (fused first color), open meshes (boundary edges; the
first color reaches part of the elements, a volume phase covers the rest) and
refined meshes with hanging edges (6 colors), and meet the oracle."""

import numpy as np
import pytest

from paper_1601_07613_gb300 import dgc
from paper_1601_07613_gb300 import workloads as W
from _parity import check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    dgc.lib()
    return torch, torch.device("cuda:0")


def _rhs(torch_dev, m, c, prec, coop):
    torch, dev = torch_dev
    dgc.dgc_set_option(m.h, dgc.DGC_OPT_COOPERATIVE, int(coop))
    cd = torch.empty(m.state_shape(), dtype=torch.float64, device=dev)
    r = torch.full_like(cd, float("nan"))
    dgc.dgc_import_state(m.h, c, cd)
    dgc.dgc_rhs(m.h, prec, cd, r)
    torch.cuda.synchronize()
    n = dgc.dgc_last_launch_count(m.h)
    return dgc.dgc_export_state(m.h, r), n


def _case(kind, p):
    if kind == "periodic":
        mi = W.periodic_square_tri(33, jitter=0.2, seed=71)
    elif kind == "open":
        mi = W.open_square_tri(27, jitter=0.2, seed=72)
    else:
        mi = W.periodic_square_tri(30, jitter=0.2, seed=73)
    return mi


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("kind", ["periodic", "open", "refined"])
def test_cooperative_rhs_bit_identical_and_matches_oracle(torch_dev, oracle_mod, kind, p):
    mi = _case(kind, p)
    m = dgc.Mesh.from_input(mi, p)
    m.color(1601)
    om = oracle_mod.OracleMesh.from_input(mi)
    if kind == "refined":
        elems = W.elements_near(mi, (0.45, 0.55), 0.3)
        col, _ = om.color(3, 1601)
        m.refine(elems)
        om = om.refine(col, elems)
        assert m.info["ncolors"] == 6
    c = W.random_state(om.ne, 4, m.info["np"], seed=p, amp=3e-3)
    ref = om.rhs(p, c)
    for prec, tol in ((dgc.DGC_FP64, 1e-12), (dgc.DGC_FP32_MIXED, 1e-5)):
        a, na = _rhs(torch_dev, m, c, prec, False)
        b, nb = _rhs(torch_dev, m, c, prec, True)
        assert nb == 1 and na > 1
        assert np.array_equal(a, b), f"{kind} p={p} prec {prec}"
        check(b, ref, tol, f"cooperative {kind} p={p}")
    m.close()


def test_cooperative_full_size_refined(torch_dev, oracle_mod):
    """The 180,512-element refined workload: one launch, the same bits as the
    seven launches (both precisions), FP32-mixed sampled against the oracle."""
    cfg = W.refined_square_vortex_p2_256()
    mi, p = cfg["mesh"], cfg["p"]
    m = dgc.Mesh.from_input(mi, p)
    m.color(1601)
    m.refine(cfg["refine"])
    om = oracle_mod.OracleMesh.from_input(mi)
    col, _ = om.color(3, 1601)
    om = om.refine(col, cfg["refine"])
    xyz, _, _ = om.eval_points(p)
    c = om.project(p, W.vortex_field(xyz[..., 0], xyz[..., 1], beta=cfg["beta"]))
    sample = np.random.default_rng(3).choice(om.ne, 1500, replace=False)
    ref = om.rhs(p, c, elems=sample)
    for prec in (dgc.DGC_FP64, dgc.DGC_FP32_MIXED):
        a, _ = _rhs(torch_dev, m, c, prec, False)
        b, n = _rhs(torch_dev, m, c, prec, True)
        assert n == 1 and np.array_equal(a, b)
        if prec == dgc.DGC_FP32_MIXED:  # (FP64: the separate launches' bits, checked against the exact result elsewhere)
            check(b[sample], ref, 1e-5, "cooperative full size FP32-mixed")
    m.close()


def test_cooperative_option_refused_on_quads(torch_dev):
    q = dgc.Mesh.from_input(W.periodic_square_quad(6, jitter=0.2, slant=0.3, seed=1), 1)
    with pytest.raises(dgc.DgcError):
        dgc.dgc_set_option(q.h, dgc.DGC_OPT_COOPERATIVE, 1)
    q.close()


@pytest.mark.parametrize("kind", ["periodic", "refined"])
def test_persistent_surface_kernels_bit_identical(torch_dev, oracle_mod, kind):
    """DGC_OPT_PERSISTENT (one wave of blocks, grid-stride over each color):
    the right-hand side in both precisions and two RK steps in every form equal
    the one-block-per-tile launches bit for bit, with tiles of 2 and 4 threads
    per edge."""
    torch, dev = torch_dev
    p = 3 if kind == "periodic" else 2
    mi = W.periodic_square_tri(96 if kind == "periodic" else 60, jitter=0.2, seed=74)
    m = dgc.Mesh.from_input(mi, p)
    m.color(1601)
    if kind == "refined":
        m.refine(W.elements_near(mi, (0.45, 0.55), 0.3))
    c = W.random_state(m.info["ne"], 4, m.info["np"], seed=5, amp=3e-3)
    for prec in (dgc.DGC_FP64, dgc.DGC_FP32_MIXED):
        dgc.dgc_set_option(m.h, dgc.DGC_OPT_PERSISTENT, 0)
        a, _ = _rhs(torch_dev, m, c, prec, False)
        dgc.dgc_set_option(m.h, dgc.DGC_OPT_PERSISTENT, 1)
        b, _ = _rhs(torch_dev, m, c, prec, False)
        assert np.array_equal(a, b), f"rhs {kind} prec {prec}"
    forms = [dgc.DGC_FP64, dgc.DGC_FP32_MIXED] + ([dgc.DGC_FP32_KAHAN] if kind == "periodic" else [])
    for prec in forms:
        for tpe in ((2, 4) if prec != dgc.DGC_FP64 and kind == "periodic" else (2,)):
            outs = []
            for pers in (0, 1):
                dgc.dgc_set_option(m.h, dgc.DGC_OPT_PERSISTENT, pers)
                dgc.dgc_set_option(m.h, dgc.DGC_OPT_EDGES_PER_BLOCK, 32)
                dgc.dgc_set_option(m.h, dgc.DGC_OPT_THREADS_PER_EDGE, tpe)
                if prec == dgc.DGC_FP32_KAHAN:
                    st = torch.empty(dgc.dgc_state_bytes(m.h, prec) // 4, dtype=torch.float32, device=dev)
                    dgc.dgc_import_state_prec(m.h, prec, c, st)
                else:
                    st = torch.empty(m.state_shape(), dtype=torch.float64, device=dev)
                    dgc.dgc_import_state(m.h, c, st)
                ws = torch.empty(dgc.dgc_workspace_size(m.h, prec) // 8 + 64, dtype=torch.float64, device=dev)
                d = torch.zeros(1, dtype=torch.float64, device=dev)
                for _ in range(2):
                    dgc.dgc_rk_step(m.h, prec, st, 0.3, d, ws)
                torch.cuda.synchronize()
                outs.append((st.clone(), d.item()))
            assert torch.equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1], f"{kind} prec {prec} tpe {tpe}"
    m.close()
