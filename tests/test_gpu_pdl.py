"""Programmatic dependent launch of the RK step's kernels (DGC_OPT_PDL): each
surface kernel starts its flux work while its predecessor drains and waits
for the predecessor before its epilogue.  The order of every read and write
is unchanged, so the step must give bit-identical states and time steps with
and without it, in every precision form, fused and unfused, on conforming and
refined meshes."""

import numpy as np
import pytest

from paper_1601_07613_gb300 import dgc
from paper_1601_07613_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    dgc.lib()
    return torch, torch.device("cuda:0")


def _steps(torch, dev, m, prec, c_host, pdl, n=4, cfl=0.3):
    dgc.dgc_set_option(m.h, dgc.DGC_OPT_PDL, int(pdl))
    if prec == dgc.DGC_FP32_KAHAN:
        st = torch.empty(dgc.dgc_state_bytes(m.h, prec) // 4, dtype=torch.float32, device=dev)
        dgc.dgc_import_state_prec(m.h, prec, c_host, st)
    else:
        st = torch.empty(m.state_shape(), dtype=torch.float64, device=dev)
        dgc.dgc_import_state(m.h, c_host, st)
    ws = torch.empty(dgc.dgc_workspace_size(m.h, prec) // 8 + 64, dtype=torch.float64, device=dev)
    dt = torch.zeros(1, dtype=torch.float64, device=dev)
    dts = []
    for _ in range(n):
        dgc.dgc_rk_step(m.h, prec, st, cfl, dt, ws)
        dts.append(float(dt.item()))
    torch.cuda.synchronize()
    out = dgc.dgc_export_state_prec(m.h, prec, st) if prec == dgc.DGC_FP32_KAHAN else dgc.dgc_export_state(m.h, st)
    assert np.isfinite(out).all() and all(0.0 < d < 1.0 for d in dts)  # a physical run
    return out, dts


@pytest.mark.parametrize("prec", [dgc.DGC_FP32_MIXED, dgc.DGC_FP32_KAHAN, dgc.DGC_FP64])
@pytest.mark.parametrize("p", [1, 3])
@pytest.mark.parametrize("fuse", [True, False])
def test_pdl_steps_bit_identical(torch_dev, prec, p, fuse):
    torch, dev = torch_dev
    mi = W.periodic_square_tri(40, jitter=0.2, seed=71)
    m = dgc.Mesh.from_input(mi, p)
    m.color(1601)
    dgc.dgc_set_option(m.h, dgc.DGC_OPT_FUSE, int(fuse))
    c = W.random_state(mi.ne, 4, m.info["np"], seed=5)
    a, da = _steps(torch, dev, m, prec, c, True)
    b, db = _steps(torch, dev, m, prec, c, False)
    assert da == db
    assert np.array_equal(a, b)
    m.close()


def test_pdl_refined_and_naive_colors_bit_identical(torch_dev):
    torch, dev = torch_dev
    mi = W.periodic_square_tri(30, jitter=0.2, seed=72)
    m = dgc.Mesh.from_input(mi, 2)
    m.color(1601)
    m.refine(W.elements_near(mi, (0.5, 0.5), 0.3))
    c = W.random_state(m.info["ne"], 4, m.info["np"], seed=6)
    for prec in (dgc.DGC_FP32_MIXED, dgc.DGC_FP64):
        a, da = _steps(torch, dev, m, prec, c, True)
        b, db = _steps(torch, dev, m, prec, c, False)
        assert da == db and np.array_equal(a, b)
    m.close()
    ev = mi.ev[np.random.default_rng(3).permutation(mi.ne)]
    m = dgc.Mesh(2, 3, mi.xyz, ev, mi.periodic_len)
    dgc.dgc_color_edges_naive(m.h, True, True)
    c = W.random_state(mi.ne, 4, m.info["np"], seed=7)
    a, da = _steps(torch, dev, m, dgc.DGC_FP32_MIXED, c, True)
    b, db = _steps(torch, dev, m, dgc.DGC_FP32_MIXED, c, False)
    assert da == db and np.array_equal(a, b)
    m.close()


@pytest.mark.parametrize("p", [1, 2])
def test_pdl_tetrahedra_bit_identical(torch_dev, p):
    torch, dev = torch_dev
    mi = W.periodic_cube_tet(5)
    m = dgc.Mesh.from_input(mi, p)
    m.color(1601)
    c = W.random_state(mi.ne, 5, m.info["np"], seed=8, mean=(0.5, 0.05, -0.04, 0.03, 1.3))
    for prec in (dgc.DGC_FP32_MIXED, dgc.DGC_FP64):
        for fuse in (True, False):
            dgc.dgc_set_option(m.h, dgc.DGC_OPT_FUSE, int(fuse))
            a, da = _steps(torch, dev, m, prec, c, True, n=3)
            b, db = _steps(torch, dev, m, prec, c, False, n=3)
            assert da == db and np.array_equal(a, b)
    m.close()


def _rhs(torch, dev, m, prec, c_host, pdl, kind):
    dgc.dgc_set_option(m.h, dgc.DGC_OPT_PDL, int(pdl))
    st = torch.empty(m.state_shape(), dtype=torch.float64, device=dev)
    dgc.dgc_import_state(m.h, c_host, st)
    r = torch.full(m.state_shape(), float("nan"), dtype=torch.float64, device=dev)
    if kind == "colored":
        dgc.dgc_rhs(m.h, prec, st, r)
    elif kind == "atomic":
        dgc.dgc_rhs_atomic(m.h, prec, st, r)
    else:
        info = m.info
        nb = dgc.dgc_two_pass_buffer_bytes(info["ns"], info["np"], info["M"], 8)
        buf = torch.empty(nb // 8, dtype=torch.float64, device=dev)
        dgc.dgc_rhs_two_pass(m.h, prec, st, r, buf)
    torch.cuda.synchronize()
    return dgc.dgc_export_state(m.h, r)


@pytest.mark.parametrize("kind", ["colored", "atomic", "two_pass"])
def test_pdl_rhs_forms_identical(torch_dev, kind):
    """dgc_rhs and the comparators with and without programmatic launch, on a
    conforming and a refined mesh: the same bits (the colored and two-pass forms
    sum in a fixed order; the atomic form's order varies, so it is compared to
    within its rounding)."""
    torch, dev = torch_dev
    mi = W.periodic_square_tri(30, jitter=0.2, seed=73)
    for refine in (False, True):
        m = dgc.Mesh.from_input(mi, 3)
        m.color(1601)
        if refine:
            m.refine(W.elements_near(mi, (0.5, 0.5), 0.3))
        c = W.random_state(m.info["ne"], 4, m.info["np"], seed=9)
        for prec in (dgc.DGC_FP32_MIXED, dgc.DGC_FP64):
            a = _rhs(torch, dev, m, prec, c, True, kind)
            b = _rhs(torch, dev, m, prec, c, False, kind)
            assert np.isfinite(a).all()
            if kind == "atomic":
                assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
            else:
                assert np.array_equal(a, b)
        m.close()
