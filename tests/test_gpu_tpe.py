"""Four threads per edge (two lanes per edge side) in the FP32 colored kernels
of the RK step on triangle meshes, against the oracle and against the default
two threads per edge.

With four threads per edge the two lanes of a side split the edge's quadrature
points, the volume integral's points (first color) and the modes of the
epilogues; their partial sums are combined by shuffles.  Only the FP32
summation order changes, so the step must meet the same tolerances against the
oracle (state change within 1e-5 relative L2, per-element max within 1e-4, dt
within 1e-13) and stay within FP32 rounding of the two-thread step.  Meshes of
p = 1, 2, 3 (odd and even mode counts: the epilogue split and the stage-2 FP64
state pairs differ), periodic (fused colors, the first color doing CFL pass 1)
and open (boundary edges, plain sequence), both FP32 forms.
"""

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


def _step(torch_dev, mi, p, c, prec, tpe, epb=64, steps=1, fuse=True):
    torch, dev = torch_dev
    m = dgc.Mesh.from_input(mi, p)
    m.color(1601)
    dgc.dgc_set_option(m.h, dgc.DGC_OPT_FUSE, int(fuse))
    dgc.dgc_set_option(m.h, dgc.DGC_OPT_EDGES_PER_BLOCK, epb)
    dgc.dgc_set_option(m.h, dgc.DGC_OPT_THREADS_PER_EDGE, tpe)
    if prec == dgc.DGC_FP32_KAHAN:
        st = torch.empty(dgc.dgc_state_bytes(m.h, prec) // 4, dtype=torch.float32, device=dev)
        dgc.dgc_import_state_prec(m.h, prec, c, st)
    else:
        st = torch.empty(m.state_shape(), dtype=torch.float64, device=dev)
        dgc.dgc_import_state(m.h, c, st)
    ws = torch.empty(dgc.dgc_workspace_size(m.h, prec) // 8 + 64, dtype=torch.float64, device=dev)
    d = torch.zeros(1, dtype=torch.float64, device=dev)
    for _ in range(steps):
        dgc.dgc_rk_step(m.h, prec, st, 0.3, d, ws)
    torch.cuda.synchronize()
    out = (dgc.dgc_export_state_prec(m.h, prec, st) if prec == dgc.DGC_FP32_KAHAN
           else dgc.dgc_export_state(m.h, st))
    n = dgc.dgc_last_launch_count(m.h)
    m.close()
    return out, float(d.item()), n


CASES = [
    ("periodic", lambda: W.periodic_square_tri(26, jitter=0.2, seed=61)),
    ("open", lambda: W.open_square_tri(23, jitter=0.2, seed=62)),
]


@pytest.mark.parametrize("prec", [dgc.DGC_FP32_MIXED, dgc.DGC_FP32_KAHAN])
@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("name,make", CASES)
def test_four_threads_per_edge_match_oracle(torch_dev, oracle_mod, name, make, p, prec):
    mi = make()
    om = oracle_mod.OracleMesh.from_input(mi)
    xyz, _, _ = om.eval_points(p)
    c = om.project(p, W.vortex_field(xyz[..., 0], xyz[..., 1], beta=5.0))
    c = c + W.uniform_perturbation(c.shape, 7, 1e-3)
    ref, dt_ref = om.rk_step(p, c, 0.3)
    got4, dt4, _ = _step(torch_dev, mi, p, c, prec, 4)
    got2, dt2, _ = _step(torch_dev, mi, p, c, prec, 2)
    assert abs(dt4 - dt_ref) < 1e-13 * dt_ref and dt4 == dt2
    check(got4 - c, ref - c, 1e-5, f"tpe 4, p = {p}, {name}")
    # the two launch shapes differ only by FP32 summation order
    check(got4 - c, got2 - c, 1e-5, "tpe 4 against tpe 2")


@pytest.mark.parametrize("epb", [16, 32, 64])
def test_four_threads_per_edge_tile_shapes_and_steps(torch_dev, oracle_mod, epb):
    """Ragged last tiles of every color (37 x 37 periodic mesh: 1,369 edges per
    color) at three tile sizes, ten steps, against ten oracle steps."""
    mi = W.periodic_square_tri(37, jitter=0.2, seed=63)
    om = oracle_mod.OracleMesh.from_input(mi)
    p = 3
    xyz, _, _ = om.eval_points(p)
    c = om.project(p, W.vortex_field(xyz[..., 0], xyz[..., 1], beta=5.0))
    ref = c
    for _ in range(10):
        ref, _ = om.rk_step(p, ref, 0.3)
    got, _, n = _step(torch_dev, mi, p, c, dgc.DGC_FP32_MIXED, 4, epb=epb, steps=10)
    assert n == 10
    check(got - c, ref - c, 1e-5, f"tpe 4, {epb} edges per block, 10 steps")


def test_four_threads_per_edge_unfused_and_static(torch_dev, oracle_mod):
    """The plain Algorithm 1 sequence (no fusions) and the allocation-free step
    take the same option."""
    torch, dev = torch_dev
    mi = W.periodic_square_tri(20, jitter=0.2, seed=64)
    om = oracle_mod.OracleMesh.from_input(mi)
    c = W.random_state(mi.ne, 4, 6, seed=5, amp=3e-3)
    ref, _ = om.rk_step(2, c, 0.3)
    got, _, _ = _step(torch_dev, mi, 2, c, dgc.DGC_FP32_MIXED, 4, fuse=False)
    check(got - c, ref - c, 1e-5, "tpe 4 unfused")
    m = dgc.Mesh.from_input(mi, 2)
    m.color(1601)
    dgc.dgc_set_option(m.h, dgc.DGC_OPT_THREADS_PER_EDGE, 4)
    st = torch.empty(m.state_shape(), dtype=torch.float64, device=dev)
    dgc.dgc_import_state(m.h, c, st)
    d = torch.zeros(1, dtype=torch.float64, device=dev)
    dgc.dgc_rk_step_static(m.h, dgc.DGC_FP32_MIXED, st, 0.3, d)
    torch.cuda.synchronize()
    check(dgc.dgc_export_state(m.h, st) - c, ref - c, 1e-5, "tpe 4 static step")
    m.close()


def test_threads_per_edge_option_refusals(torch_dev):
    mi = W.periodic_square_tri(8)
    m = dgc.Mesh.from_input(mi, 1)
    m.color(1)
    for bad in (1, 3, 8):
        with pytest.raises(dgc.DgcError):
            dgc.dgc_set_option(m.h, dgc.DGC_OPT_THREADS_PER_EDGE, bad)
    dgc.dgc_set_option(m.h, dgc.DGC_OPT_EDGES_PER_BLOCK, 128)
    with pytest.raises(dgc.DgcError):  # 4 x 128 threads exceed a block
        dgc.dgc_set_option(m.h, dgc.DGC_OPT_THREADS_PER_EDGE, 4)
    dgc.dgc_set_option(m.h, dgc.DGC_OPT_EDGES_PER_BLOCK, 64)
    dgc.dgc_set_option(m.h, dgc.DGC_OPT_THREADS_PER_EDGE, 4)
    with pytest.raises(dgc.DgcError):
        dgc.dgc_set_option(m.h, dgc.DGC_OPT_EDGES_PER_BLOCK, 128)
    m.close()
    q = dgc.Mesh.from_input(W.periodic_square_quad(6, jitter=0.2, slant=0.3, seed=1), 1)
    with pytest.raises(dgc.DgcError):
        dgc.dgc_set_option(q.h, dgc.DGC_OPT_THREADS_PER_EDGE, 4)
    q.close()


def test_per_class_tiles_match_oracle(torch_dev, oracle_mod):
    """Different tiles per kernel class (first and middle colors two threads
    per edge, last color four): the step still meets the oracle."""
    torch, dev = torch_dev
    mi = W.periodic_square_tri(31, jitter=0.2, seed=65)
    om = oracle_mod.OracleMesh.from_input(mi)
    p = 3
    xyz, _, _ = om.eval_points(p)
    c = om.project(p, W.vortex_field(xyz[..., 0], xyz[..., 1], beta=5.0))
    ref, dt_ref = om.rk_step(p, c, 0.3)
    m = dgc.Mesh.from_input(mi, p)
    m.color(1601)
    dgc.dgc_set_tile(m.h, dgc.DGC_K_FIRST, 64, 2)
    dgc.dgc_set_tile(m.h, dgc.DGC_K_COLOR, 128, 2)
    dgc.dgc_set_tile(m.h, dgc.DGC_K_LAST, 32, 4)
    assert dgc.dgc_get_tile(m.h, dgc.DGC_K_LAST) == (32, 4)
    assert dgc.dgc_get_tile(m.h, dgc.DGC_K_COLOR) == (128, 2)
    with pytest.raises(dgc.DgcError):
        dgc.dgc_set_tile(m.h, dgc.DGC_K_COLOR, 128, 4)
    with pytest.raises(dgc.DgcError):
        dgc.dgc_set_tile(m.h, 0, 64, 2)  # not a tile class
    st = torch.empty(m.state_shape(), dtype=torch.float64, device=dev)
    dgc.dgc_import_state(m.h, c, st)
    ws = torch.empty(dgc.dgc_workspace_size(m.h, dgc.DGC_FP32_MIXED) // 8 + 64, dtype=torch.float64, device=dev)
    d = torch.zeros(1, dtype=torch.float64, device=dev)
    dgc.dgc_rk_step(m.h, dgc.DGC_FP32_MIXED, st, 0.3, d, ws)
    torch.cuda.synchronize()
    assert abs(d.item() - dt_ref) < 1e-13 * dt_ref
    check(dgc.dgc_export_state(m.h, st) - c, ref - c, 1e-5, "per-class tiles")
    m.close()


def test_autotune_single_mesh(torch_dev, oracle_mod):
    """dgc_autotune picks a tile per class from the candidate set (it steps a
    scratch state); the tuned step matches the oracle."""
    torch, dev = torch_dev
    mi = W.periodic_square_tri(40, jitter=0.2, seed=66)
    om = oracle_mod.OracleMesh.from_input(mi)
    p = 2
    c = W.random_state(mi.ne, 4, 6, seed=9, amp=3e-3)
    ref, _ = om.rk_step(p, c, 0.3)
    m = dgc.Mesh.from_input(mi, p)
    m.color(1601)
    scratch = torch.empty(m.state_shape(), dtype=torch.float64, device=dev)
    dgc.dgc_import_state(m.h, c, scratch)
    ws = torch.empty(dgc.dgc_workspace_size(m.h, dgc.DGC_FP32_MIXED) // 8 + 64, dtype=torch.float64, device=dev)
    d = torch.zeros(1, dtype=torch.float64, device=dev)
    tiles, ms = dgc.dgc_autotune(m.h, dgc.DGC_FP32_MIXED, scratch, 0.3, d, ws, reps=2)
    assert ms > 0
    for cls, kc in (("first", dgc.DGC_K_FIRST), ("color", dgc.DGC_K_COLOR), ("last", dgc.DGC_K_LAST)):
        e, t = tiles[cls]
        assert e in (32, 64, 128) and t in (2, 4) and e * t <= 256
        assert dgc.dgc_get_tile(m.h, kc) == (e, t)
    st = torch.empty_like(scratch)
    dgc.dgc_import_state(m.h, c, st)
    dgc.dgc_rk_step(m.h, dgc.DGC_FP32_MIXED, st, 0.3, d, ws)
    torch.cuda.synchronize()
    check(dgc.dgc_export_state(m.h, st) - c, ref - c, 1e-5, f"autotuned tiles {tiles}")
    m.close()
