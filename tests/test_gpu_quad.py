"""GPU parity on parallelogram quadrilateral meshes (Sec. 3.1, Table 2: 4
colors; Eq. 2 with the tensor Legendre space Q_p) against the oracle.

Tolerances as for triangles: FP64 right-hand side 1e-12 relative L2, FP32-mixed
1e-5; one RK step's state change 1e-11 (FP64) and 1e-5 (mixed); dt 1e-13 (FP64)
and 1e-12 (mixed, whose CFL pass reads the same FP64 state).  Meshes: slanted
periodic parallelograms (4 colors, every element has each color once) and
jittered rectangles on the open square (boundary edges, transmissive state).
Sizes from 6 x 6 (18 edges per color, one partial block) to 16 x 16; the full
quadrilateral workload (810 x 810 periodic parallelograms, p = 3) is checked on
sampled elements and by conservation.  At h = 1/810 the terms of Eq. 2 (of size
|F|/h) cancel to a much smaller right-hand side: there the GPU's FP64 result is
compared with the oracle's extended-precision build and must be within 1e-12 of
it, or within the FP64 oracle's own error against it where that is larger.
Every comparison also bounds the largest per-element error (tests/_parity.py).
"""

import numpy as np
import pytest

from paper_1601_07613_gb300 import dgc
from paper_1601_07613_gb300 import workloads as W
from _parity import check, fp64_vs_exact, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    dgc.lib()
    return torch, torch.device("cuda:0")


class Q:
    """A quadrilateral mesh on the device and its oracle twin."""

    def __init__(self, torch_dev, oracle_mod, mi, p, seed=1601, fuse=True, epb=None):
        self.torch, self.dev = torch_dev
        self.p = p
        self.m = dgc.Mesh.from_input(mi, p)
        assert self.m.elem == dgc.DGC_QUAD and self.m.nonaffine == 0
        self.m.color(seed)
        dgc.dgc_set_option(self.m.h, dgc.DGC_OPT_FUSE, int(fuse))
        if epb:
            dgc.dgc_set_option(self.m.h, dgc.DGC_OPT_EDGES_PER_BLOCK, epb)
        self.om = oracle_mod.OracleMesh.from_input(mi)
        T = self.torch
        shape = self.m.state_shape()
        self.c = T.empty(shape, dtype=T.float64, device=self.dev)
        self.r = T.empty(shape, dtype=T.float64, device=self.dev)

    def vortex(self, beta=5.0, perturb=1e-3, seed=3):
        xyz, _, _ = self.om.eval_points(self.p)
        c = self.om.project(self.p, W.vortex_field(xyz[..., 0], xyz[..., 1], beta=beta))
        return c + W.uniform_perturbation(c.shape, seed, perturb)

    def load(self, c):
        dgc.dgc_import_state(self.m.h, c, self.c)

    def rhs(self, prec, kind="colored"):
        T = self.torch
        self.r.fill_(float("nan"))
        if kind == "colored":
            dgc.dgc_rhs(self.m.h, prec, self.c, self.r)
        elif kind == "atomic":
            dgc.dgc_rhs_atomic(self.m.h, prec, self.c, self.r)
        else:
            info = self.m.info
            nb = dgc.dgc_two_pass_buffer_bytes(info["ns"], info["np"], info["M"], 8)
            buf = T.empty(nb // 8, dtype=T.float64, device=self.dev)
            dgc.dgc_rhs_two_pass(self.m.h, prec, self.c, self.r, buf)
        T.cuda.synchronize()
        return dgc.dgc_export_state(self.m.h, self.r)

    def rk(self, prec, cfl, steps=1):
        T = self.torch
        ws = T.empty(dgc.dgc_workspace_size(self.m.h, prec) // 8 + 64, dtype=T.float64, device=self.dev)
        d = T.zeros(1, dtype=T.float64, device=self.dev)
        for _ in range(steps):
            dgc.dgc_rk_step(self.m.h, prec, self.c, cfl, d, ws)
        T.cuda.synchronize()
        return dgc.dgc_export_state(self.m.h, self.c), float(d.item())

    def close(self):
        self.m.close()


def _mesh(kind, n=12):
    if kind == "periodic":
        return W.periodic_square_quad(n, jitter=0.2, slant=0.3, seed=41)
    return W.open_square_quad(n - 1, jitter=0.2, seed=42)


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("kind", ["periodic", "open"])
def test_quad_rhs_matches_oracle(torch_dev, oracle_mod, p, kind):
    run = Q(torch_dev, oracle_mod, _mesh(kind), p)
    c = W.random_state(run.om.ne, 4, (p + 1) ** 2, seed=p)
    run.load(c)
    ref = run.om.rhs(p, c)
    check(run.rhs(dgc.DGC_FP64), ref, 1e-12, "FP64")
    check(run.rhs(dgc.DGC_FP32_MIXED), ref, 1e-5, "FP32-mixed")
    run.close()


@pytest.mark.parametrize("p", [2, 3])
def test_quad_rhs_vortex_matches_oracle(torch_dev, oracle_mod, p):
    run = Q(torch_dev, oracle_mod, _mesh("periodic", 16), p)
    c = run.vortex()
    run.load(c)
    ref = run.om.rhs(p, c)
    e64, _ = check(run.rhs(dgc.DGC_FP64), ref, 1e-12, "FP64")
    e32, _ = check(run.rhs(dgc.DGC_FP32_MIXED), ref, 1e-5, "FP32-mixed")
    print(f"quad vortex p={p}: FP64 {e64:.2e}, FP32-mixed {e32:.2e}")
    run.close()


@pytest.mark.parametrize("kind", ["atomic", "two_pass"])
@pytest.mark.parametrize("p", [1, 3])
def test_quad_comparators_match_oracle(torch_dev, oracle_mod, kind, p):
    run = Q(torch_dev, oracle_mod, _mesh("periodic"), p)
    c = W.random_state(run.om.ne, 4, (p + 1) ** 2, seed=7)
    run.load(c)
    ref = run.om.rhs(p, c)
    check(run.rhs(dgc.DGC_FP64, kind), ref, 1e-12)
    check(run.rhs(dgc.DGC_FP32_MIXED, kind), ref, 1e-5)
    run.close()


@pytest.mark.parametrize("epb", [16, 128])
@pytest.mark.parametrize("n", [6, 10])
def test_quad_tile_shapes_and_ragged_colors(torch_dev, oracle_mod, epb, n):
    """18 and 50 edges per color: a single partial block, and a ragged last one."""
    run = Q(torch_dev, oracle_mod, _mesh("periodic", n), 3, epb=epb)
    c = W.random_state(run.om.ne, 4, 16, seed=8)
    run.load(c)
    ref = run.om.rhs(3, c)
    check(run.rhs(dgc.DGC_FP64), ref, 1e-12)
    check(run.rhs(dgc.DGC_FP32_MIXED), ref, 1e-5)
    run.close()


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("fuse", [True, False])
def test_quad_rk_step_matches_oracle(torch_dev, oracle_mod, p, fuse):
    mi = _mesh("periodic")
    for prec, tol, dtol in ((dgc.DGC_FP64, 1e-11, 1e-13), (dgc.DGC_FP32_MIXED, 1e-5, 1e-12)):
        run = Q(torch_dev, oracle_mod, mi, p, fuse=fuse)
        c = run.vortex()
        ref, dt_ref = run.om.rk_step(p, c, 0.3)
        run.load(c)
        got, dt = run.rk(prec, 0.3)
        assert abs(dt - dt_ref) < dtol * dt_ref
        check(got - c, ref - c, tol)
        run.close()


def test_quad_freestream(torch_dev, oracle_mod):
    run = Q(torch_dev, oracle_mod, _mesh("periodic"), 3)
    c = np.zeros(run.m.state_shape())
    c[:, :, 0] = [1.1, 0.3, -0.2, 2.6]
    run.load(c)
    h = 1.0 / 12
    for prec in (dgc.DGC_FP64, dgc.DGC_FP32_MIXED):
        r = run.rhs(prec)
        assert np.abs(r).max() * h * h / (4 * h * 3.0) < (1e-13 if prec == dgc.DGC_FP64 else 1e-6)
    run.close()


def test_quad_pdl_on_off_identical(torch_dev, oracle_mod):
    mi = _mesh("periodic")
    out = []
    for pdl in (1, 0):
        run = Q(torch_dev, oracle_mod, mi, 3)
        dgc.dgc_set_option(run.m.h, dgc.DGC_OPT_PDL, pdl)
        run.load(run.vortex())
        out.append(run.rk(dgc.DGC_FP32_MIXED, 0.3, steps=2)[0])
        run.close()
    assert np.array_equal(out[0], out[1])


# ------------------------------------------------------------------------------------------
# Full size: 810 x 810 periodic parallelograms (656,100 elements, 1,312,200 edges), p = 3
# ------------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def full(torch_dev, oracle_mod):
    cfg = W.quad_square_vortex_p3_810()
    run = Q(torch_dev, oracle_mod, cfg["mesh"], cfg["p"])
    assert run.m.info["ne"] == 656_100
    xyz, _, _ = run.om.eval_points(cfg["p"])
    c = run.om.project(cfg["p"], W.vortex_field(xyz[..., 0], xyz[..., 1], beta=cfg["beta"]))
    c = c + W.uniform_perturbation(c.shape, cfg["seed"], cfg["perturb"])
    yield run, cfg, c
    run.close()


def test_full_size_quad_rhs_sampled(full, oracle_mod):
    run, cfg, c = full
    sample = np.sort(np.random.default_rng(0).choice(run.om.ne, 3000, replace=False))
    run.load(c)
    ref = run.om.rhs(cfg["p"], c, elems=sample)
    refx = oracle_mod.OracleMesh.from_input(cfg["mesh"], build="extended").rhs(cfg["p"], c, elems=sample)
    e64, eo = fp64_vs_exact(run.rhs(dgc.DGC_FP64)[sample], ref, refx, 1e-12, "quad full size")
    e32, _ = check(run.rhs(dgc.DGC_FP32_MIXED)[sample], ref, 1e-5, "quad full size FP32-mixed")
    print(f"quad full size: FP64 vs exact {e64:.3e} (FP64 oracle {eo:.3e}), FP32-mixed {e32:.3e}")


def test_full_size_quad_steps_conserve(full):
    run, cfg, c = full
    detj = run.om.detj()
    for prec, rtol in ((dgc.DGC_FP64, 1e-12), (dgc.DGC_FP32_MIXED, 1e-8)):
        run.load(c)
        got, dt = run.rk(prec, cfg["cfl"], steps=5)
        assert np.isfinite(got).all() and dt > 0
        t0 = (detj[:, None] * c[:, :, 0]).sum(0)
        t1 = (detj[:, None] * got[:, :, 0]).sum(0)
        np.testing.assert_allclose(t1, t0, rtol=rtol, atol=1e-13 * np.abs(t0).max())


def test_quad_static_step_equals_regular(torch_dev, oracle_mod):
    """The allocation-free step (its workspace in the library's static device
    array) runs the same launches: bit-identical states."""
    torch, dev = torch_dev
    mi = _mesh("periodic", 8)
    out = []
    for static in (False, True):
        run = Q(torch_dev, oracle_mod, mi, 2)
        run.load(run.vortex())
        d = torch.zeros(1, dtype=torch.float64, device=dev)
        if static:
            for _ in range(2):
                dgc.dgc_rk_step_static(run.m.h, dgc.DGC_FP32_MIXED, run.c, 0.3, d)
            torch.cuda.synchronize()
            out.append(dgc.dgc_export_state(run.m.h, run.c))
        else:
            out.append(run.rk(dgc.DGC_FP32_MIXED, 0.3, steps=2)[0])
        run.close()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("p", [1, 3])
def test_quad_cfl_dt_matches_oracle(torch_dev, oracle_mod, p):
    torch, dev = torch_dev
    run = Q(torch_dev, oracle_mod, _mesh("open"), p)
    c = run.vortex()
    run.load(c)
    d = torch.zeros(1, dtype=torch.float64, device=dev)
    dgc.dgc_cfl_dt(run.m.h, run.c, 0.3, d)
    torch.cuda.synchronize()
    ref = run.om.dt(p, c, 0.3)
    assert abs(float(d.item()) - ref) < 1e-13 * ref
    run.close()
