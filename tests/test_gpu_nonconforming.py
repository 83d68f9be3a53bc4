"""GPU parity on nonconforming meshes (Sec. 3.2): the 6-color colored surface
kernels with hanging edges, where the coarse element evaluates its basis on
one half of its edge, against the oracle.

Tolerances as for conforming meshes: FP64 right-hand side 1e-12 relative L2,
FP32-mixed 1e-5; one RK step's state change 1e-11 (FP64) and 1e-5 (mixed).
On vortex states the refined meshes' fine elements raise the agreement floor of
two exact FP64 evaluations (measured as the oracle against itself on the mesh
translated by half a period: 2e-12 on the 30 x 30 mesh at p = 2); there the
FP64 bound is max(1e-12, twice that floor), computed in the test.
The full-size nonconforming workload (256 x 256 x 2 periodic triangles refined
within radius 0.2 of the centre, 180,512 elements, p = 2) is checked on sampled
elements that include coarse elements with hanging edges, and run for its 200
FP64 steps with a conservation check.
"""

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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


class Refined:
    """A refined mesh on the device and its oracle twin."""

    def __init__(self, torch_dev, oracle_mod, mi, p, elems, seed=1601, epb=None):
        self.torch, self.dev = torch_dev
        self.p = p
        self.m = dgc.Mesh.from_input(mi, p)
        self.m.color(seed)
        om = oracle_mod.OracleMesh.from_input(mi)
        col, _ = om.color(3, seed)
        self.m.refine(elems)
        self.om = om.refine(col, elems)
        assert self.m.info["ne"] == self.om.ne and self.m.info["ncolors"] == 6
        if epb:
            dgc.dgc_set_option(self.m.h, dgc.DGC_OPT_EDGES_PER_BLOCK, epb)
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


def _case(kind):
    if kind == "periodic":
        mi = W.periodic_square_tri(30, jitter=0.2, seed=41)
    else:
        mi = W.open_square_tri(26, jitter=0.2, seed=42)
    return mi, W.elements_near(mi, (0.45, 0.55), 0.3)


def _floor(oracle_mod, mi, elems, p, c, sample=None, seed=1601):
    """Agreement floor of two exact FP64 evaluations: the oracle against itself
    on the same refined mesh translated by half a period (an exact symmetry;
    only the rounding of the coordinates changes)."""
    om = oracle_mod.OracleMesh.from_input(mi)
    col, _ = om.color(3, seed)
    a = om.refine(col, elems)
    t = oracle_mod.OracleMesh(2, (mi.xyz + 0.5) % 1.0, mi.ev, mi.periodic_len)
    col2, _ = t.color(3, seed)
    b = t.refine(col2, elems)
    return rel(b.rhs(p, c, elems=sample), a.rhs(p, c, elems=sample))


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("kind", ["periodic", "open"])
def test_refined_rhs_matches_oracle(torch_dev, oracle_mod, p, kind):
    mi, elems = _case(kind)
    run = Refined(torch_dev, oracle_mod, mi, p, elems)
    assert (dgc.dgc_get_hanging(run.m.h) >= 0).sum() > 20
    c = W.random_state(run.om.ne, 4, run.m.info["np"], seed=p)
    run.load(c)
    ref = run.om.rhs(p, c)
    e64 = rel(run.rhs(dgc.DGC_FP64), ref)
    e32 = rel(run.rhs(dgc.DGC_FP32_MIXED), ref)
    assert e64 < 1e-12, e64
    assert e32 < 1e-5, e32
    run.close()


@pytest.mark.parametrize("p", [2, 3])
def test_refined_rhs_vortex_matches_oracle(torch_dev, oracle_mod, p):
    mi, elems = _case("periodic")
    run = Refined(torch_dev, oracle_mod, mi, p, elems)
    c = run.vortex()
    run.load(c)
    ref = run.om.rhs(p, c)
    floor = _floor(oracle_mod, mi, elems, p, c)
    e64 = rel(run.rhs(dgc.DGC_FP64), ref)
    e32 = rel(run.rhs(dgc.DGC_FP32_MIXED), ref)
    print(f"refined vortex p={p}: FP64 {e64:.2e} (oracle floor {floor:.2e}), FP32-mixed {e32:.2e}")
    assert e64 < max(1e-12, 2.0 * floor), (e64, floor)
    assert e32 < 1e-5, e32
    run.close()


@pytest.mark.parametrize("kind", ["atomic", "two_pass"])
def test_refined_comparators_match_oracle(torch_dev, oracle_mod, kind):
    mi, elems = _case("periodic")
    run = Refined(torch_dev, oracle_mod, mi, 2, elems)
    c = W.random_state(run.om.ne, 4, 6, seed=7)
    run.load(c)
    ref = run.om.rhs(2, c)
    assert rel(run.rhs(dgc.DGC_FP64, kind), ref) < 1e-12
    assert rel(run.rhs(dgc.DGC_FP32_MIXED, kind), ref) < 1e-5
    run.close()


@pytest.mark.parametrize("epb", [16, 128])
def test_refined_tile_shapes(torch_dev, oracle_mod, epb):
    mi, elems = _case("periodic")
    run = Refined(torch_dev, oracle_mod, mi, 3, elems, epb=epb)
    c = W.random_state(run.om.ne, 4, 10, seed=8)
    run.load(c)
    assert rel(run.rhs(dgc.DGC_FP64), run.om.rhs(3, c)) < 1e-12
    run.close()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_refined_rk_step_matches_oracle(torch_dev, oracle_mod, p):
    mi, elems = _case("periodic")
    for prec, tol in ((dgc.DGC_FP64, 1e-11), (dgc.DGC_FP32_MIXED, 1e-5)):
        run = Refined(torch_dev, oracle_mod, mi, p, elems)
        c = run.vortex()
        ref, dt_ref = run.om.rk_step(p, c, 0.3)
        run.load(c)
        got, dt = run.rk(prec, 0.3)
        assert abs(dt - dt_ref) < 1e-13 * dt_ref
        assert rel(got - c, ref - c) < tol
        run.close()


def test_refined_freestream_and_refine_nothing(torch_dev, oracle_mod):
    mi = W.periodic_square_tri(12, jitter=0.2, seed=43)
    run = Refined(torch_dev, oracle_mod, mi, 2, np.array([], np.int32))
    assert run.m.info["ne"] == mi.ne
    c = np.zeros(run.m.state_shape())
    c[:, :, 0] = np.array([1.1, 0.3, -0.2, 2.6]) / np.sqrt(2.0)
    run.load(c)
    r = run.rhs(dgc.DGC_FP64)
    assert np.abs(r).max() < 1e-10
    run.close()


# ------------------------------------------------------------------------------------------
# Full size: 180,512 elements (16,480 refined parents), p = 2
# ------------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cfg4(torch_dev, oracle_mod):
    cfg = W.refined_square_vortex_p2_256()
    run = Refined(torch_dev, oracle_mod, cfg["mesh"], cfg["p"], cfg["refine"])
    assert run.m.info["ne"] == 180_512
    xyz, _, _ = run.om.eval_points(cfg["p"])
    c = run.om.project(cfg["p"], W.vortex_field(xyz[..., 0], xyz[..., 1], beta=cfg["beta"]))
    yield run, cfg, c
    run.close()


def test_full_size_refined_rhs_sampled(cfg4, oracle_mod):
    run, cfg, c = cfg4
    p = cfg["p"]
    L, R, _, _ = run.om.sides()
    hang = np.nonzero(run.om.hanging >= 0)[0]
    rng = np.random.default_rng(0)
    coarse = np.unique(R[hang])
    sample = np.unique(np.concatenate([rng.choice(run.om.ne, 1500, replace=False),
                                       rng.choice(coarse, 300, replace=False),
                                       rng.choice(L[hang], 300, replace=False)]))
    run.load(c)
    ref = run.om.rhs(p, c, elems=sample)
    floor = _floor(oracle_mod, cfg["mesh"], cfg["refine"], p, c, sample)
    e64 = rel(run.rhs(dgc.DGC_FP64)[sample], ref)
    e32 = rel(run.rhs(dgc.DGC_FP32_MIXED)[sample], ref)
    print(f"nonconforming full size: FP64 rel L2 {e64:.3e} (oracle floor {floor:.3e}), FP32-mixed {e32:.3e}")
    assert e64 < max(1e-12, 2.0 * floor)
    assert e32 < 1e-5


def test_full_size_refined_run_conserves(cfg4):
    """The configuration's 200 FP64 SSP-RK3 steps: the means' totals stay put
    (periodic mesh; hanging-edge fluxes cancel between the halves and the coarse
    edge), and the state stays finite and positive."""
    run, cfg, c = cfg4
    run.load(c)
    detj = run.om.detj()
    got, dt = run.rk(dgc.DGC_FP64, cfg["cfl"], steps=cfg["steps"])
    assert np.isfinite(got).all() and dt > 0
    t0 = (detj[:, None] * c[:, :, 0]).sum(0)
    t1 = (detj[:, None] * got[:, :, 0]).sum(0)
    np.testing.assert_allclose(t1, t0, rtol=1e-12, atol=1e-13 * np.abs(t0).max())
    assert (got[:, 0, 0] > 0).all()
