"""GPU parity on nonconforming meshes (Sec. 3.2): the 6-color colored surface
kernels with hanging edges, where the coarse element evaluates its basis on
one half of its edge, against the oracle.

Tolerances as for conforming meshes: FP64 right-hand side 1e-12 relative L2,
FP32-mixed 1e-5; one RK step's state change 1e-11 (FP64) and 1e-5 (mixed).
On vortex states the refined meshes' fine elements make Eq. 2's terms cancel
to a much smaller sum, and no FP64 evaluation reaches 1e-12 of the exact
result: there the GPU's FP64 right-hand side is compared with the oracle's
extended-precision build and must be within 1e-12 of it, or within the FP64
oracle's own error against it where that is larger.  Every comparison also
bounds the largest per-element error (tests/_parity.py).
The full-size nonconforming workload (256 x 256 x 2 periodic triangles refined
within radius 0.2 of the centre, 180,512 elements, p = 2) is checked on sampled
elements that include coarse elements with hanging edges, and run for its 200
FP64 steps with a conservation check.
"""

import numpy as np
import pytest

from paper_1601_07613_gb300 import dgc
from paper_1601_07613_gb300 import workloads as W
from _amr import second_level
from _parity import check, fp64_vs_exact, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    dgc.lib()
    return torch, torch.device("cuda:0")


class Refined:
    """A refined mesh on the device and its oracle twin."""

    def __init__(self, torch_dev, oracle_mod, mi, p, elems, seed=1601, epb=None, second=None):
        self.torch, self.dev = torch_dev
        self.p = p
        self.m = dgc.Mesh.from_input(mi, p)
        self.m.color(seed)
        om = oracle_mod.OracleMesh.from_input(mi)
        col, _ = om.color(3, seed)
        self.m.refine(elems)
        self.om = om.refine(col, elems)
        if second is not None:
            # a second level: the elements second(oracle mesh) picks, refined again
            e2 = second(self.om)
            self.m.refine(e2)
            self.om = self.om.refine(self.om.colors, e2)
        assert self.m.info["ne"] == self.om.ne
        assert self.m.info["ncolors"] == (6 if second is None else 12)
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


def _exact(oracle_mod, mi, elems, seed=1601):
    """The refined mesh in the oracle's extended-precision build (the same
    coloring, refinement and map as the FP64 oracle's)."""
    om = oracle_mod.OracleMesh.from_input(mi, build="extended")
    col, _ = om.color(3, seed)
    return om.refine(col, elems)


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("kind", ["periodic", "open"])
def test_refined_rhs_matches_oracle(torch_dev, oracle_mod, p, kind):
    mi, elems = _case(kind)
    run = Refined(torch_dev, oracle_mod, mi, p, elems)
    assert (dgc.dgc_get_hanging(run.m.h) >= 0).sum() > 20
    c = W.random_state(run.om.ne, 4, run.m.info["np"], seed=p)
    run.load(c)
    ref = run.om.rhs(p, c)
    check(run.rhs(dgc.DGC_FP64), ref, 1e-12, "FP64")
    check(run.rhs(dgc.DGC_FP32_MIXED), ref, 1e-5, "FP32-mixed")
    run.close()


@pytest.mark.parametrize("p", [2, 3])
def test_refined_rhs_vortex_matches_oracle(torch_dev, oracle_mod, p):
    mi, elems = _case("periodic")
    run = Refined(torch_dev, oracle_mod, mi, p, elems)
    c = run.vortex()
    run.load(c)
    ref = run.om.rhs(p, c)
    refx = _exact(oracle_mod, mi, elems).rhs(p, c)
    e64, eo = fp64_vs_exact(run.rhs(dgc.DGC_FP64), ref, refx, 1e-12, "refined vortex")
    e32, _ = check(run.rhs(dgc.DGC_FP32_MIXED), ref, 1e-5, "refined vortex FP32-mixed")
    print(f"refined vortex p={p}: FP64 vs exact {e64:.2e} (FP64 oracle {eo:.2e}), FP32-mixed {e32:.2e}")
    run.close()


@pytest.mark.parametrize("kind", ["atomic", "two_pass"])
def test_refined_comparators_match_oracle(torch_dev, oracle_mod, kind):
    mi, elems = _case("periodic")
    run = Refined(torch_dev, oracle_mod, mi, 2, elems)
    c = W.random_state(run.om.ne, 4, 6, seed=7)
    run.load(c)
    ref = run.om.rhs(2, c)
    check(run.rhs(dgc.DGC_FP64, kind), ref, 1e-12)
    check(run.rhs(dgc.DGC_FP32_MIXED, kind), ref, 1e-5)
    run.close()


@pytest.mark.parametrize("epb", [16, 128])
def test_refined_tile_shapes(torch_dev, oracle_mod, epb):
    mi, elems = _case("periodic")
    run = Refined(torch_dev, oracle_mod, mi, 3, elems, epb=epb)
    c = W.random_state(run.om.ne, 4, 10, seed=8)
    run.load(c)
    check(run.rhs(dgc.DGC_FP64), run.om.rhs(3, c), 1e-12)
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
        check(got - c, ref - c, tol)
        run.close()


def _second(rm):
    return second_level(rm, (0.45, 0.55), 0.18, 0.36)


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("kind", ["periodic", "open"])
def test_two_level_rhs_matches_oracle(torch_dev, oracle_mod, p, kind):
    """A second level (12 colors; level-2 elements beside level-1 ones, and
    level-0 elements beside level-1 ones that were refined from their hanging
    side): the right-hand side in both precisions, and the comparators."""
    mi, elems = _case(kind)
    run = Refined(torch_dev, oracle_mod, mi, p, elems, second=_second)
    lev = run.om.levels
    L, _, _, _ = run.om.sides()
    hang = run.om.hanging >= 0
    assert (lev == 2).sum() > 100 and (hang & (lev[L] == 2)).sum() > 20 and (hang & (lev[L] == 1)).sum() > 20
    c = W.random_state(run.om.ne, 4, run.m.info["np"], seed=p)
    run.load(c)
    ref = run.om.rhs(p, c)
    check(run.rhs(dgc.DGC_FP64), ref, 1e-12, "two levels FP64")
    check(run.rhs(dgc.DGC_FP32_MIXED), ref, 1e-5, "two levels FP32-mixed")
    if p == 2:
        check(run.rhs(dgc.DGC_FP64, "atomic"), ref, 1e-12, "two levels atomic")
        check(run.rhs(dgc.DGC_FP64, "two_pass"), ref, 1e-12, "two levels two-pass")
    run.close()


@pytest.mark.parametrize("p", [2, 3])
def test_two_level_rk_step_matches_oracle(torch_dev, oracle_mod, p):
    mi, elems = _case("periodic")
    for prec, tol in ((dgc.DGC_FP64, 1e-11), (dgc.DGC_FP32_MIXED, 1e-5)):
        run = Refined(torch_dev, oracle_mod, mi, p, elems, second=_second)
        c = run.vortex()
        ref, dt_ref = run.om.rk_step(p, c, 0.3)
        run.load(c)
        got, dt = run.rk(prec, 0.3)
        assert abs(dt - dt_ref) < 1e-13 * dt_ref
        check(got - c, ref - c, tol, f"two levels RK step prec {prec}")
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
    refx = _exact(oracle_mod, cfg["mesh"], cfg["refine"]).rhs(p, c, elems=sample)
    e64, eo = fp64_vs_exact(run.rhs(dgc.DGC_FP64)[sample], ref, refx, 1e-12, "nonconforming full size")
    e32, _ = check(run.rhs(dgc.DGC_FP32_MIXED)[sample], ref, 1e-5, "nonconforming full size FP32-mixed")
    print(f"nonconforming full size: FP64 vs exact {e64:.3e} (FP64 oracle {eo:.3e}), FP32-mixed {e32:.3e}")


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
