"""GPU parity of the FP32 Kahan form (FP32 flux, FP32 pair state updated by
compensated summation) and of the increment form of the step shared with the
mixed form, against the oracle.

Tolerances: right-hand side and one RK step's state change within 1e-5
relative L2 (FP32 flux); dt within 1e-12 (the CFL reduction runs in FP64 on the
pair values, which carry 48 bits); import/export round trip within 2^-46
relative per value.
"""

import numpy as np
import pytest

from paper_1601_07613_gb300 import dgc
from paper_1601_07613_gb300 import workloads as W
from _parity import check, rel

pytestmark = pytest.mark.gpu
KAHAN, MIXED, FP64 = dgc.DGC_FP32_KAHAN, dgc.DGC_FP32_MIXED, dgc.DGC_FP64


@pytest.fixture(scope="module")
def torch_dev():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    dgc.lib()
    return torch, torch.device("cuda:0")


class K:
    def __init__(self, torch_dev, mi, p, seed=1601, fuse=True):
        self.torch, self.dev = torch_dev
        self.m = dgc.Mesh.from_input(mi, p)
        self.m.color(seed)
        dgc.dgc_set_option(self.m.h, dgc.DGC_OPT_FUSE, int(fuse))
        T = self.torch
        self.k = T.empty(dgc.dgc_state_bytes(self.m.h, KAHAN) // 4, dtype=T.float32, device=self.dev)
        self.c = T.empty(self.m.state_shape(), dtype=T.float64, device=self.dev)
        self.r = T.empty(self.m.state_shape(), dtype=T.float64, device=self.dev)

    def load(self, c):
        dgc.dgc_import_state_prec(self.m.h, KAHAN, c, self.k)
        dgc.dgc_import_state(self.m.h, c, self.c)

    def state(self, prec):
        self.torch.cuda.synchronize()
        if prec == KAHAN:
            return dgc.dgc_export_state_prec(self.m.h, KAHAN, self.k)
        return dgc.dgc_export_state(self.m.h, self.c)

    def rhs(self, prec):
        self.r.fill_(float("nan"))
        dgc.dgc_rhs(self.m.h, prec, self.k if prec == KAHAN else self.c, self.r)
        self.torch.cuda.synchronize()
        return dgc.dgc_export_state(self.m.h, self.r)

    def rk(self, prec, cfl, steps=1):
        T = self.torch
        ws = T.empty(dgc.dgc_workspace_size(self.m.h, prec) // 8 + 64, dtype=T.float64, device=self.dev)
        d = T.zeros(1, dtype=T.float64, device=self.dev)
        for _ in range(steps):
            dgc.dgc_rk_step(self.m.h, prec, self.k if prec == KAHAN else self.c, cfl, d, ws)
        return self.state(prec), float(d.item())

    def close(self):
        self.m.close()


def _vortex(oracle_mod, mi, p, beta=5.0):
    om = oracle_mod.OracleMesh.from_input(mi)
    xyz, _, _ = om.eval_points(p)
    c = om.project(p, W.vortex_field(xyz[..., 0], xyz[..., 1], beta=beta))
    return om, c + W.uniform_perturbation(c.shape, 3, 1e-3)


def test_kahan_import_export_round_trip(torch_dev):
    mi = W.periodic_square_tri(17, jitter=0.2, seed=51)
    run = K(torch_dev, mi, 3)
    c = W.random_state(mi.ne, 4, 10, seed=5, amp=5e-2)
    run.load(c)
    back = run.state(KAHAN)
    assert np.all(np.abs(back - c) <= 2.0 ** -46 * np.abs(c) + 1e-300)
    assert run.k.numel() * 4 == dgc.dgc_state_size(run.m.h)  # the pair state of a triangle: FP64's size
    run.close()


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("kind", ["periodic", "open"])
def test_kahan_rhs_matches_oracle(torch_dev, oracle_mod, p, kind):
    mi = (W.periodic_square_tri(27, jitter=0.2, seed=52) if kind == "periodic"
          else W.open_square_tri(23, jitter=0.2, seed=52))
    om, c = _vortex(oracle_mod, mi, p)
    run = K(torch_dev, mi, p)
    run.load(c)
    ref = om.rhs(p, c)
    check(run.rhs(KAHAN), ref, 1e-5)
    run.close()


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("fuse", [True, False])
def test_kahan_and_mixed_rk_step_match_oracle(torch_dev, oracle_mod, p, fuse):
    mi = W.periodic_square_tri(26, jitter=0.2, seed=53)
    om, c = _vortex(oracle_mod, mi, p)
    ref, dt_ref = om.rk_step(p, c, 0.3)
    run = K(torch_dev, mi, p, fuse=fuse)
    for prec in (KAHAN, MIXED):
        run.load(c)
        got, dt = run.rk(prec, 0.3)
        assert abs(dt - dt_ref) < 1e-12 * dt_ref
        check(got - c, ref - c, 1e-5, f"prec {prec}")
    run.close()


def test_kahan_tracks_fp64_over_many_small_steps(torch_dev, oracle_mod):
    """200 steps at CFL 0.02: the per-step change is ~1e-4 of the state, so an
    FP32 state without compensation would lose ~2^-24 / 1e-4 of every update;
    the compensated pair state stays with the FP64 run to the FP32 flux's
    accuracy, as does the FP64-state mixed form."""
    mi = W.periodic_square_tri(20, jitter=0.2, seed=54)
    _, c = _vortex(oracle_mod, mi, 2)
    run = K(torch_dev, mi, 2)
    run.load(c)
    ref, _ = run.rk(FP64, 0.02, steps=200)
    run.load(c)
    gk, _ = run.rk(KAHAN, 0.02, steps=200)
    run.load(c)
    gm, _ = run.rk(MIXED, 0.02, steps=200)
    ek, em = rel(gk - c, ref - c), rel(gm - c, ref - c)
    print(f"200 small steps: du rel L2 Kahan {ek:.2e}, mixed {em:.2e}")
    check(gk - c, ref - c, 1e-5)
    check(gm - c, ref - c, 1e-5)
    # the whole state: both within a few FP32 ulps of the FP64 run (not drifting)
    check(gk, ref, 1e-7)
    check(gm, ref, 1e-7)
    run.close()


def test_kahan_conserves(torch_dev, oracle_mod):
    mi = W.periodic_square_tri(24, jitter=0.2, seed=55)
    om, c = _vortex(oracle_mod, mi, 3)
    run = K(torch_dev, mi, 3)
    run.load(c)
    got, _ = run.rk(KAHAN, 0.3, steps=20)
    detj = om.detj()
    t0 = (detj[:, None] * c[:, :, 0]).sum(0)
    t1 = (detj[:, None] * got[:, :, 0]).sum(0)
    # each step's mean increments cancel to FP32 rounding of the fluxes
    np.testing.assert_allclose(t1, t0, rtol=1e-8)
    run.close()


def test_kahan_static_step_equals_regular(torch_dev):
    mi = W.periodic_square_tri(18, jitter=0.2, seed=56)
    run = K(torch_dev, mi, 2)
    c = W.random_state(mi.ne, 4, 6, seed=9)
    run.load(c)
    a, _ = run.rk(KAHAN, 0.3, steps=2)
    run.load(c)
    d = run.torch.zeros(1, dtype=run.torch.float64, device=run.dev)
    for _ in range(2):
        dgc.dgc_rk_step_static(run.m.h, KAHAN, run.k, 0.3, d)
    b = run.state(KAHAN)
    assert np.array_equal(a, b)
    run.close()


def test_kahan_refuses_tetrahedra(torch_dev):
    m = dgc.Mesh.from_input(W.periodic_cube_tet(3), 1)
    m.color(1)
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_state_bytes(m.h, KAHAN)
    assert e.value.status == 4
    m.close()
