"""GPU parity on hybrid triangle/parallelogram meshes (Sec. 3.1, Table 2's hybrid
mesh, 4 colors; Eq. 2 with each element in its own space, P_p or Q_p; states
with (p+1)^2 coefficients per variable, a triangle using the first
(p+1)(p+2)/2).  FP64, the plain Algorithm 1 sequence (volume integral, then
each color), against the oracle: right-hand side within 1e-12 relative L2, one
RK step's state change within 1e-11 (per-element max as in tests/_parity.py),
dt within 1e-13; the atomic comparator too; the FP32-mixed form (FP32 fluxes
and projections in perturbation form, FP64 state) within 1e-5; freestream; a
200 x 200 mesh sampled against the extended oracle."""

import numpy as np
import pytest

from paper_1601_07613_gb300 import dgc
from paper_1601_07613_gb300 import workloads as W
from _parity import check, fp64_vs_exact

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    dgc.lib()
    return torch, torch.device("cuda:0")


def _mesh(kind, n=12, frac=0.4, seed=5):
    periodic = kind == "periodic"
    return W.hybrid_square(n, frac, periodic=periodic, jitter=0.2, slant=0.3 if periodic else 0.0, seed=seed,
                           mode="parallelogram")


def _state(mi, p, seed, amp=3e-3):
    c = W.random_state(mi.ne, 4, (p + 1) ** 2, seed=seed, amp=amp)
    tri = mi.ev[:, 3] < 0
    c[tri, :, (p + 1) * (p + 2) // 2:] = 0.0  # a triangle's unused coefficients
    return c


class H:
    def __init__(self, torch_dev, mi, p, seed=1601):
        self.torch, self.dev = torch_dev
        self.m = dgc.Mesh.from_input(mi, p)
        assert self.m.elem == dgc.DGC_QUAD and self.m.nonaffine == 0
        nc, _ = self.m.color(seed)
        assert nc == 4
        T = self.torch
        self.c = T.empty(self.m.state_shape(), dtype=T.float64, device=self.dev)
        self.r = T.empty_like(self.c)

    def rhs(self, c, kind="colored", prec=dgc.DGC_FP64):
        dgc.dgc_import_state(self.m.h, c, self.c)
        self.r.fill_(float("nan"))
        if kind == "colored":
            dgc.dgc_rhs(self.m.h, prec, self.c, self.r)
        else:
            dgc.dgc_rhs_atomic(self.m.h, prec, self.c, self.r)
        self.torch.cuda.synchronize()
        return dgc.dgc_export_state(self.m.h, self.r)

    def rk(self, c, cfl, steps=1, prec=dgc.DGC_FP64):
        T = self.torch
        dgc.dgc_import_state(self.m.h, c, self.c)
        ws = T.empty(dgc.dgc_workspace_size(self.m.h, prec) // 8 + 64, dtype=T.float64, device=self.dev)
        d = T.zeros(1, dtype=T.float64, device=self.dev)
        for _ in range(steps):
            dgc.dgc_rk_step(self.m.h, prec, self.c, cfl, d, ws)
        T.cuda.synchronize()
        return dgc.dgc_export_state(self.m.h, self.c), float(d.item())

    def close(self):
        self.m.close()


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("kind", ["periodic", "open"])
def test_hybrid_rhs_matches_oracle(torch_dev, oracle_mod, kind, p):
    mi = _mesh(kind)
    run = H(torch_dev, mi, p)
    c = _state(mi, p, seed=p)
    ref = oracle_mod.OracleMesh.from_input(mi).rhs(p, c)
    got = run.rhs(c)
    check(got, ref, 1e-12, f"hybrid {kind} p = {p}")
    tri = mi.ev[:, 3] < 0
    assert np.all(got[tri][:, :, (p + 1) * (p + 2) // 2:] == 0.0)
    check(run.rhs(c, "atomic"), ref, 1e-12, f"hybrid atomic {kind} p = {p}")
    got = run.rhs(c, prec=dgc.DGC_FP32_MIXED)
    check(got, ref, 1e-5, f"hybrid FP32-mixed {kind} p = {p}")
    assert np.all(got[tri][:, :, (p + 1) * (p + 2) // 2:] == 0.0)
    check(run.rhs(c, "atomic", dgc.DGC_FP32_MIXED), ref, 1e-5, f"hybrid FP32-mixed atomic {kind} p = {p}")
    run.close()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_hybrid_rk_step_matches_oracle(torch_dev, oracle_mod, p):
    mi = _mesh("periodic", n=14, seed=6)
    om = oracle_mod.OracleMesh.from_input(mi)
    xyz, _, _ = om.eval_points(p)
    c = om.project(p, W.vortex_field(xyz[..., 0], xyz[..., 1], beta=5.0))
    ref, dt_ref = om.rk_step(p, c, 0.3)
    run = H(torch_dev, mi, p)
    got, dt = run.rk(c, 0.3)
    assert abs(dt - dt_ref) < 1e-13 * dt_ref
    check(got - c, ref - c, 1e-11, f"hybrid RK step p = {p}")
    got, dt = run.rk(c, 0.3, prec=dgc.DGC_FP32_MIXED)
    assert abs(dt - dt_ref) < 1e-13 * dt_ref
    check(got - c, ref - c, 1e-5, f"hybrid FP32-mixed RK step p = {p}")
    run.close()


def test_hybrid_freestream_and_refusals(torch_dev, oracle_mod):
    torch, dev = torch_dev
    mi = _mesh("periodic", n=10)
    run = H(torch_dev, mi, 2)
    c = np.zeros(run.m.state_shape())
    ub = np.array([1.1, 0.3, -0.2, 2.6])
    tri = mi.ev[:, 3] < 0
    c[:, :, 0] = ub
    c[tri, :, 0] = ub / np.sqrt(2.0)
    r = run.rhs(c)
    h = 0.1
    assert np.abs(r).max() * (0.5 * h * h) / (3.4 * h * 3.0) < 1e-13
    r32 = run.rhs(c, prec=dgc.DGC_FP32_MIXED)  # the perturbation form: the flux of the mean cancels exactly
    assert np.abs(r32).max() * (0.5 * h * h) / (3.4 * h * 3.0) < 1e-6
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_rhs(run.m.h, dgc.DGC_FP32_KAHAN, run.c, run.r)
    assert e.value.status == 4
    buf = torch.empty(1 << 20, dtype=torch.float64, device=dev)
    with pytest.raises(dgc.DgcError):
        dgc.dgc_rhs_two_pass(run.m.h, dgc.DGC_FP64, run.c, run.r, buf)
    run.close()


def test_hybrid_larger_mesh_sampled(torch_dev, oracle_mod):
    """200 x 200 cells, 30 % split (about 52,000 elements), p = 3, vortex state:
    FP64 against the extended oracle on 2,000 sampled elements."""
    mi = W.hybrid_square(200, 0.3, periodic=True, jitter=0.2, slant=0.3, seed=8, mode="parallelogram")
    p = 3
    om = oracle_mod.OracleMesh.from_input(mi)
    xyz, _, _ = om.eval_points(p)
    c = om.project(p, W.vortex_field(xyz[..., 0], xyz[..., 1], beta=5.0))
    c = c + W.uniform_perturbation(c.shape, 9, 1e-3)
    tri = mi.ev[:, 3] < 0
    c[tri, :, (p + 1) * (p + 2) // 2:] = 0.0
    sample = np.sort(np.random.default_rng(0).choice(om.ne, 2000, replace=False))
    ref = om.rhs(p, c, elems=sample)
    refx = oracle_mod.OracleMesh.from_input(mi, build="extended").rhs(p, c, elems=sample)
    run = H(torch_dev, mi, p)
    got = run.rhs(c)[sample]
    e, eo = fp64_vs_exact(got, ref, refx, 1e-12, "hybrid 200 x 200")
    print(f"hybrid 200 x 200: FP64 vs exact {e:.2e} (FP64 oracle {eo:.2e}), {om.ne} elements")
    run.close()
