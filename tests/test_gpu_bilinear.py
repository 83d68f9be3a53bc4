"""GPU parity on general (bilinear) quadrilaterals, alone and in hybrid meshes
with triangles (Sec. 3.1, Table 2's quadrilateral and hybrid meshes; Eq. 2 with
detJ J^-1 taken at every volume point and each element's own mass matrix
M = int phi_i phi_j detJ applied after the colors).  FP64, the plain
Algorithm 1 sequence, against the oracle: right-hand side within 1e-12
relative L2 (colored and atomic), one RK step's state change within 1e-11, dt
within 1e-13 (per-element max as in tests/_parity.py); the allocation-free step
bit-identical to the regular one; the FP32-mixed form (FP32 fluxes and
projections in perturbation form, FP64 state) within 1e-5; freestream; a
160 x 160 mesh of jittered quadrilaterals sampled against the extended
oracle."""

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


def _mesh(kind, n=12, seed=5):
    if kind == "quad":
        return W.periodic_square_quad(n, "vertex", 0.2, seed=seed)
    if kind == "quad_open":
        return W.open_square_quad(n, "vertex", 0.2, seed=seed)
    return W.hybrid_square(n, 0.4, periodic=True, jitter=0.2, seed=seed)


def _zero_tri(mi, p, c):
    tri = mi.ev[:, 3] < 0
    c[tri, :, (p + 1) * (p + 2) // 2:] = 0.0  # a triangle's unused coefficients
    return c


class B:
    def __init__(self, torch_dev, mi, p, seed=1601):
        self.torch, self.dev = torch_dev
        self.m = dgc.Mesh.from_input(mi, p)
        assert self.m.elem == dgc.DGC_QUAD and self.m.nonaffine > 0
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

    def rk(self, c, cfl, steps=1, static=False, prec=dgc.DGC_FP64):
        T = self.torch
        dgc.dgc_import_state(self.m.h, c, self.c)
        ws = T.empty(dgc.dgc_workspace_size(self.m.h, prec) // 8 + 64, dtype=T.float64, device=self.dev)
        d = T.zeros(1, dtype=T.float64, device=self.dev)
        for _ in range(steps):
            if static:
                dgc.dgc_rk_step_static(self.m.h, prec, self.c, cfl, d)
            else:
                dgc.dgc_rk_step(self.m.h, prec, self.c, cfl, d, ws)
        T.cuda.synchronize()
        return dgc.dgc_export_state(self.m.h, self.c), float(d.item())

    def close(self):
        self.m.close()


def _vortex(om, mi, p, perturb=1e-3, seed=9):
    xyz, _, _ = om.eval_points(p)
    c = om.project(p, W.vortex_field(xyz[..., 0], xyz[..., 1], beta=5.0))
    return _zero_tri(mi, p, c + W.uniform_perturbation(c.shape, seed, perturb))


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("kind", ["quad", "quad_open", "hybrid"])
def test_bilinear_rhs_matches_oracle(torch_dev, oracle_mod, kind, p):
    mi = _mesh(kind)
    run = B(torch_dev, mi, p)
    c = _zero_tri(mi, p, W.random_state(mi.ne, 4, (p + 1) ** 2, seed=p, amp=3e-3))
    ref = oracle_mod.OracleMesh.from_input(mi).rhs(p, c)
    check(run.rhs(c), ref, 1e-12, f"bilinear {kind} p = {p}")
    check(run.rhs(c, "atomic"), ref, 1e-12, f"bilinear atomic {kind} p = {p}")
    check(run.rhs(c, prec=dgc.DGC_FP32_MIXED), ref, 1e-5, f"bilinear FP32-mixed {kind} p = {p}")
    check(run.rhs(c, "atomic", dgc.DGC_FP32_MIXED), ref, 1e-5, f"bilinear FP32-mixed atomic {kind} p = {p}")
    run.close()


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("kind", ["quad", "hybrid"])
def test_bilinear_rk_step_matches_oracle(torch_dev, oracle_mod, kind, p):
    mi = _mesh(kind, n=14, seed=6)
    om = oracle_mod.OracleMesh.from_input(mi)
    c = _vortex(om, mi, p)
    ref, dt_ref = om.rk_step(p, c, 0.3)
    run = B(torch_dev, mi, p)
    got, dt = run.rk(c, 0.3)
    assert abs(dt - dt_ref) < 1e-13 * dt_ref
    check(got - c, ref - c, 1e-11, f"bilinear {kind} RK step p = {p}")
    got_s, dt_s = run.rk(c, 0.3, static=True)
    assert np.array_equal(got_s, got) and dt_s == dt
    got, dt = run.rk(c, 0.3, prec=dgc.DGC_FP32_MIXED)
    assert abs(dt - dt_ref) < 1e-13 * dt_ref
    check(got - c, ref - c, 1e-5, f"bilinear FP32-mixed {kind} RK step p = {p}")
    got_s, dt_s = run.rk(c, 0.3, static=True, prec=dgc.DGC_FP32_MIXED)
    assert np.array_equal(got_s, got) and dt_s == dt
    run.close()


def test_bilinear_freestream(torch_dev, oracle_mod):
    """A uniform state: its projection on every element (a multiple of the
    first basis function, which is constant) gives a zero right-hand side to
    rounding, the face and volume integrals of a constant flux cancelling."""
    mi = _mesh("hybrid", n=10)
    om = oracle_mod.OracleMesh.from_input(mi)
    xyz, _, _ = om.eval_points(2)
    ub = np.array([1.1, 0.3, -0.2, 2.6])
    c = om.project(2, np.broadcast_to(ub, xyz.shape[:2] + (4,)).copy())
    run = B(torch_dev, mi, 2)
    r = run.rhs(c)
    h = 0.1
    assert np.abs(r).max() * (0.5 * h * h) / (3.4 * h * 3.0) < 1e-12
    r32 = run.rhs(c, prec=dgc.DGC_FP32_MIXED)
    assert np.abs(r32).max() * (0.5 * h * h) / (3.4 * h * 3.0) < 1e-6
    run.close()


def test_bilinear_larger_mesh_sampled(torch_dev, oracle_mod):
    """160 x 160 jittered (general) quadrilaterals, p = 3, vortex state: FP64
    against the extended oracle on 2,000 sampled elements."""
    mi = W.periodic_square_quad(160, "vertex", 0.2, seed=8)
    p = 3
    om = oracle_mod.OracleMesh.from_input(mi)
    c = _vortex(om, mi, p)
    sample = np.sort(np.random.default_rng(0).choice(om.ne, 2000, replace=False))
    ref = om.rhs(p, c, elems=sample)
    refx = oracle_mod.OracleMesh.from_input(mi, build="extended").rhs(p, c, elems=sample)
    run = B(torch_dev, mi, p)
    got = run.rhs(c)[sample]
    e, eo = fp64_vs_exact(got, ref, refx, 1e-12, "bilinear 160 x 160")
    print(f"bilinear 160 x 160: FP64 vs exact {e:.2e} (FP64 oracle {eo:.2e}), {om.ne} elements")
    run.close()
