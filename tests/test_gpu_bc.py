"""GPU parity of the boundary conditions, the limiter and the mesh's time
(the double Mach reflection run of Sec. 5, Table 7: slip walls, prescribed
states, the moving incident shock and a limiter after every RK stage; readings
of [giuliani], dg_oracle.c bc_state / orc_limit) against the oracle, FP64.

Tolerances: FP64 right-hand side 1e-12 relative L2 (colored, atomic, two-pass),
FP32-mixed 1e-5; the FP32 forms' RK step (boundary conditions, no limiter)
1e-5;
the limiter alone 1e-13; one limited RK step's state change 1e-11; ten
limited steps of the double Mach setup 1e-10 (per-element max as in
tests/_parity.py); dt and the advanced time 1e-13.  The allocation-free step
is bit-identical to the regular one.  Batches, refinement and the cooperative
right-hand side refuse boundary conditions, and the FP32 forms the limiter.
"""

import numpy as np
import pytest

from paper_1601_07613_gb300 import dgc
from paper_1601_07613_gb300 import workloads as W
from _parity import check

pytestmark = pytest.mark.gpu
FP64 = dgc.DGC_FP64


@pytest.fixture(scope="module")
def torch_dev():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    dgc.lib()
    return torch, torch.device("cuda:0")


class Run:
    """A double Mach-type mesh with its boundary conditions on the device and
    in the oracle."""

    def __init__(self, torch_dev, oracle_mod, mi, p, limiter=False, seed=1601, states=None):
        self.torch, self.dev = torch_dev
        self.p = p
        self.m = dgc.Mesh.from_input(mi, p)
        self.m.color(seed)
        l, r, ql, qr = dgc.dgc_get_sides(self.m.h)
        self.om = oracle_mod.OracleMesh.from_input(mi)
        lo, ro, qlo, _ = self.om.sides()
        assert np.array_equal(l, lo) and np.array_equal(r, ro) and np.array_equal(ql, qlo)
        kind, sidx = W.double_mach_boundary(mi, l, r, ql)
        self.kind = kind
        S = W.double_mach_states() if states is None else states
        dgc.dgc_set_boundary(self.m.h, kind, sidx, S, W.DMR_SHOCK, (0, 1))
        self.om.set_bc(kind, sidx, S, W.DMR_SHOCK, (0, 1))
        if limiter:
            dgc.dgc_set_option(self.m.h, dgc.DGC_OPT_LIMITER, 1)
            self.om.set_limiter(True)
        T = self.torch
        self.c = T.empty(self.m.state_shape(), dtype=T.float64, device=self.dev)
        self.r = T.empty_like(self.c)

    def set_time(self, t):
        dgc.dgc_set_time(self.m.h, t)
        self.om.set_time(t)

    def ic(self):
        xyz, _, _ = self.om.eval_points(self.p)
        return self.om.limit(self.p, self.om.project(self.p, W.double_mach_field(xyz[..., 0], xyz[..., 1])))

    def rhs(self, c, kind="colored", prec=FP64):
        T = self.torch
        dgc.dgc_import_state(self.m.h, c, self.c)
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

    def rk(self, c, cfl=0.3, steps=1, static=False):
        T = self.torch
        dgc.dgc_import_state(self.m.h, c, self.c)
        ws = T.empty(dgc.dgc_workspace_size(self.m.h, FP64) // 8 + 64, dtype=T.float64, device=self.dev)
        d = T.zeros(1, dtype=T.float64, device=self.dev)
        dts = []
        for _ in range(steps):
            if static:
                dgc.dgc_rk_step_static(self.m.h, FP64, self.c, cfl, d)
            else:
                dgc.dgc_rk_step(self.m.h, FP64, self.c, cfl, d, ws)
            dts.append(float(d.item()))
        T.cuda.synchronize()
        return dgc.dgc_export_state(self.m.h, self.c), dts

    def close(self):
        self.m.close()


def _mesh(nx=32, ny=8, seed=21):
    return W.open_rect_tri(nx, ny, 4.0, 1.0, jitter=0.2, seed=seed)


def _conserved(rho, u, v, pr):
    return [rho, rho * u, rho * v, pr / 0.4 + 0.5 * rho * (u * u + v * v)]


# Prescribed states near the smooth field below, for the unlimited RK steps:
# the double Mach states (density 8 behind a Mach 10 shock) against that field
# make a discontinuity that an unlimited step turns non-physical.
MILD_STATES = np.array([_conserved(1.6, 1.1, -0.6, 2.1), _conserved(1.4, 0.9, -0.8, 1.9)])


def _smooth(run, seed):
    """A positive smooth state with large velocities at every boundary."""
    xyz, _, _ = run.om.eval_points(run.p)
    x, y = xyz[..., 0], xyz[..., 1]
    rho = 1.5 + 0.3 * np.sin(2 * x + 3 * y)
    u = 1.0 + 0.5 * np.cos(3 * x - y)
    v = -0.7 + 0.4 * np.sin(x + 2 * y)
    pr = 2.0 + 0.2 * np.cos(x * y)
    U = np.stack([rho, rho * u, rho * v, pr / 0.4 + 0.5 * rho * (u * u + v * v)], axis=-1)
    c = run.om.project(run.p, U)
    return c + W.uniform_perturbation(c.shape, seed, 1e-2)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_boundary_rhs_matches_oracle(torch_dev, oracle_mod, p):
    run = Run(torch_dev, oracle_mod, _mesh(), p)
    assert set(np.unique(run.kind[run.om.sides()[1] < 0])) == {0, 1, 2, 3}
    run.set_time(0.05)  # the shock's trace on the top boundary mid-domain
    c = _smooth(run, p)
    ref = run.om.rhs(p, c)
    for kind in ("colored", "atomic", "two_pass"):
        check(run.rhs(c, kind), ref, 1e-12, f"boundary rhs {kind} p = {p}")
    run.close()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_boundary_rhs_fp32_matches_oracle(torch_dev, oracle_mod, p):
    """The FP32-mixed right-hand side with the same boundaries: the second lane
    of a boundary face evaluates the outside state as a deviation from the
    element's reference (walls mirror it, state and shock faces replace it)."""
    run = Run(torch_dev, oracle_mod, _mesh(), p)
    run.set_time(0.05)
    c = _smooth(run, 20 + p)
    ref = run.om.rhs(p, c)
    for kind in ("colored", "atomic", "two_pass"):
        check(run.rhs(c, kind, dgc.DGC_FP32_MIXED), ref, 1e-5, f"boundary rhs FP32 {kind} p = {p}")
    run.close()


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("fuse", [True, False])
def test_boundary_rk_step_fp32_matches_oracle(torch_dev, oracle_mod, p, fuse):
    """The FP32 forms' RK step with boundaries (no limiter): the state change
    against the oracle's, and the mesh's time advanced by dt.  Walls, the
    transmissive outflow and a moving shock between two prescribed states
    near the smooth field (the stage times t, t + dt, t + dt / 2 move the
    shock's foot along the bottom)."""
    run = Run(torch_dev, oracle_mod, _mesh(seed=25), p, states=MILD_STATES)
    dgc.dgc_set_option(run.m.h, dgc.DGC_OPT_FUSE, int(fuse))
    c = _smooth(run, 30 + p)
    T = run.torch
    for prec in (dgc.DGC_FP32_MIXED, dgc.DGC_FP32_KAHAN):
        run.set_time(0.05)
        ref, dt_ref = run.om.rk_step(p, c, 0.3)
        assert np.isfinite(ref).all()
        d = T.zeros(1, dtype=T.float64, device=run.dev)
        ws = T.empty(dgc.dgc_workspace_size(run.m.h, prec) // 8 + 64, dtype=T.float64, device=run.dev)
        if prec == dgc.DGC_FP32_KAHAN:
            k = T.empty(dgc.dgc_state_bytes(run.m.h, prec) // 4, dtype=T.float32, device=run.dev)
            dgc.dgc_import_state_prec(run.m.h, prec, c, k)
            dgc.dgc_rk_step(run.m.h, prec, k, 0.3, d, ws)
            T.cuda.synchronize()
            got = dgc.dgc_export_state_prec(run.m.h, prec, k)
        else:
            dgc.dgc_import_state(run.m.h, c, run.c)
            dgc.dgc_rk_step(run.m.h, prec, run.c, 0.3, d, ws)
            T.cuda.synchronize()
            got = dgc.dgc_export_state(run.m.h, run.c)
        dt = float(d.item())
        assert abs(dt - dt_ref) < 1e-12 * dt_ref
        check(got - c, ref - c, 1e-5, f"FP32 RK step with boundaries, prec {prec}, p = {p}")
        t = dgc.dgc_get_time(run.m.h)
        assert abs(t - run.om.time()) < 1e-13 * t
    run.close()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_limiter_matches_oracle(torch_dev, oracle_mod, p):
    run = Run(torch_dev, oracle_mod, _mesh(seed=22), p)
    c = _smooth(run, 10 + p)
    c[:, :, 1:] += np.random.default_rng(p).uniform(-0.3, 0.3, c[:, :, 1:].shape)
    ref = run.om.limit(p, c)
    dgc.dgc_import_state(run.m.h, c, run.c)
    dgc.dgc_limit(run.m.h, FP64, run.c)
    run.torch.cuda.synchronize()
    got = dgc.dgc_export_state(run.m.h, run.c)
    assert np.array_equal(got[:, :, 0], c[:, :, 0])
    assert np.abs(ref - c).max() > 1e-2  # the limiter acted
    check(got, ref, 1e-13, f"limiter p = {p}")
    run.close()


@pytest.mark.parametrize("p", [1, 2])
def test_limited_rk_step_matches_oracle(torch_dev, oracle_mod, p):
    """One limited SSP-RK3 step from the double Mach state a few oracle steps
    after the start (the shock has moved off the grid lines)."""
    run = Run(torch_dev, oracle_mod, _mesh(), p, limiter=True)
    c = run.ic()
    for _ in range(3):
        c, _ = run.om.rk_step(p, c, 0.3)
    t0 = run.om.time()
    run.set_time(t0)
    ref, dt_ref = run.om.rk_step(p, c, 0.3)
    got, dts = run.rk(c)
    assert abs(dts[0] - dt_ref) < 1e-13 * dt_ref
    check(got - c, ref - c, 1e-11, f"limited RK step p = {p}")
    t = dgc.dgc_get_time(run.m.h)
    assert abs(t - run.om.time()) < 1e-13 * t
    run.set_time(t0)
    got_s, dts_s = run.rk(c, static=True)
    assert np.array_equal(got_s, got) and dts_s == dts
    run.close()


def test_double_mach_ten_steps_match_oracle(torch_dev, oracle_mod):
    run = Run(torch_dev, oracle_mod, _mesh(64, 16, seed=23), 1, limiter=True)
    c0 = run.ic()
    ref = c0.copy()
    for _ in range(10):
        ref, _ = run.om.rk_step(1, ref, 0.3)
    got, dts = run.rk(c0, steps=10)
    check(got - c0, ref - c0, 1e-10, "double Mach, 10 limited steps")
    assert abs(dgc.dgc_get_time(run.m.h) - run.om.time()) < 1e-13 * run.om.time()
    U = got[:, :, 0] * np.sqrt(2.0)
    pr = 0.4 * (U[:, 3] - 0.5 * (U[:, 1] ** 2 + U[:, 2] ** 2) / U[:, 0])
    assert (U[:, 0] > 0).all() and (pr > 0).all()
    run.close()


def test_boundary_refusals(torch_dev, oracle_mod):
    run = Run(torch_dev, oracle_mod, _mesh(8, 2, seed=24), 1, limiter=True)
    for prec in (dgc.DGC_FP32_MIXED, dgc.DGC_FP32_KAHAN):
        with pytest.raises(dgc.DgcError) as e:
            dgc.dgc_rhs(run.m.h, prec, run.c, run.r)
        assert e.value.status == 4
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_refine(run.m.h, np.array([0], np.int32))
    assert e.value.status == 4
    dgc.dgc_set_option(run.m.h, dgc.DGC_OPT_COOPERATIVE, 1)
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_rhs(run.m.h, FP64, run.c, run.r)
    assert e.value.status == 4
    run.close()
    q = dgc.Mesh.from_input(W.open_square_quad(4), 1)
    q.color(1)
    ns = q.info["ns"]
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_set_boundary(q.h, np.ones(ns, np.int8))
    assert e.value.status == 4
    q.close()
