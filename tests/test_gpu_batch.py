"""Batched meshes (one persistent launch per kernel class and RK stage over many
meshes of uneven size and order, replayed from a CUDA graph) against the same
meshes stepped one at a time with dgc_rk_step: the batched kernels run the same
per-edge and per-element code, so the states and time steps must be identical.
"""

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


SPECS = [(7, 1), (16, 3), (9, 2), (23, 3), (12, 1), (5, 2)]


def _meshes_and_states(seed=0):
    meshes, states = [], []
    for i, (n, p) in enumerate(SPECS):
        mi = W.periodic_square_tri(n, jitter=0.2, seed=100 + i)
        m = dgc.Mesh.from_input(mi, p)
        m.color(1601 + i)
        xyz = dgc.dgc_vol_points(m.h)
        c = dgc.dgc_project(m.h, W.vortex_field(xyz[..., 0], xyz[..., 1], beta=3.0 + 0.5 * i, xc=0.4 + 0.03 * i))
        meshes.append(m)
        states.append(c)
    return meshes, states


@pytest.mark.parametrize("tpe", [2, 4])
def test_batch_four_threads_per_edge_equal_single_mesh(torch_dev, tpe):
    """Batched FP32-mixed step with 2 or 4 threads per edge (all classes, 32
    edges per block) equals the single-mesh step with the same tiles bit for
    bit: the same per-edge code."""
    torch, dev = torch_dev
    meshes, states = _meshes_and_states()
    prec = dgc.DGC_FP32_MIXED
    cb = [torch.empty(m.state_shape(), dtype=torch.float64, device=dev) for m in meshes]
    cs = [torch.empty_like(x) for x in cb]
    for m, c, a, b in zip(meshes, states, cb, cs):
        dgc.dgc_import_state(m.h, c, a)
        dgc.dgc_import_state(m.h, c, b)
        dgc.dgc_set_option(m.h, dgc.DGC_OPT_EDGES_PER_BLOCK, 32)
        dgc.dgc_set_option(m.h, dgc.DGC_OPT_THREADS_PER_EDGE, tpe)
    batch = dgc.dgc_batch_create(meshes)
    dgc.dgc_batch_set_option(batch, dgc.DGC_OPT_EDGES_PER_BLOCK, 32)
    dgc.dgc_batch_set_option(batch, dgc.DGC_OPT_THREADS_PER_EDGE, tpe)
    ws = torch.empty(dgc.dgc_batch_workspace_size(batch, prec) // 8 + 64, dtype=torch.float64, device=dev)
    dts = torch.zeros(len(meshes), dtype=torch.float64, device=dev)
    for _ in range(2):
        dgc.dgc_batch_rk_step(batch, prec, cb, 0.3, dts, ws)
    torch.cuda.synchronize()
    for i, m in enumerate(meshes):
        wsi = torch.empty(dgc.dgc_workspace_size(m.h, prec) // 8 + 64, dtype=torch.float64, device=dev)
        d = torch.zeros(1, dtype=torch.float64, device=dev)
        for _ in range(2):
            dgc.dgc_rk_step(m.h, prec, cs[i], 0.3, d, wsi)
        torch.cuda.synchronize()
        assert dts[i].item() == d.item()
        assert torch.equal(cb[i], cs[i]), f"mesh {i}"
    with pytest.raises(dgc.DgcError):  # 4 x 128 threads exceed a block
        dgc.dgc_batch_set_option(batch, dgc.DGC_OPT_EDGES_PER_BLOCK, 128 if tpe == 4 else 256)
    dgc.dgc_batch_destroy(batch)
    for m in meshes:
        m.close()


@pytest.mark.parametrize("prec", [dgc.DGC_FP64, dgc.DGC_FP32_MIXED])
@pytest.mark.parametrize("graph", [True, False])
def test_batch_equals_single_mesh_steps(torch_dev, prec, graph):
    torch, dev = torch_dev
    meshes, states = _meshes_and_states()
    cb = [torch.empty(m.state_shape(), dtype=torch.float64, device=dev) for m in meshes]
    cs = [torch.empty_like(x) for x in cb]
    for m, c, a, b in zip(meshes, states, cb, cs):
        dgc.dgc_import_state(m.h, c, a)
        dgc.dgc_import_state(m.h, c, b)
    batch = dgc.dgc_batch_create(meshes)
    dgc.dgc_batch_set_option(batch, dgc.DGC_OPT_GRAPH, int(graph))
    ws = torch.empty(dgc.dgc_batch_workspace_size(batch, prec) // 8 + 64, dtype=torch.float64, device=dev)
    dts = torch.zeros(len(meshes), dtype=torch.float64, device=dev)
    for _ in range(2):
        dgc.dgc_batch_rk_step(batch, prec, cb, 0.3, dts, ws)
    assert dgc.dgc_batch_launch_count(batch) == 12
    torch.cuda.synchronize()
    for i, m in enumerate(meshes):
        wsi = torch.empty(dgc.dgc_workspace_size(m.h, prec) // 8 + 64, dtype=torch.float64, device=dev)
        d = torch.zeros(1, dtype=torch.float64, device=dev)
        for _ in range(2):
            dgc.dgc_rk_step(m.h, prec, cs[i], 0.3, d, wsi)
        torch.cuda.synchronize()
        assert dts[i].item() == d.item()
        assert torch.equal(cb[i], cs[i]), f"mesh {i}"
    dgc.dgc_batch_destroy(batch)
    for m in meshes:
        m.close()


def test_batch_autotune_and_refusals(torch_dev):
    torch, dev = torch_dev
    meshes, states = _meshes_and_states()
    cb = [torch.empty(m.state_shape(), dtype=torch.float64, device=dev) for m in meshes]
    for m, c, a in zip(meshes, states, cb):
        dgc.dgc_import_state(m.h, c, a)
    batch = dgc.dgc_batch_create(meshes)
    prec = dgc.DGC_FP32_MIXED
    need = dgc.dgc_batch_workspace_size(batch, prec)
    ws = torch.empty(need // 8 + 64, dtype=torch.float64, device=dev)
    dts = torch.zeros(len(meshes), dtype=torch.float64, device=dev)
    tiles, ms = dgc.dgc_batch_autotune(batch, prec, cb, 0.3, dts, ws, reps=2)
    assert ms > 0
    for e, t in tiles.values():
        assert e in (16, 32, 64, 128) and t in (2, 4) and e * t <= 256
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_batch_rk_step(batch, prec, cb, 0.3, dts, ws, workspace_bytes=need - 1)
    assert e.value.status == 1
    for c in cb:
        assert torch.isfinite(c).all()
    dgc.dgc_batch_destroy(batch)
    for m in meshes:
        m.close()


# ------------------------------------------------------------------------------------------
# Batch members against the oracle
# ------------------------------------------------------------------------------------------

def _rings(om, seeds, depth):
    l, r, _, _ = om.sides()
    nbr = [[] for _ in range(om.ne)]
    for a, b in zip(l, r):
        if b >= 0:
            nbr[a].append(b)
            nbr[b].append(a)
    sets = [np.unique(seeds)]
    for _ in range(depth):
        cur = set(sets[-1].tolist())
        for e in sets[-1]:
            cur.update(nbr[e])
        sets.append(np.array(sorted(cur)))
    return sets


def _sampled_step(o, p, c, dt, rings):
    """One SSP-RK3 step on the elements s0, each stage on the rings the next needs."""
    s0, s1, s2 = rings
    R = o.real
    c = np.asarray(c, dtype=R)
    dt = R(dt)
    u1 = np.zeros_like(c)
    u1[s2] = c[s2] + dt * o.rhs(p, c, elems=s2)
    u2 = np.zeros_like(c)
    u2[s1] = R(0.75) * c[s1] + R(0.25) * (u1[s1] + dt * o.rhs(p, u1, elems=s1))
    return c[s0] / 3 + R(2) / 3 * (u2[s0] + dt * o.rhs(p, u2, elems=s0))


@pytest.mark.parametrize("prec,tol", [(dgc.DGC_FP64, 1e-11), (dgc.DGC_FP32_MIXED, 1e-5)])
def test_batch_members_match_oracle(torch_dev, oracle_mod, prec, tol):
    """One batched step of six meshes (p = 1, 2, 3; 50 to 1,058 elements):
    every member's state change and time step against the oracle's SSP-RK3
    step of that mesh alone, states projected by the oracle."""
    torch, dev = torch_dev
    meshes, oms, states = [], [], []
    for i, (n, p) in enumerate(SPECS):
        mi = W.periodic_square_tri(n, jitter=0.2, seed=100 + i)
        m = dgc.Mesh.from_input(mi, p)
        m.color(1601 + i)
        om = oracle_mod.OracleMesh.from_input(mi)
        xyz, _, _ = om.eval_points(p)
        states.append(om.project(p, W.vortex_field(xyz[..., 0], xyz[..., 1], beta=3.0 + 0.5 * i, xc=0.4 + 0.03 * i)))
        meshes.append(m)
        oms.append(om)
    cb = [torch.empty(m.state_shape(), dtype=torch.float64, device=dev) for m in meshes]
    for m, c, a in zip(meshes, states, cb):
        dgc.dgc_import_state(m.h, c, a)
    batch = dgc.dgc_batch_create(meshes)
    ws = torch.empty(dgc.dgc_batch_workspace_size(batch, prec) // 8 + 64, dtype=torch.float64, device=dev)
    dts = torch.zeros(len(meshes), dtype=torch.float64, device=dev)
    dgc.dgc_batch_rk_step(batch, prec, cb, 0.3, dts, ws)
    torch.cuda.synchronize()
    for i, (m, om, c) in enumerate(zip(meshes, oms, states)):
        p = SPECS[i][1]
        ref, dt_ref = om.rk_step(p, c, 0.3)
        assert abs(dts[i].item() - dt_ref) < 1e-13 * dt_ref, i
        got = dgc.dgc_export_state(m.h, cb[i])
        check(got - c, ref - c, tol, f"mesh {i} (p = {p})")
    dgc.dgc_batch_destroy(batch)
    for m in meshes:
        m.close()


@pytest.fixture(scope="module")
def batch64(torch_dev, oracle_mod):
    """The 64-mesh batch (2,029,848 triangles, p in {1, 2, 3}), vortex states
    projected by the oracle, on the device."""
    torch, dev = torch_dev
    specs = W.batched_square_meshes()
    mis = [W.periodic_square_tri(s["n"], jitter=0.2, seed=500 + i) for i, s in enumerate(specs)]
    meshes, states = [], []
    for i, (s, mi) in enumerate(zip(specs, mis)):
        m = dgc.Mesh.from_input(mi, s["p"])
        m.color(1601 + i)
        meshes.append(m)
        om = oracle_mod.OracleMesh.from_input(mi)
        xyz, _, _ = om.eval_points(s["p"])
        states.append(om.project(s["p"], W.vortex_field(xyz[..., 0], xyz[..., 1], beta=s["beta"], xc=s["xc"],
                                                        yc=s["yc"])))
        del om
    assert sum(m.info["ne"] for m in meshes) == 2_029_848
    batch = dgc.dgc_batch_create(meshes)
    yield specs, mis, meshes, states, batch
    dgc.dgc_batch_destroy(batch)
    for m in meshes:
        m.close()


@pytest.mark.parametrize("prec", [dgc.DGC_FP64, dgc.DGC_FP32_MIXED])
def test_full_size_batch_sampled(torch_dev, oracle_mod, batch64, prec):
    """The 64-mesh batch at its autotuned tile shape: one batched step, checked
    on ~2,000 sampled elements of the largest mesh of each order against the
    oracle's stages on the rings they need (FP64: within 1e-11 of the extended
    build's exact state change, or the FP64 oracle's own error; FP32-mixed:
    within 1e-5 of the FP64 oracle), and every mesh's dt against the oracle's."""
    torch, dev = torch_dev
    specs, mis, meshes, states, batch = batch64
    ws = torch.empty(dgc.dgc_batch_workspace_size(batch, prec) // 8 + 64, dtype=torch.float64, device=dev)
    dts = torch.zeros(len(meshes), dtype=torch.float64, device=dev)
    scratch = [torch.empty(m.state_shape(), dtype=torch.float64, device=dev) for m in meshes]
    for m, c, a in zip(meshes, states, scratch):
        dgc.dgc_import_state(m.h, c, a)
    best, _ = dgc.dgc_batch_autotune(batch, prec, scratch, 0.3, dts, ws, reps=1)
    best = ", ".join(f"{k} {e}x{t}" for k, (e, t) in best.items())
    cb = [torch.empty(m.state_shape(), dtype=torch.float64, device=dev) for m in meshes]
    for m, c, a in zip(meshes, states, cb):
        dgc.dgc_import_state(m.h, c, a)
    del scratch
    dgc.dgc_batch_rk_step(batch, prec, cb, 0.3, dts, ws)
    torch.cuda.synchronize()
    picks = [max((i for i, s in enumerate(specs) if s["p"] == p), key=lambda i: meshes[i].info["ne"])
             for p in (1, 2, 3)]
    rng = np.random.default_rng(5)
    for i in picks:
        p = specs[i]["p"]
        om = oracle_mod.OracleMesh.from_input(mis[i])
        c = states[i]
        dt = om.dt(p, c, 0.3)
        assert abs(dts[i].item() - dt) < 1e-13 * dt
        seeds = rng.choice(om.ne, 150, replace=False)
        s0, s1, s2, _ = _rings(om, seeds, 3)
        got = dgc.dgc_export_state(meshes[i].h, cb[i])[s0] - c[s0]
        u3 = _sampled_step(om, p, c, dt, (s0, s1, s2)) - c[s0]
        what = f"batch mesh {i} ({meshes[i].info['ne']} elements, p = {p}, tiles {best})"
        if prec == dgc.DGC_FP64:
            ox = oracle_mod.OracleMesh.from_input(mis[i], build="extended")
            u3x = _sampled_step(ox, p, c, dt, (s0, s1, s2)) - c[s0]
            e, eo = fp64_vs_exact(got, u3, u3x, 1e-11, what)
            print(f"{what}: FP64 du vs exact {e:.2e} (FP64 oracle {eo:.2e}), {s0.size} elements")
        else:
            e, _ = check(got, u3, 1e-5, what)
            print(f"{what}: FP32-mixed du {e:.2e}, {s0.size} elements")
    # every mesh's time step
    for i in range(len(meshes)):
        om = oracle_mod.OracleMesh.from_input(mis[i])
        dt = om.dt(specs[i]["p"], states[i], 0.3)
        assert abs(dts[i].item() - dt) < 1e-13 * dt, i


def test_batch_profile_collect(torch_dev):
    """DGC_OPT_PROFILE on a batch: event pairs per launch (graph off), the same
    states as the graph replay."""
    torch, dev = torch_dev
    meshes, states = _meshes_and_states()
    prec = dgc.DGC_FP32_MIXED
    out = []
    for profile in (0, 1):
        cb = [torch.empty(m.state_shape(), dtype=torch.float64, device=dev) for m in meshes]
        for m, c, a in zip(meshes, states, cb):
            dgc.dgc_import_state(m.h, c, a)
        batch = dgc.dgc_batch_create(meshes)
        dgc.dgc_batch_set_option(batch, dgc.DGC_OPT_PROFILE, profile)
        ws = torch.empty(dgc.dgc_batch_workspace_size(batch, prec) // 8 + 64, dtype=torch.float64, device=dev)
        dts = torch.zeros(len(meshes), dtype=torch.float64, device=dev)
        for _ in range(2):
            dgc.dgc_batch_rk_step(batch, prec, cb, 0.3, dts, ws)
        torch.cuda.synchronize()
        if profile:
            prof = dgc.dgc_batch_profile_collect(batch)
            assert {k: v[1] for k, v in prof.items()} == {"cfl": 4, "first": 6, "color": 6, "last": 6}
            assert all(v[0] > 0 for v in prof.values())
        out.append([x.clone() for x in cb])
        dgc.dgc_batch_destroy(batch)
    for a, b in zip(*out):
        assert torch.equal(a, b)
    for m in meshes:
        m.close()
