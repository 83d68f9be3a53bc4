"""Batched meshes (one persistent launch per kernel class and RK stage over many
meshes of uneven size and order, replayed from a CUDA graph) against the same
meshes stepped one at a time with dgc_rk_step: the batched kernels run the same
per-edge and per-element code, so the states and time steps must be identical.
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
    best, ms = dgc.dgc_batch_autotune(batch, prec, cb, 0.3, dts, ws, reps=2)
    assert best in (16, 32, 64, 128) and all(v > 0 for v in ms.values())
    assert ms[best] == min(ms.values())
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_batch_rk_step(batch, prec, cb, 0.3, dts, ws, workspace_bytes=need - 1)
    assert e.value.status == 1
    for c in cb:
        assert torch.isfinite(c).all()
    dgc.dgc_batch_destroy(batch)
    for m in meshes:
        m.close()
