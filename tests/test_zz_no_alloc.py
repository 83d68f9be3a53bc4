"""dgc_rk_step_static: the allocation-free RK step, against dgc_rk_step.

Some callers cannot allocate device memory -- their device memory belongs to a
host framework's own pool, or their time loop must keep a fixed footprint once
running -- so they cannot hand dgc_rk_step the workspace it needs.
dgc_rk_step_static takes that workspace from a fixed 16 MiB array the library
holds on the device.  This file checks, through the C ABI, that two steps in a
row give the same state and time step as the regular entry point (within the
tolerances of the other RK tests), that the static calls leave the device's free
memory unchanged (the array is reserved by the mesh upload, with the module
loading left at the CUDA default), that a mesh not yet on the device and a mesh
too large for the array are refused, and it runs the same way alone in a fresh
process or after the rest of the suite (the file is collected last).
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


@pytest.mark.parametrize("prec,tol", [(dgc.DGC_FP64, 1e-11), (dgc.DGC_FP32_MIXED, 1e-5)])
def test_static_step_matches_regular_step(torch_dev, prec, tol):
    torch, dev = torch_dev
    mi = W.periodic_square_tri(24, jitter=0.2, seed=12)
    mesh = dgc.Mesh.from_input(mi, 2)
    mesh.color(1601)
    xyz = dgc.dgc_vol_points(mesh.h)
    c0 = dgc.dgc_project(mesh.h, W.vortex_field(xyz[..., 0], xyz[..., 1]))
    a = torch.empty(mesh.state_shape(), dtype=torch.float64, device=dev)
    b = torch.empty_like(a)
    dgc.dgc_import_state(mesh.h, c0, a)  # first device call: uploads the mesh
    dgc.dgc_import_state(mesh.h, c0, b)
    ws = torch.empty(dgc.dgc_workspace_size(mesh.h, prec) // 8 + 64, dtype=torch.float64, device=dev)
    dta = torch.zeros(1, dtype=torch.float64, device=dev)
    dtb = torch.zeros(1, dtype=torch.float64, device=dev)
    for step in range(2):  # two calls in a row
        dgc.dgc_rk_step(mesh.h, prec, a, 0.3, dta, ws)
        torch.cuda.synchronize()
        # the regular step has launched every kernel the static one uses, so the
        # driver has loaded their code: the static call itself must not change
        # the device's free memory (the array was reserved at the mesh upload)
        free_before = torch.cuda.mem_get_info()[0]
        torch_before = torch.cuda.memory_allocated()
        dgc.dgc_rk_step_static(mesh.h, prec, b, 0.3, dtb)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before, f"call {step}: free device memory changed"
        assert torch.cuda.memory_allocated() == torch_before
        ua = dgc.dgc_export_state(mesh.h, a)
        ub = dgc.dgc_export_state(mesh.h, b)
        assert abs(dtb.item() - dta.item()) <= 1e-13 * dta.item()
        check(ub - c0, ua - c0, tol, f"call {step}")
    mesh.close()


def test_static_step_refusals(torch_dev):
    torch, dev = torch_dev
    c = torch.zeros(16, dtype=torch.float64, device=dev)
    dt = torch.zeros(1, dtype=torch.float64, device=dev)
    # colored but never on the device: uploading would allocate, so it is refused
    small = dgc.Mesh.from_input(W.periodic_square_tri(10), 1)
    small.color(1)
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_rk_step_static(small.h, dgc.DGC_FP64, c, 0.3, dt)
    assert e.value.status == 1 and "first" in str(e.value)
    small.close()
    # 32,768 triangles at p = 3 need more scratch than the 16 MiB array holds
    big = dgc.Mesh.from_input(W.periodic_square_tri(128), 3)
    big.color(1)
    with pytest.raises(dgc.DgcError) as e:
        dgc.dgc_rk_step_static(big.h, dgc.DGC_FP32_MIXED, c, 0.3, dt)
    assert e.value.status == 1 and "too large" in str(e.value)
    big.close()
