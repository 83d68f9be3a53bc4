"""Dynamic adaptivity on the device (Sec. 3.2): the 6-color map of a refined mesh
evaluated by a GPU kernel, the state moved between a mesh and its refinement by
GPU kernels, and a refine -> step -> coarsen cycle against the oracle.

* the device color map equals the host's refinement colors and the oracle's
  (bit for bit), on a test mesh and on the 180,512-element refined workload;
* prolongation and restriction equal the oracle's L2 projections (computed by
  quadrature through physical points, independent of the library's child
  projection matrices) within 1e-13 relative;
* a cycle: the coarse vortex state, refined, prolonged, five SSP-RK3 steps on the
  refined mesh (FP64 and FP32-mixed), restricted and coarsened, against the
  oracle doing the same (FP64: its extended build, the exact result of the same
  inputs); the state change within 1e-11 (FP64) and 1e-5 (FP32-mixed) relative
  L2, and the total of the means conserved.
"""

import numpy as np
import pytest

from paper_1601_07613_gb300 import dgc
from paper_1601_07613_gb300 import workloads as W
from _amr import second_level
from _parity import check, fp64_vs_exact

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    dgc.lib()
    return torch, torch.device("cuda:0")


def _mesh(kind):
    if kind == "periodic":
        mi = W.periodic_square_tri(30, jitter=0.2, seed=91)
    else:
        mi = W.open_square_tri(24, jitter=0.2, seed=92)
    return mi, W.elements_near(mi, (0.45, 0.55), 0.3)


def _host_colors(m):
    return dgc.dgc_get_ordering(m.h)[2]  # color of each original edge


@pytest.mark.parametrize("kind", ["periodic", "open", "full"])
def test_device_color_map_bit_exact(torch_dev, oracle_mod, kind):
    if kind == "full":
        cfg = W.refined_square_vortex_p2_256()
        mi, elems = cfg["mesh"], cfg["refine"]
    else:
        mi, elems = _mesh(kind)
    m = dgc.Mesh.from_input(mi, 2)
    m.color(1601)
    om = oracle_mod.OracleMesh.from_input(mi)
    col, _ = om.color(3, 1601)
    m.refine(elems)
    got, ms = dgc.dgc_refine_colors_device(m.h, m.info["ns"])
    assert ms >= 0.0
    assert np.array_equal(got, _host_colors(m))
    assert np.array_equal(got, om.refine(col, elems).colors)
    assert set(np.unique(got)) == {1, 2, 3, 4, 5, 6}
    m.close()


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("kind", ["periodic", "open"])
def test_prolong_and_restrict_match_oracle(torch_dev, oracle_mod, kind, p):
    torch, dev = torch_dev
    mi, elems = _mesh(kind)
    om = oracle_mod.OracleMesh.from_input(mi)
    col, _ = om.color(3, 1601)
    fm = om.refine(col, elems)
    m = dgc.Mesh.from_input(mi, p)
    m.color(1601)
    np_ = m.info["np"]
    c0 = W.random_state(om.ne, 4, np_, seed=p, amp=5e-2)
    cc = torch.empty(m.state_shape(), dtype=torch.float64, device=dev)
    dgc.dgc_import_state(m.h, c0, cc)
    m.refine(elems)
    cf = torch.empty(m.state_shape(), dtype=torch.float64, device=dev)
    dgc.dgc_prolong_state(m.h, cc, cf)
    torch.cuda.synchronize()
    got = dgc.dgc_export_state(m.h, cf)
    ref = fm.prolong(p, c0)
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()
    f = W.random_state(fm.ne, 4, np_, seed=10 + p, amp=5e-2)
    dgc.dgc_import_state(m.h, f, cf)
    cc2 = torch.empty_like(cc)
    dgc.dgc_restrict_state(m.h, cf, cc2)
    m.coarsen()
    torch.cuda.synchronize()
    got = dgc.dgc_export_state(m.h, cc2)
    ref = fm.restrict(p, f)
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()
    m.close()


@pytest.mark.parametrize("prec,tol", [(dgc.DGC_FP64, 1e-11), (dgc.DGC_FP32_MIXED, 1e-5)])
def test_refine_step_coarsen_cycle(torch_dev, oracle_mod, prec, tol):
    torch, dev = torch_dev
    mi, elems = _mesh("periodic")
    p, steps = 2, 5
    om = oracle_mod.OracleMesh.from_input(mi)
    col, _ = om.color(3, 1601)
    fm = om.refine(col, elems)
    xyz, _, _ = om.eval_points(p)
    c0 = om.project(p, W.vortex_field(xyz[..., 0], xyz[..., 1], beta=5.0))
    # oracle (FP64, and the extended build for the FP64 comparison): prolong,
    # steps on the refined mesh, restrict
    def cycle(o, f):
        u = f.prolong(p, c0)
        for _ in range(steps):
            u, _ = f.rk_step(p, u, 0.3)
        return f.restrict(p, u)

    ref = cycle(om, fm)
    if prec == dgc.DGC_FP64:
        ox = oracle_mod.OracleMesh.from_input(mi, build="extended")
        refx = cycle(ox, ox.refine(col, elems))
    # device
    m = dgc.Mesh.from_input(mi, p)
    m.color(1601)
    cc = torch.empty(m.state_shape(), dtype=torch.float64, device=dev)
    dgc.dgc_import_state(m.h, c0, cc)
    m.refine(elems)
    cf = torch.empty(m.state_shape(), dtype=torch.float64, device=dev)
    dgc.dgc_prolong_state(m.h, cc, cf)
    ws = torch.empty(dgc.dgc_workspace_size(m.h, prec) // 8 + 64, dtype=torch.float64, device=dev)
    d = torch.zeros(1, dtype=torch.float64, device=dev)
    for _ in range(steps):
        dgc.dgc_rk_step(m.h, prec, cf, 0.3, d, ws)
    dgc.dgc_restrict_state(m.h, cf, cc)
    m.coarsen()
    torch.cuda.synchronize()
    got = dgc.dgc_export_state(m.h, cc)
    if prec == dgc.DGC_FP64:
        e, _ = fp64_vs_exact(got - c0, ref - c0, refx - c0, tol, "refine-step-coarsen FP64")
    else:
        e, _ = check(got - c0, ref - c0, tol, f"refine-step-coarsen prec {prec}")
    print(f"refine -> {steps} steps -> coarsen, prec {prec}: du rel L2 {e:.2e}")
    dj = om.detj()
    t0 = (dj[:, None] * c0[:, :, 0]).sum(0)
    t1 = (dj[:, None] * got[:, :, 0]).sum(0)
    np.testing.assert_allclose(t1, t0, rtol=1e-12, atol=1e-13 * np.abs(t0).max())
    # the mesh is the coarse one again: a step runs on it
    assert m.info["ncolors"] == 3 and m.info["ne"] == om.ne
    ws = torch.empty(dgc.dgc_workspace_size(m.h, prec) // 8 + 64, dtype=torch.float64, device=dev)
    dgc.dgc_rk_step(m.h, prec, cc, 0.3, d, ws)
    torch.cuda.synchronize()
    assert torch.isfinite(cc).all()
    m.close()


def test_two_level_color_map_and_cycle(torch_dev, oracle_mod):
    """A second level on the device: its color map (the palette doubled again,
    12 colors) bit for bit against the host's and the oracle's; then the coarse
    vortex state prolonged through both levels, three FP64 steps on the
    two-level mesh, restricted and coarsened back through both levels, against
    the oracle (its extended build for the FP64 comparison)."""
    torch, dev = torch_dev
    mi, elems = _mesh("periodic")
    p, steps = 2, 3
    om = oracle_mod.OracleMesh.from_input(mi)
    col, _ = om.color(3, 1601)
    f1 = om.refine(col, elems)
    e2 = second_level(f1, (0.45, 0.55), 0.18, 0.36)
    f2 = f1.refine(f1.colors, e2)
    xyz, _, _ = om.eval_points(p)
    c0 = om.project(p, W.vortex_field(xyz[..., 0], xyz[..., 1], beta=5.0))

    def cycle(g1, g2):
        u = g2.prolong(p, g1.prolong(p, c0))
        for _ in range(steps):
            u, _ = g2.rk_step(p, u, 0.3)
        return g1.restrict(p, g2.restrict(p, u))

    ref = cycle(f1, f2)
    ox = oracle_mod.OracleMesh.from_input(mi, build="extended")
    x1 = ox.refine(col, elems)
    refx = cycle(x1, x1.refine(x1.colors, e2))
    m = dgc.Mesh.from_input(mi, p)
    m.color(1601)
    cc = torch.empty(m.state_shape(), dtype=torch.float64, device=dev)
    dgc.dgc_import_state(m.h, c0, cc)
    m.refine(elems)
    c1 = torch.empty(m.state_shape(), dtype=torch.float64, device=dev)
    dgc.dgc_prolong_state(m.h, cc, c1)
    m.refine(e2)
    got, _ = dgc.dgc_refine_colors_device(m.h, m.info["ns"])
    assert np.array_equal(got, _host_colors(m)) and np.array_equal(got, f2.colors)
    assert set(np.unique(got)) == set(range(1, 13))
    c2 = torch.empty(m.state_shape(), dtype=torch.float64, device=dev)
    dgc.dgc_prolong_state(m.h, c1, c2)
    ws = torch.empty(dgc.dgc_workspace_size(m.h, dgc.DGC_FP64) // 8 + 64, dtype=torch.float64, device=dev)
    d = torch.zeros(1, dtype=torch.float64, device=dev)
    for _ in range(steps):
        dgc.dgc_rk_step(m.h, dgc.DGC_FP64, c2, 0.3, d, ws)
    dgc.dgc_restrict_state(m.h, c2, c1)
    m.coarsen()
    dgc.dgc_restrict_state(m.h, c1, cc)
    m.coarsen()
    torch.cuda.synchronize()
    out = dgc.dgc_export_state(m.h, cc)
    e, _ = fp64_vs_exact(out - c0, ref - c0, refx - c0, 1e-11, "two-level cycle FP64")
    print(f"two levels: refine, refine, {steps} steps, coarsen, coarsen: du rel L2 {e:.2e}")
    dj = om.detj()
    np.testing.assert_allclose((dj[:, None] * out[:, :, 0]).sum(0), (dj[:, None] * c0[:, :, 0]).sum(0),
                               rtol=1e-12, atol=1e-13 * np.abs(c0[:, :, 0]).max())
    assert m.info["ncolors"] == 3 and m.info["ne"] == om.ne
    m.close()


def test_transfer_refusals(torch_dev):
    torch, dev = torch_dev
    m = dgc.Mesh.from_input(W.periodic_square_tri(8), 1)
    m.color(1)
    x = torch.zeros(m.state_shape(), dtype=torch.float64, device=dev)
    with pytest.raises(dgc.DgcError):
        dgc.dgc_prolong_state(m.h, x, x)
    with pytest.raises(dgc.DgcError):
        dgc.dgc_restrict_state(m.h, x, x)
    with pytest.raises(dgc.DgcError):
        dgc.dgc_refine_colors_device(m.h, m.info["ns"])
    m.close()
