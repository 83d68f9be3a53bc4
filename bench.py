#!/usr/bin/env python
"""Benchmark: DOF-RHS updates/s of the colored DG right-hand side on GB300.

One step = one SSP-RK3 step (CFL reduction + three right-hand sides with their
stage updates) of the 2D Euler modal DG scheme, p = 3, on the periodic
724x724 jittered square split into 1,048,352 triangles (41,934,080 scalar
DOFs), state = isentropic vortex + 1e-3 uniform perturbation.  The headline
path computes flux, quadrature and projection in FP32 and keeps the state and
stage update in FP64; FP64, the atomicAdd-scatter and the per-edge-buffer
comparators are timed beside it on the same GPU.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dgc|reference]

Under torchrun (N > 1) every rank advances its own replica of the workload
(weak scaling, no collective on the data path); the reported time is the
maximum over ranks.  ``--impl reference`` times the CPU oracle on the host
cores instead (rank 0 only).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1601_07613_gb300 import workloads as W  # noqa: E402

METRIC = "DOF-RHS updates/s, FP64 colored vs FP32-mixed/batched; % of HBM roofline"
UNIT = "DOF-RHS updates/s"
WORKLOAD = "2D Euler DG p=3 on 1,048,352 jittered periodic triangles (724x724), vortex + 1e-3 perturbation"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 peak derived from unit counts and clock: 152 SMs x 4 FP64 flop/clk/SM
# (2 DFMA/clk/SM, the GB300's FP64 rate) x 2.07 GHz; the roofline uses the
# measured figure (fp64_peak_tflops) and keeps this one beside it.
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12


def fp64_peak_tflops(torch, dev, n: int = 4096, reps: int = 3) -> float:
    """Measured FP64 rate of this GPU: a library FP64 GEMM (torch float64 matmul,
    cuBLAS DGEMM) of n^3, best of reps, CUDA events; 2 n^3 flops."""
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    best = float("inf")
    for _ in range(reps):
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        s.record()
        torch.matmul(a, b)
        e.record()
        torch.cuda.synchronize()
        best = min(best, s.elapsed_time(e))
    del a, b
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    def __init__(self, index: int):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def class_bytes(cls: str, E: int, nedges: int, NV: int, dim: int, form: str, rec: int = 0,
                first_est: bool = False) -> float:
    """Algorithmic DRAM bytes of one launch (one call for the two-pass CFL) of a
    kernel class, averaged over the three RK stages; each element is touched once
    per color on a closed conforming mesh.  form: "fp64", or "mixed" / "kahan"
    (the FP32 forms, increment form of the step); rec = bytes of an element's FP32
    record.  Per element, FP32 forms, last color: stage 0 reads the record and
    the partial rhs and writes the increment and the stage record (2 rec + 8 NV);
    stage 1 also reads rec0 and the increment (3 rec + 12 NV); stage 2 reads the
    record, rhs, increment and the state, writes the state (rec + 24 NV): on
    average (6 rec + 44 NV) / 3.  (The Kahan pair state of a triangle has the FP64
    state's size.)  first_est: the mixed triangle step whose first color of stage
    0 reads the FP64 state and writes the record of u0 and the CFL estimates (the
    work of CFL pass 1); the CFL class is then pass 2 alone, which reads the
    estimates."""
    f32 = form != "fp64"
    s_in = rec if f32 else 8 * NV      # state read for traces
    s_rhs = (4 if f32 else 8) * NV     # rhs element block
    edge = 16 + 16 * (2 if dim == 2 else 3)
    if cls == "first":
        if first_est:
            s_in = ((8 * NV + rec + 4) + 2 * rec) / 3
        return E * (s_in + 8 * dim * dim + s_rhs) + nedges * edge
    if cls == "color":
        return E * (s_in + 2 * s_rhs) + nedges * edge
    if cls == "last":
        per = (6 * rec + 44 * NV) / 3 if f32 else 8 * NV * (3 + 2.0 / 3.0)
        return E * per + nedges * edge
    if cls == "cfl":
        if first_est:
            return 4.0 * E
        return E * ((rec + 12) if form == "kahan" else (8 * NV + 12 + (rec if f32 else 0)))
    if cls == "volume":
        return E * (s_in + 8 * dim * dim + s_rhs)
    if cls == "stage":
        return E * ((4 * rec + 44 * NV) / 3 if f32 else 8 * NV * (3 + 2.0 / 3.0))
    return float("nan")


def flops_per_rhs(E, NV, nqv, nqe, nfaces=3):
    """FP arithmetic of one right-hand side (FMA = 2): per element the volume
    term (trace 2 NV, projection 4 NV, flux ~40 per point) and its share of
    the surface terms (trace + projection 4 NV, flux ~70 per point and side)."""
    return E * (nqv * (6 * NV + 40) + nfaces * nqe * (4 * NV + 70))


def setup_workload(dgc, torch, dev, n: int = 724):
    cfg = W.jittered_square_vortex_p3_724x724(n)
    mi, p = cfg["mesh"], cfg["p"]
    t0 = time.time()
    mesh = dgc.Mesh.from_input(mi, p)
    t1 = time.time()
    ncol, per = mesh.color(1601)
    t2 = time.time()
    xyz = dgc.dgc_vol_points(mesh.h)
    vals = W.vortex_field(xyz[..., 0], xyz[..., 1], beta=cfg["beta"], xc=cfg["xc"], yc=cfg["yc"])
    c = dgc.dgc_project(mesh.h, vals)
    c += W.uniform_perturbation(c.shape, cfg["perturb_seed"], cfg["perturb"])
    del xyz, vals
    prep = {"mesh_s": round(t1 - t0, 3), "color_reorder_s": round(t2 - t1, 3), "colors": ncol,
            "edges_per_color": per}
    return cfg, mi, mesh, c, prep


def time_steps(torch, fn, steps, stream):
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record(stream)
    for _ in range(steps):
        fn()
    e.record(stream)
    torch.cuda.synchronize()
    return s.elapsed_time(e) / steps


def kernel_source_hash() -> str:
    """Hash of the sources the triangle kernels are built from (their file, the
    shared device kernels and every device header, launch shapes included); the
    DRAM traffic quoted below holds only for the sources it was measured with.
    The host library, the mesh code and the other element types' kernels are
    not part of it."""
    import hashlib

    root = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1601_07613_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(root)):
        if name in ("kernels_tri.cu", "kernels_common.cu") or name.endswith((".cuh", ".h")):
            with open(os.path.join(root, name), "rb") as f:
                h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, averaged
# over the launches of each class as one step has them: the first color once
# with the FP64 state and twice with the record, the last color once per
# stage) from ncu captures of this benchmark's own command at full size with
# the tiles 64x2, 64x2, 32x4 (one kernel and two launches per capture), taken
# with the kernel sources of hash TRAFFIC_SOURCES.
TRAFFIC_SOURCES = "4a0049ffaf80ecb9"
TRAFFIC_BYTES = {"last": 1123873706, "first": 480706858, "color": 592563712, "cfl": 4220672}


def fp64_roofline(flops: float, ms: float, p64: float) -> dict:
    """The FP64 form against the FP64 pipe.  flops = Eq. 2's floating-point
    operations as a term-by-term FP64 evaluation does them; on triangle meshes
    the basis contractions among them run as FP32 pairs on the FP32 pipe, so the
    effective rate can exceed the FP64 pipe's peak: reported as such (frac = null)."""
    eff = flops / (ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": None, "peak": round(p64, 3), "unit": "TFLOP/s",
            "peak_source": "measured in this run: cuBLAS DGEMM 4096^3 (torch)", "frac": None,
            "effective_fp64_equivalent": round(eff, 3), "effective_vs_fp64_peak": round(eff / p64, 3),
            "derived_peak": round(FP64_PEAK_TFLOPS, 3),
            "note": "Eq. 2's FP64 flop count over the step time; the basis contractions run as FP32 pairs on the "
                    "FP32 pipe (fluxes, geometry and the stage update on the FP64 pipe), so no fraction of the "
                    "FP64 peak is claimed"}


def replica_throughput(torch, ms: float, world: int, units_per_step: float, dev):
    """Replicas only: every rank runs the whole workload; the job's time per step
    is the slowest rank's (all-reduce MAX), and the throughput counts the units
    of all ranks.  Returns (ms per step, units per second)."""
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * units_per_step / (ms * 1e-3)


def run_dgc(args, rank, world, local_rank):
    import torch

    from paper_1601_07613_gb300 import dgc

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dgc.lib()
    cfg, mi, mesh, c_host, prep = setup_workload(dgc, torch, dev, args.n)
    if args.epb:
        dgc.dgc_set_option(mesh.h, dgc.DGC_OPT_EDGES_PER_BLOCK, args.epb)
    if args.tpe:
        dgc.dgc_set_option(mesh.h, dgc.DGC_OPT_THREADS_PER_EDGE, args.tpe)
    if args.no_pdl:
        dgc.dgc_set_option(mesh.h, dgc.DGC_OPT_PDL, 0)
    info = mesh.info
    E, NV, p = info["ne"], info["M"] * info["np"], info["p"]
    dofs = E * NV
    stream = torch.cuda.current_stream()
    c = torch.empty(mesh.state_shape(), dtype=torch.float64, device=dev)
    dt = torch.zeros(1, dtype=torch.float64, device=dev)
    mixed, fp64 = dgc.DGC_FP32_MIXED, dgc.DGC_FP64
    wsb = max(dgc.dgc_workspace_size(mesh.h, fp64), dgc.dgc_workspace_size(mesh.h, mixed))
    ws = torch.empty(wsb // 8 + 64, dtype=torch.float64, device=dev)
    dgc.dgc_import_state(mesh.h, c_host, c)

    def step(prec):
        dgc.dgc_rk_step(mesh.h, prec, c, cfg["cfl"], dt, ws)

    # ---- tiles: the library's autotuner (edges per block x threads per edge of the
    # first, middle and last colors) on a scratch copy of the state, untimed
    tiles = None
    if args.tiles:
        for kc, t in zip((dgc.DGC_K_FIRST, dgc.DGC_K_COLOR, dgc.DGC_K_LAST), args.tiles.split(",")):
            e, tp = (int(v) for v in t.split("x"))
            dgc.dgc_set_tile(mesh.h, kc, e, tp)
    if not (args.no_autotune or args.epb or args.tpe or args.tiles):
        scratch = torch.empty_like(c)
        dgc.dgc_import_state(mesh.h, c_host, scratch)
        tiles, tune_ms = dgc.dgc_autotune(mesh.h, mixed, scratch, cfg["cfl"], dt, ws, reps=3)
        del scratch
    else:
        tiles = {k: dgc.dgc_get_tile(mesh.h, kc) for k, kc in (("first", dgc.DGC_K_FIRST),
                                                                ("color", dgc.DGC_K_COLOR), ("last", dgc.DGC_K_LAST))}

    # ---- headline: FP32-mixed RK step -------------------------------------------------
    for _ in range(args.warmup):
        step(mixed)
    launches_per_step = dgc.dgc_last_launch_count(mesh.h)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local_rank)
    ms = time_steps(torch, lambda: step(mixed), args.steps, stream)
    clocks = clk.stop()
    # Per-kernel durations: the same number of steps again with a CUDA event pair
    # around every launch.  The events order the launches strictly, so the
    # kernels of this pass do not overlap (programmatic dependent launch) and
    # the pass takes a little longer than the headline's.
    dgc.dgc_set_option(mesh.h, dgc.DGC_OPT_PROFILE, 1)
    dgc.dgc_profile_collect(mesh.h)
    ms_prof = time_steps(torch, lambda: step(mixed), args.steps, stream)
    prof = dgc.dgc_profile_collect(mesh.h)
    dgc.dgc_set_option(mesh.h, dgc.DGC_OPT_PROFILE, 0)
    ms, value = replica_throughput(torch, ms, world, 3 * dofs, dev)

    hbm, hbm_kind = peaks()
    ncolors = info["ncolors"]
    per_color = prep["edges_per_color"]
    kernels = {}
    # the mixed step's first color of stage 0 does CFL pass 1; the CFL class is pass 2
    kernels_per_call = {"cfl": 1}
    for cls, (tms, nl) in prof.items():
        n = nl // kernels_per_call.get(cls, 1)
        if cls == "first":
            ne_ = per_color[0]
        elif cls == "last":
            ne_ = per_color[-1]
        elif cls == "color":
            ne_ = sum(per_color[1:-1]) / max(1, ncolors - 2)
        else:
            ne_ = 0
        b = class_bytes(cls, E, ne_, NV, 2, "mixed", rec=4 * info["M"] * (info["np"] + 1), first_est=True)
        avg = tms / n
        kernels[cls] = {"launches": nl, "calls": n, "avg_ms": round(avg, 5), "share": round(tms / (ms_prof * args.steps), 4),
                        "alg_bytes": int(b), "alg_gbs": round(b / (avg * 1e-3) / 1e9, 1),
                        "frac_hbm": round(b / (avg * 1e-3) / 1e9 / hbm, 3)}
    dom = max(kernels, key=lambda k: kernels[k]["avg_ms"] * kernels[k]["calls"])
    step_bytes = sum(kernels[k]["alg_bytes"] * kernels[k]["calls"] for k in kernels) / args.steps
    measured = TRAFFIC_SOURCES == kernel_source_hash() and args.n == 724
    traffic = TRAFFIC_BYTES.get(dom) if measured else None
    if measured:
        # the same kernels by the DRAM bytes ncu measured per launch (launch list in profiles/)
        for k, kv in kernels.items():
            if k in TRAFFIC_BYTES:
                g = TRAFFIC_BYTES[k] / (kv["avg_ms"] * 1e-3) / 1e9
                kv["dram_gbs"] = round(g, 1)
                kv["dram_frac_hbm"] = round(g / hbm, 3)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": kernels[dom]["alg_gbs"], "peak": hbm,
                "unit": "GB/s", "frac": kernels[dom]["frac_hbm"], "traffic": traffic,
                "dram_frac": kernels[dom].get("dram_frac_hbm"),
                "peak_source": f"{hbm_kind} (MEASURED_PEAKS.json hbm_gbs)" if hbm_kind == "measured" else "fallback",
                "profiled_ms_per_step": round(ms_prof, 5),
                "step_alg_gbs": round(step_bytes / (ms * 1e-3) / 1e9, 1),
                "step_frac": round(step_bytes / (ms * 1e-3) / 1e9 / hbm, 3)}
    # the paper-structure model of one RHS with an FP32 state block S: volume pass,
    # then per edge read both neighbours and read-modify-write both rhs blocks,
    # (2 + 3F) S + 40 + (F/2) 48 bytes per element (F = 3 edges); timed as the
    # RK step / 3, which also carries the CFL pass and the stage updates
    S32 = 4 * NV
    pm_bytes = E * ((2 + 3 * 3) * S32 + 40 + 1.5 * 48)
    t_rhs = ms / 3.0
    roofline["paper_structure"] = {"bytes_per_rhs": int(pm_bytes), "t_rhs_ms": round(t_rhs, 4),
                                   "gbs": round(pm_bytes / (t_rhs * 1e-3) / 1e9, 1),
                                   "frac": round(pm_bytes / (t_rhs * 1e-3) / 1e9 / hbm, 3)}
    # the same two figures as plain keys beside frac (the whole step's measure)
    roofline["paper_structure_gbs"] = roofline["paper_structure"]["gbs"]
    roofline["paper_structure_frac"] = roofline["paper_structure"]["frac"]

    variants = {}
    if not args.no_variants:
        # ---- FP64 colored RK step (FP64-ALU bound on this GPU) ------------------------
        dgc.dgc_import_state(mesh.h, c_host, c)
        step(fp64)
        k64 = max(3, args.steps // 5)
        ms64 = time_steps(torch, lambda: step(fp64), k64, stream)
        fl = 3 * flops_per_rhs(E, NV, info["nqv"], info["nqf"])
        # the headline step in plain stream order (no programmatic dependent launch)
        dgc.dgc_import_state(mesh.h, c_host, c)
        dgc.dgc_set_option(mesh.h, dgc.DGC_OPT_PDL, 0)
        step(mixed)
        ms_plain = time_steps(torch, lambda: step(mixed), args.steps, stream)
        dgc.dgc_set_option(mesh.h, dgc.DGC_OPT_PDL, 0 if args.no_pdl else 1)
        variants["rk_fp32mixed_plain_launch"] = {"value": 3 * dofs / (ms_plain * 1e-3), "ms_per_step": round(ms_plain, 4)}
        p64 = fp64_peak_tflops(torch, dev)
        variants["rk_fp64"] = {"value": 3 * dofs / (ms64 * 1e-3), "ms_per_step": round(ms64, 4),
                               "roofline": fp64_roofline(fl, ms64, p64)}
        # ---- Kahan form: FP32 pair state, compensated update --------------------------
        kst = torch.empty(dgc.dgc_state_bytes(mesh.h, dgc.DGC_FP32_KAHAN) // 4, dtype=torch.float32, device=dev)
        wsk = torch.empty(dgc.dgc_workspace_size(mesh.h, dgc.DGC_FP32_KAHAN) // 8 + 64, dtype=torch.float64,
                          device=dev)
        dgc.dgc_import_state_prec(mesh.h, dgc.DGC_FP32_KAHAN, c_host, kst)
        stepk = lambda: dgc.dgc_rk_step(mesh.h, dgc.DGC_FP32_KAHAN, kst, cfg["cfl"], dt, wsk)
        stepk()
        msk = time_steps(torch, stepk, max(3, args.steps), stream)
        variants["rk_fp32kahan"] = {"value": 3 * dofs / (msk * 1e-3), "ms_per_step": round(msk, 4)}
        del wsk
        # ---- right-hand side alone: colored vs atomicAdd vs two-pass buffer ----------
        r = torch.empty_like(c)
        nbuf = dgc.dgc_two_pass_buffer_bytes(info["ns"], info["np"], info["M"], 8)
        buf = torch.empty(nbuf // 8, dtype=torch.float64, device=dev)
        dgc.dgc_import_state(mesh.h, c_host, c)
        reps = max(5, args.steps)
        for prec, tag in ((mixed, "fp32mixed"), (fp64, "fp64")):
            rr = reps if prec == mixed else max(3, reps // 5)
            calls = {
                "colored": lambda: dgc.dgc_rhs(mesh.h, prec, c, r),
                "atomic": lambda: dgc.dgc_rhs_atomic(mesh.h, prec, c, r),
                "two_pass": lambda: dgc.dgc_rhs_two_pass(mesh.h, prec, c, r, buf),
            }
            for name, fn in calls.items():
                fn()
                t_ = time_steps(torch, fn, rr, stream)
                variants[f"rhs_{name}_{tag}"] = {"value": dofs / (t_ * 1e-3), "ms_per_rhs": round(t_, 4)}
            dgc.dgc_set_option(mesh.h, dgc.DGC_OPT_FUSE, 0)
            fn = calls["colored"]
            fn()
            t_ = time_steps(torch, fn, rr, stream)
            variants[f"rhs_colored_unfused_{tag}"] = {"value": dofs / (t_ * 1e-3), "ms_per_rhs": round(t_, 4)}
            dgc.dgc_set_option(mesh.h, dgc.DGC_OPT_FUSE, 1)
        variants["two_pass_buffer_bytes"] = nbuf
        del buf, r
        variants.update(run_batched(dgc, torch, dev, stream, args))
        variants.update(run_other_meshes(dgc, torch, dev, stream, args))
        variants["nonconforming_two_level_p2_256"] = run_two_level(dgc, torch, dev, stream, args)
        variants.update(run_table7(dgc, torch, dev, stream, args, cfg, c_host))
        variants.update(run_double_mach(dgc, torch, dev, stream, args))
        variants["coloring_tables"] = run_coloring_tables(dgc)

    # ---- end to end through the C ABI with pinned host buffers -----------------------------
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(dgc, torch, dev, mesh, c_host, cfg, dofs, args)

    workload = WORKLOAD if args.n == 724 else f"2D Euler DG p=3 on {E} jittered periodic triangles ({args.n}x{args.n})"
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (flux/quadrature/projection; f64 state, stage update, CFL)",
        "data": "synthetic",
        "config": {"workload": workload, "elements": E, "edges": info["ns"], "p": p, "Np": info["np"],
                   "M": info["M"], "edge_points": info["nqf"], "area_points": info["nqv"],
                   "dofs": dofs, "step": "SSP-RK3 (3 RHS) with FP64 CFL reduction",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "no flush: state 335 MB FP64 + 168 MB FP32 copy per replica exceed the 129 MB L2",
                   "host_prep": prep,
                   "tiles": {k: {"edges_per_block": v[0], "threads_per_edge": v[1]} for k, v in tiles.items()}},
        "roofline": roofline, "kernels": kernels, "gpu_launches": int(launches_per_step * args.steps),
        "clocks": clocks, "e2e": e2e, "variants": variants,
    }
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(mi, p, c_host, dofs)
    mesh.close()
    return out


def run_e2e(dgc, torch, dev, mesh, c_host, cfg, dofs, args):
    """End to end through the C ABI: every step takes its input state from
    page-locked host memory and returns its result there (import, mixed RK
    step, export).  Steps of independent states (an ensemble, as a serving loop
    would see) run three at a time on rotating streams with their own buffers,
    so one state's upload, another's step and a third's download overlap (the
    host link moves ~210 GB/s each way, ~340 GB/s both ways at once, so the
    copies of one step take about as long as its kernels); the synchronous
    sequence (one step at a time, blocking calls) is reported beside it."""
    mixed = dgc.DGC_FP32_MIXED
    nb = 3
    shape = c_host.shape
    streams = [torch.cuda.Stream() for _ in range(nb)]
    host_in, host_out = [], []
    for _ in range(nb):
        hi = torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
        hi[...] = c_host
        host_in.append(hi)
        host_out.append(torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy())
    cd = [torch.empty(shape, dtype=torch.float64, device=dev) for _ in range(nb)]
    xf = [torch.empty(shape, dtype=torch.float64, device=dev) for _ in range(nb)]
    wsb = dgc.dgc_workspace_size(mesh.h, mixed)
    ws = [torch.empty(wsb // 8 + 64, dtype=torch.float64, device=dev) for _ in range(nb)]
    dts = [torch.zeros(1, dtype=torch.float64, device=dev) for _ in range(nb)]

    def one(i):
        b = i % nb
        s = streams[b].cuda_stream
        dgc.dgc_import_state_async(mesh.h, host_in[b], cd[b], xf[b], s)
        dgc.dgc_rk_step(mesh.h, mixed, cd[b], cfg["cfl"], dts[b], ws[b], stream=s)
        dgc.dgc_export_state_async(mesh.h, cd[b], host_out[b], xf[b], s)

    k = max(4, args.steps)
    for i in range(nb * 2):
        one(i)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(k):
        one(i)
    torch.cuda.synchronize()
    te = (time.perf_counter() - t0) / k
    # one step at a time through the blocking calls
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        dgc.dgc_import_state(mesh.h, host_in[0], cd[0])
        dgc.dgc_rk_step(mesh.h, mixed, cd[0], cfg["cfl"], dts[0], ws[0])
        dgc.dgc_export_state(mesh.h, cd[0], host_out[0])
    torch.cuda.synchronize()
    ts = (time.perf_counter() - t0) / 3
    nbytes = int(host_in[0].nbytes)
    return {"value": 3 * dofs / te, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "ms_per_step": round(te * 1e3, 3), "pipeline": f"{nb} independent states in flight on {nb} streams",
            "sync_ms_per_step": round(ts * 1e3, 3), "sync_value": 3 * dofs / ts}


def run_batched(dgc, torch, dev, stream, args):
    """64 independent periodic meshes, element counts log-uniform on [1e3, 2e5],
    p uniform in {1, 2, 3}, random vortices: one persistent launch per kernel class
    and stage over all meshes, replayed from a CUDA graph, tile size autotuned."""
    specs = W.batched_square_meshes()
    meshes, states = [], []
    for i, s in enumerate(specs):
        m = dgc.Mesh.from_input(W.periodic_square_tri(s["n"], jitter=0.2, seed=500 + i), s["p"])
        m.color(1601 + i)
        xyz = dgc.dgc_vol_points(m.h)
        c = dgc.dgc_project(m.h, W.vortex_field(xyz[..., 0], xyz[..., 1], beta=s["beta"], xc=s["xc"], yc=s["yc"]))
        meshes.append(m)
        states.append(c)
    dofs = sum(m.info["ne"] * m.info["M"] * m.info["np"] for m in meshes)
    cdev = [torch.empty(m.state_shape(), dtype=torch.float64, device=dev) for m in meshes]
    for m, c, d in zip(meshes, states, cdev):
        dgc.dgc_import_state(m.h, c, d)
    batch = dgc.dgc_batch_create(meshes)
    out = {}
    try:
        for prec, tag in ((dgc.DGC_FP32_MIXED, "fp32mixed"), (dgc.DGC_FP64, "fp64")):
            ws = torch.empty(dgc.dgc_batch_workspace_size(batch, prec) // 8 + 64, dtype=torch.float64, device=dev)
            dts = torch.zeros(len(meshes), dtype=torch.float64, device=dev)
            if args.tiles:  # fixed tiles (a profiler's command), else the autotuner's
                for kc, t in zip((dgc.DGC_K_FIRST, dgc.DGC_K_COLOR, dgc.DGC_K_LAST), args.tiles.split(",")):
                    e, tp = (int(v) for v in t.split("x"))
                    dgc.dgc_batch_set_tile(batch, kc, e, tp if tag == "fp32mixed" else 2)
                tiles_b = {k: (int(t.split("x")[0]), int(t.split("x")[1]) if tag == "fp32mixed" else 2)
                           for k, t in zip(("first", "color", "last"), args.tiles.split(","))}
                tune_ms = None
            else:
                tiles_b, tune_ms = dgc.dgc_batch_autotune(batch, prec, cdev, 0.3, dts, ws,
                                                          reps=3 if tag == "fp32mixed" else 1)
            k = max(3, args.steps) if tag == "fp32mixed" else 3
            ms = time_steps(torch, lambda: dgc.dgc_batch_rk_step(batch, prec, cdev, 0.3, dts, ws), k, stream)
            out[f"batched_{tag}"] = {
                "value": 3 * dofs / (ms * 1e-3), "ms_per_step": round(ms, 4), "meshes": len(meshes),
                "elements": sum(m.info["ne"] for m in meshes), "dofs": dofs,
                "launches_per_step": dgc.dgc_batch_launch_count(batch), "graph": True,
                "tiles": {k: {"edges_per_block": v[0], "threads_per_edge": v[1]} for k, v in tiles_b.items()},
                "autotune_best_ms": round(tune_ms, 4) if tune_ms is not None else None}
            hbm, _ = peaks()
            infos = [m.info for m in meshes]
            if tag == "fp32mixed":
                # whole step against the paper-structure model, and per kernel class from
                # a profiled pass (event pairs around every launch, graph off)
                pm = sum(i["ne"] * ((2 + 3 * 3) * 4 * i["M"] * i["np"] + 40 + 1.5 * 48) for i in infos)
                out[f"batched_{tag}"]["paper_structure"] = {
                    "bytes_per_rhs": int(pm), "gbs": round(pm / (ms / 3 * 1e-3) / 1e9, 1),
                    "frac": round(pm / (ms / 3 * 1e-3) / 1e9 / hbm, 3)}
                dgc.dgc_batch_set_option(batch, dgc.DGC_OPT_PROFILE, 1)
                dgc.dgc_batch_profile_collect(batch)
                msp = time_steps(torch, lambda: dgc.dgc_batch_rk_step(batch, prec, cdev, 0.3, dts, ws), k, stream)
                prof = dgc.dgc_batch_profile_collect(batch)
                dgc.dgc_batch_set_option(batch, dgc.DGC_OPT_PROFILE, 0)
                kern = {}
                for cls, (tms, nl) in prof.items():
                    calls = nl // k if cls == "cfl" else nl
                    b = 0.0
                    for i in infos:
                        nv, rec = i["M"] * i["np"], 4 * i["M"] * (i["np"] + 1)
                        b += class_bytes(cls, i["ne"], i["ne"] // 2, nv, 2, "mixed", rec=rec)
                    avg = tms / (k if cls == "cfl" else calls)  # the CFL class: both passes and the reset, per step
                    kern[cls] = {"launches_per_step": nl // k, "avg_ms": round(avg, 5),
                                 "share": round(tms / (msp * k), 4), "alg_bytes": int(b),
                                 "alg_gbs": round(b / (avg * 1e-3) / 1e9, 1),
                                 "frac_hbm": round(b / (avg * 1e-3) / 1e9 / hbm, 3)}
                out[f"batched_{tag}"]["profiled_ms_per_step"] = round(msp, 4)
                out[f"batched_{tag}"]["kernels"] = kern
            else:
                fl = 3 * sum(flops_per_rhs(i["ne"], i["M"] * i["np"], i["nqv"], i["nqf"]) for i in infos)
                p64 = fp64_peak_tflops(torch, dev)
                out[f"batched_{tag}"]["roofline"] = fp64_roofline(fl, ms, p64)
            del ws
    finally:
        dgc.dgc_batch_destroy(batch)
        for m in meshes:
            m.close()
    return out


def run_other_meshes(dgc, torch, dev, stream, args, only=None):
    """The other workloads, each an RK step in FP64 and in mixed precision, and
    its right-hand side colored / atomicAdd / two-pass:
    1,572,864 periodic Kuhn tetrahedra at p = 2 (4 face colors; seeded random
    state),
    the 256 x 256 x 2 periodic triangle mesh refined once within radius 0.2 of the
    centre (180,512 elements, hanging edges, 6 colors) at p = 2, and
    656,100 periodic parallelograms (810 x 810, 4 edge colors) at p = 3, the
    hybrid 512 x 512 grid with 30 % of its cells split into triangles at p = 3,
    and 262,144 general (bilinear) quadrilaterals (512 x 512, every vertex
    jittered) at p = 3, the last two through the table-driven kernels.
    On the tetrahedra and the parallelograms the mixed step also gets a per-kernel
    breakdown from a profiled pass against the HBM roofline."""
    out = {}
    tube = W.cube_tube_p2_64()
    ref = W.refined_square_vortex_p2_256()
    quad = W.quad_square_vortex_p3_810()
    hyb = W.hybrid_square_vortex_p3_512()
    bil = W.bilinear_square_vortex_p3_512()
    hbm, _ = peaks()
    for tag, mi, p, refine in (("tet_p2_64cube", tube["mesh"], tube["p"], None),
                               ("nonconforming_p2_256", ref["mesh"], ref["p"], ref["refine"]),
                               ("quad_p3_810", quad["mesh"], quad["p"], None),
                               ("hybrid_p3_512", hyb["mesh"], hyb["p"], None),
                               ("bilinear_p3_512", bil["mesh"], bil["p"], None)):
        if only is not None and not tag.startswith(only):
            continue
        t0 = time.perf_counter()
        m = dgc.Mesh.from_input(mi, p)
        _, per_color = m.color(1601)
        if refine is not None:
            m.refine(refine)
        prep_s = time.perf_counter() - t0
        if args.epb:
            dgc.dgc_set_option(m.h, dgc.DGC_OPT_EDGES_PER_BLOCK, args.epb)
        info = m.info
        if mi.dim == 3:
            # seeded mean state + perturbed modes (projecting the tube at 100M
            # volume points costs minutes of host time; the kernels' work does not
            # depend on the field)
            c_host = W.random_state(info["ne"], 5, info["np"], seed=7, amp=3e-3, mean=(0.7, 0.1, -0.05, 0.03, 1.8))
        else:
            xyz = dgc.dgc_vol_points(m.h)
            c_host = dgc.dgc_project(m.h, W.vortex_field(xyz[..., 0], xyz[..., 1], beta=5.0))
        dofs = info["ne"] * info["M"] * info["np"]
        c = torch.empty(m.state_shape(), dtype=torch.float64, device=dev)
        r = torch.empty_like(c)
        dt = torch.zeros(1, dtype=torch.float64, device=dev)
        entry = {"elements": info["ne"], "faces": info["ns"], "p": p, "dofs": dofs, "colors": info["ncolors"],
                 "host_mesh_color_s": round(prep_s, 2)}
        # (hybrid meshes and general quadrilaterals: the table-driven kernels, FP64 and FP32-mixed)
        hybrid = tag.startswith(("hybrid", "bilinear"))
        for prec, name in ((dgc.DGC_FP32_MIXED, "fp32mixed"), (dgc.DGC_FP64, "fp64")):
            ws = torch.empty(dgc.dgc_workspace_size(m.h, prec) // 8 + 64, dtype=torch.float64, device=dev)
            dgc.dgc_import_state(m.h, c_host, c)
            fn = lambda: dgc.dgc_rk_step(m.h, prec, c, 0.3, dt, ws)
            fn()
            k = max(3, args.steps // (1 if prec == dgc.DGC_FP32_MIXED else 5))
            ms = time_steps(torch, fn, k, stream)
            entry[f"rk_{name}"] = {"value": 3 * dofs / (ms * 1e-3), "ms_per_step": round(ms, 4),
                                   "launches_per_step": dgc.dgc_last_launch_count(m.h)}
            if prec == dgc.DGC_FP32_MIXED and refine is None and not hybrid:
                dgc.dgc_set_option(m.h, dgc.DGC_OPT_PROFILE, 1)
                dgc.dgc_profile_collect(m.h)
                msp = time_steps(torch, fn, k, stream)
                prof = dgc.dgc_profile_collect(m.h)
                dgc.dgc_set_option(m.h, dgc.DGC_OPT_PROFILE, 0)
                rec = 4 * ((info["M"] * (info["np"] + 1) + 3) // 4 * 4)
                kern = {}
                for cls, (tms, nl) in prof.items():
                    n = nl // (2 if cls == "cfl" else 1)
                    ne_ = per_color[0] if cls in ("first", "color", "last") else 0
                    b = class_bytes(cls, info["ne"], ne_, info["M"] * info["np"], mi.dim, "mixed", rec=rec)
                    avg = tms / n
                    kern[cls] = {"calls": n, "avg_ms": round(avg, 5), "share": round(tms / (msp * k), 4),
                                 "alg_bytes": int(b), "alg_gbs": round(b / (avg * 1e-3) / 1e9, 1),
                                 "frac_hbm": round(b / (avg * 1e-3) / 1e9 / hbm, 3)}
                entry["rk_fp32mixed"]["profiled_ms_per_step"] = round(msp, 4)
                entry["rk_fp32mixed"]["kernels"] = kern
            del ws
            nbuf = dgc.dgc_two_pass_buffer_bytes(info["ns"], info["np"], info["M"], 8)
            buf = torch.empty(nbuf // 8, dtype=torch.float64, device=dev)
            dgc.dgc_import_state(m.h, c_host, c)
            forms = [("colored", lambda: dgc.dgc_rhs(m.h, prec, c, r)),
                     ("atomic", lambda: dgc.dgc_rhs_atomic(m.h, prec, c, r))]
            if not hybrid:
                forms.append(("two_pass", lambda: dgc.dgc_rhs_two_pass(m.h, prec, c, r, buf)))
            for kind, call in forms:
                call()
                t_ = time_steps(torch, call, max(3, args.steps // 5), stream)
                entry[f"rhs_{kind}_{name}"] = {"value": dofs / (t_ * 1e-3), "ms_per_rhs": round(t_, 4)}
            if mi.dim == 2 and not m.elem == dgc.DGC_QUAD:
                # the colored right-hand side as one cooperative launch (grid barriers between colors)
                dgc.dgc_set_option(m.h, dgc.DGC_OPT_COOPERATIVE, 1)
                call = lambda: dgc.dgc_rhs(m.h, prec, c, r)
                call()
                t_ = time_steps(torch, call, max(3, args.steps // 5), stream)
                entry[f"rhs_colored_coop_{name}"] = {"value": dofs / (t_ * 1e-3), "ms_per_rhs": round(t_, 4)}
                dgc.dgc_set_option(m.h, dgc.DGC_OPT_COOPERATIVE, 0)
                # one wave of blocks per color, grid-stride
                dgc.dgc_set_option(m.h, dgc.DGC_OPT_PERSISTENT, 1)
                call()
                t_ = time_steps(torch, call, max(3, args.steps // 5), stream)
                entry[f"rhs_colored_persistent_{name}"] = {"value": dofs / (t_ * 1e-3), "ms_per_rhs": round(t_, 4)}
                # back to the library's default: persistent on refined meshes, else off
                dgc.dgc_set_option(m.h, dgc.DGC_OPT_PERSISTENT, int(refine is not None))
            dgc.dgc_set_option(m.h, dgc.DGC_OPT_FUSE, 0)
            call = lambda: dgc.dgc_rhs(m.h, prec, c, r)
            call()
            t_ = time_steps(torch, call, max(3, args.steps // 5), stream)
            entry[f"rhs_colored_unfused_{name}"] = {"value": dofs / (t_ * 1e-3), "ms_per_rhs": round(t_, 4)}
            dgc.dgc_set_option(m.h, dgc.DGC_OPT_FUSE, 1)
            del buf
        if refine is not None:
            # dynamic adaptivity on the device: the Sec. 3.2 color map of the refined
            # sides, and the state moved to and from the mesh before refinement
            _, map_ms = dgc.dgc_refine_colors_device(m.h, info["ns"])
            ne0 = mi.ne
            cc = torch.zeros((ne0, info["M"], info["np"]), dtype=torch.float64, device=dev)
            pro = lambda: dgc.dgc_prolong_state(m.h, cc, c)
            res = lambda: dgc.dgc_restrict_state(m.h, c, cc)
            pro()
            res()
            entry["adapt"] = {"host_refine_s": round(prep_s, 4), "device_color_map_ms": round(map_ms, 4),
                              "prolong_ms": round(time_steps(torch, pro, 10, stream), 4),
                              "restrict_ms": round(time_steps(torch, res, 10, stream), 4)}
            del cc
        out[tag] = entry
        del c, r
        m.close()
    return out


def run_two_level(dgc, torch, dev, stream, args) -> dict:
    """The nonconforming workload refined a second time (the palette doubled
    again, 12 colors): the 256 x 256 x 2 mesh refined within radius 0.2 of the
    vortex centre, then its children within 0.1 and the coarse elements beside
    hanging halves right of the centre within 0.23 refined again; p = 2.  The
    mixed and FP64 RK steps, the colored right-hand side, and the device color
    map of the second level."""
    ref = W.refined_square_vortex_p2_256()
    mi, p = ref["mesh"], ref["p"]
    t0 = time.perf_counter()
    m = dgc.Mesh.from_input(mi, p)
    m.color(1601)
    m.refine(ref["refine"])
    l, r, _, _ = dgc.dgc_get_sides(m.h)
    _, xyz = dgc.dgc_get_elements(m.h)
    e2 = W.second_level_elements(ref["refine"], mi.ne, l, r, dgc.dgc_get_hanging(m.h), xyz, (0.5, 0.5), 0.1, 0.23)
    m.refine(e2)
    prep_s = time.perf_counter() - t0
    info = m.info
    xyzv = dgc.dgc_vol_points(m.h)
    c_host = dgc.dgc_project(m.h, W.vortex_field(xyzv[..., 0], xyzv[..., 1], beta=ref["beta"]))
    dofs = info["ne"] * info["M"] * info["np"]
    _, map_ms = dgc.dgc_refine_colors_device(m.h, info["ns"])
    off = dgc.dgc_get_ordering(m.h)[3]
    entry = {"elements": info["ne"], "sides": info["ns"], "colors": info["ncolors"], "p": p,
             "second_level_parents": int(len(e2)), "per_color": np.diff(off).tolist(),
             "host_refine_s": round(prep_s, 3), "device_color_map_ms": round(map_ms, 4)}
    c = torch.empty(m.state_shape(), dtype=torch.float64, device=dev)
    rr = torch.empty_like(c)
    dt = torch.zeros(1, dtype=torch.float64, device=dev)
    for prec, name in ((dgc.DGC_FP32_MIXED, "fp32mixed"), (dgc.DGC_FP64, "fp64")):
        ws = torch.empty(dgc.dgc_workspace_size(m.h, prec) // 8 + 64, dtype=torch.float64, device=dev)
        dgc.dgc_import_state(m.h, c_host, c)
        fn = lambda: dgc.dgc_rk_step(m.h, prec, c, ref["cfl"], dt, ws)
        fn()
        ms = time_steps(torch, fn, max(3, args.steps // (1 if prec == dgc.DGC_FP32_MIXED else 5)), stream)
        entry[f"rk_{name}"] = {"value": 3 * dofs / (ms * 1e-3), "ms_per_step": round(ms, 4),
                               "launches_per_step": dgc.dgc_last_launch_count(m.h)}
        call = lambda: dgc.dgc_rhs(m.h, prec, c, rr)
        call()
        t_ = time_steps(torch, call, max(3, args.steps // 5), stream)
        entry[f"rhs_colored_{name}"] = {"value": dofs / (t_ * 1e-3), "ms_per_rhs": round(t_, 4)}
        del ws
    m.close()
    return entry


def run_coloring_tables(dgc) -> list:
    """Tables 1-3's kind of statistics on this library (host only): triangle,
    quadrilateral and tetrahedral meshes of growing size (each about 4x the last,
    as the rectangle meshes A-E; tetrahedra 8x) and hybrid triangle/quadrilateral
    meshes; edges (faces) per color, the greedy pass and conflict resolution with
    the reordering, in seconds."""
    rows = []
    for kind, n in (("tri", 64), ("tri", 128), ("tri", 256), ("tri", 512),
                    ("quad", 32), ("quad", 64), ("quad", 128), ("quad", 256), ("quad", 512),
                    ("hybrid", 40), ("hybrid", 160), ("tet", 8), ("tet", 16), ("tet", 32)):
        mi = {"tri": lambda: W.open_square_tri(n, jitter=0.2, seed=n),
              "quad": lambda: W.open_square_quad(n, "vertex", jitter=0.2, seed=n),
              "hybrid": lambda: W.hybrid_square(n, 0.3, periodic=False, jitter=0.2, seed=n),
              "tet": lambda: W.periodic_cube_tet(n)}[kind]()
        m = dgc.Mesh.from_input(mi, 1)
        t0 = time.perf_counter()
        nc, per = m.color(1601)
        rows.append({"mesh": kind, "elements": m.info["ne"], "sides": m.info["ns"], "colors": nc,
                     "per_color": per, "coloring_s": round(time.perf_counter() - t0, 4)})
        m.close()
    return rows


def run_table7(dgc, torch, dev, stream, args, cfg, c_base):
    """Color count and data ordering on GB300 (the ablation of Table 7): the
    naive greedy (5 colors) or the modified coloring (3), with and without the
    color-1 element renumbering and the left-ascending edge order of Sec. 5.
    The mesh is the benchmark's with its element list in a seeded random order,
    standing in for a mesh generator's unstructured numbering (on the grid's own
    order the naive greedy already finds 3 colors).  Each row times the mixed RK
    step and the FP64 right-hand side; pct = speed-up over the first row."""
    mi = cfg["mesh"]
    perm = np.random.default_rng(1601).permutation(mi.ne)
    m = dgc.Mesh(2, cfg["p"], mi.xyz, mi.ev[perm], mi.periodic_len)
    c_host = np.ascontiguousarray(c_base[perm])  # the same elements (same vertex lists), permuted
    info = m.info
    dofs = info["ne"] * info["M"] * info["np"]
    c = torch.empty((info["ne"], info["M"], info["np"]), dtype=torch.float64, device=dev)
    r = torch.empty_like(c)
    dt = torch.zeros(1, dtype=torch.float64, device=dev)
    rows = []
    for colors, renumber, reorder in ((5, False, False), (3, False, False), (5, True, False), (3, True, False),
                                      (5, True, True), (3, True, True)):
        if colors == 5:
            nc, _ = dgc.dgc_color_edges_naive(m.h, renumber, reorder)
        else:
            nc, _ = dgc.dgc_color_edges(m.h, 1601, 0)
            dgc.dgc_reorder(m.h, renumber, reorder)
        ws = torch.empty(dgc.dgc_workspace_size(m.h, dgc.DGC_FP32_MIXED) // 8 + 64, dtype=torch.float64, device=dev)
        dgc.dgc_import_state(m.h, c_host, c)
        fn = lambda: dgc.dgc_rk_step(m.h, dgc.DGC_FP32_MIXED, c, cfg["cfl"], dt, ws)
        fn()
        t_rk = time_steps(torch, fn, max(3, args.steps // 2), stream)
        dgc.dgc_import_state(m.h, c_host, c)
        fr = lambda: dgc.dgc_rhs(m.h, dgc.DGC_FP64, c, r)
        fr()
        t_rhs = time_steps(torch, fr, 3, stream)
        rows.append({"colors": int(nc), "renumber": renumber, "reorder": reorder,
                     "rk_fp32mixed_ms": round(t_rk, 4), "rhs_fp64_ms": round(t_rhs, 4),
                     "launches_per_step": dgc.dgc_last_launch_count(m.h)})
        del ws
    for row in rows:
        row["pct_rk"] = round(100.0 * (rows[0]["rk_fp32mixed_ms"] - row["rk_fp32mixed_ms"]) / rows[0]["rk_fp32mixed_ms"], 1)
        row["pct_rhs_fp64"] = round(100.0 * (rows[0]["rhs_fp64_ms"] - row["rhs_fp64_ms"]) / rows[0]["rhs_fp64_ms"], 1)
    m.close()
    return {"table7_ablation": {"mesh": "1,048,352 jittered periodic triangles, element list in seeded random order",
                                "p": cfg["p"], "dofs": dofs, "rows": rows}}


def run_double_mach(dgc, torch, dev, stream, args):
    """The double Mach reflection run Table 7 times (Sec. 5; its setup is
    [giuliani]'s, not the paper's: the standard Mach 10 problem on [0, 4] x
    [0, 1]): 1120 x 280 cells of two jittered triangles (627,200 elements, mesh
    D's size), p = 1, FP64, slip wall / inflow / moving-shock / outflow
    boundaries and the limiter after every RK stage.  Times the limited RK step
    (CUDA events over the paper's 1000 steps from the initial state), checks the
    means stay physical, and repeats Table 7's ablation on this mesh with its
    element list in a seeded random order (naive greedy 5 colors or the
    modified coloring's 3, with and without the color-1 renumbering and the
    left-ascending edge order; 200 steps each; pct = speed-up over the first row)."""
    cfg = W.double_mach_p1()
    p = cfg["p"]

    def build(mi):
        m = dgc.Mesh.from_input(mi, p)
        l, r, ql, _ = dgc.dgc_get_sides(m.h)
        kind, sidx = W.double_mach_boundary(mi, l, r, ql)
        dgc.dgc_set_boundary(m.h, kind, sidx, cfg["states"], cfg["shock"], cfg["shock_states"])
        dgc.dgc_set_option(m.h, dgc.DGC_OPT_LIMITER, 1)
        xyz = dgc.dgc_vol_points(m.h)
        return m, dgc.dgc_project(m.h, W.double_mach_field(xyz[..., 0], xyz[..., 1]))

    out = {}
    t0 = time.perf_counter()
    m, c_host = build(cfg["mesh"])
    m.color(1601)
    prep = time.perf_counter() - t0
    info = m.info
    dofs = info["ne"] * info["M"] * info["np"]
    c = torch.empty(m.state_shape(), dtype=torch.float64, device=dev)
    dt = torch.zeros(1, dtype=torch.float64, device=dev)
    ws = torch.empty(dgc.dgc_workspace_size(m.h, dgc.DGC_FP64) // 8 + 64, dtype=torch.float64, device=dev)
    dgc.dgc_import_state(m.h, c_host, c)
    dgc.dgc_limit(m.h, dgc.DGC_FP64, c)
    dgc.dgc_set_time(m.h, 0.0)
    fn = lambda: dgc.dgc_rk_step(m.h, dgc.DGC_FP64, c, cfg["cfl"], dt, ws)
    ms = time_steps(torch, fn, 1000, stream)
    t_end = dgc.dgc_get_time(m.h)
    U = dgc.dgc_export_state(m.h, c)[:, :, 0] * np.sqrt(2.0)  # element means (phi_0 = sqrt 2)
    # per kernel class from a profiled pass (event pairs around every launch)
    dgc.dgc_set_option(m.h, dgc.DGC_OPT_PROFILE, 1)
    dgc.dgc_profile_collect(m.h)
    msp = time_steps(torch, fn, 50, stream)
    prof = dgc.dgc_profile_collect(m.h)
    dgc.dgc_set_option(m.h, dgc.DGC_OPT_PROFILE, 0)
    kern = {cls: {"launches": nl, "ms_per_step": round(tms / 50, 4), "share": round(tms / (msp * 50), 3)}
            for cls, (tms, nl) in prof.items()}
    pr = 0.4 * (U[:, 3] - 0.5 * (U[:, 1] ** 2 + U[:, 2] ** 2) / U[:, 0])
    out["run"] = {"elements": info["ne"], "p": p, "dofs": dofs, "colors": info["ncolors"], "steps": 1000,
                  "ms_per_step": round(ms, 4), "s_1000_steps": round(ms, 3),
                  "value": 3 * dofs / (ms * 1e-3), "unit": "DOF-RHS updates/s",
                  "launches_per_step": dgc.dgc_last_launch_count(m.h), "t_end": t_end,
                  "min_density": float(U[:, 0].min()), "min_pressure": float(pr.min()),
                  "finite": bool(np.isfinite(U).all()), "host_prep_s": round(prep, 2),
                  "profiled_ms_per_step": round(msp, 4), "kernels": kern}
    m.close()
    # Table 7 on this mesh, its elements in a seeded random order
    mi = cfg["mesh"]
    perm = np.random.default_rng(1601).permutation(mi.ne)
    mp = W.MeshInput(2, mi.xyz, np.ascontiguousarray(mi.ev[perm]), None, name=mi.name + "_shuffled")
    m, c_host = build(mp)
    rows = []
    for colors, renumber, reorder in ((5, False, False), (3, False, False), (5, True, False), (3, True, False),
                                      (5, True, True), (3, True, True)):
        if colors == 5:
            nc, _ = dgc.dgc_color_edges_naive(m.h, renumber, reorder)
        else:
            nc, _ = dgc.dgc_color_edges(m.h, 1601, 0)
            dgc.dgc_reorder(m.h, renumber, reorder)
        ws = torch.empty(dgc.dgc_workspace_size(m.h, dgc.DGC_FP64) // 8 + 64, dtype=torch.float64, device=dev)
        dgc.dgc_import_state(m.h, c_host, c)
        dgc.dgc_set_time(m.h, 0.0)
        fn = lambda: dgc.dgc_rk_step(m.h, dgc.DGC_FP64, c, cfg["cfl"], dt, ws)
        fn()
        t_rk = time_steps(torch, fn, 200, stream)
        rows.append({"colors": int(nc), "renumber": renumber, "reorder": reorder, "ms_per_step": round(t_rk, 4),
                     "launches_per_step": dgc.dgc_last_launch_count(m.h)})
        del ws
    for row in rows:
        row["pct"] = round(100.0 * (rows[0]["ms_per_step"] - row["ms_per_step"]) / rows[0]["ms_per_step"], 1)
    m.close()
    out["table7"] = {"mesh": "the same mesh, element list in seeded random order", "steps_per_row": 200,
                     "rows": rows}
    return {"double_mach_p1_627200": out}


def host_cores() -> int:
    """Host cores this process may run on (nproc)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(mi, p, c_host, dofs, single_elements: int = 100_000):
    """The CPU oracle as it stands (FP64 C, element by element as Eq. 2 is
    written): its threaded build (gcc -O3 -fopenmp, the element loop split over
    all host cores) on one whole right-hand side of the same workload, and its
    sequential build on a random sample of single_elements elements."""
    import oracle

    E = mi.ne
    nv = c_host.shape[1] * c_host.shape[2]
    cores = host_cores()
    mt = oracle.OracleMesh.from_input(mi, build="threads")
    used = oracle.set_threads(cores)
    t0 = time.perf_counter()
    mt.rhs(p, c_host)
    t = time.perf_counter() - t0
    del mt
    om = oracle.OracleMesh.from_input(mi)
    n1 = min(single_elements, E)
    sel = np.random.default_rng(0).choice(E, n1, replace=False)
    t1 = time.perf_counter()
    om.rhs(p, c_host, elems=sel)
    ts = time.perf_counter() - t1
    return {"value": E * nv / t, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"one FP64 right-hand side of all {E} elements, {t:.2f} s on {used} threads "
                      f"(gcc -O3 -fopenmp, no FMA contraction)",
            "single_thread": {"value": n1 * nv / ts, "unit": UNIT, "cores": 1,
                              "sample": f"{n1} random elements of one right-hand side, {ts:.2f} s, sequential build"}}


def run_reference(args):
    """The CPU oracle on the host cores: each step is one right-hand side of a
    bounded random sample of the workload's elements."""
    import oracle

    cfg = W.jittered_square_vortex_p3_724x724(args.n)
    mi, p = cfg["mesh"], cfg["p"]
    workload = WORKLOAD if args.n == 724 else f"2D Euler DG p=3 on {mi.ne} jittered periodic triangles ({args.n}x{args.n})"
    om = oracle.OracleMesh.from_input(mi)
    xyz, _, _ = om.eval_points(p)
    c = om.project(p, W.vortex_field(xyz[..., 0], xyz[..., 1], beta=cfg["beta"]))
    c += W.uniform_perturbation(c.shape, cfg["perturb_seed"], cfg["perturb"])
    del xyz
    E = mi.ne
    NV = c.shape[1] * c.shape[2]
    per_step = min(args.ref_elements, E) if args.ref_elements > 0 else E
    cores = host_cores()
    mt = oracle.OracleMesh.from_input(mi, build="threads")
    used = oracle.set_threads(cores)
    del om
    rng = np.random.default_rng(0)

    def sample():
        return None if per_step == E else rng.choice(E, per_step, replace=False)

    for _ in range(args.warmup):
        mt.rhs(p, c, elems=sample())
    t0 = time.perf_counter()
    for _ in range(args.steps):
        mt.rhs(p, c, elems=sample())
    t = (time.perf_counter() - t0) / args.steps
    value = per_step * NV / t
    what = "all" if per_step == E else f"{per_step} random"
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t * 1e3, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload, "elements": E, "p": p,
                   "step": f"one oracle right-hand side of {what} elements"},
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": used,
                         "sample": f"{what} elements per step, FP64 C oracle, threaded build on {used} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["dgc", "reference"], default="dgc")
    ap.add_argument("--no-variants", action="store_true", help="skip the FP64 and comparator timings")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffers) timing")
    ap.add_argument("--ref-elements", type=int, default=0,
                    help="oracle elements per reference step (0 = the whole mesh)")
    ap.add_argument("--epb", type=int, default=0, help="edges per block of the surface kernels (0 = library default)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default tiles")
    ap.add_argument("--tiles", default="", help="tiles of the first, middle and last colors as EPBxTPE,EPBxTPE,"
                    "EPBxTPE (edges per block x threads per edge), instead of the autotuner's")
    ap.add_argument("--tpe", type=int, default=0, help="threads per edge of the FP32 surface kernels (0 = library "
                    "default: 2)")
    ap.add_argument("--no-pdl", action="store_true", help="launch the headline step's kernels in plain stream order")
    ap.add_argument("--n", type=int, default=724, help="grid size n (n x n squares, 2 n^2 triangles); "
                    "724 is the benchmark workload, smaller n is for profiler captures")
    ap.add_argument("--only", choices=["tet", "nonconforming", "quad", "hybrid", "bilinear", "batch", "double_mach",
                                       "two_level"],
                    help="time only that one of the other workloads (its variants entry, printed alone)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.only:
        import torch

        from paper_1601_07613_gb300 import dgc

        dgc.lib()
        dev = torch.device("cuda:0")
        st = torch.cuda.current_stream()
        if args.only == "batch":
            print(json.dumps(run_batched(dgc, torch, dev, st, args)), flush=True)
        elif args.only == "double_mach":
            print(json.dumps(run_double_mach(dgc, torch, dev, st, args)), flush=True)
        elif args.only == "two_level":
            print(json.dumps({"nonconforming_two_level_p2_256": run_two_level(dgc, torch, dev, st, args)}), flush=True)
        else:
            print(json.dumps(run_other_meshes(dgc, torch, dev, st, args, only=args.only)), flush=True)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args)), flush=True)
        return

    if world > 1:
        import torch

        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    out = run_dgc(args, rank, world, local_rank)
    if world > 1:
        import torch

        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
