"""Thin ctypes binding of the C ABI in include/dgc.h (same function names).

Only argument marshalling lives here: numpy arrays are passed as host
pointers, torch CUDA tensors (or integers) as device pointers, and the current
torch stream as the ``cudaStream_t``.  All computation happens in the compiled
library; if it is missing, importing this module's ``lib()`` raises.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build_lib

DGC_FP64 = 0
DGC_FP32_MIXED = 1
DGC_FP32_KAHAN = 2
DGC_OPT_FUSE = 0
DGC_OPT_EDGES_PER_BLOCK = 1
DGC_OPT_THREADS_PER_EDGE = 2
DGC_OPT_PROFILE = 3
DGC_OPT_GRAPH = 4
DGC_OPT_PDL = 5
DGC_OPT_COOPERATIVE = 6
DGC_OPT_PERSISTENT = 7
DGC_OPT_LIMITER = 8
DGC_BC_TRANSMISSIVE, DGC_BC_WALL, DGC_BC_STATE, DGC_BC_SHOCK = 0, 1, 2, 3  # dgc_bc
DGC_TRI, DGC_QUAD, DGC_TET = 0, 1, 2  # dgc_elem
KERNEL_CLASSES = ["cfl", "volume", "first", "color", "last", "stage", "atomic", "buffer", "gather", "limit"]

STATUS = {0: "DGC_OK", 1: "DGC_ERR_ARG", 2: "DGC_ERR_MESH", 3: "DGC_ERR_COLORING_LIMIT",
          4: "DGC_ERR_UNSUPPORTED", 5: "DGC_ERR_CUDA", 6: "DGC_ERR_OOM", 7: "DGC_ERR_NONFINITE"}

# Every function the header declares, with its ctypes signature.
_P = C.c_void_p
_I64 = C.c_int64
_I32P = C.POINTER(C.c_int32)
_I64P = C.POINTER(C.c_int64)
_DP = C.POINTER(C.c_double)
SIGNATURES = {
    "dgc_mesh_create": (C.c_int, [C.c_int, C.c_int, _I64, _DP, _I64, _I32P, _DP, C.POINTER(_P)]),
    "dgc_mesh_create_elem": (C.c_int, [C.c_int, C.c_int, _I64, _DP, _I64, _I32P, _DP, C.POINTER(_P)]),
    "dgc_mesh_element": (C.c_int, [_P, _I32P, _I64P]),
    "dgc_color_edges": (C.c_int, [_P, C.c_uint64, _I64, _I32P, _I64P]),
    "dgc_color_edges_naive": (C.c_int, [_P, C.c_int, C.c_int, _I32P, _I64P]),
    "dgc_mesh_info": (C.c_int, [_P, _I64P]),
    "dgc_get_sides": (C.c_int, [_P, _I32P, _I32P, C.POINTER(C.c_int8), C.POINTER(C.c_int8)]),
    "dgc_refine": (C.c_int, [_P, _I64, _I32P]),
    "dgc_reorder": (C.c_int, [_P, C.c_int, C.c_int]),
    "dgc_coarsen": (C.c_int, [_P]),
    "dgc_get_hanging": (C.c_int, [_P, C.POINTER(C.c_int8)]),
    "dgc_get_elements": (C.c_int, [_P, _I32P, _DP]),
    "dgc_get_ordering": (C.c_int, [_P, _I32P, _I32P, C.POINTER(C.c_int8), _I32P]),
    "dgc_vol_points": (C.c_int, [_P, _DP]),
    "dgc_project": (C.c_int, [_P, _DP, _DP]),
    "dgc_state_size": (C.c_int, [_P, _I64P]),
    "dgc_workspace_size": (C.c_int, [_P, C.c_int, _I64P]),
    "dgc_import_state": (C.c_int, [_P, _DP, _P, _P]),
    "dgc_state_bytes": (C.c_int, [_P, C.c_int, _I64P]),
    "dgc_import_state_async": (C.c_int, [_P, _DP, _P, _P, _P]),
    "dgc_export_state_async": (C.c_int, [_P, _P, _DP, _P, _P]),
    "dgc_import_state_prec": (C.c_int, [_P, C.c_int, _DP, _P, _P]),
    "dgc_export_state_prec": (C.c_int, [_P, C.c_int, _P, _DP, _P]),
    "dgc_export_state": (C.c_int, [_P, _P, _DP, _P]),
    "dgc_rhs": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "dgc_cfl_dt": (C.c_int, [_P, _P, C.c_double, _P, _P]),
    "dgc_rk_step": (C.c_int, [_P, C.c_int, _P, C.c_double, _P, _P, _I64, _P]),
    "dgc_rhs_atomic": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "dgc_rhs_two_pass": (C.c_int, [_P, C.c_int, _P, _P, _P, _I64, _P]),
    "dgc_two_pass_buffer_bytes": (C.c_int, [_I64, C.c_int, C.c_int, C.c_int, _I64P]),
    "dgc_set_option": (C.c_int, [_P, C.c_int, _I64]),
    "dgc_profile_collect": (C.c_int, [_P, _DP, _I64P]),
    "dgc_last_launch_count": (C.c_int, [_P, _I64P]),
    "dgc_last_error": (C.c_char_p, []),
    "dgc_rk_step_static": (C.c_int, [_P, C.c_int, _P, C.c_double, _P, _P]),
    "dgc_set_tile": (C.c_int, [_P, C.c_int, C.c_int, C.c_int]),
    "dgc_prolong_state": (C.c_int, [_P, _P, _P, _P]),
    "dgc_restrict_state": (C.c_int, [_P, _P, _P, _P]),
    "dgc_refine_colors_device": (C.c_int, [_P, C.POINTER(C.c_int8), _DP, _P]),
    "dgc_get_tile": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "dgc_autotune": (C.c_int, [_P, C.c_int, _P, C.c_double, _P, _P, _I64, C.c_int, _P, C.POINTER(C.c_int),
                               C.POINTER(C.c_int), _DP]),
    "dgc_batch_create": (C.c_int, [C.c_int, C.POINTER(_P), C.POINTER(_P)]),
    "dgc_batch_workspace_size": (C.c_int, [_P, C.c_int, _I64P]),
    "dgc_batch_set_option": (C.c_int, [_P, C.c_int, _I64]),
    "dgc_batch_rk_step": (C.c_int, [_P, C.c_int, C.POINTER(_P), C.c_double, _P, _P, _I64, _P]),
    "dgc_batch_autotune": (C.c_int, [_P, C.c_int, C.POINTER(_P), C.c_double, _P, _P, _I64, C.c_int, _P,
                                     C.POINTER(C.c_int), C.POINTER(C.c_int), _DP]),
    "dgc_batch_launch_count": (C.c_int, [_P, _I64P]),
    "dgc_batch_profile_collect": (C.c_int, [_P, _DP, _I64P]),
    "dgc_batch_set_tile": (C.c_int, [_P, C.c_int, C.c_int, C.c_int]),
    "dgc_set_boundary": (C.c_int, [_P, C.POINTER(C.c_int8), C.POINTER(C.c_int8), C.c_int, _DP, _DP,
                                   C.POINTER(C.c_int8)]),
    "dgc_set_time": (C.c_int, [_P, C.c_double]),
    "dgc_get_time": (C.c_int, [_P, _DP]),
    "dgc_limit": (C.c_int, [_P, C.c_int, _P, _P]),
    "dgc_batch_destroy": (None, [_P]),
    "dgc_destroy": (None, [_P]),
}

_lib = None


class DgcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def lib(build: bool = True):
    """Load the compiled library (building it first if asked); raises if it is unavailable."""
    global _lib
    if _lib is None:
        path = _build_lib.LIB
        if build:
            path = _build_lib.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path}")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise DgcError(status, lib().dgc_last_error().decode())


def _dptr(a) -> int:
    """Device pointer of a torch tensor (or an integer address)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    return a.data_ptr()


def _stream(stream) -> int | None:
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


def _h(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(C.POINTER(np.ctypeslib.as_ctypes_type(dtype)))


# --- the C ABI, one wrapper per function -----------------------------------------------

def dgc_mesh_create(dim: int, p: int, xyz, ev, periodic_len=None):
    xyz, xp = _h(xyz, np.float64)
    ev, ep = _h(ev, np.int32)
    lp = None
    if periodic_len is not None:
        L, lp = _h(periodic_len, np.float64)
    out = _P()
    _check(lib().dgc_mesh_create(dim, p, xyz.shape[0], xp, ev.shape[0], ep, lp, C.byref(out)))
    return out


def dgc_mesh_create_elem(elem: int, p: int, xyz, ev, periodic_len=None):
    xyz, xp = _h(xyz, np.float64)
    ev, ep = _h(ev, np.int32)
    lp = None
    if periodic_len is not None:
        L, lp = _h(periodic_len, np.float64)
    out = _P()
    _check(lib().dgc_mesh_create_elem(elem, p, xyz.shape[0], xp, ev.shape[0], ep, lp, C.byref(out)))
    return out


def dgc_mesh_element(mesh):
    """(element type DGC_TRI / DGC_QUAD / DGC_TET, elements the kernels do not take)"""
    t = C.c_int32()
    n = C.c_int64()
    _check(lib().dgc_mesh_element(mesh, C.byref(t), C.byref(n)))
    return t.value, n.value


def dgc_color_edges(mesh, seed: int, max_swaps: int = 0):
    nc = C.c_int32()
    per = (C.c_int64 * 8)()
    _check(lib().dgc_color_edges(mesh, seed, max_swaps, C.byref(nc), per))
    return nc.value, list(per)[: nc.value]


def dgc_color_edges_naive(mesh, renumber: bool = True, reorder: bool = True):
    nc = C.c_int32()
    per = (C.c_int64 * 8)()
    _check(lib().dgc_color_edges_naive(mesh, int(renumber), int(reorder), C.byref(nc), per))
    return nc.value, list(per)[: min(nc.value, 8)]


def dgc_mesh_info(mesh) -> dict:
    a = (C.c_int64 * 10)()
    _check(lib().dgc_mesh_info(mesh, a))
    keys = ["ne", "ns", "np", "M", "nqf", "nqv", "ncolors", "dim", "p", "perfect"]
    return dict(zip(keys, list(a)))


def dgc_get_sides(mesh):
    ns = dgc_mesh_info(mesh)["ns"]
    l, r = np.zeros(ns, np.int32), np.zeros(ns, np.int32)
    ql, qr = np.zeros(ns, np.int8), np.zeros(ns, np.int8)
    _check(lib().dgc_get_sides(mesh, *(x.ctypes.data_as(_I32P) for x in (l, r)),
                               *(x.ctypes.data_as(C.POINTER(C.c_int8)) for x in (ql, qr))))
    return l, r, ql, qr


def dgc_reorder(mesh, renumber: bool, reorder_left: bool):
    _check(lib().dgc_reorder(mesh, int(renumber), int(reorder_left)))


def dgc_refine(mesh, elems):
    e = np.ascontiguousarray(np.asarray(elems, dtype=np.int32).ravel())
    _check(lib().dgc_refine(mesh, len(e), e.ctypes.data_as(_I32P)))


def dgc_coarsen(mesh):
    _check(lib().dgc_coarsen(mesh))


def dgc_get_hanging(mesh):
    h = np.zeros(dgc_mesh_info(mesh)["ns"], np.int8)
    _check(lib().dgc_get_hanging(mesh, h.ctypes.data_as(C.POINTER(C.c_int8))))
    return h


def dgc_get_elements(mesh):
    info = dgc_mesh_info(mesh)
    nvpe = info["dim"] + 1
    ev = np.zeros((info["ne"], nvpe), np.int32)
    X = np.zeros((info["ne"], nvpe, info["dim"]))
    _check(lib().dgc_get_elements(mesh, ev.ctypes.data_as(_I32P), X.ctypes.data_as(_DP)))
    return ev, X


def dgc_get_ordering(mesh):
    info = dgc_mesh_info(mesh)
    en = np.zeros(info["ne"], np.int32)
    sn = np.zeros(info["ns"], np.int32)
    col = np.zeros(info["ns"], np.int8)
    off = np.zeros(info["ncolors"] + 1, np.int32)
    _check(lib().dgc_get_ordering(mesh, en.ctypes.data_as(_I32P), sn.ctypes.data_as(_I32P),
                                  col.ctypes.data_as(C.POINTER(C.c_int8)), off.ctypes.data_as(_I32P)))
    return en, sn, col, off


def dgc_vol_points(mesh) -> np.ndarray:
    info = dgc_mesh_info(mesh)
    out = np.zeros((info["ne"], info["nqv"], info["dim"]))
    _check(lib().dgc_vol_points(mesh, out.ctypes.data_as(_DP)))
    return out


def dgc_project(mesh, vals) -> np.ndarray:
    info = dgc_mesh_info(mesh)
    vals, vp = _h(vals, np.float64)
    out = np.zeros((info["ne"], info["M"], info["np"]))
    _check(lib().dgc_project(mesh, vp, out.ctypes.data_as(_DP)))
    return out


def dgc_state_size(mesh) -> int:
    b = C.c_int64()
    _check(lib().dgc_state_size(mesh, C.byref(b)))
    return b.value


def dgc_workspace_size(mesh, prec: int) -> int:
    b = C.c_int64()
    _check(lib().dgc_workspace_size(mesh, prec, C.byref(b)))
    return b.value


def dgc_import_state(mesh, c_host, c_dev, stream=None):
    c_host, cp = _h(c_host, np.float64)
    _check(lib().dgc_import_state(mesh, cp, _dptr(c_dev), _stream(stream)))


def dgc_export_state(mesh, c_dev, out=None, stream=None):
    info = dgc_mesh_info(mesh)
    if out is None:
        out = np.zeros((info["ne"], info["M"], info["np"]))
    _check(lib().dgc_export_state(mesh, _dptr(c_dev), out.ctypes.data_as(_DP), _stream(stream)))
    return out


def dgc_import_state_async(mesh, c_host, c_dev, xfer_dev, stream=None):
    """c_host: a C-contiguous float64 numpy view of pinned host memory."""
    _check(lib().dgc_import_state_async(mesh, c_host.ctypes.data_as(_DP), _dptr(c_dev), _dptr(xfer_dev),
                                        _stream(stream)))


def dgc_export_state_async(mesh, c_dev, c_host, xfer_dev, stream=None):
    _check(lib().dgc_export_state_async(mesh, _dptr(c_dev), c_host.ctypes.data_as(_DP), _dptr(xfer_dev),
                                        _stream(stream)))


def dgc_state_bytes(mesh, prec: int) -> int:
    b = C.c_int64()
    _check(lib().dgc_state_bytes(mesh, prec, C.byref(b)))
    return b.value


def dgc_import_state_prec(mesh, prec: int, c_host, c_dev, stream=None):
    c_host, cp = _h(c_host, np.float64)
    _check(lib().dgc_import_state_prec(mesh, prec, cp, _dptr(c_dev), _stream(stream)))


def dgc_export_state_prec(mesh, prec: int, c_dev, out=None, stream=None):
    info = dgc_mesh_info(mesh)
    if out is None:
        out = np.zeros((info["ne"], info["M"], info["np"]))
    _check(lib().dgc_export_state_prec(mesh, prec, _dptr(c_dev), out.ctypes.data_as(_DP), _stream(stream)))
    return out


def dgc_rhs(mesh, prec: int, c_dev, rhs_dev, stream=None):
    _check(lib().dgc_rhs(mesh, prec, _dptr(c_dev), _dptr(rhs_dev), _stream(stream)))


def dgc_set_boundary(mesh, kind, state_idx=None, states=None, shock=None, shock_states=None):
    """kind[s], state_idx[s] per side in dgc_get_sides order; states [n][4]."""
    k = np.ascontiguousarray(kind, dtype=np.int8)
    si = None if state_idx is None else np.ascontiguousarray(state_idx, dtype=np.int8)
    st = np.ascontiguousarray(np.zeros((0, 4)) if states is None else np.asarray(states, dtype=np.float64).reshape(-1, 4))
    sh = None if shock is None else np.ascontiguousarray(shock, dtype=np.float64)
    ss = None if shock_states is None else np.ascontiguousarray(shock_states, dtype=np.int8)
    i8 = C.POINTER(C.c_int8)
    _check(lib().dgc_set_boundary(mesh, k.ctypes.data_as(i8), si.ctypes.data_as(i8) if si is not None else None,
                                  st.shape[0], st.ctypes.data_as(_DP) if st.size else None,
                                  sh.ctypes.data_as(_DP) if sh is not None else None,
                                  ss.ctypes.data_as(i8) if ss is not None else None))


def dgc_set_time(mesh, t: float):
    _check(lib().dgc_set_time(mesh, float(t)))


def dgc_get_time(mesh) -> float:
    t = C.c_double(0.0)
    _check(lib().dgc_get_time(mesh, C.byref(t)))
    return t.value


def dgc_limit(mesh, prec: int, c_dev, stream=None):
    _check(lib().dgc_limit(mesh, prec, _dptr(c_dev), _stream(stream)))


def dgc_cfl_dt(mesh, c_dev, cfl: float, dt_dev, stream=None):
    _check(lib().dgc_cfl_dt(mesh, _dptr(c_dev), cfl, _dptr(dt_dev), _stream(stream)))


def _nbytes(a, nbytes):
    if nbytes is not None:
        return nbytes
    return a.numel() * a.element_size()


def dgc_rk_step(mesh, prec: int, c_dev, cfl: float, dt_dev, workspace_dev, workspace_bytes=None, stream=None):
    """workspace_bytes defaults to the size of the workspace tensor."""
    _check(lib().dgc_rk_step(mesh, prec, _dptr(c_dev), cfl, _dptr(dt_dev), _dptr(workspace_dev),
                             _nbytes(workspace_dev, workspace_bytes), _stream(stream)))


def dgc_rhs_atomic(mesh, prec: int, c_dev, rhs_dev, stream=None):
    _check(lib().dgc_rhs_atomic(mesh, prec, _dptr(c_dev), _dptr(rhs_dev), _stream(stream)))


def dgc_rhs_two_pass(mesh, prec: int, c_dev, rhs_dev, buffer_dev, buffer_bytes=None, stream=None):
    """buffer_bytes defaults to the size of the buffer tensor."""
    _check(lib().dgc_rhs_two_pass(mesh, prec, _dptr(c_dev), _dptr(rhs_dev), _dptr(buffer_dev),
                                  _nbytes(buffer_dev, buffer_bytes), _stream(stream)))


def dgc_two_pass_buffer_bytes(sides: int, np_: int, neq: int, word_bytes: int = 8) -> int:
    b = C.c_int64()
    _check(lib().dgc_two_pass_buffer_bytes(sides, np_, neq, word_bytes, C.byref(b)))
    return b.value


def dgc_set_option(mesh, opt: int, value: int):
    _check(lib().dgc_set_option(mesh, opt, value))


DGC_K_FIRST, DGC_K_COLOR, DGC_K_LAST = 2, 3, 4


def dgc_prolong_state(mesh, c_coarse_dev, c_fine_dev, stream=None):
    _check(lib().dgc_prolong_state(mesh, _dptr(c_coarse_dev), _dptr(c_fine_dev), _stream(stream)))


def dgc_restrict_state(mesh, c_fine_dev, c_coarse_dev, stream=None):
    _check(lib().dgc_restrict_state(mesh, _dptr(c_fine_dev), _dptr(c_coarse_dev), _stream(stream)))


def dgc_refine_colors_device(mesh, ns: int, stream=None):
    """Returns (colors int8[Ns] in original side order, map kernel ms)."""
    out = np.zeros(ns, np.int8)
    ms = C.c_double()
    _check(lib().dgc_refine_colors_device(mesh, out.ctypes.data_as(C.POINTER(C.c_int8)), C.byref(ms),
                                          _stream(stream)))
    return out, ms.value


def dgc_set_tile(mesh, kclass: int, edges_per_block: int, threads_per_edge: int):
    _check(lib().dgc_set_tile(mesh, kclass, edges_per_block, threads_per_edge))


def dgc_get_tile(mesh, kclass: int):
    e, t = C.c_int(), C.c_int()
    _check(lib().dgc_get_tile(mesh, kclass, C.byref(e), C.byref(t)))
    return e.value, t.value


def dgc_autotune(mesh, prec: int, c_dev, cfl: float, dt_dev, workspace_dev, reps: int = 5, workspace_bytes=None,
                 stream=None):
    """Returns ({"first"|"color"|"last": (edges per block, threads per edge)}, best ms per step)."""
    e = (C.c_int * 3)()
    t = (C.c_int * 3)()
    ms = C.c_double()
    _check(lib().dgc_autotune(mesh, prec, _dptr(c_dev), cfl, _dptr(dt_dev), _dptr(workspace_dev),
                              _nbytes(workspace_dev, workspace_bytes), reps, _stream(stream), e, t, C.byref(ms)))
    return {k: (e[i], t[i]) for i, k in enumerate(("first", "color", "last"))}, ms.value


def dgc_profile_collect(mesh) -> dict:
    ms = (C.c_double * 16)()
    n = (C.c_int64 * 16)()
    _check(lib().dgc_profile_collect(mesh, ms, n))
    return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_CLASSES) if n[i] > 0}


def dgc_last_launch_count(mesh) -> int:
    b = C.c_int64()
    _check(lib().dgc_last_launch_count(mesh, C.byref(b)))
    return b.value


def dgc_rk_step_static(mesh, prec: int, c_dev, cfl: float, dt_dev, stream=None):
    """dgc_rk_step without a caller workspace (small meshes; see include/dgc.h)."""
    _check(lib().dgc_rk_step_static(mesh, prec, _dptr(c_dev), cfl, _dptr(dt_dev), _stream(stream)))


def _ptr_array(tensors):
    arr = (_P * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = _dptr(t)
    return arr


def dgc_batch_create(meshes):
    handles = (_P * len(meshes))(*[m.h if isinstance(m, Mesh) else m for m in meshes])
    out = _P()
    _check(lib().dgc_batch_create(len(meshes), handles, C.byref(out)))
    return out


def dgc_batch_workspace_size(batch, prec: int) -> int:
    b = C.c_int64()
    _check(lib().dgc_batch_workspace_size(batch, prec, C.byref(b)))
    return b.value


def dgc_batch_set_option(batch, opt: int, value: int):
    _check(lib().dgc_batch_set_option(batch, opt, value))


def dgc_batch_rk_step(batch, prec: int, c_devs, cfl: float, dt_devs, workspace_dev, workspace_bytes=None,
                      stream=None):
    _check(lib().dgc_batch_rk_step(batch, prec, _ptr_array(c_devs), cfl, _dptr(dt_devs), _dptr(workspace_dev),
                                   _nbytes(workspace_dev, workspace_bytes), _stream(stream)))


def dgc_batch_autotune(batch, prec: int, c_devs, cfl: float, dt_devs, workspace_dev, reps: int = 5,
                       workspace_bytes=None, stream=None):
    """Returns ({"first"|"color"|"last": (edges per block, threads per edge)}, best ms per step)."""
    e = (C.c_int * 3)()
    t = (C.c_int * 3)()
    ms = C.c_double()
    _check(lib().dgc_batch_autotune(batch, prec, _ptr_array(c_devs), cfl, _dptr(dt_devs), _dptr(workspace_dev),
                                    _nbytes(workspace_dev, workspace_bytes), reps, _stream(stream), e, t,
                                    C.byref(ms)))
    return {k: (e[i], t[i]) for i, k in enumerate(("first", "color", "last"))}, ms.value


def dgc_batch_launch_count(batch) -> int:
    b = C.c_int64()
    _check(lib().dgc_batch_launch_count(batch, C.byref(b)))
    return b.value


def dgc_batch_set_tile(batch, kclass: int, edges_per_block: int, threads_per_edge: int):
    _check(lib().dgc_batch_set_tile(batch, kclass, edges_per_block, threads_per_edge))


def dgc_batch_profile_collect(batch) -> dict:
    ms = (C.c_double * 16)()
    n = (C.c_int64 * 16)()
    _check(lib().dgc_batch_profile_collect(batch, ms, n))
    return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_CLASSES) if n[i] > 0}


def dgc_batch_destroy(batch):
    if batch:
        lib().dgc_batch_destroy(batch)


def dgc_last_error() -> str:
    return lib().dgc_last_error().decode()


def dgc_destroy(mesh):
    if mesh:
        lib().dgc_destroy(mesh)


class Mesh:
    """Owns a dgc_mesh handle; convenience accessors over the functions above."""

    def __init__(self, dim, p, xyz, ev, periodic_len=None):
        ev = np.asarray(ev)
        if dim == 2 and ev.shape[1] == 4:  # quadrilateral or hybrid mesh
            self.h = dgc_mesh_create_elem(DGC_QUAD, p, xyz, ev, periodic_len)
        else:
            self.h = dgc_mesh_create(dim, p, xyz, ev, periodic_len)
        self.info = dgc_mesh_info(self.h)
        self.elem, self.nonaffine = dgc_mesh_element(self.h)

    @classmethod
    def from_input(cls, mi, p):
        return cls(mi.dim, p, mi.xyz, mi.ev, mi.periodic_len)

    def color(self, seed: int, max_swaps: int = 0):
        r = dgc_color_edges(self.h, seed, max_swaps)
        self.info = dgc_mesh_info(self.h)
        return r

    def refine(self, elems):
        dgc_refine(self.h, elems)
        self.info = dgc_mesh_info(self.h)

    def coarsen(self):
        dgc_coarsen(self.h)
        self.info = dgc_mesh_info(self.h)

    def state_shape(self):
        return (self.info["ne"], self.info["M"], self.info["np"])

    def close(self):
        if self.h:
            dgc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
