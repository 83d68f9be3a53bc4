"""CPU oracle for the colored DG right-hand side -- TEST INFRASTRUCTURE ONLY.

A plain, slow FP64 C implementation (``dg_oracle.c``) of what the CUDA path
computes: the edge table, the paper's coloring and reordering (Sec. 3.1, Sec. 5)
and the modal DG right-hand side of Eq. 2 evaluated element by element, plus the
CFL rule and SSP-RK3 step.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  Quadrilateral and
hybrid triangle/quadrilateral meshes are built from a [E][4] element list (-1 as
the fourth vertex of a triangle).  It shares no code with
``paper_1601_07613_gb300`` (the product), and the product never imports it.

This module only builds the C file with gcc and marshals numpy arrays through
ctypes; all arithmetic is in ``dg_oracle.c``.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dg_oracle.c")
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

EULER = 0
ADVECTION = 1


def build(force: bool = False) -> str:
    """Compile dg_oracle.c into oracle/_build/liboracle.so (gcc, -O2, no FMA contraction)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i32(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _i64(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _i8(a):
    return a.ctypes.data_as(C.POINTER(C.c_int8))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            P = C.c_void_p
            dp = C.POINTER(C.c_double)
            L.orc_last_error.restype = C.c_char_p
            L.orc_gauss_jacobi.argtypes = [C.c_int, C.c_double, dp, dp]
            L.orc_tri_rule.argtypes = [C.c_int, dp, dp, dp]
            L.orc_tet_rule.argtypes = [C.c_int, dp, dp, dp, dp]
            L.orc_basis_tri.argtypes = [C.c_int, C.c_double, C.c_double, dp, dp, dp]
            L.orc_basis_tet.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, dp, dp, dp, dp]
            L.orc_basis_quad.argtypes = [C.c_int, C.c_double, C.c_double, dp, dp, dp]
            L.orc_quad_rule.argtypes = [C.c_int, dp, dp, dp]
            L.orc_mesh_new_quad.restype = P
            L.orc_mesh_new_quad.argtypes = [C.c_int64, dp, C.c_int64, C.POINTER(C.c_int32), dp]
            L.orc_mesh_is_quad.argtypes = [P]
            L.orc_mesh_nonaffine.restype = C.c_int64
            L.orc_mesh_nonaffine.argtypes = [P]
            L.orc_mesh_new.restype = P
            L.orc_mesh_new.argtypes = [C.c_int, C.c_int64, dp, C.c_int64, C.POINTER(C.c_int32), dp]
            L.orc_mesh_free.argtypes = [P]
            L.orc_mesh_nsides.restype = C.c_int64
            L.orc_mesh_nsides.argtypes = [P]
            L.orc_mesh_sides.argtypes = [P, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                         C.POINTER(C.c_int8), C.POINTER(C.c_int8)]
            L.orc_mesh_detj.argtypes = [P, dp]
            L.orc_color.argtypes = [P, C.c_int, C.c_uint64, C.c_int64, C.POINTER(C.c_int8),
                                    C.POINTER(C.c_int64)]
            L.orc_color_naive.argtypes = [P, C.POINTER(C.c_int8)]
            L.orc_reorder.argtypes = [P, C.c_int, C.POINTER(C.c_int8), C.POINTER(C.c_int32),
                                      C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
            L.orc_lf_flux.argtypes = [C.c_int, dp, dp, dp, dp]
            L.orc_rhs.argtypes = [P, C.c_int, C.c_int, dp, dp, dp, C.POINTER(C.c_int64), C.c_int64,
                                  C.c_int, C.c_int]
            L.orc_dt.argtypes = [P, C.c_int, dp, C.c_double, dp]
            L.orc_rk_step.argtypes = [P, C.c_int, dp, C.c_double, C.c_double, dp]
            L.orc_num_vol_points.argtypes = [C.c_int, C.c_int]
            L.orc_eval_points.argtypes = [P, C.c_int, C.c_int, dp, C.c_int, dp, dp, dp]
            L.orc_project.argtypes = [P, C.c_int, C.c_int, dp, dp]
            L.orc_refine.restype = P
            L.orc_refine.argtypes = [P, C.POINTER(C.c_int8), C.POINTER(C.c_uint8)]
            L.orc_mesh_nelem.restype = C.c_int64
            L.orc_mesh_nelem.argtypes = [P]
            L.orc_mesh_nvert.restype = C.c_int64
            L.orc_mesh_nvert.argtypes = [P]
            L.orc_mesh_elements.argtypes = [P, C.POINTER(C.c_int32), dp]
            L.orc_mesh_refined.argtypes = [P, C.POINTER(C.c_int8), C.POINTER(C.c_int8)]
            _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise RuntimeError("oracle: " + lib().orc_last_error().decode())


def gauss_jacobi(n: int, a: float = 0.0):
    x = np.zeros(n)
    w = np.zeros(n)
    _check(lib().orc_gauss_jacobi(n, a, _d(x), _d(w)))
    return x, w


def tri_rule(n: int):
    r, s, w = (np.zeros(n * n) for _ in range(3))
    _check(lib().orc_tri_rule(n, _d(r), _d(s), _d(w)))
    return r, s, w


def tet_rule(n: int):
    r, s, t, w = (np.zeros(n ** 3) for _ in range(4))
    _check(lib().orc_tet_rule(n, _d(r), _d(s), _d(t), _d(w)))
    return r, s, t, w


def quad_rule(n: int):
    r, s, w = (np.zeros(n * n) for _ in range(3))
    _check(lib().orc_quad_rule(n, _d(r), _d(s), _d(w)))
    return r, s, w


def npoly(dim: int, p: int, quad: bool = False) -> int:
    if quad:
        return (p + 1) ** 2
    return (p + 1) * (p + 2) // 2 if dim == 2 else (p + 1) * (p + 2) * (p + 3) // 6


def basis_quad(p: int, r, s):
    """Q_p tensor Legendre basis on [0,1]^2: phi, dphi/dr, dphi/ds, arrays (npts, (p+1)^2)."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    n = npoly(2, p, quad=True)
    out = [np.zeros((r.size, n)) for _ in range(3)]
    buf = [np.zeros(n) for _ in range(3)]
    for i in range(r.size):
        _check(lib().orc_basis_quad(p, float(r[i]), float(s[i]), _d(buf[0]), _d(buf[1]), _d(buf[2])))
        for k in range(3):
            out[k][i] = buf[k]
    return tuple(out)


def basis_tri(p: int, r, s):
    """phi, dphi/dr, dphi/ds at the points (r, s): arrays (npts, Np)."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    n = npoly(2, p)
    out = [np.zeros((r.size, n)) for _ in range(3)]
    buf = [np.zeros(n) for _ in range(3)]
    for i in range(r.size):
        lib().orc_basis_tri(p, float(r[i]), float(s[i]), _d(buf[0]), _d(buf[1]), _d(buf[2]))
        for k in range(3):
            out[k][i] = buf[k]
    return tuple(out)


def basis_tet(p: int, r, s, t):
    r, s, t = (np.atleast_1d(np.asarray(v, dtype=np.float64)) for v in (r, s, t))
    n = npoly(3, p)
    out = [np.zeros((r.size, n)) for _ in range(4)]
    buf = [np.zeros(n) for _ in range(4)]
    for i in range(r.size):
        lib().orc_basis_tet(p, float(r[i]), float(s[i]), float(t[i]), *(_d(b) for b in buf))
        for k in range(4):
            out[k][i] = buf[k]
    return tuple(out)


def lf_flux(dim: int, um, up, n):
    um, up, n = (np.ascontiguousarray(v, dtype=np.float64) for v in (um, up, n))
    out = np.zeros(dim + 2)
    lib().orc_lf_flux(dim, _d(um), _d(up), _d(n), _d(out))
    return out


class OracleMesh:
    """The oracle's own mesh: edge table, geometry, coloring, reordering, Eq. 2."""

    def __init__(self, dim: int, xyz: np.ndarray, ev: np.ndarray, periodic_len=None):
        self.dim = dim
        self._xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self._ev = np.ascontiguousarray(ev, dtype=np.int32)
        self.ne = int(self._ev.shape[0])
        self.quad = dim == 2 and self._ev.shape[1] == 4
        self._L = None if periodic_len is None else np.ascontiguousarray(periodic_len, dtype=np.float64)
        L = _d(self._L) if self._L is not None else None
        if self.quad:
            h = lib().orc_mesh_new_quad(self._xyz.shape[0], _d(self._xyz), self.ne, _i32(self._ev), L)
        else:
            h = lib().orc_mesh_new(dim, self._xyz.shape[0], _d(self._xyz), self.ne, _i32(self._ev), L)
        if not h:
            raise ValueError("oracle: " + lib().orc_last_error().decode())
        self._h = h
        self.ns = int(lib().orc_mesh_nsides(h))
        self.nonaffine = int(lib().orc_mesh_nonaffine(h))

    def np_modes(self, p: int) -> int:
        return npoly(self.dim, p, self.quad)

    @classmethod
    def from_input(cls, mi):
        return cls(mi.dim, mi.xyz, mi.ev, mi.periodic_len)

    def refine(self, col: np.ndarray, elems) -> "OracleMesh":
        """One level of refinement of the listed elements with the 6-color map of
        Sec. 3.2 (dg_oracle.c, orc_refine); col holds this mesh's colors 1..3.
        The new mesh carries .colors and .hanging (per side)."""
        col = np.ascontiguousarray(col, dtype=np.int8)
        flag = np.zeros(self.ne, np.uint8)
        flag[np.asarray(elems, dtype=np.int64)] = 1
        h = lib().orc_refine(self._h, _i8(col), flag.ctypes.data_as(C.POINTER(C.c_uint8)))
        if not h:
            raise ValueError("oracle: " + lib().orc_last_error().decode())
        m = OracleMesh.__new__(OracleMesh)
        m.dim = self.dim
        m.quad = False
        m.nonaffine = 0
        m._h = h
        m.ne = int(lib().orc_mesh_nelem(h))
        m.ns = int(lib().orc_mesh_nsides(h))
        m.nv = int(lib().orc_mesh_nvert(h))
        m._L = self._L
        m.colors = np.zeros(m.ns, np.int8)
        m.hanging = np.zeros(m.ns, np.int8)
        _check(lib().orc_mesh_refined(h, _i8(m.colors), _i8(m.hanging)))
        return m

    def elements(self):
        """Vertex ids [E][nvpe] and unwrapped coordinates [E][nvpe][dim] (nvpe = 4 for
        quadrilateral meshes, else dim + 1)."""
        nvpe = 4 if self.quad else self.dim + 1
        ev = np.zeros((self.ne, nvpe), np.int32)
        X = np.zeros((self.ne, nvpe, self.dim))
        lib().orc_mesh_elements(self._h, _i32(ev), _d(X))
        return ev, X

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_mesh_free(h)
            self._h = None

    @property
    def M(self) -> int:
        return self.dim + 2

    def sides(self):
        l = np.zeros(self.ns, np.int32)
        r = np.zeros(self.ns, np.int32)
        ql = np.zeros(self.ns, np.int8)
        qr = np.zeros(self.ns, np.int8)
        lib().orc_mesh_sides(self._h, _i32(l), _i32(r), _i8(ql), _i8(qr))
        return l, r, ql, qr

    def detj(self):
        d = np.zeros(self.ne)
        lib().orc_mesh_detj(self._h, _d(d))
        return d

    def color(self, nc: int, seed: int, max_swaps: int = 0):
        """Sec. 3.1 coloring.  Returns (colors int8[Ns], stats) or raises on the swap cap."""
        col = np.zeros(self.ns, np.int8)
        stats = np.zeros(4, np.int64)
        rc = lib().orc_color(self._h, nc, seed, max_swaps, _i8(col), _i64(stats))
        if rc != 0:
            raise RuntimeError("oracle: " + lib().orc_last_error().decode())
        return col, dict(greedy_conflicts=int(stats[0]), swaps=int(stats[1]),
                         breaks=int(stats[2]), deferrals=int(stats[3]))

    def color_naive(self):
        col = np.zeros(self.ns, np.int8)
        nc = lib().orc_color_naive(self._h, _i8(col))
        if nc < 0:
            raise RuntimeError("oracle: " + lib().orc_last_error().decode())
        return col, int(nc)

    def reorder(self, col: np.ndarray, nc: int):
        col = np.ascontiguousarray(col, dtype=np.int8)
        en = np.zeros(self.ne, np.int32)
        sn = np.zeros(self.ns, np.int32)
        off = np.zeros(nc + 1, np.int32)
        _check(lib().orc_reorder(self._h, nc, _i8(col), _i32(en), _i32(sn), _i32(off)))
        return en, sn, off

    def rhs(self, p: int, c: np.ndarray, elems=None, kind: int = EULER, adv=None,
            nq_face1: int = 0, nq_vol1: int = 0) -> np.ndarray:
        c = np.ascontiguousarray(c, dtype=np.float64)
        M = c.shape[1]
        n = self.np_modes(p)
        assert c.shape == (self.ne, M, n), c.shape
        if elems is None:
            out = np.zeros_like(c)
            el, ne = None, -1
        else:
            elems = np.ascontiguousarray(elems, dtype=np.int64)
            out = np.zeros((elems.size, M, n))
            el, ne = _i64(elems), elems.size
        a = None if adv is None else np.ascontiguousarray(adv, dtype=np.float64)
        _check(lib().orc_rhs(self._h, p, kind, _d(a) if a is not None else None, _d(c), _d(out),
                             el, ne, nq_face1, nq_vol1))
        return out

    def dt(self, p: int, c: np.ndarray, cfl: float) -> float:
        c = np.ascontiguousarray(c, dtype=np.float64)
        out = np.zeros(1)
        _check(lib().orc_dt(self._h, p, _d(c), cfl, _d(out)))
        return float(out[0])

    def rk_step(self, p: int, c: np.ndarray, cfl: float, dt: float = 0.0):
        """Returns (new state, dt); the input array is not modified."""
        u = np.array(c, dtype=np.float64, copy=True, order="C")
        out = np.zeros(1)
        _check(lib().orc_rk_step(self._h, p, _d(u), cfl, dt, _d(out)))
        return u, float(out[0])

    def eval_points(self, p: int, c=None, n1: int = 0, M: int | None = None):
        """Volume points (unwrapped), physical weights and, if c is given, U there."""
        M = M if M is not None else (c.shape[1] if c is not None else self.M)
        nq1 = n1 if n1 > 0 else (p + 1 if self.dim == 2 else p + 2)
        nq = nq1 ** self.dim
        xyz = np.zeros((self.ne, nq, self.dim))
        w = np.zeros((self.ne, nq))
        U = np.zeros((self.ne, nq, M)) if c is not None else None
        cc = np.ascontiguousarray(c, dtype=np.float64) if c is not None else None
        r = lib().orc_eval_points(self._h, p, M, _d(cc) if cc is not None else None, n1, _d(xyz),
                                  _d(w), _d(U) if U is not None else None)
        if r < 0:
            raise RuntimeError("oracle: " + lib().orc_last_error().decode())
        return xyz, w, U

    def project(self, p: int, vals: np.ndarray) -> np.ndarray:
        vals = np.ascontiguousarray(vals, dtype=np.float64)
        M = vals.shape[2]
        c = np.zeros((self.ne, M, self.np_modes(p)))
        _check(lib().orc_project(self._h, p, M, _d(vals), _d(c)))
        return c
