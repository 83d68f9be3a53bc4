"""CPU oracle for the colored DG right-hand side -- TEST INFRASTRUCTURE ONLY.

A plain, slow FP64 C implementation (``dg_oracle.c``) of what the CUDA path
computes: the edge table, the paper's coloring and reordering (Sec. 3.1, Sec. 5)
and the modal DG right-hand side of Eq. 2 evaluated element by element, plus the
CFL rule and SSP-RK3 step.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  Quadrilateral and
hybrid triangle/quadrilateral meshes are built from a [E][4] element list (-1 as
the fourth vertex of a triangle).  It shares no code with
``paper_1601_07613_gb300`` (the product), and the product never imports it.

This module only builds the C file with gcc (an FP64, an extended-precision and
a threaded build) and marshals numpy arrays through ctypes; all arithmetic is in
``dg_oracle.c``.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dg_oracle.c")
_lock = threading.Lock()

# The same C file in three builds:
#   "fp64"     FP64, sequential: the oracle of the tests;
#   "extended" long double arithmetic (x87 80-bit on x86-64, IEEE binary128 on
#              aarch64), sequential: the reference an FP64 evaluation's rounding
#              error is measured against;
#   "threads"  FP64, -O3, OpenMP over the elements of a right-hand side: the
#              CPU baseline on all host cores (the same arithmetic per element).
# No build uses FMA contraction or -march=native (the host code must give the
# same results on x86-64 and aarch64).
_BUILDS = {
    "fp64": ("liboracle.so", ["-O2"]),
    "extended": ("liboracle_ext.so", ["-O2", "-DORC_REAL=long double"]),
    "threads": ("liboracle_mt.so", ["-O3", "-fopenmp"]),
}
_libs: dict = {}

EULER = 0
ADVECTION = 1


def _so(kind: str) -> str:
    return os.path.join(_HERE, "_build", _BUILDS[kind][0])


def build(force: bool = False, kinds=("fp64", "extended", "threads")) -> str:
    """Compile dg_oracle.c into oracle/_build/ (gcc, no FMA contraction), one
    shared object per build kind; returns the FP64 build's path."""
    os.makedirs(os.path.join(_HERE, "_build"), exist_ok=True)
    for kind in kinds:
        so = _so(kind)
        if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
            tmp = so + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", *_BUILDS[kind][1], "-std=c11", "-fPIC", "-shared",
                                   "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, so)
    return _so("fp64")


class _Build:
    """One loaded build: the CDLL, its real type (ctypes and numpy) and the
    argument types of every exported function."""

    def __init__(self, kind: str):
        build(kinds=(kind,))
        self.kind = kind
        L = C.CDLL(_so(kind))
        L.orc_real_bytes.restype = C.c_int
        L.orc_real_mant_dig.restype = C.c_int
        ext = kind == "extended"
        self.ct = C.c_longdouble if ext else C.c_double
        self.dtype = np.longdouble if ext else np.float64
        if L.orc_real_bytes() != C.sizeof(self.ct) or np.dtype(self.dtype).itemsize != C.sizeof(self.ct):
            raise RuntimeError(f"oracle build {kind}: real type size mismatch")
        self.mant_dig = int(L.orc_real_mant_dig())
        P = C.c_void_p
        R = self.ct
        dp = C.POINTER(R)
        L.orc_last_error.restype = C.c_char_p
        L.orc_gauss_jacobi.argtypes = [C.c_int, R, dp, dp]
        L.orc_tri_rule.argtypes = [C.c_int, dp, dp, dp]
        L.orc_tet_rule.argtypes = [C.c_int, dp, dp, dp, dp]
        L.orc_basis_tri.argtypes = [C.c_int, R, R, dp, dp, dp]
        L.orc_basis_tet.argtypes = [C.c_int, R, R, R, dp, dp, dp, dp]
        L.orc_basis_quad.argtypes = [C.c_int, R, R, dp, dp, dp]
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
        L.orc_dt.argtypes = [P, C.c_int, dp, R, dp]
        L.orc_rk_step.argtypes = [P, C.c_int, dp, R, R, dp]
        L.orc_rk_step_kind.argtypes = [P, C.c_int, C.c_int, dp, dp, R, R, dp]
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
        L.orc_mesh_levels.restype = None
        L.orc_mesh_levels.argtypes = [P, C.POINTER(C.c_int8)]
        L.orc_transfer.argtypes = [P, P, C.POINTER(C.c_uint8), C.c_int, C.c_int, C.c_int, dp, dp]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_set_threads.restype = C.c_int
        i8 = C.POINTER(C.c_int8)
        L.orc_set_bc.argtypes = [P, i8, i8, C.c_int, dp, dp, i8]
        L.orc_boundary_state.argtypes = [P, C.c_int32, dp, dp, dp, dp]
        L.orc_set_time.argtypes = [P, R]
        L.orc_get_time.argtypes = [P, dp]
        L.orc_set_limiter.argtypes = [P, C.c_int]
        L.orc_limit.argtypes = [P, C.c_int, dp]
        self.L = L

    def arr(self, a):
        """a as a C-contiguous array of this build's real type."""
        return np.ascontiguousarray(a, dtype=self.dtype)

    def ptr(self, a):
        assert a.dtype == self.dtype and a.flags["C_CONTIGUOUS"]
        return a.ctypes.data_as(C.POINTER(self.ct))

    def check(self, rc):
        if rc != 0:
            raise RuntimeError(f"oracle ({self.kind}): " + self.L.orc_last_error().decode())


def get(kind: str = "fp64") -> _Build:
    """The loaded build of this kind ("fp64", "extended" or "threads")."""
    with _lock:
        if kind not in _libs:
            _libs[kind] = _Build(kind)
        return _libs[kind]


def lib():
    """The FP64 build's CDLL."""
    return get("fp64").L


def _d(a):
    return get("fp64").ptr(a)


def _i32(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _i64(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _i8(a):
    return a.ctypes.data_as(C.POINTER(C.c_int8))


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
    """The oracle's own mesh: edge table, geometry, coloring, reordering, Eq. 2.

    build: "fp64" (default), "extended" (the same steps in long double; inputs
    are converted exactly, results come back as numpy longdouble arrays) or
    "threads" (FP64, right-hand sides over all threads set by set_threads)."""

    def __init__(self, dim: int, xyz: np.ndarray, ev: np.ndarray, periodic_len=None, build: str = "fp64"):
        self._b = B = get(build)
        self.dim = dim
        self._xyz = B.arr(xyz)
        self._ev = np.ascontiguousarray(ev, dtype=np.int32)
        self.ne = int(self._ev.shape[0])
        self.quad = dim == 2 and self._ev.shape[1] == 4
        self._L = None if periodic_len is None else B.arr(periodic_len)
        L = B.ptr(self._L) if self._L is not None else None
        if self.quad:
            h = B.L.orc_mesh_new_quad(self._xyz.shape[0], B.ptr(self._xyz), self.ne, _i32(self._ev), L)
        else:
            h = B.L.orc_mesh_new(dim, self._xyz.shape[0], B.ptr(self._xyz), self.ne, _i32(self._ev), L)
        if not h:
            raise ValueError("oracle: " + B.L.orc_last_error().decode())
        self._h = h
        self.ns = int(B.L.orc_mesh_nsides(h))
        self.nonaffine = int(B.L.orc_mesh_nonaffine(h))

    @property
    def real(self):
        """numpy type of this mesh's arithmetic and results"""
        return self._b.dtype

    def np_modes(self, p: int) -> int:
        return npoly(self.dim, p, self.quad)

    @classmethod
    def from_input(cls, mi, build: str = "fp64"):
        return cls(mi.dim, mi.xyz, mi.ev, mi.periodic_len, build=build)

    def refine(self, col: np.ndarray, elems) -> "OracleMesh":
        """One level of refinement of the listed elements with the color map of
        Sec. 3.2 (dg_oracle.c, orc_refine); col holds this mesh's colors (1..3 on
        a conforming mesh; a refined mesh's .colors for a further level).  The
        new mesh carries .colors and .hanging (per side) and .levels (per
        element)."""
        B = self._b
        col = np.ascontiguousarray(col, dtype=np.int8)
        flag = np.zeros(self.ne, np.uint8)
        flag[np.asarray(elems, dtype=np.int64)] = 1
        h = B.L.orc_refine(self._h, _i8(col), flag.ctypes.data_as(C.POINTER(C.c_uint8)))
        if not h:
            raise ValueError("oracle: " + B.L.orc_last_error().decode())
        m = OracleMesh.__new__(OracleMesh)
        m._b = B
        m.dim = self.dim
        m.quad = False
        m.nonaffine = 0
        m._h = h
        m.ne = int(B.L.orc_mesh_nelem(h))
        m.ns = int(B.L.orc_mesh_nsides(h))
        m.nv = int(B.L.orc_mesh_nvert(h))
        m._L = self._L
        m._parent = self
        m._flag = flag
        m.colors = np.zeros(m.ns, np.int8)
        m.hanging = np.zeros(m.ns, np.int8)
        B.check(B.L.orc_mesh_refined(h, _i8(m.colors), _i8(m.hanging)))
        m.levels = np.zeros(m.ne, np.int8)
        B.L.orc_mesh_levels(h, _i8(m.levels))
        return m

    def prolong(self, p: int, c_coarse: np.ndarray) -> np.ndarray:
        """For a mesh made by refine(): the parent mesh's state [E0][M][Np] projected
        onto this mesh (each child the L2 projection of its parent's polynomial)."""
        B = self._b
        c = B.arr(c_coarse)
        out = np.zeros((self.ne, c.shape[1], c.shape[2]), self.real)
        B.check(B.L.orc_transfer(self._parent._h, self._h, self._flag.ctypes.data_as(C.POINTER(C.c_uint8)), p,
                                 c.shape[1], 0, B.ptr(c), B.ptr(out)))
        return out

    def restrict(self, p: int, c_fine: np.ndarray) -> np.ndarray:
        """For a mesh made by refine(): this mesh's state projected onto the parent mesh
        (each parent the L2 projection of its children's piecewise polynomial)."""
        B = self._b
        c = B.arr(c_fine)
        out = np.zeros((self._parent.ne, c.shape[1], c.shape[2]), self.real)
        B.check(B.L.orc_transfer(self._parent._h, self._h, self._flag.ctypes.data_as(C.POINTER(C.c_uint8)), p,
                                 c.shape[1], 1, B.ptr(c), B.ptr(out)))
        return out

    def elements(self):
        """Vertex ids [E][nvpe] and unwrapped coordinates [E][nvpe][dim] (nvpe = 4 for
        quadrilateral meshes, else dim + 1)."""
        nvpe = 4 if self.quad else self.dim + 1
        ev = np.zeros((self.ne, nvpe), np.int32)
        X = np.zeros((self.ne, nvpe, self.dim), self.real)
        self._b.L.orc_mesh_elements(self._h, _i32(ev), self._b.ptr(X))
        return ev, X

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._b.L.orc_mesh_free(h)
            self._h = None

    @property
    def M(self) -> int:
        return self.dim + 2

    def sides(self):
        l = np.zeros(self.ns, np.int32)
        r = np.zeros(self.ns, np.int32)
        ql = np.zeros(self.ns, np.int8)
        qr = np.zeros(self.ns, np.int8)
        self._b.L.orc_mesh_sides(self._h, _i32(l), _i32(r), _i8(ql), _i8(qr))
        return l, r, ql, qr

    def detj(self):
        d = np.zeros(self.ne, self.real)
        self._b.L.orc_mesh_detj(self._h, self._b.ptr(d))
        return d

    def color(self, nc: int, seed: int, max_swaps: int = 0):
        """Sec. 3.1 coloring.  Returns (colors int8[Ns], stats) or raises on the swap cap."""
        col = np.zeros(self.ns, np.int8)
        stats = np.zeros(4, np.int64)
        self._b.check(self._b.L.orc_color(self._h, nc, seed, max_swaps, _i8(col), _i64(stats)))
        return col, dict(greedy_conflicts=int(stats[0]), swaps=int(stats[1]),
                         breaks=int(stats[2]), deferrals=int(stats[3]))

    def color_naive(self):
        col = np.zeros(self.ns, np.int8)
        nc = self._b.L.orc_color_naive(self._h, _i8(col))
        if nc < 0:
            raise RuntimeError("oracle: " + self._b.L.orc_last_error().decode())
        return col, int(nc)

    def reorder(self, col: np.ndarray, nc: int):
        col = np.ascontiguousarray(col, dtype=np.int8)
        en = np.zeros(self.ne, np.int32)
        sn = np.zeros(self.ns, np.int32)
        off = np.zeros(nc + 1, np.int32)
        self._b.check(self._b.L.orc_reorder(self._h, nc, _i8(col), _i32(en), _i32(sn), _i32(off)))
        return en, sn, off

    def rhs(self, p: int, c: np.ndarray, elems=None, kind: int = EULER, adv=None,
            nq_face1: int = 0, nq_vol1: int = 0) -> np.ndarray:
        B = self._b
        c = B.arr(c)
        M = c.shape[1]
        n = self.np_modes(p)
        assert c.shape == (self.ne, M, n), c.shape
        if elems is None:
            out = np.zeros_like(c)
            el, ne = None, -1
        else:
            elems = np.ascontiguousarray(elems, dtype=np.int64)
            out = np.zeros((elems.size, M, n), self.real)
            el, ne = _i64(elems), elems.size
        a = None if adv is None else B.arr(adv)
        B.check(B.L.orc_rhs(self._h, p, kind, B.ptr(a) if a is not None else None, B.ptr(c), B.ptr(out),
                            el, ne, nq_face1, nq_vol1))
        return out

    def dt(self, p: int, c: np.ndarray, cfl: float) -> float:
        B = self._b
        c = B.arr(c)
        out = np.zeros(1, self.real)
        B.check(B.L.orc_dt(self._h, p, B.ptr(c), cfl, B.ptr(out)))
        return float(out[0])

    def rk_step(self, p: int, c: np.ndarray, cfl: float, dt: float = 0.0, kind: int = EULER, adv=None):
        """One SSP-RK3 step: returns (new state, dt); the input array is not
        modified.  kind=ADVECTION (one equation, velocity adv) needs dt > 0."""
        B = self._b
        u = np.array(c, dtype=self.real, copy=True, order="C")
        out = np.zeros(1, self.real)
        a = None if adv is None else B.arr(adv)
        B.check(B.L.orc_rk_step_kind(self._h, p, kind, B.ptr(a) if a is not None else None, B.ptr(u), cfl, dt,
                                     B.ptr(out)))
        return u, float(out[0])

    # boundary conditions, time and limiter (triangle meshes; dg_oracle.c
    # orc_set_bc, orc_limit)
    BC_TRANSMISSIVE, BC_WALL, BC_STATE, BC_SHOCK = 0, 1, 2, 3

    def set_bc(self, kind, sidx=None, states=None, shock=None, shock_states=None):
        """kind[s] per side (boundary sides only matter), sidx[s] the state of a
        BC_STATE side, states [n][4], shock (a, b, c): the state shock_states[0]
        where x < a + b y + c t, else shock_states[1]."""
        B = self._b
        kind = np.ascontiguousarray(kind, dtype=np.int8)
        assert kind.shape == (self.ns,)
        sidx = None if sidx is None else np.ascontiguousarray(sidx, dtype=np.int8)
        st = B.arr(np.zeros((0, 4)) if states is None else np.asarray(states).reshape(-1, 4))
        sh = None if shock is None else B.arr(shock)
        ss = None if shock_states is None else np.ascontiguousarray(shock_states, dtype=np.int8)
        B.check(B.L.orc_set_bc(self._h, _i8(kind), _i8(sidx) if sidx is not None else None, st.shape[0],
                               B.ptr(st) if st.size else None, B.ptr(sh) if sh is not None else None,
                               _i8(ss) if ss is not None else None))

    def boundary_state(self, s: int, Um, n, x):
        B = self._b
        Um, n, x = B.arr(Um), B.arr(n), B.arr(x)
        out = np.zeros(4, self.real)
        B.check(B.L.orc_boundary_state(self._h, int(s), B.ptr(Um), B.ptr(n), B.ptr(x), B.ptr(out)))
        return out

    def set_time(self, t: float):
        self._b.check(self._b.L.orc_set_time(self._h, t))

    def time(self) -> float:
        out = np.zeros(1, self.real)
        self._b.check(self._b.L.orc_get_time(self._h, self._b.ptr(out)))
        return float(out[0])

    def set_limiter(self, on: bool):
        self._b.check(self._b.L.orc_set_limiter(self._h, int(bool(on))))

    def limit(self, p: int, c: np.ndarray) -> np.ndarray:
        """The limited copy of state c (the limiter alone, as after an RK stage)."""
        B = self._b
        u = np.array(c, dtype=self.real, copy=True, order="C")
        B.check(B.L.orc_limit(self._h, p, B.ptr(u)))
        return u

    def eval_points(self, p: int, c=None, n1: int = 0, M: int | None = None):
        """Volume points (unwrapped), physical weights and, if c is given, U there."""
        B = self._b
        M = M if M is not None else (c.shape[1] if c is not None else self.M)
        nq1 = n1 if n1 > 0 else (p + 1 if self.dim == 2 else p + 2)
        nq = nq1 ** self.dim
        xyz = np.zeros((self.ne, nq, self.dim), self.real)
        w = np.zeros((self.ne, nq), self.real)
        U = np.zeros((self.ne, nq, M), self.real) if c is not None else None
        cc = B.arr(c) if c is not None else None
        r = B.L.orc_eval_points(self._h, p, M, B.ptr(cc) if cc is not None else None, n1, B.ptr(xyz),
                                B.ptr(w), B.ptr(U) if U is not None else None)
        if r < 0:
            raise RuntimeError("oracle: " + B.L.orc_last_error().decode())
        return xyz, w, U

    def project(self, p: int, vals: np.ndarray) -> np.ndarray:
        B = self._b
        vals = B.arr(vals)
        M = vals.shape[2]
        c = np.zeros((self.ne, M, self.np_modes(p)), self.real)
        B.check(B.L.orc_project(self._h, p, M, B.ptr(vals), B.ptr(c)))
        return c


def set_threads(n: int) -> int:
    """Threads of the "threads" build's right-hand side (0: leave as is);
    returns the count in effect."""
    return int(get("threads").L.orc_set_threads(int(n)))
