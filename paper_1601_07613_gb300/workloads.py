"""Seeded synthetic inputs shared by the library's callers, the tests and the bench.

This module only *generates inputs*: mesh vertex/element lists, random modal
coefficient arrays and the point values of the isentropic-vortex field.  It
contains none of the DG method's arithmetic (no basis, quadrature, geometry,
flux, coloring or time stepping), so the CUDA path and the CPU oracle can both
draw their inputs from here without sharing any of the computation they are
checked on.

The paper's meshes (rectangles A-E, NACA-0012, spherical shells, Table 1-3) are
not available; the generators below build meshes of the same kind and scale:

* ``periodic_square_tri``: an ``n x n`` periodic unit square, every grid square
  split into two triangles, optionally with every vertex jittered uniformly by
  up to ``jitter * h`` in x and y.  Periodic meshes have no boundary, so every
  element has exactly one edge of each color, as for the closed spherical
  meshes of Table 1.
* ``open_square_tri``: the same split on a non-periodic square (boundary edges).
* ``periodic_cube_tet``: an ``n^3`` periodic unit cube, each cube split into six
  tetrahedra along its main diagonal (Kuhn/Freudenthal split).
* ``periodic_square_quad`` / ``open_square_quad``: ``n x n`` quadrilaterals on
  the unit square (Table 2's rectangular domains).  ``mode="parallelogram"``
  jitters the grid lines and shifts every row of vertices sideways, so every
  element is a parallelogram of its own width, height and slant;
  ``mode="vertex"`` jitters every vertex (general convex quadrilaterals,
  colored only).
* ``hybrid_square``: the quadrilateral grid with a seeded fraction of its
  squares split into two triangles (Table 2's hybrid tri/quad mesh).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 1.4


@dataclass
class MeshInput:
    """Vertex and element lists in the layout ``dgc_mesh_create`` takes."""

    dim: int
    xyz: np.ndarray  # (nv, dim) float64
    # (ne, dim+1) int32, CCW triangles / positive-volume tets; (ne, 4) CCW
    # quadrilaterals, -1 as the fourth id of a triangle of a hybrid mesh
    ev: np.ndarray
    periodic_len: np.ndarray | None  # (dim,) float64 or None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def ne(self) -> int:
        return int(self.ev.shape[0])

    @property
    def nv(self) -> int:
        return int(self.xyz.shape[0])


def periodic_square_tri(n: int, jitter: float = 0.0, seed: int | None = None) -> MeshInput:
    """``n x n`` periodic unit square, each square split into two CCW triangles.

    Vertex (i, j) has id ``j*n + i`` and sits at ``(i/n, j/n)`` (plus jitter);
    vertex ids wrap, so periodic edges are shared by vertex id.  Square (i, j),
    numbered j-major, becomes [(i,j), (i+1,j), (i+1,j+1)] and
    [(i,j), (i+1,j+1), (i,j+1)].  ``n >= 3`` keeps every edge key unique.
    """
    if n < 3:
        raise ValueError("periodic meshes need n >= 3")
    h = 1.0 / n
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    xyz = np.stack([ii.ravel() * h, jj.ravel() * h], axis=1).astype(np.float64)
    if jitter:
        rng = np.random.default_rng(seed)
        xyz += rng.uniform(-jitter * h, jitter * h, size=xyz.shape)

    def vid(i, j):
        return (j % n) * n + (i % n)

    i = ii.ravel()
    j = jj.ravel()
    a = vid(i, j)
    b = vid(i + 1, j)
    c = vid(i + 1, j + 1)
    d = vid(i, j + 1)
    ev = np.empty((2 * n * n, 3), dtype=np.int32)
    ev[0::2] = np.stack([a, b, c], axis=1)
    ev[1::2] = np.stack([a, c, d], axis=1)
    return MeshInput(2, xyz, ev, np.array([1.0, 1.0]), name=f"periodic_square_tri_{n}x{n}",
                     meta={"n": n, "jitter": jitter, "seed": seed})


def open_square_tri(n: int, jitter: float = 0.0, seed: int | None = None) -> MeshInput:
    """Non-periodic ``n x n`` unit square split like ``periodic_square_tri``.

    It has ``(n+1)^2`` vertices and ``4n`` boundary edges.  Only interior
    vertices are jittered.
    """
    h = 1.0 / n
    ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")
    xyz = np.stack([ii.ravel() * h, jj.ravel() * h], axis=1).astype(np.float64)
    if jitter:
        rng = np.random.default_rng(seed)
        d = rng.uniform(-jitter * h, jitter * h, size=xyz.shape)
        interior = ((ii.ravel() > 0) & (ii.ravel() < n) & (jj.ravel() > 0) & (jj.ravel() < n))
        xyz[interior] += d[interior]
    ci, cj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    i = ci.ravel()
    j = cj.ravel()

    def vid(i, j):
        return j * (n + 1) + i

    a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
    ev = np.empty((2 * n * n, 3), dtype=np.int32)
    ev[0::2] = np.stack([a, b, c], axis=1)
    ev[1::2] = np.stack([a, c, d], axis=1)
    return MeshInput(2, xyz, ev, None, name=f"open_square_tri_{n}x{n}", meta={"n": n})


def open_rect_tri(nx: int, ny: int, lx: float, ly: float, jitter: float = 0.0,
                  seed: int | None = None) -> MeshInput:
    """Non-periodic ``nx x ny`` rectangle [0, lx] x [0, ly] of cells split into
    two triangles each as in ``open_square_tri``; only interior vertices are
    jittered (by ``U(-jitter h, jitter h)`` per axis, h the cell size along that
    axis), so the four sides stay straight."""
    hx, hy = lx / nx, ly / ny
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
    xyz = np.stack([ii.ravel() * hx, jj.ravel() * hy], axis=1).astype(np.float64)
    if jitter:
        rng = np.random.default_rng(seed)
        d = rng.uniform(-jitter, jitter, size=xyz.shape) * np.array([hx, hy])
        interior = (ii.ravel() > 0) & (ii.ravel() < nx) & (jj.ravel() > 0) & (jj.ravel() < ny)
        xyz[interior] += d[interior]
    ci, cj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    i, j = ci.ravel(), cj.ravel()

    def vid(i, j):
        return j * (nx + 1) + i

    a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
    ev = np.empty((2 * nx * ny, 3), dtype=np.int32)
    ev[0::2] = np.stack([a, b, c], axis=1)
    ev[1::2] = np.stack([a, c, d], axis=1)
    return MeshInput(2, xyz, ev, None, name=f"open_rect_tri_{nx}x{ny}", meta={"nx": nx, "ny": ny})


def _quad_grid(n: int, periodic: bool, mode: str, jitter: float, slant: float, seed):
    nn = n if periodic else n + 1
    h = 1.0 / n
    rng = np.random.default_rng(seed)
    ii, jj = np.meshgrid(np.arange(nn), np.arange(nn), indexing="xy")
    i, j = ii.ravel(), jj.ravel()
    inner_x = (i > 0) & (i < n) if not periodic else np.ones(i.size, bool)
    inner_y = (j > 0) & (j < n) if not periodic else np.ones(j.size, bool)
    if mode == "parallelogram":
        # column lines x_i, row lines y_j, row shifts s_j (zero on open boundary rows)
        xl = np.arange(nn) * h + (rng.uniform(-jitter * h, jitter * h, nn) if jitter else 0.0)
        yl = np.arange(nn) * h + (rng.uniform(-jitter * h, jitter * h, nn) if jitter else 0.0)
        sl = rng.uniform(-slant * h, slant * h, nn) if slant else np.zeros(nn)
        if not periodic:
            xl[[0, n]] = [0.0, 1.0]
            yl[[0, n]] = [0.0, 1.0]
            sl[[0, n]] = 0.0
        x = xl[i] + np.where(inner_x, sl[j], 0.0)
        y = yl[j]
        xyz = np.stack([x, y], axis=1)
    elif mode == "vertex":
        xyz = np.stack([i * h, j * h], axis=1).astype(np.float64)
        if jitter:
            d = rng.uniform(-jitter * h, jitter * h, size=xyz.shape)
            xyz[:, 0] += np.where(inner_x, d[:, 0], 0.0)
            xyz[:, 1] += np.where(inner_y, d[:, 1], 0.0)
    else:
        raise ValueError(mode)

    def vid(a, b):
        return (b % nn) * nn + (a % nn)

    ci, cj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    a, b = ci.ravel(), cj.ravel()
    ev = np.stack([vid(a, b), vid(a + 1, b), vid(a + 1, b + 1), vid(a, b + 1)], axis=1).astype(np.int32)
    return xyz.astype(np.float64), ev


def periodic_square_quad(n: int, mode: str = "parallelogram", jitter: float = 0.0, slant: float = 0.0,
                         seed: int | None = None) -> MeshInput:
    """``n x n`` periodic quadrilaterals, square (i, j) numbered j-major as
    [(i,j), (i+1,j), (i+1,j+1), (i,j+1)] (CCW).  Vertex (i, j) has id ``j*n + i``.

    ``mode="parallelogram"``: column line i at ``i h + U(-jitter h, jitter h)``,
    row line j likewise, and row j of vertices shifted by ``U(-slant h, slant h)``
    in x, so every element is a parallelogram.  ``mode="vertex"``: every vertex
    jittered by ``U(-jitter h, jitter h)`` in x and y.  ``n >= 3``.
    """
    if n < 3:
        raise ValueError("periodic meshes need n >= 3")
    xyz, ev = _quad_grid(n, True, mode, jitter, slant, seed)
    return MeshInput(2, xyz, ev, np.array([1.0, 1.0]), name=f"periodic_square_quad_{n}x{n}",
                     meta={"n": n, "mode": mode, "jitter": jitter, "slant": slant, "seed": seed})


def open_square_quad(n: int, mode: str = "parallelogram", jitter: float = 0.0, slant: float = 0.0,
                     seed: int | None = None) -> MeshInput:
    """Non-periodic ``n x n`` quadrilaterals on the unit square, ``(n+1)^2`` vertices;
    boundary vertices stay on the boundary.  With ``slant`` the interior columns of
    each row are shifted (the elements next to x = 0 and x = 1 are then general
    quadrilaterals), so open parallelogram meshes use ``slant=0``."""
    xyz, ev = _quad_grid(n, False, mode, jitter, slant, seed)
    return MeshInput(2, xyz, ev, None, name=f"open_square_quad_{n}x{n}",
                     meta={"n": n, "mode": mode, "jitter": jitter, "slant": slant, "seed": seed})


def hybrid_square(n: int, frac: float = 0.25, periodic: bool = True, jitter: float = 0.0,
                  seed: int | None = None, mode: str = "vertex", slant: float = 0.0) -> MeshInput:
    """The ``n x n`` quadrilateral grid (``mode`` as for ``periodic_square_quad``:
    "vertex" jitters every vertex, "parallelogram" keeps every cell a
    parallelogram) with a seeded fraction ``frac`` of its cells split along the
    diagonal (i,j)-(i+1,j+1) into two CCW triangles, listed with -1 as their fourth
    vertex.  Elements are numbered cell by cell, a split cell's two triangles in
    place of the cell."""
    base = (periodic_square_quad(n, mode, jitter, slant, seed=seed) if periodic
            else open_square_quad(n, mode, jitter, slant, seed=seed))
    rng = np.random.default_rng(None if seed is None else seed + 1)
    split = rng.uniform(size=n * n) < frac
    rows = []
    for e in range(n * n):
        a, b, c, d = base.ev[e]
        if split[e]:
            rows.append((a, b, c, -1))
            rows.append((a, c, d, -1))
        else:
            rows.append((a, b, c, d))
    ev = np.array(rows, dtype=np.int32)
    return MeshInput(2, base.xyz, ev, base.periodic_len, name=f"hybrid_square_{n}x{n}",
                     meta={"n": n, "frac": frac, "periodic": periodic, "seed": seed, "mode": mode})


# The six tetrahedra of the Kuhn split of the unit cube: the path 000 -> 111
# visits the axes in the order of each permutation.
_KUHN_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def periodic_cube_tet(n: int) -> MeshInput:
    """``n^3`` periodic unit cube, each cube split into six Kuhn tetrahedra.

    Vertex (i, j, k) has id ``(k*n + j)*n + i``.  Each tetrahedron is the
    monotone path 000 -> 111 along one permutation of the axes; vertices are
    ordered so that the volume is positive.
    """
    if n < 3:
        raise ValueError("periodic meshes need n >= 3")
    h = 1.0 / n
    g = np.arange(n)
    kk, jj, ii = np.meshgrid(g, g, g, indexing="ij")
    xyz = np.stack([ii.ravel() * h, jj.ravel() * h, kk.ravel() * h], axis=1).astype(np.float64)
    cells = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)  # cube-major (k, j, i)

    def vid(p):
        return ((p[:, 2] % n) * n + (p[:, 1] % n)) * n + (p[:, 0] % n)

    tets = []
    for perm in _KUHN_PERMS:
        p0 = cells.copy()
        p1 = p0.copy()
        p1[:, perm[0]] += 1
        p2 = p1.copy()
        p2[:, perm[1]] += 1
        p3 = p2.copy()
        p3[:, perm[2]] += 1
        verts = [vid(p0), vid(p1), vid(p2), vid(p3)]
        # orientation: the sign of the permutation decides the volume sign
        e1 = np.eye(3)[perm[0]]
        e2 = e1 + np.eye(3)[perm[1]]
        e3 = np.ones(3)
        vol = np.linalg.det(np.stack([e1, e2, e3]))
        if vol < 0:
            verts[1], verts[2] = verts[2], verts[1]
        tets.append(np.stack(verts, axis=1))
    ev = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return MeshInput(3, xyz, ev, np.array([1.0, 1.0, 1.0]), name=f"periodic_cube_tet_{n}^3x6",
                     meta={"n": n})


def open_cube_tet(n: int, jitter: float = 0.0, seed: int | None = None) -> MeshInput:
    """Non-periodic ``n^3`` unit cube split like ``periodic_cube_tet``.

    It has ``(n+1)^3`` vertices and boundary faces on the six sides; only
    interior vertices are jittered.
    """
    h = 1.0 / n
    g = np.arange(n + 1)
    kk, jj, ii = np.meshgrid(g, g, g, indexing="ij")
    xyz = np.stack([ii.ravel() * h, jj.ravel() * h, kk.ravel() * h], axis=1).astype(np.float64)
    if jitter:
        rng = np.random.default_rng(seed)
        d = rng.uniform(-jitter * h, jitter * h, size=xyz.shape)
        inner = np.all((xyz > 0.5 * h) & (xyz < 1.0 - 0.5 * h), axis=1)
        xyz[inner] += d[inner]
    c = np.arange(n)
    ck, cj, ci = np.meshgrid(c, c, c, indexing="ij")
    cells = np.stack([ci.ravel(), cj.ravel(), ck.ravel()], axis=1)

    def vid(p):
        return (p[:, 2] * (n + 1) + p[:, 1]) * (n + 1) + p[:, 0]

    tets = []
    for perm in _KUHN_PERMS:
        p0 = cells.copy()
        p1 = p0.copy()
        p1[:, perm[0]] += 1
        p2 = p1.copy()
        p2[:, perm[1]] += 1
        p3 = p2.copy()
        p3[:, perm[2]] += 1
        verts = [vid(p0), vid(p1), vid(p2), vid(p3)]
        e1 = np.eye(3)[perm[0]]
        e2 = e1 + np.eye(3)[perm[1]]
        if np.linalg.det(np.stack([e1, e2, np.ones(3)])) < 0:
            verts[1], verts[2] = verts[2], verts[1]
        tets.append(np.stack(verts, axis=1))
    ev = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return MeshInput(3, xyz, ev, None, name=f"open_cube_tet_{n}^3x6", meta={"n": n})


def random_state(ne: int, m: int, np_: int, seed: int, amp: float = 3e-3,
                 mean=(0.7, 0.1, -0.05, 1.8), spread: float = 0.05) -> np.ndarray:
    """Random modal coefficients ``c[e][m][j]`` (float64), with a positive mean mode.

    Mode 0 of each component is ``mean[m]`` plus a uniform spread; the higher
    modes are uniform in ``(-amp, amp)``.  With the defaults the state stays
    well inside the physical region (positive density and pressure).
    """
    rng = np.random.default_rng(seed)
    c = rng.uniform(-amp, amp, size=(ne, m, np_))
    mean = np.asarray(mean, dtype=np.float64)
    if mean.size != m:
        mean = np.resize(mean, m)
    c[:, :, 0] = mean[None, :] * (1.0 + rng.uniform(-spread, spread, size=(ne, m)))
    return np.ascontiguousarray(c)


def uniform_perturbation(shape, seed: int, amp: float = 1e-3) -> np.ndarray:
    """Uniform ``(-amp, amp)`` perturbation added to projected coefficients."""
    return np.random.default_rng(seed).uniform(-amp, amp, size=shape)


def vortex_field(x: np.ndarray, y: np.ndarray, t: float = 0.0, beta: float = 5.0,
                 xc: float = 0.5, yc: float = 0.5, uinf: float = 1.0, vinf: float = 1.0,
                 radius: float = 0.1, period: float = 1.0, gamma: float = GAMMA) -> np.ndarray:
    """Conserved variables of the isentropic vortex at points (x, y), time t.

    The classic vortex on ``[-5, 5]^2`` is scaled by ``radius`` onto the
    periodic unit square and advected with ``(uinf, vinf)``; the distance to the
    centre is taken on the nearest periodic image.  Returns an array of shape
    ``x.shape + (4,)`` holding ``(rho, rho u, rho v, E)``.
    """
    dx = x - xc - uinf * t
    dy = y - yc - vinf * t
    dx = dx - period * np.round(dx / period)
    dy = dy - period * np.round(dy / period)
    xt = dx / radius
    yt = dy / radius
    f = np.exp(0.5 * (1.0 - xt * xt - yt * yt))
    rho = (1.0 - (gamma - 1.0) * beta * beta / (8.0 * gamma * math.pi ** 2) * f * f) ** (1.0 / (gamma - 1.0))
    u = uinf - beta / (2.0 * math.pi) * yt * f
    v = vinf + beta / (2.0 * math.pi) * xt * f
    p = rho ** gamma
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E], axis=-1)


def vortex_tube_field(x, y, z, t: float = 0.0, **kw) -> np.ndarray:
    """3D isentropic vortex tube: the 2D vortex in (x, y), w = 0, constant in z.

    Returns ``(rho, rho u, rho v, rho w, E)`` of shape ``x.shape + (5,)``.
    """
    q = vortex_field(x, y, t, **kw)
    out = np.zeros(q.shape[:-1] + (5,), dtype=np.float64)
    out[..., 0:3] = q[..., 0:3]
    out[..., 4] = q[..., 3]
    return out


# --- Named workloads (sizes as stated) -------------------------------------------------

def square_vortex_p1_32x32() -> dict:
    """2048-triangle periodic square, p=1, vortex beta=5 at the centre, CFL 0.3, 100 RK3 steps."""
    return dict(mesh=periodic_square_tri(32), p=1, beta=5.0, xc=0.5, yc=0.5, cfl=0.3, steps=100)


def jittered_square_vortex_p3_724x724(n: int = 724) -> dict:
    """1,048,352-triangle periodic square (724x724, nodes jittered +-0.2h, seed 1601), p=3.

    Initial state: vortex beta=5 at the centre, projected, plus a uniform
    (-1e-3, 1e-3) perturbation of every coefficient (seed 7613).
    """
    return dict(mesh=periodic_square_tri(n, jitter=0.2, seed=1601), p=3, beta=5.0, xc=0.5,
                yc=0.5, perturb=1e-3, perturb_seed=7613, cfl=0.3)


def quad_square_vortex_p3_810(n: int = 810) -> dict:
    """656,100 periodic parallelograms (810x810: grid lines jittered +-0.2h, rows
    shifted +-0.3h, seed 1601), p = 3 (16 modes, 41,990,400 scalar DOFs, the DOF
    count of the 724x724 triangle workload).  State: vortex beta = 5 at the centre,
    projected, plus U(-1e-3, 1e-3) on every coefficient (seed 7613)."""
    return dict(mesh=periodic_square_quad(n, jitter=0.2, slant=0.3, seed=1601), p=3, beta=5.0, xc=0.5,
                yc=0.5, perturb=1e-3, seed=7613, cfl=0.3)


def cube_tube_p2_64(n: int = 64) -> dict:
    """64^3 periodic cube x 6 Kuhn tets = 1,572,864 tets, p=2, vortex tube."""
    return dict(mesh=periodic_cube_tet(n), p=2, beta=5.0, xc=0.5, yc=0.5, cfl=0.3)


def elements_near(mi: MeshInput, center, radius: float) -> np.ndarray:
    """Ids of the elements whose centroid lies within ``radius`` of ``center``
    (centroids of the element's vertices unwrapped next to its first vertex)."""
    X = mi.xyz[mi.ev]  # [E][nvpe][dim]
    if mi.periodic_len is not None:
        L = np.asarray(mi.periodic_len)
        X = X - L * np.round((X - X[:, :1, :]) / L)
    cen = X.mean(axis=1)
    d = cen - np.asarray(center, dtype=np.float64)
    return np.nonzero((d * d).sum(axis=1) < radius * radius)[0].astype(np.int32)


def refined_square_vortex_p2_256(n: int = 256, radius: float = 0.2) -> dict:
    """Nonconforming workload: the periodic n x n x 2 triangle mesh, every
    element whose centroid lies within ``radius`` of the vortex centre split
    once into four (Sec. 3.2); p = 2, vortex strength 5, CFL 0.3."""
    mi = periodic_square_tri(n)
    return dict(mesh=mi, refine=elements_near(mi, (0.5, 0.5), radius), p=2, beta=5.0,
                xc=0.5, yc=0.5, cfl=0.3, steps=200)


def second_level_elements(refined, ne0: int, left, right, hanging, xyz, center, radius: float,
                          coarse_radius: float) -> np.ndarray:
    """The elements to refine a second time after one refinement of the elements
    ``refined`` of an ``ne0``-element mesh (ids in the refined mesh's expanded
    order, as the library numbers them): children (level 1) with no coarser
    neighbour -- the fine side of no hanging edge, so adjacent elements still
    differ by at most one level -- whose centroid lies within ``radius`` of
    ``center``, and coarse elements beside hanging halves within
    ``coarse_radius`` and right of ``center``.  left, right, hanging: the refined
    mesh's sides (dgc_get_sides, dgc_get_hanging); xyz: its elements' vertex
    coordinates [E][3][2] (dgc_get_elements)."""
    flag = np.zeros(ne0, bool)
    flag[np.asarray(refined, dtype=np.int64)] = True
    level = np.repeat(flag.astype(np.int8), np.where(flag, 4, 1))
    hang = np.asarray(hanging) >= 0
    fine = np.zeros(level.size, bool)
    fine[np.asarray(left)[hang]] = True
    coarse = np.zeros(level.size, bool)
    coarse[np.asarray(right)[hang]] = True
    d = np.asarray(xyz).mean(axis=1) - np.asarray(center, dtype=np.float64)
    d2 = (d * d).sum(axis=1)
    sel = ((level == 1) & ~fine & (d2 < radius * radius)) | (coarse & (d2 < coarse_radius ** 2) & (d[:, 0] > 0))
    return np.nonzero(sel)[0].astype(np.int32)


def hybrid_square_vortex_p3_512(n: int = 512, frac: float = 0.3) -> dict:
    """Hybrid workload (Table 2's hybrid mesh at benchmark scale): the periodic
    n x n parallelogram grid with a fraction ``frac`` of its cells split into two
    triangles (about 340,000 elements at n = 512), p = 3, vortex strength 5."""
    mi = hybrid_square(n, frac, periodic=True, jitter=0.2, slant=0.3, seed=8, mode="parallelogram")
    return dict(mesh=mi, p=3, beta=5.0, cfl=0.3)


def bilinear_square_vortex_p3_512(n: int = 512) -> dict:
    """General-quadrilateral workload: the periodic n x n grid with every vertex
    jittered by U(-0.2 h, 0.2 h) (bilinear elements, 262,144 at n = 512), p = 3,
    vortex strength 5."""
    mi = periodic_square_quad(n, "vertex", 0.2, seed=9)
    return dict(mesh=mi, p=3, beta=5.0, cfl=0.3)


# ---------------------------------------------------------------------------
# Double Mach reflection (Sec. 5 times Table 7 on it: mesh D, 627,326 triangles,
# p = 1, 1000 steps; the setup is [giuliani]'s and not in the paper; this is the
# standard one of Woodward and Colella): a Mach 10 shock in air (gamma = 1.4)
# at 60 degrees to a reflecting wall y = 0, x >= 1/6, on [0, 4] x [0, 1].
# ---------------------------------------------------------------------------
BC_TRANSMISSIVE, BC_WALL, BC_STATE, BC_SHOCK = 0, 1, 2, 3
DMR_SHOCK = (1.0 / 6.0, 1.0 / np.sqrt(3.0), 20.0 / np.sqrt(3.0))  # x_s = a + b y + c t


def _conserved(rho, u, v, p, gamma=1.4):
    return np.array([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def double_mach_states() -> np.ndarray:
    """[2][4] conserved states: 0 behind the shock (rho 8, p 116.5, speed 8.25
    at -30 degrees), 1 ahead of it (rho 1.4, p 1, at rest)."""
    return np.stack([_conserved(8.0, 8.25 * np.cos(np.pi / 6), -8.25 * np.sin(np.pi / 6), 116.5),
                     _conserved(1.4, 0.0, 0.0, 1.0)])


def double_mach_field(x: np.ndarray, y: np.ndarray, t: float = 0.0) -> np.ndarray:
    """The shock's two states on either side of x_s(y, t): [..., 4]."""
    S = double_mach_states()
    a, b, c = DMR_SHOCK
    behind = x < a + b * y + c * t
    return np.where(behind[..., None], S[0], S[1])


def double_mach_boundary(mi: MeshInput, left: np.ndarray, right: np.ndarray, qleft: np.ndarray):
    """Boundary kind and state index per side (sides as both the library and the
    oracle list them: left/right element, local face of the left), from each
    boundary face's midpoint: the bottom up to x = 1/6 and the left side take
    the state behind the shock, the bottom beyond it is a slip wall, the top
    follows the moving shock (states 0 behind, 1 ahead), the right side is
    transmissive."""
    kind = np.zeros(left.size, np.int8)
    sidx = np.zeros(left.size, np.int8)
    b = np.nonzero(right < 0)[0]
    v0 = mi.ev[left[b], qleft[b]]
    v1 = mi.ev[left[b], (qleft[b] + 1) % 3]
    mid = 0.5 * (mi.xyz[v0] + mi.xyz[v1])
    lx = mi.xyz[:, 0].max()
    ly = mi.xyz[:, 1].max()
    tol = 1e-9
    k = np.full(b.size, BC_TRANSMISSIVE, np.int8)
    bottom, top = mid[:, 1] < tol, mid[:, 1] > ly - tol
    leftb, rightb = mid[:, 0] < tol, mid[:, 0] > lx - tol
    k[bottom & (mid[:, 0] < DMR_SHOCK[0])] = BC_STATE
    k[bottom & (mid[:, 0] >= DMR_SHOCK[0])] = BC_WALL
    k[top] = BC_SHOCK
    k[leftb & ~bottom & ~top] = BC_STATE
    k[rightb & ~bottom & ~top] = BC_TRANSMISSIVE
    kind[b] = k
    return kind, sidx


def double_mach_p1(ny: int = 280) -> dict:
    """The double Mach workload: [0, 4] x [0, 1] as 4 ny x ny cells of two
    jittered triangles (627,200 at ny = 280, mesh D's size), p = 1, the shock
    states of ``double_mach_states`` at t = 0, CFL 0.3, the limiter on."""
    mi = open_rect_tri(4 * ny, ny, 4.0, 1.0, jitter=0.2, seed=482)
    return dict(mesh=mi, p=1, cfl=0.3, states=double_mach_states(), shock=DMR_SHOCK, shock_states=(0, 1))


def batched_square_meshes(count: int = 64, seed: int = 5, e_min: float = 1e3,
                          e_max: float = 2e5) -> list[dict]:
    """Independent periodic square meshes of uneven size and order.

    Element counts are log-uniform on [e_min, e_max] (grid ``n = round(sqrt(E/2))``),
    p uniform in {1, 2, 3}, vortex strength in U[3, 6], centre in U[0.3, 0.7]^2.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        e = math.exp(rng.uniform(math.log(e_min), math.log(e_max)))
        n = max(3, int(round(math.sqrt(e / 2.0))))
        p = int(rng.integers(1, 4))
        beta = float(rng.uniform(3.0, 6.0))
        xc, yc = (float(v) for v in rng.uniform(0.3, 0.7, size=2))
        out.append(dict(n=n, p=p, beta=beta, xc=xc, yc=yc))
    return out
