"""Element selections for meshes refined more than once (test inputs only)."""

import numpy as np


def second_level(rm, center, radius, coarse_radius=None):
    """Elements of the refined oracle mesh rm to refine once more: level-1
    elements with no coarser neighbour (the fine side of no hanging edge, so
    adjacent elements still differ by at most one level) whose centroid lies
    within radius of center, and coarse elements with hanging halves within
    coarse_radius (default radius) and right of center."""
    _, X = rm.elements()
    d = X.mean(axis=1) - np.asarray(center, dtype=np.float64)
    d2 = (d * d).sum(axis=1)
    cr = radius if coarse_radius is None else coarse_radius
    l, r, _, _ = rm.sides()
    hang = rm.hanging >= 0
    fine = np.zeros(rm.ne, bool)
    fine[l[hang]] = True
    coarse = np.zeros(rm.ne, bool)
    coarse[r[hang]] = True
    sel = ((rm.levels == 1) & ~fine & (d2 < radius * radius)) | (coarse & (d2 < cr * cr) & (d[:, 0] > 0))
    return np.nonzero(sel)[0].astype(np.int32)
