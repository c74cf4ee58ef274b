"""Structured-to-unstructured tetrahedral meshes (Kuhn / Freudenthal split).

Each hexahedron of a tensor-product grid is cut into six tetrahedra along its
main diagonal: for every permutation (a, b, c) of the three axes the tet
(v000, v000 + e_a, v000 + e_a + e_b, v111).  The split is conforming across
hexahedra, so the result is a valid unstructured conforming tet mesh; it is
handed to the solvers as plain arrays (coordinates, connectivity, face tags),
exactly what a user would upload from a mesh file.

Conventions (shared by every consumer of these arrays):
  * tets are positively oriented: det[v1-v0, v2-v0, v3-v0] > 0;
  * local face f of a tet is the face opposite local vertex f;
  * face tags: 0 interior, 1 free surface, 2 gravitational free surface,
    3 absorbing, 4 periodic (partner given), 5 dynamic-rupture fault,
    6 rigid wall;
  * face_partner[t, f] = t' * 4 + f' for periodic faces, else -1.
"""

from dataclasses import dataclass, field
from itertools import permutations

import numpy as np

TAG_INTERIOR = 0
TAG_FREE = 1
TAG_GRAVITY = 2
TAG_ABSORB = 3
TAG_PERIODIC = 4
TAG_FAULT = 5
TAG_RIGID = 6

SIDES = ("x-", "x+", "y-", "y+", "z-", "z+")


@dataclass
class Mesh:
    xyz: np.ndarray            # (nv, 3) float64
    tets: np.ndarray           # (nt, 4) int64, positively oriented
    face_tag: np.ndarray       # (nt, 4) int32
    face_partner: np.ndarray   # (nt, 4) int64, -1 unless periodic
    hex_index: np.ndarray      # (nt, 3) int64 structured (i, j, k) of the parent hex
    dims: tuple                # (nx, ny, nz)
    extra: dict = field(default_factory=dict)

    @property
    def nt(self):
        return self.tets.shape[0]

    @property
    def nv(self):
        return self.xyz.shape[0]

    def centroids(self):
        return self.xyz[self.tets].mean(axis=1)


def graded_axis(x0, x1, n, ratio=1.0):
    """n cells on [x0, x1] whose widths grow geometrically from the x0 end so
    that the last cell is `ratio` times the first (ratio=1: uniform)."""
    if n < 1:
        raise ValueError("need at least one cell")
    if ratio == 1.0 or n == 1:
        return np.linspace(x0, x1, n + 1)
    q = ratio ** (1.0 / (n - 1))
    w = q ** np.arange(n)
    w = w / w.sum() * (x1 - x0)
    return np.concatenate([[x0], x0 + np.cumsum(w)])


def _vid(i, j, k, nx, ny):
    return i + (nx + 1) * (j + (ny + 1) * k)


def kuhn_box(xs, ys, zs, tags=None, warp=None, fault=None):
    """Kuhn-split tensor grid with node coordinates xs, ys, zs (monotone).

    tags:  dict side -> tag for the six box sides (default: absorbing).
           Periodic sides must come in pairs (x-/x+ etc.).
    warp:  optional function (xyz (nv,3), ijk (nv,3)) -> xyz applied to nodes
           after the grid is built (e.g. a bathymetry warp); it must keep every
           tet positively oriented and periodic sides translation-equivalent.
    fault: optional dict(c=int, jrange=(j0, j1), krange=(k0, k1)) marking the
           interior faces on the index plane i - k = c with j in [j0, j1) and
           k in [k0, k1) as dynamic-rupture faces (tag 5 on both sides).
    """
    xs, ys, zs = (np.asarray(a, dtype=np.float64) for a in (xs, ys, zs))
    nx, ny, nz = len(xs) - 1, len(ys) - 1, len(zs) - 1
    tags = dict(tags or {})
    for s in SIDES:
        tags.setdefault(s, TAG_ABSORB)
    for a in "xyz":
        if (tags[a + "-"] == TAG_PERIODIC) != (tags[a + "+"] == TAG_PERIODIC):
            raise ValueError("periodic sides must be paired")

    I, J, K = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    I, J, K = (a.transpose(2, 1, 0).ravel() for a in (I, J, K))  # i fastest
    ijk = np.stack([I, J, K], axis=1).astype(np.int32)
    xyz = np.stack([xs[I], ys[J], zs[K]], axis=1)
    if warp is not None:
        xyz = np.asarray(warp(xyz.copy(), ijk), dtype=np.float64)

    hi, hj, hk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    hi, hj, hk = (a.transpose(2, 1, 0).ravel() for a in (hi, hj, hk))
    nh = hi.size
    unit = np.eye(3, dtype=np.int64)
    tets = []
    hexid = []
    for perm in permutations(range(3)):
        offs = [np.zeros(3, np.int64), unit[perm[0]], unit[perm[0]] + unit[perm[1]],
                np.ones(3, np.int64)]
        cols = []
        for o in offs:
            cols.append(_vid(hi + o[0], hj + o[1], hk + o[2], nx, ny))
        tets.append(np.stack(cols, axis=1))
        hexid.append(np.stack([hi, hj, hk], axis=1))
    tets = np.concatenate(tets, axis=0).astype(np.int64)
    hexid = np.concatenate(hexid, axis=0)
    # order tets hex by hex (better locality than permutation-major)
    order = np.argsort(np.repeat(np.arange(nh)[None, :], 6, axis=0).ravel(), kind="stable")
    tets, hexid = tets[order], hexid[order]

    # positive orientation
    p = xyz[tets]
    det = np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0])
    if np.any(np.abs(det) == 0):
        raise ValueError("degenerate tet")
    neg = det < 0
    tets[neg, 1], tets[neg, 2] = tets[neg, 2].copy(), tets[neg, 1].copy()

    nt = tets.shape[0]
    face_tag = np.zeros((nt, 4), np.int32)
    face_partner = -np.ones((nt, 4), np.int64)
    fv = np.stack([np.delete(tets, f, axis=1) for f in range(4)], axis=1)  # (nt,4,3)
    fijk = ijk[fv]  # (nt,4,3,3)
    side_faces = {}
    for ax, a in enumerate("xyz"):
        nmax = (nx, ny, nz)[ax]
        for s, val in (("-", 0), ("+", nmax)):
            on = np.all(fijk[:, :, :, ax] == val, axis=2)
            face_tag[on] = tags[a + s]
            side_faces[a + s] = np.argwhere(on)
    for ax, a in enumerate("xyz"):
        if tags[a + "-"] != TAG_PERIODIC:
            continue
        other = [d for d in range(3) if d != ax]
        keys = {}
        for t, f in side_faces[a + "+"]:
            key = tuple(sorted(tuple(fijk[t, f, v, other]) for v in range(3)))
            keys[key] = (t, f)
        for t, f in side_faces[a + "-"]:
            key = tuple(sorted(tuple(fijk[t, f, v, other]) for v in range(3)))
            tp, fp = keys[key]
            face_partner[t, f] = tp * 4 + fp
            face_partner[tp, fp] = t * 4 + f
    if fault is not None:
        c = fault["c"]
        j0, j1 = fault["jrange"]
        k0, k1 = fault["krange"]
        d = fijk[..., 0] - fijk[..., 2]  # (nt,4,3)
        on = np.all(d == c, axis=2)
        on &= np.all((fijk[..., 1] >= j0) & (fijk[..., 1] <= j1), axis=2)
        on &= np.all((fijk[..., 2] >= k0) & (fijk[..., 2] <= k1), axis=2)
        on &= face_tag == TAG_INTERIOR
        face_tag[on] = TAG_FAULT
    return Mesh(xyz=xyz, tets=tets, face_tag=face_tag, face_partner=face_partner,
                hex_index=hexid, dims=(nx, ny, nz))


def unit_cube_periodic(n):
    """n^3 hexes x 6 tets on the periodic unit cube."""
    g = np.linspace(0.0, 1.0, n + 1)
    t = {s: TAG_PERIODIC for s in SIDES}
    return kuhn_box(g, g, g, tags=t)
