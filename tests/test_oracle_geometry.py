"""Pins for the oracle's element geometry, face connectivity, CFL length and
rate-2 clusters (Sec. 4.4) against closed forms and brute force."""

from collections import deque

import numpy as np
import pytest

import synthetic as syn
from oracle.basis import FACE_VERTS
from oracle.geometry import Geometry, clusters

rng = np.random.default_rng(21)


def _random_tets(n):
    """n well-shaped random tets (positively oriented), as a mesh of their own."""
    P = rng.standard_normal((n, 4, 3))
    P[:, 1:] += 2.0 * np.eye(3)[None]
    d = np.linalg.det(np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=2))
    P[d < 0] = P[d < 0][:, [0, 2, 1, 3]]
    tets = np.arange(4 * n).reshape(n, 4)
    return P.reshape(-1, 3), tets


def test_regular_tetrahedron_closed_forms():
    """Edge a: volume a^3/(6 sqrt 2), face area sqrt(3)/4 a^2, insphere
    radius a/(2 sqrt 6), so the CFL length h = 2 r_in = a/sqrt(6)."""
    a = 1.7
    P = a / np.sqrt(8.0) * np.array([[1.0, 1, 1], [-1, 1, -1], [1, -1, -1], [-1, -1, 1]])
    g = Geometry(P, np.array([[0, 1, 2, 3]]), np.full((1, 4), 3, np.int32))
    assert g.volume[0] == pytest.approx(a ** 3 / (6 * np.sqrt(2.0)), rel=1e-14)
    assert np.allclose(g.area[0], np.sqrt(3.0) / 4 * a * a, rtol=1e-14)
    assert g.h[0] == pytest.approx(a / np.sqrt(6.0), rel=1e-14)


def test_normals_areas_and_insphere_of_random_tets():
    """Outward unit normals (away from the opposite vertex) with
    sum_f area_f n_f = 0 (a closed surface); the incentre
    sum_f area_f P_f / sum_f area_f (P_f the vertex opposite face f) lies at
    the same distance h/2 from all four face planes."""
    xyz, tets = _random_tets(50)
    g = Geometry(xyz, tets, np.full((50, 4), 3, np.int32))
    P = xyz[tets]
    assert np.allclose(np.linalg.norm(g.normal, axis=2), 1.0, rtol=1e-14)
    assert np.allclose(np.einsum("ef,efd->ed", g.area, g.normal), 0.0, atol=1e-12 * g.area.max())
    for f in range(4):
        on_face = P[:, FACE_VERTS[f][0]]
        assert np.all(np.einsum("ed,ed->e", g.normal[:, f], on_face - P[:, f]) > 0)
    centre = np.einsum("ef,efd->ed", g.area, P) / g.area.sum(1)[:, None]
    for f in range(4):
        on_face = P[:, FACE_VERTS[f][0]]
        dist = np.einsum("ed,ed->e", g.normal[:, f], on_face - centre)
        assert np.allclose(dist, g.h / 2, rtol=1e-12)
    # volume against the scalar triple product of the edges
    vol = np.abs(np.einsum("ed,ed->e", P[:, 1] - P[:, 0], np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]))) / 6
    assert np.allclose(g.volume, vol, rtol=1e-13)


def test_face_neighbours_share_vertices_and_periodic_faces_are_translates():
    m = syn.kuhn_box(np.linspace(0, 1, 4), np.linspace(0, 2, 3), np.linspace(0, 1, 3),
                     tags={"x-": 4, "x+": 4, "y-": 3, "y+": 3, "z-": 6, "z+": 2})
    g = Geometry(m.xyz, m.tets, m.face_tag, m.face_partner)
    for e in range(g.E):
        for f in range(4):
            t = g.face_tag[e, f]
            nb, nf = g.nbr[e, f], g.nbr_face[e, f]
            if t in (3, 6, 2):
                assert nb < 0
                continue
            assert nb >= 0 and g.nbr[nb, nf] == e and g.nbr_face[nb, nf] == f
            mine = g.xyz[g.tets[e, list(FACE_VERTS[f])]]
            theirs = g.xyz[g.tets[nb, list(FACE_VERTS[nf])]] - g.shift[e, f]
            # the same three points (any order), opposite normals, equal areas
            assert np.allclose(np.sort(mine, axis=0), np.sort(theirs, axis=0), atol=1e-14)
            assert np.allclose(g.normal[e, f], -g.normal[nb, nf], atol=1e-14)
            assert g.area[e, f] == pytest.approx(g.area[nb, nf], rel=1e-14)
            if t == 4:
                assert np.count_nonzero(np.abs(g.shift[e, f]) > 1e-14) == 1
                assert abs(abs(g.shift[e, f, 0]) - 1.0) < 1e-14


def _greatest_clustering(g, dt, max_clusters):
    """Closed form of the largest cluster index per element that keeps
    2^c dt_min <= dt_e (the CFL bound), c <= max_clusters - 1, face
    neighbours at most one apart and fault neighbours equal:
    c_e = min_j (c0_j + dist(e, j)), the graph distance with weight 1 across
    ordinary faces and 0 across fault faces (0-1 breadth-first search)."""
    dtmin = dt.min()
    c0 = np.minimum(np.floor(np.log2(dt / dtmin) + 1e-12).astype(np.int64), max_clusters - 1)
    out = c0.copy()
    for j in range(g.E):
        dist = np.full(g.E, np.iinfo(np.int64).max)
        dist[j] = 0
        dq = deque([j])
        while dq:
            u = dq.popleft()
            for f in range(4):
                v = g.nbr[u, f]
                if v < 0:
                    continue
                w = 0 if g.face_tag[u, f] == 5 else 1
                if dist[u] + w < dist[v]:
                    dist[v] = dist[u] + w
                    (dq.appendleft if w == 0 else dq.append)(v)
        out = np.minimum(out, c0[j] + dist)
    return out


@pytest.mark.parametrize("max_clusters", [2, 4, 6])
def test_clusters_are_the_greatest_admissible_clustering(max_clusters):
    """Rate-2 clusters (Sec. 4.4) on seeded random element time steps spanning
    2^0 .. 2^6 dt_min, on a box with a fault: equal to the brute-force closed
    form, and every constraint holds."""
    m = syn.kuhn_box(np.linspace(0, 4, 5), np.linspace(0, 2, 3), np.linspace(-2, 0, 3),
                     fault=dict(c=0, jrange=(0, 2), krange=(0, 2)))
    g = Geometry(m.xyz, m.tets, m.face_tag, m.face_partner)
    for seed in range(3):
        dt = 2.0 ** np.random.default_rng(seed).uniform(0, 6, g.E)
        c, dtmin = clusters(g, dt, max_clusters)
        assert dtmin == dt.min()
        assert np.array_equal(c, _greatest_clustering(g, dt, max_clusters))
        assert np.all((2.0 ** c) * dtmin <= dt * (1 + 1e-12)) and c.max() <= max_clusters - 1
        for f in range(4):
            nb = g.nbr[:, f]
            has = nb >= 0
            d = c[has] - c[nb[has]]
            fault = g.face_tag[has, f] == 5
            assert np.all(np.abs(d) <= 1) and np.all(d[fault] == 0)
