"""Element geometry, face connectivity, CFL time steps and rate-2 clusters
(oracle; test infrastructure).

Affine map x = x0 + J xi from the reference tet; outward unit normals and
face areas per local face (face f opposite vertex f).  Interior faces are
matched through their sorted global vertex triples; periodic faces use the
given partner (and a translation between the two faces' centroids).

CFL (Sec. 4.4): dt_e = C(N) h_e / c_p,e with C(N) = cfl/(2N+1).
Reading: h = insphere diameter 2 r_in = 6 V / (sum of face areas).
Rate-2 clusters (Sec. 4.4), reading: cluster c holds the elements with
dt_e in [2^c dt_min, 2^(c+1) dt_min) and steps with 2^c dt_min; it is capped
at max_clusters-1; then face neighbours are made to differ by at most one
cluster by moving the coarser element down (never violates the CFL bound);
both sides of a fault face go to the smaller of their clusters.
"""

import numpy as np

from .basis import FACE_VERTS


class Geometry:
    def __init__(self, xyz, tets, face_tag, face_partner=None):
        self.xyz = np.asarray(xyz, dtype=np.float64)
        self.tets = np.asarray(tets, dtype=np.int64)
        self.face_tag = np.asarray(face_tag, dtype=np.int32)
        E = self.tets.shape[0]
        self.E = E
        if face_partner is None:
            face_partner = -np.ones((E, 4), np.int64)
        self.face_partner = np.asarray(face_partner, dtype=np.int64)
        P = self.xyz[self.tets]  # (E,4,3)
        self.x0 = P[:, 0]
        self.J = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=2)
        self.detJ = np.linalg.det(self.J)
        if np.any(self.detJ <= 0):
            raise ValueError("inverted or degenerate tetrahedron")
        self.Jinv = np.linalg.inv(self.J)  # Jinv[e, a, d] = d xi_a / d x_d
        self.volume = self.detJ / 6.0
        self.normal = np.empty((E, 4, 3))
        self.area = np.empty((E, 4))
        self.face_centroid = np.empty((E, 4, 3))
        for f in range(4):
            a, b, c = (P[:, v] for v in FACE_VERTS[f])
            cr = np.cross(b - a, c - a)
            ar = np.linalg.norm(cr, axis=1)
            n = cr / ar[:, None]
            opp = P[:, f]
            sgn = np.sign(np.einsum("ij,ij->i", n, a - opp))
            self.normal[:, f] = n * sgn[:, None]
            self.area[:, f] = 0.5 * ar
            self.face_centroid[:, f] = (a + b + c) / 3.0
        self.h = 6.0 * self.volume / self.area.sum(axis=1)
        self._connect()

    def _connect(self):
        E = self.E
        self.nbr = -np.ones((E, 4), np.int64)
        self.nbr_face = -np.ones((E, 4), np.int64)
        self.shift = np.zeros((E, 4, 3))
        table = {}
        for e in range(E):
            for f in range(4):
                if self.face_tag[e, f] in (0, 5):
                    key = tuple(sorted(self.tets[e, list(FACE_VERTS[f])]))
                    table.setdefault(key, []).append((e, f))
        for key, lst in table.items():
            if len(lst) != 2:
                raise ValueError(f"non-matching interior face {key}: {lst}")
            (e1, f1), (e2, f2) = lst
            self.nbr[e1, f1], self.nbr_face[e1, f1] = e2, f2
            self.nbr[e2, f2], self.nbr_face[e2, f2] = e1, f1
        per = np.argwhere(self.face_tag == 4)
        for e, f in per:
            p = self.face_partner[e, f]
            if p < 0:
                raise ValueError("periodic face without partner")
            self.nbr[e, f], self.nbr_face[e, f] = p // 4, p % 4
            self.shift[e, f] = self.face_centroid[p // 4, p % 4] - self.face_centroid[e, f]

    def to_ref(self, e, x):
        """Reference coordinates of physical points x (..., 3) in elements e."""
        return np.einsum("...ad,...d->...a", self.Jinv[e], x - self.x0[e])

    def to_phys(self, e, xi):
        return self.x0[e] + np.einsum("...da,...a->...d", self.J[e], xi)


def cfl_dt(geom, rho, lam, mu, N, cfl):
    cp = np.sqrt((np.asarray(lam) + 2 * np.asarray(mu)) / np.asarray(rho))
    return cfl / (2 * N + 1) * geom.h / cp


def clusters(geom, dt, max_clusters):
    dtmin = dt.min()
    c = np.floor(np.log2(dt / dtmin) + 1e-12).astype(np.int64)
    c = np.clip(c, 0, max_clusters - 1)
    # dt_e in [2^c dtmin, 2^(c+1) dtmin); an exact power of two goes up (tie-break)
    changed = True
    while changed:
        changed = False
        for f in range(4):
            nb = geom.nbr[:, f]
            has = nb >= 0
            cn = np.where(has, c[np.where(has, nb, 0)], 1 << 30)
            tag = geom.face_tag[:, f]
            lim = np.where(tag == 5, cn, cn + 1)
            newc = np.minimum(c, lim)
            if np.any(newc != c):
                c = newc
                changed = True
    return c, dtmin
