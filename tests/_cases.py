"""Shared builders for the GPU parity tests: the same seeded inputs go to the
oracle (test infrastructure) and to the C-ABI library."""

import numpy as np

import synthetic as syn
from oracle.ader import Oracle
from synthetic.workloads import coupled_box, random_dofs


def to_gpu_layout(Q_oracle):
    """oracle Q[e, l, p] -> library Q[e, p, l]"""
    return np.ascontiguousarray(np.transpose(Q_oracle, (0, 2, 1)))


def to_oracle_layout(Q_gpu):
    return np.ascontiguousarray(np.transpose(Q_gpu, (0, 2, 1)))


def rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def make_pair(mesh, mat, N, precision=0, cfl=0.5, g=9.81, max_clusters=1, ensemble=1, acoustic_ocean=False):
    from paper_2107_06640_gb300 import Solver
    rho, lam, mu = mat
    o = Oracle(mesh.xyz, mesh.tets, mesh.face_tag, mesh.face_partner, rho, lam, mu, N, cfl=cfl, g=g,
               max_clusters=max_clusters)
    s = Solver(mesh.xyz, mesh.tets, mesh.face_tag, rho, lam, mu, face_partner=mesh.face_partner,
               degree=N, precision=precision, cfl=cfl, gravity=g, max_clusters=max_clusters,
               ensemble=ensemble, acoustic_ocean=acoustic_ocean)
    return o, s


def small_coupled(nxy=3, n_water=2, n_crust=2, rigid_bottom=False, bathy=None):
    """A few-hundred-tet version of the coupled ocean-crust box (all face kinds)."""
    return coupled_box(nxy=nxy, n_water=n_water, n_crust=n_crust, L=6e3, depth=4e3, water=1e3,
                       rigid_bottom=rigid_bottom, bathy=bathy)


def eta_poly(x, y):
    """A global degree-2 sea-surface polynomial: exact on every face for N >= 2."""
    return 0.3 + 1e-4 * x - 2e-4 * y + 1e-8 * x * y


def oracle_eta_at_nodes(o, elem_face, node_chi, N):
    """Oracle eta (values at its face quadrature points, a P_N polynomial) fitted
    on each face and evaluated at the library's face nodes."""
    mono = [(a, b) for a in range(N + 1) for b in range(N + 1 - a)]
    Vq = np.array([[x ** a * y ** b for (a, b) in mono] for x, y in o.chi])
    Vn = np.array([[x ** a * y ** b for (a, b) in mono] for x, y in node_chi])
    out = np.empty((len(elem_face), len(node_chi)))
    for g, ef in enumerate(elem_face):
        e, f = divmod(int(ef), 4)
        c, *_ = np.linalg.lstsq(Vq, o.eta[e, f], rcond=None)
        out[g] = Vn @ c
    return out


def node_chi(N):
    return np.array([[i1 / N, i2 / N] for i2 in range(N + 1) for i1 in range(N + 1 - i2)])


def submesh(mesh, mat, elems):
    """The elements `elems` plus their face neighbours as a stand-alone mesh.
    Faces of the added neighbours that lead outside become absorbing; the
    one-step update of every element of `elems` is then the same as in the
    full mesh (it only reads its own and its neighbours' dofs)."""
    import synthetic as syn
    fv = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    tri = np.sort(mesh.tets[:, fv], axis=2)                    # (nt, 4, 3)
    nv = mesh.xyz.shape[0]
    key = (tri[..., 0] * nv + tri[..., 1]) * nv + tri[..., 2]  # (nt, 4)
    flat = key.ravel()
    order = np.argsort(flat, kind="stable")
    sk = flat[order]

    def nbr_of(e, f):
        if mesh.face_tag[e, f] not in (syn.TAG_INTERIOR, syn.TAG_FAULT):
            return -1
        k = key[e, f]
        lo = np.searchsorted(sk, k, "left")
        hi = np.searchsorted(sk, k, "right")
        for idx in order[lo:hi]:
            if idx // 4 != e:
                return int(idx // 4)
        raise ValueError("unmatched face")

    keep = set(int(e) for e in elems)
    nbrs = {}
    for e in list(keep):
        for f in range(4):
            nb = nbr_of(e, f)
            nbrs[(e, f)] = nb
            if nb >= 0:
                keep.add(nb)
    keep = np.array(sorted(keep))
    pos = -np.ones(mesh.nt, np.int64)
    pos[keep] = np.arange(keep.size)
    tets = mesh.tets[keep]
    vids, inv = np.unique(tets, return_inverse=True)
    tags = mesh.face_tag[keep].copy()
    for i, e in enumerate(keep):
        for f in range(4):
            nb = nbrs[(e, f)] if (e, f) in nbrs else nbr_of(e, f)
            if nb >= 0 and pos[nb] < 0:
                tags[i, f] = syn.TAG_ABSORB
            if tags[i, f] == syn.TAG_PERIODIC:
                raise ValueError("periodic faces not supported in submeshes")
    sub = syn.Mesh(xyz=mesh.xyz[vids], tets=inv.reshape(-1, 4), face_tag=tags,
                   face_partner=-np.ones_like(tags, dtype=np.int64), hex_index=mesh.hex_index[keep],
                   dims=mesh.dims)
    return sub, tuple(np.asarray(a)[keep] for a in mat), keep, pos
