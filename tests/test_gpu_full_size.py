"""GPU parity at the full sizes the benchmark runs, on sampled outputs the
oracle recomputes one by one: after one step, the update of an element only
reads its own and its face neighbours' state, so the oracle steps a small mesh
made of the sampled elements and their neighbours (tests._cases.submesh)."""

import numpy as np
import pytest

import synthetic as syn
from tests._cases import node_chi, oracle_eta_at_nodes, rel_l2, submesh, to_oracle_layout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2107_06640_gb300 import build
    build.build()


def _eta_to_oracle(o, sub, keep, gmap, eta_nodes, N):
    """Hand the oracle the library's nodal sea-surface values through their
    P_N interpolant on every gravitational face of the small mesh."""
    mono = [(a, b) for a in range(N + 1) for b in range(N + 1 - a)]
    Vn = np.array([[x ** a * y ** b for (a, b) in mono] for x, y in node_chi(N)])
    Vq = np.array([[x ** a * y ** b for (a, b) in mono] for x, y in o.chi])
    for i, e in enumerate(keep):
        for f in range(4):
            if sub.face_tag[i, f] == syn.TAG_GRAVITY:
                o.eta[i, f] = Vq @ np.linalg.solve(Vn, eta_nodes[gmap[int(e) * 4 + f]])


def test_full_size_ensemble_sampled():
    """The ensemble workload as the benchmark runs it (1,019,304-tet coupled
    box, N = 5, tensor-core 3xTF32 form, 32 scenarios at once), each scenario
    with its own seeded dofs and sea-surface uplift (8 Gaussian bumps): one
    step, then 30 sampled elements (random, at the sea surface, at the sea
    floor) of 8 of the scenarios against the oracle.  The dofs are non-zero
    only on the samples' neighbourhood (the full-size FP32 upload is mostly
    untouched zero pages); the samples are read with adg_get_dofs_subset.
    Tolerance as for the 1.5 M-tet box in this form (1e-5)."""
    from oracle.ader import Oracle
    from paper_2107_06640_gb300 import ADG_3XTF32, Solver
    from synthetic.workloads import coupled_box, uplift_scenarios
    m, mat = coupled_box(nxy=66)
    assert m.nt == 1019304
    S = 32
    rho, lam, mu = mat
    s = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, degree=5, cfl=0.35, precision=ADG_3XTF32, ensemble=S)
    rng = np.random.default_rng(21)
    wet = m.hex_index[:, 2] >= 35
    top = np.nonzero(np.any(m.face_tag == syn.TAG_GRAVITY, axis=1))[0]
    floor = np.nonzero(wet & (m.hex_index[:, 2] == 35))[0]
    pick = np.concatenate([rng.choice(m.nt, 10, replace=False), rng.choice(top, 10, replace=False),
                           rng.choice(floor, 10, replace=False)])
    sub, smat, keep, pos = submesh(m, mat, pick)
    Qk = (rng.standard_normal((keep.size, S, 9, s.B)) * 1e-3).astype(np.float32)
    Q0 = np.zeros((m.nt, S, 9, s.B), np.float32)
    Q0[keep] = Qk
    s.set_dofs_f32(Q0)
    del Q0
    ef, nxyz = s.gravity_faces()
    eta0 = np.stack([f(nxyz[..., 0], nxyz[..., 1]) for f in uplift_scenarios(S, seed=3)], axis=1)
    s.set_eta(eta0)
    s.advance(1)
    Q1 = s.get_dofs_subset(pick)
    eta1 = s.read_ssh()
    o = Oracle(sub.xyz, sub.tets, sub.face_tag, sub.face_partner, *smat, 5, cfl=0.35, dt=s.info.dt_min)
    gmap = {int(v): g for g, v in enumerate(ef)}
    sel = pos[pick]
    for k in (0, 5, 11, 16, 22, 27, 30, 31):
        o.Q = np.ascontiguousarray(np.transpose(Qk[:, k].astype(np.float64), (0, 2, 1)))
        o.eta[:] = 0.0
        _eta_to_oracle(o, sub, keep, gmap, eta0[:, k], 5)
        o.t = 0.0
        o.step_gts()
        got = to_oracle_layout(Q1[:, k])
        assert rel_l2(got, o.Q[sel]) <= 1e-5, (k, rel_l2(got, o.Q[sel]))
        for i, e in enumerate(keep):
            if pos[e] not in set(sel):
                continue
            for f in range(4):
                if sub.face_tag[i, f] == syn.TAG_GRAVITY:
                    want = oracle_eta_at_nodes(o, [i * 4 + f], node_chi(5), 5)[0]
                    assert rel_l2(eta1[gmap[int(e) * 4 + f], k], want) <= 1e-6


def test_full_size_megathrust_sampled():
    """The megathrust workload at its benchmark size (17,280,000 tets, N = 4,
    15-degree fault with 32,000 faces under a 2 km ocean with gravity,
    rate-and-state friction) in the form the benchmark runs (FP32 dofs, FP64
    friction): one step from seeded dofs, then 25 sampled elements on both
    sides of the fault and 5 elsewhere against the oracle, and the fault state
    (slip rate, state, slip) of every fault face whose two sides are in the
    small mesh.  The dofs are non-zero only on the samples' neighbourhood (a
    sparse FP32 upload; the samples are read with adg_get_dofs_subset).
    Tolerances: FP32 dofs and traces, one step (2e-5 dofs, 1e-4 fault state,
    relative L2)."""
    if _mem_available_gb() < 160.0:
        pytest.skip("needs 160 GB of free host memory for the 17.3 M-tet setup")
    from oracle import rupture as ru
    from oracle.ader import Oracle
    from paper_2107_06640_gb300 import ADG_FP32, Solver, _lib
    from synthetic.workloads import fault_box, rs_fault_params
    r = 5
    m, mat = fault_box(nx=32 * r, ny=40 * r, nz=16 * r, dz=1e3 / r, dip_deg=15.0, ocean_layers=2 * r, water=2e3)
    assert m.nt == 17280000
    rho, lam, mu = mat
    s = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, degree=4, cfl=0.35, precision=ADG_FP32)
    nff = int(s.info.n_fault_faces)
    mf, pf, fxyz, fn = _lib.adg_fault_faces(s.ctx, nff, s.Bf)
    par = rs_fault_params(fxyz, fn, seed=0, patch_center=fxyz.reshape(-1, 3).mean(0), patch_radius=8e3)
    _lib.adg_set_fault(s.ctx, par[:, None])
    rng = np.random.default_rng(31)
    faces = rng.choice(nff, 25, replace=False)
    pick = np.unique(np.concatenate([mf[faces[:15]] // 4, pf[faces[15:]] // 4, rng.choice(m.nt, 5, replace=False)]))
    sub, smat, keep, pos = submesh(m, mat, pick)
    Qk = (rng.standard_normal((keep.size, 9, s.B)) * np.array([1e5] * 6 + [1e-2] * 3)[None, :, None]).astype(np.float32)
    Q0 = np.zeros((m.nt, 9, s.B), np.float32)
    Q0[keep] = Qk
    s.set_dofs_f32(Q0)
    del Q0
    ef, _ = s.gravity_faces()
    s.set_eta(np.zeros((len(ef), 1, s.Bf)))
    s.advance(1)
    st = np.empty((nff, 1, s.Bf, 8))
    st = _lib.adg_read_fault(s.ctx, st)[:, 0]
    o = Oracle(sub.xyz, sub.tets, sub.face_tag, sub.face_partner, *smat, 4, cfl=0.35, dt=s.info.dt_min)
    lib_face = {int(v): k for k, v in enumerate(mf)}
    idx = np.array([lib_face[int(keep[e]) * 4 + int(f)] for e, f in o.fm])
    assert np.allclose(o.f_xyz, fxyz[idx], rtol=0, atol=1e-6)
    o.set_fault({k: par[idx, :, i] for i, k in enumerate(ru.PARAMS)})
    o.Q = to_oracle_layout(Qk.astype(np.float64))
    o.step_gts()
    sel = pos[pick]
    got = to_oracle_layout(s.get_dofs_subset(pick))
    assert rel_l2(got, o.Q[sel]) <= 2e-5, rel_l2(got, o.Q[sel])
    assert rel_l2(st[idx, :, 0], o.fault["V"]) <= 1e-4
    assert rel_l2(st[idx, :, 1], o.fault["psi"]) <= 1e-4
    assert rel_l2(st[idx, :, 2:5], o.fault["slip"]) <= 1e-4


def _mem_available_gb():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 0.0


def test_full_size_lts_first_tick_sampled():
    """The LTS workload at its benchmark size (9,360,000 tets graded 32x in x
    and y under a sinusoidal seafloor, 6 rate-2 clusters, degree 5, 3xTF32).
    After the first tick, cluster 0 has finished one step of dt_min; in it a
    coarser neighbour contributes the integral of its Taylor expansion over
    [0, dt_min], as one global step of dt_min does.  Sampled elements with
    dt_e < 2 dt_min (cluster 0 whatever their neighbours) against the oracle on
    their neighbourhood with dt = dt_min, through adg_get_dofs_subset.  The
    dofs are non-zero only on that neighbourhood, so the full-size FP32 upload
    is mostly untouched zero pages.  Tolerance as for the other 3xTF32 steps."""
    if _mem_available_gb() < 40.0:
        pytest.skip("needs 40 GB of free host memory for the 9.36 M-tet mesh")
    from oracle.ader import Oracle
    from paper_2107_06640_gb300 import ADG_3XTF32, Solver
    from synthetic.workloads import coupled_box
    L = 100e3
    bathy = lambda x, y: -2000.0 + 500.0 * np.sin(2 * np.pi * x / L) * np.sin(2 * np.pi * y / L)
    m, mat = coupled_box(nxy=200, bathy=bathy, grading=32.0)
    assert m.nt == 9360000
    rho, lam, mu = mat
    s = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, degree=5, cfl=0.35, precision=ADG_3XTF32, max_clusters=6)
    assert s.info.n_clusters == 6
    dtmin = s.info.dt_min
    rng = np.random.default_rng(41)
    cand = rng.choice(m.nt, 600, replace=False)
    sub, smat, keep, pos = submesh(m, mat, cand)
    oc = Oracle(sub.xyz, sub.tets, sub.face_tag, sub.face_partner, *smat, 5, cfl=0.35)
    fine = cand[oc.dt_e[pos[cand]] < 2.0 * dtmin * (1.0 - 1e-9)]
    assert fine.size >= 10
    pick = fine[:40]
    sub, smat, keep, pos = submesh(m, mat, pick)
    Qk = (rng.standard_normal((keep.size, 9, s.B)) * 1e-3).astype(np.float32)
    Q0 = np.zeros((m.nt, 9, s.B), np.float32)
    Q0[keep] = Qk
    s.set_dofs_f32(Q0)
    del Q0
    s.step_tick()
    got = s.get_dofs_subset(pick)
    o = Oracle(sub.xyz, sub.tets, sub.face_tag, sub.face_partner, *smat, 5, cfl=0.35, dt=dtmin)
    o.Q = to_oracle_layout(Qk.astype(np.float64))
    o.step_gts()
    sel = pos[pick]
    assert rel_l2(to_oracle_layout(got), o.Q[sel]) <= 1e-5, rel_l2(to_oracle_layout(got), o.Q[sel])
    # the samples moved (a zero update would pass trivially)
    assert rel_l2(to_oracle_layout(Qk[sel].astype(np.float64)), o.Q[sel]) > 1e-3


def _face_neighbours(tets):
    """[nt][4] face neighbour of each tet face (-1 on the boundary), by
    matching the sorted vertex triples of all faces."""
    fv = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    tri = np.sort(tets[:, fv], axis=2)
    nv = int(tets.max()) + 1
    key = ((tri[..., 0] * nv + tri[..., 1]) * nv + tri[..., 2]).ravel()
    order = np.argsort(key, kind="stable")
    sk = key[order]
    same = np.nonzero(sk[1:] == sk[:-1])[0]
    a, b = order[same], order[same + 1]
    nbr = np.full(key.size, -1, np.int64)
    nbr[a] = b // 4
    nbr[b] = a // 4
    return nbr.reshape(-1, 4)


def _lts_support(nbr, cl, patch, cmax):
    """A superset of the elements whose dofs can be non-zero after one rate-2
    LTS macro step (Sec. 4.4) that starts from dofs non-zero only on `patch`:
    at every tick s, in cluster order, each cluster c with (s+1) % 2^c == 0
    ends a step, and an element of it joins when a face neighbour is already
    in (a prediction, an LTS buffer or a Taylor integral of a neighbour only
    carries data the neighbour had by then)."""
    supp = np.zeros(cl.size, bool)
    supp[patch] = True
    idx = np.array(patch, np.int64)
    for s in range(1 << cmax):
        for c in range(cmax + 1):
            if (s + 1) % (1 << c):
                continue
            cand = np.unique(nbr[idx].ravel())
            cand = cand[cand >= 0]
            cand = cand[(cl[cand] == c) & ~supp[cand]]
            supp[cand] = True
            idx = np.concatenate([idx, cand])
    return np.sort(idx)


def test_full_size_lts_whole_macro_step_sampled():
    """The LTS workload at its benchmark size and launch configuration
    (9,360,000 tets graded 32x, 6 rate-2 clusters, degree 5, 3xTF32, acoustic
    ocean) over one whole macro step of 32 ticks.  The dofs start non-zero on
    three patches only, each a tet and its face neighbours at a cluster border
    (1|0, 2|3 and 4|5), chosen with a seeded search for small supports, so
    that between them every cluster steps with data, takes LTS buffers from a
    finer neighbour and Taylor integrals from a coarser one.  Every element outside
    the patches' support (a superset of where data can arrive within the
    macro step) must still be exactly zero; the support, as a small mesh with
    the library's clusters and dt_min, is stepped by the oracle's LTS macro
    step and compared element by element.  Tolerance as for the other 3xTF32
    macro steps."""
    if _mem_available_gb() < 48.0:
        pytest.skip("needs 48 GB of free host memory for the 9.36 M-tet mesh")
    from oracle.ader import Oracle
    from paper_2107_06640_gb300 import ADG_3XTF32, Solver
    from synthetic.workloads import coupled_box
    L = 100e3
    bathy = lambda x, y: -2000.0 + 500.0 * np.sin(2 * np.pi * x / L) * np.sin(2 * np.pi * y / L)
    m, mat = coupled_box(nxy=200, bathy=bathy, grading=32.0)
    assert m.nt == 9360000
    s = Solver(m.xyz, m.tets, m.face_tag, *mat, degree=5, cfl=0.35, precision=ADG_3XTF32, max_clusters=6,
               acoustic_ocean=True)
    _, cl, dtmin, ncl = s.plan()
    assert ncl == 6
    cmax = ncl - 1
    nbr = _face_neighbours(m.tets)
    rng = np.random.default_rng(43)
    taken = np.zeros(m.nt, bool)
    patches, supports = [], []
    for a, b in ((1, 0), (2, 3), (4, 5)):
        inner = np.nonzero(cl == a)[0]
        nb = nbr[inner]
        border = np.zeros(inner.size, bool)
        for f in range(4):
            v = nb[:, f] >= 0
            border[v] |= cl[nb[v, f]] == b
        best = None
        for e in rng.choice(inner[border], 24, replace=False):
            p = np.unique(np.concatenate([[e], nbr[e][nbr[e] >= 0]]))
            F = _lts_support(nbr, cl, p, cmax)
            ring = nbr[F].ravel()
            if taken[F].any() or taken[ring[ring >= 0]].any():
                continue
            work = int(sum(np.count_nonzero(cl[F] == c) << (cmax - c) for c in range(ncl)))
            if best is None or work < best[0]:
                best = (work, p, F)
        assert best is not None
        patches.append(best[1])
        supports.append(best[2])
        taken[best[2]] = True
    F = np.unique(np.concatenate(supports))
    P = np.concatenate(patches)
    sub, smat, keep, pos = submesh(m, mat, F)
    o = Oracle(sub.xyz, sub.tets, sub.face_tag, sub.face_partner, *smat, 5, cfl=0.35, max_clusters=ncl)
    o.cluster = cl[keep].astype(np.int64)
    o.dtmin = dtmin
    assert set(np.unique(cl[F])) == set(range(ncl))
    Qp = rng.standard_normal((P.size, s.B, 9)) * 1e-3
    fluid = mat[2][P] == 0.0
    mean = Qp[fluid, :, 0:3].mean(axis=2)
    Qp[fluid, :, 0] = Qp[fluid, :, 1] = Qp[fluid, :, 2] = mean    # fluid stress -p I
    Qp[fluid, :, 3:6] = 0.0
    Qp = Qp.astype(np.float32).astype(np.float64)
    o.Q[pos[P]] = Qp
    Qbig = np.zeros((m.nt, 9, s.B), np.float32)
    Qbig[P] = np.swapaxes(Qp, 1, 2)
    s.set_dofs_f32(Qbig)
    s.advance(1)
    s.get_dofs_f32(out=Qbig)
    inside = np.zeros(m.nt, bool)
    inside[F] = True
    step = 1 << 19
    for lo in range(0, m.nt, step):
        rows = np.any(Qbig[lo:lo + step].reshape(-1, 9 * s.B) != 0.0, axis=1)
        stray = np.nonzero(rows & ~inside[lo:lo + step])[0]
        assert stray.size == 0, ("data outside the support", lo + stray[:8])
    got = to_oracle_layout(Qbig[F].astype(np.float64))
    del Qbig
    o.advance_macro()
    want = o.Q[pos[F]]
    assert rel_l2(got, want) <= 2e-5, rel_l2(got, want)
    start = 0
    for p, Fi in zip(patches, supports):
        sel = np.searchsorted(F, Fi)
        assert rel_l2(got[sel], want[sel]) <= 2e-5, (rel_l2(got[sel], want[sel]), np.bincount(cl[Fi], minlength=ncl))
        # the patch moved (a zero update would pass trivially)
        assert rel_l2(Qp[start:start + p.size], want[np.searchsorted(F, p)]) > 1e-3
        start += p.size
    # the data travelled: every cluster holds non-zero dofs after the step
    for c in range(ncl):
        assert np.abs(want[cl[F] == c]).max() > 0.0, c
