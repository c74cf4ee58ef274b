"""The library's host-side set-up, checked on the CPU (no device) against the
oracle.  adg_plan: the CFL time step and rate-2 cluster of every element
(Sec. 4.4) on meshes with periodic faces, a fluid layer with a gravitational
surface, a fault and randomly jittered nodes; cluster indices bit for bit.
adg_face_flux: the Godunov flux matrices of every face kind (Sec. 4.2)."""

import numpy as np
import pytest

import synthetic as syn
from oracle.basis import FACE_VERTS
from oracle.geometry import Geometry, cfl_dt, clusters
from synthetic.mesh import kuhn_box
from synthetic.workloads import coupled_box


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2107_06640_gb300 import build
    build.build()


def _warped_periodic(n, a):
    phi = lambda u: u - a * np.sin(2 * np.pi * u) / (2 * np.pi)
    g = np.linspace(0, 1, n + 1)
    return syn.kuhn_box(g, g, g, tags={s: 4 for s in syn.mesh.SIDES}, warp=lambda x, ijk: phi(x))


def _jittered(n, amp, seed):
    rng = np.random.default_rng(seed)
    g = np.linspace(0.0, 1.0, n + 1)

    def warp(x, ijk):
        inner = np.all((ijk > 0) & (ijk < n), axis=1)
        x[inner] += rng.uniform(-amp, amp, (inner.sum(), 3)) / n
        return x

    return kuhn_box(g, g, g, warp=warp)


def _fault_graded():
    return kuhn_box(np.linspace(0, 4e3, 5), np.linspace(0, 2e3, 3), np.array([-2e3, -1.6e3, 0.0]),
                    fault=dict(c=0, jrange=(0, 2), krange=(0, 2)))


def _cases():
    m = _warped_periodic(4, 0.95)
    yield "periodic-warped", m, syn.elastic_uniform(m.nt), 3, 0.5, 3
    m, mat = coupled_box(nxy=3, n_water=2, n_crust=3, L=6e3, depth=4e3, water=1.5e3, grading=1.6)
    yield "ocean-gravity", m, mat, 5, 0.35, 4
    m = _fault_graded()
    g = np.random.default_rng(3)
    mu = 3.2e10 * (1 + 0.2 * g.uniform(-1, 1, m.nt))
    yield "fault", m, (2700.0 * (1 + 0.2 * g.uniform(-1, 1, m.nt)), mu * 1.1, mu), 4, 0.35, 2
    for seed in range(2):
        m = _jittered(4, 0.35, seed)
        yield f"jittered-{seed}", m, syn.elastic_uniform(m.nt), 2, 0.5, 8


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_plan_equals_the_oracle(case):
    from paper_2107_06640_gb300 import plan
    name, m, (rho, lam, mu), N, cfl, mc = case
    dt, cl, dtmin, ncl = plan(m.xyz, m.tets, m.face_tag, rho, lam, mu, face_partner=m.face_partner, degree=N,
                              cfl=cfl, max_clusters=mc)
    geo = Geometry(m.xyz, m.tets, m.face_tag, m.face_partner)
    want_dt = cfl_dt(geo, rho, lam, mu, N, cfl)
    want_cl, want_min = clusters(geo, want_dt, mc)
    assert np.allclose(dt, want_dt, rtol=1e-14, atol=0)
    assert dtmin == pytest.approx(want_min, rel=1e-14)
    assert np.array_equal(cl, want_cl)
    assert ncl == want_cl.max() + 1
    if name in ("periodic-warped", "ocean-gravity"):
        assert ncl >= 2


def test_jittered_mesh_spans_several_clusters():
    from paper_2107_06640_gb300 import plan
    m = _jittered(4, 0.35, 0)
    _, cl, _, ncl = plan(m.xyz, m.tets, m.face_tag, *syn.elastic_uniform(m.nt), degree=2, cfl=0.5, max_clusters=8)
    assert ncl >= 3 and np.bincount(cl).min() > 0


def test_plan_reports_mesh_and_material_errors():
    from paper_2107_06640_gb300 import AdgError, _lib as L
    m = _warped_periodic(2, 0.3)
    rho, lam, mu = syn.elastic_uniform(m.nt)
    ctx = L.adg_create(L.adg_default_config())
    try:
        L.adg_upload_mesh(ctx, m.xyz, m.tets, m.face_tag, m.face_partner)
        with pytest.raises(AdgError) as ei:   # no material yet
            L.adg_plan(ctx)
        assert ei.value.code == -3
        bad = mu.copy()
        bad[5] = -1.0
        L.adg_upload_material(ctx, rho, lam, bad)
        with pytest.raises(AdgError) as ei:
            L.adg_plan(ctx)
        assert ei.value.code == -1
    finally:
        L.adg_destroy(ctx)
    # an inverted tet, and an interior face without its neighbour
    for mutate in ("invert", "unmatched"):
        tets, tag = m.tets.copy(), m.face_tag.copy()
        if mutate == "invert":
            tets[7, [1, 2]] = tets[7, [2, 1]]
            tag[7, [1, 2]] = tag[7, [2, 1]]
        else:
            tag = np.where(tag == 4, 0, tag)  # periodic faces declared interior: no matching face
        ctx = L.adg_create(L.adg_default_config())
        try:
            L.adg_upload_mesh(ctx, m.xyz, tets, tag, m.face_partner)
            L.adg_upload_material(ctx, rho, lam, mu)
            with pytest.raises(AdgError) as ei:
                L.adg_plan(ctx)
            assert ei.value.code == -2, mutate
        finally:
            L.adg_destroy(ctx)


def _flux_case(m, mat, N=2):
    from paper_2107_06640_gb300 import _lib as L
    cfg = L.adg_default_config()
    cfg.degree = N
    ctx = L.adg_create(cfg)
    L.adg_upload_mesh(ctx, m.xyz, m.tets, m.face_tag, m.face_partner)
    L.adg_upload_material(ctx, *mat)
    return L, ctx


def _oracle_flux(n, tag, qm, qp, matm, matp):
    """The oracle's Godunov flux T A^- w^b through a face with outward normal n."""
    from oracle import physics as ph
    R = ph.frame(n)
    wm = ph.rotate_in(qm, R)
    Zpm, Zsm = ph.impedances(*matm)
    if tag in (0, 4):
        Zpp, Zsp = ph.impedances(*matp)
        wb = ph.middle_state(wm, ph.rotate_in(qp, R), Zpm, Zpp, Zsm, Zsp)
    else:
        wb = ph.middle_state(wm, ph.ghost(wm, tag), Zpm, Zpm, Zsm, Zsm)
    return ph.rotate_out(ph.flux_rotated(wb, *matm), R)


def test_face_flux_matrices_equal_the_oracle_flux():
    """adg_face_flux returns the 9 x 9 matrices the kernels apply; with random
    states on both sides they give the oracle's Godunov flux (Sec. 4.2) on
    solid-solid (two materials), solid-fluid, fluid-fluid, periodic, free,
    rigid and absorbing faces, and zero on gravitational and fault faces."""
    rng = np.random.default_rng(12)
    scale = np.array([1e6] * 6 + [1.0] * 3)
    # ocean over crust with a gravitational top and absorbing sides; a second
    # box with periodic x, free y and rigid z sides and a fault
    m1, (rho, lam, mu) = coupled_box(nxy=2, n_water=1, n_crust=2, L=4e3, depth=3e3, water=1e3)
    rho = rho * (1 + 0.1 * rng.uniform(-1, 1, m1.nt))
    m2 = kuhn_box(np.linspace(0, 4e3, 5), np.linspace(0, 2e3, 3), np.linspace(-2e3, 0, 3),
                  tags={"x-": 4, "x+": 4, "y-": 1, "y+": 1, "z-": 6, "z+": 6},
                  fault=dict(c=0, jrange=(0, 2), krange=(0, 2)))
    mu2 = 3.2e10 * (1 + 0.2 * rng.uniform(-1, 1, m2.nt))
    cases = [(m1, (rho, lam, mu)), (m2, (2700.0 * (1 + 0.2 * rng.uniform(-1, 1, m2.nt)), 1.1 * mu2, mu2))]
    seen = set()
    for m, mat in cases:
        L, ctx = _flux_case(m, mat)
        geo = Geometry(m.xyz, m.tets, m.face_tag, m.face_partner)
        try:
            for e in range(m.nt):
                for f in range(4):
                    tag = int(m.face_tag[e, f])
                    nb = geo.nbr[e, f]
                    fluid_pair = (mat[2][e] == 0, nb >= 0 and mat[2][nb] == 0)
                    key = (tag, fluid_pair)
                    if key in seen and rng.uniform() > 0.05:
                        continue
                    seen.add(key)
                    Fm, Fp = L.adg_face_flux(ctx, e, f)
                    if tag in (2, 5):
                        assert not Fm.any() and not Fp.any()
                        continue
                    qm = rng.standard_normal(9) * scale
                    qp = rng.standard_normal(9) * scale
                    matm = tuple(a[e] for a in mat)
                    matp = tuple(a[nb] for a in mat) if nb >= 0 else matm
                    want = _oracle_flux(geo.normal[e, f], tag, qm, qp, matm, matp)
                    got = Fm @ qm + Fp @ qp
                    sc = np.abs(want).max()
                    assert np.max(np.abs(got - want)) <= 1e-12 * sc, (tag, fluid_pair)
                    if tag not in (0, 4):
                        assert not Fp.any()
        finally:
            L.adg_destroy(ctx)
    tags = {k[0] for k in seen}
    assert tags == {0, 1, 2, 3, 4, 5, 6}
    assert (0, (True, False)) in seen and (0, (False, True)) in seen and (0, (True, True)) in seen
    from paper_2107_06640_gb300 import AdgError
    L, ctx = _flux_case(m2, cases[1][1])
    try:
        with pytest.raises(AdgError) as ei:
            L.adg_face_flux(ctx, m2.nt, 0)
        assert ei.value.code == -1
    finally:
        L.adg_destroy(ctx)


def _face_nodes(xyz, tet, f, N):
    """Physical points of the equispaced face nodes chi = (i1/N, i2/N), i2 outer,
    i1 inner, on local face f (opposite local vertex f; vertices a < b < c)."""
    a, b, c = (xyz[tet[v]] for v in FACE_VERTS[f])
    chi = np.array([(i1 / N, i2 / N) for i2 in range(N + 1) for i1 in range(N + 1 - i2)])
    return a + chi[:, :1] * (b - a) + chi[:, 1:] * (c - a)


@pytest.mark.parametrize("N", [3, 5])
def test_face_node_maps_match_physical_points(N):
    """adg_face_neighbour: for every interior, periodic and fault face the
    neighbour and its face are the oracle's, and node_map (the permutation the
    neighbour flux applies to the neighbour's trace, Sec. 4.2) carries each face
    node onto the neighbour's node at the same physical point, on a warped
    periodic box, a warped fault box and a jittered box."""
    from paper_2107_06640_gb300 import _lib as L

    def warp(x, ijk):
        x[:, 0] += 150 * np.sin(x[:, 2] / 700.0) + 90 * np.cos(x[:, 1] / 500.0)
        x[:, 2] += 120 * np.sin(x[:, 0] / 900.0)
        return x

    meshes = [_warped_periodic(3, 0.6),
              kuhn_box(np.linspace(0, 4e3, 5), np.linspace(0, 2e3, 3), np.linspace(-2e3, 0, 3), warp=warp,
                       fault=dict(c=0, jrange=(0, 2), krange=(0, 2))),
              _jittered(3, 0.3, 4)]
    Bf = (N + 1) * (N + 2) // 2
    kinds = set()
    for m in meshes:
        geo = Geometry(m.xyz, m.tets, m.face_tag, m.face_partner)
        mat = syn.elastic_uniform(m.nt)
        L_, ctx = _flux_case(m, mat, N=N)
        try:
            for e in range(m.nt):
                for f in range(4):
                    nb, nf, node_map = L.adg_face_neighbour(ctx, e, f, Bf)
                    assert nb == geo.nbr[e, f] and (nb < 0 or nf == geo.nbr_face[e, f])
                    if nb < 0:
                        continue
                    kinds.add(int(m.face_tag[e, f]))
                    assert sorted(node_map) == list(range(Bf))
                    mine = _face_nodes(m.xyz, m.tets[e], f, N) + geo.shift[e, f]
                    theirs = _face_nodes(m.xyz, m.tets[nb], nf, N)
                    scale = np.abs(m.xyz).max()
                    assert np.max(np.abs(theirs[node_map] - mine)) <= 1e-12 * scale, (e, f)
        finally:
            L.adg_destroy(ctx)
    assert kinds == {0, 4, 5}


def test_a_new_upload_replaces_the_kept_plan():
    from paper_2107_06640_gb300 import _lib as L
    m = _warped_periodic(2, 0.3)
    rho, lam, mu = syn.elastic_uniform(m.nt)
    ctx = L.adg_create(L.adg_default_config())
    try:
        L.adg_upload_mesh(ctx, m.xyz, m.tets, m.face_tag, m.face_partner)
        L.adg_upload_material(ctx, rho, lam, mu)
        dt1 = L.adg_plan(ctx)[0]
        L.adg_upload_material(ctx, rho, 4.0 * lam + 6.0 * mu, mu)  # c_p doubled: half the time steps
        dt2 = L.adg_plan(ctx)[0]
        assert np.allclose(dt2, dt1 / 2, rtol=1e-14)
        Fm, _ = L.adg_face_flux(ctx, 0, 0)
        want = _oracle_flux(Geometry(m.xyz, m.tets, m.face_tag, m.face_partner).normal[0, 0], int(m.face_tag[0, 0]),
                            np.eye(9)[6], np.zeros(9), (rho[0], 4 * lam[0] + 6 * mu[0], mu[0]),
                            (rho[0], 4 * lam[0] + 6 * mu[0], mu[0]))
        assert np.allclose(Fm[:, 6], want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    finally:
        L.adg_destroy(ctx)
