"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  Bar: relative L2 <= 1e-10 for the FP64 path (dofs and
sea-surface height); FP32 within the tolerance stated in each test."""

import numpy as np
import pytest

import synthetic as syn
from synthetic.workloads import plane_wave_case, plane_wave_field, random_dofs
from tests._cases import (eta_poly, make_pair, node_chi, oracle_eta_at_nodes, rel_l2, small_coupled,
                          submesh, to_gpu_layout, to_oracle_layout)

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2107_06640_gb300 import build
    build.build()


def test_plane_wave_small_config_fp64():
    # 8^3 hexes x 6 tets periodic, rho=1 lambda=2 mu=1, N=3, CFL 0.5, 100 steps
    m, mat = plane_wave_case(8)
    o, s = make_pair(m, mat, 3, cfl=0.5)
    assert s.nt == 3072 and np.isclose(s.info.dt_min, o.dtmin, rtol=1e-14)
    o.Q = o.project(plane_wave_field(0.0))
    s.set_dofs(to_gpu_layout(o.Q))
    for _ in range(100):
        o.step_gts()
    s.advance(100)
    Qg = to_oracle_layout(s.get_dofs())
    assert rel_l2(Qg, o.Q) <= FP64_TOL, rel_l2(Qg, o.Q)
    ref = np.linalg.norm(o.l2_error(plane_wave_field(o.t), Q=0 * o.Q))
    assert np.linalg.norm(o.l2_error(plane_wave_field(o.t), Q=Qg)) / ref < 2e-4
    assert np.isclose(s.time, o.t, rtol=1e-13)


def _coupled_run(N, precision, steps=3, seed=1):
    m, mat = small_coupled()
    o, s = make_pair(m, mat, N, precision=precision, cfl=0.5)
    Q0 = random_dofs((m.nt, s.B, 9), seed, N=N) * 1e-3
    o.Q = Q0.copy()
    s.set_dofs(to_gpu_layout(Q0))
    ef, nxyz = s.gravity_faces()
    assert len(ef) == int(np.sum(m.face_tag == syn.TAG_GRAVITY)) > 0
    s.set_eta(eta_poly(nxyz[..., 0], nxyz[..., 1])[:, None, :])
    for e, f in np.argwhere(m.face_tag == syn.TAG_GRAVITY):
        o.eta[e, f] = eta_poly(o.face_x[e, f, :, 0], o.face_x[e, f, :, 1])
    for _ in range(steps):
        o.step_gts()
    s.advance(steps)
    Qg = to_oracle_layout(s.get_dofs())
    eta_g = s.read_ssh()[:, 0, :]
    eta_o = oracle_eta_at_nodes(o, ef, node_chi(N), N)
    return rel_l2(Qg, o.Q), rel_l2(eta_g, eta_o)


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_coupled_random_dofs_fp64(N):
    # ocean over crust: solid-fluid interface, gravitational top, absorbing sides
    eq, ee = _coupled_run(N, 0)
    assert eq <= FP64_TOL and ee <= FP64_TOL, (eq, ee)


@pytest.mark.parametrize("precision,N", [(1, 5), (2, 5), (2, 4)])
def test_coupled_random_dofs_fp32(precision, N):
    # FP32 dofs (1: CUDA-core products, 2: tensor-core 3xTF32 products at
    # degrees 5 and 4; FP64 eta): per-output tolerance after 3 steps
    eq, ee = _coupled_run(N, precision)
    assert eq <= 2e-5 and ee <= 1e-6, (eq, ee)


@pytest.mark.parametrize("N", [5, 4])
def test_lts_coupled_graded_3xtf32(N):
    m, mat = syn.workloads.coupled_box(nxy=4, n_water=2, n_crust=2, L=8e3, depth=4e3, water=1e3,
                                       grading=4.0)
    o, s = make_pair(m, mat, N, precision=2, cfl=0.5, max_clusters=4)
    assert s.info.n_clusters >= 2
    Q0 = random_dofs((m.nt, s.B, 9), 3, N=N)
    o.Q = Q0.copy()
    s.set_dofs(to_gpu_layout(Q0))
    o.advance_macro()
    s.advance(1)
    assert rel_l2(to_oracle_layout(s.get_dofs()), o.Q) <= 2e-5


@pytest.mark.parametrize("N", [5, 4])
def test_periodic_cube_tensor_core_local_kernel(N):
    """Every element of a periodic cube takes the tensor-core local kernel
    (no gravitational, fault or LTS-boundary faces); 384 elements = 32 tiles
    of 12, ragged against the 2 x 152 tiles in flight.  Degree 4 stages its
    140-byte dofs rows through shared memory."""
    m, mat = syn.unit_cube_periodic(4), syn.materials.elastic_uniform(384)
    o, s = make_pair(m, mat, N, precision=2, cfl=0.5)
    from paper_2107_06640_gb300 import _lib
    Q0 = random_dofs((m.nt, s.B, 9), 5, N=N)
    o.Q = Q0.copy()
    s.set_dofs(to_gpu_layout(Q0))
    for _ in range(3):
        o.step_gts()
    s.advance(3)
    assert rel_l2(to_oracle_layout(s.get_dofs()), o.Q) <= 2e-5
    _, launches = _lib.adg_profile(s.ctx, 1)
    assert launches[0] == 1 and launches[1] == 1  # tensor-core launches only, no CUDA-core remainder
    assert int(s.info.tensor_core_updates_per_macro) == m.nt


@pytest.mark.parametrize("N", [5, 4])
def test_coupled_box_gravity_elements_on_the_tensor_cores(N):
    """Ocean over crust with a gravitational top: every element takes the
    tensor-core kernels, those with a sea-surface face on their own local
    launch (derivative traces of that face and the FP64 (eta, H) update on the
    tile), which the neighbour kernel's stored-flux path lifts.  Parity
    against the oracle (dofs and sea surface) is _coupled_run's."""
    m, mat = small_coupled()
    from paper_2107_06640_gb300 import _lib
    s = make_pair(m, mat, N, precision=2, cfl=0.5)[1]
    ms, launches = _lib.adg_profile(s.ctx, 1)
    assert launches[0] == 2 and launches[1] == 1   # local: elastic + gravitational-face launches; neighbour: one
    assert launches[3] == 1 and launches[4] == 1   # (phases with a tensor-core part)
    assert 0 < ms[3] <= ms[0] and 0 < ms[4] <= ms[1]
    assert int(s.info.tensor_core_updates_per_macro) == m.nt
    eq, ee = _coupled_run(N, 2, seed=9)
    assert eq <= 2e-5 and ee <= 1e-6, (eq, ee)


@pytest.mark.parametrize("N", [5, 4])
def test_ensemble_equals_independent_runs_3xtf32(N):
    m, mat = small_coupled(nxy=2)
    S = 5
    from paper_2107_06640_gb300 import ADG_3XTF32, Solver
    rho, lam, mu = mat
    kw = dict(degree=N, cfl=0.5, precision=ADG_3XTF32)
    ens = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, ensemble=S, **kw)
    Qs = np.stack([to_gpu_layout(random_dofs((m.nt, ens.B, 9), 20 + k, N=N)) for k in range(S)], axis=1)
    ens.set_dofs(Qs.astype(np.float32))
    ens.advance(2)
    out = ens.get_dofs()
    for k in range(S):
        one = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, **kw)
        one.set_dofs(Qs[:, k].astype(np.float32))
        one.advance(2)
        assert np.array_equal(one.get_dofs(), out[:, k])


def test_free_surface_and_rigid_wall_fp64():
    m, mat = small_coupled(rigid_bottom=True)
    m.face_tag[m.face_tag == syn.TAG_GRAVITY] = syn.TAG_FREE
    o, s = make_pair(m, mat, 4, cfl=0.5)
    Q0 = random_dofs((m.nt, s.B, 9), 7, N=4)
    o.Q = Q0.copy()
    s.set_dofs(to_gpu_layout(Q0))
    for _ in range(2):
        o.step_gts()
    s.advance(2)
    assert rel_l2(to_oracle_layout(s.get_dofs()), o.Q) <= FP64_TOL


@pytest.mark.parametrize("N", [5, 4])
def test_free_surface_rigid_wall_absorbing_on_the_tensor_cores(N):
    """Free-surface top, rigid-wall bottom and absorbing sides in the 3xTF32
    form: with no gravitational face every element takes both tensor-core
    kernels, whose neighbour kernel forms each face's Godunov flux (ghost
    states of the linear boundaries included) in the face frame."""
    m, mat = small_coupled(rigid_bottom=True)
    m.face_tag[m.face_tag == syn.TAG_GRAVITY] = syn.TAG_FREE
    o, s = make_pair(m, mat, N, precision=2, cfl=0.5)
    assert int(s.info.tensor_core_updates_per_macro) == m.nt
    Q0 = random_dofs((m.nt, s.B, 9), 8, N=N)
    o.Q = Q0.copy()
    s.set_dofs(to_gpu_layout(Q0))
    for _ in range(3):
        o.step_gts()
    s.advance(3)
    assert rel_l2(to_oracle_layout(s.get_dofs()), o.Q) <= 2e-5


def _warped_periodic(n, a=0.6):
    phi = lambda u: u - a * np.sin(2 * np.pi * u) / (2 * np.pi)
    g = np.linspace(0, 1, n + 1)
    return syn.kuhn_box(g, g, g, tags={sd: syn.TAG_PERIODIC for sd in syn.mesh.SIDES},
                        warp=lambda x, ijk: phi(x))


def test_lts_two_clusters_fp64():
    m = _warped_periodic(4)
    mat = syn.elastic_uniform(m.nt)
    o, s = make_pair(m, mat, 3, cfl=0.5, max_clusters=3)
    assert s.info.n_clusters == int(o.cluster.max()) + 1 >= 2
    sizes = np.bincount(o.cluster)
    assert list(s.info.cluster_size[: s.info.n_clusters]) == list(sizes)
    o.Q = o.project(plane_wave_field(0.0))
    s.set_dofs(to_gpu_layout(o.Q))
    for _ in range(3):
        o.advance_macro()
    s.advance(3)
    assert rel_l2(to_oracle_layout(s.get_dofs()), o.Q) <= FP64_TOL



@pytest.mark.parametrize("N", [3, 4])
def test_f32_dofs_transfer(N):
    """adg_set_dofs_f32 / adg_get_dofs_f32 (device-side reordering; rows of
    S 9 B = 360 values at N = 3 move in 16-byte chunks, 630 at N = 4 one by
    one): the caller's order survives bit for bit in both dofs precisions, the
    double API sees the same values, a step from an FP32 upload equals the step
    from the same values through the double API, and a call inside an LTS macro
    step is refused."""
    from paper_2107_06640_gb300 import ADG_FP32, ADG_FP64, AdgError, Solver
    m, (rho, lam, mu) = small_coupled()
    rng = np.random.default_rng(5)
    for prec in (ADG_FP32, ADG_FP64):
        kw = dict(degree=N, cfl=0.5, precision=prec, ensemble=2)
        a = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, **kw)
        b = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, **kw)
        Q32 = (rng.standard_normal((m.nt, 2, 9, a.B)) * 1e-2).astype(np.float32)
        a.set_dofs_f32(Q32)
        assert np.array_equal(a.get_dofs_f32(), Q32)
        assert np.array_equal(a.get_dofs(), Q32.astype(np.float64))
        b.set_dofs(Q32.astype(np.float64))
        a.advance(1)
        b.advance(1)
        assert np.array_equal(a.get_dofs(), b.get_dofs())
        assert np.array_equal(a.get_dofs_f32(), b.get_dofs().astype(np.float32))
        idx = [m.nt - 1, 0, 7, 7]
        assert np.array_equal(a.get_dofs_subset(idx), a.get_dofs()[idx])
    w = _warped_periodic(4)
    s = Solver(w.xyz, w.tets, w.face_tag, *syn.elastic_uniform(w.nt), face_partner=w.face_partner, degree=3,
               cfl=0.5, max_clusters=3)
    assert s.info.n_clusters >= 2
    s.step_tick()
    with pytest.raises(AdgError) as ei:
        s.set_dofs_f32(np.zeros((w.nt, 9, s.B), np.float32))
    assert ei.value.code == -3
    # the subset readout works inside the macro step
    assert np.array_equal(s.get_dofs_subset([3, 0]), s.get_dofs()[[3, 0]])
    with pytest.raises(AdgError):
        s.get_dofs_subset([w.nt])

@pytest.mark.parametrize("prec_name,S,N,acoustic", [("ADG_3XTF32", 1, 5, True), ("ADG_FP64", 2, 3, False)])
def test_f32_dofs_pipelined_transfers(prec_name, S, N, acoustic):
    """adg_set_dofs_f32_async / adg_advance_async / adg_get_dofs_f32_async then
    adg_sync: four steps enqueued back to back, each from its own upload and
    into its own download, give bit for bit the results of the synchronous
    calls (the uploads' fluid stress projected as there), the context ends at
    the same time, a synchronous call after the pipeline sees the last state,
    and an input that would need converting is refused before anything is
    enqueued."""
    import torch
    import paper_2107_06640_gb300 as pkg
    from paper_2107_06640_gb300 import Solver
    m, (rho, lam, mu) = small_coupled()
    kw = dict(degree=N, cfl=0.5, precision=getattr(pkg, prec_name), ensemble=S, acoustic_ocean=acoustic)
    a = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, **kw)
    b = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, **kw)
    shape = (m.nt, S, 9, a.B)
    rng = np.random.default_rng(11)
    K = 4
    ins = [torch.empty(shape, dtype=torch.float32, pin_memory=True).numpy() for _ in range(K)]
    outs = [torch.empty(shape, dtype=torch.float32, pin_memory=True).numpy() for _ in range(K)]
    for x in ins:
        x[...] = (rng.standard_normal(shape) * 1e-2).astype(np.float32)
    for k in range(K):
        a.set_dofs_f32_async(ins[k])
        a.advance_async(1)
        a.get_dofs_f32_async(outs[k])
    a.sync()
    for k in range(K):
        b.set_dofs_f32(ins[k])
        b.advance(1)
        assert np.array_equal(outs[k], b.get_dofs_f32()), k
    assert a.info.time == b.info.time
    assert np.array_equal(a.get_dofs_f32(), outs[-1])
    with pytest.raises(ValueError):
        a.set_dofs_f32_async(ins[0].astype(np.float64))
    with pytest.raises(ValueError):
        a.get_dofs_f32_async(np.empty(shape, np.float64))

def test_lts_coupled_graded_fp64():
    m, mat = syn.workloads.coupled_box(nxy=4, n_water=2, n_crust=2, L=8e3, depth=4e3, water=1e3,
                                       grading=4.0)
    o, s = make_pair(m, mat, 3, cfl=0.5, max_clusters=4)
    assert s.info.n_clusters >= 2
    Q0 = random_dofs((m.nt, s.B, 9), 3, N=3)
    o.Q = Q0.copy()
    s.set_dofs(to_gpu_layout(Q0))
    o.advance_macro()
    s.advance(1)
    assert rel_l2(to_oracle_layout(s.get_dofs()), o.Q) <= FP64_TOL


def test_ensemble_equals_independent_runs():
    m, mat = small_coupled()
    S = 3
    from paper_2107_06640_gb300 import Solver
    rho, lam, mu = mat
    ens = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, degree=3, cfl=0.5, ensemble=S)
    Qs = np.stack([to_gpu_layout(random_dofs((m.nt, ens.B, 9), 10 + k, N=3)) for k in range(S)], axis=1)
    ens.set_dofs(Qs)
    ens.advance(2)
    out = ens.get_dofs()
    for k in range(S):
        one = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, degree=3, cfl=0.5)
        one.set_dofs(Qs[:, k])
        one.advance(2)
        assert np.array_equal(one.get_dofs(), out[:, k])


def test_receivers_checkpoint_and_advance_to():
    m, mat = small_coupled()
    o, s = make_pair(m, mat, 3, cfl=0.5)
    Q0 = random_dofs((m.nt, s.B, 9), 5, N=3)
    o.Q = Q0.copy()
    s.set_dofs(to_gpu_layout(Q0))
    # checkpoint at t=0, run, restore, run again: bitwise identical
    buf = s.save_state()
    s.advance(2)
    first = s.get_dofs()
    s.load_state(buf)
    assert s.time == 0.0
    s.advance(2)
    assert np.array_equal(s.get_dofs(), first)
    # advance_to with a shortened final step
    s.load_state(buf)
    T = 2.37 * s.info.dt_min
    s.advance_to(T)
    o.step_gts()
    o.step_gts()
    o.step_gts(0.37 * o.dtmin)
    assert np.isclose(s.time, T)
    assert rel_l2(to_oracle_layout(s.get_dofs()), o.Q) <= FP64_TOL
    # receivers
    rng = np.random.default_rng(0)
    c = m.centroids()
    pts = c[rng.choice(m.nt, 7, replace=False)] + 10.0
    s.add_receivers(pts)
    got = s.read_receivers()[:, 0, :]
    from oracle.geometry import Geometry
    inside = []
    for p in pts:
        lam_ = np.einsum("ead,ed->ea", o.geo.Jinv, p[None] - o.geo.x0)
        bary = np.concatenate([lam_, 1 - lam_.sum(1, keepdims=True)], axis=1)
        inside.append(int(np.argmax(bary.min(1))))
    want = o.evaluate(np.array(inside), pts)
    assert rel_l2(got, want) <= FP64_TOL


def test_nan_is_reported():
    from paper_2107_06640_gb300 import AdgError
    m, mat = small_coupled()
    o, s = make_pair(m, mat, 2, cfl=0.5)
    Q = np.zeros((m.nt, 9, s.B))
    Q[5, 2, 1] = np.nan
    s.set_dofs(Q)
    with pytest.raises(AdgError) as ei:
        s.advance(1)
    assert ei.value.code == -6



def test_nan_is_reported_by_the_tensor_core_kernels():
    """A NaN in one dof of a periodic cube (every element on the tensor-core
    kernels) is reported after the step, in the first tile and in the last."""
    from paper_2107_06640_gb300 import AdgError, Solver, ADG_3XTF32
    m, mat = syn.unit_cube_periodic(4), syn.materials.elastic_uniform(384)
    for e in (5, 383):
        s = Solver(m.xyz, m.tets, m.face_tag, *mat, face_partner=m.face_partner, degree=5, cfl=0.5,
                   precision=ADG_3XTF32)
        Q = np.zeros((m.nt, 9, s.B))
        Q[e, 4, 17] = np.nan
        s.set_dofs(Q)
        with pytest.raises(AdgError) as ei:
            s.advance(1)
        assert ei.value.code == -6

@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (2, 1e-5)])
def test_full_size_coupled_box_sampled(precision, tol):
    """The 1.5 M-tet coupled ocean-crust box at N=5 (the benchmark workload),
    FP64 and the tensor-core 3xTF32 form: one global step from seeded dofs;
    60 sampled elements (interior, interface, surface, boundary) recomputed by
    the oracle on their neighbourhood.  3xTF32 tolerance: FP32 rounding of the
    dofs and one step of FP32-accumulated products (1e-5 relative L2)."""
    from synthetic.workloads import coupled_box, seafloor_pulse
    m, mat = coupled_box()
    assert m.nt == 1497600
    from paper_2107_06640_gb300 import Solver
    rho, lam, mu = mat
    s = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, degree=5, cfl=0.35, precision=precision)
    rng = np.random.default_rng(11)
    Q0 = rng.standard_normal((m.nt, 9, s.B)) * 1e-3
    s.set_dofs(Q0)
    ef, nxyz = s.gravity_faces()
    eta0 = 0.5 * np.sin(nxyz[..., 0] / 7e3)[:, None, :]
    s.set_eta(eta0)
    s.advance(1)
    Q1 = s.get_dofs()
    eta1 = s.read_ssh()[:, 0]
    # sample: 20 random, 20 at the sea surface, 20 at the sea floor
    wet = m.hex_index[:, 2] >= 35
    top = np.nonzero(np.any(m.face_tag == syn.TAG_GRAVITY, axis=1))[0]
    floor = np.nonzero(wet & (m.hex_index[:, 2] == 35))[0]
    side = np.nonzero(np.any(m.face_tag == syn.TAG_ABSORB, axis=1))[0]
    pick = np.concatenate([rng.choice(m.nt, 15, replace=False), rng.choice(top, 15, replace=False),
                           rng.choice(floor, 15, replace=False), rng.choice(side, 15, replace=False)])
    sub, smat, keep, pos = submesh(m, mat, pick)
    from oracle.ader import Oracle
    o = Oracle(sub.xyz, sub.tets, sub.face_tag, sub.face_partner, *smat, 5, cfl=0.35, dt=s.info.dt_min)
    o.Q = to_oracle_layout(Q0[keep])
    gmap = {int(v): g for g, v in enumerate(ef)}
    for i, e in enumerate(keep):
        for f in range(4):
            if sub.face_tag[i, f] == syn.TAG_GRAVITY:
                # eta0 = 0.5 sin(x/7e3) is not a polynomial: hand the oracle the
                # library's nodal values through their P_N interpolant
                g = gmap[int(e) * 4 + f]
                mono = [(a, b) for a in range(6) for b in range(6 - a)]
                Vn = np.array([[x ** a * y ** b for (a, b) in mono] for x, y in node_chi(5)])
                Vq = np.array([[x ** a * y ** b for (a, b) in mono] for x, y in o.chi])
                o.eta[i, f] = Vq @ np.linalg.solve(Vn, eta0[g, 0])
    o.step_gts()
    sel = pos[pick]
    got = to_oracle_layout(Q1[pick])
    assert rel_l2(got, o.Q[sel]) <= tol, rel_l2(got, o.Q[sel])
    for i, e in enumerate(keep):
        if pos[e] not in set(sel):
            continue
        for f in range(4):
            if sub.face_tag[i, f] == syn.TAG_GRAVITY:
                g = gmap[int(e) * 4 + f]
                want = oracle_eta_at_nodes(o, [i * 4 + f], node_chi(5), 5)[0]
                assert rel_l2(eta1[g], want) <= (FP64_TOL if precision == 0 else 1e-6)
