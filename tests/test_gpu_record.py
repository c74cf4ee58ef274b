"""Recording at a cadence (adg_record_*): the samples a ring collects while
adg_advance runs equal the synchronous readouts of the same states, the
ring keeps the newest samples and counts the overwritten ones, and the calls
refuse what they cannot do."""

import numpy as np
import pytest

from tests._cases import small_coupled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2107_06640_gb300 import build
    build.build()


def _pair(precision):
    from paper_2107_06640_gb300 import Solver
    m, (rho, lam, mu) = small_coupled()
    kw = dict(degree=3, cfl=0.5, precision=precision, ensemble=2)
    a = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, **kw)
    b = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, **kw)
    rng = np.random.default_rng(7)
    Q = rng.standard_normal((m.nt, 2, 9, a.B)) * 1e-3
    rec = np.stack([m.xyz[m.tets[k]].mean(0) for k in (0, m.nt // 3, m.nt // 2, m.nt - 1)])
    for s in (a, b):
        s.set_dofs(Q)
        ef, xyz = s.gravity_faces()
        s.set_eta(np.stack([np.sin(xyz[..., 0] / 7e3), np.cos(xyz[..., 1] / 5e3)], axis=1))
        s.add_receivers(rec)
    return m, a, b


@pytest.mark.parametrize("precision", [0, 1])
def test_recorded_samples_equal_synchronous_readouts(precision):
    from paper_2107_06640_gb300 import _lib
    m, a, b = _pair(precision)
    R, H = _lib.ADG_RECORD_RECEIVERS, _lib.ADG_RECORD_SSH
    a.record(R, every=2, capacity=3)
    a.record(H, every=3, capacity=4)
    a.advance(6)
    want_r, want_h, t_r, t_h = [], [], [], []
    for k in range(1, 7):
        b.advance(1)
        if k % 2 == 0:
            want_r.append(b.read_receivers())
            t_r.append(b.query().time)
        if k % 3 == 0:
            want_h.append(b.read_ssh())
            t_h.append(b.query().time)
    t, got, dropped = a.read_record(R)
    assert dropped == 0 and len(t) == 3
    assert np.array_equal(got, np.array(want_r)) and np.array_equal(t, np.array(t_r))
    t, got, dropped = a.read_record(H)
    assert dropped == 0 and len(t) == 2
    assert np.array_equal(got, np.array(want_h)) and np.array_equal(t, np.array(t_h))
    # nothing new until the next due step
    t, got, _ = a.read_record(R)
    assert len(t) == 0


def test_ring_keeps_the_newest_and_counts_the_dropped():
    from paper_2107_06640_gb300 import _lib
    m, a, b = _pair(1)
    R = _lib.ADG_RECORD_RECEIVERS
    a.record(R, every=1, capacity=2)
    a.advance(5)
    b.advance(4)
    r4 = b.read_receivers()
    b.advance(1)
    r5 = b.read_receivers()
    t, got, dropped = a.read_record(R, max_samples=1)
    assert dropped == 3 and len(t) == 1 and np.array_equal(got[0], r4)
    t, got, dropped = a.read_record(R)
    assert dropped == 3 and len(t) == 1 and np.array_equal(got[0], r5)


def test_partial_step_of_advance_to_is_sampled_at_the_target_time():
    from paper_2107_06640_gb300 import _lib
    m, a, b = _pair(0)
    H = _lib.ADG_RECORD_SSH
    dt = a.query().macro_dt
    a.record(H, every=1, capacity=8)
    a.advance_to(2.5 * dt)
    t, got, _ = a.read_record(H)
    assert len(t) == 3 and t[-1] == pytest.approx(2.5 * dt, rel=1e-14)
    assert np.array_equal(got[-1], a.read_ssh())


def test_record_calls_refuse_what_they_cannot_do():
    from paper_2107_06640_gb300 import AdgError, _lib
    m, a, b = _pair(1)
    R, H = _lib.ADG_RECORD_RECEIVERS, _lib.ADG_RECORD_SSH
    with pytest.raises(AdgError) as ei:
        a.read_record(H)  # not started
    assert ei.value.code == -3
    with pytest.raises(AdgError):
        a.record(R, every=0, capacity=4)
    a.record(R, every=1, capacity=4)
    with pytest.raises(AdgError) as ei:
        a.add_receivers(np.zeros((1, 3)) + m.xyz.mean(0))
    assert ei.value.code == -3
    a.stop_record(R)
    a.add_receivers(np.zeros((1, 3)) + m.xyz.mean(0))  # allowed again


@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 2e-6)])
def test_hydrostatic_start_is_exact_for_a_polynomial_sea_surface(precision, tol):
    """adg_hydrostatic_start: with a sea surface of degree 3 on the flat top of
    the coupled box, p' = rho g eta(x, y) is a cubic in every water tet, so its
    projection at degree 3 is exact: receivers in the water read
    s_xx = s_yy = s_zz = -rho g eta(x, y), zero shear stress and velocity, in
    both scenarios (each its own surface); the solid keeps its dofs."""
    from paper_2107_06640_gb300 import AdgError, Solver
    m, (rho, lam, mu) = small_coupled()
    s = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, degree=3, cfl=0.5, precision=precision, ensemble=2)
    rng = np.random.default_rng(9)
    Q0 = rng.standard_normal((m.nt, 2, 9, s.B)) * 1e-3
    s.set_dofs(Q0)
    surf = [lambda x, y: 0.3 + 1e-4 * x - 2e-4 * y + 3e-11 * x * x * y,
            lambda x, y: -0.2 + 5e-8 * x * y - 4e-12 * y ** 3]
    ef, xyz = s.gravity_faces()
    s.set_eta(np.stack([f(xyz[..., 0], xyz[..., 1]) for f in surf], axis=1))
    s.hydrostatic_start()
    water = np.nonzero(mu == 0.0)[0]
    solid = np.nonzero(mu > 0.0)[0]
    assert water.size and solid.size
    got = s.get_dofs_subset(solid)
    want = Q0[solid].astype(np.float32).astype(np.float64) if precision == 1 else Q0[solid]
    assert np.array_equal(got, want)
    # points inside water tets (random barycentric weights)
    pick = rng.choice(water, 12, replace=False)
    lam4 = rng.dirichlet(np.ones(4), size=pick.size)
    pts = np.einsum("rk,rkd->rd", lam4, m.xyz[m.tets[pick]])
    s.add_receivers(pts)
    r = s.read_receivers()  # [n][S][9]
    g = 9.81
    for k, f in enumerate(surf):
        p = rho[pick] * g * f(pts[:, 0], pts[:, 1])
        scale = np.abs(p).max()
        for q in range(3):
            assert np.max(np.abs(r[:, k, q] + p)) <= tol * scale
        assert np.max(np.abs(r[:, k, 3:])) <= tol * scale


def test_hydrostatic_start_needs_a_sea_surface():
    from paper_2107_06640_gb300 import AdgError, Solver
    import synthetic as syn
    m = syn.unit_cube_periodic(2)
    s = Solver(m.xyz, m.tets, m.face_tag, *syn.materials.elastic_uniform(m.nt), face_partner=m.face_partner,
               degree=2, cfl=0.5)
    with pytest.raises(AdgError) as ei:
        s.hydrostatic_start()
    assert ei.value.code == -3
