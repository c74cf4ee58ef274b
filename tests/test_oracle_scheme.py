"""Whole-scheme pins for the oracle: analytic solutions the paper's equations fix.

  * P plane wave in a periodic cube: error vs the analytic solution and
    convergence order N+1 (Sec. 4.1 ADER-DG, homogeneous elastic medium);
  * normal-incidence P wave on a solid/fluid interface: reflection and
    transmission coefficients (Z1-Z2)/(Z1+Z2), 2 Z1/(Z1+Z2) (Sec. 4.2);
  * standing surface-gravity wave in a uniform ocean over a rigid bottom:
    omega^2 = g m tanh(m H), m^2 = k^2 - omega^2/c^2, obtained from
    Eqs. (acoustics-pde) and (gravitational-bc) with the right-hand side
    dropped (Secs. 3, 4.3);
  * energy does not grow under the upwind flux;
  * rate-2 LTS: one cluster is bitwise global time stepping, two clusters
    keep the plane-wave error (Sec. 4.4).
"""

import numpy as np
import pytest
from scipy.optimize import brentq

import synthetic as syn
from oracle.ader import Oracle

R_P = np.array([-2.0, -1, -1, 0, 0, 0, 1, 0, 0])  # right-going P eigenvector, rho=1, lam=2, mu=1


def plane_wave(t, amp=1e-3):
    # q = amp r sin(k.x - omega t), k = 2 pi e_x, omega = c_p |k| = 4 pi
    return lambda x: amp * R_P * np.sin(2 * np.pi * x[..., 0:1] - 4 * np.pi * t)


def _periodic_oracle(n, N, **kw):
    m = syn.unit_cube_periodic(n)
    rho, lam, mu = syn.elastic_uniform(m.nt)
    return Oracle(m.xyz, m.tets, m.face_tag, m.face_partner, rho, lam, mu, N, **kw)


def _run_plane_wave(n, N, T):
    o = _periodic_oracle(n, N, cfl=0.5)
    o.Q = o.project(plane_wave(0.0))
    ns = int(np.ceil(T / o.dtmin))
    for _ in range(ns):
        o.step_gts(T / ns)
    return np.linalg.norm(o.l2_error(plane_wave(o.t)))


@pytest.mark.parametrize("N,n", [(2, 4), (3, 2), (5, 2)])
def test_plane_wave_convergence_order(N, n):
    e1 = _run_plane_wave(n, N, 0.05)
    e2 = _run_plane_wave(2 * n, N, 0.05)
    order = np.log2(e1 / e2)
    assert order > N + 1 - 0.35, (e1, e2, order)


def test_plane_wave_small_config():
    # 8^3 hexes x 6 tets, N=3, CFL 0.5, 100 steps, amplitude 1e-3
    o = _periodic_oracle(8, 3, cfl=0.5)
    assert o.E == 3072
    o.Q = o.project(plane_wave(0.0))
    for _ in range(100):
        o.step_gts()
    err = np.linalg.norm(o.l2_error(plane_wave(o.t)))
    ref = np.linalg.norm(o.l2_error(plane_wave(o.t), Q=0 * o.Q))
    assert 0.18 < o.t < 0.19
    assert err / ref < 2e-4, err / ref


def _interface_exact(t, Rc, Tc, c1=2.0, Z1=2.0, c2=1.0, Z2=1.0, x0=-0.8, w=0.2, amp=1e-3):
    f = lambda s: amp * np.exp(-((s - x0) / w) ** 2)

    def fn(x):
        X = x[..., 0]
        out = np.zeros(x.shape[:-1] + (9,))
        solid = X < 0
        vi, vr, vt = f(X - c1 * t), Rc * f(-X - c1 * t), Tc * f(X * c1 / c2 - c1 * t)
        out[..., 6] = np.where(solid, vi + vr, vt)
        out[..., 0] = np.where(solid, -Z1 * vi + Z1 * vr, -Z2 * vt)
        syy = np.where(solid, -(2.0 / c1) * vi + (2.0 / c1) * vr, -Z2 * vt)
        out[..., 1] = syy
        out[..., 2] = syy
        return out
    return fn


def test_solid_fluid_reflection_transmission():
    xs = np.linspace(-2, 2, 33)
    yz = np.linspace(0, 0.125, 2)
    m = syn.kuhn_box(xs, yz, yz, tags={"x-": 3, "x+": 3, "y-": 4, "y+": 4, "z-": 4, "z+": 4})
    cx = m.centroids()[:, 0]
    rho = np.ones(m.nt)
    lam = np.where(cx < 0, 2.0, 1.0)     # solid c_p = 2, Z = 2 | fluid c = 1, Z = 1
    mu = np.where(cx < 0, 1.0, 0.0)
    o = Oracle(m.xyz, m.tets, m.face_tag, m.face_partner, rho, lam, mu, 3, cfl=0.5)
    Z1, Z2 = 2.0, 1.0
    Rc, Tc = (Z1 - Z2) / (Z1 + Z2), 2 * Z1 / (Z1 + Z2)
    o.Q = o.project(_interface_exact(0.0, Rc, Tc))
    T = 0.8
    ns = int(np.ceil(T / o.dtmin))
    for _ in range(ns):
        o.step_gts(T / ns)
    ref = np.linalg.norm(o.l2_error(_interface_exact(o.t, Rc, Tc), Q=0 * o.Q))
    err = np.linalg.norm(o.l2_error(_interface_exact(o.t, Rc, Tc))) / ref
    bad = np.linalg.norm(o.l2_error(_interface_exact(o.t, -Rc, 2 - Tc))) / ref
    assert err < 1e-2 and bad > 0.5, (err, bad)


def _gravity_case(nx=4, nz=2, N=3, g=1.0, H=1.0, c=2.0, rho=1.0, L=2.0, amp=1e-2, zs=None, max_clusters=1):
    k = 2 * np.pi / L
    om = brentq(lambda w: w * w - g * np.sqrt(k * k - w * w / c / c) * np.tanh(np.sqrt(k * k - w * w / c / c) * H),
                1e-3, c * k * 0.999)
    m_ = np.sqrt(k * k - om * om / c / c)

    def exact(t, om=om, m_=m_):
        def fn(x):
            X, Zc = x[..., 0], x[..., 2]
            P = np.cosh(m_ * (Zc + H))
            out = np.zeros(x.shape[:-1] + (9,))
            p = amp * P * np.cos(k * X) * np.cos(om * t)
            out[..., 0] = out[..., 1] = out[..., 2] = -p
            out[..., 6] = amp * k * P * np.sin(k * X) * np.sin(om * t) / (rho * om)
            out[..., 8] = -amp * m_ * np.sinh(m_ * (Zc + H)) * np.cos(k * X) * np.sin(om * t) / (rho * om)
            return out
        return fn

    xs = np.linspace(0, L, nx + 1)
    ys = np.linspace(0, L / nx, 2)
    zs = np.linspace(-H, 0, nz + 1) if zs is None else np.asarray(zs, np.float64) * H
    msh = syn.kuhn_box(xs, ys, zs, tags={"x-": 4, "x+": 4, "y-": 4, "y+": 4, "z-": 6, "z+": 2})
    o = Oracle(msh.xyz, msh.tets, msh.face_tag, msh.face_partner, np.full(msh.nt, rho),
               np.full(msh.nt, rho * c * c), np.zeros(msh.nt), N, cfl=0.5, g=g, max_clusters=max_clusters)
    o.Q = o.project(exact(0.0))
    for e, f in np.argwhere(o.geo.face_tag == 2):
        o.eta[e, f] = amp * np.cosh(m_ * H) * np.cos(k * o.face_x[e, f, :, 0]) / (rho * g)
    return o, exact, om, k


def test_surface_gravity_wave_dispersion():
    o, exact, om, k = _gravity_case()
    T = np.pi / om  # half a period
    ns = int(np.ceil(T / o.dtmin))
    E0 = o.energy()
    for _ in range(ns):
        o.step_gts(T / ns)
    ref = np.linalg.norm(o.l2_error(exact(o.t), Q=0 * o.Q))
    err = np.linalg.norm(o.l2_error(exact(o.t))) / ref
    # the same mode with the shallow-water frequency sqrt(gH) k is far off
    bad = np.linalg.norm(o.l2_error(exact(o.t, om=k * 1.0))) / ref
    assert err < 1e-2 and bad > 0.1, (err, bad)
    assert o.energy() <= E0 * (1 + 1e-12)


@pytest.mark.parametrize("zs,top", [([-1, -0.9, -0.45, 0], 1), ([-1, -0.6, -0.2, -0.1, 0], 0)])
def test_surface_gravity_wave_with_lts(zs, top):
    """The standing surface-gravity wave under rate-2 LTS (Sec. 4.4) on a grid
    graded in depth: two clusters, with the gravitational surface in the
    coarse (top = 1) or the fine (top = 0) cluster, so the (eta, H) ODE runs
    over that cluster's step from its own Taylor expansion.  The error after
    half a period stays that of global time stepping on the same grid, and the
    energy (mechanical plus surface) does not grow."""
    g_, exact, om, k = _gravity_case(zs=zs, max_clusters=1)
    o, *_ = _gravity_case(zs=zs, max_clusters=2)
    assert np.bincount(o.cluster).size == 2
    assert set(o.cluster[np.argwhere(o.geo.face_tag == 2)[:, 0]]) == {top}
    T = np.pi / om
    errs = []
    for r in (g_, o):
        macro = r.dtmin * (1 << int(r.cluster.max()))
        ns = int(np.ceil(T / macro))
        E0 = r.energy()
        for _ in range(ns):
            r.advance_macro(T / ns / macro)
            assert r.energy() <= E0 * (1 + 1e-12)
        assert r.t == pytest.approx(T, rel=1e-13)
        ref = np.linalg.norm(r.l2_error(exact(r.t), Q=0 * r.Q))
        errs.append(np.linalg.norm(r.l2_error(exact(r.t))) / ref)
    assert errs[0] < 3e-3 and errs[1] < 1.05 * errs[0], errs


def test_energy_does_not_grow_periodic():
    o = _periodic_oracle(2, 3, cfl=0.5)
    rng = np.random.default_rng(3)
    o.Q = o.project(lambda x: np.sin(2 * np.pi * (x @ rng.standard_normal((3, 9)))))
    E = [o.energy()]
    for _ in range(20):
        o.step_gts()
        E.append(o.energy())
    E = np.array(E)
    assert np.all(E[1:] <= E[:-1] * (1 + 1e-12)), np.diff(E)


def test_energy_does_not_grow_with_absorbing_and_gravitational_boundaries():
    """The coupled box (ocean over crust, gravitational sea surface, absorbing
    sides and bottom): the energy, surface term included, does not grow in any
    step under the upwind flux; and the absorbing faces carry energy out,
    since the same box with rigid walls in their place keeps well over twice
    as much after the same 60 steps (there only the upwind dissipation of the
    rough start acts)."""
    from synthetic.workloads import coupled_box
    m, (rho, lam, mu) = coupled_box(nxy=2, n_water=1, n_crust=2, L=4e3, depth=3e3, water=1e3)
    assert set(np.unique(m.face_tag)) == {syn.TAG_INTERIOR, syn.TAG_GRAVITY, syn.TAG_ABSORB}
    W = np.random.default_rng(5).standard_normal((3, 9))
    fluid = mu == 0.0
    ends = []
    for tags in (m.face_tag, np.where(m.face_tag == syn.TAG_ABSORB, syn.TAG_RIGID, m.face_tag)):
        o = Oracle(m.xyz, m.tets, tags, m.face_partner, rho, lam, mu, 2, cfl=0.5)
        o.Q = o.project(lambda x: 1e-3 * np.sin(2 * np.pi * (x @ W) / 3e3))
        o.Q[fluid, :, 1] = o.Q[fluid, :, 0]
        o.Q[fluid, :, 2] = o.Q[fluid, :, 0]
        o.Q[fluid, :, 3:6] = 0.0
        o.eta[:] = np.random.default_rng(6).standard_normal(o.eta.shape) * 1e-3
        E = [o.energy()]
        for _ in range(60):
            o.step_gts()
            E.append(o.energy())
        E = np.array(E)
        assert np.all(E[1:] <= E[:-1] * (1 + 1e-12)), np.max(np.diff(E) / E[:-1])
        ends.append(E[-1] / E[0])
    assert ends[0] < 0.5 * ends[1], ends


def _warped_periodic(n, a=0.6):
    phi = lambda u: u - a * np.sin(2 * np.pi * u) / (2 * np.pi)
    g = np.linspace(0, 1, n + 1)
    return syn.kuhn_box(g, g, g, tags={s: 4 for s in syn.mesh.SIDES}, warp=lambda x, ijk: phi(x))


def test_lts_one_cluster_is_bitwise_gts_and_two_clusters_keep_accuracy():
    m = _warped_periodic(4)
    rho, lam, mu = syn.elastic_uniform(m.nt)
    mk = lambda mc: Oracle(m.xyz, m.tets, m.face_tag, m.face_partner, rho, lam, mu, 3, cfl=0.5,
                           max_clusters=mc)
    g1 = mk(1)
    g1.Q = g1.project(plane_wave(0.0))
    l1 = mk(1)
    l1.Q = g1.Q.copy()
    for _ in range(8):
        g1.step_gts()
        l1.advance_macro()
    assert np.array_equal(g1.Q, l1.Q)
    l2 = mk(2)
    assert np.bincount(l2.cluster).size == 2 and np.all(np.bincount(l2.cluster) > 0)
    l2.Q = l2.project(plane_wave(0.0))
    for _ in range(4):
        l2.advance_macro()
    assert np.isclose(l2.t, g1.t)
    e_gts = np.linalg.norm(g1.l2_error(plane_wave(g1.t)))
    e_lts = np.linalg.norm(l2.l2_error(plane_wave(l2.t)))
    assert e_lts < 1.5 * e_gts, (e_lts, e_gts)


@pytest.mark.parametrize("a,n_clusters", [(0.6, 2), (0.95, 3)])
def test_lts_conserves_the_element_means(a, n_clusters):
    """In a uniform periodic medium Eq. (elasticity-pde) is in conservation
    form and the Godunov flux is linear in the two time-integrated traces, so
    the scheme changes sum_e |J_e| Q_e,0 (the integral of q) by face terms that
    cancel between neighbours whenever both sides integrate the same states.
    Rate-2 LTS (Sec. 4.4) gives them the same states: the coarse side takes the
    fine side's buffer (the sum of its integrals over the coarse step), the
    fine side the coarse Taylor expansion integrated over each sub-interval,
    which sum to the coarse integral.  So the integral of q is conserved to
    rounding with any number of clusters."""
    m = _warped_periodic(4, a)
    rho, lam, mu = syn.elastic_uniform(m.nt)
    o = Oracle(m.xyz, m.tets, m.face_tag, m.face_partner, rho, lam, mu, 3, cfl=0.5, max_clusters=n_clusters)
    assert np.bincount(o.cluster).size == n_clusters
    rng = np.random.default_rng(11)
    W = rng.standard_normal((3, 9))
    o.Q = o.project(lambda x: 1.0 + np.sin(2 * np.pi * (x @ W)))
    total = lambda: np.einsum("e,ep->p", o.geo.detJ, o.Q[:, 0, :])
    t0 = total()
    scale = np.einsum("e,ep->p", o.geo.detJ, np.abs(o.Q[:, 0, :])).max()
    for _ in range(3):
        o.advance_macro()
    assert np.max(np.abs(total() - t0)) <= 1e-13 * scale
    # the solution did change
    assert np.max(np.abs(o.Q[:, 1:, :])) > 0 and not np.allclose(o.Q, o.project(lambda x: 1.0 + np.sin(2 * np.pi * (x @ W))))


def test_fluid_stress_stays_isotropic():
    """The acoustic special case of Sec. 4.1 (mu = 0, s_ij = -p delta_ij) is an
    invariant subspace of the discrete scheme: with mu = 0 every stress
    update of a fluid element, in the volume term and in the Godunov flux (also
    across the fluid-solid interface and the gravitational surface), is lambda
    times a divergence or a normal velocity jump times the identity.  So fluid
    elements that start with s_xx = s_yy = s_zz and no shear stress keep that
    form.  The 4-quantity (p, v) ocean is this restriction."""
    from synthetic.workloads import coupled_box
    m, (rho, lam, mu) = coupled_box(nxy=2, n_water=1, n_crust=1, L=4e3, depth=2e3, water=1e3)
    N = 3
    o = Oracle(m.xyz, m.tets, m.face_tag, m.face_partner, rho, lam, mu, N, cfl=0.5)
    rng = np.random.default_rng(4)
    Q = rng.standard_normal(o.Q.shape) * 1e-3
    fluid = mu == 0.0
    assert fluid.any() and (~fluid).any()
    p = rng.standard_normal(Q[fluid].shape[:2]) * 1e-3
    for i in range(3):
        Q[fluid, :, i] = -p
    Q[fluid, :, 3:6] = 0.0
    o.Q = Q
    o.eta[:] = rng.standard_normal(o.eta.shape) * 1e-2
    for _ in range(3):
        o.step_gts()
    Qf = o.Q[fluid]
    scale = np.abs(Qf[..., 0]).max()
    assert scale > 0
    assert np.max(np.abs(Qf[..., 1] - Qf[..., 0])) <= 1e-12 * scale
    assert np.max(np.abs(Qf[..., 2] - Qf[..., 0])) <= 1e-12 * scale
    assert np.max(np.abs(Qf[..., 3:6])) <= 1e-12 * scale


@pytest.mark.parametrize("N", [2, 4])
def test_projection_and_point_evaluation_reproduce_a_polynomial(N):
    """The receiver readout (Sec. 5 outputs): a field that is a polynomial of
    degree N in x, y, z lies in every element's space P_N, so its L2
    projection is exact and evaluating the element polynomial at any point
    inside the element returns the field, on a warped (non-uniform) mesh
    where each tet has its own affine map."""
    m = _warped_periodic(3)
    rho, lam, mu = syn.elastic_uniform(m.nt)
    o = Oracle(m.xyz, m.tets, m.face_tag, m.face_partner, rho, lam, mu, N, cfl=0.5)
    rng = np.random.default_rng(5)
    terms = [(i, j, k) for i in range(N + 1) for j in range(N + 1 - i) for k in range(N + 1 - i - j)]
    coef = rng.standard_normal((len(terms), 9))

    def field(x):
        mono = np.stack([x[..., 0] ** i * x[..., 1] ** j * x[..., 2] ** k for (i, j, k) in terms], axis=-1)
        return mono @ coef

    o.Q = o.project(field)
    e = rng.integers(0, o.E, 40)
    lam4 = rng.dirichlet(np.ones(4), size=e.size)
    x = np.einsum("rk,rkd->rd", lam4, m.xyz[m.tets[e]])
    want = field(x)
    got = o.evaluate(e, x)
    assert np.max(np.abs(got - want)) <= 1e-11 * np.abs(want).max()


def test_energy_is_the_integral_of_the_energy_density():
    """Oracle.energy (used by the non-growth pins) against a direct quadrature:
    1/2 rho |v|^2 + 1/2 sigma . C^-1 sigma with C the 6 x 6 Voigt stiffness
    (engineering shear strain) inverted numerically in the solid, p^2 / (2 K)
    with p = -tr(sigma)/3 in the fluid, plus 1/2 rho g eta^2 on the
    gravitational surface (Secs. 3, 4.3)."""
    from oracle import basis as ob
    from oracle.quadrature import tet_rule, tri_rule
    from synthetic.workloads import coupled_box
    m, (rho, lam, mu) = coupled_box(nxy=2, n_water=1, n_crust=1, L=4e3, depth=2e3, water=1e3)
    N = 2
    o = Oracle(m.xyz, m.tets, m.face_tag, m.face_partner, rho, lam, mu, N, cfl=0.5)
    rng = np.random.default_rng(8)
    o.Q = rng.standard_normal(o.Q.shape) * np.array([1e5] * 6 + [1e-2] * 3)
    fluid = mu == 0
    o.Q[fluid, :, 1] = o.Q[fluid, :, 0]
    o.Q[fluid, :, 2] = o.Q[fluid, :, 0]
    o.Q[fluid, :, 3:6] = 0.0
    o.eta[:] = rng.standard_normal(o.eta.shape) * 0.1
    pts, w = tet_rule(2 * N)
    phi = ob.eval_basis(N, pts)
    want = 0.0
    for e in range(o.E):
        q = phi @ o.Q[e]                                      # (nq, 9)
        kin = 0.5 * rho[e] * np.sum(q[:, 6:] ** 2, axis=1)
        if fluid[e]:
            p = -q[:, :3].sum(1) / 3
            pot = p ** 2 / (2 * lam[e])
        else:
            C = np.zeros((6, 6))
            C[:3, :3] = lam[e]
            C[np.arange(3), np.arange(3)] += 2 * mu[e]
            C[np.arange(3, 6), np.arange(3, 6)] = mu[e]
            Sinv = np.linalg.inv(C)
            pot = 0.5 * np.einsum("qi,ij,qj->q", q[:, :6], Sinv, q[:, :6])
        want += o.geo.volume[e] * 6 * np.sum(w * (kin + pot))   # |J| = 6 V, sum w = 1/6
    _, fw = tri_rule(2 * N)
    for e, f in np.argwhere(o.geo.face_tag == 2):
        want += o.geo.area[e, f] * 2 * np.sum(fw * 0.5 * rho[e] * o.g * o.eta[e, f] ** 2)
    assert o.energy() == pytest.approx(want, rel=1e-12)
