"""Pins of the oracle's linear slip-weakening friction (Sec. 5, Scenario-A
fault; Eq. bc-dynrup with the slip path length as state) against closed
forms: the friction coefficient, a fault that stays locked, and a fault under
constant load, whose state obeys dpsi/dt = A + B psi until psi = D_c and
slides at a constant rate after."""

import numpy as np
import pytest

from oracle import rupture as ru

RHO, LAM, MU = 3000.0, 3.0e10, 3.0e10
ETA = np.sqrt(RHO * MU) / 2.0  # both sides alike: Zs- Zs+ / (Zs- + Zs+)


def _par(npts, mu_s=0.6, mu_d=0.4, Dc=0.5, C=2e6, sn0=-40e6, tau=20e6, psi=0.0, V=0.0):
    """Parameters of npts points with the shear prestress along x on a fault
    with normal z (its normal part zero)."""
    p = {k: np.zeros(npts) for k in ru.LSW_PARAMS}
    p.update(mu_s=np.full(npts, mu_s), mu_d=np.full(npts, mu_d), Dc=np.full(npts, Dc), C=np.full(npts, C),
             sn0=np.full(npts, sn0), t0x=np.full(npts, tau), psi=np.full(npts, psi), V=np.full(npts, V))
    return p


def _run(par, dt, steps, N=3):
    """Both sides at rest (zero perturbation), so Theta = |tau0| and S = -sn0
    at every time point; returns psi, |V|, slip, traction after each step."""
    npts = par["psi"].size
    n = np.tile([0.0, 0.0, 1.0], (npts, 1))
    q = np.zeros((N + 1, npts, 9))
    mat = tuple(np.full(npts, v) for v in (RHO, LAM, MU))
    hist = []
    slip = np.zeros((npts, 3))
    for _ in range(steps):
        Gm, Gp, psi, V, dslip, iters, tau = ru.solve_step(n, q, q, mat, mat, par, dt, N, law="lsw")
        assert not iters.any()
        par = dict(par, psi=psi, V=V)
        slip = slip + dslip
        hist.append((psi.copy(), V.copy(), slip.copy(), tau.copy()))
    return hist


def test_friction_coefficient_is_linear_in_slip_then_constant():
    p = dict(mu_s=0.6, mu_d=0.4, Dc=0.5)
    psi = np.array([0.0, 0.125, 0.25, 0.5, 0.9, 7.0])
    assert np.allclose(ru.lsw_friction(psi, p), [0.6, 0.55, 0.5, 0.4, 0.4, 0.4], rtol=0, atol=1e-15)


def test_fault_below_strength_stays_locked():
    # |tau0| = 20 MPa < C + mu_s S = 2 + 0.6 * 40 = 26 MPa
    hist = _run(_par(4, tau=20e6), dt=1e-3, steps=5)
    psi, V, slip, tau = hist[-1]
    assert np.all(V == 0) and np.all(psi == 0) and np.all(slip == 0)
    assert np.allclose(tau, [[20e6, 0, 0]] * 4, rtol=1e-15)


def _closed_form(t, Th, S, C, mu_s, mu_d, Dc, eta, psi0=0.0):
    """Slip path length under constant Theta and S: dpsi/dt = A + B psi with
    A = (Th - C - mu_s S)/eta, B = (mu_s - mu_d) S / (Dc eta) until psi = Dc,
    then constant V_d = (Th - C - mu_d S)/eta."""
    A = (Th - C - mu_s * S) / eta
    B = (mu_s - mu_d) * S / (Dc * eta)
    tc = np.log((Dc + A / B) / (psi0 + A / B)) / B
    return np.where(t <= tc, (psi0 + A / B) * np.exp(B * t) - A / B, Dc + (Th - C - mu_d * S) / eta * (t - tc))


@pytest.mark.parametrize("N", [2, 3])
def test_overloaded_fault_follows_the_closed_form(N):
    """Theta = 27 MPa above the static strength 26 MPa: the slip path
    length grows as the exponential closed form until it reaches D_c, then
    the fault slides at (Theta - C - mu_d S)/eta; the scheme converges at
    first order in dt (each step's tail, after the last time point, advances
    the state with the frozen last rate), and while sliding the traction
    equals the strength."""
    Th, S, C, mu_s, mu_d, Dc = 27e6, 40e6, 2e6, 0.6, 0.4, 0.5
    A = (Th - C - mu_s * S) / ETA
    T = 1.0
    errs = []
    for steps in (40, 80, 160):
        dt = T / steps
        hist = _run(_par(1, mu_s=mu_s, mu_d=mu_d, Dc=Dc, C=C, sn0=-S, tau=Th, V=A), dt, steps, N=N)
        t = dt * np.arange(1, steps + 1)
        psi = np.array([h[0][0] for h in hist])
        want = _closed_form(t, Th, S, C, mu_s, mu_d, Dc, ETA)
        errs.append(np.max(np.abs(psi - want)))
        assert want[-1] > 2 * Dc  # the run covers both regimes
        # slip runs along the prestress; its Gauss-weighted integral of |V|
        # approximates the same path length
        slip = np.array([h[2][0] for h in hist])
        assert np.all(slip[:, 1:] == 0)
        assert np.max(np.abs(slip[:, 0] - want)) < 2e-3 * want[-1]
        # once weakened: constant rate and the traction at the dynamic strength
        psi_end, V_end, _, tau_end = hist[-1]
        assert psi_end[0] > Dc
        assert V_end[0] == pytest.approx((Th - C - mu_d * S) / ETA, rel=1e-13)
        assert np.linalg.norm(tau_end[0]) == pytest.approx(C + mu_d * S, rel=1e-13)
    assert errs[0] < 2e-3 * want[-1]
    assert errs[0] / errs[1] > 1.8 and errs[1] / errs[2] > 1.8


def test_traction_is_the_strength_while_weakening():
    """Mid-weakening (psi < D_c) the fault traction is C + f(psi) S with the
    state at the last time point, and theta - eta |V| gives it."""
    Th, S, C = 27e6, 40e6, 2e6
    hist = _run(_par(1, C=C, sn0=-S, tau=Th, V=(Th - C - 0.6 * S) / ETA), dt=2e-3, steps=3, N=3)
    psi, V, _, tau = hist[-1]
    assert 0 < psi[0] < 0.5
    # the last time point's state is psi advanced by the rest of the step
    tj, _ = ru.time_points(3, 2e-3)
    psi_last = psi[0] - V[0] * (2e-3 - tj[-1])
    want = C + ru.lsw_friction(np.array([psi_last]), dict(mu_s=0.6, mu_d=0.4, Dc=0.5))[0] * S
    assert np.linalg.norm(tau[0]) == pytest.approx(want, rel=1e-12)
    assert Th - ETA * V[0] == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("N,zs,lts", [(2, (-2e3, -1e3, 0.0), False), (3, (-2e3, -1e3, 0.0), False),
                                      (3, (-2e3, -1.6e3, 0.0), True)])
def test_locked_fault_in_the_scheme_equals_welded_interior_faces(N, zs, lts):
    """A fault that cannot slip (cohesion far above any traction, so |V| = 0
    exactly) is a welded interface: the whole scheme with it equals the same
    mesh with those faces interior, to rounding.  This pins the fault path at
    element level: its traces at the fault nodes (exact, the states are of
    degree N on the face), the N+1 Gauss points in time (exact for the degree-N
    time dependence), the nodal-to-Gauss interpolation and the lift into both
    elements with the area / |J| scaling of each side (Sec. 4.2, Eq.
    bc-dynrup); the elements on either side have different materials and,
    on a warped grid (so the fault is not planar either), different volumes.
    With rate-2 LTS (Sec. 4.4) the fault faces lie in both clusters and the
    fault is solved over each cluster's step from the stored expansions; the
    welded mesh takes the same clusters."""
    from oracle.ader import Oracle
    from synthetic.mesh import kuhn_box

    def warp(x, ijk):
        x[:, 0] += 150 * np.sin(x[:, 2] / 700.0) + 90 * np.cos(x[:, 1] / 500.0)
        x[:, 2] += 120 * np.sin(x[:, 0] / 900.0)
        return x

    m = kuhn_box(np.linspace(0, 4e3, 5), np.linspace(0, 2e3, 3), np.array(zs), warp=warp,
                 fault=dict(c=0, jrange=(0, 2), krange=(0, 2)))
    g = np.random.default_rng(3)
    rho = 2700.0 * (1 + 0.2 * g.uniform(-1, 1, m.nt))
    mu = 3.2e10 * (1 + 0.2 * g.uniform(-1, 1, m.nt))
    lam = mu * (1 + 0.3 * g.uniform(0, 1, m.nt))
    mc = 2 if lts else 1
    fault = Oracle(m.xyz, m.tets, m.face_tag, m.face_partner, rho, lam, mu, N, cfl=0.5, max_clusters=mc)
    welded = Oracle(m.xyz, m.tets, np.where(m.face_tag == 5, 0, m.face_tag), m.face_partner, rho, lam, mu, N,
                    cfl=0.5, max_clusters=mc)
    welded.cluster = fault.cluster.copy()
    assert fault.nff == 8 and welded.nff == 0
    assert np.unique(fault.cluster[fault.fm[:, 0]]).size == (2 if lts else 1)
    Bf = (N + 1) * (N + 2) // 2
    par = {k: np.zeros((fault.nff, Bf)) for k in ru.LSW_PARAMS}
    par.update(mu_s=np.full((fault.nff, Bf), 0.6), mu_d=np.full((fault.nff, Bf), 0.4),
               Dc=np.full((fault.nff, Bf), 0.5), C=np.full((fault.nff, Bf), 1e30),
               sn0=np.full((fault.nff, Bf), -40e6))
    fault.set_fault(par, law="lsw")
    Q0 = g.standard_normal(fault.Q.shape) * np.array([1e6] * 6 + [1.0] * 3)
    fault.Q, welded.Q = Q0.copy(), Q0.copy()
    for _ in range(3):
        for o in (fault, welded):
            o.advance_macro() if lts else o.step_gts()
    assert np.all(fault.fault["V"] == 0) and np.all(fault.fault["slip"] == 0)
    for p in range(9):
        sc = np.abs(welded.Q[..., p]).max()
        assert np.max(np.abs(fault.Q[..., p] - welded.Q[..., p])) <= 1e-11 * sc, p
    assert not np.allclose(welded.Q, Q0)


@pytest.mark.parametrize("dP", [5e6, -5e6])
def test_normal_stress_change_moves_the_strength(dP):
    """The strength acts on the total normal stress (Eq. bc-dynrup: S from the
    background sigma_n0 plus the dynamic normal stress of the middle state).
    Both sides carry an extra isotropic stress -dP I, which puts no shear on
    the fault (Theta = |tau0| stays 27 MPa) and makes the welded normal stress
    -dP: extra compression (dP > 0) raises the static strength
    C + mu_s (40 MPa + dP) above Theta and the fault stays locked; extra
    tension lowers it and the fault slides with the traction at the strength
    C + f(psi) (40 MPa + dP)."""
    Th, S0, C = 27e6, 40e6, 2e6
    N, dt = 3, 2e-3
    n = np.tile([0.0, 0.0, 1.0], (1, 1))
    q = np.zeros((N + 1, 1, 9))
    q[..., :3] = -dP
    mat = tuple(np.full(1, v) for v in (RHO, LAM, MU))
    par = _par(1, C=C, sn0=-S0, tau=Th)
    Gm, Gp, psi, V, dslip, iters, tau = ru.solve_step(n, q, q, mat, mat, par, dt, N, law="lsw")
    S = S0 + dP
    if dP > 0:
        assert V[0] == 0 and psi[0] == 0 and np.allclose(tau[0], [Th, 0, 0], rtol=1e-15)
    else:
        assert V[0] > 0 and psi[0] > 0
        tj, _ = ru.time_points(N, dt)
        psi_last = psi[0] - V[0] * (dt - tj[-1])
        want = C + ru.lsw_friction(np.array([psi_last]), dict(mu_s=0.6, mu_d=0.4, Dc=0.5))[0] * S
        assert np.linalg.norm(tau[0]) == pytest.approx(want, rel=1e-12)
