"""Pins for the oracle's fault solve (Sec. 3, Eq. bc-dynrup, and its readings)."""

import numpy as np

from oracle import physics as ph
from oracle import rupture as ru

rng = np.random.default_rng(5)


def _par(n, **over):
    p = dict(a=np.full(n, 0.01), b=np.full(n, 0.014), L=np.full(n, 0.2), f0=np.full(n, 0.6),
             V0=np.full(n, 1e-6), fw=np.full(n, 0.1), Vw=np.full(n, 0.1), sn0=np.full(n, -40e6),
             t0x=np.zeros(n), t0y=np.zeros(n), t0z=np.zeros(n), psi=np.full(n, 0.6), V=np.full(n, 1e-12))
    p.update({k: np.broadcast_to(v, (n,)).astype(float).copy() for k, v in over.items()})
    return p


def test_steady_state_law_is_consistent():
    # f(V, psi_ss(V)) = f_ss(V): the two halves of the law agree
    p = _par(50)
    V = np.logspace(-14, 1, 50)
    assert np.allclose(ru.friction(V, ru.psi_ss(V, p), p), ru.f_ss(V, p), rtol=1e-12)
    # low slip rate: f_ss -> f0 - (b-a) ln(V/V0);  high: -> f_w
    assert np.isclose(ru.f_ss(np.array([1e-6]), _par(1))[0], 0.6, rtol=1e-9)
    assert abs(ru.f_ss(np.array([1e3]), _par(1))[0] - 0.1) < 1e-3


def test_state_relaxation_is_the_exact_ode_solution():
    p = _par(1)
    V, psi0, h = np.array([0.3]), np.array([0.7]), 0.05
    # fine RK4 integration of dpsi/dt = -(V/L)(psi - psi_ss(V))
    y = psi0.copy()
    n = 2000
    ss = ru.psi_ss(V, p)
    rhs = lambda y: -(V / p["L"]) * (y - ss)
    for _ in range(n):
        k1 = rhs(y)
        k2 = rhs(y + 0.5 * h / n * k1)
        k3 = rhs(y + 0.5 * h / n * k2)
        k4 = rhs(y + h / n * k3)
        y = y + h / n / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    assert np.allclose(ru.psi_relax(psi0, V, h, p), y, rtol=1e-12)


def test_newton_agrees_with_bisection_and_has_zero_residual():
    n = 200
    p = _par(n)
    Theta = rng.uniform(0, 40e6, n)
    S = rng.uniform(1e6, 60e6, n)
    eta = rng.uniform(2e6, 8e6, n)
    psi = rng.uniform(0.3, 0.9, n)
    V, it, ok = ru.newton_slip_rate(Theta, S, eta, psi, p, np.full(n, 1e-12))
    assert np.all(ok) and it.max() < 100
    Vb = ru.bisect_slip_rate(Theta, S, eta, psi, p)
    ok_ = (Vb > 1e-290)
    assert np.allclose(V[ok_], Vb[ok_], rtol=1e-9, atol=0)
    # the root is bracketed within a relative 1e-8 (g is steep near V ~ 2 V0 e^{-psi/a})
    g = lambda v: Theta - eta * v - S * ru.friction(v, psi, p)
    assert np.all(g(V * (1 - 1e-8)) >= 0) and np.all(g(V * (1 + 1e-8)) <= 0)
    assert it.max() <= 12


def _states(npts):
    n = rng.standard_normal((npts, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    qm = rng.standard_normal((npts, 9)) * 1e6
    qp = rng.standard_normal((npts, 9)) * 1e6
    qm[:, 6:] *= 1e-6
    qp[:, 6:] *= 1e-6
    return n, qm, qp


def _mat(npts, rho, vp, vs):
    return (np.full(npts, rho), np.full(npts, rho * (vp ** 2 - 2 * vs ** 2)), np.full(npts, rho * vs ** 2))


def test_locked_fault_is_the_welded_interface():
    # infinite strength (V = 0): the fault flux equals the interior Godunov flux
    npts = 20
    n, qm, qp = _states(npts)
    matm, matp = _mat(npts, 2700, 6000, 3464), _mat(npts, 3000, 6500, 3700)
    st = ru.fault_states(n, qm, qp, matm, matp, np.zeros((npts, 3)), np.full(npts, -1e30))
    t_b, vb, vc, Vv, _ = ru.middle_traction_velocity(st, np.zeros(npts), n)
    Fm = ru.ahat_apply(n, t_b, vb, *matm)
    R = ph.frame(n)
    wm, wp = ph.rotate_in(qm, R), ph.rotate_in(qp, R)
    Zpm, Zsm = ph.impedances(*matm)
    Zpp, Zsp = ph.impedances(*matp)
    wb = ph.middle_state(wm, wp, Zpm, Zpp, Zsm, Zsp)
    F = ph.rotate_out(ph.flux_rotated(wb, *matm), R)
    assert np.allclose(Fm, F, rtol=1e-10, atol=1e-12 * np.abs(F).max())
    # the plus side sees the same interface from the other side
    Fp = -ru.ahat_apply(n, t_b, vc, *matp)
    Rn = ph.frame(-n)
    wm2, wp2 = ph.rotate_in(qp, Rn), ph.rotate_in(qm, Rn)
    wb2 = ph.middle_state(wm2, wp2, Zpp, Zpm, Zsp, Zsm)
    F2 = ph.rotate_out(ph.flux_rotated(wb2, *matp), Rn)
    assert np.allclose(Fp, F2, rtol=1e-10, atol=1e-12 * np.abs(F2).max())


def test_slipping_fault_obeys_the_friction_conditions():
    npts = 30
    n, qm, qp = _states(npts)
    mat = _mat(npts, 2700, 6000, 3464)
    tau0 = rng.standard_normal((npts, 3)) * 30e6
    p = _par(npts)
    st = ru.fault_states(n, qm, qp, mat, mat, tau0, p["sn0"])
    Th = np.linalg.norm(st["Thv"], axis=-1)
    V, _, ok = ru.newton_slip_rate(Th, st["S"], st["eta"], p["psi"], p, np.full(npts, 1e-12))
    t_b, vb, vc, Vv, tau_tot = ru.middle_traction_velocity(st, V, n)
    # |tau| = S f(|V|, psi) and V parallel to tau (Eq. bc-dynrup)
    assert np.allclose(np.linalg.norm(tau_tot, axis=1), st["S"] * ru.friction(V, p["psi"], p), rtol=1e-8)
    cross = np.cross(tau_tot, Vv)
    assert np.all(np.linalg.norm(cross, axis=1) <= 1e-9 * np.linalg.norm(tau_tot, axis=1) * (V + 1e-30))
    # slip rate is the tangential velocity jump between the two middle states
    assert np.allclose(vc - vb, Vv, atol=1e-9 * (np.abs(Vv).max() + 1e-30))
    # V tangential, normal velocity and normal stress continuous
    assert np.allclose(np.sum(Vv * n, 1), 0.0, atol=1e-12 * np.abs(Vv).max())


def test_zero_strength_leaves_no_shear_traction():
    npts = 10
    n, qm, qp = _states(npts)
    mat = _mat(npts, 2700, 6000, 3464)
    tau0 = rng.standard_normal((npts, 3)) * 1e6
    st = ru.fault_states(n, qm, qp, mat, mat, tau0, np.full(npts, 1e30))  # tension: S = 0
    assert np.all(st["S"] == 0)
    Th = np.linalg.norm(st["Thv"], axis=-1)
    V, _, _ = ru.newton_slip_rate(Th, st["S"], st["eta"], np.full(npts, 0.6), _par(npts), np.zeros(npts))
    assert np.allclose(V, Th / st["eta"], rtol=1e-12)
    *_, tau_tot = ru.middle_traction_velocity(st, V, n)
    assert np.abs(tau_tot).max() < 1e-6


def test_step_under_constant_load_converges_to_the_fault_ode():
    """With both sides at rest the fault sees constant Theta and S, and Eq.
    bc-dynrup with the slip-law state evolution is the scalar DAE
    dpsi/dt = -(V/L)(psi - psi_ss(V)),  Theta - eta V = S f(V, psi).
    Solved independently (scipy's DOP853, the root by Brent's method) it is the
    limit of the oracle's steps: psi and V converge at first order in dt (each
    step's tail after the last time point advances the state with the frozen
    last rate) through a strong weakening (psi 0.6 -> 0.09, V x 20)."""
    from scipy.integrate import solve_ivp
    from scipy.optimize import brentq
    rho, lam, mu = 3000.0, 3.0e10, 3.0e10
    eta = np.sqrt(rho * mu) / 2.0
    Th, S, T, N = 30e6, 40e6, 0.2, 3
    p1 = _par(1, sn0=-S, t0x=Th)

    def V_of(psi):
        g = lambda lv: Th - eta * np.exp(lv) - S * ru.friction(np.array([np.exp(lv)]), np.array([psi]), p1)[0]
        return np.exp(brentq(g, -700.0, np.log(Th / eta), xtol=1e-14, rtol=1e-15))

    def rhs(t, y):
        V = np.array([V_of(y[0])])
        return -(V / p1["L"]) * (y - ru.psi_ss(V, p1))

    errs = []
    for steps in (40, 80, 160):
        dt = T / steps
        p = dict(p1, V=np.array([V_of(0.6)]))
        n = np.array([[0.0, 0.0, 1.0]])
        q = np.zeros((N + 1, 1, 9))
        mat = tuple(np.full(1, v) for v in (rho, lam, mu))
        hist = []
        for _ in range(steps):
            _, _, psi, V, _, _, _ = ru.solve_step(n, q, q, mat, mat, p, dt, N)
            p = dict(p, psi=psi, V=V)
            hist.append((psi[0], V[0]))
        hist = np.array(hist)
        t = dt * np.arange(1, steps + 1)
        ref = solve_ivp(rhs, (0.0, T), [0.6], method="DOP853", rtol=1e-12, atol=1e-14, t_eval=t).y[0]
        Vref = np.array([V_of(x) for x in ref])
        errs.append((np.max(np.abs(hist[:, 0] - ref)), np.max(np.abs(hist[:, 1] / Vref - 1))))
    assert ref[-1] < 0.1 and Vref[-1] > 15 * V_of(0.6)
    errs = np.array(errs)
    assert errs[-1, 0] < 2e-4 and errs[-1, 1] < 4e-3, errs
    assert np.all(errs[:-1] / errs[1:] > 1.8), errs
