"""Pins for the oracle's Jacobians, rotation and Riemann solver (Secs. 3, 4.2, 4.3)."""

import numpy as np
import pytest

from oracle import physics as ph

rng = np.random.default_rng(1)


def _unit(n):
    return n / np.linalg.norm(n)


def _Ahat(n, rho, lam, mu):
    A = ph.jacobians(rho, lam, mu)
    return n[0] * A[0] + n[1] * A[1] + n[2] * A[2]


@pytest.mark.parametrize("mat", [(2700.0, 3.24e10, 3.24e10), (1.0, 2.0, 1.0), (1000.0, 2.25e9, 0.0)])
def test_eigenvalues_are_wave_speeds(mat):
    rho, lam, mu = mat
    cp = np.sqrt((lam + 2 * mu) / rho)
    cs = np.sqrt(mu / rho)
    for _ in range(5):
        n = _unit(rng.standard_normal(3))
        ev = np.sort(np.linalg.eigvals(_Ahat(n, rho, lam, mu)).real)
        want = np.sort([-cp, -cs, -cs, 0, 0, 0, cs, cs, cp])
        # the acoustic zero eigenvalue is defective: eig resolves it to ~sqrt(eps) cp
        assert np.allclose(ev, want, atol=1e-7 * cp)


def test_acoustic_special_case():
    # mu = 0, lambda = K, sigma = -p I turns Eq. (elasticity-pde) into linear acoustics
    rho, K = 1000.0, 2.25e9
    A = ph.jacobians(rho, K, 0.0)
    # dp/dt + K div v = 0 with p = -s_xx: row s_xx of A_x has -K on v_x
    for d in range(3):
        for i in range(3):
            assert A[d, i, 6 + d] == -K
        # rho dv/dt + grad p = 0  ->  dv_d/dt - (1/rho) d s_dd/dx_d
        assert A[d, 6 + d, d] == -1 / rho
    # no shear coupling into stresses
    assert np.all(A[:, 3:6, :] == 0)


def test_rotation_identity():
    # n.(A,B,C) = T(n) A T^-1(n)  (Sec. 4.2)
    rho, lam, mu = 2.0, 3.0, 1.5
    A = ph.jacobians(rho, lam, mu)
    for _ in range(5):
        n = _unit(rng.standard_normal(3))
        R = ph.frame(n)
        assert np.allclose(R.T @ R, np.eye(3)) and np.allclose(R[:, 0], n)
        T = np.stack([ph.rotate_out(np.eye(9)[i], R) for i in range(9)], axis=1)
        Ti = np.stack([ph.rotate_in(np.eye(9)[i], R) for i in range(9)], axis=1)
        assert np.allclose(T @ Ti, np.eye(9))
        assert np.allclose(T @ A[0] @ Ti, _Ahat(n, rho, lam, mu), atol=1e-12)


def _flux(qm, qp, n, matm, matp, R=None):
    R = ph.frame(n) if R is None else R
    wm, wp = ph.rotate_in(qm, R), ph.rotate_in(qp, R)
    Zpm, Zsm = ph.impedances(*matm)
    Zpp, Zsp = ph.impedances(*matp)
    wb = ph.middle_state(wm, wp, Zpm, Zpp, Zsm, Zsp)
    return ph.rotate_out(ph.flux_rotated(wb, *matm), R), wb, wm, wp


def test_godunov_equals_upwind_flux_for_equal_materials():
    # textbook: with equal materials the Godunov flux is A+ q- + A- q+ (eigen-split)
    mat = (2.0, 3.0, 1.5)
    for _ in range(5):
        n = _unit(rng.standard_normal(3))
        qm, qp = rng.standard_normal(9), rng.standard_normal(9)
        F, *_ = _flux(qm, qp, n, mat, mat)
        Ah = _Ahat(n, *mat)
        lam_, V = np.linalg.eig(Ah)
        Vi = np.linalg.inv(V)
        Ap = (V @ np.diag(np.maximum(lam_.real, 0)) @ Vi).real
        Am = (V @ np.diag(np.minimum(lam_.real, 0)) @ Vi).real
        assert np.allclose(F, Ap @ qm + Am @ qp, atol=1e-10)


def test_tangent_choice_does_not_matter():
    matm, matp = (2700.0, 3.24e10, 3.24e10), (1000.0, 2.25e9, 0.0)
    n = _unit(np.array([0.3, -0.2, 0.9]))
    R = ph.frame(n)
    a = 0.7
    s2 = np.cos(a) * R[:, 1] + np.sin(a) * R[:, 2]
    R2 = np.stack([n, s2, np.cross(n, s2)], axis=1)
    qm, qp = rng.standard_normal(9), rng.standard_normal(9)
    F1, *_ = _flux(qm, qp, n, matm, matp, R)
    F2, *_ = _flux(qm, qp, n, matm, matp, R2)
    assert np.allclose(F1, F2, rtol=1e-12, atol=1e-6)


def test_elastic_acoustic_state_consistency():
    # Sec. 4.2: with w- = w+ on 1 and 7 and w4 = w6 = 0, w^b is the physical state
    Zpm, Zsm, Zpp = 2.0e7, 1.1e7, 1.5e6
    w = rng.standard_normal(9)
    w[[3, 5]] = 0.0
    wp = rng.standard_normal(9)
    wp[[0, 6]] = w[[0, 6]]
    wb = ph.middle_state(w, wp, Zpm, Zpp, Zsm, 0.0)
    assert np.allclose(wb[[0, 3, 5, 6, 7, 8]], w[[0, 3, 5, 6, 7, 8]])


def test_solid_solid_shear_tends_to_acoustic_rule():
    # stresses ~ 1e6 Pa, velocities ~ 1 m/s, so that sigma / Z_s is of the size of v
    Zpm, Zsm, Zpp = 2.0e7, 1.1e7, 1.5e6
    scale = np.array([1e6] * 6 + [1.0] * 3)
    wm, wp = rng.standard_normal(9) * scale, rng.standard_normal(9) * scale
    wp[[3, 5]] = 0.0
    wb0 = ph.middle_state(wm, wp, Zpm, Zpp, Zsm, 0.0)
    wbe = ph.middle_state(wm, wp, Zpm, Zpp, Zsm, 1e-3)
    assert np.allclose(wb0, wbe, rtol=0, atol=1e-6 * scale)
    # Eq. (boundary-state) entries
    assert wb0[3] == 0 and wb0[5] == 0
    assert wb0[7] == pytest.approx(wm[7] - wm[3] / Zsm, rel=1e-14, abs=1e-15)
    assert wb0[8] == pytest.approx(wm[8] - wm[5] / Zsm, rel=1e-14, abs=1e-15)


def test_middle_state_obeys_rankine_hugoniot():
    # w- - w^b lies in the span of the left-going eigenvectors of A- (relevant comps)
    matm, matp = (2700.0, 3.24e10, 3.24e10), (1000.0, 2.25e9, 0.0)
    wm, wp = rng.standard_normal(9), rng.standard_normal(9)
    Zpm, Zsm = ph.impedances(*matm)
    Zpp, Zsp = ph.impedances(*matp)
    wb = ph.middle_state(wm, wp, Zpm, Zpp, Zsm, Zsp)
    A = ph.jacobians(*matm)[0]
    lam_, V = np.linalg.eig(A)
    left = V[:, lam_.real < -1e-6].real
    rel = [0, 3, 5, 6, 7, 8]
    jump = (wm - wb)[rel]
    coef, *_ = np.linalg.lstsq(left[rel], jump, rcond=None)
    assert np.allclose(left[rel] @ coef, jump, atol=1e-9 * np.abs(jump).max())
    # interface conditions: traction continuity on 1 (acoustic side: -p), zero shear
    assert wb[3] == 0 and wb[5] == 0


@pytest.mark.parametrize("matp", [(2000.0, 1.2e10, 0.8e10), (1000.0, 2.25e9, 0.0)])
def test_middle_states_of_both_sides_meet_the_interface_conditions(matp):
    """The Godunov middle state is the exact Riemann solution at the interface
    (Sec. 4.2), so the states each side computes for the same face (its own
    frame, normal n and -n) satisfy the interface conditions: a welded
    solid-solid contact has one traction sigma.n and one velocity; at a
    solid-fluid contact the normal traction and normal velocity agree and
    neither side carries shear traction.  Each side's state keeps the
    characteristics that leave it through the face (sigma - Z v for the P
    pair and, in a solid, the two S pairs)."""
    matm = (2700.0, 3.24e10, 3.24e10)
    Zpm, Zsm = ph.impedances(*matm)
    Zpp, Zsp = ph.impedances(*matp)
    fluid = matp[2] == 0.0
    for _ in range(5):
        n = _unit(rng.standard_normal(3))
        qm = rng.standard_normal(9) * np.array([1e6] * 6 + [1.0] * 3)
        qp = rng.standard_normal(9) * np.array([1e6] * 6 + [1.0] * 3)
        if fluid:
            qp[:3] = qp[0]
            qp[3:6] = 0.0
        R, Rn = ph.frame(n), ph.frame(-n)
        wm, wp = ph.rotate_in(qm, R), ph.rotate_in(qp, Rn)
        wbm = ph.middle_state(wm, ph.rotate_in(qp, R), Zpm, Zpp, Zsm, Zsp)
        wbp = ph.middle_state(wp, ph.rotate_in(qm, Rn), Zpp, Zpm, Zsp, Zsm)
        bm, bp = ph.rotate_out(wbm, R), ph.rotate_out(wbp, Rn)
        # each side keeps its outgoing characteristics sigma - Z v (P; S pairs in a solid)
        for w, wb, Zp_, Zs_ in ((wm, wbm, Zpm, Zsm), (wp, wbp, Zpp, Zsp)):
            pairs = [(0, 6, Zp_)] + ([(3, 7, Zs_), (5, 8, Zs_)] if Zs_ > 0 else [])
            for i, j, Z in pairs:
                assert abs((wb[i] - Z * wb[j]) - (w[i] - Z * w[j])) <= 1e-12 * (abs(w[i]) + Z * abs(w[j]))

        def traction(q):
            S = np.array([[q[0], q[3], q[5]], [q[3], q[1], q[4]], [q[5], q[4], q[2]]])
            return S @ n

        tm, tp = traction(bm), traction(bp)
        ts = 1e-12 * 1e6
        vs = 1e-12
        if fluid:
            assert abs(tm @ n - tp @ n) <= ts and abs(bm[6:] @ n - bp[6:] @ n) <= vs
            assert np.allclose(tm - (tm @ n) * n, 0.0, atol=ts) and np.allclose(tp - (tp @ n) * n, 0.0, atol=ts)
        else:
            assert np.allclose(tm, tp, rtol=0, atol=ts) and np.allclose(bm[6:], bp[6:], rtol=0, atol=vs)


def test_gravity_ghost_reproduces_boundary_state():
    # Eq. (free-surface-boundary-state): v_n^b = v_n^- - (rho g eta - p^-)/Z, p^b = rho g eta
    rho, K, g, eta = 1000.0, 2.25e9, 9.81, 0.37
    Z, _ = ph.impedances(rho, K, 0.0)
    wm = rng.standard_normal(9)
    wp = ph.ghost(wm, 2, eta=eta, rho=rho, g=g)
    wb = ph.middle_state(wm, wp, Z, Z, 0.0, 0.0)
    pm = -wm[0]
    assert np.isclose(-wb[0], rho * g * eta)
    assert np.isclose(wb[6], wm[6] - (rho * g * eta - pm) / Z)


def test_free_surface_is_gravity_with_zero_eta():
    rho, lam, mu = 2.0, 3.0, 1.5
    Zp, Zs = ph.impedances(rho, lam, mu)
    wm = rng.standard_normal(9)
    a = ph.middle_state(wm, ph.ghost(wm, 1), Zp, Zp, Zs, Zs)
    b = ph.middle_state(wm, ph.ghost(wm, 2, eta=0.0, rho=rho, g=9.81), Zp, Zp, Zs, Zs)
    assert np.allclose(a, b)
    assert abs(a[0]) < 1e-15 and abs(a[3]) < 1e-15 and abs(a[5]) < 1e-15


def _upwind_plus(A):
    """A+ = the part of the rotated Jacobian with positive speeds (waves that
    leave through the face): V diag(max(lambda, 0)) V^-1 where A is
    diagonalisable; for a fluid (whose zero eigenvalue is defective) the sum
    over the simple positive eigenvalues of lambda r l^T / (l^T r)."""
    lam, V = np.linalg.eig(A)
    if np.linalg.cond(V) < 1e8:
        return (V @ np.diag(np.maximum(lam.real, 0.0)) @ np.linalg.inv(V)).real
    lamL, W = np.linalg.eig(A.T)
    out = np.zeros_like(A)
    for i in np.nonzero(lam.real > 1e-6 * np.abs(lam).max())[0]:
        r = V[:, i].real
        l = W[:, np.argmin(np.abs(lamL - lam[i]))].real
        out += lam[i].real * np.outer(r, l) / (l @ r)
    return out


@pytest.mark.parametrize("mat", [(2700.0, 3.24e10, 3.24e10), (1.0, 2.0, 1.0), (1000.0, 2.25e9, 0.0)])
def test_absorbing_flux_is_the_upwind_flux_of_the_interior_state(mat):
    """Absorbing boundary (ghost q+ = 0 with the interior material): the flux
    A w^b equals A+ w^-, the classical upwind flux with nothing entering from
    outside; a transparent ghost (q+ = q-) gives A w^- instead."""
    rho, lam, mu = mat
    Zp, Zs = ph.impedances(rho, lam, mu)
    A = ph.jacobians(rho, lam, mu)[0]
    Ap = _upwind_plus(A)
    for _ in range(4):
        wm = rng.standard_normal(9) * np.array([1e6] * 6 + [1.0] * 3)
        wb = ph.middle_state(wm, ph.ghost(wm, 3), Zp, Zp, Zs, Zs)
        got = ph.flux_rotated(wb, rho, lam, mu)
        assert np.allclose(got, Ap @ wm, rtol=0, atol=1e-10 * np.abs(A @ wm).max())
        assert not np.allclose(got, A @ wm, rtol=0, atol=1e-3 * np.abs(A @ wm).max())


@pytest.mark.parametrize("mat", [(1.0, 2.0, 1.0), (1000.0, 2.25e9, 0.0)])
@pytest.mark.parametrize("tag", [1, 6])
def test_wall_middle_states_keep_the_outgoing_waves_and_meet_the_wall_conditions(mat, tag):
    """Free surface (tag 1): zero traction, w1 = w4 = w6 = 0.  Rigid wall with
    free slip (tag 6): zero normal velocity and zero shear traction, w7 = w4 =
    w6 = 0.  In both, the characteristics leaving the element through the face
    (sigma - Z v on (w1, w7) with Z_p, on (w4, w8) and (w6, w9) with Z_s in a
    solid) equal the interior's: the wall only sets the incoming ones."""
    rho, lam, mu = mat
    Zp, Zs = ph.impedances(rho, lam, mu)
    for _ in range(4):
        wm = rng.standard_normal(9) * np.array([1e3] * 6 + [1.0] * 3)
        wb = ph.middle_state(wm, ph.ghost(wm, tag), Zp, Zp, Zs, Zs)
        sc = 1e-13 * np.abs(wm).max() * max(Zp, 1.0)
        assert abs((wb[0] - Zp * wb[6]) - (wm[0] - Zp * wm[6])) <= sc
        if mu > 0:
            for ts, tv in ((3, 7), (5, 8)):
                assert abs((wb[ts] - Zs * wb[tv]) - (wm[ts] - Zs * wm[tv])) <= sc
        assert wb[3] == pytest.approx(0.0, abs=sc) and wb[5] == pytest.approx(0.0, abs=sc)
        if tag == 1:
            assert wb[0] == pytest.approx(0.0, abs=sc)
        else:
            assert wb[6] == pytest.approx(0.0, abs=sc / max(Zp, 1.0))


def test_gravity_ode_closed_forms():
    dt, kappa = 0.7, 0.3
    # f = 0: eta = eta0 e^{-kappa dt}, H = eta0 (1 - e^{-kappa dt})/kappa
    eta, H = ph.gravity_ode_taylor(np.array([1.3]), np.zeros((1, 4)), kappa, dt)
    assert np.isclose(eta[0], 1.3 * np.exp(-kappa * dt), rtol=1e-15)
    assert np.isclose(H[0], 1.3 * (1 - np.exp(-kappa * dt)) / kappa, rtol=1e-14)
    # kappa = 0: plain polynomial integrals
    f = np.array([[0.5, -1.0, 2.0, 0.25]])
    eta, H = ph.gravity_ode_taylor(np.array([0.1]), f, 0.0, dt)
    e_exp = 0.1 + sum(f[0, m] * dt ** (m + 1) / (m + 1) for m in range(4))
    h_exp = 0.1 * dt + sum(f[0, m] * dt ** (m + 2) / ((m + 1) * (m + 2)) for m in range(4))
    assert np.isclose(eta[0], e_exp, rtol=1e-14) and np.isclose(H[0], h_exp, rtol=1e-14)
    # constant forcing: eta = f/k + (eta0 - f/k) e^{-k t}
    eta, H = ph.gravity_ode_taylor(np.array([0.2]), np.array([[1.5]]), kappa, dt)
    ex = 1.5 / kappa + (0.2 - 1.5 / kappa) * np.exp(-kappa * dt)
    hx = 1.5 / kappa * dt + (0.2 - 1.5 / kappa) * (1 - np.exp(-kappa * dt)) / kappa
    assert np.isclose(eta[0], ex, rtol=1e-14) and np.isclose(H[0], hx, rtol=1e-13)
