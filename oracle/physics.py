"""Physics of the coupled elastic-acoustic system (oracle; test infrastructure).

q = (s_xx, s_yy, s_zz, s_xy, s_yz, s_xz, v_x, v_y, v_z)        (Sec. 3)
Jacobians A, B, C of dq/dt + A dq/dx + B dq/dy + C dq/dz = 0 written out from
Eq. (elasticity-pde); the acoustic case is lambda = K, mu = 0 (Sec. 4.1).

Riemann problem (Sec. 4.2): rotate into the face frame R = [n s t] with the
outward normal n, w = T^-1 q (stress R^T S R, velocity R^T v), solve for the
middle state w^b and return the flux T A^- w^b, Eq. (numerical-flux).

Readings recorded here (the paper prints only the elastic-acoustic case):
  * solid-solid shear: the same welded-contact form as the P part, with Z_s
    (alpha_2 on (w4, w8), alpha_3 on (w6, w9)); it tends to Eq.
    (boundary-state) as Z_s^+ -> 0;
  * if either side is a fluid: w4^b = w6^b = 0 (Sec. 4.2 closure), the minus
    side's tangential velocities penalised by its own shear traction;
  * ghost states (Sec. 4.3, "inverse Riemann problem"): absorbing q+ = 0 with
    the minus material; free surface: tractions (w1, w4, w6) mirrored;
    rigid wall (free slip): w7, w4, w6 mirrored; gravitational surface:
    u_n+ = v_n-, p+ = 2 rho g eta - p-, Eq. (free-surface-boundary-state).
"""

import numpy as np


def jacobians(rho, lam, mu):
    """A, B, C as arrays (..., 9, 9) from Eq. (elasticity-pde)."""
    rho, lam, mu = (np.asarray(a, dtype=np.float64) for a in (rho, lam, mu))
    shp = np.broadcast(rho, lam, mu).shape
    A = np.zeros(shp + (3, 9, 9))
    l2m = lam + 2 * mu
    ir = 1.0 / rho
    # stress rows: d s_ij/dt - lam delta_ij div v - mu (dv_i/dx_j + dv_j/dx_i) = 0
    # velocity rows: rho dv_i/dt - d s_ij/dx_j = 0
    # index of s_ij in q:
    S = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3, (1, 2): 4, (2, 1): 4,
         (0, 2): 5, (2, 0): 5}
    for d in range(3):  # derivative direction x_d
        M = A[..., d, :, :]
        # normal stresses
        for i in range(3):
            M[..., S[(i, i)], 6 + d] -= lam
        M[..., S[(d, d)], 6 + d] -= 2 * mu
        # shear stresses s_ij (i<j): -mu (dv_i/dx_j + dv_j/dx_i)
        for (i, j) in ((0, 1), (1, 2), (0, 2)):
            if d == j:
                M[..., S[(i, j)], 6 + i] -= mu
            if d == i:
                M[..., S[(i, j)], 6 + j] -= mu
        # velocities: dv_i/dt - (1/rho) d s_ij/dx_j
        for i in range(3):
            M[..., 6 + i, S[(i, d)]] -= ir
    del l2m
    return A


def star_matrices(Jinv, rho, lam, mu):
    """A*_e = sum_d (d xi_e / d x_d) A_d  -> (E, 3, 9, 9)."""
    A = jacobians(rho, lam, mu)  # (E,3,9,9)
    return np.einsum("xed,xdij->xeij", Jinv, A)


def impedances(rho, lam, mu):
    rho, lam, mu = (np.asarray(a, dtype=np.float64) for a in (rho, lam, mu))
    return np.sqrt(rho * (lam + 2 * mu)), np.sqrt(rho * mu)


def frame(n):
    """Orthonormal frames R (..., 3, 3) with columns (n, s, t) for unit normals n."""
    n = np.asarray(n, dtype=np.float64)
    a = np.zeros_like(n)
    # pick the coordinate axis least aligned with n
    k = np.argmin(np.abs(n), axis=-1)
    np.put_along_axis(a, k[..., None], 1.0, axis=-1)
    s = a - np.sum(a * n, axis=-1, keepdims=True) * n
    s /= np.linalg.norm(s, axis=-1, keepdims=True)
    t = np.cross(n, s)
    return np.stack([n, s, t], axis=-1)


_VOIGT = ((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2))


def _stress_tensor(q):
    S = np.empty(q.shape[:-1] + (3, 3))
    for c, (i, j) in enumerate(_VOIGT):
        S[..., i, j] = q[..., c]
        S[..., j, i] = q[..., c]
    return S


def _voigt(S):
    return np.stack([S[..., i, j] for (i, j) in _VOIGT], axis=-1)


def rotate_in(q, R):
    """w = T^-1 q: stress R^T S R, velocity R^T v (R broadcast against q)."""
    S = _stress_tensor(q[..., :6])
    Sr = np.einsum("...ji,...jk,...kl->...il", R, S, R, optimize=True)
    v = np.einsum("...ji,...j->...i", R, q[..., 6:])
    return np.concatenate([_voigt(Sr), v], axis=-1)


def rotate_out(w, R):
    """q = T w: stress R S' R^T, velocity R v'."""
    S = _stress_tensor(w[..., :6])
    Sq = np.einsum("...ij,...jk,...lk->...il", R, S, R, optimize=True)
    v = np.einsum("...ij,...j->...i", R, w[..., 6:])
    return np.concatenate([_voigt(Sq), v], axis=-1)


def middle_state(wm, wp, Zpm, Zpp, Zsm, Zsp):
    """Godunov middle state w^b on the minus side, Eq. (boundary-state) and the
    solid-solid reading.  Paper indices w1..w9 are 0-based here (w1 -> 0)."""
    Zpm, Zpp, Zsm, Zsp = (np.asarray(z, dtype=np.float64)[..., None] for z in (Zpm, Zpp, Zsm, Zsp))
    wb = wm.copy()
    a1 = Zpm * Zpp / (Zpm + Zpp) * ((wm[..., 0:1] - wp[..., 0:1]) / Zpp + wm[..., 6:7] - wp[..., 6:7])
    wb[..., 0:1] = wm[..., 0:1] - a1
    wb[..., 6:7] = wm[..., 6:7] - a1 / Zpm
    solid = (Zsm > 0) & (Zsp > 0)
    with np.errstate(divide="ignore", invalid="ignore"):
        for (ts, tv) in ((3, 7), (5, 8)):
            a = Zsm * Zsp / (Zsm + Zsp) * ((wm[..., ts:ts + 1] - wp[..., ts:ts + 1]) / Zsp
                                           + wm[..., tv:tv + 1] - wp[..., tv:tv + 1])
            ws_solid = wm[..., ts:ts + 1] - a
            wv_solid = wm[..., tv:tv + 1] - a / Zsm
            # fluid on either side: zero shear traction, penalised tangential velocity
            wv_fluid = np.where(Zsm > 0, wm[..., tv:tv + 1] - wm[..., ts:ts + 1] / np.where(Zsm > 0, Zsm, 1.0),
                                wm[..., tv:tv + 1])
            wb[..., ts:ts + 1] = np.where(solid, ws_solid, 0.0)
            wb[..., tv:tv + 1] = np.where(solid, wv_solid, wv_fluid)
    return wb


def flux_rotated(wb, rho, lam, mu):
    """A^- w^b with the x-Jacobian of the minus material (rotated frame)."""
    A = jacobians(rho, lam, mu)[..., 0, :, :]
    return np.einsum("...ij,...j->...i", A, wb)


def ghost(wm, tag, eta=None, rho=None, g=None):
    """Ghost state w+ for the boundary tags (rotated frame)."""
    wp = wm.copy()
    if tag == 3:      # absorbing: q+ = 0
        wp[...] = 0.0
    elif tag == 1:    # free surface: traction mirrored
        wp[..., [0, 3, 5]] *= -1.0
    elif tag == 6:    # rigid wall, free slip
        wp[..., [6, 3, 5]] *= -1.0
    elif tag == 2:    # gravitational surface: u_n+ = v_n-, p+ = 2 rho g eta - p-
        pm = -wm[..., 0]
        wp[..., 0] = -(2.0 * rho * g * eta - pm)
        wp[..., [3, 5]] *= -1.0
    else:
        raise ValueError(tag)
    return wp


def gravity_ode_taylor(eta_n, f, kappa, dt, tol=1e-17, max_terms=200):
    """Exact solution over one step of  eta' = f(tau) - kappa eta,  H' = eta,
    eta(0) = eta_n, H(0) = 0, Eq. (coupled-ode-system) with
    f = v_n^- + p^-/Z and kappa = rho g / Z.

    f: (..., N+1) Taylor coefficients in tau = t - t_n.  Reading: the paper's
    7th-order Runge-Kutta scheme is replaced by the exact power series
    c_0 = eta_n, c_{m+1} = (f_m - kappa c_m)/(m+1), summed until the terms
    drop below tol relative to the running sum.  Returns (eta(dt), H(dt))."""
    eta_n = np.asarray(eta_n, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    c = eta_n.copy()
    eta = c.copy()
    H = c * dt
    pw = np.ones_like(eta_n)  # dt^m
    for m in range(max_terms):
        fm = f[..., m] if m < f.shape[-1] else 0.0
        c = (fm - kappa * c) / (m + 1)
        pw = pw * dt
        term = c * pw
        eta = eta + term
        H = H + term * dt / (m + 2)
        if m >= f.shape[-1] and np.all(np.abs(term) <= tol * (np.abs(eta) + 1e-300)):
            break
    return eta, H
