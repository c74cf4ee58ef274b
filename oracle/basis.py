"""Orthonormal Dubiner basis on the reference tetrahedron (oracle; test
infrastructure).  Sec. 4.1: q = sum_l Q_l phi_l with B_N = C(N+3, 3) modes.

Reading (the paper names the basis but prints no formula): the Dubiner
(Koornwinder) product basis in collapsed coordinates,
    phi_ijk = c_ijk * s^i P_i^(0,0)(2 xi/s - 1)
                    * t^j P_j^(2i+1,0)(2 eta/t - 1)
                    * P_k^(2i+2j+2,0)(2 zeta - 1),
    s = 1 - eta - zeta,  t = 1 - zeta,
with c_ijk > 0 chosen so that the reference mass matrix is the identity.
Order: total degree n = i+j+k ascending, then i ascending, then j ascending.
Jacobi polynomial coefficients come from scipy (a library primitive); each
factor is evaluated in its homogeneous form, defined on the whole closed tet;
all integrals use the collapsed Gauss rules of quadrature.py.
"""

from functools import lru_cache

import numpy as np
from scipy.special import jacobi

from .quadrature import tet_rule


def n_basis(N):
    return (N + 1) * (N + 2) * (N + 3) // 6


def n_face_basis(N):
    return (N + 1) * (N + 2) // 2


def triples(N):
    out = []
    for n in range(N + 1):
        for i in range(n + 1):
            for j in range(n - i + 1):
                out.append((i, j, n - i - j))
    return out


@lru_cache(maxsize=None)
def _jac_coeffs(n, a):
    """Monomial coefficients c_k of P_n^(a,0)(y) = sum_k c_k y^k (scipy)."""
    return tuple(jacobi(n, a, 0.0).coeffs[::-1])


def _G(n, a, x, tau):
    """tau^n P_n^(a,0)(2x/tau - 1) with its partial derivatives in x and tau,
    written in the homogeneous form sum_k c_k (2x - tau)^k tau^(n-k), which is
    the same polynomial and stays defined where tau = 0 (tet vertices/edges)."""
    c = _jac_coeffs(n, a)
    u = 2.0 * x - tau
    val = np.zeros_like(x)
    dx = np.zeros_like(x)
    dtau = np.zeros_like(x)
    for k, ck in enumerate(c):
        uk = u ** k
        tk = tau ** (n - k)
        val += ck * uk * tk
        if k > 0:
            uk1 = u ** (k - 1)
            dx += ck * 2.0 * k * uk1 * tk
            dtau += ck * (-k) * uk1 * tk
        if n - k > 0:
            dtau += ck * (n - k) * uk * tau ** (n - k - 1)
    return val, dx, dtau


def _raw(N, pts):
    xi, eta, zeta = pts[:, 0], pts[:, 1], pts[:, 2]
    s = 1.0 - eta - zeta
    t = 1.0 - zeta
    T = triples(N)
    val = np.empty((pts.shape[0], len(T)))
    grad = np.empty((pts.shape[0], len(T), 3))
    for l, (i, j, k) in enumerate(T):
        f1, f1x, f1s = _G(i, 0, xi, s)
        f2, f2y, f2t = _G(j, 2 * i + 1, eta, t)
        f3, f3z, _ = _G(k, 2 * i + 2 * j + 2, zeta, np.ones_like(zeta))
        val[:, l] = f1 * f2 * f3
        # d/dxi: only f1 through x
        grad[:, l, 0] = f1x * f2 * f3
        # d/deta: f1 through s (ds/deta = -1), f2 through x
        grad[:, l, 1] = -f1s * f2 * f3 + f1 * f2y * f3
        # d/dzeta: f1 through s (-1), f2 through t (-1), f3
        grad[:, l, 2] = -f1s * f2 * f3 - f1 * f2t * f3 + f1 * f2 * f3z
    return val, grad


@lru_cache(maxsize=None)
def _norms(N):
    pts, w = tet_rule(2 * N)
    v, _ = _raw(N, pts)
    return 1.0 / np.sqrt(np.einsum("q,ql,ql->l", w, v, v))


def eval_basis(N, pts):
    """phi_l at reference points pts (npts, 3) -> (npts, B)."""
    v, _ = _raw(N, np.atleast_2d(np.asarray(pts, dtype=np.float64)))
    return v * _norms(N)[None, :]


def eval_grad(N, pts):
    """d phi_l / d xi_e at pts -> (npts, B, 3)."""
    _, g = _raw(N, np.atleast_2d(np.asarray(pts, dtype=np.float64)))
    return g * _norms(N)[None, :, None]


@lru_cache(maxsize=None)
def mass_matrix(N, degree=None):
    pts, w = tet_rule(2 * N if degree is None else degree)
    v = eval_basis(N, pts)
    return np.einsum("q,qk,ql->kl", w, v, v)


@lru_cache(maxsize=None)
def stiffness(N):
    """K[e][k, l] = int_ref d phi_k/d xi_e * phi_l  -> (3, B, B)."""
    pts, w = tet_rule(2 * N)
    v = eval_basis(N, pts)
    g = eval_grad(N, pts)
    return np.einsum("q,qke,ql->ekl", w, g, v)


# Reference-tet vertices and faces.  Face f is opposite vertex f; its three
# vertices are listed in increasing local index, and the face is parametrised
# by x(chi) = Va + chi1 (Vb - Va) + chi2 (Vc - Va).
REF_VERTS = np.array([[0.0, 0, 0], [1.0, 0, 0], [0.0, 1, 0], [0.0, 0, 1]])
FACE_VERTS = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))


def face_to_ref(f, chi):
    """Map reference-triangle points chi (nq, 2) onto face f of the reference tet."""
    a, b, c = (REF_VERTS[v] for v in FACE_VERTS[f])
    chi = np.atleast_2d(chi)
    return a[None, :] + chi[:, :1] * (b - a)[None, :] + chi[:, 1:2] * (c - a)[None, :]
