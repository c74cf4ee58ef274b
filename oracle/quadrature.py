"""Collapsed (conical-product) Gauss-Legendre rules on the reference triangle
and tetrahedron (oracle; test infrastructure).

Reference tetrahedron: vertices (0,0,0), (1,0,0), (0,1,0), (0,0,1), volume 1/6.
Reference triangle: vertices (0,0), (1,0), (0,1), area 1/2.

The Duffy collapse maps the unit cube onto the simplex,
    tet: zeta = w, eta = v (1-w), xi = u (1-v)(1-w), dV = (1-v)(1-w)^2 du dv dw
    tri: chi2 = v, chi1 = u (1-v),                  dA = (1-v) du dv
and a tensor Gauss-Legendre rule with n points per direction integrates a
polynomial of total degree d exactly when 2n-1 >= d+2 (tet) or d+1 (tri).
The 1-D rule is numpy's Gauss-Legendre (a library primitive).
"""

import numpy as np
from numpy.polynomial.legendre import leggauss


def gauss01(n):
    x, w = leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def tet_rule(degree):
    """Points (nq, 3) and weights (nq,) exact for total degree `degree`."""
    n = max(1, int(np.ceil((degree + 3) / 2.0)))
    x, w = gauss01(n)
    u, v, s = np.meshgrid(x, x, x, indexing="ij")
    wu, wv, ws = np.meshgrid(w, w, w, indexing="ij")
    zeta = s
    eta = v * (1 - s)
    xi = u * (1 - v) * (1 - s)
    wt = wu * wv * ws * (1 - v) * (1 - s) ** 2
    pts = np.stack([xi.ravel(), eta.ravel(), zeta.ravel()], axis=1)
    return pts, wt.ravel()


def tri_rule(degree):
    """Points (nq, 2) and weights (nq,) on the reference triangle, exact for
    total degree `degree` (weights sum to 1/2)."""
    n = max(1, int(np.ceil((degree + 2) / 2.0)))
    x, w = gauss01(n)
    u, v = np.meshgrid(x, x, indexing="ij")
    wu, wv = np.meshgrid(w, w, indexing="ij")
    chi2 = v
    chi1 = u * (1 - v)
    wt = wu * wv * (1 - v)
    return np.stack([chi1.ravel(), chi2.ravel()], axis=1), wt.ravel()
