"""Pins for the oracle's basis and reference operators (Sec. 4.1)."""

from math import comb

import numpy as np
import pytest

from oracle import basis as ob
from oracle.quadrature import tet_rule, tri_rule


@pytest.mark.parametrize("N", [0, 1, 2, 3, 4, 5])
def test_basis_size(N):
    # B_N = C(N+3, 3) (Sec. 4.1)
    assert ob.n_basis(N) == comb(N + 3, 3) == len(ob.triples(N))


@pytest.mark.parametrize("N", [1, 3, 5])
def test_orthonormal_with_finer_rule(N):
    M = ob.mass_matrix(N, 2 * N + 4)
    assert np.abs(M - np.eye(ob.n_basis(N))).max() < 1e-13


def test_quadrature_exact_on_monomials():
    # int_tet x^a y^b z^c = a! b! c! / (a+b+c+3)!  (closed form)
    from math import factorial
    pts, w = tet_rule(7)
    for a, b, c in [(0, 0, 0), (3, 2, 1), (0, 7, 0), (2, 2, 3)]:
        exact = factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 3)
        got = np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
        assert abs(got - exact) < 1e-15 * max(1.0, 1 / exact) * exact + 1e-17
    pts, w = tri_rule(6)
    for a, b in [(0, 0), (6, 0), (3, 3), (1, 4)]:
        exact = factorial(a) * factorial(b) / factorial(a + b + 2)
        assert abs(np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b) - exact) < 1e-15


def _random_poly(N, rng):
    terms = [(a, b, c) for a in range(N + 1) for b in range(N + 1) for c in range(N + 1)
             if a + b + c <= N]
    coef = rng.standard_normal(len(terms))
    return terms, coef


def _poly_eval(terms, coef, x, d=None):
    out = np.zeros(x.shape[0])
    for (a, b, c), k in zip(terms, coef):
        e = [a, b, c]
        f = k
        if d is not None:
            f = f * e[d]
            if e[d] == 0:
                continue
            e[d] -= 1
        out += f * x[:, 0] ** e[0] * x[:, 1] ** e[1] * x[:, 2] ** e[2]
    return out


@pytest.mark.parametrize("N", [2, 3, 5])
def test_basis_spans_PN_and_stiffness_matches_monomial_derivatives(N):
    rng = np.random.default_rng(0)
    terms, coef = _random_poly(N, rng)
    pts, w = tet_rule(2 * N + 2)
    phi = ob.eval_basis(N, pts)
    P = phi.T @ (w * _poly_eval(terms, coef, pts))  # L2 projection (exact: p in P_N)
    x = rng.uniform(0, 0.3, size=(20, 3))
    assert np.allclose(ob.eval_basis(N, x) @ P, _poly_eval(terms, coef, x), atol=1e-12)
    K = ob.stiffness(N)
    for e in range(3):
        dP = phi.T @ (w * _poly_eval(terms, coef, pts, d=e))
        # projection of dp/dxi_e = K_e^T P (strong-form derivative operator)
        assert np.allclose(K[e].T @ P, dP, atol=1e-11)


def test_gradient_matches_finite_differences():
    N = 4
    x = np.array([[0.1, 0.2, 0.3], [0.6, 0.1, 0.05], [0.05, 0.05, 0.05]])
    g = ob.eval_grad(N, x)
    h = 1e-6
    for e in range(3):
        d = np.zeros(3)
        d[e] = h
        fd = (ob.eval_basis(N, x + d) - ob.eval_basis(N, x - d)) / (2 * h)
        assert np.abs(fd - g[:, :, e]).max() < 1e-6


def test_hierarchical_by_degree():
    # the first B_{N-1} functions span P_{N-1}: derivatives of P_N land there
    N = 4
    K = ob.stiffness(N)
    Bm = ob.n_basis(N - 1)
    for e in range(3):
        assert np.abs(K[e].T[Bm:, :]).max() < 1e-12


def test_face_maps_lie_on_faces():
    chi, _ = tri_rule(4)
    planes = [lambda p: p.sum(1) - 1, lambda p: p[:, 0], lambda p: p[:, 1], lambda p: p[:, 2]]
    for f in range(4):
        p = ob.face_to_ref(f, chi)
        assert np.abs(planes[f](p)).max() < 1e-15
