"""Pins of the oracle phi-functions and augmented exponentials.

Independent references: the closed form phi_k(z) = (e^z - sum_{j<k} z^j/j!)/z^k
and the power series sum_j z^j/(j+k)! (Eq. (eq3.6) expanded), evaluated per
eigenvalue; phi_k(0) = 1/k!; and the recurrence of Eq. (eq3.7).
"""
import math

import numpy as np
import pytest

from oracle.phi import (augmented_norm1, phi_combination_dense, phi_krylov,
                        phi_matrices)


def phi_series(k, z, terms=80):
    return sum(z ** j / math.factorial(j + k) for j in range(terms))


def phi_closed(k, z):
    if abs(z) <= 4.0:
        return phi_series(k, z)
    return (np.exp(z) - sum(z ** j / math.factorial(j) for j in range(k))) / z ** k


def test_phi_at_zero_is_inverse_factorial():
    for p in range(0, 6):
        ph = phi_matrices(np.zeros((1, 1)), 6)
        for k in range(7):
            assert abs(ph[k][0, 0] - 1.0 / math.factorial(k)) < 1e-15


@pytest.mark.parametrize("lam", [-30.0, -3.0, -0.2, 0.0, 0.3, 2.0])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_krylov_phi_scalar(lam, p):
    for tau in (1.0, 0.37):
        a, b = phi_krylov(np.array([[lam]]), tau, p)
        z = tau * lam
        assert a[0] == pytest.approx(phi_closed(p, z), rel=1e-13, abs=1e-15)
        assert b[0] == pytest.approx(phi_closed(p + 1, z), rel=1e-13, abs=1e-15)


@pytest.mark.parametrize("p", [1, 3, 4])
def test_krylov_phi_rotation_block(p):
    # H acts like multiplication by i*w on x + i y: phi(tau H) e_1 = (Re, Im) phi(i tau w)
    w = 7.5
    H = np.array([[0.0, -w], [w, 0.0]])
    for tau in (1.0, 0.2):
        a, b = phi_krylov(H, tau, p)
        for vec, k in ((a, p), (b, p + 1)):
            ref = phi_closed(k, 1j * tau * w)
            assert vec[0] == pytest.approx(ref.real, abs=1e-14)
            assert vec[1] == pytest.approx(ref.imag, abs=1e-14)


def test_krylov_phi_tridiagonal_by_eigendecomposition():
    rng = np.random.default_rng(3)
    m, p = 12, 3
    H = np.diag(rng.standard_normal(m)) + np.diag(rng.standard_normal(m - 1), 1) \
        + np.diag(rng.standard_normal(m - 1), -1)
    H *= 2.0
    lam, X = np.linalg.eig(H)
    e1 = np.zeros(m)
    e1[0] = 1.0
    c = np.linalg.solve(X, e1)
    for tau in (1.0, 0.4):
        a, b = phi_krylov(H, tau, p)
        ref_a = (X @ (np.array([phi_closed(p, tau * l) for l in lam]) * c)).real
        ref_b = (X @ (np.array([phi_closed(p + 1, tau * l) for l in lam]) * c)).real
        assert np.allclose(a, ref_a, rtol=1e-11, atol=1e-13)
        assert np.allclose(b, ref_b, rtol=1e-11, atol=1e-13)
        # recurrence, Eq. (eq3.7): phi_p(z) = z phi_{p+1}(z) + 1/p!
        assert np.allclose(a, tau * H @ b + e1 / math.factorial(p), atol=1e-13)


def test_augmented_norm():
    H = np.array([[1.0, -2.0], [3.0, 0.5]])
    assert augmented_norm1(H, 2.0, 3) == pytest.approx(8.0)
    assert augmented_norm1(H, 0.01, 3) == pytest.approx(1.0)


def test_dense_combination_diagonal():
    rng = np.random.default_rng(1)
    lam = np.array([-5.0, -0.7, 0.0, 0.4, 1.3])
    A = np.diag(lam)
    v = [rng.standard_normal(5) for _ in range(4)]
    v[2] = None
    for rho in (1.0, 0.5, 0.9):
        y = phi_combination_dense(A, v, rho)
        ref = np.zeros(5)
        for l, vl in enumerate(v):
            if vl is not None:
                ref += rho ** l * np.array([phi_closed(l, rho * x) for x in lam]) * vl
        assert np.allclose(y, ref, rtol=1e-13, atol=1e-14)


def test_phi_matrices_against_eigendecomposition():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((6, 6))
    lam, X = np.linalg.eig(A)
    Xi = np.linalg.inv(X)
    ph = phi_matrices(A, 5)
    for k in range(6):
        ref = (X @ np.diag([phi_closed(k, l) for l in lam]) @ Xi).real
        assert np.allclose(ph[k], ref, rtol=1e-10, atol=1e-12)
