"""phi-functions and the small matrix exponentials of Algorithm 1 (oracle).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``): never used by the product path.

* phi_k (Eqs. (eq3.6)-(eq3.7)): phi_0(z) = e^z, phi_{k+1}(z) = (phi_k(z) - 1/k!)/z.
* Algorithm 1, remark after step 6: phi_p(tau H_m) e_1 and phi_{p+1}(tau H_m) e_1
  come out of one exponential of an augmented matrix.  Reading of the
  augmentation (size m+p+1, as the (m+p+1)^3 term of Eq. (eq:cost) implies):

      Hhat[0:m, 0:m] = tau H_m,   Hhat[0, m] = 1,
      Hhat[m+k, m+k+1] = 1  for k = 0 .. p-1,

  so that exp(Hhat)[0:m, m+j-1] = phi_j(tau H_m) e_1 for j = 1 .. p+1.
* A dense reference for y(rho) = sum_l rho^l phi_l(rho A) v_l, the solution at
  t = rho of the ODE of Eq. (eq3.15): with W = [v_p, ..., v_1] and S_p the p x p
  upshift, y(rho) = [I 0] exp(rho [[A, W], [0, S_p]]) [v_0; e_p].

The exponential itself is the library primitive ``scipy.linalg.expm``.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla


def augmented_krylov_matrix(H: np.ndarray, tau: float, p: int) -> np.ndarray:
    m = H.shape[0]
    M = m + p + 1
    Hh = np.zeros((M, M))
    Hh[0:m, 0:m] = tau * H
    Hh[0, m] = 1.0
    for k in range(p):
        Hh[m + k, m + k + 1] = 1.0
    return Hh


def phi_krylov(H: np.ndarray, tau: float, p: int) -> tuple[np.ndarray, np.ndarray]:
    """(phi_p(tau H) e_1, phi_{p+1}(tau H) e_1) from one exponential of Hhat."""
    m = H.shape[0]
    E = sla.expm(augmented_krylov_matrix(H, tau, p))
    return E[0:m, m + p - 1].copy(), E[0:m, m + p].copy()


def augmented_norm1(H: np.ndarray, tau: float, p: int) -> float:
    """||tau Hhat||_1 of the augmented matrix above (enters M of Eq. (eq:cost))."""
    return float(np.max(np.sum(np.abs(augmented_krylov_matrix(H, tau, p)), axis=0)))


def phi_matrices(A: np.ndarray, kmax: int) -> list[np.ndarray]:
    """[phi_0(A), ..., phi_kmax(A)] for a small dense A from one block exponential.

    exp([[A, I, 0, ...], [0, 0, I, ...], ..., [0, ..., 0]]) has phi_k(A) in its
    first block row (the integral definition Eq. (eq3.6) with Delta t = 1).
    """
    n = A.shape[0]
    K = kmax + 1
    B = np.zeros((K * n, K * n))
    B[0:n, 0:n] = A
    for k in range(1, K):
        B[(k - 1) * n:k * n, k * n:(k + 1) * n] = np.eye(n)
    E = sla.expm(B)
    return [E[0:n, k * n:(k + 1) * n].copy() for k in range(K)]


def phi_combination_dense(A: np.ndarray, v: list, rho: float) -> np.ndarray:
    """y(rho) = sum_{l=0}^p rho^l phi_l(rho A) v_l for dense A (v_l may be None)."""
    n = A.shape[0]
    p = len(v) - 1
    vs = [np.zeros(n) if x is None else np.asarray(x, dtype=np.float64) for x in v]
    if p == 0:
        return sla.expm(rho * A) @ vs[0]
    B = np.zeros((n + p, n + p))
    B[0:n, 0:n] = A
    for k in range(p):
        B[0:n, n + k] = vs[p - k]          # W = [v_p, ..., v_1]
    for k in range(p - 1):
        B[n + k, n + k + 1] = 1.0          # S_p
    rhs = np.concatenate([vs[0], np.zeros(p)])
    rhs[n + p - 1] = 1.0                   # e_p
    return (sla.expm(rho * B) @ rhs)[0:n]


def phi_scalar(k: int, z: complex) -> complex:
    """phi_k(z) for a scalar by the recurrence of Eq. (eq3.7) (|z| not small)."""
    val = np.exp(z)
    for j in range(k):
        val = (val - 1.0 / math.factorial(j)) / z
    return val
