"""Exponential integrators of Sec. 3.3 driven as in Sec. 4.4 (oracle).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``): never used by the product path.

A model provides F(u) and Jv(u_lin, x) (and, for dense phi, jacobian(u)).
A phi-evaluator ``phi(u_lin, dt, rho, v, slot)`` returns
[sum_l rho_i^l phi_l(rho_i A) v_l for rho_i in rho] with A = dt J(u_lin); the
Krylov one is Algorithm 1 (``KrylovPhi``), the dense one the exact augmented
exponential (``DensePhi``).  With A = dt J_n and v = dt F(u_n) (Sec. 4.4):

EPI2 / exponential Rosenbrock-Euler, Eq. (eq3.5):
    u_{n+1} = u_n + Y(1),  p = 1, v_1 = v.
exprb42, Eq. (eq3.11), two calls:
    U_2 = u_n + Y(3/4) [p=1, v_1 = v];  D_2 = N_n(U_2) - N_n(u_n)
    u_{n+1} = u_n + Y(1) [p=3, v_1 = v, v_3 = (32/9) dt D_2].
pexprb43, Eq. (eq3.12), two calls:
    U_2 = u_n + Y(1/2), U_3 = u_n + Y(1) [one call, rho = (1/2, 1), v_1 = v]
    u_{n+1} = U_3 + Y(1) [p=4, v_3 = dt(16 D_2 - 2 D_3), v_4 = dt(-48 D_2 + 12 D_3)].
exprb53, Eq. (eq3.13), three calls:
    Y_1(1/2), Y_1(9/10) [rho = (1/2, 9/10), p=1, v_1 = v];  U_2 = u_n + Y_1(1/2)
    Y_3(1/2), Y_3(9/10) [rho = (1/2, 9/10), p=3, v_3 = dt D_2]
    U_3 = u_n + Y_1(9/10) + (27/25)/(1/2)^3 Y_3(1/2) + (729/125)/(9/10)^3 Y_3(9/10)
    u_{n+1} = u_n + Y(1) [p=4, v_1 = v, v_3 = dt(18 D_2 - 250/81 D_3),
                                         v_4 = dt(-60 D_2 + 500/27 D_3)].
    Reading: the driver text of Sec. 4.4 prints 725/125 and "h D_n2"; Eq. (eq3.13)
    prints 729/125 and the step is dt, and only 729/125 satisfies the order
    condition 4 of Table 1 (the 729/125 term cancels c_3^3 phi_3(c_3 Z)).
    Y_3(rho) = rho^3 phi_3(rho A) v_3 carries rho^3, hence the division.
epi3, Eq. (eq_epi3), one call per step after one EPI2 starting step:
    u_{n+1} = u_n + Y(1) [p=2, v_1 = v, v_2 = (2/3) dt R_{n-1}],
    R_{n-1} = F(u_{n-1}) - F(u_n) - J_n (u_{n-1} - u_n).

D_ni = N_n(U_ni) - N_n(u_n) is evaluated literally (Eq. (eqDni)), with
N_n(u) = F(u) - J_n u (Eq. (eq3.2)).
"""
from __future__ import annotations

from typing import Optional

import numpy as np

from .phi import phi_combination_dense
from .phipm import PhiOpts, phipm_simul_iom2

SCHEMES = ("epi2", "exprb42", "pexprb43", "exprb53", "epi3")


class KrylovPhi:
    """Algorithm 1 as the phi-evaluator; carries m between steps per call slot."""

    def __init__(self, model, opts: Optional[PhiOpts] = None, m_carry: bool = True):
        self.model = model
        self.opts = opts or PhiOpts()
        self.m_carry = m_carry
        self.slots: dict = {}
        self.stats: list = []

    def __call__(self, u_lin, dt, rho, v, slot):
        model = self.model

        def Amul(x):
            return dt * model.Jv(u_lin, x)

        m_start = self.slots.get(slot) if self.m_carry else None
        W, st = phipm_simul_iom2(Amul, rho, v, self.opts, model.nA, m_start=m_start)
        if st.m_last > 0:
            self.slots[slot] = st.m_last
        self.stats.append((slot, st))
        return W


class DensePhi:
    """Exact phi-combinations through the dense augmented exponential."""

    def __init__(self, model):
        self.model = model

    def __call__(self, u_lin, dt, rho, v, slot):
        J = self.model.jacobian(u_lin)
        J = J.toarray() if hasattr(J, "toarray") else np.asarray(J)
        return [phi_combination_dense(dt * J, list(v), r) for r in rho]


def _D(model, u_n, U):
    """D = N_n(U) - N_n(u_n), Eq. (eqDni)."""
    return (model.F(U) - model.Jv(u_n, U)) - (model.F(u_n) - model.Jv(u_n, u_n))


def step(scheme: str, model, u_n: np.ndarray, dt: float, phi,
         u_prev: Optional[np.ndarray] = None) -> np.ndarray:
    """One step of ``scheme``; epi3 needs ``u_prev`` (None -> EPI2 starting step)."""
    v = dt * model.F(u_n)
    if scheme == "epi2" or (scheme == "epi3" and u_prev is None):
        (y,) = phi(u_n, dt, [1.0], [None, v], "epi2")
        return u_n + y
    if scheme == "exprb42":
        (y1,) = phi(u_n, dt, [0.75], [None, v], "s1")
        D2 = _D(model, u_n, u_n + y1)
        (w,) = phi(u_n, dt, [1.0], [None, v, None, (32.0 / 9.0) * dt * D2], "s2")
        return u_n + w
    if scheme == "pexprb43":
        y_half, y_one = phi(u_n, dt, [0.5, 1.0], [None, v], "s1")
        U2 = u_n + y_half
        U3 = u_n + y_one
        D2 = _D(model, u_n, U2)
        D3 = _D(model, u_n, U3)
        (w,) = phi(u_n, dt, [1.0],
                   [None, None, None, dt * (16.0 * D2 - 2.0 * D3), dt * (-48.0 * D2 + 12.0 * D3)],
                   "s2")
        return U3 + w
    if scheme == "exprb53":
        y1_half, y1_nine = phi(u_n, dt, [0.5, 0.9], [None, v], "s1")
        U2 = u_n + y1_half
        D2 = _D(model, u_n, U2)
        y3_half, y3_nine = phi(u_n, dt, [0.5, 0.9], [None, None, None, dt * D2], "s2")
        U3 = (u_n + y1_nine + ((27.0 / 25.0) / 0.5 ** 3) * y3_half
              + ((729.0 / 125.0) / 0.9 ** 3) * y3_nine)
        D3 = _D(model, u_n, U3)
        (w,) = phi(u_n, dt, [1.0],
                   [None, v, None, dt * (18.0 * D2 - (250.0 / 81.0) * D3),
                    dt * (-60.0 * D2 + (500.0 / 27.0) * D3)], "s3")
        return u_n + w
    if scheme == "epi3":
        R = model.F(u_prev) - model.F(u_n) - model.Jv(u_n, u_prev - u_n)
        (w,) = phi(u_n, dt, [1.0], [None, v, (2.0 / 3.0) * dt * R], "s1")
        return u_n + w
    raise ValueError(f"unknown scheme {scheme!r}")


def integrate(scheme: str, model, u0: np.ndarray, dt: float, nsteps: int, phi) -> np.ndarray:
    """nsteps steps from u0 (epi3 starts with one EPI2 step, Sec. 3.3)."""
    u_prev, u = None, u0
    for _ in range(nsteps):
        u_next = step(scheme, model, u, dt, phi, u_prev=u_prev)
        u_prev, u = u, u_next
    return u
