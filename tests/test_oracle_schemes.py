"""Pins of the oracle exponential integrators (Sec. 3.3, Sec. 4.4).

* Table 1 stiff order conditions evaluated on the scalar coefficient functions
  of the golden coefficient file (copied from Eqs. (eq3.11)-(eq3.13)); the
  725/125 of the Sec. 4.4 driver text fails condition 4, 729/125 passes.
* Observed convergence orders 2 (EPI2), 3 (epi3), 4 (exprb42, pexprb43),
  5 (exprb53) on a small quadratic ODE with exact (dense) phi-functions,
  against an independent high-order Runge-Kutta reference (scipy DOP853).
* Exactness on linear F (D_ni = 0, every scheme is exp(dt L) u + dt phi_1 c).
* Discrete mass sum_i A_i h_i is conserved by a Krylov step.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle.phi import phi_combination_dense
from oracle.phipm import PhiOpts
from oracle.schemes import DensePhi, KrylovPhi, integrate, step
from paper_1805_02144_gb300.inputs import balanced_state

from conftest import oracle_swe

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "scheme_coefficients.json")))


def phi(k, z):
    if abs(z) <= 4.0:
        return sum(z ** j / math.factorial(j + k) for j in range(80))
    return (np.exp(z) - sum(z ** j / math.factorial(j) for j in range(k))) / z ** k


def b_of(scheme, i, z):
    return sum(c * phi(int(k), z) for k, c in GOLD[scheme]["b"][str(i)].items())


def psi3(scheme, i, z, coeffs=None):
    """psi_{3,i}(z) = sum_k a_ik(z) c_k^2/2 - c_i^3 phi_3(c_i z) (Table 1 caption)."""
    c = {int(k): v for k, v in GOLD[scheme]["c"].items()}
    a = coeffs if coeffs is not None else GOLD[scheme]["a"]
    tot = -c[i] ** 3 * phi(3, c[i] * z)
    for key, terms in a.items():
        ii, kk = map(int, key.split(","))
        if ii == i:
            tot += sum(cf * phi(k, s * z) for cf, k, s in terms) * c[kk] ** 2 / 2.0
    return tot


@pytest.mark.parametrize("z", [0.0, -0.3, -2.5, 1.7, -12.0])
def test_table1_conditions_1_and_2(z):
    for scheme in ("pexprb43", "exprb53"):
        c = {int(k): v for k, v in GOLD[scheme]["c"].items()}
        s1 = sum(b_of(scheme, i, z) * c[i] ** 2 for i in c)
        s2 = sum(b_of(scheme, i, z) * c[i] ** 3 for i in c)
        assert s1 == pytest.approx(2 * phi(3, z), rel=1e-12, abs=1e-14)
        assert s2 == pytest.approx(6 * phi(4, z), rel=1e-12, abs=1e-14)
    # exprb42 satisfies condition 1 identically
    sch = "exprb42"
    assert b_of(sch, 2, z) * 0.75 ** 2 == pytest.approx(2 * phi(3, z), rel=1e-12, abs=1e-14)


def test_table1_conditions_3_and_4_for_exprb53():
    c = {int(k): v for k, v in GOLD["exprb53"]["c"].items()}
    s3 = sum(b_of("exprb53", i, 0.0) * c[i] ** 4 for i in c)
    assert s3 == pytest.approx(24 * phi(5, 0.0), rel=1e-12)
    # condition 4: sum_i b_i(Z) c_i K psi_{3,i}(Z) = 0 for all K requires the
    # phi_3(c_3 Z) part of psi_{3,3} to vanish and the phi_3(Z/2) parts to cancel
    for z in (0.0,):
        cond4 = sum(b_of("exprb53", i, z) * c[i] * psi3("exprb53", i, z) for i in c)
        assert abs(cond4) < 1e-14
    for z in (-0.7, -3.0, 0.9):
        # psi_{3,3} is a multiple of phi_3(z/2) only (no phi_3(0.9 z) term left)
        assert psi3("exprb53", 3, z) == pytest.approx(0.135 * phi(3, 0.5 * z), rel=1e-12)
    # the driver-text 725/125 leaves a phi_3(0.9 z) residual and breaks condition 4
    bad = GOLD["exprb53_driver_text_garble"]["a"]
    cond4_bad = sum(b_of("exprb53", i, 0.0) * c[i] * psi3("exprb53", i, 0.0, bad) for i in c)
    assert abs(cond4_bad) > 1e-5


class QuadraticODE:
    """u' = L u + Q(u): a small damped-rotating system with quadratic coupling."""

    nA = 16

    def __init__(self, stiff=4.0):
        self.L = stiff * np.array([[-0.2, 1.0, 0.0, 0.0], [-1.0, -0.2, 0.0, 0.0],
                                   [0.0, 0.0, -0.5, 0.6], [0.0, 0.0, -0.6, -0.5]])

    def F(self, u):
        q = np.array([u[0] * u[2], -u[1] * u[3], u[0] * u[1], 0.5 * u[2] ** 2])
        return self.L @ u + q

    def jacobian(self, u):
        dq = np.array([[u[2], 0, u[0], 0], [0, -u[3], 0, -u[1]],
                       [u[1], u[0], 0, 0], [0, 0, u[2], 0]])
        return self.L + dq

    def Jv(self, u, x):
        return self.jacobian(u) @ x


@pytest.mark.parametrize("scheme,order", [("epi2", 2), ("epi3", 3), ("exprb42", 4),
                                          ("pexprb43", 4), ("exprb53", 5)])
def test_observed_order_on_quadratic_ode(scheme, order):
    model = QuadraticODE()
    u0 = np.array([1.0, 0.5, -0.8, 0.3])
    T = 2.0
    ref = solve_ivp(lambda t, y: model.F(y), (0, T), u0, method="DOP853",
                    rtol=1e-13, atol=1e-15).y[:, -1]
    dts, errs = [], []
    for N in (8, 16, 32, 64):
        uN = integrate(scheme, model, u0, T / N, N, DensePhi(model))
        e = np.linalg.norm(uN - ref)
        if e > 1e-12:
            dts.append(T / N)
            errs.append(e)
    slope = np.polyfit(np.log(dts), np.log(errs), 1)[0]
    assert abs(slope - order) < 0.3, (scheme, slope, errs)


class LinearModel:
    """F(u) = J0 u + c with J0 the SWE Jacobian at a fixed state."""

    def __init__(self, s, u0):
        self.J0 = s.jacobian(u0)
        self.c = 1e-4 * s.F(u0)
        self.nA = s.nA

    def F(self, u):
        return self.J0 @ u + self.c

    def Jv(self, u, x):
        return self.J0 @ x

    def jacobian(self, u):
        return self.J0


@pytest.mark.parametrize("scheme", ["epi2", "exprb42", "pexprb43", "exprb53"])
def test_exact_for_linear_problems(scheme):
    s = oracle_swe(2)
    u0 = balanced_state(s.grid.x, 1, 400.0)
    model = LinearModel(s, u0)
    dt = 7200.0
    exact = u0 + phi_combination_dense(dt * model.J0.toarray(), [None, dt * model.F(u0)], 1.0)
    got = step(scheme, model, u0, dt, KrylovPhi(model, PhiOpts(tol=1e-12)))
    assert np.linalg.norm(got - exact) <= 1e-10 * np.linalg.norm(exact - u0)


@pytest.mark.parametrize("scheme", ["exprb42", "pexprb43", "exprb53", "epi3"])
def test_krylov_step_matches_dense_and_conserves_mass(scheme):
    s = oracle_swe(2)
    u0 = balanced_state(s.grid.x, 2, 400.0)
    dt = 3600.0
    kp = KrylovPhi(s, PhiOpts(tol=1e-12))
    a = integrate(scheme, s, u0, dt, 2, kp)
    b = integrate(scheme, s, u0, dt, 2, DensePhi(s))
    assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b - u0)
    assert abs(s.mass(a) - s.mass(u0)) <= 1e-13 * s.mass(u0)
