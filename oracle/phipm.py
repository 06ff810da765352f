"""phipm_simul_iom2 (Algorithm 1) with the IOM2 Krylov projection (oracle).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``): never used by the product path.

Computes, for 0 < rho_1 < ... < rho_Ns <= 1 and vectors v_0..v_p (None = 0),

    W[i] = y(rho_i) = sum_{l=0}^{p} rho_i^l phi_l(rho_i A) v_l            (*)

the solution of the ODE of Eq. (eq3.15) at t = rho_i, by the substepping of
Eqs. (eq3.17)-(eq3.18) with one Krylov approximation of phi_p(tau_k A) w_p per
substep (Sec. 4.3, Algorithm 1).

Readings where the paper is silent, garbled or inconsistent
-----------------------------------------------------------
R1  Output form (*) carries rho^l: the drivers of Sec. 4.4 only work in this
    form (Eq. (eq:exp_multistage) prints it without rho^l).
R2  The sum in Eq. (eq3.17) and Algorithm 1 step 6 runs over j = 0..p-1
    (printed with upper limit p-i); this is what Eq. (eq3.16) and the
    recurrence Eq. (eq3.7) give.
R3  beta = ||w_p||_2 of the current substep (the initialisation's
    beta = ||v_0|| cannot be the Krylov norm: the basis is built for w_p).
R4  IOM2: each new vector is orthogonalised against the previous iom = 2 basis
    vectors with both coefficients taken from the unmodified A v_j (classical
    Gram-Schmidt over the window), so H_m is tridiagonal.  Happy breakdown
    when h_{j+1,j} <= 1e-13 (|h_{j-1,j}| + |h_{j,j}|): the space is invariant,
    m is capped at j and the error estimate is 0.
R5  The corrected Krylov formula of step 2(ii) is used with the factor tau on
    the correction term, tau^p phi_p(tau A) w_p ~
    tau^p beta [V_m phi_p(tau H) e_1 + tau h_{m+1,m} (e_m^T phi_{p+1}(tau H) e_1) v_{m+1}].
R6  Error estimate: eps = tau^p beta tau |h_{m+1,m}| |e_m^T phi_{p+1}(tau H) e_1|,
    the size of that correction's contribution to y_{k+1} (step 3 prints it
    without the tau factors).
R7  Tolerance: accept when omega = t_out eps / (tau Tol s) <= delta (step 6),
    with s = max_l ||v_l||_2 in "relative" mode (the default) and s = 1 in
    "absolute" mode (the literal step 6).
R8  Controller (steps 4-5; the cited rules of the earlier works are not in
    the paper).  With target gamma = 0.8, order guess q = max(1, m/4) and rate
    kappa = 2:
        tau_new = tau (omega/gamma)^(-1/q), clamped to [tau/5, 2 tau]
                  (omega = 0 gives 2 tau);
        m_new   = m + ceil(log(omega/gamma)/log(kappa)), clamped to
                  [ceil(3m/4), floor(4m/3) + 1] and to [1, m_max]
                  (omega = 0 gives ceil(3m/4)).
    The proposal with the smaller cost of Eq. (eq:cost) is taken, comparing
    C(tau_new, m) with C(tau, m_new), where nint is round-half-up, the count
    of remaining substeps is at least 1, M = 44/3 + 2 max(0, nint(log2(
    ||tau Hhat_m||_1 / 5.37))) with the current H_m in both costs (H of size
    m_new may not exist yet), and n_A is the structural nonzero count of J.
    After a rejection the step size is taken whenever m_new = m (m at m_max
    or at the breakdown size).  The basis is kept across rejections (it
    depends on A and w_p only); a larger m extends it.
R9  Substeps land exactly on each rho_i: tau_k = rho_i - t_k whenever
    tau >= (rho_i - t_k)(1 - 1e-12), and t_k is set to rho_i after such a step.  When a step was shortened this way
    and accepted, the next step size is max(tau_new, tau) so the shortening
    does not shrink later substeps.  tau and m carry over to the next output.
R10 Zero skip (step 1): A w_{j-1} is skipped when w_{j-1} is exactly zero.
R11 Bounds (not in the paper): a call fails with NoConvergence after
    max_substeps accepted substeps (an option), after max_reject rejections,
    when an accepted substep would not move t, or when the error estimate is
    not finite, so a run whose state or step size has gone wrong ends instead
    of running on.  The exponential itself has no size limit here.

The controller of steps 4-6 is split into three functions, each pinned on its
own: ``cost`` (Eq. (eq:cost)), ``proposals`` (step 4, R8) and
``prefer_step_size`` (step 5, R8); ``accepts`` is the test of step 6.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional, Sequence

import numpy as np

from .phi import augmented_norm1, phi_krylov


class NoConvergence(RuntimeError):
    pass


@dataclasses.dataclass
class PhiOpts:
    tol: float = 1e-8
    tol_mode: str = "relative"        # "relative" | "absolute"   (R7)
    m_init: int = 1                   # Algorithm 1 initialisation
    m_max: int = 64
    iom: int = 2
    delta: float = 1.4                # Algorithm 1 initialisation
    gamma: float = 0.8                # R8
    kappa: float = 2.0                # R8
    max_reject: int = 200
    max_substeps: int = 4096          # NoConvergence beyond this many accepted substeps per call
    breakdown: float = 1e-13          # R4


@dataclasses.dataclass
class Attempt:
    t: float
    tau: float
    m: int
    omega: float
    accepted: bool


@dataclasses.dataclass
class PhiStats:
    n_jv: int = 0
    n_substeps: int = 0
    n_reject: int = 0
    m_last: int = 0
    m_max_used: int = 0
    trace: list = dataclasses.field(default_factory=list)


def nint(x: float) -> int:
    """Round half up (the paper's nint delimiter in Eq. (eq:cost))."""
    return int(math.floor(x + 0.5))


def cost(tau: float, m: int, p: int, remaining: float, N: int, nA: int, hnorm: float) -> float:
    """C(tau, m) of Eq. (eq:cost); hnorm = ||tau Hhat_m||_1, remaining = t_out - t_k.

    Readings (R8): the substep count nint(remaining / tau) is at least 1, and
    the nint of M's logarithm is at least 0 (so M >= 44/3 for small norms).
    """
    nsub = max(1, nint(remaining / tau))
    M = 44.0 / 3.0 + 2.0 * max(0, nint(math.log2(hnorm / 5.37)))
    return (nsub * m * (N + nA) + 2 * (p - 1) * (nA + N)
            + M * (m + p + 1) ** 3 + (2 * p + 1) * N)


def accepts(omega: float, delta: float) -> bool:
    """Algorithm 1 step 6: accept the substep when t_out eps / (tau Tol s) <= delta."""
    return omega <= delta


def proposals(omega: float, tau: float, m: int, cap: int, opts: "PhiOpts") -> tuple[float, int]:
    """Algorithm 1 step 4 (reading R8): (tau_new, m_new) from omega of the attempt (tau, m).

    cap: the largest usable Krylov size (m_max, or the breakdown size).
    """
    if omega == 0.0:
        tau_new = 2.0 * tau
        m_new = max(1, math.ceil(3 * m / 4))
    else:
        q = max(1.0, m / 4.0)
        tau_new = tau * (omega / opts.gamma) ** (-1.0 / q)
        tau_new = min(max(tau_new, tau / 5.0), 2.0 * tau)
        dm = math.ceil(math.log(omega / opts.gamma) / math.log(opts.kappa))
        m_new = m + dm
        m_new = min(max(m_new, math.ceil(3 * m / 4)), m * 4 // 3 + 1)
    m_new = max(1, min(m_new, opts.m_max, cap))
    return tau_new, m_new


def prefer_step_size(c_tau: float, c_m: float, accepted: bool, m_new: int, m: int) -> bool:
    """Algorithm 1 step 5 (reading R8): True to update tau, False to update m.

    The step size is updated when C(tau_new, m) <= C(tau, m_new), and after a
    rejection whenever the Krylov size cannot change (m_new = m).
    """
    return c_tau <= c_m or (not accepted and m_new == m)


class IOM2Basis:
    """Incomplete orthogonalisation (window ``iom``) of the Krylov space of A, w_p (R4)."""

    def __init__(self, Amul: Callable, v1: np.ndarray, iom: int, m_max: int, bd: float):
        self.Amul = Amul
        self.iom = iom
        self.bd = bd
        self.V = [v1]
        self.H = np.zeros((m_max + 1, m_max))
        self.size = 0              # number of columns of H built
        self.broken = False
        self.n_jv = 0

    def extend(self, m: int) -> int:
        """Build columns until m are available (or breakdown); return the usable m."""
        while self.size < m and not self.broken:
            j = self.size
            z = self.Amul(self.V[j])
            self.n_jv += 1
            window = range(max(0, j - self.iom + 1), j + 1)
            for i in window:
                self.H[i, j] = float(np.dot(z, self.V[i]))
            for i in window:
                z = z - self.H[i, j] * self.V[i]
            hn = float(np.linalg.norm(z))
            self.H[j + 1, j] = hn
            self.size = j + 1
            if hn <= self.bd * sum(abs(self.H[i, j]) for i in window):
                self.broken = True
                self.H[j + 1, j] = 0.0
                self.V.append(np.zeros_like(z))
            else:
                self.V.append(z / hn)
        return min(m, self.size)


def phipm_simul_iom2(Amul: Callable[[np.ndarray], np.ndarray],
                     rho: Sequence[float],
                     v: Sequence[Optional[np.ndarray]],
                     opts: PhiOpts,
                     nA: int,
                     m_start: Optional[int] = None,
                     replay: Optional[list] = None) -> tuple[list, PhiStats]:
    """Algorithm 1.  Returns ([y(rho_1), ..., y(rho_Ns)], stats).

    ``replay``: optional list of Attempt records; when given, the step sizes,
    Krylov sizes and accept/reject decisions are taken from it instead of the
    controller (used to force substep partitions).
    """
    rho = [float(r) for r in rho]
    if not rho or rho[0] <= 0.0 or rho[-1] > 1.0 or any(b <= a for a, b in zip(rho, rho[1:])):
        raise ValueError("rho must satisfy 0 < rho_1 < ... < rho_Ns <= 1")
    p = len(v) - 1
    if p < 1:
        raise ValueError("p >= 1 required")
    N = next(x.size for x in v if x is not None) if any(x is not None for x in v) else None
    if N is None:
        raise ValueError("at least one v_l must be given")
    vs = [None if x is None else np.asarray(x, dtype=np.float64) for x in v]
    stats = PhiStats()
    norms = [0.0 if x is None else float(np.linalg.norm(x)) for x in vs]
    scale = max(norms) if opts.tol_mode == "relative" else 1.0
    if scale == 0.0:
        return [np.zeros(N) for _ in rho], stats

    t = 0.0
    y = np.zeros(N) if vs[0] is None else vs[0].copy()
    tau = rho[0]                                  # initial substep (initialisation)
    m = m_start if m_start is not None else opts.m_init
    m = max(1, min(m, opts.m_max))
    out = []
    rp = iter(replay) if replay is not None else None

    for t_out in rho:
        while t < t_out:
            # step 1: w_0 = y_k, w_j = A w_{j-1} + sum_l t^l/l! v_{j+l} (eq3.18), R10
            w = [y]
            for j in range(1, p + 1):
                acc = np.zeros(N)
                for l in range(0, p - j + 1):
                    if vs[j + l] is not None:
                        acc = acc + (t ** l / math.factorial(l)) * vs[j + l]
                if np.any(w[j - 1] != 0.0):
                    wj = Amul(w[j - 1]) + acc
                    stats.n_jv += 1
                else:
                    wj = acc
                w.append(wj)
            beta = float(np.linalg.norm(w[p]))
            basis = IOM2Basis(Amul, w[p] / beta, opts.iom, opts.m_max, opts.breakdown) \
                if beta > 0.0 else None

            while True:                           # attempts on this substep
                remaining = t_out - t
                land = tau >= remaining * (1.0 - 1e-12)
                tau_k = remaining if land else tau
                if rp is not None:
                    rec = next(rp)
                    tau_k, m = rec.tau, rec.m
                    land = tau_k >= remaining * (1.0 - 1e-12)
                    if land:
                        tau_k = remaining
                # step 2: Krylov approximation of phi_p(tau A) w_p
                if basis is not None:
                    m_use = basis.extend(m)
                    Hm = basis.H[0:m_use, 0:m_use]
                    hnext = basis.H[m_use, m_use - 1]
                    hnorm = augmented_norm1(Hm, tau_k, p)
                    phi_p, phi_p1 = phi_krylov(Hm, tau_k, p)
                    eps = tau_k ** p * beta * tau_k * abs(hnext) * abs(phi_p1[m_use - 1])  # R6
                else:
                    m_use, eps, hnorm = m, 0.0, 1.0
                # step 6 test (R7)
                omega = t_out * eps / (tau_k * opts.tol * scale)
                if not math.isfinite(omega):
                    raise NoConvergence("phipm_simul_iom2: non-finite error estimate")
                accepted = accepts(omega, opts.delta) if rp is None else rec.accepted
                stats.trace.append(Attempt(t=t, tau=tau_k, m=m_use, omega=omega, accepted=accepted))
                stats.m_max_used = max(stats.m_max_used, m_use)

                # steps 4-5: proposals and cost comparison (R8)
                cap = basis.size if (basis is not None and basis.broken) else opts.m_max
                tau_new, m_new = proposals(omega, tau_k, m_use, cap, opts)
                hnorm_new = augmented_norm1(Hm, tau_new, p) if basis is not None else 1.0
                c_tau = cost(tau_new, m_use, p, remaining, N, nA, hnorm_new)
                c_m = cost(tau_k, m_new, p, remaining, N, nA, hnorm)
                take_tau = prefer_step_size(c_tau, c_m, accepted, m_new, m_use)

                if accepted:
                    # y_{k+1} = tau^p phi_p(tau A) w_p + sum_{j<p} tau^j/j! w_j (eq3.17, R2, R5)
                    ynew = np.zeros(N)
                    for j in range(p):
                        ynew = ynew + (tau_k ** j / math.factorial(j)) * w[j]
                    if basis is not None:
                        Vm = np.stack(basis.V[0:m_use], axis=1)
                        krylov = Vm @ phi_p
                        krylov = krylov + tau_k * hnext * phi_p1[m_use - 1] * basis.V[m_use]
                        ynew = ynew + (tau_k ** p * beta) * krylov
                    y = ynew
                    t_next = t_out if land else t + tau_k
                    if not t_next > t or stats.n_substeps >= opts.max_substeps:
                        raise NoConvergence(f"phipm_simul_iom2: {stats.n_substeps} substeps, no progress at t={t}")
                    t = t_next
                    stats.n_substeps += 1
                    if take_tau:
                        tau = max(tau_new, tau) if land else tau_new
                    else:
                        tau = max(tau_k, tau) if land else tau_k
                        m = m_new
                    stats.m_last = m_use
                    break
                stats.n_reject += 1
                if stats.n_reject > opts.max_reject or tau_k < 1e-14:
                    raise NoConvergence(f"phipm_simul_iom2: {stats.n_reject} rejections, tau={tau_k}")
                if take_tau:
                    tau = tau_new
                    m = m_use
                else:
                    tau = tau_k
                    m = m_new
            if basis is not None:
                stats.n_jv += basis.n_jv
        out.append(y.copy())
    return out, stats
