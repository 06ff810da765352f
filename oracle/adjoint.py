"""Gradient of exprb steps with frozen substep decisions (oracle).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``): never used by the product path.

A step u_{n+1} = S(u_n) of Sec. 3.3, evaluated by Algorithm 1, is only
piecewise smooth in u_n: the controller's choices (substep sizes tau_k, Krylov
sizes m_k, accept/reject) jump.  With those choices held at the values of the
forward run (its attempt trace), S is a smooth map (a composition of F,
J(u_n) x, dot products, norms and the small matrix exponential), and its
derivative is what a central finite difference with the same frozen choices
measures.  This module evaluates that map once more, in torch float64 CPU
ops, and differentiates it with torch.autograd (a library primitive):

* ``TorchSWE``: F(u) and J(u) x of ``oracle.swe`` written again term by term
  (Eqs. (eq:sweqsinv), (eq:dynja)-(eq:dynjc), reading of the second J_r row as
  in ``oracle.swe``); the sparse operators are applied through a small
  autograd function whose backward is the transposed sparse product.
* ``phi_replay``: Algorithm 1 along the accepted attempts of a trace:
  w_j of Eq. (eq3.18) with the zero skip, the IOM2 basis of the oracle's
  reading R4, phi_p(tau H) e_1 and phi_{p+1}(tau H) e_1 from the augmented
  exponential (``torch.linalg.matrix_exp``), and the update of Eq. (eq3.17)
  with the corrected formula (reading R5).  Rejected attempts do not touch
  the result and are skipped.
* ``step_replay``: the schemes of ``oracle.schemes`` (EPI2, exprb42,
  pexprb43, exprb53) on top of it, D_ni evaluated literally (Eq. (eqDni)).
* ``loss_and_gradient``: the quadratic observation misfit of a forecast and
  its gradient with respect to the initial state, stepping backwards with
  one recomputed step per checkpoint (the forward states are the checkpoints).

Reading (the paper defines no adjoint): the derivative is the one of the
computed map with frozen decisions, not of the exact scheme; the two differ
at the level of the Krylov tolerance.  The misfit is taken at the end of
the forecast only: 0.5 * sum_i (h(x_i) - y_i)^2 / sigma^2.
"""
from __future__ import annotations

import math
from typing import Optional, Sequence

import numpy as np
import torch

from .phipm import Attempt, PhiOpts, phipm_simul_iom2
from .schemes import KrylovPhi, step as np_step

ADJOINT_SCHEMES = ("epi2", "exprb42", "pexprb43", "exprb53")
NCALLS = {"epi2": 1, "exprb42": 2, "pexprb43": 2, "exprb53": 3}


class _SpMV(torch.autograd.Function):
    """y = M x for a scipy sparse matrix M; backward gives M^T g."""

    @staticmethod
    def forward(ctx, x, M):
        ctx.M = M
        return torch.from_numpy(M @ x.detach().numpy())

    @staticmethod
    def backward(ctx, g):
        return torch.from_numpy(ctx.M.T @ g.detach().numpy()), None


def spmv(M, x: torch.Tensor) -> torch.Tensor:
    return _SpMV.apply(x, M)


class TorchSWE:
    """F(u) and J(u) x of ``oracle.swe.SWE`` in torch float64 (same operators)."""

    def __init__(self, swe):
        self.swe = swe
        self.ng = swe.ng
        self.n = swe.n
        self.ops = swe.ops
        self.nrm = torch.from_numpy(np.ascontiguousarray(swe.grid.x))
        self.f = torch.from_numpy(swe.f)
        self.nu = swe.nu
        self.g = swe.g
        self.nA = swe.nA
        self.hs = None if swe.hs is None else torch.from_numpy(np.asarray(swe.hs, dtype=np.float64))
        L = swe.ops.L
        self.LL = (L @ L).tocsr()

    def split(self, u):
        ng = self.ng
        return u[0:ng], u[ng:2 * ng], u[2 * ng:3 * ng], u[3 * ng:4 * ng]

    def cross_n(self, vx, vy, vz):
        n = self.nrm
        return (n[:, 1] * vz - n[:, 2] * vy, n[:, 2] * vx - n[:, 0] * vz, n[:, 0] * vy - n[:, 1] * vx)

    def vorticity(self, ux, uy, uz):
        V = self.ops.V
        return spmv(V[0], ux) + spmv(V[1], uy) + spmv(V[2], uz)

    def Df(self, psi):
        return -self.nu * spmv(self.LL, psi)

    def F(self, u):
        ux, uy, uz, h = self.split(u)
        G, D = self.ops.G, self.ops.D
        eta = self.vorticity(ux, uy, uz) + self.f
        P = self.cross_n(ux, uy, uz)
        E = 0.5 * (ux * ux + uy * uy + uz * uz) + self.g * h
        if self.hs is not None:
            E = E + self.g * self.hs
        parts = [-eta * P[c] - spmv(G[c], E) + self.Df(uc) for c, uc in enumerate((ux, uy, uz))]
        parts.append(-(spmv(D[0], ux * h) + spmv(D[1], uy * h) + spmv(D[2], uz * h)) + self.Df(h))
        return torch.cat(parts)

    def Jv(self, u, x):
        ux, uy, uz, h = self.split(u)
        xx, xy, xz, xh = self.split(x)
        G, D = self.ops.G, self.ops.D
        n = self.nrm
        nx, ny, nz = n[:, 0], n[:, 1], n[:, 2]
        P = self.cross_n(ux, uy, uz)
        eta = self.vorticity(ux, uy, uz) + self.f
        Vx = self.vorticity(xx, xy, xz)
        s = ux * xx + uy * xy + uz * xz + self.g * xh
        rot = (eta * nz * xy - eta * ny * xz,
               -eta * nz * xx + eta * nx * xz,
               eta * ny * xx - eta * nx * xy)
        parts = [-P[c] * Vx + self.Df((xx, xy, xz)[c]) + rot[c] - spmv(G[c], s) for c in range(3)]
        parts.append(self.Df(xh) - (spmv(D[0], h * xx) + spmv(D[1], h * xy) + spmv(D[2], h * xz)
                                    + spmv(D[0], ux * xh) + spmv(D[1], uy * xh) + spmv(D[2], uz * xh)))
        return torch.cat(parts)


def augmented_exp(H: torch.Tensor, tau: float, p: int) -> tuple[torch.Tensor, torch.Tensor]:
    """(phi_p(tau H) e_1, phi_{p+1}(tau H) e_1) from exp of the augmented matrix
    (the same augmentation as ``oracle.phi.augmented_krylov_matrix``)."""
    m = H.shape[0]
    M = m + p + 1
    top = torch.cat([tau * H, torch.zeros(m, p + 1, dtype=H.dtype)], dim=1)
    Hh = torch.cat([top, torch.zeros(p + 1, M, dtype=H.dtype)], dim=0)
    const = torch.zeros(M, M, dtype=H.dtype)
    const[0, m] = 1.0
    for k in range(p):
        const[m + k, m + k + 1] = 1.0
    E = torch.linalg.matrix_exp(Hh + const)
    return E[0:m, m + p - 1], E[0:m, m + p]


def phi_replay(Amul, rho: Sequence[float], v: Sequence[Optional[torch.Tensor]],
               attempts: Sequence[Attempt], breakdown: float = 1e-13) -> list:
    """y(rho_i) = sum_l rho_i^l phi_l(rho_i A) v_l along the accepted attempts."""
    p = len(v) - 1
    N = next(x.numel() for x in v if x is not None)
    acc = [a for a in attempts if a.accepted]
    it = iter(acc)
    y = torch.zeros(N, dtype=torch.float64) if v[0] is None else v[0]
    t = 0.0
    out = []
    for t_out in rho:
        while t < t_out:
            rec = next(it)
            tau, m = rec.tau, rec.m
            remaining = t_out - t
            land = tau >= remaining * (1.0 - 1e-12)
            if land:
                tau = remaining
            # Eq. (eq3.18) with the zero skip (R10)
            w = [y]
            for j in range(1, p + 1):
                c = torch.zeros(N, dtype=torch.float64)
                for l in range(0, p - j + 1):
                    if v[j + l] is not None:
                        c = c + (t ** l / math.factorial(l)) * v[j + l]
                if bool(torch.any(w[j - 1] != 0.0)):
                    c = Amul(w[j - 1]) + c
                w.append(c)
            ynew = sum((tau ** j / math.factorial(j)) * w[j] for j in range(p))
            beta = torch.linalg.norm(w[p])
            if float(beta.detach()) > 0.0:
                # IOM2 basis of m columns (R4, classical window of two)
                V = [w[p] / beta]
                Hcols = []
                hnext = None
                for j in range(m):
                    z = Amul(V[j])
                    lo = max(0, j - 1)
                    hw = [torch.dot(z, V[i]) for i in range(lo, j + 1)]
                    for i, hij in zip(range(lo, j + 1), hw):
                        z = z - hij * V[i]
                    hn = torch.linalg.norm(z)
                    if float(hn.detach()) <= breakdown * sum(abs(float(x.detach())) for x in hw):
                        raise RuntimeError("happy breakdown: the frozen-decision map is not smooth here")
                    col = [torch.zeros((), dtype=torch.float64)] * (m + 1)
                    for i, hij in zip(range(lo, j + 1), hw):
                        col[i] = hij
                    col[j + 1] = hn
                    Hcols.append(torch.stack(col))
                    V.append(z / hn)
                    hnext = hn
                Hfull = torch.stack(Hcols, dim=1)           # (m+1) x m
                phi_p, phi_p1 = augmented_exp(Hfull[0:m, :], tau, p)
                krylov = torch.stack(V[0:m], dim=1) @ phi_p + tau * hnext * phi_p1[m - 1] * V[m]
                ynew = ynew + (tau ** p) * beta * krylov
            y = ynew
            t = t_out if land else t + tau
        out.append(y)
    return out


def _D(model, u_n, U):
    """D = N_n(U) - N_n(u_n), Eq. (eqDni), literally."""
    return (model.F(U) - model.Jv(u_n, U)) - (model.F(u_n) - model.Jv(u_n, u_n))


def step_replay(scheme: str, tm: TorchSWE, u_n: torch.Tensor, dt: float, calls: Sequence) -> torch.Tensor:
    """One step of ``scheme`` with the attempts of each phi call frozen
    (``calls[k]``: attempt list of the k-th phi evaluation of the step)."""
    def Amul(x):
        return dt * tm.Jv(u_n, x)

    v = dt * tm.F(u_n)
    if scheme == "epi2":
        (y,) = phi_replay(Amul, [1.0], [None, v], calls[0])
        return u_n + y
    if scheme == "exprb42":
        (y1,) = phi_replay(Amul, [0.75], [None, v], calls[0])
        D2 = _D(tm, u_n, u_n + y1)
        (w,) = phi_replay(Amul, [1.0], [None, v, None, (32.0 / 9.0) * dt * D2], calls[1])
        return u_n + w
    if scheme == "pexprb43":
        y_half, y_one = phi_replay(Amul, [0.5, 1.0], [None, v], calls[0])
        U2, U3 = u_n + y_half, u_n + y_one
        D2, D3 = _D(tm, u_n, U2), _D(tm, u_n, U3)
        (w,) = phi_replay(Amul, [1.0], [None, None, None, dt * (16.0 * D2 - 2.0 * D3),
                                         dt * (-48.0 * D2 + 12.0 * D3)], calls[1])
        return U3 + w
    if scheme == "exprb53":
        y1_half, y1_nine = phi_replay(Amul, [0.5, 0.9], [None, v], calls[0])
        D2 = _D(tm, u_n, u_n + y1_half)
        y3_half, y3_nine = phi_replay(Amul, [0.5, 0.9], [None, None, None, dt * D2], calls[1])
        U3 = (u_n + y1_nine + ((27.0 / 25.0) / 0.5 ** 3) * y3_half
              + ((729.0 / 125.0) / 0.9 ** 3) * y3_nine)
        D3 = _D(tm, u_n, U3)
        (w,) = phi_replay(Amul, [1.0], [None, v, None, dt * (18.0 * D2 - (250.0 / 81.0) * D3),
                                         dt * (-60.0 * D2 + (500.0 / 27.0) * D3)], calls[2])
        return u_n + w
    raise ValueError(f"no adjoint for scheme {scheme!r}; supported: {ADJOINT_SCHEMES}")


def step_vjp(scheme: str, tm: TorchSWE, u_n: np.ndarray, dt: float, calls: Sequence,
             lam: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(u_{n+1}, (d u_{n+1} / d u_n)^T lam) with frozen decisions."""
    u = torch.from_numpy(np.array(u_n, dtype=np.float64)).requires_grad_(True)
    out = step_replay(scheme, tm, u, dt, calls)
    out.backward(torch.from_numpy(np.asarray(lam, dtype=np.float64)))
    return out.detach().numpy().copy(), u.grad.numpy().copy()


class ReplayPhi:
    """phi-evaluator for ``oracle.schemes.step`` that replays given traces."""

    def __init__(self, model, calls: Sequence, opts: Optional[PhiOpts] = None):
        self.model = model
        self.calls = list(calls)
        self.k = 0
        self.opts = opts or PhiOpts()

    def __call__(self, u_lin, dt, rho, v, slot):
        tr = self.calls[self.k]
        self.k += 1
        W, _ = phipm_simul_iom2(lambda x: dt * self.model.Jv(u_lin, x), rho, v, self.opts,
                                self.model.nA, replay=list(tr))
        return W


def forward_with_traces(scheme: str, swe, u0: np.ndarray, dt: float, nsteps: int,
                        opts: Optional[PhiOpts] = None):
    """Oracle forecast; returns (states u_0..u_N, per-step list of per-call traces)."""
    ncalls = NCALLS[scheme]
    phi = KrylovPhi(swe, opts or PhiOpts())
    states = [np.array(u0, dtype=np.float64)]
    traces = []
    for _ in range(nsteps):
        k0 = len(phi.stats)
        states.append(np_step(scheme, swe, states[-1], dt, phi))
        traces.append([st.trace for _, st in phi.stats[k0:k0 + ncalls]])
    return states, traces


def misfit(h_obs_cells: np.ndarray, y_obs: np.ndarray, sigma: float, u: np.ndarray, ng: int):
    """(J, dJ/du) of J = 0.5 sum_i (h_{c_i} - y_i)^2 / sigma^2 at state u."""
    h = u[3 * ng:]
    r = (h[h_obs_cells] - y_obs) / sigma
    g = np.zeros_like(u)
    np.add.at(g, 3 * ng + h_obs_cells, r / sigma)
    return 0.5 * float(r @ r), g


def loss_and_gradient(scheme: str, swe, u0: np.ndarray, dt: float, nsteps: int,
                      obs_cells: np.ndarray, y_obs: np.ndarray, sigma: float,
                      opts: Optional[PhiOpts] = None):
    """(J, dJ/du_0, traces) for the misfit at the end of an nsteps forecast."""
    states, traces = forward_with_traces(scheme, swe, u0, dt, nsteps, opts)
    J, lam = misfit(obs_cells, y_obs, sigma, states[-1], swe.ng)
    tm = TorchSWE(swe)
    for k in reversed(range(nsteps)):
        _, lam = step_vjp(scheme, tm, states[k], dt, traces[k], lam)
    return J, lam, traces


def loss_replayed(scheme: str, swe, u0: np.ndarray, dt: float, traces: Sequence,
                  obs_cells: np.ndarray, y_obs: np.ndarray, sigma: float,
                  opts: Optional[PhiOpts] = None) -> float:
    """J of the forecast from u0 with every step's decisions replayed (numpy oracle)."""
    u = np.array(u0, dtype=np.float64)
    for calls in traces:
        u = np_step(scheme, swe, u, dt, ReplayPhi(swe, calls, opts))
    return misfit(obs_cells, y_obs, sigma, u, swe.ng)[0]
