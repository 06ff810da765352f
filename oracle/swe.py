"""Semi-discrete shallow-water equations F(u) and their Jacobian (oracle).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``): never used by the product path.

State layout, Eq. (eq:dynu): u = (u_x, u_y, u_z, h), each a column of N_g
cell averages, so n = 4 N_g.

F(u) follows Eq. (eq:sweqsinv) with the absolute vorticity of Eq. (eq:vort) and
the dissipation D_f = -nu L^2 of Eq. (eq:swdis) added to every prognostic
variable, nu from Eq. (eq:niu):

    du_c/dt = -eta * P_c - G_c E - nu L(L u_c),        c = x, y, z
    dh/dt   = -(D_x (u_x h) + D_y (u_y h) + D_z (u_z h)) - nu L(L h)
    eta = V_x u_x + V_y u_y + V_z u_z + f,  f = 2 Omega n_z,  P = n x u,
    E   = (u_x^2 + u_y^2 + u_z^2)/2 + g (h + h_s),  h_s = 0 unless given.

With topography (``hs``, the surface height h_s per cell, constant in time)
only E changes: F gains -G (g h_s); J(u) does not depend on h_s.

The Jacobian J = J_v + J_r + J_m is applied block by block as printed in
Eqs. (eq:dynja)-(eq:dynjc).  Reading: the second row of J_r is printed as
[eta n_z, D_f, -eta n_x, 0]; differentiating -eta P_y = -eta (n_z u_x - n_x u_z)
gives [-eta n_z, D_f, +eta n_x, 0], and this module uses the derivative (the
first and third rows agree with F as printed).  The central-difference test
pins this: F is quadratic, so (F(u+e x) - F(u-e x))/(2e) equals J x exactly up
to rounding.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from .mesh import Grid, Operators, build_grid, build_operators, nnz_jacobian

EARTH_RADIUS = 6.37122e6      # a [m]
GRAVITY = 9.80616             # g [m s^-2]
OMEGA = 7.292e-5              # Omega [s^-1]
GAMMA_H = 0.04e-2             # gamma_h of Eq. (eq:niu), Sec. 5 default
DT_E = 240.0                  # Delta t_e [s], Eq. (eq:niu)
N_GAMMA = 4                   # n_gamma, Eq. (eq:niu)


def dissipation_coefficient(ncells: int, radius: float, gamma_h: float) -> float:
    """nu = gamma_h * dx^n_gamma / dt_e with dx = sqrt(4 pi a^2 / N_g), Eq. (eq:niu)."""
    dx = np.sqrt(4.0 * np.pi * radius * radius / ncells)
    return gamma_h * dx ** N_GAMMA / DT_E


@dataclasses.dataclass
class SWE:
    grid: Grid
    ops: Operators
    g: float = GRAVITY
    omega: float = OMEGA
    gamma_h: float = GAMMA_H
    hs: np.ndarray = None          # surface height h_s per cell [m] (None = 0)

    @property
    def ng(self) -> int:
        return self.grid.ncells

    @property
    def n(self) -> int:
        return self.grid.n

    @property
    def nu(self) -> float:
        return dissipation_coefficient(self.ng, self.grid.radius, self.gamma_h)

    @property
    def f(self) -> np.ndarray:
        """Coriolis parameter f = 2 Omega sin(theta) = 2 Omega n_z at cell centres."""
        return 2.0 * self.omega * self.grid.x[:, 2]

    @property
    def nA(self) -> int:
        return nnz_jacobian(self.grid)

    # -- helpers ------------------------------------------------------------
    def split(self, u: np.ndarray):
        ng = self.ng
        return u[0:ng], u[ng:2 * ng], u[2 * ng:3 * ng], u[3 * ng:4 * ng]

    def cross_n(self, vx, vy, vz):
        """(n x v) per cell: P_x = n_y v_z - n_z v_y etc. (Sec. 2, below Eq. (eq:vort))."""
        n = self.grid.x
        return (n[:, 1] * vz - n[:, 2] * vy,
                n[:, 2] * vx - n[:, 0] * vz,
                n[:, 0] * vy - n[:, 1] * vx)

    def vorticity(self, ux, uy, uz):
        """Relative vorticity V_x u_x + V_y u_y + V_z u_z (Eq. (eq:vort) without f)."""
        V = self.ops.V
        return V[0] @ ux + V[1] @ uy + V[2] @ uz

    def Df(self, psi):
        """Dissipation operator D_f psi = -nu L(L psi), Eq. (eq:swdis)."""
        L = self.ops.L
        return -self.nu * (L @ (L @ psi))

    # -- F -------------------------------------------------------------------
    def F(self, u: np.ndarray) -> np.ndarray:
        ux, uy, uz, h = self.split(u)
        G, D = self.ops.G, self.ops.D
        eta = self.vorticity(ux, uy, uz) + self.f
        P = self.cross_n(ux, uy, uz)
        E = 0.5 * (ux * ux + uy * uy + uz * uz) + self.g * h
        if self.hs is not None:
            E = E + self.g * self.hs
        out = np.empty_like(u)
        ng = self.ng
        for c, uc in enumerate((ux, uy, uz)):
            out[c * ng:(c + 1) * ng] = -eta * P[c] - G[c] @ E + self.Df(uc)
        out[3 * ng:] = -(D[0] @ (ux * h) + D[1] @ (uy * h) + D[2] @ (uz * h)) + self.Df(h)
        return out

    # -- J x ----------------------------------------------------------------
    def Jv(self, u: np.ndarray, x: np.ndarray) -> np.ndarray:
        """J(u) x = J_v x + J_r x + J_m x, Eqs. (eq:dynja)-(eq:dynjc)."""
        ux, uy, uz, h = self.split(u)
        xx, xy, xz, xh = self.split(x)
        G, D, V = self.ops.G, self.ops.D, self.ops.V
        n = self.grid.x
        nx, ny, nz = n[:, 0], n[:, 1], n[:, 2]
        P = self.cross_n(ux, uy, uz)
        eta = self.vorticity(ux, uy, uz) + self.f
        ng = self.ng
        out = np.zeros_like(x)

        # J_v (Eq. (eq:dynja)): row c = -{P_c^i V_d^{ij}}, d = x, y, z
        Vx = V[0] @ xx + V[1] @ xy + V[2] @ xz
        for c in range(3):
            out[c * ng:(c + 1) * ng] -= P[c] * Vx

        # J_r (Eq. (eq:dynjb)): D_f on the diagonal blocks plus the rotation
        # rows x: [., eta n_z, -eta n_y], y: [-eta n_z, ., eta n_x] (reading),
        # z: [eta n_y, -eta n_x, .]
        out[0:ng] += self.Df(xx) + eta * nz * xy - eta * ny * xz
        out[ng:2 * ng] += -eta * nz * xx + self.Df(xy) + eta * nx * xz
        out[2 * ng:3 * ng] += eta * ny * xx - eta * nx * xy + self.Df(xz)
        out[3 * ng:] += self.Df(xh)

        # J_m (Eq. (eq:dynjc)): row c = -[G_c u_x, G_c u_y, G_c u_z, g G_c],
        # row h = -[D_x h, D_y h, D_z h, D_x u_x + D_y u_y + D_z u_z]
        s = ux * xx + uy * xy + uz * xz + self.g * xh
        for c in range(3):
            out[c * ng:(c + 1) * ng] -= G[c] @ s
        out[3 * ng:] -= (D[0] @ (h * xx) + D[1] @ (h * xy) + D[2] @ (h * xz)
                         + D[0] @ (ux * xh) + D[1] @ (uy * xh) + D[2] @ (uz * xh))
        return out

    def jacobian(self, u: np.ndarray) -> sp.csr_matrix:
        """J(u) assembled as a sparse (4N_g x 4N_g) matrix from the same blocks."""
        ux, uy, uz, h = self.split(u)
        G, D, V = self.ops.G, self.ops.D, self.ops.V
        n = self.grid.x
        P = self.cross_n(ux, uy, uz)
        eta = self.vorticity(ux, uy, uz) + self.f
        L = self.ops.L
        Dfm = -self.nu * (L @ L)
        dg = sp.diags
        Z = None
        Jv = [[-dg(P[c]) @ V[d] for d in range(3)] + [Z] for c in range(3)]
        Jv.append([Z, Z, Z, Z])
        en = [dg(eta * n[:, k]) for k in range(3)]
        Jr = [[Dfm, en[2], -en[1], Z],
              [-en[2], Dfm, en[0], Z],
              [en[1], -en[0], Dfm, Z],
              [Z, Z, Z, Dfm]]
        uc = (ux, uy, uz)
        Jm = [[-(G[c] @ dg(uc[d])) for d in range(3)] + [-self.g * G[c]] for c in range(3)]
        Jm.append([-(D[d] @ dg(h)) for d in range(3)]
                  + [-(D[0] @ dg(ux) + D[1] @ dg(uy) + D[2] @ dg(uz))])
        blocks = []
        for r in range(4):
            row = []
            for c in range(4):
                terms = [b for b in (Jv[r][c], Jr[r][c], Jm[r][c]) if b is not None]
                row.append(sum(terms[1:], terms[0]) if terms else None)
            blocks.append(row)
        return sp.bmat(blocks, format="csr")

    # -- nonlinear remainder ---------------------------------------------------
    def N(self, u_lin: np.ndarray, u: np.ndarray) -> np.ndarray:
        """N_n(u) = F(u) - J_n u with J_n = J(u_lin), Eq. (eq3.2)."""
        return self.F(u) - self.Jv(u_lin, u)

    # -- diagnostics ---------------------------------------------------------
    def mass(self, u: np.ndarray) -> float:
        """Total mass sum_i A_i h_i (the conserved quantity of Sec. 5.2)."""
        return float(np.sum(self.grid.area * self.split(u)[3]))

    def energy(self, u: np.ndarray) -> float:
        """Total energy sum_i A_i h_i (|u_i|^2/2 + g h_i/2) (conservation
        diagnostics of the Rossby-Haurwitz section).  Reading: the paper prints
        the density g h + |u|^2/2, which is the Bernoulli function E of
        Eq. (eq:sweqsinv); the quantity the shallow-water equations conserve is
        its mass-weighted form with the potential term halved, used here."""
        ux, uy, uz, h = self.split(u)
        return float(np.sum(self.grid.area * h * (0.5 * (ux * ux + uy * uy + uz * uz) + 0.5 * self.g * h)))

    def potential_enstrophy(self, u: np.ndarray) -> float:
        """Total potential enstrophy sum_i A_i (zeta_i + f_i)^2 / (2 h_i), with the
        relative vorticity zeta = V . u of Eq. (eq:vort) (same section)."""
        ux, uy, uz, h = self.split(u)
        eta = self.vorticity(ux, uy, uz) + self.f
        return float(np.sum(self.grid.area * eta * eta / (2.0 * h)))


def make_swe(level: int, radius: float = EARTH_RADIUS, g: float = GRAVITY,
             omega: float = OMEGA, gamma_h: float = GAMMA_H) -> SWE:
    grid = build_grid(level, radius)
    return SWE(grid=grid, ops=build_operators(grid), g=g, omega=omega, gamma_h=gamma_h)
