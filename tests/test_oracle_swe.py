"""Pins of the oracle F(u) and J(u)x.

* F is quadratic in u, so the central difference (F(u+e x) - F(u-e x))/(2e) is
  exactly J(u)x up to rounding for any e: this pins every term of the Jacobian
  blocks of Eqs. (eq:dynja)-(eq:dynjc) against F of Eq. (eq:sweqsinv), and in
  particular the reading of the second row of J_r (the printed signs fail).
* Mass: sum_i A_i (dh/dt)_i = 0 for every state (flux form), and a^T J = 0 for
  the mass functional a.
* A fluid at rest with flat height is a steady state: F = 0.
* Quadratic structure: F(u+d) - F(u) - J(u)d does not depend on u; it is the
  quadratic part Q(d) = F(d) - J(0)d (used for D_ni and R_{n-1}).
"""
import numpy as np
import pytest

from paper_1805_02144_gb300.inputs import balanced_state, random_vector

from conftest import oracle_swe


@pytest.mark.parametrize("lev,seed", [(2, 1), (3, 2), (4, 3)])
def test_jv_equals_central_difference(lev, seed):
    s = oracle_swe(lev)
    u = balanced_state(s.grid.x, seed, 400.0)
    for k in range(3):
        x = random_vector(s.n, 100 + k) * np.concatenate([np.full(3 * s.ng, 10.0), np.full(s.ng, 100.0)])
        jx = s.Jv(u, x)
        eps = 1.0
        fd = (s.F(u + eps * x) - s.F(u - eps * x)) / (2 * eps)
        assert np.linalg.norm(fd - jx) <= 1e-12 * np.linalg.norm(jx)


def test_printed_jr_row2_signs_fail_the_difference_check():
    """Planting the printed signs [eta n_z, ., -eta n_x] in J_r row 2 breaks J = dF/du."""
    s = oracle_swe(3)
    u = balanced_state(s.grid.x, 1, 200.0)
    x = random_vector(s.n, 5)
    ng = s.ng
    n = s.grid.x
    eta = s.vorticity(*s.split(u)[:3]) + s.f
    xx, xy, xz, _ = s.split(x)
    printed = s.Jv(u, x).copy()
    printed[ng:2 * ng] += 2.0 * eta * (n[:, 2] * xx - n[:, 0] * xz)
    fd = (s.F(u + x) - s.F(u - x)) / 2.0
    assert np.linalg.norm(fd - printed) > 1e-6 * np.linalg.norm(fd)


def test_assembled_jacobian_matches_matrix_free():
    s = oracle_swe(2)
    u = balanced_state(s.grid.x, 3, 300.0)
    J = s.jacobian(u)
    x = random_vector(s.n, 9)
    assert np.linalg.norm(J @ x - s.Jv(u, x)) <= 1e-14 * np.linalg.norm(J @ x)


def test_mass_is_conserved_by_F_and_J():
    s = oracle_swe(4)
    u = balanced_state(s.grid.x, 2, 400.0)
    a = s.grid.area
    Fh = s.split(s.F(u))[3]
    assert abs(np.sum(a * Fh)) <= 1e-13 * np.sum(a * np.abs(Fh))
    x = random_vector(s.n, 4)
    Jh = s.split(s.Jv(u, x))[3]
    assert abs(np.sum(a * Jh)) <= 1e-13 * np.sum(a * np.abs(Jh))


def test_rest_state_is_steady():
    s = oracle_swe(3)
    u = np.concatenate([np.zeros(3 * s.ng), np.full(s.ng, 5960.0)])
    F = s.F(u)
    # momentum: -G(g h) of a constant; continuity: -D(0); both vanish
    assert np.max(np.abs(F)) < 1e-12 * s.g * 5960.0 / s.grid.radius


def test_quadratic_remainder_is_independent_of_base_state():
    s = oracle_swe(3)
    u1 = balanced_state(s.grid.x, 1, 200.0)
    u2 = balanced_state(s.grid.x, 7, 400.0)
    d = balanced_state(s.grid.x, 11, 50.0)
    d[3 * s.ng:] -= 5960.0
    r1 = s.F(u1 + d) - s.F(u1) - s.Jv(u1, d)
    r2 = s.F(u2 + d) - s.F(u2) - s.Jv(u2, d)
    q = s.F(d) - s.Jv(np.zeros(s.n), d)
    scale = np.linalg.norm(s.F(u1))
    assert np.linalg.norm(r1 - q) <= 1e-12 * scale
    assert np.linalg.norm(r2 - q) <= 1e-12 * scale
    assert np.linalg.norm(q) > 1e-8 * scale


# -- conservation diagnostics (Rossby-Haurwitz section) -------------------------
def _solid_body(s, w, H):
    """u = w (e_z x r) (rotation about the axis with angular speed w), h = H."""
    n = s.grid.x
    a = s.grid.radius
    vel = w * a * np.stack([-n[:, 1], n[:, 0], np.zeros(s.ng)], axis=1)
    return np.concatenate([vel[:, 0], vel[:, 1], vel[:, 2], np.full(s.ng, H)])


def test_energy_and_enstrophy_of_rest_state():
    s = oracle_swe(4)
    H = 5960.0
    u = np.concatenate([np.zeros(3 * s.ng), np.full(s.ng, H)])
    a = s.grid.radius
    area = 4.0 * np.pi * a * a
    assert s.energy(u) == pytest.approx(area * 0.5 * s.g * H * H, rel=1e-12)
    # sum_i A_i f_i^2 / (2H) -> (2 Omega)^2 / (2H) * a^2 * 4 pi / 3 (quadrature error O(dx^2))
    exact = (2.0 * s.omega) ** 2 / (2.0 * H) * a * a * 4.0 * np.pi / 3.0
    assert s.potential_enstrophy(u) == pytest.approx(exact, rel=2e-3)


def test_diagnostics_of_solid_body_rotation_converge_to_closed_forms():
    """Energy and potential enstrophy of u = w e_z x r, h = H against their
    integrals: kinetic H w^2 a^4 (4 pi/3)... via int cos^2 = 8 pi/3, and the
    absolute vorticity (2w + 2 Omega) sin(lat) (zeta of a solid-body rotation
    is 2 w sin(lat)), so errors shrink about fourfold per level."""
    H, w = 5960.0, 2e-6
    errs = []
    for lev in (3, 4, 5):
        s = oracle_swe(lev)
        a = s.grid.radius
        u = _solid_body(s, w, H)
        e_exact = H * 0.5 * (w * a) ** 2 * a * a * 8.0 * np.pi / 3.0 + 4.0 * np.pi * a * a * 0.5 * s.g * H * H
        z_exact = (2.0 * w + 2.0 * s.omega) ** 2 / (2.0 * H) * a * a * 4.0 * np.pi / 3.0
        ee = abs(s.energy(u) - e_exact) / e_exact
        ez = abs(s.potential_enstrophy(u) - z_exact) / z_exact
        errs.append((ee, ez))
    assert errs[-1][0] <= 1e-5 and errs[-1][1] <= 1e-3, errs
    assert errs[2][1] < 0.5 * errs[0][1], errs      # the vorticity term converges


# -- topography -------------------------------------------------------------
def _with_hs(s, hs):
    import dataclasses
    return dataclasses.replace(s, hs=hs)


def test_topography_enters_F_through_the_gradient_only():
    """F(u; h_s) - F(u; 0) = (-G_c(g h_s), 0) exactly, and J does not change."""
    from paper_1805_02144_gb300.inputs import topography
    s = oracle_swe(3)
    hs = topography(s.grid.x, 9, 2000.0)
    st = _with_hs(s, hs)
    u = balanced_state(s.grid.x, 2, 300.0)
    dF = st.F(u) - s.F(u)
    ng = s.ng
    for c in range(3):
        ref = -(s.ops.G[c] @ (s.g * hs))
        assert np.abs(dF[c * ng:(c + 1) * ng] - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(dF[3 * ng:]).max() == 0.0
    x = random_vector(s.n, 3)
    assert np.array_equal(st.Jv(u, x), s.Jv(u, x))


def test_lake_at_rest_over_topography_has_no_momentum_tendency():
    """u = 0, h + h_s = const: the pressure gradient of a constant vanishes
    (edge values of a constant are that constant), so F_u = 0 to rounding;
    only the hyperdiffusion of h remains in F_h."""
    from paper_1805_02144_gb300.inputs import topography
    s = oracle_swe(4)
    hs = topography(s.grid.x, 9, 2000.0)
    st = _with_hs(s, hs)
    u = np.concatenate([np.zeros(3 * s.ng), 5960.0 - hs])
    F = st.F(u)
    scale = np.abs(s.ops.G[0] @ (s.g * hs)).max()     # the size of either gradient alone
    assert np.abs(F[:3 * s.ng]).max() <= 1e-12 * scale
    assert np.abs(F[3 * s.ng:] - (-s.nu * (s.ops.L @ (s.ops.L @ u[3 * s.ng:])))).max() \
        <= 1e-12 * np.abs(F[3 * s.ng:]).max()
