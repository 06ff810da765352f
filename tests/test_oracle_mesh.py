"""Pins of the oracle grid and finite-volume operators against closed forms.

The discrete operators must reproduce, with an error that shrinks under
refinement, the continuous surface operators of Sec. 2 on fields whose
derivatives are known in closed form (phi = b.n, psi = c.n, P = I - n n^T):
  * gradient of psi                      -> (c - n psi) / a
  * divergence of q = phi P c            -> -2 phi psi / a + (P c).(P b) / a
  * normal vorticity of u = phi a w x n  -> 2 phi w.n + n.(grad phi x a w x n)
  * Laplacian of n_z (degree-1 harmonic) -> -2 n_z / a^2
The fields are anisotropic so that an inconsistent edge quadrature, a sign
error, a missing factor or a transposed operand all change the limit.
"""
import json
import os

import numpy as np
import pytest

from oracle.mesh import build_grid, build_operators, nnz_jacobian

GOLD = os.path.join(os.path.dirname(__file__), "golden")
A = 6.37122e6


def test_grid_counts_match_paper_formula():
    gold = json.load(open(os.path.join(GOLD, "grid_counts.json")))
    for lev in range(0, 6):
        g = build_grid(lev)
        assert g.ncells == gold["levels"][str(lev)]
        assert g.edge_i.size // 2 == 3 * g.ncells - 6
        deg = g.degree()
        assert np.sum(deg == 5) == 12 and np.all((deg == 5) | (deg == 6))
    assert 4 * gold["levels"]["6"] == gold["level6_unknowns"]


@pytest.mark.parametrize("lev", [0, 2, 4, 5])
def test_areas_tile_the_sphere(lev):
    g = build_grid(lev)
    assert abs(np.sum(g.area) / (4 * np.pi * A * A) - 1.0) < 1e-13
    assert np.all(g.area > 0)


def test_edge_geometry_antisymmetry():
    g = build_grid(3)
    key = {(i, j): k for k, (i, j) in enumerate(zip(g.edge_i, g.edge_j))}
    rev = np.array([key[(j, i)] for i, j in zip(g.edge_i, g.edge_j)])
    assert np.allclose(g.nu[rev], -g.nu, atol=1e-15)
    assert np.allclose(g.te[rev], -g.te, atol=1e-15)
    assert np.allclose(g.le[rev], g.le, rtol=1e-14)
    # nu is tangent at the Voronoi edge and unit
    assert np.allclose(np.linalg.norm(g.nu, axis=1), 1.0)
    # mean cell spacing matches dx = sqrt(4 pi a^2 / N_g) of Eq. (eq:niu) to O(1)
    dx = np.sqrt(4 * np.pi * A * A / g.ncells)
    assert 0.8 < np.mean(g.de) / dx < 1.3


def _errors(lev):
    g = build_grid(lev)
    ops = build_operators(g)
    n = g.x
    c = np.array([0.3, -0.5, 0.8])
    w = np.array([0.2, 0.7, -0.4])
    b = np.array([-0.6, 0.1, 0.5])
    psi, phi = n @ c, n @ b
    Pc = c[None, :] - n * psi[:, None]
    gphi = (b[None, :] - n * phi[:, None]) / A
    out = {}
    grad_exact = Pc / A
    grad = np.stack([ops.G[k] @ psi for k in range(3)], axis=1)
    out["G"] = np.max(np.abs(grad - grad_exact)) / np.max(np.abs(grad_exact))
    q = phi[:, None] * Pc
    div_exact = phi * (-2.0 * psi / A) + np.sum(Pc * gphi, axis=1)
    div = sum(ops.D[k] @ q[:, k] for k in range(3))
    out["D"] = np.max(np.abs(div - div_exact)) / np.max(np.abs(div_exact))
    v = A * np.cross(w[None, :], n)
    u = phi[:, None] * v
    vort_exact = 2.0 * phi * (n @ w) + np.sum(n * np.cross(gphi, v), axis=1)
    vort = sum(ops.V[k] @ u[:, k] for k in range(3))
    out["V"] = np.max(np.abs(vort - vort_exact)) / np.max(np.abs(vort_exact))
    lap = ops.L @ n[:, 2]
    out["L"] = np.max(np.abs(lap + 2 * n[:, 2] / A ** 2)) / (2 / A ** 2)
    return out


def test_operators_converge_to_continuous_limits():
    e3, e4, e5 = _errors(3), _errors(4), _errors(5)
    for k in ("G", "V", "D", "L"):
        assert e5[k] < 0.01, (k, e5[k])
        assert e4[k] < e3[k] and e5[k] < e4[k], (k, e3[k], e4[k], e5[k])
        # at least first order in dx (a factor ~2 per level)
        assert e5[k] < 0.7 * e4[k], (k, e4[k], e5[k])


def test_operators_exact_structure():
    g = build_grid(3)
    ops = build_operators(g)
    one = np.ones(g.ncells)
    # gradient and Laplacian annihilate constants (to rounding: the edge
    # interpolation weights sum to one)
    for k in range(3):
        assert np.max(np.abs(ops.G[k] @ one)) < 1e-13 / A
    assert np.max(np.abs(ops.L @ one)) < 1e-14 * abs(ops.L).max()
    # conservation: sum_i A_i (D q)_i = 0 and sum_i A_i (L psi)_i = 0
    rng = np.random.default_rng(0)
    q = rng.standard_normal((g.ncells, 3))
    div = sum(ops.D[k] @ q[:, k] for k in range(3))
    psi = rng.standard_normal(g.ncells)
    scale = np.sum(g.area * np.abs(div))
    assert abs(np.sum(g.area * div)) < 1e-13 * scale
    lap = ops.L @ psi
    assert abs(np.sum(g.area * lap)) < 1e-13 * np.sum(g.area * np.abs(lap))
    # gradient is tangent: n . G psi = 0
    grad = np.stack([ops.G[k] @ psi for k in range(3)], axis=1)
    assert np.max(np.abs(np.sum(grad * g.x, axis=1))) < 1e-12 * np.max(np.abs(grad))


def test_structural_nnz_counts_rings():
    g = build_grid(2)
    # brute force: count distinct cells within 1 and 2 edge hops per cell
    nbr = [set() for _ in range(g.ncells)]
    for i, j in zip(g.edge_i, g.edge_j):
        nbr[i].add(j)
    total = 0
    for i in range(g.ncells):
        r1 = {i} | nbr[i]
        r2 = set(r1)
        for j in nbr[i]:
            r2 |= nbr[j]
        total += 4 * (3 * len(r1) + len(r2))
    assert nnz_jacobian(g) == total
