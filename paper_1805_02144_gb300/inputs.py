"""Seeded synthetic inputs: balanced shallow-water states on any cell set.

This module holds no arithmetic of the time-stepping method.  It maps cell
centre positions (unit vectors, in whatever cell order the caller uses) and a
seed to a state vector u = (u_x, u_y, u_z, h) (the planar layout of
Eq. (eq:dynu)), so that the CUDA library and the CPU oracle receive the same
input although each builds its own grid.

Height: h = h0 + h', h0 = 5960 m, with

    h'(n) = amp * sum_i A_i Re(e^{i alpha_i} (x + i y)^{k_i}) cos(l_i pi z + beta_i),
                                                     i = 1..8

divided by the maximum of |sum_i ...| over a fixed 1-degree latitude-longitude
sample of the sphere (so max |h'| is amp up to the sampling, whatever the
grid).  n = (x, y, z) is the unit position, k_i in {0..4}, l_i in {1..4},
alpha_i, beta_i ~ U[0, 2 pi), A_i ~ U[-1, 1].  On the sphere (x + i y)^k equals
cos^k(lat) e^{i k lon}, so each term is a smooth low-wavenumber lon/lat
sinusoid with no pole singularity.

Velocity: geostrophic balance u = (g / f0) n x grad_s h' with f0 = 2 Omega
(the balance with f = 2 Omega sin(lat) is singular at the equator); grad_s is
the exact tangential gradient of the formula above at the cell centre.
"""
from __future__ import annotations

import numpy as np

H0 = 5960.0
NTERMS = 8


def _params(seed: int):
    rng = np.random.Generator(np.random.PCG64(seed))
    k = rng.integers(0, 5, size=NTERMS)
    l = rng.integers(1, 5, size=NTERMS)
    alpha = rng.uniform(0.0, 2.0 * np.pi, size=NTERMS)
    beta = rng.uniform(0.0, 2.0 * np.pi, size=NTERMS)
    amp = rng.uniform(-1.0, 1.0, size=NTERMS)
    return k, l, alpha, beta, amp


def _sample_points() -> np.ndarray:
    lat = np.deg2rad(np.arange(-90.0, 90.5, 1.0))
    lon = np.deg2rad(np.arange(0.0, 360.0, 1.0))
    la, lo = np.meshgrid(lat, lon, indexing="ij")
    return np.stack([np.cos(la) * np.cos(lo), np.cos(la) * np.sin(lo), np.sin(la)],
                    axis=-1).reshape(-1, 3)


def _raw_sum(xyz: np.ndarray, seed: int):
    """Un-normalised sum of the eight terms and its Cartesian gradient."""
    xyz = np.asarray(xyz, dtype=np.float64)
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    k, l, alpha, beta, amp = _params(seed)
    w = x + 1j * y
    hp = np.zeros_like(x)
    grad = np.zeros_like(xyz)
    for i in range(NTERMS):
        rot = np.exp(1j * alpha[i])
        horiz = np.real(rot * w ** k[i])
        # d/dx (x+iy)^k = k (x+iy)^(k-1); d/dy = i k (x+iy)^(k-1)
        dw = k[i] * w ** (k[i] - 1) if k[i] > 0 else np.zeros_like(w)
        dhx = np.real(rot * dw)
        dhy = np.real(rot * 1j * dw)
        arg = l[i] * np.pi * z + beta[i]
        vert = np.cos(arg)
        dvert = -l[i] * np.pi * np.sin(arg)
        hp += amp[i] * horiz * vert
        grad[:, 0] += amp[i] * dhx * vert
        grad[:, 1] += amp[i] * dhy * vert
        grad[:, 2] += amp[i] * horiz * dvert
    return hp, grad


def height_perturbation(xyz: np.ndarray, seed: int, amplitude: float):
    """h'(n) and its Cartesian gradient d h'/d(x, y, z) on the unit sphere."""
    hp, grad = _raw_sum(xyz, seed)
    ref, _ = _raw_sum(_sample_points(), seed)
    scale = amplitude / np.max(np.abs(ref))
    return hp * scale, grad * scale


def balanced_state(xyz: np.ndarray, seed: int, amplitude: float,
                   radius: float = 6.37122e6, g: float = 9.80616,
                   omega: float = 7.292e-5) -> np.ndarray:
    """State u = (u_x, u_y, u_z, h) of length 4 N_g for cell centres ``xyz`` (N_g x 3)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    hp, grad = height_perturbation(xyz, seed, amplitude)
    # tangential gradient on the sphere of radius a: (I - n n^T) grad / a
    radial = np.sum(grad * xyz, axis=1, keepdims=True)
    gs = (grad - radial * xyz) / radius
    f0 = 2.0 * omega
    vel = (g / f0) * np.cross(xyz, gs)
    return np.concatenate([vel[:, 0], vel[:, 1], vel[:, 2], H0 + hp])


def random_vector(n: int, seed: int) -> np.ndarray:
    """A seeded standard-normal vector (test directions, Krylov inputs)."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(n)


def ensemble_config(seed: int = 4, nmem: int = 64, levels=(5, 6, 7), dts=(900.0, 1800.0, 3600.0),
                    horizon: float = 6 * 3600.0) -> list:
    """Seeded ensemble members: level, dt, steps over the horizon, amplitude, seed.

    Each member draws its grid level and time step uniformly from the given
    sets and its perturbation amplitude from U[50, 400] m; nsteps = horizon/dt.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for m in range(nmem):
        lev = int(rng.choice(levels))
        dt = float(rng.choice(dts))
        amp = float(rng.uniform(50.0, 400.0))
        out.append({"level": lev, "dt": dt, "nsteps": int(round(horizon / dt)), "amplitude": amp,
                    "seed": 1000 * seed + m})
    return out


def observation_network(xyz: np.ndarray, nobs: int = 1000, seed: int = 7, sigma: float = 5.0,
                        truth_seed: int = 8, truth_amplitude: float = 400.0, h_truth=None):
    """Synthetic height observations for the adjoint misfit.

    Cells: the cell nearest to each of a seeded sequence of uniformly random
    unit vectors, duplicates dropped, until ``nobs`` distinct cells are found
    (so the set depends on positions only, not on the cell order).
    Values: the truth height at those cells plus Gaussian noise of standard
    deviation ``sigma`` [m].  The truth is ``h_truth`` (heights of all cells
    in the caller's order, e.g. a truth forecast at the observation time) or,
    when it is None, the height of the balanced state ``truth_seed``.
    Returns (cells, y, sigma) with cells indexing the caller's order.
    """
    ng = xyz.shape[0]
    if not 0 < nobs <= ng:
        raise ValueError("need 0 < nobs <= number of cells")
    rng = np.random.Generator(np.random.PCG64(seed))
    cells: list = []
    seen = set()
    while len(cells) < nobs:
        d = rng.normal(size=(nobs, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        for c in _nearest(xyz, d):
            if int(c) not in seen:
                seen.add(int(c))
                cells.append(int(c))
                if len(cells) == nobs:
                    break
    cells = np.asarray(cells, dtype=np.int64)
    if h_truth is None:
        h_obs = H0 + height_perturbation(xyz[cells], truth_seed, truth_amplitude)[0]
    else:
        h_obs = np.asarray(h_truth, dtype=np.float64)[cells]
    noise = np.random.Generator(np.random.PCG64(seed + 1)).normal(size=nobs)
    return cells, h_obs + sigma * noise, sigma


def fd_directions(u0: np.ndarray, k: int = 8, seed: int = 11, rel: float = 1e-6):
    """k seeded standard-normal directions d_i for central differences of a
    function of u0, each with its step eps_i = rel * ||u0|| / ||d_i||."""
    out = []
    for i in range(k):
        d = random_vector(u0.size, seed + i)
        out.append((d, rel * float(np.linalg.norm(u0)) / float(np.linalg.norm(d))))
    return out


def _nearest(xyz: np.ndarray, d: np.ndarray) -> np.ndarray:
    out = np.empty(d.shape[0], dtype=np.int64)
    for a in range(0, d.shape[0], 64):
        out[a:a + 64] = np.argmax(d[a:a + 64] @ xyz.T, axis=1)
    return out


def topography(xyz: np.ndarray, seed: int = 9, height: float = 2000.0) -> np.ndarray:
    """A smooth seeded surface height h_s in [0, height] [m]: (height + h') / 2
    with h' the sinusoid sum above (amplitude ``height``, seed ``seed``)."""
    hp, _ = height_perturbation(np.asarray(xyz, dtype=np.float64), seed, height)
    return 0.5 * (height + hp)
