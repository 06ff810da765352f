"""Helpers shared by the GPU parity tests: grid pairs and order conversion.

The library orders cells along a space-filling curve, the oracle in
generation order; the library's exported generation index ("gen") maps one
to the other, and the matched positions agree up to rounding.
Inputs are generated once in oracle order and permuted, so both sides see the
same numbers.
"""
import functools

import numpy as np

from conftest import oracle_swe


@functools.lru_cache(maxsize=None)
def pair(level: int):
    from paper_1805_02144_gb300.api import Grid
    G = Grid(level)
    s = oracle_swe(level)
    idx = G.export("gen")                      # grid cell k is oracle cell idx[k]
    assert np.abs(s.grid.x[idx] - G.cell_centres()).max() < 1e-14
    return G, s, idx


def to_prod(u_o: np.ndarray, idx: np.ndarray) -> np.ndarray:
    ng = idx.size
    return np.concatenate([u_o[c * ng:(c + 1) * ng][idx] for c in range(4)])


def to_oracle(u_p: np.ndarray, idx: np.ndarray) -> np.ndarray:
    ng = idx.size
    out = np.empty_like(u_p)
    for c in range(4):
        out[c * ng + idx] = u_p[c * ng:(c + 1) * ng]
    return out


def dev(x: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def host(t) -> np.ndarray:
    return t.detach().cpu().numpy()


def rel_l2_parts(a: np.ndarray, b: np.ndarray, ng: int):
    """(relative L2 error of h, of the stacked velocity components) of a vs b."""
    ha, hb = a[3 * ng:], b[3 * ng:]
    va, vb = a[:3 * ng], b[:3 * ng]
    eh = np.linalg.norm(ha - hb) / max(np.linalg.norm(hb), 1e-300)
    ev = np.linalg.norm(va - vb) / max(np.linalg.norm(vb), 1e-300)
    return eh, ev


def term_scale(s, u: np.ndarray, x: np.ndarray = None) -> float:
    """Largest sum of |terms| of F(u) (or of J(u)x) over cells and components.

    Both grids are built independently, so cell positions agree only to
    ~1e-16 and edge geometry to ~1e-16/dx relative; F and J x are sums of
    terms much larger than their result (pressure gradient of g h, flux
    divergence of u h).  Parity of one stencil evaluation is therefore
    bounded relative to this term scale, not to |F|.
    """
    A = lambda M: abs(M)
    ops = s.ops
    ux, uy, uz, h = s.split(np.abs(u))
    if x is None:
        E = 0.5 * (ux ** 2 + uy ** 2 + uz ** 2) + s.g * h
        q = [ux * h, uy * h, uz * h]
        vel = (ux, uy, uz)
        rot = (A(ops.V[0]) @ ux + A(ops.V[1]) @ uy + A(ops.V[2]) @ uz + np.abs(s.f)) * (ux + uy + uz)
    else:
        xx, xy, xz, xh = s.split(np.abs(x))
        E = ux * xx + uy * xy + uz * xz + s.g * xh
        q = [xx * h + ux * xh, xy * h + uy * xh, xz * h + uz * xh]
        vel = (xx, xy, xz)
        eta = A(ops.V[0]) @ ux + A(ops.V[1]) @ uy + A(ops.V[2]) @ uz + np.abs(s.f)
        rot = (A(ops.V[0]) @ xx + A(ops.V[1]) @ xy + A(ops.V[2]) @ xz) * (ux + uy + uz) \
            + eta * (xx + xy + xz)
    L = A(ops.L)
    diss = [s.nu * (L @ (L @ c)) for c in (*vel, h if x is None else s.split(np.abs(x))[3])]
    mom = max(np.max(A(ops.G[c]) @ E + rot + diss[c]) for c in range(3))
    cont = np.max(sum(A(ops.D[c]) @ q[c] for c in range(3)) + diss[3])
    return float(max(mom, cont))


def stencil_tol(s) -> float:
    """Relative tolerance (to term_scale) of one stencil evaluation.

    Voronoi vertices are circumcentres computed from differences of nearby
    unit vectors, so a rounding of 1e-16 in a node position moves them by
    ~1e-16 / (dx/a) and changes edge lengths by ~eps (a/dx)^2 relative, with
    (a/dx)^2 = N_g / (4 pi).  Two independently built grids therefore carry
    operator coefficients that differ by that much; 20x margin, floor 1e-13.
    """
    return max(1e-13, 20 * 1.1e-16 * s.ng / (4 * np.pi))


def abs_jacobian(s, u: np.ndarray, quad_only: bool = False):
    """Sparse matrix of the summed |terms| of J(u) (or of J(u) - J(0)).

    Entry (r, c) bounds the sum of absolute values of every product that the
    stencil adds into J_rc, so |J|^T |lam| bounds the terms of (J^T lam)_c.
    """
    import scipy.sparse as sp
    ops = s.ops
    A = abs
    ux, uy, uz, h = s.split(u)
    au = [np.abs(ux), np.abs(uy), np.abs(uz)]
    P = [np.abs(c) for c in s.cross_n(ux, uy, uz)]
    eta = sum(A(ops.V[d]) @ au[d] for d in range(3)) + (0.0 if quad_only else np.abs(s.f))
    L = A(ops.L)
    dis = None if quad_only else s.nu * (L @ L)
    dg = sp.diags
    blocks = [[None] * 4 for _ in range(4)]
    for c in range(3):
        for d in range(3):
            t = dg(P[c]) @ A(ops.V[d]) + A(ops.G[c]) @ dg(au[d])
            if c != d:
                t = t + dg(eta)
            elif dis is not None:
                t = t + dis
            blocks[c][d] = t
        blocks[c][3] = None if quad_only else s.g * A(ops.G[c])
        blocks[3][c] = A(ops.D[c]) @ dg(np.abs(h))
    hh = sum(A(ops.D[d]) @ dg(au[d]) for d in range(3))
    blocks[3][3] = hh if dis is None else hh + dis
    return sp.bmat(blocks, format="csr")
