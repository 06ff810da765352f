"""Icosahedral geodesic Voronoi grid and the finite-volume operators (oracle).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``): never used by the product path.

Sec. 2 of the paper discretises the shallow-water equations by a finite-volume
method on control volumes around the nodes of a geodesic grid of level l with
N_g = 10 * 2^(2l) + 2 nodes (Sec. 2, after Eq. (eq:niu)), and writes the
discrete operators as sparse matrices G_x, G_y, G_z (gradient), D_x, D_y, D_z
(divergence), V_x, V_y, V_z (normal vorticity) and L (Laplacian)
(Eqs. (eq:sweqsinv), (eq:vort), (eq:swdis)).  The paper delegates the exact mesh
and operator construction to an earlier work that is not available here, so
this module fixes one concrete definition and states it in full:

Mesh
  * level 0: the regular icosahedron with vertices at the two poles and two
    rings of five at latitude +-atan(1/2), the southern ring rotated by 36 deg;
  * level l -> l+1: every triangle is split in four by its edge midpoints,
    each midpoint being (a+b)/|a+b| (bisection on the unit sphere);
  * cells are the spherical Voronoi regions of the nodes; the Voronoi vertices
    are the triangle circumcentres (b-a)x(c-a)/|(b-a)x(c-a)| (CCW triangles).

Per directed edge e = (i -> j), with c1, c2 the Voronoi-edge endpoints:
  * l_e  = a * arc(c1, c2)                 (Voronoi edge length)
  * d_e  = a * arc(x_i, x_j)               (node separation)
  * m_e  = (c1 + c2)/|c1 + c2|             (Voronoi edge midpoint)
  * nu_e = (x_j - x_i)/|x_j - x_i|         (unit outward normal, tangent at m_e
                                            because the Voronoi edge lies on the
                                            bisecting great circle of x_i, x_j)
  * t_e  = m_e x nu_e                      (counter-clockwise edge tangent)
  * A_i  = a^2 * sum of the spherical triangles (x_i, c1, c2) over the cell's
           edges, each by the Oosterom-Strackee formula
           E = 2 atan2(|x.(y x z)|, 1 + x.y + y.z + z.x)

Edge values: the trapezoid rule along the Voronoi edge,
    psi_e = (psi(c1) + psi(c2)) / 2,   psi(c) = sum_{v in T(c)} lambda_v psi_v,
where T(c) is the Delaunay triangle whose circumcentre is c and lambda are the
barycentric coordinates of the circumcentre of the flat triangle through its
three nodes (that point lies on the ray through c):
    lambda_a ~ |b-c|^2 (|c-a|^2 + |a-b|^2 - |b-c|^2), and cyclically.
On a bisection mesh the Voronoi edge is not cut in its middle by the Delaunay
edge, so the plain average (psi_i + psi_j)/2 makes the Green-Gauss gradient
inconsistent (an O(1) error that does not shrink under refinement); the
trapezoid rule is exact for linear fields and keeps the one-ring stencil.

Operators (P_i = I - n_i n_i^T):
  * (G psi)_i = P_i (1/A_i) sum_e l_e nu_e (psi_e - psi_i)
  * (D . q)_i = (1/A_i) sum_e l_e nu_e . q_e                      (flux form)
  * (V . u)_i = (1/A_i) sum_e l_e t_e  . u_e                      (circulation)
  * (L psi)_i = (1/A_i) sum_e (l_e/d_e)(psi_j - psi_i)

These follow Gauss' and Stokes' theorems on each control volume.  Mass
conservation is structural: the flux of D and L through an edge is the same
number seen from both cells, with opposite normals.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

# ---------------------------------------------------------------------------
# geometry helpers (unit sphere)
# ---------------------------------------------------------------------------


def _normalize(v: np.ndarray) -> np.ndarray:
    return v / np.sqrt(np.sum(v * v, axis=-1, keepdims=True))


def _arc(p: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Great-circle angle between unit vectors, the well-conditioned atan2 form."""
    return np.arctan2(np.linalg.norm(np.cross(p, q), axis=-1), np.sum(p * q, axis=-1))


def _spherical_triangle_area(x: np.ndarray, y: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Area (solid angle) of the spherical triangle x, y, z (Oosterom-Strackee)."""
    num = np.abs(np.sum(x * np.cross(y, z), axis=-1))
    den = 1.0 + np.sum(x * y, axis=-1) + np.sum(y * z, axis=-1) + np.sum(z * x, axis=-1)
    return 2.0 * np.arctan2(num, den)


def icosahedron() -> tuple[np.ndarray, np.ndarray]:
    """Level-0 nodes (12 x 3, unit vectors) and faces (20 x 3, CCW from outside)."""
    s = 1.0 / np.sqrt(5.0)          # sin(atan(1/2))
    c = 2.0 / np.sqrt(5.0)          # cos(atan(1/2))
    pts = [(0.0, 0.0, 1.0)]
    for k in range(5):
        lon = 2.0 * np.pi * k / 5.0
        pts.append((c * np.cos(lon), c * np.sin(lon), s))
    for k in range(5):
        lon = 2.0 * np.pi * k / 5.0 + np.pi / 5.0
        pts.append((c * np.cos(lon), c * np.sin(lon), -s))
    pts.append((0.0, 0.0, -1.0))
    x = np.array(pts, dtype=np.float64)
    faces = []
    for k in range(5):
        k1 = (k + 1) % 5
        faces.append((0, 1 + k, 1 + k1))            # northern cap
        faces.append((1 + k, 6 + k, 1 + k1))        # upper band
        faces.append((1 + k1, 6 + k, 6 + k1))       # lower band
        faces.append((11, 6 + k1, 6 + k))           # southern cap
    f = np.array(faces, dtype=np.int64)
    return x, _orient_ccw(x, f)


def _orient_ccw(x: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Reorder each face so that (b-a)x(c-a) points away from the origin."""
    a, b, c = x[f[:, 0]], x[f[:, 1]], x[f[:, 2]]
    s = np.sum(np.cross(b - a, c - a) * (a + b + c), axis=-1)
    f = f.copy()
    flip = s < 0
    f[flip, 1], f[flip, 2] = f[flip, 2].copy(), f[flip, 1].copy()
    return f


def bisect(x: np.ndarray, f: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """One refinement: split every triangle in four at its normalised edge midpoints."""
    nv = x.shape[0]
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
    key = np.sort(e, axis=1)
    uniq, inv = np.unique(key, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    mid = _normalize(x[uniq[:, 0]] + x[uniq[:, 1]])
    nf = f.shape[0]
    m01 = nv + inv[0:nf]
    m12 = nv + inv[nf:2 * nf]
    m20 = nv + inv[2 * nf:3 * nf]
    a, b, c = f[:, 0], f[:, 1], f[:, 2]
    children = np.concatenate([
        np.stack([a, m01, m20], axis=1),
        np.stack([m01, b, m12], axis=1),
        np.stack([m20, m12, c], axis=1),
        np.stack([m01, m12, m20], axis=1),
    ], axis=0)
    return np.concatenate([x, mid], axis=0), children


# ---------------------------------------------------------------------------
# grid
# ---------------------------------------------------------------------------


@dataclasses.dataclass
class Grid:
    """Voronoi finite-volume grid of one level, in generation order."""

    level: int
    radius: float
    x: np.ndarray            # (N_g, 3) unit cell centres n_i
    faces: np.ndarray        # (T, 3) Delaunay triangles (CCW)
    area: np.ndarray         # (N_g,) cell areas A_i [m^2]
    edge_i: np.ndarray       # (2E,) directed edge source cell
    edge_j: np.ndarray       # (2E,) directed edge target cell
    le: np.ndarray           # (2E,) Voronoi edge length l_e [m]
    de: np.ndarray           # (2E,) node separation d_e [m]
    nu: np.ndarray           # (2E, 3) unit outward normal nu_e
    te: np.ndarray           # (2E, 3) edge tangent t_e = m_e x nu_e
    # edge-value interpolation psi_e = sum_k ew[e, k] psi[en[e, k]] (6 terms:
    # three nodes of each of the two triangles, already halved)
    en: np.ndarray           # (2E, 6) node indices
    ew: np.ndarray           # (2E, 6) weights

    @property
    def ncells(self) -> int:
        return self.x.shape[0]

    @property
    def n(self) -> int:
        """Length of the state vector u = (u_x, u_y, u_z, h), Eq. (eq:dynu)."""
        return 4 * self.ncells

    def degree(self) -> np.ndarray:
        return np.bincount(self.edge_i, minlength=self.ncells)


def build_grid(level: int, radius: float = 6.37122e6) -> Grid:
    """Build the level-``level`` grid defined in the module docstring."""
    x, f = icosahedron()
    for _ in range(level):
        x, f = bisect(x, f)
    ng = x.shape[0]
    a, b, c = x[f[:, 0]], x[f[:, 1]], x[f[:, 2]]
    cc = _normalize(np.cross(b - a, c - a))          # circumcentres (outward)

    # Each CCW triangle (p, q, r) lies to the left of its directed edges
    # p->q, q->r, r->p.  The Voronoi edge dual to {i, j} joins the circumcentres
    # of the triangles left of i->j and left of j->i.
    src = np.concatenate([f[:, 0], f[:, 1], f[:, 2]])
    dst = np.concatenate([f[:, 1], f[:, 2], f[:, 0]])
    tri = np.tile(np.arange(f.shape[0]), 3)
    order = np.lexsort((dst, src))
    src, dst, tri = src[order], dst[order], tri[order]
    # partner of each directed edge (j -> i)
    # Sorting the edges by (dst, src) lists the reversed pairs (d, s) in the
    # same lexicographic order as the (s, d) list, so the k-th entry of that
    # permutation is the index of the reverse of edge k.
    partner = np.lexsort((src, dst))
    # sanity: partner maps (s,d) to (d,s)
    if not (np.all(src[partner] == dst) and np.all(dst[partner] == src)):
        raise RuntimeError("mesh is not a closed manifold triangulation")
    c_left = cc[tri]                                  # left of i->j
    c_right = cc[tri[partner]]                        # left of j->i
    xi, xj = x[src], x[dst]

    le = radius * _arc(c_left, c_right)
    de = radius * _arc(xi, xj)
    me = _normalize(c_left + c_right)
    nu = _normalize(xj - xi)
    te = np.cross(me, nu)
    tri_area = _spherical_triangle_area(xi, c_left, c_right)
    area = radius * radius * np.bincount(src, weights=tri_area, minlength=ng)
    lam = _circumcentre_barycentric(a, b, c)         # (T, 3)
    t_l, t_r = tri, tri[partner]
    en = np.concatenate([f[t_l], f[t_r]], axis=1)
    ew = 0.5 * np.concatenate([lam[t_l], lam[t_r]], axis=1)
    return Grid(level=level, radius=radius, x=x, faces=f, area=area,
                edge_i=src, edge_j=dst, le=le, de=de, nu=nu, te=te, en=en, ew=ew)


def _circumcentre_barycentric(a: np.ndarray, b: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Barycentric coordinates of the circumcentre of the flat triangle a, b, c."""
    la = np.sum((b - c) ** 2, axis=-1)
    lb = np.sum((c - a) ** 2, axis=-1)
    lc = np.sum((a - b) ** 2, axis=-1)
    w = np.stack([la * (lb + lc - la), lb * (lc + la - lb), lc * (la + lb - lc)], axis=-1)
    return w / np.sum(w, axis=-1, keepdims=True)


# ---------------------------------------------------------------------------
# sparse operators
# ---------------------------------------------------------------------------


@dataclasses.dataclass
class Operators:
    """The sparse N_g x N_g matrices of Eqs. (eq:sweqsinv), (eq:vort), (eq:swdis)."""

    G: tuple[sp.csr_matrix, sp.csr_matrix, sp.csr_matrix]
    D: tuple[sp.csr_matrix, sp.csr_matrix, sp.csr_matrix]
    V: tuple[sp.csr_matrix, sp.csr_matrix, sp.csr_matrix]
    L: sp.csr_matrix


def _edge_value_operator(g: Grid, w: np.ndarray, minus_self: bool) -> sp.csr_matrix:
    """Sparse M with (M psi)_i = sum_e w_e (psi_e [- psi_i]), psi_e interpolated."""
    ng = g.ncells
    rows = np.repeat(g.edge_i, 6)
    cols = g.en.reshape(-1)
    vals = (w[:, None] * g.ew).reshape(-1)
    if minus_self:
        rows = np.concatenate([rows, g.edge_i])
        cols = np.concatenate([cols, g.edge_i])
        vals = np.concatenate([vals, -w])
    return sp.csr_matrix((vals, (rows, cols)), shape=(ng, ng))


def build_operators(g: Grid) -> Operators:
    inva = 1.0 / g.area[g.edge_i]
    # raw gradient R_c psi = (1/A) sum l nu_c (psi_e - psi_i), then G = P R
    R = [_edge_value_operator(g, g.le * g.nu[:, c] * inva, True) for c in range(3)]
    n = g.x
    nR = sum(sp.diags(n[:, d]) @ R[d] for d in range(3))       # n . R
    G = tuple((R[c] - sp.diags(n[:, c]) @ nR).tocsr() for c in range(3))
    D = tuple(_edge_value_operator(g, g.le * g.nu[:, c] * inva, False) for c in range(3))
    V = tuple(_edge_value_operator(g, g.le * g.te[:, c] * inva, False) for c in range(3))
    ng = g.ncells
    wl = g.le / g.de * inva
    L = sp.csr_matrix((np.concatenate([wl, -wl]),
                       (np.concatenate([g.edge_i, g.edge_i]), np.concatenate([g.edge_j, g.edge_i]))),
                      shape=(ng, ng))
    return Operators(G=G, D=D, V=V, L=L)


def nnz_jacobian(g: Grid) -> int:
    """Structural number of nonzeros n_A of J (used by the cost of Eq. (eq:cost)).

    A momentum row of cell i couples to all four variables on the one-ring
    R1(i) (cell plus neighbours: V, G and the rotation terms) and to its own
    component on the two-ring R2(i) (the L^2 dissipation); the continuity row
    likewise.  So the count per cell is 4 * (3 |R1(i)| + |R2(i)|).
    """
    ng = g.ncells
    adj = sp.csr_matrix((np.ones(g.edge_i.size), (g.edge_i, g.edge_j)), shape=(ng, ng))
    one = sp.identity(ng, format="csr") + adj
    r1 = np.diff(one.indptr)
    two = (one @ one).tocsr()
    r2 = np.diff(two.indptr)
    return int(np.sum(4 * (3 * r1 + r2)))
