"""Host-side checks of the CUDA library (no GPU needed).

* The library loads and exports every function declared in include/*.h.
* The library's own grid (C++ generator, space-filling-curve order) is the
  oracle's grid: the same cell centres up to rounding, the same areas, the same
  n_A, and operator tables that rebuild exactly the oracle's sparse G, D, V, L
  once cells are matched by position.
"""
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.spatial import cKDTree

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1805_02144_gb300 import build
    build.build()
    from paper_1805_02144_gb300 import _lib
    return _lib.load()


def _declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, re.M):
                if m.group(1) not in ("if", "return"):
                    names.add(m.group(1))
    return names


def test_library_exports_every_declared_function(lib):
    from paper_1805_02144_gb300 import _lib
    declared = _declared_functions()
    assert set(_lib.EXPORTS) == declared, (set(_lib.EXPORTS) ^ declared)
    for name in declared:
        assert hasattr(lib, name), name


def _match(G, og):
    d, idx = cKDTree(og.x).query(G.cell_centres())
    assert d.max() < 1e-14
    assert len(np.unique(idx)) == G.ncells
    return idx        # product cell k is oracle cell idx[k]


def _slot_matrix(nbr, coef, diag, ng):
    rows = np.concatenate([np.tile(np.arange(ng), 6), np.arange(ng)])
    cols = np.concatenate([nbr.reshape(-1), np.arange(ng)])
    vals = np.concatenate([coef.reshape(-1), diag])
    return sp.csr_matrix((vals, (rows, cols)), shape=(ng, ng))


@pytest.mark.parametrize("lev", [0, 1, 3, 4])
def test_library_grid_equals_oracle_grid(lib, lev):
    from paper_1805_02144_gb300.api import Grid
    from oracle.mesh import build_grid, build_operators, nnz_jacobian
    G = Grid(lev, host_only=True)
    og = build_grid(lev)
    ops = build_operators(og)
    idx = _match(G, og)
    P = sp.csr_matrix((np.ones(G.ncells), (np.arange(G.ncells), idx)), shape=(G.ncells, G.ncells))
    assert np.allclose(G.cell_areas(), og.area[idx], rtol=1e-12)
    assert G.nA == nnz_jacobian(og)
    nbr = G.export("nbr")
    ng = G.ncells

    def to_oracle(M):
        return P.T @ M @ P

    def close(A, B):
        d = abs(A - B).max()
        assert d <= 1e-11 * abs(B).max(), d

    close(to_oracle(_slot_matrix(nbr, G.export("wl"), G.export("wld"), ng)), ops.L)
    nc, ndd, sdg = G.export("nc"), G.export("ndd"), G.export("sdg")
    vc, vd = G.export("vc"), G.export("vd")
    nrm = G.cell_centres()
    raw = [_slot_matrix(nbr, nc[c], ndd[c] - sdg[c], ng) for c in range(3)]
    nR = sum(sp.diags(nrm[:, d]) @ raw[d] for d in range(3))
    for c in range(3):
        close(to_oracle(_slot_matrix(nbr, nc[c], ndd[c], ng)), ops.D[c])
        close(to_oracle(_slot_matrix(nbr, vc[c], vd[c], ng)), ops.V[c])
        close(to_oracle(raw[c] - sp.diags(nrm[:, c]) @ nR), ops.G[c])


@pytest.mark.parametrize("lev", [0, 2, 4])
def test_transposed_slot_tables(lib, lev):
    """The transposed tables (used by J^T) give exactly the transposed matrices."""
    from paper_1805_02144_gb300.api import Grid
    G = Grid(lev, host_only=True)
    ng = G.ncells
    nbr = G.export("nbr")
    wld, ndd, vd = G.export("wld"), G.export("ndd"), G.export("vd")

    def same(A, B):
        assert abs(A - B).max() == 0.0

    same(_slot_matrix(nbr, G.export("wlT"), wld, ng), _slot_matrix(nbr, G.export("wl"), wld, ng).T)
    nc, ncT, vc, vcT = G.export("nc"), G.export("ncT"), G.export("vc"), G.export("vcT")
    for c in range(3):
        same(_slot_matrix(nbr, ncT[c], ndd[c], ng), _slot_matrix(nbr, nc[c], ndd[c], ng).T)
        same(_slot_matrix(nbr, vcT[c], vd[c], ng), _slot_matrix(nbr, vc[c], vd[c], ng).T)
    # the pad slot of each pentagon carries no weight in either table
    pad = nbr == np.arange(ng)[None, :]
    assert pad.sum() == 12
    assert not np.any(G.export("wl")[pad]) and not np.any(G.export("wlT")[pad])


def test_hilbert_order_improves_locality(lib):
    from paper_1805_02144_gb300.api import Grid
    spread = {}
    for reorder in (False, True):
        G = Grid(5, host_only=True, reorder=reorder)
        nbr = G.export("nbr")
        spread[reorder] = np.median(np.abs(nbr - np.arange(G.ncells)[None, :]))
    assert spread[True] < 0.25 * spread[False], spread


def test_host_grid_rejects_compute_and_bad_arguments(lib):
    from paper_1805_02144_gb300 import _lib
    from paper_1805_02144_gb300.api import Grid
    import ctypes as C
    G = Grid(2, host_only=True)
    rc = lib.swe_rhs(G.handle, C.c_void_p(8), C.c_void_p(16), None)
    assert rc == -1 and b"host only" in lib.swe_last_error()
    buf = np.empty(3)
    assert lib.swe_grid_export(G.handle, b"wl", buf.ctypes.data_as(C.c_void_p), 3) == -1
    h = C.c_void_p()
    assert lib.swe_create_grid_host(11, 6.4e6, 9.8, 7e-5, 4e-4, 1, C.byref(h)) == -1
    assert lib.swe_create_grid_host(2, -1.0, 9.8, 7e-5, 4e-4, 1, C.byref(h)) == -1


@pytest.mark.parametrize("lev", [0, 1, 2, 4, 6])
def test_generation_index_is_the_oracle_order(lib, lev):
    """The exported generation index maps the grid's cells to the order in
    which refinement creates the nodes: it is a permutation and picks the
    oracle's node (built in that order) at the same position."""
    from paper_1805_02144_gb300.api import Grid
    from oracle.mesh import build_grid
    G = Grid(lev, host_only=True)
    gen = G.export("gen")
    assert np.array_equal(np.sort(gen), np.arange(G.ncells))
    og = build_grid(lev)
    assert np.abs(og.x[gen] - G.cell_centres()).max() < 1e-14
    # without reordering the grid is in generation order up to the midpoint
    # numbering of each refinement; the first 12 cells are the icosahedron
    H = Grid(lev, host_only=True, reorder=False)
    assert np.array_equal(H.export("gen")[:12], np.arange(12))
