"""GPU parity of the model variants: surface topography h_s and the
high-dissipation gamma_h = 1.25e-2 (Sec. 2 and Eq. (eq:niu)).

Fresh grids are built here (the shared parity grids stay without topography).
"""
import dataclasses

import numpy as np
import pytest

from oracle.phipm import PhiOpts
from oracle.schemes import KrylovPhi, integrate
from oracle.swe import make_swe
from paper_1805_02144_gb300.inputs import balanced_state, topography
from parity_utils import dev, host, pair, rel_l2_parts, stencil_tol, term_scale, to_oracle, to_prod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_02144_gb300 import build
    build.build()


def _topo_pair(lev):
    from paper_1805_02144_gb300.api import Grid, swe_grid_set_topography
    _, s0, idx = pair(lev)
    hs = topography(s0.grid.x, 9, 2000.0)
    s = dataclasses.replace(s0, hs=hs)
    G = Grid(lev)
    swe_grid_set_topography(G, hs[idx])
    return G, s, idx, hs


@pytest.mark.parametrize("lev", [3, 5])
def test_rhs_with_topography_matches_oracle(lev):
    from paper_1805_02144_gb300.api import swe_rhs
    G, s, idx, hs = _topo_pair(lev)
    u = balanced_state(s.grid.x, 2, 300.0)
    u[3 * s.ng:] -= hs                  # the free surface h + h_s keeps its balance
    ref = s.F(u)
    got = to_oracle(host(swe_rhs(G, dev(to_prod(u, idx)))), idx)
    scale = term_scale(s, u) + s.g * np.abs(hs).max()
    assert np.abs(got - ref).max() <= stencil_tol(s) * scale
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_exprb53_steps_with_topography_match_oracle():
    from paper_1805_02144_gb300.api import SchemeState, exprb_step
    G, s, idx, hs = _topo_pair(3)
    u0 = balanced_state(s.grid.x, 2, 300.0)
    u0[3 * s.ng:] -= hs
    ref = integrate("exprb53", s, u0, 3600.0, 2, KrylovPhi(s, PhiOpts(tol=1e-8)))
    st = SchemeState(G)
    u = dev(to_prod(u0, idx))
    for _ in range(2):
        u, info = exprb_step(G, "exprb53", 3600.0, u, state=st, opts={"tol": 1e-8}, stats=True)
        assert info["status"] == 0
    eh, ev = rel_l2_parts(to_oracle(host(u), idx), ref, s.ng)
    assert eh <= 1e-10 and ev <= 1e-10, (eh, ev)


def test_topography_can_be_removed():
    from paper_1805_02144_gb300.api import swe_grid_set_topography, swe_rhs
    G, s, idx, hs = _topo_pair(2)
    Gp, _, _ = pair(2)
    u = dev(to_prod(balanced_state(s.grid.x, 2, 300.0), idx))
    assert not np.array_equal(host(swe_rhs(G, u)), host(swe_rhs(Gp, u)))
    swe_grid_set_topography(G, None)
    assert np.array_equal(host(swe_rhs(G, u)), host(swe_rhs(Gp, u)))


def test_high_dissipation_variant_matches_oracle():
    """gamma_h = 1.25e-2 (the high-dissipation setting of Sec. 5) with exprb42."""
    from paper_1805_02144_gb300.api import Grid, SchemeState, exprb_step
    _, s0, idx = pair(3)
    s = make_swe(3, gamma_h=1.25e-2)
    G = Grid(3, gamma_h=1.25e-2)
    assert G.nu == pytest.approx(s.nu, rel=1e-14)
    u0 = balanced_state(s.grid.x, 1, 200.0)
    ref = integrate("exprb42", s, u0, 900.0, 3, KrylovPhi(s, PhiOpts(tol=1e-8)))
    st = SchemeState(G)
    u = dev(to_prod(u0, idx))
    for _ in range(3):
        u, info = exprb_step(G, "exprb42", 900.0, u, state=st, opts={"tol": 1e-8}, stats=True)
        assert info["status"] == 0
    eh, ev = rel_l2_parts(to_oracle(host(u), idx), ref, s.ng)
    assert eh <= 1e-10 and ev <= 1e-10, (eh, ev)
