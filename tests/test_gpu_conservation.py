"""GPU parity of the conservation diagnostics (Rossby-Haurwitz section:
total mass, total energy, potential enstrophy) and of their evolution over a
15-day run with 6 h exprb53 steps.

swe_diagnostics is compared with the oracle's sums on the same states; the
15-day run compares the diagnostics of the GPU trajectory with those of the
oracle trajectory (same scheme, Tol and decisions), and checks that mass is
conserved to rounding (flux-form divergence and Laplacian), that energy
drifts by less than the paper's 0.1 % over 15 days, and that potential
enstrophy (dissipated by the hyperdiffusion on this coarse grid) stays
within 2 %.
"""
import multiprocessing as mp
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

from oracle.phipm import PhiOpts
from oracle.schemes import KrylovPhi, step
from paper_1805_02144_gb300.inputs import balanced_state, random_vector
from parity_utils import dev, host, pair, to_oracle, to_prod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_02144_gb300 import build
    build.build()


def _oracle_diag(s, u):
    return {"mass": s.mass(u), "energy": s.energy(u), "potential_enstrophy": s.potential_enstrophy(u)}


@pytest.mark.parametrize("lev", [3, 5, 7])
def test_diagnostics_match_oracle(lev):
    from paper_1805_02144_gb300.api import swe_diagnostics
    G, s, idx = pair(lev)
    u = balanced_state(s.grid.x, 3, 400.0)
    u[:3 * s.ng] += 2.0 * random_vector(3 * s.ng, 4)     # add a rough rotational part
    got = swe_diagnostics(G, dev(to_prod(u, idx)))
    ref = _oracle_diag(s, u)
    for k in ("mass", "energy"):
        assert got[k] == pytest.approx(ref[k], rel=1e-13), k
    assert got["potential_enstrophy"] == pytest.approx(ref["potential_enstrophy"], rel=1e-11)


def test_fifteen_day_run_conservation_matches_oracle():
    from paper_1805_02144_gb300.api import SchemeState, exprb_step, swe_diagnostics
    G, s, idx = pair(4)
    dt, nsteps, tol = 6 * 3600.0, 60, 1e-8
    u = balanced_state(s.grid.x, 2, 400.0)
    phi = KrylovPhi(s, PhiOpts(tol=tol))
    st = SchemeState(G)
    ug = dev(to_prod(u, idx))
    d0_o, d0_g = _oracle_diag(s, u), swe_diagnostics(G, ug)
    for k in range(nsteps):
        u = step("exprb53", s, u, dt, phi)
        ug = exprb_step(G, "exprb53", dt, ug, state=st, opts={"tol": tol})
        if (k + 1) % 20 == 0:
            do, dg = _oracle_diag(s, u), swe_diagnostics(G, ug)
            for key in do:
                drift_o = (do[key] - d0_o[key]) / d0_o[key]
                drift_g = (dg[key] - d0_g[key]) / d0_g[key]
                assert abs(drift_g - drift_o) <= 1e-9, (k, key, drift_g, drift_o)
    assert abs(dg["mass"] - d0_g["mass"]) <= 1e-12 * d0_g["mass"]
    # energy within the paper's 0.1 %; potential enstrophy is dissipated by the
    # hyperdiffusion -nu L^2 of Eq. (eq:swdis) as it cascades to the grid scale
    # of this coarse (level-4) grid: about 1.3 % over 15 days
    assert abs(dg["energy"] - d0_g["energy"]) <= 1e-3 * d0_g["energy"]
    assert abs(dg["potential_enstrophy"] - d0_g["potential_enstrophy"]) <= 2e-2 * d0_g["potential_enstrophy"]


L6_RUNS = {
    # the paper's high-dissipation setting: stable for 15 days at 6 h steps; the
    # first 5 days (20 steps) are compared with the oracle
    "gamma_h_1.25e-2": (1.25e-2, 20),
    # the default dissipation: this grid's discrete gravity-wave modes grow (the
    # linearised operator has eigenvalues with positive real part at levels >= 4)
    # and the run blows up after about 3 days in both; the first 2 days (8
    # steps) are compared, into the growth
    "gamma_h_4e-4": (4e-4, 8),
}


@pytest.fixture(scope="module")
def level6_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle_runs as orun
    ex = ProcessPoolExecutor(max_workers=len(L6_RUNS), mp_context=mp.get_context("spawn"))
    futs = {k: ex.submit(orun.diagnostics_run, "exprb53", 6, 2, 400.0, 6 * 3600.0, n, 1e-8, gh)
            for k, (gh, n) in L6_RUNS.items()}
    yield futs
    ex.shutdown(wait=True, cancel_futures=True)


@pytest.mark.parametrize("case", list(L6_RUNS))
def test_level6_exprb53_6h_steps_match_oracle(case, level6_oracle):
    """exprb53 with 6 h steps on the level-6 grid (40,962 cells): the GPU
    trajectory and its diagnostics after every step against the oracle's."""
    from paper_1805_02144_gb300.api import Grid, SchemeState, exprb_step, swe_diagnostics
    from parity_utils import rel_l2_parts
    gh, nsteps = L6_RUNS[case]
    G = Grid(6, gamma_h=gh)
    from conftest import oracle_swe
    s = oracle_swe(6)
    idx = G.export("gen")
    u0 = balanced_state(s.grid.x, 2, 400.0)
    st = SchemeState(G)
    ug = dev(to_prod(u0, idx))
    dg = [swe_diagnostics(G, ug)]
    for k in range(nsteps):
        ug, info = exprb_step(G, "exprb53", 6 * 3600.0, ug, state=st, opts={"tol": 1e-8}, stats=True)
        assert info["status"] == 0, (k, info["status"])
        dg.append(swe_diagnostics(G, ug))
    ref, do = level6_oracle[case].result(timeout=1800)
    eh, ev = rel_l2_parts(to_oracle(host(ug), idx), ref, s.ng)
    assert eh <= 1e-10 and ev <= 1e-10, (eh, ev)
    keys = ("mass", "energy", "potential_enstrophy")
    for k in range(nsteps + 1):
        for q, key in enumerate(keys):
            drift_o = (do[k][q] - do[0][q]) / do[0][q]
            drift_g = (dg[k][key] - dg[0][key]) / dg[0][key]
            assert abs(drift_g - drift_o) <= 1e-9, (k, key, drift_g, drift_o)
        assert abs(dg[k]["mass"] - dg[0]["mass"]) <= 1e-12 * dg[0]["mass"]
    if gh > 1e-3:   # stable setting: energy within the paper's 0.1 % over the 5 days
        assert abs(dg[-1]["energy"] - dg[0]["energy"]) <= 1e-3 * dg[0]["energy"]
