"""GPU parity of the ensemble launch (batching): swe_ensemble_*.

Every member of one persistent launch must reproduce its own exprb42
trajectory: against the FP64 oracle on small grids (1e-10 relative L2 in h
and velocity, increments 1e-8) and against the single-trajectory GPU path on
the full 64-member, levels 5/6/7, 6 h ensemble.  Tuning must not change the
results, and the run must replay identically from a captured CUDA graph.
"""
import numpy as np
import pytest

from oracle.phipm import PhiOpts
from oracle.schemes import KrylovPhi, integrate
from paper_1805_02144_gb300.inputs import balanced_state, ensemble_config
from parity_utils import dev, host, pair, rel_l2_parts, to_oracle, to_prod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_02144_gb300 import build
    build.build()


def _sequential(G, u0, dt, nsteps):
    from paper_1805_02144_gb300.api import SchemeState, exprb_step
    st = SchemeState(G)
    u = u0.clone()
    for _ in range(nsteps):
        u = exprb_step(G, "exprb42", dt, u, state=st)
    return u


def test_small_ensemble_matches_oracle_per_member():
    from paper_1805_02144_gb300.api import Ensemble
    members = [(2, 900.0, 3, 120.0), (3, 1800.0, 2, 300.0), (4, 3600.0, 2, 400.0), (3, 900.0, 4, 50.0)]
    grids, states, refs = [], [], []
    for k, (lev, dt, ns, amp) in enumerate(members):
        G, s, idx = pair(lev)
        u0 = balanced_state(s.grid.x, 20 + k, amp)
        refs.append((s, idx, u0, integrate("exprb42", s, u0, dt, ns, KrylovPhi(s, PhiOpts(tol=1e-8)))))
        grids.append(G)
        states.append(dev(to_prod(u0, idx)))
    E = Ensemble(grids, [m[1] for m in members], [m[2] for m in members], opts={"tol": 1e-8})
    for k, u in enumerate(states):
        E.set_state(k, u)
    E.run()
    st = E.stats()
    assert all(x == 0 for x in st["status"]), st
    for k, (s, idx, u0, ref) in enumerate(refs):
        got = to_oracle(host(E.get_state(k)), idx)
        eh, ev = rel_l2_parts(got, ref, s.ng)
        assert eh <= 1e-10 and ev <= 1e-10, (k, eh, ev)
        assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref - u0)


def _full_ensemble():
    import torch
    from paper_1805_02144_gb300.api import Ensemble, Grid
    cfg = ensemble_config()
    grids = {lev: Grid(lev) for lev in sorted({c["level"] for c in cfg})}
    gl = [grids[c["level"]] for c in cfg]
    u0 = [torch.from_numpy(balanced_state(g.cell_centres(), c["seed"], c["amplitude"])).cuda()
          for g, c in zip(gl, cfg)]
    E = Ensemble(gl, [c["dt"] for c in cfg], [c["nsteps"] for c in cfg], opts={"tol": 1e-8})
    return cfg, gl, u0, E


def test_full_ensemble_matches_single_trajectories_tuned_and_graphed():
    import torch
    cfg, gl, u0, E = _full_ensemble()
    assert {c["level"] for c in cfg} == {5, 6, 7}
    assert {c["dt"] for c in cfg} == {900.0, 1800.0, 3600.0}
    for m, u in enumerate(u0):
        E.set_state(m, u)
    E.tune(rounds=2)                       # states restored afterwards
    st = E.stats()
    assert all(x == 0 for x in st["status"])
    assert sum(st["blocks"]) > 0 and min(st["blocks"]) >= 1
    # the tuned launch is one of the shapes; every member is in exactly one
    # group, a group's members share its block count, the groups fit the launch
    sh = E.shape()
    assert (sh["threads"], sh["blocks_per_sm"]) in {(96, 4), (128, 3), (192, 2), (384, 1)}
    mg = sh["member_group"]
    assert sorted(set(mg)) == list(range(sh["groups"]))
    nbg = {}
    for m, g in enumerate(mg):
        assert nbg.setdefault(g, st["blocks"][m]) == st["blocks"][m]
    assert sum(nbg.values()) == sh["nblocks"] <= 152 * sh["blocks_per_sm"]
    # eager run (fresh trajectories: no Krylov size carried from the tuning runs)
    E.reset()
    E.run()
    torch.cuda.synchronize()
    eager = [E.get_state(m).clone() for m in range(len(cfg))]
    assert all(x == 0 for x in E.stats()["status"])
    # the same run captured in a CUDA graph and replayed
    for m, u in enumerate(u0):
        E.set_state(m, u)
    E.reset()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            E.run(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for m, u in enumerate(u0):
        E.set_state(m, u)
    E.reset()
    g.replay()
    torch.cuda.synchronize()
    for m in range(len(cfg)):
        assert torch.equal(E.get_state(m), eager[m]), m
    # each member against its own single-trajectory run
    for m, (G, c) in enumerate(zip(gl, cfg)):
        ref = _sequential(G, u0[m], c["dt"], c["nsteps"])
        eh, ev = rel_l2_parts(host(eager[m]), host(ref), G.ncells)
        assert eh <= 1e-10 and ev <= 1e-10, (m, c, eh, ev)
