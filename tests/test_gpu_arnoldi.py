"""GPU parity of wider orthogonalisation windows (phi_opts.iom > 2, up to
full Arnoldi): Algorithm 1 with the basis orthogonalised against the last
iom vectors (classical Gram-Schmidt over the window), H_m upper Hessenberg.
The oracle's IOM2Basis takes the same window; decisions must be identical.
"""
import numpy as np
import pytest

from oracle.phipm import PhiOpts, phipm_simul_iom2
from oracle.schemes import KrylovPhi, integrate
from paper_1805_02144_gb300.inputs import balanced_state, random_vector
from parity_utils import dev, host, pair, rel_l2_parts, to_oracle, to_prod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_02144_gb300 import build
    build.build()


@pytest.mark.parametrize("lev,iom", [(3, 4), (3, 64), (5, 64)])
def test_phi_action_with_wide_window_matches_oracle(lev, iom):
    from paper_1805_02144_gb300.api import phi_action
    G, s, idx = pair(lev)
    u = balanced_state(s.grid.x, 5, 400.0)
    dt = 3600.0
    v = [None, random_vector(s.n, 41), None, random_vector(s.n, 43)]
    rho = [0.5, 1.0]
    W, st = phipm_simul_iom2(lambda x: dt * s.Jv(u, x), rho, v, PhiOpts(tol=1e-8, iom=iom), s.nA)
    outs, gst = phi_action(G, dev(to_prod(u, idx)), dt, [None if x is None else dev(to_prod(x, idx)) for x in v],
                           rho, opts={"tol": 1e-8, "iom": iom}, stats=True, trace_cap=512)
    assert gst["status"] == 0
    assert [(a["m"], a["accepted"]) for a in gst["trace"]] == [(a.m, a.accepted) for a in st.trace]
    assert gst["n_jv"] == st.n_jv
    for w_ref, o in zip(W, outs):
        got = to_oracle(host(o), idx)
        assert np.linalg.norm(got - w_ref) <= 1e-10 * np.linalg.norm(w_ref)


def test_exprb53_steps_with_full_arnoldi_match_oracle():
    from paper_1805_02144_gb300.api import SchemeState, exprb_step
    G, s, idx = pair(3)
    u0 = balanced_state(s.grid.x, 2, 400.0)
    ref = integrate("exprb53", s, u0, 3600.0, 3, KrylovPhi(s, PhiOpts(tol=1e-8, iom=64)))
    st = SchemeState(G)
    u = dev(to_prod(u0, idx))
    for _ in range(3):
        u, info = exprb_step(G, "exprb53", 3600.0, u, state=st, opts={"tol": 1e-8, "iom": 64}, stats=True)
        assert info["status"] == 0
    eh, ev = rel_l2_parts(to_oracle(host(u), idx), ref, s.ng)
    assert eh <= 1e-10 and ev <= 1e-10, (eh, ev)


def test_mixed_precision_full_arnoldi_matches_oracle():
    from paper_1805_02144_gb300.api import phi_action
    G, s, idx = pair(5)
    u = balanced_state(s.grid.x, 3, 400.0)
    dt = 1800.0
    v = [None, dt * s.F(u)]
    W, _ = phipm_simul_iom2(lambda x: dt * s.Jv(u, x), [1.0], v, PhiOpts(tol=1e-10, iom=64), s.nA)
    outs = phi_action(G, dev(to_prod(u, idx)), dt, [None, dev(to_prod(v[1], idx))], [1.0],
                      opts={"precision": 1, "tol": 1e-6, "iom": 64})
    got = to_oracle(host(outs[0]), idx)
    assert np.linalg.norm(got - W[0]) <= 1e-5 * np.linalg.norm(W[0])


def test_adjoint_and_ensembles_take_iom2_only():
    from paper_1805_02144_gb300._lib import SweError
    from paper_1805_02144_gb300.api import Ensemble, Grid, SchemeState, exprb_step, exprb_step_adjoint
    G = Grid(2)
    u = dev(balanced_state(G.cell_centres(), 4, 300.0))
    u1, info = exprb_step(G, "exprb42", 900.0, u, state=SchemeState(G), stats=True, trace_cap=256)
    with pytest.raises(SweError):
        exprb_step_adjoint(G, "exprb42", 900.0, u, info["trace"], u1, opts={"iom": 64})
    with pytest.raises(SweError):
        Ensemble([G], [900.0], [1], opts={"iom": 64})
