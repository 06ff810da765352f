"""GPU parity: the CUDA library through its C ABI against the FP64 oracle.

Tolerances: F and J x are single FP64 stencil evaluations on two
independently built grids whose operator coefficients differ by
~eps (a/dx)^2 relative (circumcentre conditioning); they must agree within
parity_utils.stencil_tol of the largest sum of |terms| (term_scale), and
within 1e-10 in relative L2.  phi_action and exprb_step are compared within 1e-10 relative L2
in h and in the stacked velocity, and the increments u_{n+1} - u_n (the part
the schemes compute) within 1e-8 relative; the controller decisions (Krylov
sizes, accept/reject sequence) must be identical.
"""
import numpy as np
import pytest

from oracle.phipm import PhiOpts, phipm_simul_iom2
from oracle.schemes import KrylovPhi, integrate, step
from paper_1805_02144_gb300.inputs import balanced_state, random_vector
from parity_utils import (dev, host, pair, rel_l2_parts, stencil_tol, term_scale, to_oracle,
                          to_prod)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_02144_gb300 import build
    build.build()


def _state(s, seed, amp):
    return balanced_state(s.grid.x, seed, amp)


@pytest.mark.parametrize("lev", [0, 3, 5, 7])
def test_rhs_matches_oracle(lev):
    from paper_1805_02144_gb300.api import swe_rhs
    G, s, idx = pair(lev)
    u = _state(s, 2, 400.0)
    ref = s.F(u)
    got = to_oracle(host(swe_rhs(G, dev(to_prod(u, idx)))), idx)
    assert np.abs(got - ref).max() <= stencil_tol(s) * term_scale(s, u)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("lev", [0, 3, 5, 7])
def test_jv_matches_oracle(lev):
    from paper_1805_02144_gb300.api import swe_jv
    G, s, idx = pair(lev)
    u = _state(s, 3, 400.0)
    x = random_vector(s.n, 11)
    ref = s.Jv(u, x)
    got = to_oracle(host(swe_jv(G, dev(to_prod(u, idx)), dev(to_prod(x, idx)))), idx)
    assert np.abs(got - ref).max() <= stencil_tol(s) * term_scale(s, u, x)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def _phi_case(lev, dt, pattern, rho, tol, seed=5):
    from paper_1805_02144_gb300.api import phi_action
    G, s, idx = pair(lev)
    u = _state(s, seed, 400.0)
    v = [None if not on else random_vector(s.n, 40 + i) for i, on in enumerate(pattern)]
    opts = PhiOpts(tol=tol)
    W, st = phipm_simul_iom2(lambda x: dt * s.Jv(u, x), rho, v, opts, s.nA)
    outs, gst = phi_action(G, dev(to_prod(u, idx)), dt,
                           [None if x is None else dev(to_prod(x, idx)) for x in v], rho,
                           opts={"tol": tol}, stats=True, trace_cap=512)
    return G, s, idx, W, st, outs, gst


@pytest.mark.parametrize("pattern,rho", [
    ((0, 1), [0.75]),
    ((0, 1), [0.5, 0.9]),
    ((0, 0, 0, 1), [0.5, 0.9]),
    ((0, 1, 0, 1), [1.0]),
    ((0, 0, 0, 1, 1), [1.0]),
    ((0, 1, 0, 1, 1), [1.0]),
    ((1, 1, 1), [0.3, 1.0]),
])
@pytest.mark.parametrize("tol", [1e-8, 1e-12])
def test_phi_action_matches_oracle(pattern, rho, tol):
    G, s, idx, W, st, outs, gst = _phi_case(3, 3600.0, pattern, rho, tol)
    assert gst["status"] == 0
    gm = [(a["m"], a["accepted"]) for a in gst["trace"]]
    om = [(a.m, a.accepted) for a in st.trace]
    assert gm == om
    assert gst["n_jv"] == st.n_jv and gst["n_substeps"] == st.n_substeps
    for w_ref, o in zip(W, outs):
        got = to_oracle(host(o), idx)
        assert np.linalg.norm(got - w_ref) <= 1e-10 * np.linalg.norm(w_ref)


def test_phi_action_level5_long_step():
    G, s, idx, W, st, outs, gst = _phi_case(5, 3600.0, (0, 1, 0, 1, 1), [1.0], 1e-8)
    assert [(a["m"], a["accepted"]) for a in gst["trace"]] == [(a.m, a.accepted) for a in st.trace]
    got = to_oracle(host(outs[0]), idx)
    assert np.linalg.norm(got - W[0]) <= 1e-10 * np.linalg.norm(W[0])


def test_phi_action_zero_inputs_and_replay():
    from paper_1805_02144_gb300.api import phi_action
    G, s, idx = pair(3)
    u = _state(s, 1, 200.0)
    import torch
    z = torch.zeros(G.n, dtype=torch.float64, device="cuda")
    outs = phi_action(G, dev(to_prod(u, idx)), 900.0, [None, z], [0.5, 1.0])
    assert all(float(o.abs().max()) == 0.0 for o in outs)
    # replaying the oracle's decisions reproduces its substep partition exactly
    x = random_vector(s.n, 3)
    forced = [(0.25, 12, 1), (0.25, 12, 1), (0.5, 20, 1)]
    from oracle.phipm import Attempt
    trace = [Attempt(t=0, tau=a, m=b, omega=0, accepted=bool(c)) for a, b, c in forced]
    W, st = phipm_simul_iom2(lambda y: 900.0 * s.Jv(u, y), [1.0], [None, x], PhiOpts(), s.nA,
                             replay=trace)
    outs, gst = phi_action(G, dev(to_prod(u, idx)), 900.0, [None, dev(to_prod(x, idx))], [1.0],
                           opts={"replay": forced}, stats=True, trace_cap=16)
    assert [(round(a["tau"], 12), a["m"]) for a in gst["trace"]] == [(0.25, 12), (0.25, 12), (0.5, 20)]
    assert gst["n_jv"] == st.n_jv
    got = to_oracle(host(outs[0]), idx)
    assert np.linalg.norm(got - W[0]) <= 1e-11 * np.linalg.norm(W[0])


def test_phi_action_reports_no_convergence():
    from paper_1805_02144_gb300.api import phi_action
    G, s, idx = pair(3)
    u = _state(s, 1, 200.0)
    x = random_vector(s.n, 3)
    outs, gst = phi_action(G, dev(to_prod(u, idx)), 3600.0, [None, dev(to_prod(x, idx))], [1.0],
                           opts={"tol": 1e-30, "max_reject": 3, "m_max": 4}, stats=True)
    assert gst["status"] == -3      # SWE_ERR_NOCONV, reported without a device fault
    # the grid stays usable
    outs, gst = phi_action(G, dev(to_prod(u, idx)), 900.0, [None, dev(to_prod(x, idx))], [1.0],
                           stats=True)
    assert gst["status"] == 0


@pytest.mark.parametrize("case", ["substeps", "exponent"])
def test_phi_action_bounds_end_runaway_calls(case):
    """A call that would need more than max_substeps accepted substeps ends
    with NOCONV like the oracle's NoConvergence under the same option.  An
    augmented matrix with ||tau Hhat||_1 beyond 4096 (dt = 1e9 s, a step size
    gone wrong) exceeds what the device's scaled Taylor exponential accepts
    (1024 scaling steps): the device ends the call with NOCONV on its own
    terms (the oracle has no such bound).  The grid stays usable."""
    from oracle.phipm import NoConvergence
    from paper_1805_02144_gb300.api import phi_action
    G, s, idx = pair(3)
    u = _state(s, 1, 200.0)
    x = random_vector(s.n, 3)
    if case == "substeps":
        dt, gopts = 3600.0, {"max_substeps": 1, "m_max": 4}
        with pytest.raises(NoConvergence):
            phipm_simul_iom2(lambda y: dt * s.Jv(u, y), [1.0], [None, x], PhiOpts(max_substeps=1, m_max=4),
                             s.nA)
    else:
        dt, gopts = 1e9, {}
    outs, gst = phi_action(G, dev(to_prod(u, idx)), dt, [None, dev(to_prod(x, idx))], [1.0],
                           opts=gopts, stats=True, trace_cap=64)
    assert gst["status"] == -3
    if case == "exponent":
        # the norm bound ends the call within the first attempts (h_{j+1,j} ~ dt |J|
        # enters the norm from m = 2 on), not the rejection limit of 200
        assert len(gst["trace"]) <= 3
    outs, gst = phi_action(G, dev(to_prod(u, idx)), 900.0, [None, dev(to_prod(x, idx))], [1.0],
                           stats=True)
    assert gst["status"] == 0


@pytest.mark.parametrize("scheme,lev,dt,nsteps", [
    ("exprb42", 3, 900.0, 1),          # the level-3 exprb42 single-step workload
    ("exprb42", 3, 3600.0, 3),
    ("pexprb43", 3, 3600.0, 3),
    ("exprb53", 3, 3600.0, 3),
    ("epi3", 3, 900.0, 4),
    ("epi2", 3, 900.0, 2),
    ("exprb53", 5, 3600.0, 2),
])
def test_exprb_step_matches_oracle(scheme, lev, dt, nsteps):
    from paper_1805_02144_gb300.api import SchemeState, exprb_step
    G, s, idx = pair(lev)
    amp = 200.0 if lev == 3 and dt == 900.0 else 400.0
    u0 = _state(s, 1 if amp == 200.0 else 2, amp)
    kp = KrylovPhi(s, PhiOpts(tol=1e-8))
    ref = integrate(scheme, s, u0, dt, nsteps, kp)
    st = SchemeState(G)
    u = dev(to_prod(u0, idx))
    njv = 0
    for _ in range(nsteps):
        u, gst = exprb_step(G, scheme, dt, u, state=st, stats=True)
        assert gst["status"] == 0
        njv += gst["n_jv"]
    got = to_oracle(host(u), idx)
    eh, ev = rel_l2_parts(got, ref, s.ng)
    assert eh <= 1e-10 and ev <= 1e-10, (eh, ev)
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref - u0)
    assert njv == sum(x.n_jv for _, x in kp.stats)
    # discrete mass is conserved by the device path too
    area = G.cell_areas()
    m0 = np.sum(area * to_prod(u0, idx)[3 * s.ng:])
    m1 = np.sum(area * host(u)[3 * s.ng:])
    assert abs(m1 - m0) <= 1e-13 * m0


def test_exprb53_level7_step_matches_oracle():
    """Full size: the level-7 exprb53 dt = 3600 s step the benchmark times."""
    from paper_1805_02144_gb300.api import SchemeState, exprb_step
    G, s, idx = pair(7)
    u0 = _state(s, 2, 400.0)
    kp = KrylovPhi(s, PhiOpts(tol=1e-8))
    ref = step("exprb53", s, u0, 3600.0, kp)
    st = SchemeState(G)
    u, gst = exprb_step(G, "exprb53", 3600.0, dev(to_prod(u0, idx)), state=st, stats=True, trace_cap=256)
    assert gst["status"] == 0
    got = to_oracle(host(u), idx)
    eh, ev = rel_l2_parts(got, ref, s.ng)
    assert eh <= 1e-10 and ev <= 1e-10, (eh, ev)
    assert gst["n_jv"] == sum(x.n_jv for _, x in kp.stats)
