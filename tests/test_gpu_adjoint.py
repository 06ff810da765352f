"""GPU parity of the transposed stencils (adjoint building blocks).

swe_jtv gives J(u)^T lam and swe_dqtv gives (J(x) - J(0))^T lam, the
transposes of the Jacobian of Eqs. (eq:dynja)-(eq:dynjc) and of the
derivative of the quadratic part of F.  They are compared element by element
with the transposed sparse matrices the oracle assembles, within the
stencil tolerance of one evaluation (relative to the summed |terms|), and
checked against swe_jv by the dot-product identity <lam, J x> = <J^T lam, x>
on the same device grid.
"""
import numpy as np
import pytest

from oracle.phipm import PhiOpts

from paper_1805_02144_gb300.inputs import balanced_state, random_vector
from parity_utils import abs_jacobian, dev, host, pair, stencil_tol, to_oracle, to_prod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_02144_gb300 import build
    build.build()


def _check(s, got, ref, absJ, lam):
    bound = stencil_tol(s) * np.max(absJ.T @ np.abs(lam))
    assert np.abs(got - ref).max() <= bound, (np.abs(got - ref).max(), bound)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("lev", [0, 3, 5, 7])
def test_jtv_matches_oracle(lev):
    from paper_1805_02144_gb300.api import swe_jtv
    G, s, idx = pair(lev)
    u = balanced_state(s.grid.x, 3, 400.0)
    lam = random_vector(s.n, 21)
    ref = s.jacobian(u).T @ lam
    got = to_oracle(host(swe_jtv(G, dev(to_prod(u, idx)), dev(to_prod(lam, idx)))), idx)
    _check(s, got, ref, abs_jacobian(s, u), lam)


@pytest.mark.parametrize("lev", [0, 3, 5])
def test_dqtv_matches_oracle(lev):
    from paper_1805_02144_gb300.api import swe_dqtv
    G, s, idx = pair(lev)
    x = balanced_state(s.grid.x, 4, 300.0) + 1e-2 * random_vector(s.n, 5)
    lam = random_vector(s.n, 22)
    ref = (s.jacobian(x) - s.jacobian(np.zeros_like(x))).T @ lam
    got = to_oracle(host(swe_dqtv(G, dev(to_prod(x, idx)), dev(to_prod(lam, idx)))), idx)
    _check(s, got, ref, abs_jacobian(s, x, quad_only=True), lam)


@pytest.mark.parametrize("lev", [2, 6])
def test_transpose_dot_identity(lev):
    """<lam, J x> = <J^T lam, x> and <lam, Q'(w) x> = <Q'(w)^T lam, x> on one grid."""
    import torch
    from paper_1805_02144_gb300.api import Grid, swe_dqtv, swe_jtv, swe_jv
    G = Grid(lev)
    u = dev(balanced_state(G.cell_centres(), 6, 400.0))
    x, lam = dev(random_vector(G.n, 31)), dev(random_vector(G.n, 32))
    zero = torch.zeros_like(u)
    a = torch.dot(lam, swe_jv(G, u, x)).item()
    b = torch.dot(swe_jtv(G, u, lam), x).item()
    scale = torch.dot(lam.abs(), swe_jv(G, u.abs(), x.abs()).abs()).item()
    assert abs(a - b) <= 1e-13 * scale, (a, b, scale)
    # Q'(w) x = J(w) x - J(0) x
    qa = torch.dot(lam, swe_jv(G, u, x) - swe_jv(G, zero, x)).item()
    qb = torch.dot(swe_dqtv(G, u, lam), x).item()
    assert abs(qa - qb) <= 1e-12 * scale, (qa, qb, scale)


def test_transposed_entry_points_reject_aliasing():
    from paper_1805_02144_gb300 import _lib
    from paper_1805_02144_gb300.api import Grid
    G = Grid(1)
    lam = dev(random_vector(G.n, 1))
    lib = _lib.load()
    p = lam.data_ptr()
    assert lib.swe_jtv(G.handle, p, p, p, None) == -1
    assert lib.swe_dqtv(G.handle, p, p, p, None) == -1


# ---------------------------------------------------------------------------
# adjoint of whole steps (exprb_step_adjoint)
# ---------------------------------------------------------------------------
TRACE_CAP = 4096


def _gpu_forward(G, scheme, u0p, dt, nsteps, opts=None):
    from paper_1805_02144_gb300.api import SchemeState, exprb_step
    st = SchemeState(G)
    u = dev(u0p)
    states, traces = [u], []
    for _ in range(nsteps):
        u, info = exprb_step(G, scheme, dt, u, state=st, opts=opts, stats=True, trace_cap=TRACE_CAP)
        assert info["status"] == 0 and len(info["trace"]) < TRACE_CAP
        states.append(u)
        traces.append(info["trace"])
    return states, traces


def _same_decisions(gtrace, ocalls):
    """Identical Krylov sizes and accept/reject sequence.  Step sizes follow
    omega continuously, and omega comes from a small correction term whose
    rounding differs between the two evaluations, so tau agrees to ~1e-9."""
    flat = [(c, a) for c, call in enumerate(ocalls) for a in call]
    assert len(gtrace) == len(flat)
    for g, (c, o) in zip(gtrace, flat):
        assert g["call"] == c and g["m"] == o.m and g["accepted"] == o.accepted
        assert abs(g["tau"] - o.tau) <= 1e-7 * o.tau


def _replay(trace):
    return [[r["tau"], r["m"], 1.0 if r["accepted"] else 0.0] for r in trace]


@pytest.mark.parametrize("scheme,lev", [("epi2", 3), ("exprb42", 3), ("exprb42", 5), ("pexprb43", 3),
                                        ("pexprb43", 5), ("exprb53", 3), ("exprb53", 5)])
def test_step_adjoint_matches_oracle(scheme, lev):
    from oracle.adjoint import TorchSWE, forward_with_traces, step_vjp
    from paper_1805_02144_gb300.api import exprb_step_adjoint
    G, s, idx = pair(lev)
    dt = 1800.0
    u0 = balanced_state(s.grid.x, 2, 400.0)
    ostates, otraces = forward_with_traces(scheme, s, u0, dt, 2)
    gstates, gtraces = _gpu_forward(G, scheme, to_prod(u0, idx), dt, 2)
    tm = TorchSWE(s)
    for k in range(2):
        _same_decisions(gtraces[k], otraces[k])
        lam = random_vector(s.n, 50 + k)
        _, ref = step_vjp(scheme, tm, ostates[k], dt, otraces[k], lam)
        got, info = exprb_step_adjoint(G, scheme, dt, gstates[k], gtraces[k], dev(to_prod(lam, idx)), stats=True)
        assert info["status"] == 0
        got = to_oracle(host(got), idx)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 1e-9, err


@pytest.mark.parametrize("scheme", ["exprb42", "pexprb43", "exprb53"])
def test_step_adjoint_matches_gpu_frozen_central_difference(scheme):
    """<lam, dS/du d> by a central difference of the GPU step replaying the
    forward's decisions, against <S'^T lam, d> from the adjoint."""
    from paper_1805_02144_gb300.api import SchemeState, exprb_step, exprb_step_adjoint, Grid
    G = Grid(4)
    x = G.cell_centres()
    u0 = balanced_state(x, 3, 400.0)
    dt = 1800.0
    states, traces = _gpu_forward(G, scheme, u0, dt, 2)
    ng = G.ncells
    for k in range(2):
        lam = random_vector(G.n, 70 + k)
        d = random_vector(G.n, 80 + k)
        un = host(states[k])
        d[:3 * ng] *= np.abs(un[:3 * ng]).max()
        d[3 * ng:] *= 400.0
        adj = host(exprb_step_adjoint(G, scheme, dt, states[k], traces[k], dev(lam)))
        eps = 1e-6
        rp = {"replay": _replay(traces[k])}
        up = host(exprb_step(G, scheme, dt, dev(un + eps * d), state=SchemeState(G), opts=rp))
        um = host(exprb_step(G, scheme, dt, dev(un - eps * d), state=SchemeState(G), opts=rp))
        fd = lam @ (up - um) / (2 * eps)
        assert abs(fd - adj @ d) <= 1e-7 * abs(fd), (fd, adj @ d)


def _misfit_gpu(u, cells_t, y_t, sigma, ng):
    import torch
    h = u[3 * ng:]
    r = (h[cells_t] - y_t) / sigma
    lam = torch.zeros_like(u)
    lam.index_add_(0, 3 * ng + cells_t, r / sigma)
    return 0.5 * float(torch.dot(r, r)), lam


def test_forecast_gradient_level6_12_steps():
    """Gradient of the observation misfit of a 6 h exprb42 forecast: level 6,
    dt = 1800 s, 12 steps, Tol 1e-10; observations = the oracle's 6 h truth
    forecast from the balanced state of seed 5 at 1000 seeded cells plus
    N(0, 5^2) noise; first guess = the balanced state of seed 6.  Checked
    against the oracle gradient and against central differences of the GPU
    forecast with frozen decisions along 8 seeded directions,
    eps = 1e-6 ||u_0|| / ||d||."""
    import torch
    from oracle.adjoint import loss_and_gradient
    from oracle.schemes import KrylovPhi, integrate
    from paper_1805_02144_gb300.api import SchemeState, exprb_step, exprb_step_adjoint
    from paper_1805_02144_gb300.inputs import fd_directions, observation_network
    G, s, idx = pair(6)
    dt, nsteps, tol = 1800.0, 12, 1e-10
    ng = s.ng
    truth = integrate("exprb42", s, balanced_state(s.grid.x, 5, 400.0), dt, nsteps,
                      KrylovPhi(s, PhiOpts(tol=tol)))
    cells, y, sigma = observation_network(s.grid.x, 1000, 7, 5.0, h_truth=truth[3 * ng:])
    u0 = balanced_state(s.grid.x, 6, 400.0)
    J_o, g_o, otraces = loss_and_gradient("exprb42", s, u0, dt, nsteps, cells, y, sigma, PhiOpts(tol=tol))
    # the same observation set in the library's cell order
    inv = np.empty_like(idx)
    inv[idx] = np.arange(idx.size)
    cells_p = torch.from_numpy(inv[cells]).to("cuda")
    y_t = torch.from_numpy(y).to("cuda")
    opts = {"tol": tol}
    states, traces = _gpu_forward(G, "exprb42", to_prod(u0, idx), dt, nsteps, opts)
    for k in range(nsteps):
        _same_decisions(traces[k], otraces[k])
    J_g, lam = _misfit_gpu(states[-1], cells_p, y_t, sigma, G.ncells)
    assert abs(J_g - J_o) <= 1e-9 * J_o
    for k in reversed(range(nsteps)):
        lam = exprb_step_adjoint(G, "exprb42", dt, states[k], traces[k], lam, opts=opts)
    g = to_oracle(host(lam), idx)
    err = np.linalg.norm(g - g_o) / np.linalg.norm(g_o)
    assert err <= 1e-8, err

    def J_replayed(u):
        st = SchemeState(G)
        x = dev(u)
        for k in range(nsteps):
            x = exprb_step(G, "exprb42", dt, x, state=st, opts={"tol": tol, "replay": _replay(traces[k])})
        return _misfit_gpu(x, cells_p, y_t, sigma, G.ncells)[0]

    u0p = to_prod(u0, idx)
    gp = host(lam)
    for d, eps in fd_directions(u0p, 8, 11):
        fd = (J_replayed(u0p + eps * d) - J_replayed(u0p - eps * d)) / (2 * eps)
        assert abs(fd - gp @ d) <= 1e-6 * abs(fd), (fd, gp @ d)


def test_autograd_function_uses_the_adjoint():
    import torch
    from paper_1805_02144_gb300.api import (Grid, SchemeState, exprb_step_adjoint,
                                            exprb_step_differentiable)
    G = Grid(3)
    u0 = dev(balanced_state(G.cell_centres(), 4, 300.0)).requires_grad_(True)
    st = SchemeState(G)
    u1 = exprb_step_differentiable(G, "exprb42", 1800.0, u0, st)
    u2 = exprb_step_differentiable(G, "exprb42", 1800.0, u1, st)
    w = dev(random_vector(G.n, 5))
    (g,) = torch.autograd.grad(torch.dot(w, u2), u0)
    # the same by two explicit adjoint steps
    from paper_1805_02144_gb300.api import exprb_step
    st2 = SchemeState(G)
    a1, i1 = exprb_step(G, "exprb42", 1800.0, u0.detach(), state=st2, stats=True, trace_cap=TRACE_CAP)
    a2, i2 = exprb_step(G, "exprb42", 1800.0, a1, state=st2, stats=True, trace_cap=TRACE_CAP)
    l1 = exprb_step_adjoint(G, "exprb42", 1800.0, a1, i2["trace"], w)
    l0 = exprb_step_adjoint(G, "exprb42", 1800.0, u0.detach(), i1["trace"], l1)
    assert torch.equal(g, l0)


def test_adjoint_rejects_mismatched_traces():
    from paper_1805_02144_gb300 import _lib
    from paper_1805_02144_gb300.api import Grid, exprb_step_adjoint
    G = Grid(2)
    u = dev(balanced_state(G.cell_centres(), 4, 300.0))
    lam = dev(random_vector(G.n, 1))
    _, traces = _gpu_forward(G, "exprb42", host(u), 900.0, 1)
    with pytest.raises(RuntimeError):      # exprb42 trace given as EPI2
        exprb_step_adjoint(G, "epi2", 900.0, u, traces[0], lam)
    bad = [dict(r) for r in traces[0] if r["call"] == 0]
    with pytest.raises(RuntimeError):      # second call missing
        exprb_step_adjoint(G, "exprb42", 900.0, u, bad, lam)
    with pytest.raises(RuntimeError):      # epi3 needs the adjoint of its history term
        exprb_step_adjoint(G, "epi3", 900.0, u, traces[0], lam)
