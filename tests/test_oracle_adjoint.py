"""Pins of the oracle gradient (oracle/adjoint.py) to things other than itself.

* The torch re-evaluation of a step equals the numpy oracle step (which the
  other oracle tests pin to the paper) to rounding.
* The gradient equals a central finite difference of the numpy oracle with
  the same frozen decisions (a derivative computed without autograd).
* The misfit gradient is checked entry by entry against its definition.
* The observation network is a function of cell positions only.
"""
import numpy as np
import pytest
import torch

from conftest import oracle_swe
from oracle.adjoint import (TorchSWE, forward_with_traces, loss_and_gradient, loss_replayed, misfit,
                            step_replay, step_vjp)
from oracle.phipm import PhiOpts
from paper_1805_02144_gb300.inputs import balanced_state, observation_network, random_vector


def _direction(s, u, seed):
    """A random direction scaled like the state (velocity and height parts)."""
    d = random_vector(s.n, seed)
    ng = s.ng
    d[:3 * ng] *= np.abs(u[:3 * ng]).max()
    d[3 * ng:] *= 400.0
    return d


@pytest.mark.parametrize("scheme", ["epi2", "exprb42", "pexprb43", "exprb53"])
def test_torch_step_equals_numpy_step(scheme):
    s = oracle_swe(3)
    u0 = balanced_state(s.grid.x, 2, 400.0)
    states, traces = forward_with_traces(scheme, s, u0, 1800.0, 2)
    tm = TorchSWE(s)
    for k in range(2):
        got = step_replay(scheme, tm, torch.from_numpy(states[k]), 1800.0, traces[k]).numpy()
        assert np.linalg.norm(got - states[k + 1]) <= 1e-13 * np.linalg.norm(states[k + 1])


@pytest.mark.parametrize("scheme,lev,nsteps", [("exprb42", 3, 2), ("epi2", 3, 2), ("exprb42", 4, 3),
                                               ("pexprb43", 3, 2), ("exprb53", 3, 2)])
def test_gradient_matches_frozen_central_difference(scheme, lev, nsteps):
    s = oracle_swe(lev)
    u0 = balanced_state(s.grid.x, 2, 400.0)
    cells, y, sigma = observation_network(s.grid.x, min(1000, s.ng // 4), 7, 5.0)
    J, g, traces = loss_and_gradient(scheme, s, u0, 1800.0, nsteps, cells, y, sigma)
    assert J > 0.0
    for seed in (3, 4):
        d = _direction(s, u0, seed)
        eps = 1e-5
        jp = loss_replayed(scheme, s, u0 + eps * d, 1800.0, traces, cells, y, sigma)
        jm = loss_replayed(scheme, s, u0 - eps * d, 1800.0, traces, cells, y, sigma)
        fd = (jp - jm) / (2 * eps)
        assert abs(fd - g @ d) <= 1e-8 * abs(fd), (fd, g @ d)


def test_single_step_vjp_matches_central_difference_of_the_state():
    """(du_{n+1}/du_n)^T lam against <lam, central difference of u_{n+1}>."""
    s = oracle_swe(3)
    u0 = balanced_state(s.grid.x, 5, 300.0)
    _, traces = forward_with_traces("exprb42", s, u0, 900.0, 1)
    lam = random_vector(s.n, 9)
    _, g = step_vjp("exprb42", TorchSWE(s), u0, 900.0, traces[0], lam)
    from oracle.adjoint import ReplayPhi
    from oracle.schemes import step
    d = _direction(s, u0, 10)
    eps = 1e-5
    up = step("exprb42", s, u0 + eps * d, 900.0, ReplayPhi(s, traces[0]))
    um = step("exprb42", s, u0 - eps * d, 900.0, ReplayPhi(s, traces[0]))
    fd = lam @ (up - um) / (2 * eps)
    assert abs(fd - g @ d) <= 1e-8 * abs(fd), (fd, g @ d)


def test_misfit_gradient_definition():
    ng = 50
    u = random_vector(4 * ng, 1) + 10.0
    cells = np.array([3, 7, 7, 20])       # a repeated cell counts twice
    y = np.array([9.0, 11.0, 10.5, 10.0])
    J, g = misfit(cells, y, 2.0, u, ng)
    h = u[3 * ng:]
    assert J == pytest.approx(0.5 * sum((h[c] - yy) ** 2 for c, yy in zip(cells, y)) / 4.0, rel=1e-15)
    ref = np.zeros(4 * ng)
    for c, yy in zip(cells, y):
        ref[3 * ng + c] += (h[c] - yy) / 4.0
    assert np.array_equal(g, ref)


def test_observation_network_depends_on_positions_only():
    s = oracle_swe(4)
    x = s.grid.x
    cells, y, sigma = observation_network(x, 1000, 7, 5.0)
    assert len(np.unique(cells)) == 1000 and sigma == 5.0
    perm = np.random.Generator(np.random.PCG64(0)).permutation(s.ng)
    cells_p, y_p, _ = observation_network(x[perm], 1000, 7, 5.0)
    assert np.array_equal(perm[cells_p], cells)
    assert np.array_equal(y_p, y)
    # values: truth height plus noise of the stated size
    resid = y - balanced_state(x, 8, 400.0)[3 * s.ng:][cells]
    assert 4.0 < np.std(resid) < 6.0
