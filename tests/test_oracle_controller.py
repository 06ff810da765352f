"""Pins of the oracle's substep controller (Algorithm 1 steps 4-6, Eq. eq:cost).

Every GPU parity test demands the GPU's (m, accept) decisions equal the
oracle's, so a mistake in the oracle's controller would be copied by a GPU
that agrees with it.  These pins fix the controller to values evaluated by
hand from the printed cost function and from the stated proposal rules
(``tests/golden/controller_*.json``), plus properties of the rules:

* ``cost``: seven hand-evaluated values of Eq. eq:cost, including the
  round-half-up substep count, the at-least-one-substep and M >= 44/3
  readings and the rounding of M's logarithm on both sides of .5;
* ``proposals``: eight hand-evaluated (tau_new, m_new) pairs covering both
  clamps of tau and of m, omega = 0, the m_max and breakdown caps and m = 1;
* ``accepts`` / ``prefer_step_size``: the acceptance boundary and the choice
  between the two updates.

The last tests plant plausible mistakes in the oracle (monkeypatched on the
CPU) and check that at least one pin fails for each.  The terms
2(p-1)(n_A+N) and (2p+1)N appear identically in C(tau_new, m) and
C(tau, m_new), and N and n_A enter the first term only as N + n_A, so none
of them can change which update is chosen: the golden cost values pin them.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import phipm
from oracle.phipm import PhiOpts

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)["cases"]


COST = _load("controller_cost.json")
PROP = _load("controller_proposals.json")


def _cost_failures(cost_fn):
    bad = []
    for c in COST:
        got = cost_fn(c["tau"], c["m"], c["p"], c["remaining"], c["N"], c["nA"], c["hnorm"])
        if not abs(got - c["expected"]) <= 1e-12 * abs(c["expected"]):
            bad.append((c["name"], got, c["expected"]))
    return bad


def _proposal_failures(prop_fn):
    bad = []
    opts = PhiOpts()
    for c in PROP:
        tn, mn = prop_fn(c["omega"], c["tau"], c["m"], c["cap"], opts)
        if not (abs(tn - c["tau_new"]) <= 1e-14 * c["tau_new"] and mn == c["m_new"]):
            bad.append((c["name"], (tn, mn), (c["tau_new"], c["m_new"])))
    return bad


def test_cost_matches_hand_evaluated_values():
    assert _cost_failures(phipm.cost) == []


def test_proposals_match_hand_evaluated_values():
    assert _proposal_failures(phipm.proposals) == []


def test_acceptance_boundary_is_delta():
    delta = PhiOpts().delta
    assert delta == 1.4                                  # Algorithm 1 initialisation
    assert phipm.accepts(delta, delta)
    assert phipm.accepts(0.0, delta)
    assert not phipm.accepts(math.nextafter(delta, math.inf), delta)


def test_cheaper_update_is_chosen():
    f = phipm.prefer_step_size
    assert f(10.0, 11.0, True, 9, 8)            # C(tau_new, m) cheaper: update tau
    assert not f(11.0, 10.0, True, 9, 8)        # C(tau, m_new) cheaper: update m
    assert f(10.0, 10.0, True, 9, 8)            # tie: tau
    assert not f(11.0, 10.0, False, 9, 8)       # rejected, m can grow: m
    assert f(11.0, 10.0, False, 8, 8)           # rejected, m cannot change: tau


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 7, 8, 12, 20, 33, 48, 63, 64])
@pytest.mark.parametrize("omega", [0.0, 1e-300, 1e-9, 0.3, 0.8, 1.0, 1.4, 1.41, 7.0, 1e3, 1e12, 1e300])
def test_proposals_respect_their_clamps(m, omega):
    opts = PhiOpts()
    tau = 0.37
    tn, mn = phipm.proposals(omega, tau, m, opts.m_max, opts)
    assert tau / 5.0 <= tn <= 2.0 * tau
    assert 1 <= mn <= opts.m_max
    assert mn >= min(math.ceil(3 * m / 4), opts.m_max) and mn <= m * 4 // 3 + 1
    if omega <= opts.gamma:          # at or below the target: tau does not shrink
        assert tn >= tau
    if omega > opts.delta:           # a rejection never proposes a shorter Krylov space and a longer step
        assert tn < tau
        assert mn >= m or m == opts.m_max


def test_omega_zero_grows_the_step():
    tn, mn = phipm.proposals(0.0, 0.25, 10, 64, PhiOpts())
    assert tn == 0.5 and mn == 8


def test_proposals_are_monotone_in_omega():
    opts = PhiOpts()
    om = np.geomspace(1e-8, 1e8, 400)
    res = [phipm.proposals(w, 0.5, 16, 64, opts) for w in om]
    taus = [r[0] for r in res]
    ms = [r[1] for r in res]
    assert all(a >= b for a, b in zip(taus, taus[1:]))
    assert all(a <= b for a, b in zip(ms, ms[1:]))


def test_cost_counts_work_as_printed():
    # each extra substep adds m (N + n_A); each extra Krylov vector adds
    # nsub (N + n_A) plus the growth of the (m+p+1)^3 exponential term
    N, nA, p = 1000, 7000, 2
    c4 = phipm.cost(0.25, 10, p, 1.0, N, nA, 1.0)
    c5 = phipm.cost(0.2, 10, p, 1.0, N, nA, 1.0)
    assert c5 - c4 == pytest.approx(10 * (N + nA))
    c11 = phipm.cost(0.25, 11, p, 1.0, N, nA, 1.0)
    assert c11 - c4 == pytest.approx(4 * (N + nA) + (44.0 / 3.0) * (14 ** 3 - 13 ** 3))


# --- planted mistakes: each must fail at least one pin ------------------------
def _nint(x):
    return int(math.floor(x + 0.5))


def _cost_variant(kind):
    def f(tau, m, p, remaining, N, nA, hnorm):
        nsub = max(1, _nint(remaining / tau))
        e = max(0, _nint(math.log2(hnorm / 5.37)))
        if kind == "swap_N_nA":
            N, nA = nA, N
        if kind == "floor_substeps":
            nsub = max(1, math.floor(remaining / tau))
        if kind == "ceil_substeps":
            nsub = max(1, math.ceil(remaining / tau))
        if kind == "no_min_substep":
            nsub = _nint(remaining / tau)
        if kind == "floor_log":
            e = max(0, math.floor(math.log2(hnorm / 5.37)))
        if kind == "ceil_log":
            e = max(0, math.ceil(math.log2(hnorm / 5.37)))
        if kind == "natural_log":
            e = max(0, _nint(math.log(hnorm / 5.37)))
        M = 44.0 / 3.0 + (1.0 if kind == "M_factor_1" else 2.0) * e
        k3 = (m + p) if kind == "cube_m_p" else (m + p + 1)
        c = nsub * m * (N + nA) + M * k3 ** 3
        if kind != "drop_2p_minus_1":
            c += 2 * (p - 1) * (nA + N)
        if kind != "drop_2p_plus_1_N":
            c += (2 * p + 1) * N
        return c
    return f


@pytest.mark.parametrize("kind", ["swap_N_nA", "floor_substeps", "ceil_substeps", "no_min_substep",
                                  "floor_log", "ceil_log", "natural_log", "M_factor_1", "cube_m_p",
                                  "drop_2p_minus_1", "drop_2p_plus_1_N"])
def test_planted_cost_mistake_fails_a_pin(kind, monkeypatch):
    monkeypatch.setattr(phipm, "cost", _cost_variant(kind))
    assert _cost_failures(phipm.cost) != []
    assert _cost_variant("none")(0.25, 10, 2, 1.0, 100, 700, 42.96) == pytest.approx(COST[0]["expected"])


def _prop_variant(kind):
    def f(omega, tau, m, cap, opts):
        gamma = opts.delta if kind == "delta_as_target" else opts.gamma
        if omega == 0.0:
            tn = 2.0 * tau
            mn = m if kind == "zero_keeps_m" else max(1, math.ceil(3 * m / 4))
        else:
            q = m / 4.0 if kind == "q_no_floor" else max(1.0, m / 4.0)
            expo = 1.0 / q if kind == "wrong_sign" else -1.0 / q
            tn = tau * (omega / gamma) ** expo
            lo = tau / 2.0 if kind == "tau_clamp_half" else tau / 5.0
            tn = min(max(tn, lo), 2.0 * tau)
            dm = math.ceil(math.log(omega / gamma) / math.log(opts.kappa))
            mn = m + dm
            hi = m * 4 // 3 if kind == "m_clamp_no_plus1" else m * 4 // 3 + 1
            mn = min(max(mn, math.ceil(3 * m / 4)), hi)
        cap_ = opts.m_max if kind == "ignore_cap" else cap
        mn = max(1, min(mn, opts.m_max, cap_))
        return tn, mn
    return f


@pytest.mark.parametrize("kind", ["delta_as_target", "zero_keeps_m", "q_no_floor", "wrong_sign",
                                  "tau_clamp_half", "m_clamp_no_plus1", "ignore_cap"])
def test_planted_proposal_mistake_fails_a_pin(kind, monkeypatch):
    monkeypatch.setattr(phipm, "proposals", _prop_variant(kind))
    assert _proposal_failures(phipm.proposals) != []
    assert _proposal_failures(_prop_variant("none")) == []


def test_chosen_update_is_applied_to_the_next_attempt():
    """In a real call the update chosen after each attempt is the one the next
    attempt uses: the Krylov size changes to m_new exactly when the m update
    was chosen (a spy on prefer_step_size records the choice)."""
    from conftest import oracle_swe
    from paper_1805_02144_gb300.inputs import balanced_state, random_vector
    s = oracle_swe(2)
    u = balanced_state(s.grid.x, 1, 400.0)
    dt = 14400.0
    v = [None, random_vector(s.n, 2)]
    calls = []
    real_pref = phipm.prefer_step_size

    def spy(c_tau, c_m, accepted, m_new, m):
        r = real_pref(c_tau, c_m, accepted, m_new, m)
        calls.append((m_new, m, r))
        return r
    orig = phipm.prefer_step_size
    try:
        phipm.prefer_step_size = spy
        W, st = phipm.phipm_simul_iom2(lambda x: dt * s.Jv(u, x), [0.5, 1.0], v, PhiOpts(tol=1e-8), s.nA)
    finally:
        phipm.prefer_step_size = orig
    assert len(calls) == len(st.trace) >= 3
    assert {r for *_, r in calls} == {True, False}      # both updates occur
    for k in range(len(st.trace) - 1):
        m_new, m, take_tau = calls[k]
        assert st.trace[k + 1].m == (m if take_tau else m_new), k


@pytest.mark.parametrize("pattern", [(0, 1), (1, 1, 0, 1), (0, 0, 0, 1, 1)])
def test_relative_tolerance_makes_the_decisions_scale_invariant(pattern):
    """Reading R7: with s = max_l ||v_l|| the accept test is invariant under
    v_l -> c v_l, so the same decisions are taken and y scales by c; with the
    absolute test (s = 1) a large c forces more work."""
    from conftest import oracle_swe
    from paper_1805_02144_gb300.inputs import balanced_state, random_vector
    s = oracle_swe(2)
    u = balanced_state(s.grid.x, 1, 400.0)
    dt = 7200.0
    v = [None if not on else random_vector(s.n, 30 + i) for i, on in enumerate(pattern)]
    run = lambda vv, mode: phipm.phipm_simul_iom2(lambda x: dt * s.Jv(u, x), [0.5, 1.0], vv,
                                                  PhiOpts(tol=1e-8, tol_mode=mode), s.nA)
    W1, st1 = run(v, "relative")
    c = 1e6
    Wc, stc = run([None if x is None else c * x for x in v], "relative")
    assert [(a.m, a.accepted) for a in st1.trace] == [(a.m, a.accepted) for a in stc.trace]
    for a, b in zip(W1, Wc):
        assert np.linalg.norm(b - c * a) <= 1e-12 * np.linalg.norm(c * a)
    # the absolute test sees the scaled error estimate against the same Tol
    _, sta = run([None if x is None else c * x for x in v], "absolute")
    _, st0 = run(v, "absolute")
    assert sta.n_jv > st0.n_jv
