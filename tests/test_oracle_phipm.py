"""Pins of the oracle phipm_simul_iom2 (Algorithm 1).

The reference is the exact combination y(rho) = sum_l rho^l phi_l(rho A) v_l of
Eq. (eq3.15) computed by one dense exponential of the augmented block matrix
(a different route: no substepping, no Krylov space).  On tiny grids the
Krylov result must agree within a small multiple of Tol.  Substepping
invariance (Eqs. (eq3.16)-(eq3.18)): any partition of [0, 1] gives the same
y(1).
"""
import numpy as np
import pytest

from oracle.phi import phi_combination_dense
from oracle.phipm import Attempt, NoConvergence, PhiOpts, phipm_simul_iom2
from paper_1805_02144_gb300.inputs import balanced_state, random_vector

from conftest import oracle_swe


def _setup(lev=2, dt=3600.0, seed=1):
    s = oracle_swe(lev)
    u = balanced_state(s.grid.x, seed, 400.0)
    J = s.jacobian(u).toarray()
    A = dt * J

    def Amul(x):
        return dt * s.Jv(u, x)
    return s, u, A, Amul


def _vecs(s, pattern, seed=0):
    return [None if not on else random_vector(s.n, seed + i) for i, on in enumerate(pattern)]


@pytest.mark.parametrize("pattern,rho", [
    ((0, 1), [0.75]),
    ((0, 1), [0.5, 1.0]),
    ((0, 1), [0.5, 0.9]),
    ((0, 0, 0, 1), [0.5, 0.9]),
    ((0, 1, 0, 1), [1.0]),
    ((0, 0, 0, 1, 1), [1.0]),
    ((0, 1, 0, 1, 1), [1.0]),
    ((1, 1, 1), [0.3, 1.0]),
])
def test_matches_dense_exponential(pattern, rho):
    s, u, A, Amul = _setup()
    v = _vecs(s, pattern)
    W, st = phipm_simul_iom2(Amul, rho, v, PhiOpts(tol=1e-12), s.nA)
    for r, w in zip(rho, W):
        ref = phi_combination_dense(A, v, r)
        assert np.linalg.norm(w - ref) <= 1e-10 * np.linalg.norm(ref)
    assert st.n_substeps >= len(rho)
    assert sum(a.accepted for a in st.trace) == st.n_substeps
    assert len(st.trace) == st.n_substeps + st.n_reject


def test_tolerance_is_respected_at_production_tol():
    s, u, A, Amul = _setup(lev=3) if False else _setup(lev=2, dt=14400.0)
    v = _vecs(s, (0, 1, 0, 1, 1))
    for tol in (1e-6, 1e-8):
        W, st = phipm_simul_iom2(Amul, [1.0], v, PhiOpts(tol=tol), s.nA)
        ref = phi_combination_dense(A, v, 1.0)
        scale = max(np.linalg.norm(x) for x in v if x is not None)
        assert np.linalg.norm(W[0] - ref) <= 10 * tol * scale


def test_substep_partition_invariance():
    s, u, A, Amul = _setup(lev=1, dt=3600.0)
    v = _vecs(s, (1, 1, 0, 1))
    ref = phi_combination_dense(A, v, 1.0)
    results = []
    for nsub, m in ((1, 60), (3, 40), (7, 30)):
        trace = [Attempt(t=0, tau=1.0 / nsub, m=m, omega=0, accepted=True) for _ in range(nsub)]
        W, st = phipm_simul_iom2(Amul, [1.0], v, PhiOpts(tol=1e-12, m_max=64), s.nA, replay=trace)
        assert st.n_substeps == nsub
        results.append(W[0])
        assert np.linalg.norm(W[0] - ref) <= 1e-11 * np.linalg.norm(ref)
    assert np.linalg.norm(results[1] - results[2]) <= 1e-11 * np.linalg.norm(ref)


def test_zero_skip_counts_matvecs():
    s, u, A, Amul = _setup()
    v = _vecs(s, (0, 0, 0, 1))
    m = 25
    trace = [Attempt(t=0, tau=1.0, m=m, omega=0, accepted=True)]
    W, st = phipm_simul_iom2(Amul, [1.0], v, PhiOpts(tol=1e-12), s.nA, replay=trace)
    # w_0 = w_1 = w_2 = 0 at t = 0: no A w products, only the m Krylov ones
    assert st.n_jv == m
    ref = phi_combination_dense(A, v, 1.0)
    assert np.linalg.norm(W[0] - ref) <= 1e-9 * np.linalg.norm(ref)
    # two substeps: the second has w_0 = y_1 != 0, so p = 3 products are added
    trace = [Attempt(t=0, tau=0.5, m=m, omega=0, accepted=True)] * 2
    W, st = phipm_simul_iom2(Amul, [1.0], v, PhiOpts(tol=1e-12), s.nA, replay=trace)
    assert st.n_jv == 2 * m + 3


def test_outputs_equal_separate_calls():
    s, u, A, Amul = _setup()
    v = _vecs(s, (0, 1))
    W2, _ = phipm_simul_iom2(Amul, [0.5, 0.9], v, PhiOpts(tol=1e-12), s.nA)
    W1, _ = phipm_simul_iom2(Amul, [0.5], v, PhiOpts(tol=1e-12), s.nA)
    assert np.linalg.norm(W2[0] - W1[0]) <= 1e-10 * np.linalg.norm(W1[0])


def test_happy_breakdown_is_exact():
    rng = np.random.default_rng(2)
    n = 40
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([[-2.0, 0.5, 1.5], rng.standard_normal(n - 3)])
    A = Q @ np.diag(lam) @ Q.T
    v1 = Q[:, :3] @ np.array([1.0, -2.0, 0.5])     # in a 3-dim invariant subspace
    W, st = phipm_simul_iom2(lambda x: A @ x, [1.0], [None, v1], PhiOpts(tol=1e-12), nA=n * n)
    ref = phi_combination_dense(A, [None, v1], 1.0)
    assert np.linalg.norm(W[0] - ref) <= 1e-12 * np.linalg.norm(ref)
    assert st.m_max_used <= 3


def test_zero_input_gives_zero():
    s, u, A, Amul = _setup()
    W, st = phipm_simul_iom2(Amul, [0.5, 1.0], [None, np.zeros(s.n)], PhiOpts(), s.nA)
    assert all(np.all(w == 0) for w in W) and st.n_jv == 0


def test_rejects_bad_rho_and_reports_no_convergence():
    s, u, A, Amul = _setup()
    v = _vecs(s, (0, 1))
    with pytest.raises(ValueError):
        phipm_simul_iom2(Amul, [0.9, 0.5], v, PhiOpts(), s.nA)
    with pytest.raises(NoConvergence):
        phipm_simul_iom2(Amul, [1.0], v, PhiOpts(tol=1e-30, max_reject=3, m_max=4), s.nA)


# --- wider orthogonalisation windows (iom > 2, full Arnoldi at iom >= m) -----
def test_full_arnoldi_basis_is_orthonormal_and_satisfies_the_arnoldi_relation():
    """iom >= m: V_m orthonormal, H_m upper Hessenberg, A V_m = V_{m+1} Hbar_m."""
    from oracle.phipm import IOM2Basis
    s, u, A, Amul = _setup()
    v1 = random_vector(s.n, 5)
    v1 /= np.linalg.norm(v1)
    m = 20
    B = IOM2Basis(lambda x: A @ x, v1, iom=64, m_max=m, bd=1e-13)
    assert B.extend(m) == m
    V = np.stack(B.V[:m + 1], axis=1)
    assert np.abs(V.T @ V - np.eye(m + 1)).max() <= 1e-10
    H = B.H[:m + 1, :m]
    assert np.all(np.tril(H, -2) == 0.0)                       # upper Hessenberg
    assert np.linalg.norm(A @ V[:, :m] - V @ H) <= 1e-12 * np.linalg.norm(A @ V[:, :m])


def test_symmetric_matrix_gives_the_same_tridiagonal_h_for_any_window():
    """For symmetric A, Arnoldi reduces to Lanczos: the full-window H equals the
    IOM2 H (tridiagonal), up to rounding."""
    from oracle.phipm import IOM2Basis
    rng = np.random.default_rng(7)
    n, m = 60, 15
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.linspace(-3.0, 2.0, n)) @ Q.T
    v1 = rng.standard_normal(n)
    v1 /= np.linalg.norm(v1)
    H2 = IOM2Basis(lambda x: A @ x, v1, iom=2, m_max=m, bd=1e-13)
    Hf = IOM2Basis(lambda x: A @ x, v1, iom=64, m_max=m, bd=1e-13)
    H2.extend(m)
    Hf.extend(m)
    assert np.abs(Hf.H - H2.H).max() <= 1e-9
    assert np.abs(np.triu(Hf.H[:m, :m], 2)).max() <= 1e-9


@pytest.mark.parametrize("iom", [4, 64])
def test_wide_window_phi_action_matches_dense_reference(iom):
    s, u, A, Amul = _setup()
    v = _vecs(s, (0, 1, 0, 1), seed=3)
    W, st = phipm_simul_iom2(Amul, [0.5, 1.0], v, PhiOpts(tol=1e-12, iom=iom), s.nA)
    for w, rho in zip(W, [0.5, 1.0]):
        ref = phi_combination_dense(A, v, rho)
        assert np.linalg.norm(w - ref) <= 1e-10 * np.linalg.norm(ref)
    assert st.n_jv > 0
