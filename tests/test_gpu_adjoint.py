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
