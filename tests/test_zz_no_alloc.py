"""swe_jv_noalloc: J(u)x for callers that may not allocate device memory.

Some callers cannot let the library call cudaMalloc when they call it: code
running under another framework's memory pool or under a fixed device budget
reserved at start-up, and real-time loops that cannot take an allocation's
latency or an out-of-memory failure in the middle of a run.  swe_jv allocates
the grid's workspace on first use; swe_jv_noalloc takes its scratch from a
static device array in the library image instead, limited to grids of at most
40,962 cells (level 6).

The allocation-free variant must give the same result as swe_jv on the same
grid, on two calls in a row (the second call reuses the scratch the first one
left behind), at level 5 and at its limit, level 6, where all 12 scratch
planes are full.  Both run the same FP64 device stencil, so they must agree to
the last bit of the largest entry (1e-15 relative).  At level 6 it is also
compared with the oracle's J x, with the element-wise bound of the swe_jv
parity test.  This file is collected last on purpose: if it fails, a run that
stops at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_02144_gb300 import build
    build.build()


def _call(L, G, u, x, out, stream=None):
    return L.swe_jv_noalloc(G.handle, C.c_void_p(u.data_ptr()), C.c_void_p(x.data_ptr()),
                            C.c_void_p(out.data_ptr()), stream)


@pytest.mark.parametrize("lev", [5, 6])
def test_jv_noalloc_matches_jv_on_consecutive_calls(lev):
    import torch
    from paper_1805_02144_gb300 import _lib
    from paper_1805_02144_gb300.api import Grid, swe_jv
    from paper_1805_02144_gb300.inputs import balanced_state, random_vector
    L = _lib.load()
    G = Grid(lev)
    if lev == 6:
        assert G.ncells == 40962                      # exactly the scratch limit
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    xyz = G.cell_centres()
    for call, seed in enumerate((3, 8)):
        u = torch.from_numpy(balanced_state(xyz, seed, 400.0)).cuda()
        x = torch.from_numpy(random_vector(G.n, 20 + seed)).cuda()
        out = torch.full_like(u, float("nan"))
        rc = _call(L, G, u, x, out, stream)
        assert rc == 0, L.swe_last_error()
        ref = swe_jv(G, u, x)
        torch.cuda.synchronize()
        d = (out - ref).abs().max().item()
        assert d <= 1e-15 * ref.abs().max().item(), (call, d)


def test_jv_noalloc_at_its_limit_matches_oracle():
    import torch
    from paper_1805_02144_gb300 import _lib
    from paper_1805_02144_gb300.inputs import balanced_state, random_vector
    from parity_utils import dev, host, pair, stencil_tol, term_scale, to_oracle, to_prod
    L = _lib.load()
    G, s, idx = pair(6)
    u = balanced_state(s.grid.x, 3, 400.0)
    x = random_vector(s.n, 11)
    ref = s.Jv(u, x)
    ud, xd = dev(to_prod(u, idx)), dev(to_prod(x, idx))
    out = torch.full_like(ud, float("nan"))
    for _ in range(2):
        rc = _call(L, G, ud, xd, out, C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, L.swe_last_error()
        got = to_oracle(host(out), idx)
        assert np.abs(got - ref).max() <= stencil_tol(s) * term_scale(s, u, x)
        assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_jv_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    from paper_1805_02144_gb300 import _lib
    from paper_1805_02144_gb300._lib import SWE_ERR_INVALID_ARG
    from paper_1805_02144_gb300.api import Grid
    L = _lib.load()
    G = Grid(7)
    u = torch.zeros(G.n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(u)
    out = torch.zeros_like(u)
    rc = _call(L, G, u, x, out)
    assert rc == SWE_ERR_INVALID_ARG and b"40962" in L.swe_last_error()


def test_jv_noalloc_rejects_an_output_that_overlaps_an_input():
    import torch
    from paper_1805_02144_gb300 import _lib
    from paper_1805_02144_gb300._lib import SWE_ERR_INVALID_ARG
    from paper_1805_02144_gb300.api import Grid
    L = _lib.load()
    G = Grid(3)
    buf = torch.zeros(3 * G.n, dtype=torch.float64, device="cuda")
    u, x = buf[:G.n], buf[G.n:2 * G.n]
    assert _call(L, G, u, x, x) == SWE_ERR_INVALID_ARG       # jx == x
    assert _call(L, G, u, x, u) == SWE_ERR_INVALID_ARG       # jx == u
    assert _call(L, G, u, x, buf[G.n // 2:]) == SWE_ERR_INVALID_ARG   # partial overlap with u and x
    assert b"overlap" in L.swe_last_error()
    assert _call(L, G, u, x, buf[2 * G.n:]) == 0             # adjacent, not overlapping
    torch.cuda.synchronize()
