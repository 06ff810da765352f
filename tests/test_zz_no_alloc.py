"""swe_jv_noalloc: J(u)x for callers that may not allocate device memory.

The allocation-free variant (static scratch in the library image) must give
the same result as swe_jv on the same grid, on two calls in a row (the second
call reuses the scratch the first one left behind).  Both run the same FP64
device stencil, so the results must agree to the last bit of the largest
entry (1e-15 relative).  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_jv_noalloc_matches_jv_on_consecutive_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_02144_gb300 import build
    build.build()
    from paper_1805_02144_gb300 import _lib
    from paper_1805_02144_gb300.api import Grid, swe_jv
    from paper_1805_02144_gb300.inputs import balanced_state, random_vector
    L = _lib.load()
    G = Grid(5)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    xyz = G.cell_centres()
    for call, seed in enumerate((3, 8)):
        u = torch.from_numpy(balanced_state(xyz, seed, 400.0)).cuda()
        x = torch.from_numpy(random_vector(G.n, 20 + seed)).cuda()
        out = torch.full_like(u, float("nan"))
        rc = L.swe_jv_noalloc(G.handle, C.c_void_p(u.data_ptr()), C.c_void_p(x.data_ptr()),
                              C.c_void_p(out.data_ptr()), stream)
        assert rc == 0, L.swe_last_error()
        ref = swe_jv(G, u, x)
        torch.cuda.synchronize()
        d = (out - ref).abs().max().item()
        assert d <= 1e-15 * ref.abs().max().item(), (call, d)


def test_jv_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_02144_gb300 import _lib
    from paper_1805_02144_gb300.api import Grid
    L = _lib.load()
    G = Grid(7)
    u = torch.zeros(G.n, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(u)
    rc = L.swe_jv_noalloc(G.handle, C.c_void_p(u.data_ptr()), C.c_void_p(u.data_ptr()),
                          C.c_void_p(out.data_ptr()), None)
    assert rc == -1 and b"40962" in L.swe_last_error()
