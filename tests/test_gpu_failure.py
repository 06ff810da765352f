"""Failure detection without a GPU fault: the bounded wait every grid barrier
and reduction uses, run on a flag that nothing sets, must give up at its time
limit with SWE_ERR_TIMEOUT in the abort word and leave the context usable; a
set abort word must end the wait at its first check."""
import time

import numpy as np
import pytest

from parity_utils import dev, host, pair, to_oracle, to_prod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_02144_gb300 import build
    build.build()


def test_wait_on_a_flag_nothing_sets_times_out_and_the_context_survives():
    from paper_1805_02144_gb300._lib import SWE_ERR_TIMEOUT
    from paper_1805_02144_gb300.api import swe_rhs, swe_selftest_wait
    from paper_1805_02144_gb300.inputs import balanced_state
    t0 = time.perf_counter()
    assert swe_selftest_wait(0.05) == SWE_ERR_TIMEOUT
    elapsed = time.perf_counter() - t0
    assert 0.05 <= elapsed < 5.0
    # the device still computes correctly afterwards
    G, s, idx = pair(3)
    u = balanced_state(s.grid.x, 2, 400.0)
    got = to_oracle(host(swe_rhs(G, dev(to_prod(u, idx)))), idx)
    ref = s.F(u)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_a_set_abort_word_ends_the_wait_at_once():
    from paper_1805_02144_gb300._lib import SWE_ERR_NONFINITE
    from paper_1805_02144_gb300.api import swe_selftest_wait
    t0 = time.perf_counter()
    assert swe_selftest_wait(1.0, preset_abort=SWE_ERR_NONFINITE) == SWE_ERR_NONFINITE
    assert time.perf_counter() - t0 < 0.9          # well before the 1 s limit


def test_out_of_range_limits_are_rejected():
    from paper_1805_02144_gb300._lib import SweError
    from paper_1805_02144_gb300.api import swe_selftest_wait
    for bad in (0.0, 2.0):
        with pytest.raises(SweError):
            swe_selftest_wait(bad)
    with pytest.raises(SweError):
        swe_selftest_wait(0.01, preset_abort=3)
