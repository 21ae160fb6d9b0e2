"""Failure detection without a GPU fault: a device wait that can never be
satisfied (an mbarrier armed for 16 bytes that no copy delivers) gives up
after its wall-clock limit, records the expiry, and the host reads
MG_ETIMEOUT; the CUDA context stays usable (a cycle right after it still
matches the oracle)."""
import numpy as np
import pytest

import synth
from paper_2404_02493_gb300 import binding as B

from gpu_util import lib_handle, oracle_hier, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_02493_gb300 import build
    build.build()
    B.load()


def test_expired_wait_reports_timeout_and_context_survives():
    assert B.mg_selftest_wait_timeout() == B.MG_ETIMEOUT
    I = synth.config_constant(n=64, k=20.0)
    h = lib_handle([I], "fp64", n_cmax=15)
    try:
        u = np.zeros_like(I.g)
        B.mg_cycle(h, u, I.g.copy(), 1)
        ref = oracle_hier(I, n_cmax=15).cycle(np.zeros_like(I.g), I.g)
        assert rel(u, ref) < 1e-12
    finally:
        B.mg_destroy(h)
    # and a second expiry behaves the same
    assert B.mg_selftest_wait_timeout() == B.MG_ETIMEOUT
