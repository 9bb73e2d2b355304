"""Failure handling of the device-side waits, tested without a GPU fault.

Every spin wait in the tensor-core kernels is bounded (about one second of
clock64) and reports expiry in a flag word that the host turns into
TN_ETIMEOUT.  Here a wait on a barrier that nothing completes must give up,
set the timeout bit and leave the context usable for a normal evolution."""
import numpy as np
import pytest

from oracle import bptn as OB
from oracle import graph as OG

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tnlib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_14887_gb300 import build
    build.build()
    import paper_2306_14887_gb300 as tn
    return tn


def test_expired_wait_sets_the_timeout_bit_and_the_context_survives(tnlib):
    assert tnlib.selftest_bounded_wait() == 2
    g = OG.ring(12)
    with tnlib.TNState(g.n, g.edges, g.colours, chi=8) as s:
        s.apply_floquet(0.6, 3)
        z = s.expect_z_all()
    assert np.abs(z - OB.run(g, 8, 0.6, 3).all_z()).max() < 1e-6
