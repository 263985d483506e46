"""Failure detection without a fault: a device-side wait that nothing
completes gives up after its poll bound, the call reports EFM_ETIMEOUT, and
the same network and stream then run a traversal that matches the oracle."""
import numpy as np
import pytest

from paper_1804_02867_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def efm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_02867_gb300 import build, efmgraph

    build.build()
    efmgraph.load_library()
    return efmgraph


def test_bounded_wait_gives_up_and_the_gpu_stays_usable(oracle_lib, efm):
    net = synth.tiny(2)
    targets = list(net.targets) + [-1]
    with efm.Network(net) as nw:
        for _ in range(2):
            rc, polls, ms = efm.efm_check_bounded_wait(nw.handle)
            assert rc == -4 and "wait expired" in efm.status_str(rc)
            assert polls == 1 << 20 and 0.0 < ms < 10_000.0
        got = efm.enumerate_targets(nw, targets, 8, 1)
    for t, (sup, ctr) in zip(targets, got):
        osup, octr = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(8, 1, 0, 0))
        assert np.array_equal(sup, osup) and ctr == octr, t
