"""The allocation-free sort entry point (efm_sort_supports_noalloc).

Callers that cannot allocate device memory where they work (under another
framework's allocator, in loops that must not wait on an allocator) sort
supports with this entry point; its scratch lives in a fixed device array
inside the library.  This test checks, through the C-ABI, that its output
equals the order efm_fetch_results returns and the oracle's own sorted
output, on two calls in a row that reuse the same scratch.  The file is
named so that pytest collects it last.
"""
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


def _sorted_by_library(efm, net, target):
    import oracle

    with efm.Network(net) as nw:
        (sup, ctr), = efm.enumerate_targets(nw, [target], 30, 4, 0, 2**17)
    # the same order, written by the oracle's own sort
    want, _ = oracle.enumerate_pathways(net, target, oracle.Limits(30, 4, 0, 2**17))
    assert np.array_equal(sup, want)
    return want


def test_noalloc_sort_matches_fetch_order_twice(efm):
    import torch

    net = synth.core()
    rng = np.random.default_rng(5)
    expected = [_sorted_by_library(efm, net, t) for t in (net.targets[2], net.targets[6])]
    assert all(len(e) > 5 for e in expected)
    stream = torch.cuda.current_stream()
    for call, want in enumerate(expected):
        shuffled = want[rng.permutation(len(want))]
        src = torch.from_numpy(shuffled.view(np.int64)).cuda()
        dst = torch.full_like(src, -1)
        rc = efm.efm_sort_supports_noalloc(src.data_ptr(), want.shape[0], want.shape[1], dst.data_ptr(), stream)
        assert rc == 0, efm.status_str(rc)
        torch.cuda.synchronize()
        got = dst.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, want), f"call {call}"


def test_noalloc_sort_rejects_oversize_and_aliasing(efm):
    import torch

    buf = torch.zeros(4, 2, dtype=torch.int64, device="cuda")
    assert efm.efm_sort_supports_noalloc(buf.data_ptr(), efm.EFM_NOALLOC_MAX_ROWS + 1, 2, buf.data_ptr() + 64) == -3
    assert efm.efm_sort_supports_noalloc(buf.data_ptr(), 4, 2, buf.data_ptr()) == -1
    # partly overlapping input and output (output 8 bytes past the input)
    assert efm.efm_sort_supports_noalloc(buf.data_ptr(), 2, 2, buf.data_ptr() + 8) == -1
    assert efm.efm_sort_supports_noalloc(buf.data_ptr() + 8, 2, 2, buf.data_ptr()) == -1
    # adjacent, not overlapping: accepted
    assert efm.efm_sort_supports_noalloc(buf.data_ptr(), 2, 2, buf.data_ptr() + 32) == 0
    torch.cuda.synchronize()
    assert efm.efm_sort_supports_noalloc(buf.data_ptr(), 4, 65, buf.data_ptr() + 64) == -1
