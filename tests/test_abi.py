"""Host-side checks of the C-ABI library (no GPU needed): it builds for
sm_103a, loads, and exports every symbol include/efmgraph.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "efmgraph.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(efm_[a-z_0-9]+)\s*\(", src))
    return sorted(n for n in names if not n.endswith("_fn"))


@pytest.fixture(scope="module")
def lib():
    from paper_1804_02867_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "efm_load_network" in names and "efm_find_pathways" in names and "efm_fetch_results" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_abi():
    from paper_1804_02867_gb300 import efmgraph

    assert set(_declared()) == set(efmgraph.EXPORTS)


def test_status_strings_without_gpu(lib):
    from paper_1804_02867_gb300 import efmgraph

    assert efmgraph.status_str(0) == "ok"
    assert "invalid" in efmgraph.status_str(-1)
    assert "truncated" in efmgraph.status_str(1)


def test_rank_primes_are_prime_and_below_2_31():
    """The minimality kernel's moduli p = 2^31 - c: each is prime, and the
    largest c keeps the two-step reduction within one subtraction."""
    import sympy

    with open(os.path.join(ROOT, "paper_1804_02867_gb300", "csrc", "efm_kernels.cu")) as f:
        src = f.read()
    body = re.search(r"c_prime_c\[kNumPrimes\]\s*=\s*\{([^}]*)\}", src).group(1)
    cs = [int(x) for x in re.findall(r"\d+", body)]
    assert len(cs) == 24 and len(set(cs)) == 24
    for c in cs:
        assert sympy.isprime(2**31 - c)
        assert c < 2**10


def test_load_network_rejects_out_of_range_sizes_on_the_host(lib):
    """The loader validates on the host, before any device call: one internal
    metabolite, one split column or one unit of coefficient past the limits
    of the maximal network is EFM_EINVAL."""
    import numpy as np

    from paper_1804_02867_gb300 import efmgraph, synth

    net = synth.maximal()
    assert net.split_columns() == 4096 and int((net.external == 0).sum()) == 1024

    def load(n_met=net.n_met, n_rxn=net.n_rxn, coef=net.coef, reversible=net.reversible, external=net.external):
        with pytest.raises(efmgraph.EfmError) as e:
            efmgraph.efm_load_network(n_met, n_rxn, net.row_ptr, net.col_idx, coef, reversible, external, stream=0)
        return e.value.code

    ext = net.external.copy()
    ext[net.targets[1]] = 0  # 1025 internal metabolites
    assert load(external=ext) == -1
    rev = net.reversible.copy()
    rev[np.nonzero(rev == 0)[0][-1]] = 1  # 4097 split columns
    assert load(reversible=rev) == -1
    coef = net.coef.copy()
    coef[np.argmax(np.abs(coef))] = -(synth.MAX_COEF + 1)
    assert load(coef=coef) == -1
    coef = net.coef.copy()
    coef[0] = 0
    assert load(coef=coef) == -1


def test_wait_bounds_agree_and_null_handles_are_refused(lib):
    """The traversal kernels' poll bound equals the one the failure-path
    check runs (both 2^20), and the check refuses a null network on the host."""
    from paper_1804_02867_gb300 import efmgraph

    with open(os.path.join(ROOT, "paper_1804_02867_gb300", "csrc", "efm_kernels.cu")) as f:
        kern = re.search(r"constexpr int kSpinLimit = ([^;]+);", f.read()).group(1)
    with open(os.path.join(ROOT, "paper_1804_02867_gb300", "csrc", "efm_internal.cuh")) as f:
        shared = re.search(r"constexpr int kWaitSpinLimit = ([^;]+);", f.read()).group(1)
    assert kern.strip() == shared.strip() == "1 << 20"
    with pytest.raises(efmgraph.EfmError) as e:
        efmgraph.efm_check_bounded_wait(None)
    assert e.value.code == -1
