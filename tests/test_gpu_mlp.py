"""The proposal model on the tensor cores against the fp64 reference.

Forward scores and the training gradient come from the library's own
tcgen05 kernels (through the C-ABI) and are compared with oracle/mlp.py on
the same BF16-rounded inputs.  Tolerances follow from the arithmetic:
products of BF16 values are exact in FP32, so the forward pass differs from
fp64 only by FP32 accumulation; the gradient of W1 also rounds dL/dh to BF16
(relative error <= 2^-9 per element) before the tensor-core product.
"""
import numpy as np
import pytest

from oracle import mlp
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


def _rows(rng, n, pos=0.3):
    X = rng.normal(0, 0.6, size=(n, mlp.F)).astype(np.float32)
    X[:, 10] = 1.0
    X[:, 20:64] = 0.0
    y = (rng.random(n) < pos).astype(np.float32)
    return X, y


def _params(rng):
    p = np.zeros(mlp.N_PARAMS, dtype=np.float32)
    p[:mlp.H * mlp.F] = rng.uniform(-0.2, 0.2, size=mlp.H * mlp.F)
    p[mlp.H * mlp.F:-1] = rng.uniform(-0.3, 0.3, size=mlp.H)
    p[-1] = 0.1
    return p


def _rounded(p):
    q = p.astype(np.float32).copy()
    q[:mlp.H * mlp.F] = mlp.bf16_round(q[:mlp.H * mlp.F])
    return q


@pytest.mark.parametrize("n", [1, 128, 1000, 5 * 128 * 152 + 77])
def test_forward_matches_fp64(efm, n):
    rng = np.random.default_rng(n)
    X, _ = _rows(rng, n)
    p = _params(rng)
    m = efm.efm_model_create(1)
    try:
        efm.efm_model_params(m, p)
        got = efm.efm_model_forward(m, X)
    finally:
        efm.efm_model_free(m)
    Xr = mlp.bf16_round(X)
    want, h = mlp.forward(_rounded(p), Xr)
    W1, w2, b2 = mlp.unpack(_rounded(p))
    # FP32 accumulation of exact products: <= K * 2^-24 relative to the sum of |terms| (x4 margin)
    scale_h = np.abs(Xr.astype(np.float64)) @ np.abs(W1).T
    bound = 4 * (128 * 2.0**-24 * scale_h @ np.abs(w2) + 256 * 2.0**-24 * (np.abs(np.maximum(h, 0)) @ np.abs(w2)))
    assert np.all(np.abs(got - want) <= bound + 1e-6), np.max(np.abs(got - want) - bound)


@pytest.mark.parametrize("pos_weight", [1.0, 4.0])
def test_gradient_matches_fp64(efm, pos_weight):
    rng = np.random.default_rng(11)
    n = 3 * 128 * 152 + 45   # several tiles per CTA and a ragged tail
    X, y = _rows(rng, n)
    p = _params(rng)
    m = efm.efm_model_create(2)
    try:
        efm.efm_model_params(m, p)
        efm.efm_model_add_rows(m, X, y)
        g, loss = efm.efm_model_gradient(m, pos_weight)
        assert np.array_equal(efm.efm_model_params(m), p)   # the gradient pass changes nothing
    finally:
        efm.efm_model_free(m)
    Xr = mlp.bf16_round(X).astype(np.float64)
    L, want, dh = mlp.loss_and_grad(_rounded(p), Xr, y, pos_weight)
    assert abs(loss - L) <= 1e-4 * abs(L) + 1e-6
    k = mlp.H * mlp.F
    # W1: BF16 rounding of dL/dh (2^-9 relative, taken as 2^-8) plus FP32 accumulation
    mag = np.abs(dh).T @ np.abs(Xr)
    bound = 2.0**-8 * mag + 1e-6 * np.abs(mag).max()
    err = np.abs(g[:k].reshape(mlp.H, mlp.F) - want[:k].reshape(mlp.H, mlp.F))
    assert np.all(err <= bound), err.max()
    # w2, b2: FP32 all the way
    assert np.allclose(g[k:], want[k:], rtol=1e-3, atol=1e-7)


def test_training_separates_a_learnable_rule(efm):
    rng = np.random.default_rng(3)
    n = 40 * 128
    X, _ = _rows(rng, n)
    y = ((X[:, 0] + 0.5 * X[:, 1] - X[:, 3]) > 0.2).astype(np.float32)
    m = efm.efm_model_create(7)
    try:
        efm.efm_model_add_rows(m, X, y)
        _, l0 = efm.efm_model_gradient(m)
        l1 = efm.efm_model_train(m, epochs=30, batch_tiles=4, lr=3e-3)
        s = efm.efm_model_forward(m, X)
        p_after = efm.efm_model_params(m)
    finally:
        efm.efm_model_free(m)
    acc = np.mean((s > 0) == (y > 0.5))
    assert l1 < 0.5 * l0 and acc > 0.9, (l0, l1, acc)
    # the trained weights reproduce the GPU scores in fp64
    want, _ = mlp.forward(_rounded(p_after), mlp.bf16_round(X))
    assert np.allclose(s, want, rtol=1e-3, atol=1e-3)


def test_trace_rows_and_labels(efm):
    net = synth.core()
    m = efm.efm_model_create(4)
    try:
        with efm.Network(net) as nw:
            efm.efm_model_trace(m, nw.handle, [63, 65], 30, 4, first_k=20, rows_per_level=512)
        n, pos = efm.efm_model_rows(m)
    finally:
        efm.efm_model_free(m)
    assert n > 1000 and 0 < pos < n, (n, pos)


def test_learned_order_gives_identical_first_k(oracle_lib, efm):
    """Any model, trained or not, changes the order only."""
    m = efm.efm_model_create(9)
    try:
        for seed in range(6):
            net = synth.tiny(seed)
            targets = list(net.targets) + [-1]
            with efm.Network(net) as nw:
                for k in (1, 10, 100):
                    got = efm.enumerate_targets(nw, targets, 9, 1, first_k=k, proposal=efm.EFM_LEARNED, model=m)
                    for t, (sup, _) in zip(targets, got):
                        want, _ = oracle_lib.first_k(net, t, k, 9, 1)
                        assert np.array_equal(sup, want), (seed, t, k)
        net = synth.genome()
        with efm.Network(net) as nw:
            for t, k in [(924, 200), (883, 80)]:
                (a, _), = efm.enumerate_targets(nw, [t], 40, 4, 0, 1 << 21, first_k=k)
                (b, _), = efm.enumerate_targets(nw, [t], 40, 4, 0, 1 << 21, first_k=k, proposal=efm.EFM_LEARNED,
                                                model=m)
                want, _ = oracle_lib.first_k(net, t, k, 40, 4)
                assert np.array_equal(a, want) and np.array_equal(b, want), t
    finally:
        efm.efm_model_free(m)


def test_model_argument_rules(efm):
    net = synth.tiny(1)
    m = efm.efm_model_create(1)
    try:
        with efm.Network(net) as nw:
            with pytest.raises(efm.EfmError):   # learned order without a model
                efm.efm_find_pathways(nw.handle, [-1], 8, 1, first_k=3, proposal=efm.EFM_LEARNED)
            with pytest.raises(efm.EfmError):   # a model outside a first-K search
                efm.efm_find_pathways(nw.handle, [-1], 8, 1, proposal=efm.EFM_LEARNED, model=m)
        with pytest.raises(efm.EfmError):
            efm.efm_model_add_rows(m, np.zeros((2, 128)), np.array([0.0, 0.5]))
    finally:
        efm.efm_model_free(m)


def test_trained_model_reaches_k_sooner(efm):
    """What the model gains: trained on traces of 16 genome targets, it
    orders the first-K=1000 searches of 16 other targets.  Where both orders
    certify their answer (no level overflowed the budget), the answers are
    identical and the learned order takes less time in total."""
    net = synth.genome()
    tg = [int(t) for t in net.targets]
    K = 1000
    m = efm.efm_model_create(1)
    try:
        with efm.Network(net) as nw:
            efm.efm_model_trace(m, nw.handle, tg[:16], 40, 4, K, max_frontier=1 << 22, rows_per_level=8192)
            n, pos = efm.efm_model_rows(m)
            assert 0 < pos < n
            efm.efm_model_train(m, epochs=20, batch_tiles=16, lr=1e-3, pos_weight=min(50.0, (n - pos) / pos))

            def best(t, **kw):
                runs = [efm.enumerate_targets(nw, [t], 40, 4, 0, 1 << 22, timing=True, first_k=K, **kw)[0]
                        for _ in range(2)]
                return min(runs, key=lambda r: r[2]["total_ms"])

            plain_ms = learned_ms = 0.0
            both = 0
            for t in tg[128:144]:
                a, ca, ta = best(t)
                b, cb, tb = best(t, proposal=efm.EFM_LEARNED, model=m)
                if ca["status"] & 1 or cb["status"] & 1:
                    continue
                assert np.array_equal(a, b), t
                both += 1
                plain_ms += ta["total_ms"]
                learned_ms += tb["total_ms"]
    finally:
        efm.efm_model_free(m)
    print(f"certified by both: {both}; plain {plain_ms:.1f} ms, learned {learned_ms:.1f} ms")
    assert both >= 4
    assert learned_ms < plain_ms


def test_save_and_load_reproduce_the_scores(efm, tmp_path):
    rng = np.random.default_rng(21)
    X, y = _rows(rng, 700)
    m = efm.efm_model_create(5)
    try:
        efm.efm_model_add_rows(m, X, y)
        efm.efm_model_train(m, epochs=3, batch_tiles=2, lr=1e-3)
        s1 = efm.efm_model_forward(m, X)
        efm.save_model(m, tmp_path / "model.npy")
    finally:
        efm.efm_model_free(m)
    m2 = efm.load_model(tmp_path / "model.npy")
    try:
        s2 = efm.efm_model_forward(m2, X)
    finally:
        efm.efm_model_free(m2)
    assert np.array_equal(s1, s2)
