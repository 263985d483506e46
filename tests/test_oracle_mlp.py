"""Pins of the fp64 proposal-model reference (no GPU needed): central finite
differences of its loss, closed forms at special parameters, and the BF16
rounding rule on hand-picked values."""
import numpy as np

from oracle import mlp


def _rows(rng, n):
    X = rng.normal(0, 0.5, size=(n, mlp.F))
    X[:, 10] = 1.0
    y = (rng.random(n) < 0.3).astype(np.float64)
    return X, y


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    X, y = _rows(rng, 40)
    p = rng.normal(0, 0.1, size=mlp.N_PARAMS)
    L, g, _ = mlp.loss_and_grad(p, X, y, pos_weight=3.0)
    idx = np.concatenate([rng.choice(mlp.H * mlp.F, 60, replace=False),
                          mlp.H * mlp.F + rng.choice(mlp.H, 20, replace=False), [mlp.N_PARAMS - 1]])
    eps = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = eps
        fd = (mlp.loss_and_grad(p + e, X, y, 3.0)[0] - mlp.loss_and_grad(p - e, X, y, 3.0)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_closed_forms():
    rng = np.random.default_rng(6)
    X, y = _rows(rng, 25)
    p = rng.normal(0, 0.1, size=mlp.N_PARAMS)
    p[mlp.H * mlp.F:mlp.H * mlp.F + mlp.H] = 0.0     # w2 = 0: s = b2 everywhere
    b2 = 0.7
    p[-1] = b2
    L, g, dh = mlp.loss_and_grad(p, X, y, pos_weight=2.0)
    wt = np.where(y > 0, 2.0, 1.0)
    sig = 1 / (1 + np.exp(-b2))
    assert np.isclose(L, np.mean(wt * (np.log1p(np.exp(b2)) - y * b2)))
    assert np.isclose(g[-1], np.mean(wt * (sig - y)))
    assert np.all(g[:mlp.H * mlp.F] == 0) and np.all(dh == 0)   # no signal reaches W1 through w2 = 0
    s, _ = mlp.forward(p, X)
    assert np.allclose(s, b2)


def test_bf16_rounding_rule():
    vals = np.array([1.0, 1.0 + 2**-8, 1.0 + 2**-7, 1.0 + 3 * 2**-8, -2.5, 3.0e-39], dtype=np.float32)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even mantissa (1.0) wins;
    # 1 + 3 * 2^-8 is a tie between 1 + 2^-7 and 1 + 2^-6: 1 + 2^-6 is even
    want = np.array([1.0, 1.0, 1.0 + 2**-7, 1.0 + 2**-6, -2.5, 0.0], dtype=np.float32)
    got = mlp.bf16_round(vals)
    assert np.array_equal(got[:5], want[:5])
    assert abs(got[5] - 3.0e-39) <= 2.0**-133   # subnormal: kept to BF16 spacing
