"""Pins of the dispatcher's CPU reference: finite differences for the loss
gradient, closed forms for the features."""
import numpy as np

from oracle import dispatch_ref as ref


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.3, ref.NP)
    mu = rng.normal(0, 1, ref.NF)
    sig = rng.uniform(0.5, 2.0, ref.NF)
    X = rng.normal(0, 1, (40, ref.NF)) * sig + mu
    Y = rng.normal(0, 1, (40, ref.NV))
    C = (rng.random((40, ref.NV)) < 0.3).astype(np.uint8)
    loss, g = ref.loss_grad(p, mu, sig, X, Y, C)
    idx = rng.choice(ref.NP, 400, replace=False)
    h = 1e-6
    for k in idx:
        e = np.zeros(ref.NP)
        e[k] = h
        num = (ref.loss_grad(p + e, mu, sig, X, Y, C)[0] - ref.loss_grad(p - e, mu, sig, X, Y, C)[0]) / (2 * h)
        assert abs(num - g[k]) <= 1e-6 + 1e-5 * abs(num), (k, num, g[k])
    # censoring: predictions above a censored time cost nothing
    y = ref.forward(p, mu, sig, X)
    Cc = np.ones_like(C)
    l2, g2 = ref.loss_grad(p, mu, sig, X, y - 1.0, Cc)
    assert l2 == 0.0 and not g2.any()


def test_features_closed_forms():
    n = 200
    empty = np.zeros((n, n), np.uint8)
    f = ref.features(empty)
    assert f[0] == np.log2(n) and f[1] == 0 and f[2] == 0 and f[5] == 1 and f[8] == 1 and f[15] == 1
    chain = np.eye(n, k=1, dtype=np.uint8)
    f = ref.features(chain)
    assert abs(f[2] - (n - 1) / n) < 1e-12 and f[10] == 0 and abs(f[12] - 1.0 / n) < 1e-12
    assert abs(f[13] - 1.0 / n) < 1e-12              # two steps from i reach only i + 2
    sym = chain | chain.T
    f = ref.features(sym)
    assert f[10] == 1.0                              # every sampled edge is reciprocated
    full = 1 - np.eye(n, dtype=np.uint8)
    f = ref.features(full)
    assert abs(f[2] - (n - 1)) < 1e-12 and f[3] == 0 and abs(f[13] - 1.0) < 1e-12 and f[9] == 0
