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


def _identity_params(sign2=1.0):
    """W1 = [I_16; 0], W2 = sign2 * I_64, W3 = the first four rows of I_64, zero biases."""
    p = np.zeros(ref.NP)
    W1 = np.zeros((ref.NH, ref.NF))
    W1[:ref.NF, :ref.NF] = np.eye(ref.NF)
    p[ref.OW1:ref.OB1] = W1.ravel()
    p[ref.OW2:ref.OB2] = (sign2 * np.eye(ref.NH)).ravel()
    W3 = np.zeros((ref.NV, ref.NH))
    W3[:, :ref.NV] = np.eye(ref.NV)
    p[ref.OW3:ref.OB3] = W3.ravel()
    return p


def test_forward_closed_forms():
    """The forward pass against values fixed by construction: layers that copy
    their input give the normalised features back; a ReLU zeroes negatives at
    either hidden layer; output biases add; the normalisation is (x - mu) / sigma
    once."""
    rng = np.random.default_rng(1)
    mu = rng.normal(0, 3, ref.NF)
    sig = rng.uniform(0.5, 4.0, ref.NF)
    z = rng.uniform(0.1, 5.0, (7, ref.NF))           # normalised inputs, all positive
    X = mu + sig * z
    p = _identity_params()
    y = ref.forward(p, mu, sig, X)
    assert np.allclose(y, z[:, :ref.NV], rtol=0, atol=1e-12)
    # negative normalised inputs are cut by the first ReLU: with W2[1][1] = -1 a negative input that got
    # through it would come out positive
    zn = z.copy()
    zn[:, 1] = -zn[:, 1]
    pn = p.copy()
    pn[ref.OW2 + 1 * ref.NH + 1] = -1.0
    y = ref.forward(pn, mu, sig, mu + sig * zn)
    assert np.all(y[:, 1] == 0.0) and np.allclose(y[:, 0], z[:, 0], atol=1e-12)
    # W2 = -I: every second-layer pre-activation is negative, so the second ReLU leaves zeros
    y = ref.forward(_identity_params(-1.0), mu, sig, X)
    assert np.all(y == 0.0)
    # output biases are added as they are; hidden biases pass through the copies
    p2 = p.copy()
    p2[ref.OB3:ref.NP] = [1.0, -2.0, 0.5, 3.0]
    p2[ref.OB1:ref.OB1 + ref.NV] = 0.25
    y = ref.forward(p2, mu, sig, X)
    assert np.allclose(y, z[:, :ref.NV] + 0.25 + np.array([1.0, -2.0, 0.5, 3.0]), atol=1e-12)


def test_loss_values_by_hand():
    """Loss = mean over samples x 4 outputs of the squared log2-time error; a
    censored time costs nothing when the prediction is above it."""
    mu = np.zeros(ref.NF)
    sig = np.ones(ref.NF)
    x = np.zeros((1, ref.NF))
    x[0, :4] = [1.0, 2.0, 3.0, 4.0]                  # the identity network predicts these
    t = np.array([[0.0, 2.0, 5.0, 1.0]])              # errors 1, 0, -2, 3
    p = _identity_params()
    loss, _ = ref.loss_grad(p, mu, sig, x, t, np.zeros((1, 4), np.uint8))
    assert abs(loss - (1 + 0 + 4 + 9) / 4.0) < 1e-12
    # the last output's time is censored and predicted above it: no cost; a censored one predicted
    # below still costs (error -2 on output 2)
    loss, _ = ref.loss_grad(p, mu, sig, x, t, np.array([[0, 0, 1, 1]], np.uint8))
    assert abs(loss - (1 + 0 + 4 + 0) / 4.0) < 1e-12
    # two samples: the mean runs over both samples and all outputs
    x2 = np.vstack([x, np.zeros((1, ref.NF))])
    t2 = np.vstack([t, np.full((1, 4), 2.0)])         # second sample: predictions 0, errors -2 each
    loss, _ = ref.loss_grad(p, mu, sig, x2, t2, np.zeros((2, 4), np.uint8))
    assert abs(loss - (14.0 + 16.0) / 8.0) < 1e-12
