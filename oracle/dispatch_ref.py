"""CPU reference (float64) of the learned dispatcher: the 16 graph features
and the 16 -> 64 -> 64 -> 4 MLP loss and gradient.

TEST INFRASTRUCTURE ONLY (same rules as the rest of ``oracle``). The
definitions follow the documentation of ``bmlp_dispatch_*`` in
include/bmlp.h; the paper has no dispatcher, so the loss gradient is pinned by
finite differences in ``tests/test_dispatch_ref.py``.
"""
from __future__ import annotations

import numpy as np

NF, NH, NV = 16, 64, 4
OW1 = 0
OB1 = OW1 + NH * NF
OW2 = OB1 + NH
OB2 = OW2 + NH * NH
OW3 = OB2 + NH
OB3 = OW3 + NV * NH
NP = OB3 + NV
NSAMPLE, NPROBE, NBRANCH = 1024, 64, 64


def features(m: np.ndarray) -> np.ndarray:
    """The 16 features of a dense 0/1 matrix (rows = sources)."""
    m = (np.asarray(m) != 0).astype(np.int64)
    n = m.shape[0]
    N = float(n)
    out = m.sum(1)
    nnz = float(out.sum())
    mean = nnz / N
    var = max(float((out.astype(np.float64) ** 2).sum()) / N - mean * mean, 0.0)
    ns = min(n, NSAMPLE)
    rows = np.array([k * n // ns for k in range(ns)], np.int64)
    sub = m[rows]
    indeg = sub.sum(0).astype(np.float64)
    scale = N / ns
    imean = indeg.sum() / N * scale
    ivar = max((indeg ** 2).sum() / N * scale * scale - imean * imean, 0.0)
    ii, jj = np.nonzero(sub)
    src = rows[ii]
    se = max(float(len(jj)), 1.0)
    recip = float(m[jj, src].sum())
    local = float(np.abs(jj - src).sum())
    words = (m.shape[1] + 63) // 64
    padded = np.zeros((n, words * 64), np.int64)
    padded[:, :n] = m
    nzw = float((padded.reshape(n, words, 64).sum(2) > 0).sum())
    npr = min(ns, NPROBE)
    p1 = p2 = dead = 0.0
    for k in range(npr):
        i = rows[k]
        cols = np.nonzero(m[i])[0]
        p1 += len(cols)
        br = cols[:NBRANCH]
        reach = m[br].any(0).sum() if len(br) else 0
        p2 += reach
        dead += reach == 0
    p1 /= npr
    p2 /= npr
    f = np.zeros(NF, np.float64)
    f[0] = np.log2(N)
    f[1] = np.log2(1.0 + nnz)
    f[2] = mean
    f[3] = np.sqrt(var)
    f[4] = out.max() / N
    f[5] = (out == 0).sum() / N
    f[6] = np.sqrt(ivar)
    f[7] = indeg.max() * scale / N
    f[8] = (indeg == 0).sum() / N
    f[9] = np.trace(m) / N
    f[10] = recip / se
    f[11] = nzw / (N * np.ceil(N / 64.0))
    f[12] = local / se / N
    f[13] = p2 / N
    f[14] = np.log2((p2 + 1.0) / (p1 + 1.0))
    f[15] = dead / npr
    return f


def unpack(params):
    p = np.asarray(params, np.float64)
    W1 = p[OW1:OB1].reshape(NH, NF)
    b1 = p[OB1:OW2]
    W2 = p[OW2:OB2].reshape(NH, NH)
    b2 = p[OB2:OW3]
    W3 = p[OW3:OB3].reshape(NV, NH)
    b3 = p[OB3:NP]
    return W1, b1, W2, b2, W3, b3


def forward(params, mu, sig, X):
    """Predictions (m x 4) of the MLP on raw features X (m x 16)."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    x = (np.asarray(X, np.float64) - np.asarray(mu, np.float64)) / np.asarray(sig, np.float64)
    h1 = np.maximum(x @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ W3.T + b3


def loss_grad(params, mu, sig, X, Y, C):
    """Loss = mean over samples and outputs of d^2, d = y - t, with d := 0
    where the time is censored and y > t; and its gradient (NP,)."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    x = (np.asarray(X, np.float64) - np.asarray(mu, np.float64)) / np.asarray(sig, np.float64)
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3.T + b3
    d = y - np.asarray(Y, np.float64)
    d[(np.asarray(C) != 0) & (d > 0)] = 0.0
    m = x.shape[0]
    loss = float((d ** 2).sum() / (m * NV))
    dy = 2.0 * d / (m * NV)
    g = np.zeros(NP, np.float64)
    g[OW3:OB3] = (dy.T @ h2).ravel()
    g[OB3:NP] = dy.sum(0)
    dh2 = (dy @ W3) * (z2 > 0)
    g[OW2:OB2] = (dh2.T @ h1).ravel()
    g[OB2:OW3] = dh2.sum(0)
    dh1 = (dh2 @ W2) * (z1 > 0)
    g[OW1:OB1] = (dh1.T @ x).ravel()
    g[OB1:OW2] = dh1.sum(0)
    return loss, g
