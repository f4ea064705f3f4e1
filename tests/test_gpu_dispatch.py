"""Learned dispatcher on the GPU: features and gradients against the CPU
reference, on-GPU training, save/load, and BMLP_AUTO using the model."""
import numpy as np
import pytest
import torch

import oracle
from oracle import dispatch_ref as ref
import workloads as wl

pkg = pytest.importorskip("paper_2408_10369_gb300")
from paper_2408_10369_gb300 import bmlp  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture()
def ctx():
    c = pkg.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("index", [0, 1, 2, 3, 7, 11, 12, 21])
def test_features_match_reference(ctx, index):
    g = wl.corpus_graph(index, n_min=200, n_max=3000)
    n = g["n"]
    m = wl.dense_u8(n, g["indptr"], g["indices"])
    for fmt, R in ((bmlp.BMLP_FMT_U8, m), (bmlp.BMLP_FMT_PACKED64, wl.pack_rows(m).view(np.int64))):
        f = ctx.dispatch_features(torch.from_numpy(np.ascontiguousarray(R)).cuda(), n, fmt=fmt)
        np.testing.assert_allclose(f, ref.features(m), rtol=2e-5, atol=1e-6)


def test_gradient_matches_reference(ctx):
    rng = np.random.default_rng(1)
    p = rng.normal(0, 0.2, ref.NP).astype(np.float32)
    mu = rng.normal(0, 1, ref.NF).astype(np.float32)
    sig = rng.uniform(0.5, 2.0, ref.NF).astype(np.float32)
    X = (rng.normal(0, 1, (300, ref.NF)) * sig + mu).astype(np.float32)
    Y = rng.normal(0, 2, (300, ref.NV)).astype(np.float32)
    C = (rng.random((300, ref.NV)) < 0.25).astype(np.uint8)
    ctx.dispatch_set_params(p, mu, sig)
    loss, g = ctx.dispatch_loss_grad(X, Y, C)
    p16 = p.astype(np.float16).astype(np.float64)      # the kernels use FP16 weights
    want_loss, want_g = ref.loss_grad(p16, mu, sig, X, Y, C)
    assert abs(loss - want_loss) <= 1e-4 * abs(want_loss) + 1e-6
    np.testing.assert_allclose(g, want_g, rtol=2e-3, atol=2e-5 * np.abs(want_g).max())
    pred, choice = ctx.dispatch_predict(X[:50])
    want = ref.forward(p16, mu, sig, X[:50])
    np.testing.assert_allclose(pred, want, rtol=1e-3, atol=1e-3)
    np.testing.assert_array_equal(choice, np.argmin(pred, 1) + 1)


def test_training_learns_and_roundtrips(ctx, tmp_path):
    rng = np.random.default_rng(2)
    X = rng.normal(0, 1, (3000, ref.NF)).astype(np.float32)
    A = rng.normal(0, 1, (ref.NF, ref.NV))
    Y = (np.tanh(X @ A) * 3 + X[:, :4] ** 2).astype(np.float32)
    C = np.zeros_like(Y, np.uint8)
    base = float(((Y - Y.mean(0)) ** 2).mean())
    loss = ctx.dispatch_train(X, Y, C, epochs=60, batch=256, lr=3e-3, weight_decay=0.0, seed=3)
    assert loss < 0.15 * base, (loss, base)
    pred, _ = ctx.dispatch_predict(X[:100])
    path = tmp_path / "model.bin"
    ctx.dispatch_save(path)
    c2 = pkg.Context(0)
    try:
        c2.dispatch_load(path)
        pred2, _ = c2.dispatch_predict(X[:100])
        np.testing.assert_array_equal(pred, pred2)
        p, mu, sg = c2.dispatch_get_params()
        p1, mu1, sg1 = ctx.dispatch_get_params()
        np.testing.assert_array_equal(p, p1)
    finally:
        c2.close()


@pytest.mark.parametrize("variant", [2, 3, 4])
def test_auto_runs_the_predicted_variant(ctx, variant):
    """With a model whose output biases favour one variant, BMLP_AUTO runs it
    and the closure is still exact."""
    p = np.zeros(ref.NP, np.float32)
    p[ref.OB3:ref.NP] = 5.0
    p[ref.OB3 + variant - 1] = -5.0
    ctx.dispatch_set_params(p, np.zeros(ref.NF, np.float32), np.ones(ref.NF, np.float32))
    n = 700
    ip, ix = wl.er_graph(n, 1.3, 4)
    R = torch.from_numpy(wl.dense_u8(n, ip, ix)).cuda()
    out = torch.zeros_like(R)
    ctx.rms(R, n, out)
    torch.cuda.synchronize()
    assert ctx.stats()["variant"] == variant
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.closure(n, ip, ix))


def test_budget_censors_a_long_run(ctx):
    n = 8192
    ip, ix = wl.er_graph(n, 4.0, 0)
    P = torch.from_numpy(wl.pack_rows(wl.dense_u8(n, ip, ix)).view(np.int64)).cuda()
    out = torch.zeros_like(P)
    with pytest.raises(bmlp.BmlpError) as e:
        ctx.rms(P, n, out, fmt=bmlp.BMLP_FMT_PACKED64, variant="rms_packed", budget_ns=200_000)
    assert e.value.status == bmlp.BMLP_ERR_BUDGET
    ctx.rms(P, n, out, fmt=bmlp.BMLP_FMT_PACKED64, variant="rms_packed")   # the context is still usable


def test_dispatched_heldout_corpus_matches_oracle(ctx):
    """The committed model on 40 held-out corpus graphs (seeds 9,000-9,039,
    n up to 8,192): the dispatched pipeline (features, prediction, small
    squaring problems grouped in one batch, the rest one by one with their
    predicted variant) returns the oracle's closure for every graph, every bit."""
    import os

    from paper_2408_10369_gb300 import dispatch_corpus as dc
    model = os.path.join(os.path.dirname(pkg.__file__), "dispatch_model.bin")
    ctx.dispatch_load(model)
    rows = [{"index": i} for i in range(9000, 9040)]
    rep, graphs, outs = dc.live_pipeline(ctx, rows, 8192, return_outputs=True)
    assert rep["live_bit_mismatches"] == 0 and rep["live_tc_only_bit_mismatches"] == 0
    for (g, _), o in zip(graphs, outs):
        n = g["n"]
        got = o.cpu().numpy().view(np.uint64)
        for r0, blk in oracle.closure_bits_chunks(n, g["indptr"], g["indices"], 4096):
            np.testing.assert_array_equal(got[r0:r0 + blk.shape[0], :blk.shape[1]], blk)


def test_choose_many_matches_single_calls(ctx):
    """bmlp_dispatch_choose_many on 24 corpus graphs of mixed sizes and
    formats (packed rows read in place, misaligned rows that are copied, u8
    and host-memory inputs converted) gives the features and the choices of
    bmlp_dispatch_features + bmlp_dispatch_predict, one matrix at a time; with
    no model it refuses, and an empty list is a no-op."""
    import os

    from paper_2408_10369_gb300 import dispatch_corpus as dc
    fresh = pkg.Context(0)
    try:
        with pytest.raises(bmlp.BmlpError) as e:
            fresh.dispatch_choose_many([torch.zeros((64, 2), dtype=torch.int64, device="cuda")], [64],
                                       fmt=bmlp.BMLP_FMT_PACKED64)
        assert e.value.status == bmlp.BMLP_ERR_UNSUPPORTED
    finally:
        fresh.close()
    ctx.dispatch_load(os.path.join(os.path.dirname(pkg.__file__), "dispatch_model.bin"))
    assert len(ctx.dispatch_choose_many([], [], fmt=bmlp.BMLP_FMT_PACKED64)) == 0
    graphs = [dc.graph_on_device(i, 8192) for i in range(9040, 9064)]
    mats, ns = [], []
    for k, (g, P) in enumerate(graphs):
        n = g["n"]
        if k % 4 == 1:      # the rows at an 8-byte but not 16-byte aligned address: converted, not read in place
            w = P.shape[1]
            flat = torch.zeros(n * w + 1, dtype=torch.int64, device="cuda")
            Q = flat[1:].view(n, w)
            Q.copy_(P)
            mats.append(Q)
        elif k % 4 == 2:    # host memory
            mats.append(P.cpu())
        else:
            mats.append(P)
        ns.append(n)
    choice, feats = ctx.dispatch_choose_many(mats, ns, fmt=bmlp.BMLP_FMT_PACKED64, features=True)
    single = np.stack([ctx.dispatch_features(P, g["n"], fmt=bmlp.BMLP_FMT_PACKED64) for g, P in graphs])
    _, single_choice = ctx.dispatch_predict(single)
    np.testing.assert_allclose(feats, single, rtol=1e-6, atol=1e-6)
    np.testing.assert_array_equal(choice, single_choice)
    # the same matrices as 0/1 bytes
    u8 = [torch.from_numpy(wl.unpack_rows(P.cpu().numpy().view(np.uint64), g["n"]).astype(np.uint8)).cuda()
          for g, P in graphs[:6]]
    c8, f8 = ctx.dispatch_choose_many(u8, ns[:6], fmt=bmlp.BMLP_FMT_U8, features=True)
    np.testing.assert_allclose(f8, single[:6], rtol=1e-6, atol=1e-6)
    np.testing.assert_array_equal(c8, single_choice[:6])
