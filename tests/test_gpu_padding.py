"""Packed inputs whose padding bits (columns >= n of each row's last word) are
set: the header says they are ignored. Every closure variant, a selective
query batch large enough for the bit-sliced path, and the dispatcher's
features give the same result as for the clean rows (which the parity tests
check against the oracle), and the output padding bits stay zero."""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl

pkg = pytest.importorskip("paper_2408_10369_gb300")
from paper_2408_10369_gb300 import bmlp  # noqa: E402

pytestmark = pytest.mark.gpu
F = bmlp.BMLP_FMT_PACKED64


@pytest.fixture(scope="module")
def ctx():
    c = pkg.Context(0)
    yield c
    c.close()


def dirty(P, n):
    """A copy of the packed rows with every padding bit of the last word set."""
    Q = P.clone()
    if n % 64:
        pad = np.uint64(~((1 << (n % 64)) - 1) & 0xFFFFFFFFFFFFFFFF).view(np.int64)
        Q[:, -1] |= int(pad)
    return Q


def graph(n, d, seed):
    ip, ix = wl.er_graph(n, d, seed)
    return ip, ix, torch.from_numpy(wl.csr_to_packed(n, ip, ix).view(np.int64)).cuda()


@pytest.mark.parametrize("variant", ["rms_tc", "rms_packed", "smp_packed"])
@pytest.mark.parametrize("n,d", [(4100, 3.0), (8257, 1.2)])
def test_closure_ignores_padding_bits(ctx, variant, n, d):
    ip, ix, P = graph(n, d, 7)
    clean, got = torch.zeros_like(P), torch.zeros_like(P)
    ctx.rms(P, n, clean, fmt=F, variant=variant)
    ctx.rms(dirty(P, n), n, got, fmt=F, variant=variant)
    torch.cuda.synchronize()
    assert torch.equal(got, clean)
    want, _, _ = oracle.reach_rows(n, ip, ix, np.arange(0, n, 97, dtype=np.int32))
    rows = wl.unpack_rows(got.cpu().numpy().view(np.uint64)[::97], n)
    np.testing.assert_array_equal(rows, want)
    if n % 64:
        assert int((got[:, -1].cpu().numpy().view(np.uint64) >> np.uint64(n % 64)).max()) == 0


def test_query_batch_ignores_padding_bits(ctx):
    n, q = 4100, 128
    ip, ix, P = graph(n, 6.0, 3)
    src = torch.from_numpy(wl.query_rows(n, q, 1, 64, 0).view(np.int64)).cuda()
    clean = torch.zeros((q, P.shape[1]), dtype=torch.int64, device="cuda")
    got = torch.zeros_like(clean)
    ctx.smp(P, n, src, q, clean, fmt=F)
    ctx.smp(dirty(P, n), n, src, q, got, fmt=F)
    torch.cuda.synchronize()
    assert torch.equal(got, clean)


def test_features_ignore_padding_bits(ctx):
    n = 4100
    _, _, P = graph(n, 3.0, 5)
    a = ctx.dispatch_features(P, n, fmt=F)
    b = ctx.dispatch_features(dirty(P, n), n, fmt=F)
    np.testing.assert_array_equal(a, b)
