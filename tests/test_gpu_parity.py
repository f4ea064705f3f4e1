"""Bit-exact parity of the CUDA library (through the C ABI) with the CPU oracle.

Sizes span several 128 x 256 tensor-core tiles and ragged tails (n not a
multiple of 64 / 128 / 256), degenerate inputs (empty, n = 1, self-loop,
complete graph, chain, cycle) and the paper's worked examples.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl
from golden_io import matrix, read_facts

pkg = pytest.importorskip("paper_2408_10369_gb300")

pytestmark = pytest.mark.gpu

CLOSURE_VARIANTS = ["rms_tc", "rms_packed", "smp_packed", "smp_tc"]


@pytest.fixture(scope="module")
def ctx():
    c = pkg.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_rms(ctx, dense, variant, fmt="u8", **kw):
    n = dense.shape[0]
    if fmt == "u8":
        R = dev(dense)
        out = torch.zeros_like(R)
        it = ctx.rms(R, n, out, fmt=pkg.BMLP_FMT_U8, variant=variant, **kw)
        torch.cuda.synchronize()
        return out.cpu().numpy(), it
    P = wl.pack_rows(dense)
    R = dev(P.view(np.int64))
    out = torch.zeros_like(R)
    it = ctx.rms(R, n, out, fmt=pkg.BMLP_FMT_PACKED64, variant=variant, **kw)
    torch.cuda.synchronize()
    return wl.unpack_rows(out.cpu().numpy().view(np.uint64), n), it


def er_case(n, d, seed):
    ip, ix = wl.er_graph(n, d, seed)
    return ip, ix, wl.dense_u8(n, ip, ix)


# ----------------------------------------------------------- closures --
@pytest.mark.parametrize("variant", CLOSURE_VARIANTS)
@pytest.mark.parametrize("n,d,seed", [(1, 0.0, 0), (2, 1.0, 1), (3, 1.0, 2), (63, 1.2, 3), (64, 1.5, 4),
                                      (65, 2.0, 5), (127, 1.0, 6), (128, 1.3, 7), (129, 0.9, 8), (255, 1.1, 9),
                                      (257, 1.6, 10), (600, 1.2, 11), (1000, 2.0, 12)])
def test_closure_er(ctx, variant, n, d, seed):
    ip, ix, m = er_case(n, d, seed)
    want = oracle.closure(n, ip, ix)
    got, it = run_rms(ctx, m, variant)
    np.testing.assert_array_equal(got, want)
    if variant.startswith("rms"):
        assert it == oracle.rms_iterations(oracle.longest_shortest_path(n, ip, ix))


@pytest.mark.parametrize("variant", CLOSURE_VARIANTS)
def test_closure_special(ctx, variant):
    for n in (1, 5, 130, 300):
        cases = {
            "empty": np.zeros((n, n), np.uint8),
            "self": np.eye(n, dtype=np.uint8),
            "complete": (1 - np.eye(n, dtype=np.uint8)).astype(np.uint8),
            "chain": np.eye(n, k=1, dtype=np.uint8),
            "cycle": np.roll(np.eye(n, dtype=np.uint8), 1, axis=1),
        }
        for name, m in cases.items():
            want = oracle.warshall(m) if n <= 130 else oracle.closure(n, *wl.csr_from_dense(m))
            got, it = run_rms(ctx, m, variant)
            np.testing.assert_array_equal(got, want, err_msg="%s n=%d" % (name, n))
            if variant.startswith("rms") and name == "empty":
                assert it == 1


@pytest.mark.parametrize("variant", ["rms_tc", "rms_packed", "smp_packed"])
def test_closure_packed_format_and_reflexive(ctx, variant):
    n = 333
    ip, ix, m = er_case(n, 1.4, 21)
    want = oracle.closure(n, ip, ix)
    got, _ = run_rms(ctx, m, variant, fmt="packed")
    np.testing.assert_array_equal(got, want)
    got, _ = run_rms(ctx, m, variant, reflexive=True)
    np.testing.assert_array_equal(got, want | np.eye(n, dtype=np.uint8))


def test_nonzero_bytes_count_as_one(ctx):
    n = 200
    ip, ix, m = er_case(n, 1.5, 3)
    noisy = m * np.uint8(7) + (m * np.uint8(200))
    got, _ = run_rms(ctx, noisy.astype(np.uint8), "rms_tc")
    np.testing.assert_array_equal(got, oracle.closure(n, ip, ix))


def test_host_buffers(ctx):
    """Host (numpy) input and output: the library stages them itself."""
    n = 400
    ip, ix, m = er_case(n, 1.2, 4)
    out = np.zeros_like(m)
    ctx.rms(m, n, out, variant="rms_tc")
    np.testing.assert_array_equal(out, oracle.closure(n, ip, ix))


def test_p1_example_on_gpu(ctx):
    consts, facts = read_facts("p1_edge_path.txt")
    edge = matrix(consts, facts["edge"])
    for v in CLOSURE_VARIANTS:
        got, _ = run_rms(ctx, edge, v)
        np.testing.assert_array_equal(got, matrix(consts, facts["path"]))


def test_p3_p5_example_on_gpu(ctx):
    consts, facts = read_facts("p3p5_isforeign.txt")
    n = len(consts)
    contains = matrix(consts, facts["contains"])
    adjoins = matrix(consts, facts["adjoins"])
    for v in ("rms_tc", "rms_packed"):
        has_place, _ = run_rms(ctx, contains, v)
        base = (adjoins | adjoins.T).astype(np.uint8)
        rec = np.ascontiguousarray(has_place.T)
        out = torch.zeros((n, n), dtype=torch.uint8, device="cuda")
        ctx.compose(dev(base), dev(rec), n, out, variant=v)
        torch.cuda.synchronize()
        ipo = out.cpu().numpy()
        np.testing.assert_array_equal(ipo, matrix(consts, facts["not_isForeign"]))
        assert int((1 - ipo).sum()) == n * n - 4


# ---------------------------------------------------------------- SMP --
@pytest.mark.parametrize("variant", ["smp_packed", "smp_tc"])
@pytest.mark.parametrize("n,d,q,seed", [(2000, 2000 * 2 / 2000, 1, 0), (2000, 2.0, 16, 1), (129, 1.0, 3, 2),
                                        (700, 1.3, 200, 3), (1500, 0.8, 130, 4)])
def test_smp_er(ctx, variant, n, d, q, seed):
    ip, ix, m = er_case(n, d, seed)
    src = wl.query_rows(n, q, 1, 16, seed)
    want, levels = oracle.smp(n, ip, ix, src)
    out = torch.zeros((q, src.shape[1]), dtype=torch.int64, device="cuda")
    it = ctx.smp(dev(m), n, dev(src.view(np.int64)), q, out, variant=variant)
    torch.cuda.synchronize()
    got = wl.unpack_rows(out.cpu().numpy().view(np.uint64), n)
    np.testing.assert_array_equal(got, want)
    assert it == int(levels.max()) + 1


@pytest.mark.parametrize("variant", ["smp_packed", "smp_tc"])
def test_smp_powerlaw_packed_input(ctx, variant):
    n, q = 3000, 64
    ip, ix = wl.powerlaw_csr(n, 2.1, 1000, 0)
    P = wl.pack_rows(wl.dense_u8(n, ip, ix))
    src = wl.query_rows(n, q, 1, 64, 1)
    want, _ = oracle.smp(n, ip, ix, src)
    out = torch.zeros((q, src.shape[1]), dtype=torch.int64, device="cuda")
    ctx.smp(dev(P.view(np.int64)), n, dev(src.view(np.int64)), q, out, fmt=pkg.BMLP_FMT_PACKED64, variant=variant)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(wl.unpack_rows(out.cpu().numpy().view(np.uint64), n), want)


# ------------------------------------------- long shortest paths --
def shortcut_case(n, shape, seed):
    """A chain (i -> i+1) or a right/down grid plus round(1 % of n) random
    shortcuts: many frontier heads scattered over the row, hundreds of levels."""
    if shape == "grid":
        side = max(2, int(np.sqrt(n)))
        idx = np.arange(n)
        right = idx[(idx % side + 1 < side) & (idx + 1 < n)]
        down = idx[idx + side < n]
        src, dst = np.concatenate([right, down]), np.concatenate([right + 1, down + side])
    else:
        src = np.arange(n - 1)
        dst = src + 1
    a, b = wl.random_pairs(n, max(1, round(0.01 * n)), seed)
    return wl.csr_from_pairs(n, np.concatenate([src, a]), np.concatenate([dst, b]))


@pytest.mark.parametrize("variant", CLOSURE_VARIANTS)
@pytest.mark.parametrize("n,shape,seed", [(3000, "chain", 1), (2500, "grid", 2), (4500, "chain", 3)])
def test_closure_long_paths(ctx, variant, n, shape, seed):
    ip, ix = shortcut_case(n, shape, seed)
    want = oracle.closure(n, ip, ix)
    got, it = run_rms(ctx, wl.dense_u8(n, ip, ix), variant, fmt="packed")
    np.testing.assert_array_equal(got, want)
    if variant == "smp_packed" and n >= 4096:
        # a path-like relation is squared before the frontier expansion (same closure, fewer levels)
        assert ctx.stats()["frontier_squarings"] >= 1


@pytest.mark.parametrize("n,seed", [(2560, 1), (2597, 2)])
def test_packed_squaring_forms(ctx, n, seed):
    """Whole-row bit-row squarings in both forms: edges only into the columns
    64 w keep one bit per nonzero word through every squaring, while more than
    half the words are nonzero from the start. The first whole-row step runs
    on the Four Russians tables (its input's bits per word are not counted
    yet), the later ones gather the named rows."""
    rng = np.random.default_rng(seed)
    cols = np.arange(0, n, 64)
    keep = rng.random((n, len(cols))) < 0.6
    src = np.repeat(np.arange(n), keep.sum(1))
    dst = np.concatenate([cols[k] for k in keep])
    ip, ix = wl.csr_from_pairs(n, src, dst)
    want = oracle.closure(n, ip, ix)
    got, it = run_rms(ctx, wl.dense_u8(n, ip, ix), "rms_packed", fmt="packed")
    np.testing.assert_array_equal(got, want)
    st = ctx.stats()
    assert st["sparse_squarings"] == 0 and it >= 2
    assert st["table_squarings"] == 1


def test_squaring_operand_forms(ctx):
    """Dense R: every squaring on packed E2M1 operands. Block-sparse R (a
    chain with shortcuts): E4M3 squarings with skipped K blocks first, E2M1
    once R is dense; the switch keeps the bits."""
    ip, ix, m = er_case(1500, 3.0, 21)
    got, it = run_rms(ctx, m, "rms_tc")
    np.testing.assert_array_equal(got, oracle.closure(1500, ip, ix))
    st = ctx.stats()
    assert st["e2m1_products"] == st["product_launches"] == it
    n = 4500
    ip, ix = shortcut_case(n, "chain", 3)
    want = oracle.closure(n, ip, ix)
    got, it = run_rms(ctx, wl.dense_u8(n, ip, ix), "rms_tc", tc_only=True)
    np.testing.assert_array_equal(got, want)
    st = ctx.stats()
    assert 0 < st["e2m1_products"] < st["product_launches"] == it
    # by default the sparse first squarings run on bit rows; the tensor cores finish
    got, it2 = run_rms(ctx, wl.dense_u8(n, ip, ix), "rms_tc")
    np.testing.assert_array_equal(got, want)
    st = ctx.stats()
    assert st["sparse_squarings"] >= 1
    assert st["sparse_squarings"] + st["product_launches"] + st["thin_squarings"] == it2 == it


@pytest.mark.parametrize("n,d,seed,fmt", [(1500, 3.0, 21, "u8"), (1000, 1.4, 22, "packed"), (777, 2.5, 23, "u8")])
def test_e4m3_only_option(ctx, n, d, seed, fmt):
    """options.e4m3_only keeps every tensor-core squaring on E4M3 operands
    (kind::f8f6f4, the single-CTA kernel): same bits, same product count."""
    ip, ix, m = er_case(n, d, seed)
    got, it = run_rms(ctx, m, "rms_tc", fmt=fmt, e4m3_only=True)
    np.testing.assert_array_equal(got, oracle.closure(n, ip, ix))
    assert it == oracle.rms_iterations(oracle.longest_shortest_path(n, ip, ix))
    st = ctx.stats()
    assert st["e2m1_products"] == 0 and st["product_launches"] == it


def test_smp_wide_rows_long_paths(ctx):
    """n = 135,000 (2,110 words per row, so more than 32 words of the
    touched-word bitmap per warp) on a chain with shortcuts."""
    n, q = 135_000, 6
    ip, ix = shortcut_case(n, "chain", 7)
    src = wl.query_rows(n, q, 1, 4, 8)
    want, levels = oracle.smp(n, ip, ix, src)
    P = dev(wl.csr_to_packed(n, ip, ix).view(np.int64))
    out = torch.zeros((q, src.shape[1]), dtype=torch.int64, device="cuda")
    it = ctx.smp(P, n, dev(src.view(np.int64)), q, out, fmt=pkg.BMLP_FMT_PACKED64, variant="smp_packed")
    torch.cuda.synchronize()
    np.testing.assert_array_equal(wl.unpack_rows(out.cpu().numpy().view(np.uint64), n), want)
    assert it == int(levels.max()) + 1
    del P


# ------------------------------------------------------------ compose --
@pytest.mark.parametrize("variant", ["rms_tc", "rms_packed"])
@pytest.mark.parametrize("n,seed", [(1, 0), (77, 1), (256, 2), (513, 3), (1100, 4), (2100, 5)])
def test_compose(ctx, variant, n, seed):
    ip1, ix1, m1 = er_case(n, 1.0, seed)
    ip2, ix2, m2 = er_case(n, 1.4, seed + 50)
    want = oracle.compose_rows(n, (ip1, ix1), (ip2, ix2))
    out = torch.zeros((n, n), dtype=torch.uint8, device="cuda")
    ctx.compose(dev(m1), dev(m2), n, out, variant=variant)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), want)


# --------------------------------------------------------- arguments --
def test_argument_errors(ctx):
    R = torch.zeros((4, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(pkg.BmlpError) as e:
        ctx.rms(R, -1, R)
    assert e.value.status == 1
    with pytest.raises(pkg.BmlpError):
        ctx.rms(R, 4, R, fmt=7)
    assert ctx.rms(None, 0, None) == 0            # n = 0 is a no-op
    with pytest.raises(pkg.BmlpError):
        ctx.rms(R, 4, R, variant=99)
    with pytest.raises(pkg.BmlpError) as e:
        ctx.rms(dev(np.roll(np.eye(64, dtype=np.uint8), 1, axis=1)), 64,
                torch.zeros((64, 64), dtype=torch.uint8, device="cuda"), variant="rms_tc", max_iters=2)
    assert e.value.status == 5                   # a 64-cycle needs 7 products


def test_mma_issue_rate(ctx):
    """The issue-rate probes run and report positive rates; the 4-bit kind
    carries twice the K per instruction, so it is never slower than E4M3, and
    the 2-SM form does the work of two 1-SM MMAs per instruction pair; the
    word-OR probe reports a rate too, and so does the squaring kernel's
    N = 256 + 224 mix. Unknown kinds are refused."""
    r8 = ctx.mma_issue_rate(0, iters=2000)
    r4 = ctx.mma_issue_rate(1, iters=2000)
    r4x2 = ctx.mma_issue_rate(2, iters=2000)
    ors = ctx.mma_issue_rate(3, iters=2000)
    r480 = ctx.mma_issue_rate(4, iters=2000)
    assert r8 > 0 and r4 >= r8 and r4x2 > 0.5 * r4 and ors > 0 and r480 > 0.5 * r4x2
    for bad in (-1, 5):
        with pytest.raises(pkg.BmlpError):
            ctx.mma_issue_rate(bad)


@pytest.mark.parametrize("variant", ["rms_tc", "rms_packed", "smp_packed"])
def test_pinned_host_buffers(ctx, variant):
    """Page-locked host input and output: read and written in place by the kernels."""
    n = 1100
    ip, ix, m = er_case(n, 1.7, 31)
    want = oracle.closure(n, ip, ix)
    hin = torch.from_numpy(m).pin_memory()
    hout = torch.zeros_like(hin).pin_memory()
    ctx.rms(hin, n, hout, variant=variant)
    np.testing.assert_array_equal(hout.numpy(), want)
    P = torch.from_numpy(wl.pack_rows(m).view(np.int64)).pin_memory()
    Pout = torch.zeros_like(P).pin_memory()
    ctx.rms(P, n, Pout, fmt=pkg.BMLP_FMT_PACKED64, variant=variant)
    np.testing.assert_array_equal(wl.unpack_rows(Pout.numpy().view(np.uint64), n), want)


def _as_e4m3(m, rng):
    """0/1 matrix as E4M3 bytes: ones are 1.0 (0x38) or other nonzero E4M3 values, zeros are +0 (0x00) or -0 (0x80)."""
    ones = rng.choice(np.array([0x38, 0x40, 0x30, 0xB8, 0x01], np.uint8), size=m.shape)
    zeros = rng.choice(np.array([0x00, 0x80], np.uint8), size=m.shape)
    return np.where(m != 0, ones, zeros).astype(np.uint8)


@pytest.mark.parametrize("host", [False, True])
def test_byte_formats_i8_and_e4m3(ctx, host):
    """BMLP_FMT_I8 reads like U8 (nonzero = 1, outputs 0 / 1); BMLP_FMT_E4M3
    reads 0x00 and 0x80 as zero and any other byte as one and writes 0x00 /
    0x38; closures, compositions, the relation operators and the incremental
    fact, on device and host buffers."""
    rng = np.random.default_rng(5)
    n = 300
    ip, ix, m = er_case(n, 1.4, 41)
    want = oracle.closure(n, ip, ix)
    i8 = np.where(m != 0, rng.integers(1, 128, m.shape), 0).astype(np.int8)
    e8 = _as_e4m3(m, rng)

    def put(a):
        return torch.from_numpy(np.ascontiguousarray(a)) if host else dev(a)

    for fmt, src, one in ((pkg.bmlp.BMLP_FMT_I8, i8, 1), (pkg.bmlp.BMLP_FMT_E4M3, e8, 0x38)):
        R = put(src)
        out = put(np.full((n, n), 0x55, np.uint8))
        it = ctx.rms(R, n, out, fmt=fmt, variant="rms_tc")
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint8)
        np.testing.assert_array_equal(got, want * one)
        assert it == oracle.rms_iterations(oracle.longest_shortest_path(n, ip, ix))
        # transpose and union of the same relation
        out = put(np.zeros((n, n), np.uint8))
        ctx.transpose(R, n, out, fmt=fmt)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy().view(np.uint8), (m.T != 0) * one)
    # composition (I + R2+) R1 with E4M3 operands
    ip2, ix2, m2 = er_case(n, 1.1, 42)
    out = put(np.zeros((n, n), np.uint8))
    ctx.compose(put(_as_e4m3(m, rng)), put(_as_e4m3(m2, rng)), n, out, fmt=pkg.bmlp.BMLP_FMT_E4M3, variant="rms_tc")
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint8), oracle.compose_rows(n, (ip, ix), (ip2, ix2)) * 0x38)
    # one new fact into an E4M3 closure, in place
    clo = put((want * 0x38).astype(np.uint8))
    ctx.insert(clo, n, np.array([[3, 200]], np.int32), fmt=pkg.bmlp.BMLP_FMT_E4M3)
    torch.cuda.synchronize()
    grown = wl.csr_from_pairs(n, np.concatenate([np.repeat(np.arange(n), np.diff(ip)), [3]]), np.concatenate([ix, [200]]))
    np.testing.assert_array_equal(clo.cpu().numpy().view(np.uint8), oracle.closure(n, *grown) * 0x38)
