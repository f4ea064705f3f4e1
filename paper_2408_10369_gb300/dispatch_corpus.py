"""Training data, training and evaluation of the learned variant dispatcher.

    python -m paper_2408_10369_gb300.dispatch_corpus sweep  --start 0 --count 5000 --out corpus.jsonl
    python -m paper_2408_10369_gb300.dispatch_corpus train  --data corpus.jsonl --model dispatch_model.bin
    python -m paper_2408_10369_gb300.dispatch_corpus eval   --data corpus.jsonl --model dispatch_model.bin

sweep  times the four closure variants on the mixed corpus (graph i has seed
       i; n log-uniform in [256, 32768]; ER / power law / chain-grid with
       shortcuts / 8-block SBM). Each variant runs with a time budget of 4x the
       fastest variant so far on that graph (2 s at most): a run that hits it is
       recorded as censored at the budget. Every finished variant's closure is
       compared bit for bit with the first finished one. Appends one JSON line
       per graph and resumes by index.
train  fits the MLP on the GPU (bmlp_dispatch_train) on graphs with index <
       the split (9,000 by default) and saves the model.
retime times some variants again on every graph of a corpus file (after a
       kernel changed), keeping the other variants' times, and writes a new file.
eval   on the held-out graphs: regret of the chosen variant against the best
       one, and the time of the dispatched pipeline (features + prediction +
       chosen variant, closures grouped in one bmlp_batch_run) against plain
       single-instance BMLP_RMS_TC squaring on every graph, with and without
       its bit-row squarings (options.tc_only), all measured live.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

VARIANT_NAMES = ("rms_tc", "rms_packed", "smp_tc", "smp_packed")   # bmlp_variant 1..4
ORDER = (1, 4, 2, 3)                                                # cheapest-first sweep order
CAP_S = 2.0
GROUP_MAX_N = 4096   # larger closures run on their own (the grouped workspace is 4 n^2 bytes per problem)


def _torch():
    import torch
    return torch


def load_jsonl(path):
    rows = {}
    if os.path.exists(path):
        import gzip
        with (gzip.open(path, "rt") if path.endswith(".gz") else open(path)) as f:
            for ln in f:
                ln = ln.strip()
                if ln:
                    r = json.loads(ln)
                    rows[r["index"]] = r
    return rows


def graph_on_device(index, n_max=32768):
    import workloads as wl
    torch = _torch()
    g = wl.corpus_graph(index, n_max=n_max)
    P = wl.csr_to_packed(g["n"], g["indptr"], g["indices"])
    return g, torch.from_numpy(np.ascontiguousarray(P).view(np.int64)).cuda()


def warm(ctx, n_max):
    """Grow every workspace to the largest corpus size once, before timing."""
    from . import bmlp
    torch = _torch()
    n = n_max
    words = (n + 63) // 64
    P = torch.zeros((n, words), dtype=torch.int64, device="cuda")
    P[0, 0] = 2  # one edge 0 -> 1: closures stay tiny, buffers reach full size
    out = torch.zeros_like(P)
    for v in VARIANT_NAMES:
        ctx.rms(P, n, out, fmt=bmlp.BMLP_FMT_PACKED64, variant=v)
    ctx.dispatch_features(P, n, fmt=bmlp.BMLP_FMT_PACKED64)
    torch.cuda.synchronize()


def time_variant(ctx, P, n, out, variant, budget_s):
    from . import bmlp
    torch = _torch()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    try:
        iters = ctx.rms(P, n, out, fmt=bmlp.BMLP_FMT_PACKED64, variant=variant, budget_ns=int(budget_s * 1e9))
        censored = False
    except bmlp.BmlpError as e:
        if e.status != bmlp.BMLP_ERR_BUDGET:
            raise
        iters, censored = -1, True
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    return (max(ms, budget_s * 1e3) if censored else ms), censored, iters


def sweep(args):
    from . import bmlp
    import paper_2408_10369_gb300 as pkg
    import workloads as wl
    torch = _torch()
    done = load_jsonl(args.out)
    ctx = pkg.Context(0)
    warm(ctx, args.n_max)
    t_start = time.time()
    with open(args.out, "a") as fo:
        for index in range(args.start, args.start + args.count):
            if index in done:
                continue
            if args.time_limit and time.time() - t_start > args.time_limit:
                print("time limit reached at index", index, flush=True)
                break
            g, P = graph_on_device(index, args.n_max)
            n = g["n"]
            feats = ctx.dispatch_features(P, n, fmt=bmlp.BMLP_FMT_PACKED64)
            ms = [0.0] * 4
            cens = [False] * 4
            iters = [0] * 4
            ref_out = None
            agree = True
            best = math.inf
            for v in ORDER:
                budget = min(CAP_S, 4.0 * best / 1e3) if best < math.inf else CAP_S
                out = torch.zeros_like(P)
                t, c, it = time_variant(ctx, P, n, out, VARIANT_NAMES[v - 1], budget)
                ms[v - 1], cens[v - 1], iters[v - 1] = t, c, it
                if not c:
                    best = min(best, t)
                    if ref_out is None:
                        ref_out = out
                    elif not torch.equal(out, ref_out):
                        agree = False
            rec = dict(index=index, family=g["family"], n=n, params=g["params"], nnz=int(len(g["indices"])),
                       features=[float(x) for x in feats], ms=ms, censored=cens, iters=iters, agree=agree)
            fo.write(json.dumps(rec) + "\n")
            fo.flush()
            if not agree:
                print("VARIANTS DISAGREE on graph", index, flush=True)
            del P, ref_out
    ctx.close()


def retime(args):
    """Re-time some variants on every graph of an existing corpus file (after a kernel changed): the other
    variants' times are kept; a re-timed variant runs with a budget of 4x the fastest kept time (2 s at most)
    and its output is compared bit for bit with that fastest variant's. Writes a new corpus file."""
    from . import bmlp
    import paper_2408_10369_gb300 as pkg
    torch = _torch()
    import gzip
    opener = gzip.open if args.data.endswith(".gz") else open
    with opener(args.data, "rt") as f:
        rows = [json.loads(ln) for ln in f if ln.strip()]
    which = [VARIANT_NAMES.index(v) for v in args.variants.split(",")]
    ctx = pkg.Context(0)
    warm(ctx, args.n_max)
    t_start = time.time()
    bad = 0
    with open(args.out, "w") as fo:
        for r in rows:
            keep = [k for k in range(4) if k not in which and not r["censored"][k]]
            best_k = min(keep, key=lambda k: r["ms"][k]) if keep else None
            g, P = graph_on_device(r["index"], args.n_max)
            n = g["n"]
            ref = None
            if best_k is not None:
                ref = torch.zeros_like(P)
                ctx.rms(P, n, ref, fmt=bmlp.BMLP_FMT_PACKED64, variant=VARIANT_NAMES[best_k])
            budget = min(CAP_S, 4.0 * r["ms"][best_k] / 1e3) if best_k is not None else CAP_S
            for k in which:
                out = torch.zeros_like(P)
                t, c, it = time_variant(ctx, P, n, out, VARIANT_NAMES[k], budget)
                r["ms"][k], r["censored"][k], r["iters"][k] = t, c, it
                if not c and ref is not None and not torch.equal(out, ref):
                    r["agree"] = False
                    bad += 1
            fo.write(json.dumps(r) + "\n")
            del P, ref
    ctx.close()
    print(json.dumps({"retimed": len(rows), "variants": args.variants, "disagreements": bad,
                      "seconds": time.time() - t_start}))


def arrays(rows):
    X = np.array([r["features"] for r in rows], np.float32)
    T = np.array([r["ms"] for r in rows], np.float64)
    C = np.array([r["censored"] for r in rows], np.uint8)
    return X, np.log2(np.maximum(T, 1e-3)).astype(np.float32), C, T


def train(args):
    import paper_2408_10369_gb300 as pkg
    rows = [r for i, r in sorted(load_jsonl(args.data).items()) if i < args.split]
    X, Y, C, _ = arrays(rows)
    ctx = pkg.Context(0)
    t0 = time.time()
    loss = ctx.dispatch_train(X, Y, C, epochs=args.epochs, batch=256, lr=args.lr, weight_decay=1e-4, seed=0)
    dt = time.time() - t0
    ctx.dispatch_save(args.model)
    ctx.close()
    print(json.dumps({"train_samples": len(rows), "epochs": args.epochs, "final_loss": loss, "train_s": dt}))


def evaluate(args):
    from . import bmlp
    import paper_2408_10369_gb300 as pkg
    torch = _torch()
    rows = [r for i, r in sorted(load_jsonl(args.data).items()) if i >= args.split]
    X, Y, C, T = arrays(rows)
    ctx = pkg.Context(0)
    ctx.dispatch_load(args.model)
    pred, choice = ctx.dispatch_predict(X)
    ch = choice - 1
    best = T.min(1)
    chosen = T[np.arange(len(rows)), ch]
    regret = chosen / best - 1.0
    fixed = T[:, 0] / best - 1.0
    best_choice = T.argmin(1)
    report = {
        "heldout": len(rows),
        "regret_mean": float(regret.mean()), "regret_p50": float(np.median(regret)),
        "regret_p95": float(np.percentile(regret, 95)),
        "fixed_rms_tc_regret_mean": float(fixed.mean()),
        "choice_hist": {VARIANT_NAMES[v]: int((ch == v).sum()) for v in range(4)},
        "best_hist": {VARIANT_NAMES[v]: int((best_choice == v).sum()) for v in range(4)},
        "accuracy": float((ch == best_choice).mean()),
        "sum_ms_fixed_rms_tc_table": float(T[:, 0].sum()), "sum_ms_chosen_table": float(chosen.sum()),
        "sum_ms_best_table": float(best.sum()),
    }
    if args.live:
        report.update(live_pipeline(ctx, rows, args.n_max))
    ctx.close()
    print(json.dumps(report))
    if args.report:
        with open(args.report, "w") as f:
            json.dump(report, f, indent=1)


def live_pipeline(ctx, rows, n_max, return_outputs=False):
    """Time (a) plain single-instance squaring per graph with BMLP_RMS_TC
    (bit-row squarings while R is sparse for n >= 8192, then tensor cores),
    (a') the same with every squaring on the tensor cores (options.tc_only),
    (a'') the same on E4M3 operands (options.e4m3_only: the kind::f8f6f4 form
    of the plain tensor-core path), and (b) the dispatched path: features + prediction for every graph, then
    the graphs with n <= 4,096 run grouped in one bmlp_batch_run (engine per
    problem from the prediction: tensor-core or bit-row squaring, or frontier
    expansion), the others one by one with their predicted variant. Every output is compared with (a).
    With return_outputs, also returns the graphs (corpus dict, device input)
    and the dispatched outputs (packed bit rows on the device)."""
    from . import bmlp
    torch = _torch()
    graphs = [graph_on_device(r["index"], n_max) for r in rows]
    outs_a = [torch.zeros_like(P) for _, P in graphs]
    outs_b = [torch.zeros_like(P) for _, P in graphs]
    F = bmlp.BMLP_FMT_PACKED64
    # warm-up of both paths on the first graphs
    for (g, P), o in list(zip(graphs, outs_a))[:4]:
        ctx.rms(P, g["n"], o, fmt=F, variant="rms_tc")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for (g, P), o in zip(graphs, outs_a):
        ctx.rms(P, g["n"], o, fmt=F, variant="rms_tc")
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    # the same with every squaring on the tensor cores (no bit-row squarings while R is sparse)
    for (g, P), o in list(zip(graphs, outs_b))[:4]:
        ctx.rms(P, g["n"], o, fmt=F, variant="rms_tc", tc_only=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for (g, P), o in zip(graphs, outs_b):
        ctx.rms(P, g["n"], o, fmt=F, variant="rms_tc", tc_only=True)
    torch.cuda.synchronize()
    t_tc_only = time.perf_counter() - t0
    bad_tc_only = sum(0 if torch.equal(a, b) else 1 for a, b in zip(outs_a, outs_b))
    for o in outs_b:
        o.zero_()
    # (a'') the plain tensor-core path in its 8-bit form: every squaring on the tensor cores on E4M3 operands
    # (kind::f8f6f4), no bit-row start, no 4-bit operands
    for (g, P), o in list(zip(graphs, outs_b))[:4]:
        ctx.rms(P, g["n"], o, fmt=F, variant="rms_tc", tc_only=True, e4m3_only=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for (g, P), o in zip(graphs, outs_b):
        ctx.rms(P, g["n"], o, fmt=F, variant="rms_tc", tc_only=True, e4m3_only=True)
    torch.cuda.synchronize()
    t_e4m3 = time.perf_counter() - t0
    bad_e4m3 = sum(0 if torch.equal(a, b) else 1 for a, b in zip(outs_a, outs_b))
    for o in outs_b:
        o.zero_()

    def dispatched():
        # features and prediction for every graph with one host wait
        choice = ctx.dispatch_choose_many([P for _, P in graphs], [g["n"] for g, _ in graphs], fmt=F)
        group = []
        for (g, P), o, c in zip(graphs, outs_b, choice):
            if c in (bmlp.BMLP_RMS_TC, bmlp.BMLP_RMS_PACKED, bmlp.BMLP_SMP_PACKED) and g["n"] <= GROUP_MAX_N:
                # small graphs: grouped, the prediction picks each problem's engine (the frontier ones share one
                # grouped frontier launch)
                group.append(dict(n=g["n"], R1=P, out=o, fmt=F, variant=int(c)))
            else:
                ctx.rms(P, g["n"], o, fmt=F, variant=int(c))
        if group:
            ctx.batch_run(group)
        return choice

    dispatched()   # builds and caches the batch graphs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    choice = dispatched()
    torch.cuda.synchronize()
    t_disp = time.perf_counter() - t0
    bad = sum(0 if torch.equal(a, b) else 1 for a, b in zip(outs_a, outs_b))
    rep = {"live_graphs": len(graphs), "live_plain_rms_tc_s": t_plain, "live_dispatched_s": t_disp,
            "live_speedup": t_plain / t_disp, "live_bit_mismatches": bad,
            "live_tc_only_s": t_tc_only, "live_speedup_vs_tc_only": t_tc_only / t_disp,
            "live_tc_only_bit_mismatches": bad_tc_only,
            "live_tc_only_e4m3_s": t_e4m3, "live_speedup_vs_tc_only_e4m3": t_e4m3 / t_disp,
            "live_tc_only_e4m3_bit_mismatches": bad_e4m3,
            "live_choice_hist": {VARIANT_NAMES[v - 1]: int((choice == v).sum()) for v in (1, 2, 3, 4)}}
    if return_outputs:
        del outs_a
        return rep, graphs, outs_b
    return rep


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["sweep", "train", "eval", "retime"])
    ap.add_argument("--start", type=int, default=0)
    ap.add_argument("--count", type=int, default=10000)
    ap.add_argument("--out", default="corpus.jsonl")
    ap.add_argument("--data", default="corpus.jsonl")
    ap.add_argument("--model", default="dispatch_model.bin")
    ap.add_argument("--report", default=None)
    ap.add_argument("--split", type=int, default=9000)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--n-max", type=int, default=32768)
    ap.add_argument("--time-limit", type=float, default=0.0)
    ap.add_argument("--live", action="store_true")
    ap.add_argument("--variants", default="rms_tc", help="retime: comma-separated variants to time again")
    args = ap.parse_args()
    {"sweep": sweep, "train": train, "eval": evaluate, "retime": retime}[args.cmd](args)


if __name__ == "__main__":
    main()
