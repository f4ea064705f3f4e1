"""The committed dispatcher model against the committed corpus, on the CPU.

The float64 reference forward of the MLP (``oracle/dispatch_ref.py``), run
with the weights saved in ``dispatch_model.bin``, picks variants for the
1,000 held-out corpus graphs (index >= 9,000) whose summed measured time is
within 2 % of the best variant's and well below fixed tensor-core squaring's:
what the trained network gains over the method without it. Its choices also
match the GPU evaluation recorded beside the model (FP16 weights there, so a
few near-ties may flip)."""
import gzip
import json
import os
import struct

import numpy as np

from oracle import dispatch_ref as ref

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2408_10369_gb300")
VARIANTS = ("rms_tc", "rms_packed", "smp_tc", "smp_packed")


def load_model(path):
    b = open(path, "rb").read()
    assert b[:8] == b"BMLPMLP1"
    dims = struct.unpack("<4i", b[8:24])
    assert dims == (ref.NF, ref.NH, ref.NV, ref.NP)
    mu = np.frombuffer(b, np.float32, ref.NF, 24)
    sig = np.frombuffer(b, np.float32, ref.NF, 24 + 4 * ref.NF)
    p = np.frombuffer(b, np.float32, ref.NP, 24 + 8 * ref.NF)
    assert len(b) == 24 + 8 * ref.NF + 4 * ref.NP
    return p, mu, sig


def heldout():
    with gzip.open(os.path.join(PKG, "data", "dispatch_corpus_gb300.jsonl.gz"), "rt") as f:
        rows = [json.loads(line) for line in f if line.strip()]
    rows = [r for r in rows if r["index"] >= 9000]
    X = np.array([r["features"] for r in rows], np.float64)
    T = np.array([r["ms"] for r in rows], np.float64)
    return X, T


def test_model_choices_on_the_heldout_corpus():
    p, mu, sig = load_model(os.path.join(PKG, "dispatch_model.bin"))
    X, T = heldout()
    assert X.shape == (1000, ref.NF) and T.shape == (1000, ref.NV)
    choice = ref.forward(p, mu, sig, X).argmin(1)
    chosen = T[np.arange(len(T)), choice].sum()
    best = T.min(1).sum()
    fixed_tc = T[:, 0].sum()
    assert chosen <= 1.02 * best, (chosen, best)
    assert fixed_tc > 1.4 * chosen, (fixed_tc, chosen)
    with open(os.path.join(PKG, "data", "dispatch_eval_gb300.json")) as f:
        ev = json.load(f)
    hist = np.bincount(choice, minlength=ref.NV)
    recorded = np.array([ev["choice_hist"][v] for v in VARIANTS])
    assert np.abs(hist - recorded).sum() <= 20, (hist, recorded)
