"""The sharded path on the GPU with a one-rank NCCL group: the cost partition,
the library running the rank's share (query rows through bmlp_smp, problems
through bmlp_batch_run writing into the rank's contiguous output buffer) and
the all-gather, against the oracle. Runs in a child process so that its
process group does not outlive the test."""
import os
import socket
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import os, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import torch
import torch.distributed as dist
import oracle
import workloads as wl
import paper_2408_10369_gb300 as pkg
from paper_2408_10369_gb300 import bmlp, shard

dev = torch.device("cuda", 0)
torch.cuda.set_device(dev)
dist.init_process_group("nccl", rank=0, world_size=1, device_id=dev)
ctx = pkg.Context(0)
PK = bmlp.BMLP_FMT_PACKED64
# query rows
n, q = 3000, 61
ip, ix = wl.powerlaw_csr(n, 2.1, 300, 7)
P = torch.from_numpy(wl.csr_to_packed(n, ip, ix).view(np.int64)).to(dev)
src = wl.query_rows(n, q, 1, 12, 8)
parts = shard.lpt_partition(shard.query_costs(src), 1)
mine = parts[0]
s = torch.from_numpy(np.ascontiguousarray(src[mine]).view(np.int64)).to(dev)
out = torch.zeros_like(s)
ctx.smp(P, n, s, len(mine), out, fmt=PK, variant="smp_packed")
full = shard.gather_rows(out, parts, 0, q)
want = wl.pack_rows(oracle.smp(n, ip, ix, src)[0]).view(np.int64)
assert np.array_equal(full.cpu().numpy(), want), "sharded query rows differ"
# problems, outputs written in place into the rank's contiguous buffer
graphs = [wl.er_graph(nn, d, sd) for nn, d, sd in ((500, 1.5, 1), (77, 2.0, 2), (1300, 1.1, 3), (5000, 1.4, 4))]
ns = [500, 77, 1300, 5000]
numel = [m * wl.words(m) for m in ns]
parts = shard.lpt_partition(shard.problem_costs(ns), 1)
offs, cap = shard.share_layout(parts, 0, numel)
flat = torch.zeros(cap, dtype=torch.int64, device=dev)
items, keep = [], []
for i in parts[0]:
    R = torch.from_numpy(wl.csr_to_packed(ns[i], *graphs[i]).view(np.int64)).to(dev)
    keep.append(R)
    items.append(dict(n=ns[i], R1=R, out=flat[offs[i]:offs[i] + numel[i]].view(ns[i], wl.words(ns[i])), fmt=PK))
ctx.batch_run(items)
outs = shard.gather_flat(flat, parts, numel)
for i, (m, (gip, gix)) in enumerate(zip(ns, graphs)):
    got = outs[i].cpu().numpy().view(np.uint64).reshape(m, wl.words(m))
    assert np.array_equal(got, wl.pack_rows(oracle.closure(m, gip, gix))), ("sharded problem differs", i)
ctx.close()
dist.destroy_process_group()
print("shard ok")
'''


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_sharded_path_on_one_nccl_rank():
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "shard ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
