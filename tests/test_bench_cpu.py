"""bench.py on the CPU: the multi-process timing reduction over gloo ranks
(world size 2) and the reference arm's JSON line."""
import json
import os
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.0 + rank, world, "cpu")   # rank 1 is the slow one
        q.put((rank, t, bench.whole_job_value(10, world, t)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[1] for g in got] == [2.0, 2.0]          # every rank sees the slowest time
    assert [g[2] for g in got] == [10.0, 10.0]        # 2 ranks x 10 units / 2 s


def test_single_process_unchanged():
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.whole_job_value(8, 1, 2.0) == 4.0


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "2000",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_under_two_ranks_prints_once():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "1000",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=300, cwd=ROOT,
                       env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""


@pytest.mark.parametrize("w", ["powerlaw_smp", "kg_batch"])
def test_aux_workload_flags_parse(w, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", w, "--variant", "smp_packed"])
    a = bench.parse()
    assert a.workload == w


def test_profile_summary_values(tmp_path):
    """The per-launch DRAM bytes come from the committed summary only while its
    kernel hash matches the current source."""
    import bench
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "tc_duo_kernel_er64.md").write_text(
        "# title\n- kernel_source_sha256_12: `%s`\n- dram_bytes_per_launch: `1234`  (note)\n"
        % bench.kernel_hash("tc_duo_kernel"))
    assert bench.profiled_traffic("tc_duo_kernel", 64, root=str(tmp_path)) == 1234.0
    (prof / "tc_duo_kernel_er64.md").write_text("- kernel_source_sha256_12: `000000000000`\n"
                                                 "- dram_bytes_per_launch: `1234`\n")
    assert bench.profiled_traffic("tc_duo_kernel", 64, root=str(tmp_path)) is None
    assert bench.profiled_traffic("tc_duo_kernel", 32768) is None or bench.profiled_traffic(
        "tc_duo_kernel", 32768) > 0
