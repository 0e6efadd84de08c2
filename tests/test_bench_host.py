"""Host-side pieces of bench.py: the multi-rank aggregation (two gloo ranks on
CPU; each GPU runs an independent replica, the slowest one sets the time) and
the oracle arm's JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    v = bench._max_over_ranks(2, 10.0 + 5.0 * rank, device="cpu")
    bench._barrier(2)
    out.put((rank, v))
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 15.0), (1, 15.0)]


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["unit"] == "tests/s" and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["e2e"]["h2d_bytes_per_step"] == 0


def test_walk_source_hash_ignores_comments_only(tmp_path):
    # The committed DRAM-traffic record stays valid across comment edits of the
    # walk sources and is dropped by any code edit.
    sys.path.insert(0, ROOT)
    import bench
    a, b, c = tmp_path / "a.cu", tmp_path / "b.cu", tmp_path / "c.cu"
    a.write_text("int f(int x) {\n  return x + 1;  // add one\n}\n")
    b.write_text("// a new header comment\nint f(int x) {\n\n  return x + 1;  // plus one\n}\n")
    c.write_text("int f(int x) {\n  return x + 2;  // add one\n}\n")
    assert bench._source_sha([str(a)]) == bench._source_sha([str(b)])
    assert bench._source_sha([str(a)]) != bench._source_sha([str(c)])


def test_committed_traffic_record_is_used_only_for_its_own_walk_sources():
    # The DRAM bytes of the committed capture are reported while the walk
    # sources are those it was taken on, and null (not stale) otherwise.
    sys.path.insert(0, ROOT)
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "walk_kernel_512_traffic.json")))
    assert rec["dram_bytes_per_launch"] > 0
    if rec["source_sha"] == bench._walk_source_sha():
        assert bench._traffic_record() == rec["dram_bytes_per_launch"]
    else:
        assert bench._traffic_record() is None
