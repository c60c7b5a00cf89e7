"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas, no
data-path collective) agree on the slowest rank's step time and report the
whole-job throughput; the reference arm leaves rank 1 without work."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 25.0 * rank                      # rank 1 is the slow one
        m = bench.max_over_ranks(ms, dist, "cpu")
        v = bench.job_value(4.0e9, 3, world, m)
        out.put((rank, m, v))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    for _, m, v in res:
        assert m == 125.0
        assert v == pytest.approx(4.0e9 * 3 * 2 / 0.125)


def test_reference_arm_other_ranks_do_nothing(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, gpus = 1, 0, 2
    bench.run_reference(Args())
    assert capsys.readouterr().out == ""


def test_reference_arm_line():
    """`bench.py --impl reference` (the oracle on the host cores) prints one
    JSON line with the bench contract's keys, on the same metric and workload
    as the GPU arm."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["config"]["workload"] == bench.WORKLOAD % (24, 8)      # the GPU arm's default batch
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_traffic_entries_are_tied_to_their_kernel_source(tmp_path):
    """Each stored DRAM-traffic capture names the kernel source files it was
    taken on and their SHA-1; the bench reports the traffic only while the
    files still hash to it (a missing file never matches)."""
    import hashlib
    import json
    t = json.load(open(os.path.join(ROOT, "profiles", "chain_kernel_traffic.json")))
    assert t["captures"]
    for c in t["captures"]:
        assert c["source_files"] and all(os.path.exists(os.path.join(ROOT, f)) for f in c["source_files"])
        assert len(c["source_sha1"]) == 40 and c["bytes_per_launch"] > 0
    files = t["captures"][0]["source_files"]
    h = hashlib.sha1()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    assert bench.source_sha1(files) == h.hexdigest()
    assert bench.source_sha1(files + ["no/such/file.cu"]) is None
    assert bench.source_sha1([]) is None


def test_kernel_names_match_the_traffic_entries():
    """The bench names the tuned stress kernel the way the stored captures
    do, so a capture of the kernel it times is found."""
    import json
    names = {c["kernel"] for c in json.load(open(os.path.join(ROOT, "profiles", "chain_kernel_traffic.json")))["captures"]}
    assert bench.kernel_name({"kernel": "cluster_shared", "M": 16, "CL": 5}, "f32") in names
    assert bench.kernel_name({"kernel": "cluster_shared", "M": 16, "CL": 4}, "f32") in names
    assert bench.kernel_name({"kernel": "cluster", "M": 16, "CL": 4}, "f32") in names
    assert bench.kernel_name({"kernel": "register", "M": 16, "CL": 1}, "f32") == "k_chain_reg<16>"
