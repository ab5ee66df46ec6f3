"""The benchmark's N>1 path on the CPU: ranks launched by torch.distributed.run on 127.0.0.1 with the
gloo backend, world size 2.  Checks the replica protocol (each rank its own keyframe, the slowest
rank's time, the throughput of all ranks' units over it, one report from rank 0) and that the
reference arm runs on rank 0 alone."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(nproc: int, *argv, timeout=240):
    env = dict(os.environ, OMP_NUM_THREADS="2", CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={nproc}",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", *argv]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def test_replica_timing_protocol_two_gloo_ranks(tmp_path):
    units = 15360000.0
    r = _torchrun(2, os.path.join(ROOT, "tests", "ranks_child.py"), str(tmp_path), str(units))
    assert r.returncode == 0, r.stderr[-2000:]
    seen = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(2)]
    assert [s["rank"] for s in seen] == [0, 1] and all(s["world"] == 2 for s in seen)
    assert [s["local"] for s in seen] == [0, 1]
    # the time of the region is the slowest rank's, on every rank
    assert all(s["max_ms"] == 40.0 for s in seen) and [s["own_ms"] for s in seen] == [10.0, 40.0]
    # whole-job throughput: both ranks' units over the slowest rank's time
    assert all(s["value"] == pytest.approx(2 * units / 0.040, rel=1e-12) for s in seen)
    # replicas: same work per rank, different keyframes
    assert seen[0]["residuals"] == seen[1]["residuals"] == int(units)
    assert seen[0]["keyframe_sum"] != seen[1]["keyframe_sum"]
    # rank 0 alone reports, one JSON line
    rep0 = (tmp_path / "report0.txt").read_text().splitlines()
    assert len(rep0) == 1 and json.loads(rep0[0]) == {"value": seen[0]["value"], "n_gpus": 2}
    assert (tmp_path / "report1.txt").read_text() == ""


def test_single_rank_protocol_is_local(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    ranks = bench.Ranks("gloo")
    assert ranks.dist is None and ranks.root and ranks.world == 1
    ranks.barrier()
    assert ranks.max_ms(12.5) == 12.5
    assert ranks.throughput(1000, 12.5) == pytest.approx(80000.0)
    ranks.close()


def test_reference_arm_runs_on_rank_zero_only():
    r = _torchrun(2, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
