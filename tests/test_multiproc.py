"""The N > 1 host paths of bench.py on CPU with the gloo backend
(world size 2): the timing reduction takes the max over ranks, and the
reference arm under torchrun runs on rank 0 only and prints one line."""
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


def _worker(rank, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank),
                      LOCAL_RANK=str(rank))

    class A:
        impl = "reference"
    ws, r, _ = bench.dist_setup(A)
    bench.barrier(ws)
    out[r] = bench.max_over_ranks(1.5 if r == 0 else 4.25, ws)
    dist.destroy_process_group()


def test_max_over_ranks_with_gloo():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(port, out), nprocs=2, join=True)
        assert out[0] == 4.25 and out[1] == 4.25


@pytest.mark.timeout(600)
def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--side", "64", "--steps", "2", "--warmup", "1"]
    r = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_caps_its_timed_region(monkeypatch, capsys):
    """A --steps too large for the CPU oracle ends at the wall-time cap: the
    line reports the rate over the full-grid steps actually taken and says
    so in its sample."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    oracle.build()
    monkeypatch.setattr(bench, "REFERENCE_BUDGET_S", 0.05)

    class A:
        side, warmup, steps, gpus = 64, 3, 10 ** 6, 1
    bench.run_reference(A, 1, 0)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 10 ** 6 and line["warmup"] == 3
    assert "capped" in line["cpu_baseline"]["sample"]
    done = int(line["cpu_baseline"]["sample"].split()[0])
    assert 1 <= done < 10 ** 6
    assert line["value"] > 0 and line["value"] == line["cpu_baseline"]["value"] == line["e2e"]["value"]
