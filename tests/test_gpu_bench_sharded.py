"""bench.py --sharded under torchrun: one run of the workload with its windows split over two
ranks (here both on the one GPU, gloo transfers through the host), one JSON line from rank 0."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_sharded_two_ranks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--gpus", "2",
           "--steps", "3", "--warmup", "3", "--rounds-per-step", "2", "--sharded", "--backend",
           "gloo", "--workload", "potts10_L40_h64_m16", "--no-cpu-baseline"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["n_gpus"] == 2 and d["scaling"] == "strong" and d["value"] > 0
    assert d["config"]["parallelism"] == "windows2" and d["transport"] == "gloo"
    assert d["shards"] == [[0, 32], [32, 32]]
