"""bench.py's multi-rank period-shard mode end to end on the one GPU a test
box has: two ranks under torchrun share the GPU (their kernels are
independent; nothing on the device waits for the other rank), the process
group is gloo (the halo and the objective are staged through host memory),
and the horizon is short.  Checks that rank 0 prints one JSON line with the
strong-scaling fields; the parity of the sharded outputs themselves is
tests/test_gpu_shard.py's."""
import json
import os
import socket
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_bench_period_shards_two_ranks_one_gpu():
    pytest.importorskip("torch")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--gpus", "2",
           "--steps", "3", "--warmup", "3", "--periods", "12", "--e2e-steps", "2", "--dist-backend", "gloo"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, res.stdout[-3000:]
    d = json.loads(lines[0])
    assert d["n_gpus"] == 2 and d["scaling"] == "strong"
    assert d["config"]["parallelism"].startswith("period-shards2")
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["shards"]["periods_per_rank"] == [6, 6]
    assert d["e2e"]["value"] > 0 and d["e2e"]["ranks"] == 2
    assert d["roofline"]["kernel"].startswith("k_branch") and d["roofline"]["ops_per_launch"] == 143 * 6 * 16000
