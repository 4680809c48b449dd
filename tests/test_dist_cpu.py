"""The multi-process (N > 1) path of bench.py on the CPU: world size 2 over
gloo.  bench.py runs one replica per rank with no collective on the data path;
what crosses ranks is host logic -- the slowest rank's time, the whole-job rate
over all ranks' units, and the reference arm run by rank 0 alone -- and that is
what these tests drive, with a 127.0.0.1 rendezvous."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 10.0 + 7.5 * rank                     # this rank's time
        slowest = bench.max_over_ranks(mine, dist, "cpu")
        rate = bench.whole_job_rate(1_000_000_000, world, slowest)
        dist.barrier()
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"slowest": slowest, "rate": rate, "alone": bench.max_over_ranks(mine, None, "cpu")}, f)
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_whole_job_rate_gloo(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, x in enumerate(res):
        assert x["slowest"] == 17.5                  # every rank agrees on the slowest time
        assert x["rate"] == pytest.approx(2 * 1.0 / 17.5)
        assert x["alone"] == 10.0 + 7.5 * r          # no process group: the rank's own value


def test_reference_arm_under_torchrun():
    """Rank 0 alone times the oracle and prints one JSON line; rank 1 exits 0."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--ref-side", "16", "--steps", "1",
           "--warmup", "3", "--gpus", "2"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle"
    assert rec["e2e"]["h2d_bytes_per_step"] == 0
