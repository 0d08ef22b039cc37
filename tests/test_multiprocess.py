"""The N > 1 host path on the CPU with gloo, world size 2: the bench's rank
helpers (barrier, max over ranks for the time, sum over ranks for the
samples), per-rank instances that share nothing (instance sharding with no
data-path collective), and the reference arm launched by torchrun (rank 0
prints the one JSON line, the other rank exits without work)."""
import json
import os
import socket
import subprocess
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    from paper_1802_06625_b300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        env = bench.dist_env()
        cpu = torch.device("cpu")
        bench.barrier(ws)
        t = bench.max_over_ranks(1.5 + rank, ws, cpu)          # slowest rank's time
        n = bench.sum_over_ranks(1000.0 * (rank + 1), ws, cpu)  # units of all ranks
        w = synth.PLAIN_SMALL
        f = w.frame(0, instance=rank)
        fs = [torch.zeros_like(f) for _ in range(ws)]
        dist.all_gather(fs, f)                                # test only: compare the ranks' inputs
        out[rank] = (env, t, n, bool(torch.equal(fs[0], fs[1])), float(f.abs().sum()))
    finally:
        dist.destroy_process_group()


def test_rank_helpers_and_instance_sharding_gloo():
    ws, port = 2, _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        env, t, n, same, _ = res[r]
        assert env == (2, r, r)
        assert t == 2.5 and n == 3000.0          # max of (1.5, 2.5); 1000 + 2000
        assert not same                          # each rank fires its own instance
    assert res[0][4] != res[1][4]


def test_reference_arm_under_torchrun_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3", "--workload", "plain_small", "--ref-frames", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    # every key of the line's contract, with the reference arm's values
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"] and d["e2e"]["d2h_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    for k in ("value", "unit", "cores", "kind", "sample"):
        assert k in d["cpu_baseline"], k
