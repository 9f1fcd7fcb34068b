"""The multi-rank bench path on CPU with gloo, world size 2: rank setup,
barrier, max-over-ranks of the timings, per-rank seeds, and the reference
arm printing one line from rank 0 only.  No GPU and no data-path collective
(each rank runs its own window)."""
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


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    ws, r, local, pg = bench.dist_init()
    assert (ws, r, local) == (world, rank, rank)
    bench.barrier(pg)
    m = bench.max_over_ranks(pg, float(10 * (rank + 1)))
    out.put((rank, m))
    pg.destroy_process_group()


def test_max_over_ranks_with_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 20.0), (1, 20.0)]


def test_reference_arm_under_two_ranks_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.join(ROOT, "bench.py"), "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--cpu-seconds", "0.3", "--config", "tiny"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "events/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_per_rank_windows_differ():
    sys.path.insert(0, ROOT)
    import synth
    cfg = synth.scaled(synth.CONFIGS["tiny"], 200, 5000)
    a = synth.zipf_counts(cfg.n_gates, cfg.n_events, cfg.zipf_s, cfg.cap, cfg.seed_ev + 1000 * 0)
    b = synth.zipf_counts(cfg.n_gates, cfg.n_events, cfg.zipf_s, cfg.cap, cfg.seed_ev + 1000 * 1)
    assert a.sum() == b.sum() and (a != b).any()
