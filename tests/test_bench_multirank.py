"""The N>1 path of bench.py (replicas under torchrun) on CPU with gloo,
world size 2: each rank gets its own map (seed offset), the only collective
is the max-over-ranks of the timings, the whole-job rate counts every rank's
work over the slowest rank's time, and the reference arm runs on rank 0
only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    job = bench.rank_job(W.GERLUMPH, rank)
    ms_local = 1000.0 + 250.0 * rank            # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms_local, world)
    rate = bench.aggregate_rate(bench.interactions(job), 4, ms_max, world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, job.seed, ms_max, rate))


def test_two_rank_aggregation_gloo():
    import bench
    import workloads as W
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seeds = {o[1] for o in out}
    assert len(seeds) == world                  # independent maps per rank
    assert all(o[2] == 1250.0 for o in out)     # both ranks see the slowest time
    expect = bench.interactions(W.GERLUMPH) * 4 * world / 1.25
    assert all(abs(o[3] - expect) < 1e-6 * expect for o in out)


def test_reference_arm_other_ranks_exit_quietly(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, config, precision = 1, 0, "parity", "compensated"
    bench.run_reference(Args)
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank0():
    """`bench.py --impl reference` at N=1 prints one JSON line: the oracle
    timed on the host cores on the map arm's metric and config, with its
    cpu_baseline and an e2e entry without host-device bytes."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--config", "parity",
                        "--steps", "1", "--warmup", "1"], cwd=root, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "interactions/s" and d["dtype"] == "f64"
    assert d["config"]["workload"] == "parity-256"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
