"""Host logic of bench.py on the CPU: whole-job aggregation over ranks (gloo, world size 2)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, units = bench.aggregate(100.0 + 50.0 * rank, 1000.0 * (rank + 1), dist)
        q.put((rank, ms, units))
    finally:
        dist.destroy_process_group()


def test_aggregate_max_time_sum_units_over_two_ranks():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=5) for _ in range(2))
    for rank, ms, units in out:
        assert ms == 150.0 and units == 3000.0


def test_aggregate_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(12.5, 7.0, None) == (12.5, 7.0)


def test_bench_arguments_and_workload_description():
    sys.path.insert(0, ROOT)
    import bench
    a = bench.parse_args([])
    assert a.gpus == 1 and a.steps >= 1 and a.warmup >= 3 and a.impl == "ugp"
    cfg = bench.workload_config(a, "flushed")
    # the paper-scale configuration: 5.5M primitives, 1920 x 1080, depth 12, lighting A, a tenth of
    # the surface shapes near-specular
    assert cfg["n_prims"] == 5_500_000 and cfg["width"] == 1920 and cfg["height"] == 1080
    assert cfg["max_depth"] == 12 and cfg["lighting"] == "A" and cfg["near_specular_frac"] == 0.1
    assert "5500000" in cfg["workload"] and "1920x1080" in cfg["workload"]


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` on a tiny workload (the FP64 oracle on the host): one JSON
    line with the arm's fields, the CPU-baseline block and an e2e block without copies."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n-prims", "2000",
                          "--width", "64", "--height", "64", "--steps", "1", "--warmup", "0", "--cpu-pixels", "2048"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["unit"] == "Mrays/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
