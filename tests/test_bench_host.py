"""Host-side logic of bench.py: multi-rank aggregation over gloo (world size 2, CPU)
and the reference arm's JSON contract (the CPU oracle on a small workload)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r measured (1 + r) s device time and (2 + r) s end to end
    dev, e2e = bench.world_max([1.0 + rank, 2.0 + rank], dist, "cpu")
    value = bench.replica_throughput(1000.0, world, dev)
    out.put((rank, dev, e2e, value))
    dist.barrier()
    dist.destroy_process_group()


def test_world_max_and_replica_throughput_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, dev, e2e, value in res:
        assert dev == 2.0 and e2e == 3.0            # every rank sees the slowest rank's time
        assert value == pytest.approx(1000.0 * 2 / 2.0)


def test_world_max_without_process_group():
    import bench
    assert bench.world_max([0.5, 0.25], None, "cpu") == [0.5, 0.25]
    assert bench.replica_throughput(10.0, 1, 2.0) == 5.0


def test_reference_arm_prints_contract_line():
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "lap2d_64_f64", "--steps", "3", "--warmup", "1"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["config"]["workload"] == "lap2d_64_f64"


def test_reference_arm_silent_on_other_ranks():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "lap2d_64_f64", "--steps", "1", "--warmup", "1"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip() == ""


@pytest.mark.parametrize("name", ["random_1m_f64", "random_1m_upper_f64", "lap2d_64_f64", "er_100k_f64",
                                  "nb_100k_f64", "lap3d_160_f64"])
def test_bench_workloads_are_valid_systems(name):
    # every single-factor workload hands the solver a valid factor of its triangle and a
    # right-hand side that is exactly A x* (the oracle's SpMV), with the sizes the line reports
    import numpy as np
    import bench
    import oracle
    spec = bench.WORKLOADS[name]
    A, xs, b = spec["make"]()
    if spec.get("triangle", "lower") == "upper":
        oracle.validate_upper(A)
    else:
        oracle.validate(A)
    assert xs.shape == b.shape == (A.n, spec["nrhs"])
    r = oracle.spmv(A, xs) - b
    assert np.max(np.abs(r)) <= 1e-12 * max(1.0, float(np.max(np.abs(b))))
    if name == "random_1m_f64":
        assert (A.n, A.nnz) == (1_000_000, 6_999_979)
    if name == "lap3d_160_f64":
        assert (A.n, A.nnz) == (4_096_000, 16_307_200)
