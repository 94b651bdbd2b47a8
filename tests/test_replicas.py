"""The multi-GPU form is replicas only: every rank purifies its own matrices
and the job's rate is all units over the slowest rank's time.  The host side
of that path runs here with two gloo ranks on CPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_1101_0265_gb300 import inputs as I


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def max_over_ranks(ms):
        t = torch.tensor([ms], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    ms_local = 100.0 + 50.0 * rank          # rank 1 is the slow one
    value, ms = bench.replica_rate(ms_local, 16 * 5, world, max_over_ranks)
    h = I.dense_hamiltonian(64, 32, 0.1, config=2, instance=bench.rank_instance(rank, 0))
    sig = torch.tensor([float(h.F.sum()), float(h.F[0, 1])], dtype=torch.float64)
    sigs = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(sigs, sig)
    out[rank] = (value, ms, [s.tolist() for s in sigs])
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_rate_and_distinct_inputs():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        value, ms, sigs = res[rank]
        assert ms == 150.0                              # the slowest rank's time
        assert value == pytest.approx(world * 80 / 0.150)
        assert sigs[0] != sigs[1]                       # every replica has its own matrices


def test_single_process_rate():
    value, ms = bench.replica_rate(200.0, 16, 1, lambda x: x)
    assert ms == 200.0 and value == pytest.approx(80.0)
    # the same shape of workload, distinct seeds
    assert bench.rank_instance(0, 3) != bench.rank_instance(1, 3)
    a = I.dense_hamiltonian(32, 16, 0.1, config=2, instance=bench.rank_instance(0, 0))
    b = I.dense_hamiltonian(32, 16, 0.1, config=2, instance=bench.rank_instance(1, 0))
    assert a.F.shape == b.F.shape and not np.array_equal(a.F, b.F)


def test_reference_arm_line_contract():
    # `bench.py --impl reference` times the oracle on the host cores and prints
    # one JSON line with the main arm's metric, unit and config, plus its own
    # cpu_baseline and a zero-copy e2e object
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "256", "--steps", "1",
                        "--warmup", "3"], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "matrices/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 3
    assert d["config"] == bench.main_config(256, 8, ("TC_SF", "FIXED_MU_SF"), 1e-9, "mixed", 1)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
