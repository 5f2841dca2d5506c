"""The multi-rank host logic of bench.py (replicas, no collective on the data
path) with world size 2 over gloo on the CPU: ranks from the environment, the
max-over-ranks time, the barrier, the whole-job value, and the reference arm
that only rank 0 runs."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    t_rank = 1.5 + rank                         # the slower rank decides the time
    t_max = bench.allmax(t_rank, w)
    bench.barrier(w)
    value = bench.job_value(1000, 4, w, t_max)

    class Args:                                 # the reference arm: only rank 0 works
        workload, grad, steps, warmup = "mixture4_d2", "adjoint", 1, 0
    skipped = bench.reference_arm(Args, w, r) is None if r != 0 else True
    out[rank] = (t_max, value, skipped)
    dist.destroy_process_group()


def test_two_ranks_over_gloo():
    pytest.importorskip("torch.distributed")
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.5
    assert res[0][1] == res[1][1] == 1000 * 4 * 2 / 2.5
    assert res[1][2]


def test_reference_arm_prints_the_contract_line(capsys):
    """Rank 0 of the reference arm prints one JSON line with the bench's metric keys,
    "impl": "reference", a cpu_baseline that describes the run and an e2e with no
    host-device traffic (the oracle runs on the host)."""
    import json
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        workload, grad, steps, warmup = "mixture4_d2", "adjoint", 2, 1
    bench.reference_arm(Args, 1, 0)
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["value"] > 0 and d["higher_is_better"]
    assert d["config"]["workload"] == "mixture4_d2"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
