"""The multi-GPU path on CPU: two `gloo` ranks run the benchmark's per-rank logic.

Centres are independent, so each rank processes its own batch of structures (weak scaling) and the only
collectives of a run are the job-wide reductions of the timing and of the environment count. This checks, with two
processes on the host:
* each rank draws a different batch from its rank-derived seed, with the same workload recipe;
* the coefficients a rank computes for its batch equal those a single process computes for that batch alone
  (no data-path exchange is needed);
* the max-over-ranks time and the summed environment count are what the JSON line reports.
"""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    from oracle import soap as osoap

    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    r, w, _ = bench.dist_init(None)
    system = bench.make_system("batch", r, n_structures=3)
    h = osoap.Hypers(**system.hypers)
    c = osoap.spherical_expansion(system, h, centres=[0, system.n_atoms - 1])
    ms = bench.max_over_ranks(1.5 + r, torch.device("cpu"))
    n_total = bench.sum_over_ranks(system.n_atoms, torch.device("cpu"))
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as fh:
        json.dump({"rank": r, "world": w, "n_atoms": system.n_atoms, "pos0": system.positions[0].tolist(),
                   "hypers": system.hypers, "c_sum": float(np.sum(c)), "c_abs": float(np.sum(np.abs(c))), "ms": ms,
                   "n_total": n_total}, fh)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_by_structure(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert [d["world"] for d in res] == [world] * world
    # different batches from rank-derived seeds, same recipe
    assert res[0]["pos0"] != res[1]["pos0"]
    assert res[0]["hypers"] == res[1]["hypers"]
    # job-wide reductions: slowest rank's time, all ranks' environments
    assert all(d["ms"] == 2.5 for d in res)
    assert all(d["n_total"] == res[0]["n_atoms"] + res[1]["n_atoms"] for d in res)
    # a rank's result is the single-process result for its own batch
    sys.path.insert(0, ROOT)
    import bench
    from oracle import soap as osoap

    for d in res:
        system = bench.make_system("batch", d["rank"], n_structures=3)
        h = osoap.Hypers(**system.hypers)
        c = osoap.spherical_expansion(system, h, centres=[0, system.n_atoms - 1])
        assert system.n_atoms == d["n_atoms"]
        assert np.isclose(float(np.sum(c)), d["c_sum"], rtol=1e-12, atol=0.0)
        assert np.isclose(float(np.sum(np.abs(c))), d["c_abs"], rtol=1e-12, atol=0.0)
