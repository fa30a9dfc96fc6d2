"""Multi-process host logic of replica runs (two gloo ranks on the CPU).

A run on N GPUs is N independent replicas: each rank solves its own seeded
density, and the only collectives are the barrier around the timed region
and the max-reduce of its elapsed time. These tests run that logic as two
processes with the gloo backend.
"""
import json
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1211_5244_gb300 import replicas, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    r, w, local = replicas.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        wl = synth.WORKLOADS["free32_f64"]
        rho = synth.gaussian_mixture(wl["n"], wl["h"], wl["n_gauss"], replicas.replica_seed(wl["seed"], r),
                                     noise=wl["noise"])
        replicas.barrier(dist)
        # rank r reports an elapsed time of 1 + r seconds for 100 units
        value, slowest = replicas.aggregate(1.0 + r, 100, dist)
        mx = replicas.max_over_ranks(float(r) * 3.5, dist)
        out = {"rank": r, "world": w, "local": local, "value": value, "slowest": slowest, "max": mx,
               "rho_sum": float(rho.sum()), "rho_sq": float((rho ** 2).sum())}
        with open(os.path.join(outdir, f"rank{r}.json"), "w") as f:
            json.dump(out, f)
    finally:
        dist.destroy_process_group()


def _run(world, tmp_path):
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    return [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]


def test_two_rank_aggregate(tmp_path):
    res = _run(2, tmp_path)
    for r, d in enumerate(res):
        assert (d["rank"], d["world"], d["local"]) == (r, 2, r)
        # whole-job rate: 2 ranks x 100 units over the slowest rank's 2 s
        assert d["slowest"] == pytest.approx(2.0)
        assert d["value"] == pytest.approx(100.0)
        assert d["max"] == pytest.approx(3.5)
    # the replicas solve different densities
    assert res[0]["rho_sq"] != pytest.approx(res[1]["rho_sq"], rel=1e-6)


def test_replica_density_matches_single_process(tmp_path):
    """Rank r's density is the one a single process builds with seed + r."""
    res = _run(2, tmp_path)
    wl = synth.WORKLOADS["free32_f64"]
    for r, d in enumerate(res):
        rho = synth.gaussian_mixture(wl["n"], wl["h"], wl["n_gauss"], wl["seed"] + r, noise=wl["noise"])
        assert d["rho_sq"] == pytest.approx(float((rho ** 2).sum()), rel=1e-12)
        assert d["rho_sum"] == pytest.approx(float(rho.sum()), rel=1e-9, abs=1e-9)


def test_single_process_defaults(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert replicas.dist_env() == (0, 1, 0)
    value, slowest = replicas.aggregate(0.5, 10, None)
    assert (value, slowest) == (20.0, 0.5)
    assert replicas.max_over_ranks(7.0, None) == 7.0


def test_bad_environment(monkeypatch):
    monkeypatch.setenv("RANK", "2")
    monkeypatch.setenv("WORLD_SIZE", "2")
    with pytest.raises(ValueError):
        replicas.dist_env()
    with pytest.raises(ValueError):
        replicas.throughput(1, 1, 0.0)
