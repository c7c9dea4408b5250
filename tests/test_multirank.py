"""The env-sharding convention across ranks, on CPU (gloo, world size 2), with the oracle.

Each rank renders its own range of envs with env_offset = its first global env id, so the random
streams (keyed by global env id) and hence the outputs do not depend on how envs are spread over
processes.  The gather below only checks the result; the render path itself has no collective.
This test checks the keying convention with the FP64 oracle as each rank's renderer; the library
itself is run the same way, two processes on one GPU, in test_gpu_multiprocess.py.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2602_03002_gb300 import workloads as W

SENSOR = W.Sensor(sigma_abs=0.01, p_drop=0.05, max_latency=2, seed=(21, 22))


def _shard(n_envs, rank, world):
    lo = n_envs * rank // world
    return lo, n_envs * (rank + 1) // world


def _rank_main(rank, world, port, result_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = W.config_small(n_steps=3, n_envs=6, width=12, height=8)
    lo, hi = _shard(w.n_envs, rank, world)
    osc = oracle.OracleScene.from_workload(w)
    rays = oracle.all_rays(w.cameras, hi - lo)
    out = osc.render(w.cameras, w.poses[:, lo:hi], 2, rays, SENSOR, env_offset=lo, flags=False,
                     threads=1)["depth"].reshape(hi - lo, -1)
    parts = [None] * world
    dist.all_gather_object(parts, out)
    if rank == 0:
        np.save(result_path, np.concatenate(parts))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_env_sharding_matches_single_process(tmp_path):
    path = str(tmp_path / "gathered.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), path), nprocs=2, join=True, start_method="spawn")
    gathered = np.load(path)
    w = W.config_small(n_steps=3, n_envs=6, width=12, height=8)
    osc = oracle.OracleScene.from_workload(w)
    whole = osc.render(w.cameras, w.poses, 2, oracle.all_rays(w.cameras, w.n_envs), SENSOR, flags=False,
                       threads=1)["depth"].reshape(w.n_envs, -1)
    assert np.array_equal(gathered, whole)
    # and a different offset changes the draws (the key really is the global env id)
    shifted = osc.render(w.cameras, w.poses, 2, oracle.all_rays(w.cameras, w.n_envs), SENSOR, env_offset=1,
                         flags=False, threads=1)["depth"].reshape(w.n_envs, -1)
    assert not np.array_equal(shifted, whole)
