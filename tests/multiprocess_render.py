"""One rank of the multi-process render test: renders its share of the envs through librpl.so with
env_offset = its first global env id, then gathers every rank's frames over gloo; rank 0 writes the
gathered frames to the path given.  Run with RANK, WORLD_SIZE, MASTER_ADDR and MASTER_PORT set."""
import os
import sys

import numpy as np


def workload():
    from paper_2602_03002_gb300 import workloads as W
    w = W.config_small(n_steps=3, n_envs=10)
    sen = W.Sensor(sigma_abs=0.01, p_drop=0.05, max_latency=2, seed=(0xAB, 0xCD))
    return w, sen


def shard(n_envs, rank, world):
    return n_envs * rank // world, n_envs * (rank + 1) // world


def render(lo, hi, env_offset):
    """Frames of envs lo..hi-1 for steps 0..2 through the library (env_offset + local env = global id)."""
    import torch
    from paper_2602_03002_gb300 import rpl
    w, sen = workload()
    scene = rpl.Scene.from_workload(w, device=0)
    view = rpl.View(scene, hi - lo, w.n_links)
    view.set_cameras(w.cameras)
    view.set_sensor(sen)
    poses = torch.from_numpy(np.ascontiguousarray(w.poses[:, lo:hi])).to("cuda:0")
    frames = [view.render(poses[s], s, env_offset).cpu().numpy().copy() for s in range(3)]
    view.sync()
    return np.stack(frames)


def main(path):
    import torch.distributed as dist
    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, _ = workload()
    lo, hi = shard(w.n_envs, rank, world)
    mine = render(lo, hi, 1000 + lo)
    parts = [None] * world
    dist.all_gather_object(parts, mine)
    if rank == 0:
        np.save(path, np.concatenate(parts, axis=1))
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    main(sys.argv[1])
