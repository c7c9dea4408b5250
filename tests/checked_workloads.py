"""Renders shared by the bounds-checked-build test: the same calls run in a process on the normal
library and in a process on librpl_checked.so (RPL_CHECKED=1), whose frames must be identical and
whose error words must stay clear.  Run as a script it writes the frames to the given .npz path."""
import sys

import numpy as np


def render_all():
    import torch
    from paper_2602_03002_gb300 import rpl, workloads as W
    out = {}
    sen = W.Sensor(sigma_abs=0.01, p_drop=0.05, max_latency=2, seed=(0xB0, 0x0D))
    w = W.config_small(n_steps=3, n_envs=6)
    torso = w.cameras[0].mount_link
    w.cameras = w.cameras + [W.pinhole(13, 7, 80.0, 50.0, torso, (0.0, 0.12, 0.30), 90.0, 45.0, 0.1, 3.0)]
    poses = torch.from_numpy(w.poses).cuda()
    for kind in (rpl.RPL_BVH2, rpl.RPL_BVH4, rpl.RPL_BVH8Q8):
        scene = rpl.Scene.from_workload(w, bvh_kind=kind)
        view = rpl.View.from_workload(scene, w)
        view.set_sensor(sen)
        for s in range(3):
            out["kind%d_step%d" % (kind, s)] = view.render(poses[s], s).cpu().numpy()
        view.sync()
        # the fused server launch
        v2 = rpl.View.from_workload(scene, w)
        v2.set_sensor(sen)
        server = rpl.Server(scene, max_batch=4)
        o = v2.out_tensor()
        server.wait(server.submit(v2, poses[0], 0, o))
        out["kind%d_server" % kind] = o.cpu().numpy()
        server.close()
    # downsampled cameras, randomised mounts, side masking
    p = W.config_small(n_steps=2, n_envs=4)
    cams = W.perception_cameras(p.cameras[0].mount_link, 2, raw=(40, 30), downsample=5)
    p.cameras = cams
    p.mount_delta, p.per_env_intrinsics = W.camera_randomization(4, cams, seed=3)
    p.rsm_modes, p.rsm_cols = np.array([0, 1, 2, 1], np.uint8), (0, 1, 2)
    scene = rpl.Scene.from_workload(p)
    view = rpl.View.from_workload(scene, p)
    view.set_sensor(sen)
    pp = torch.from_numpy(p.poses).cuda()
    for s in range(2):
        out["perception_step%d" % s] = view.render(pp[s], s).cpu().numpy()
    view.sync()
    # the no-allocation entry point
    o = torch.empty((w.n_envs, sum(c.width * c.height for c in w.cameras)), device="cuda")
    scene = rpl.Scene.from_workload(w)
    rpl.View.from_workload(scene, w)
    rpl.rpl_render_static_scratch(scene.h, w.cameras, w.n_envs, w.n_links, poses[0], o)
    torch.cuda.synchronize()
    rpl.rpl_static_scratch_status(scene.h)   # raises DEVICE_FAULT if the kernels recorded a fault
    out["noalloc"] = o.cpu().numpy()
    # the per-SM tile-queue launch shape
    view = rpl.View.from_workload(scene, w)
    view.set_sensor(sen)
    rpl.rpl_view_tuning_set(view.h, tile_w=4, tile_h=8, persistent=2, min_blocks=8)
    for s in range(2):
        out["queued_step%d" % s] = view.render(poses[s], s).cpu().numpy()
    view.sync()
    return out


if __name__ == "__main__":
    frames = render_all()
    np.savez(sys.argv[1], **frames)
