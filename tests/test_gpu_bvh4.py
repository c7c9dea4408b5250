"""The four-wide terrain BVH (FP32 boxes, collapsed from the binary tree).

Collapsing only regroups nodes and the triangle test is the same FP32 code, so the four-wide tree
must give bit-identical depth to the binary one on every workload and launch shape (the minimum
over the same triangle distances does not depend on the visiting order); the node count and bytes
follow the layout, and the full-size scale workload is checked against the oracle on samples."""
import itertools

import numpy as np
import pytest

import oracle
from conftest import compare_depth
from paper_2602_03002_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _scene(rpl, w, kind):
    s = rpl.Scene(w.terrain_verts, w.terrain_tris, bvh_kind=kind)
    for l, (v, t) in enumerate(zip(w.link_verts, w.link_tris)):
        s.add_link(l, v, t)
    return s


def _frames(torch, rpl, w, scene, sensor, steps, tuning=None):
    view = rpl.View(scene, w.n_envs, w.n_links)
    view.set_cameras(w.cameras, w.per_env_intrinsics)
    view.set_sensor(sensor)
    if tuning:
        rpl.rpl_view_tuning_set(view.h, **tuning)
    poses = torch.from_numpy(w.poses).cuda()
    outs = [view.render(poses[s], s).clone() for s in steps]
    view.sync()
    return outs


def test_four_wide_matches_binary_bitexact_on_every_shape(cuda, rpl_lib):
    w = W.config_small(n_steps=2)
    torso = w.cameras[0].mount_link
    w.cameras = w.cameras + [W.pinhole(13, 7, 80.0, 50.0, torso, (0.0, 0.12, 0.30), 90.0, 45.0, 0.1, 3.0)]
    sen = W.Sensor(sigma_abs=0.01, p_drop=0.05, max_latency=1, seed=(3, 4))
    b2, b4 = _scene(rpl_lib, w, rpl_lib.RPL_BVH2), _scene(rpl_lib, w, rpl_lib.RPL_BVH4)
    ref = _frames(cuda, rpl_lib, w, b2, sen, range(2))
    for tw, pers, tf, mb in itertools.product((8, 4, 16), (0, 1), (0, 1), (8, 10, 12)):
        t = dict(tile_w=tw, tile_h=32 // tw, persistent=pers, terrain_first=tf, min_blocks=mb)
        got = _frames(cuda, rpl_lib, w, b4, sen, range(2), t)
        for s in range(2):
            assert cuda.equal(got[s], ref[s]), (t, s)
    i2, i4 = b2.info(), b4.info()
    assert i4["terrain_tris"] == i2["terrain_tris"] == 3200
    assert i4["terrain_bytes"] == i4["terrain_nodes"] * 128 + 3200 * 48
    assert i4["terrain_nodes"] < i2["terrain_nodes"] / 2 and i4["terrain_depth"] < i2["terrain_depth"]


def test_four_wide_server_and_graph(cuda, rpl_lib):
    """The fused server launch and graph replay use the four-wide kernels too."""
    torch = cuda
    w = W.config_small(n_steps=3, n_envs=6)
    sen = W.Sensor(sigma_abs=0.01, p_drop=0.05, max_latency=2, seed=(5, 6))
    scene = _scene(rpl_lib, w, rpl_lib.RPL_BVH4)
    ref = _frames(torch, rpl_lib, w, _scene(rpl_lib, w, rpl_lib.RPL_BVH2), sen, range(3))
    v = rpl_lib.View(scene, w.n_envs, w.n_links)
    v.set_cameras(w.cameras)
    v.set_sensor(sen)
    server = rpl_lib.Server(scene, max_batch=4, n_streams=2)
    poses = torch.from_numpy(w.poses).cuda()
    out = v.out_tensor()
    for s in range(3):
        server.wait(server.submit(v, poses[s], s, out))
        assert torch.equal(out, ref[s]), s
    server.close()
    g = rpl_lib.View(scene, w.n_envs, w.n_links)
    g.set_cameras(w.cameras)
    g.set_sensor(sen)
    buf = poses[0].clone()
    out2 = g.out_tensor()
    for s in range(3):
        buf.copy_(poses[s])
        assert rpl_lib.rpl_render_graph(g.h, buf, 0, out2) == s
        torch.cuda.synchronize()
        assert torch.equal(out2, ref[s]), s
    g.sync()


@pytest.mark.slow
def test_four_wide_scale_sampled(cuda, rpl_lib):
    torch = cuda
    w = W.config_scale(n_steps=2)
    scene = _scene(rpl_lib, w, rpl_lib.RPL_BVH4)
    view = rpl_lib.View.from_workload(scene, w)
    poses = torch.from_numpy(w.poses).cuda()
    outs = [view.render(poses[s], s).cpu().numpy() for s in range(2)]
    view.sync()
    rng = np.random.default_rng(44)
    n = 256
    rays = np.stack([rng.integers(0, w.n_envs, n), rng.integers(0, 2, n), rng.integers(0, 64, n),
                     rng.integers(0, 48, n)], 1).astype(np.int64)
    osc = oracle.OracleScene.from_workload(w)
    ref = osc.render(w.cameras, w.poses, 1, rays, w.sensor, s_first=np.zeros(w.n_envs, np.int64))
    got = outs[1][rays[:, 0], rays[:, 1] * 3072 + rays[:, 3] * 64 + rays[:, 2]]
    compare_depth(got, ref["depth"], ref["flags"], "bvh4 scale")
    info = scene.info()
    assert info["terrain_tris"] == 20_480_000
