"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element.

Small workload (8 envs x 2 cams x 32x24, 3,200-tri terrain, 20 box links): full frames over several
steps, sensor off and on.  Edge cases: ragged tiles, uneven cameras, per-env intrinsics, empty
terrain, zero envs, links without meshes, range depth, graph capture, host buffers, env sharding.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from conftest import compare_depth
from paper_2602_03002_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _render_seq(torch, rpl, w, steps, sensor=None, env_offset=0, view=None, scene=None):
    scene = scene or rpl.Scene.from_workload(w)
    if view is None:
        view = rpl.View(scene, w.n_envs, w.n_links)
        view.set_cameras(w.cameras, w.per_env_intrinsics)
        view.set_sensor(sensor if sensor is not None else w.sensor)
    poses = torch.from_numpy(w.poses).cuda()
    outs = []
    for s in steps:
        outs.append(view.render(poses[s - w.step0], s, env_offset).cpu().numpy().copy())
    torch.cuda.synchronize()
    view.sync()
    return outs, scene, view


def test_small_sensor_off_full_frames(cuda, rpl_lib):
    w = W.config_small(n_steps=3)
    outs, _, _ = _render_seq(cuda, rpl_lib, w, range(3))
    osc = oracle.OracleScene.from_workload(w)
    rays = oracle.all_rays(w.cameras, w.n_envs)
    for s in range(3):
        ref = osc.render(w.cameras, w.poses, s, rays, w.sensor)
        compare_depth(outs[s], ref["depth"], ref["flags"], "small step %d" % s)
        assert np.mean(ref["depth"] < 3.0) > 0.5   # the frames do see geometry


def test_small_sensor_on(cuda, rpl_lib):
    w = W.config_small(n_steps=6)
    sen = W.Sensor(sigma_abs=0.01, sigma_rel=0.02, p_drop=0.05, fill=0.0, max_latency=3, seed=(0x1234, 0xBEEF))
    outs, _, _ = _render_seq(cuda, rpl_lib, w, range(6), sensor=sen, env_offset=17)
    osc = oracle.OracleScene.from_workload(w)
    rays = oracle.all_rays(w.cameras, w.n_envs)
    for s in range(6):
        ref = osc.render(w.cameras, w.poses, s, rays, sen, s_first=np.zeros(w.n_envs, np.int64), env_offset=17)
        got = outs[s].reshape(-1)
        # dropout decisions are integer comparisons of Philox words: bit-exact
        dropped = (ref["flags"] & oracle.FLAG_DROPPED) != 0
        assert np.array_equal(got == np.float32(sen.fill), dropped), "dropout mask differs at step %d" % s
        compare_depth(got, ref["depth"], ref["flags"], "small sensor step %d" % s)


@pytest.mark.parametrize("leaf,node_cost", [(1, 0.0), (2, 0.0), (8, 100.0)])
def test_leaf_sizes(cuda, rpl_lib, leaf, node_cost):
    """Leaves of 1 to 8 triangles (the range the device node layout encodes) give the oracle's frames.

    A node cost of 100 makes the builder keep leaves as large as allowed, so the 8-triangle case
    holds leaves with 5 to 8 triangles (checked through the node count)."""
    w = W.config_small(n_steps=1)
    scene = rpl_lib.Scene.from_workload(w, max_leaf_size=leaf, sah_node_cost=node_cost)
    info = scene.info()
    if leaf == 8:
        # a binary tree with k leaves has k - 1 nodes: mean leaf size above 5
        assert info["terrain_nodes"] * 5 < info["terrain_tris"], info
    else:
        assert info["terrain_nodes"] * leaf >= info["terrain_tris"] - leaf, info
    outs, _, _ = _render_seq(cuda, rpl_lib, w, [0], scene=scene)
    osc = oracle.OracleScene.from_workload(w)
    rays = oracle.all_rays(w.cameras, w.n_envs)
    ref = osc.render(w.cameras, w.poses, 0, rays, w.sensor)
    compare_depth(outs[0], ref["depth"], ref["flags"], "leaf size %d" % leaf)


def test_latency_is_a_delayed_raw_frame_bitexact(cuda, rpl_lib):
    """Output of step s with latency k equals the undelayed output of step s' = max(s-k, first)."""
    w = W.config_small(n_steps=8)
    delayed = W.Sensor(max_latency=3, seed=(7, 9))
    plain = W.Sensor(max_latency=0, seed=(7, 9))
    a, scene, _ = _render_seq(cuda, rpl_lib, w, range(8), sensor=delayed)
    b, _, _ = _render_seq(cuda, rpl_lib, w, range(8), sensor=plain, scene=scene)
    P = w.pixels_per_env
    offs = w.cam_offsets()
    seen = set()
    for s in range(8):
        for e in range(w.n_envs):
            for c in range(len(w.cameras)):
                wl = oracle.philox4x32_10([e, c, 0xFFFFFFFF, s], [7, 9])
                k = (int(wl[0]) * 4) >> 32
                src = max(s - k, 0)
                seen.add(k)
                sl = slice(offs[c], offs[c + 1])
                assert np.array_equal(a[s][e, sl], b[src][e, sl]), (s, e, c, k)
    assert seen == {0, 1, 2, 3}


def test_env_sharding_is_bitexact(cuda, rpl_lib):
    w = W.config_small(n_steps=4)
    sen = W.Sensor(sigma_abs=0.01, p_drop=0.03, max_latency=2, seed=(5, 6))
    full, scene, _ = _render_seq(cuda, rpl_lib, w, range(4), sensor=sen, env_offset=100)
    import copy
    halves = []
    for lo, hi in ((0, 3), (3, 8)):
        wh = copy.copy(w)
        wh.poses = w.poses[:, lo:hi]
        o, _, _ = _render_seq(cuda, rpl_lib, wh, range(4), sensor=sen, env_offset=100 + lo, scene=scene)
        halves.append(o)
    for s in range(4):
        assert np.array_equal(full[s], np.concatenate([halves[0][s], halves[1][s]]))


def test_ragged_uneven_cameras_per_env_intrinsics(cuda, rpl_lib):
    w = W.config_small(n_steps=2, n_envs=5)
    torso = w.cameras[0].mount_link
    w.cameras = [W.pinhole(13, 7, 80.0, 50.0, torso, (0.10, 0.0, 0.30), 0.0, 45.0, 0.1, 3.0),
                 W.pinhole(21, 11, 90.0, 60.0, torso, (-0.10, 0.0, 0.30), 180.0, 40.0, 0.2, 2.5),
                 W.pinhole(3, 2, 60.0, 40.0, 0, (0.0, 0.15, 0.1), 90.0, 30.0, 0.05, 4.0)]
    rng = np.random.default_rng(3)
    intr = np.empty((w.n_envs, 3, 4), np.float32)
    for c, cam in enumerate(w.cameras):
        intr[:, c, 0] = cam.fx * rng.uniform(0.9, 1.1, w.n_envs)
        intr[:, c, 1] = cam.fy * rng.uniform(0.9, 1.1, w.n_envs)
        intr[:, c, 2] = cam.cx + rng.uniform(-0.5, 0.5, w.n_envs)
        intr[:, c, 3] = cam.cy + rng.uniform(-0.5, 0.5, w.n_envs)
    w.per_env_intrinsics = intr
    outs, _, view = _render_seq(cuda, rpl_lib, w, range(2))
    offs, total = view.layout()
    assert total == 13 * 7 + 21 * 11 + 3 * 2 and offs[:3] == [0, 91, 322]
    osc = oracle.OracleScene.from_workload(w)
    rays = oracle.all_rays(w.cameras, w.n_envs)
    for s in range(2):
        ref = osc.render(w.cameras, w.poses, s, rays, w.sensor, per_env_intrinsics=intr)
        compare_depth(outs[s], ref["depth"], ref["flags"], "ragged step %d" % s)


@pytest.mark.parametrize("tile,depth_kind", [((4, 8), 0), ((8, 4), 1), ((16, 2), 0)])
def test_principal_point_outside_the_image(cuda, rpl_lib, tile, depth_kind):
    """Per-tile view pyramids stay conservative when the optical axis misses the image (principal
    point above the image, and left of it for one camera, right of it for the other), for every tile
    shape and both depth kinds.  Moving the principal point up turns the torso cameras towards the
    legs: about a fifth of the pixels see link meshes (2,391 of 12,288 in the oracle's frames)."""
    import dataclasses
    torch = cuda
    w = W.config_small(n_steps=1)
    w.cameras = [dataclasses.replace(cam, cx=(-3.0 if c == 0 else cam.width + 2.0), cy=-3.0)
                 for c, cam in enumerate(w.cameras)]
    sen = W.Sensor(depth_kind=depth_kind)
    scene = rpl_lib.Scene.from_workload(w)
    view = rpl_lib.View(scene, w.n_envs, w.n_links)
    view.set_cameras(w.cameras)
    view.set_sensor(sen)
    rpl_lib.rpl_view_tuning_set(view.h, tile[0], tile[1], 0, 1, 10)
    poses = torch.from_numpy(w.poses).cuda()
    got = view.render(poses[0], 0).cpu().numpy().copy()
    osc = oracle.OracleScene.from_workload(w)
    rays = oracle.all_rays(w.cameras, w.n_envs)
    ref = osc.render(w.cameras, w.poses, 0, rays, sen)
    compare_depth(got, ref["depth"], ref["flags"], "principal point outside, tile %dx%d" % tile)
    # the links are in view: without their meshes some pixels see further
    bare = rpl_lib.Scene(w.terrain_verts, w.terrain_tris)
    bview = rpl_lib.View(bare, w.n_envs, w.n_links)
    bview.set_cameras(w.cameras)
    bview.set_sensor(sen)
    far = bview.render(poses[0], 0).cpu().numpy()
    assert np.count_nonzero(far.reshape(-1) > got.reshape(-1) + 1e-3) > 1000


def test_range_depth_kind(cuda, rpl_lib):
    w = W.config_small(n_steps=1, n_envs=3)
    sen = W.Sensor(depth_kind=1)
    outs, _, _ = _render_seq(cuda, rpl_lib, w, [0], sensor=sen)
    osc = oracle.OracleScene.from_workload(w)
    rays = oracle.all_rays(w.cameras, w.n_envs)
    ref = osc.render(w.cameras, w.poses, 0, rays, sen)
    compare_depth(outs[0], ref["depth"], ref["flags"], "range")


def test_empty_terrain_and_missing_links(cuda, rpl_lib):
    w = W.config_small(n_steps=1, n_envs=4)
    w.terrain_verts = np.zeros((0, 3), np.float32)
    w.terrain_tris = np.zeros((0, 3), np.int32)
    # links 5 and 7 have no mesh
    w.link_verts[5] = np.zeros((0, 3), np.float32)
    w.link_tris[5] = np.zeros((0, 3), np.int32)
    w.link_verts[7] = np.zeros((0, 3), np.float32)
    w.link_tris[7] = np.zeros((0, 3), np.int32)
    outs, scene, _ = _render_seq(cuda, rpl_lib, w, [0])
    info = scene.info()
    assert info["terrain_tris"] == 0 and info["n_links"] == 18
    osc = oracle.OracleScene.from_workload(w)
    rays = oracle.all_rays(w.cameras, w.n_envs)
    ref = osc.render(w.cameras, w.poses, 0, rays, w.sensor)
    compare_depth(outs[0], ref["depth"], ref["flags"], "no terrain")


def test_zero_envs(cuda, rpl_lib):
    w = W.config_small(n_steps=1)
    scene = rpl_lib.Scene.from_workload(w)
    view = rpl_lib.View(scene, 0, w.n_links)
    view.set_cameras(w.cameras)
    poses = cuda.zeros((0, w.n_links, 7), device="cuda")
    out = cuda.zeros((0, w.pixels_per_env), device="cuda")
    view.render(poses, 0, 0, out)
    view.sync()


def test_graph_capture_replays_the_same_frame(cuda, rpl_lib):
    torch = cuda
    w = W.config_small(n_steps=2)
    scene = rpl_lib.Scene.from_workload(w)
    view = rpl_lib.View.from_workload(scene, w)
    poses = torch.from_numpy(w.poses[0]).cuda()
    direct = view.render(poses, 0).clone()
    out = torch.zeros_like(direct)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rpl_lib.rpl_render(view.h, poses, 0, 0, out, s)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, direct)


def test_host_buffers_match_device_path(cuda, rpl_lib):
    torch = cuda
    w = W.config_small(n_steps=2)
    scene = rpl_lib.Scene.from_workload(w)
    va = rpl_lib.View.from_workload(scene, w)
    vb = rpl_lib.View.from_workload(scene, w)
    for s in range(2):
        dev = va.render(torch.from_numpy(w.poses[s]).cuda(), s).cpu()
        host_out = torch.empty_like(dev).pin_memory()
        vb.render(torch.from_numpy(w.poses[s]).pin_memory(), s, out=host_out)
        assert torch.equal(host_out, dev)


def test_argument_errors(cuda, rpl_lib):
    torch = cuda
    w = W.config_small(n_steps=3)
    scene = rpl_lib.Scene.from_workload(w)
    view = rpl_lib.View.from_workload(scene, w)
    poses = torch.from_numpy(w.poses[0]).cuda()
    view.render(poses, 10)
    with pytest.raises(rpl_lib.RplError) as ei:
        view.render(poses, 12)          # skipped a step
    assert ei.value.status == 1
    view.render(poses, 11)
    view.reset(None, 40)
    view.render(poses, 40)
    bad = [dict(width=4, height=4, fx=1.0, fy=1.0, cx=1.5, cy=1.5, mount_link=w.n_links, offset_pos=(0, 0, 0),
                offset_quat=(0, 0, 0, 1), d_min=0.1, d_max=3.0)]
    with pytest.raises(rpl_lib.RplError):
        view.set_cameras(bad)
    with pytest.raises(rpl_lib.RplError):
        rpl_lib.Scene(np.zeros((2, 3), np.float32), np.array([[0, 1, 2]], np.int32))   # index out of range
    with pytest.raises(rpl_lib.RplError):
        scene.add_link(0, w.link_verts[0], w.link_tris[0])                           # frozen by the view


def test_partial_reset_restarts_history(cuda, rpl_lib):
    torch = cuda
    w = W.config_small(n_steps=6)
    sen = W.Sensor(max_latency=3, seed=(11, 12))
    scene = rpl_lib.Scene.from_workload(w)
    view = rpl_lib.View(scene, w.n_envs, w.n_links)
    view.set_cameras(w.cameras)
    view.set_sensor(sen)
    poses = torch.from_numpy(w.poses).cuda()
    outs = []
    mask = np.zeros(w.n_envs, np.uint8)
    mask[[1, 4]] = 1
    for s in range(6):
        if s == 3:
            view.reset(mask, 3)
        outs.append(view.render(poses[s], s).cpu().numpy())
    s_first = np.where(mask > 0, 3, 0).astype(np.int64)
    osc = oracle.OracleScene.from_workload(w)
    rays = oracle.all_rays(w.cameras, w.n_envs)
    for s in (3, 4, 5):
        ref = osc.render(w.cameras, w.poses, s, rays, sen, s_first=s_first)
        compare_depth(outs[s], ref["depth"], ref["flags"], "reset step %d" % s)


def test_counters(cuda, rpl_lib):
    torch = cuda
    w = W.config_small(n_steps=1)
    scene = rpl_lib.Scene.from_workload(w)
    view = rpl_lib.View.from_workload(scene, w)
    poses = torch.from_numpy(w.poses[0]).cuda()
    plain = view.render(poses, 0).clone()
    out = torch.empty_like(plain)
    c = view.render_counters(poses, 0, out=out)
    assert torch.equal(out, plain)
    assert c["rays"] == w.rays_per_step
    assert c["terrain_nodes"] >= c["rays"] and c["terrain_tris"] > 0
    assert 0 < c["link_boxes"] < w.rays_per_step * w.n_links      # links outside the view volume are culled


def test_max_cameras_and_links(cuda, rpl_lib):
    """RPL_MAX_CAMERAS cameras of different sizes and RPL_MAX_LINKS links in one view."""
    w = W.config_small(n_steps=1, n_envs=3)
    rng = np.random.default_rng(9)
    n_links = rpl_lib.RPL_MAX_LINKS
    extra = n_links - w.n_links
    P = w.poses[0]
    # the extra links are small boxes floating around each env's robot
    add = np.zeros((3, extra, 7), np.float32)
    add[..., :3] = P[:, :1, :3] + rng.uniform(-1.2, 1.2, (3, extra, 3)).astype(np.float32)
    add[..., 2] = P[:, :1, 2] - rng.uniform(0.2, 0.9, (3, extra)).astype(np.float32)
    add[..., 3:] = np.asarray([Rotation.random(random_state=k).as_quat() for k in range(3 * extra)],
                              np.float32).reshape(3, extra, 4)
    w.poses = np.concatenate([P, add], axis=1)[None]
    for k in range(extra):
        v, t = W.box_mesh(rng.uniform(0.03, 0.12, 3), (0, 0, 0), subdiv=1 + k % 2)
        w.link_verts.append(v)
        w.link_tris.append(t)
    torso = w.cameras[0].mount_link
    w.cameras = [W.pinhole(5 + 3 * c, 4 + 2 * c, 70.0 + 3 * c, 50.0, torso, (0.1 * math.cos(c), 0.1 * math.sin(c), 0.3),
                           45.0 * c, 40.0 + 3 * c, 0.1, 3.0) for c in range(rpl_lib.RPL_MAX_CAMERAS)]
    outs, _, _ = _render_seq(cuda, rpl_lib, w, [0])
    osc = oracle.OracleScene.from_workload(w)
    rays = oracle.all_rays(w.cameras, w.n_envs)
    ref = osc.render(w.cameras, w.poses, 0, rays, w.sensor)
    compare_depth(outs[0], ref["depth"], ref["flags"], "max sizes")
    with pytest.raises(rpl_lib.RplError):
        rpl_lib.View(rpl_lib.Scene.from_workload(W.config_small(n_steps=1)), 2, n_links + 1)


def test_async_host_output_equals_synchronous(cuda, rpl_lib):
    """With rpl_view_host_async the host copies run on the view's copy stream from two staging
    buffers in turn; after rpl_sync every step's host frame equals the synchronous result."""
    torch = cuda
    w = W.config_small(n_steps=6, n_envs=5)
    sen = W.Sensor(sigma_abs=0.01, p_drop=0.05, max_latency=2, seed=(0xA5, 0x5A))
    scene = rpl_lib.Scene.from_workload(w)
    a = rpl_lib.View.from_workload(scene, w)
    a.set_sensor(sen)
    b = rpl_lib.View.from_workload(scene, w)
    b.set_sensor(sen)
    rpl_lib.rpl_view_host_async(b.h, True)
    poses = [torch.from_numpy(w.poses[s]).pin_memory() for s in range(6)]
    P = b.layout()[1]
    ref = [a.render(poses[s], s).cpu().clone() for s in range(6)]     # synchronous host path
    outs = [torch.empty((w.n_envs, P), dtype=torch.float32).pin_memory() for _ in range(6)]
    for s in range(6):
        rpl_lib.rpl_render(b.h, poses[s], s, 0, outs[s], None)
    b.sync()
    for s in range(6):
        assert torch.equal(outs[s], ref[s]), s
    rpl_lib.rpl_view_host_async(b.h, False)
    again = torch.empty((w.n_envs, P), dtype=torch.float32).pin_memory()
    rpl_lib.rpl_render(b.h, poses[5], 5, 0, again, None)          # synchronous again: re-render step 5
    assert torch.equal(again, ref[5])
