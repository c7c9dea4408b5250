"""Batching: uneven cameras in one launch, launch shapes chosen by the autotuner, graph replay.

The launch shape (tile of 32 rays, one warp per tile / persistent grid-stride loop / per-SM tile
queues, contiguous or dealt in chunks, env index order or spatial order, query order, registers per
thread) must never change the depth: every shape gives bit-identical frames, also on ragged
cameras where tiles hang over the image edge.  Replaying the captured graph of the whole path must
continue the sensor history exactly like step-by-step rpl_render calls.
"""
import itertools

import numpy as np
import pytest

import oracle
from conftest import compare_depth
from paper_2602_03002_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [dict(tile_w=tw, tile_h=32 // tw, persistent=p, terrain_first=tf, min_blocks=mb, env_order=0, chunk_envs=0)
          for tw, p, tf, mb in itertools.product((8, 4, 16), (0, 1, 2), (0, 1), (8, 9, 10, 12))]
# the spatial env order with each scheduling, and per-SM queues dealt in chunks of 1, 3 and 7 envs
SHAPES += [dict(tile_w=tw, tile_h=32 // tw, persistent=p, terrain_first=0, min_blocks=8, env_order=o, chunk_envs=k)
           for tw, p, o, k in itertools.product((8, 4), (0, 1, 2), (0, 1), (0, 1, 3, 7)) if (o or k) and (p == 2 or k == 0)]


# the autotuner's 192 shapes
AUTOTUNE_SHAPES = [dict(tile_w=tw, tile_h=32 // tw, persistent=p, terrain_first=tf, min_blocks=mb, env_order=o,
                        chunk_envs=k)
                   for tw, (p, o, k), tf, mb in itertools.product(
                       (8, 4, 16), ((0, 0, 0), (0, 1, 0), (1, 0, 0), (1, 1, 0), (2, 0, 0), (2, 1, 0), (2, 0, 1), (2, 1, 1)),
                       (0, 1), (8, 9, 10, 12))]


def _ragged(w):
    torso = w.cameras[0].mount_link
    w.cameras = [W.pinhole(13, 7, 80.0, 50.0, torso, (0.10, 0.0, 0.30), 0.0, 45.0, 0.1, 3.0),
                 W.pinhole(21, 11, 90.0, 60.0, torso, (-0.10, 0.0, 0.30), 180.0, 40.0, 0.2, 2.5),
                 W.pinhole(3, 2, 60.0, 40.0, 0, (0.0, 0.15, 0.1), 90.0, 30.0, 0.05, 4.0)]
    return w


@pytest.mark.parametrize("ragged", [False, True])
def test_every_launch_shape_gives_identical_depth(cuda, rpl_lib, ragged):
    torch = cuda
    w = W.config_small(n_steps=2)
    if ragged:
        w = _ragged(w)
    sen = W.Sensor(sigma_abs=0.01, p_drop=0.05, max_latency=2, seed=(1, 2))
    scene = rpl_lib.Scene.from_workload(w)
    view = rpl_lib.View(scene, w.n_envs, w.n_links)
    view.set_cameras(w.cameras)
    view.set_sensor(sen)
    poses = torch.from_numpy(w.poses).cuda()
    view.render(poses[0], 0)
    ref = view.render(poses[1], 1).clone()
    for shape in SHAPES:
        rpl_lib.rpl_view_tuning_set(view.h, **shape)
        assert rpl_lib.rpl_view_tuning_get(view.h) == shape
        out = view.render(poses[1], 1)                      # re-render the same step
        assert torch.equal(out, ref), shape
    view.sync()


def test_graph_replay_continues_the_sensor_history(cuda, rpl_lib):
    torch = cuda
    w = W.config_small(n_steps=8)
    sen = W.Sensor(sigma_abs=0.01, p_drop=0.05, max_latency=3, seed=(31, 32))
    scene = rpl_lib.Scene.from_workload(w)
    poses = torch.from_numpy(w.poses).cuda()
    a = rpl_lib.View.from_workload(scene, w)
    a.set_sensor(sen)
    ref = [a.render(poses[s], s).clone() for s in range(8)]
    b = rpl_lib.View.from_workload(scene, w)
    b.set_sensor(sen)
    rpl_lib.rpl_view_tuning_set(b.h, tile_w=16, tile_h=2, persistent=1)
    stream = torch.cuda.Stream()
    pose_buf = torch.empty_like(poses[0])
    out = b.out_tensor()
    # the side stream must wait for the default stream: the caching allocator may have given pose_buf
    # and out memory that the direct renders' pending work on the default stream still uses
    stream.wait_stream(torch.cuda.current_stream())
    got = []
    with torch.cuda.stream(stream):
        for s in range(6):
            pose_buf.copy_(poses[s])
            step = rpl_lib.rpl_render_graph(b.h, pose_buf, 0, out, stream)
            assert step == s
            got.append(out.clone())
        # a plain render in between, then replays again
        got.append(b.render(poses[6], 6, 0, None, stream).clone())
        pose_buf.copy_(poses[7])
        assert rpl_lib.rpl_render_graph(b.h, pose_buf, 0, out, stream) == 7
        got.append(out.clone())
    stream.synchronize()
    b.sync()
    for s in range(8):
        assert torch.equal(got[s], ref[s]), s


def test_autotune_picks_a_shape_and_keeps_results(cuda, rpl_lib):
    torch = cuda
    w = W.config_small(n_steps=1)
    scene = rpl_lib.Scene.from_workload(w)
    view = rpl_lib.View.from_workload(scene, w)
    poses = torch.from_numpy(w.poses[0]).cuda()
    ref = view.render(poses, 0).clone()
    out = torch.empty_like(ref)
    best, ms = rpl_lib.rpl_view_autotune(view.h, poses, 0, 0, out, None, 2)
    assert best in AUTOTUNE_SHAPES and ms > 0 and len(AUTOTUNE_SHAPES) == 192
    assert rpl_lib.rpl_view_tuning_get(view.h) == best
    assert torch.equal(view.render(poses, 0), ref)


def test_uneven_four_cameras_vs_oracle(cuda, rpl_lib):
    """The batching configuration's camera set (front/back 80x60, left/right 48x36) on a small scene."""
    torch = cuda
    w = W.config_uneven(n_steps=1, n_envs=6, tiles=1, cell=0.2)
    scene = rpl_lib.Scene.from_workload(w)
    view = rpl_lib.View.from_workload(scene, w)
    offs, total = view.layout()
    assert offs == [0, 4800, 9600, 11328, 13056] and total == 13056
    poses = torch.from_numpy(w.poses[0]).cuda()
    best, _ = rpl_lib.rpl_view_autotune(view.h, poses, 0, 0, view.out_tensor(), None, 1)
    out = view.render(poses, 0).cpu().numpy()
    rng = np.random.default_rng(12)
    rays = oracle.all_rays(w.cameras, w.n_envs)
    rays = rays[rng.choice(len(rays), 4000, replace=False)]
    osc = oracle.OracleScene.from_workload(w)
    ref = osc.render(w.cameras, w.poses, 0, rays, w.sensor)
    o = np.asarray(offs)
    cam_w = np.array([c.width for c in w.cameras])
    got = out[rays[:, 0], o[rays[:, 1]] + rays[:, 3] * cam_w[rays[:, 1]] + rays[:, 2]]
    compare_depth(got, ref["depth"], ref["flags"], "uneven cameras")
    assert np.mean(ref["depth"] < 3.0) > 0.3


@pytest.mark.slow
def test_batching_configuration_at_full_size_in_graph_replay(cuda, rpl_lib):
    """4096 envs x 4 uneven cameras on the 20.48M-triangle terrain, replayed as the CUDA graph the
    benchmark times with the autotuned launch shape: sampled pixels against the oracle, and the
    replayed frame equal to a direct render of the same step."""
    torch = cuda
    w = W.config_uneven(n_steps=2)
    scene = rpl_lib.Scene.from_workload(w)
    view = rpl_lib.View.from_workload(scene, w)
    direct = rpl_lib.View.from_workload(scene, w)
    poses = torch.from_numpy(w.poses).cuda()
    out = view.out_tensor()
    best, _ = rpl_lib.rpl_view_autotune(view.h, poses[0], 0, 0, out, None, 1)
    rpl_lib.rpl_view_tuning_set(direct.h, **best)
    view.reset(None, 0)
    buf = poses[0].clone()
    frames = []
    for s in range(2):
        buf.copy_(poses[s])
        assert rpl_lib.rpl_render_graph(view.h, buf, 0, out) == s
        torch.cuda.synchronize()
        frames.append(out.cpu().numpy().copy())
        assert torch.equal(out, direct.render(poses[s], s)), s
    view.sync()
    offs, total = view.layout()
    rng = np.random.default_rng(31)
    n = 240
    c = rng.integers(0, 4, n)
    cw = np.array([cam.width for cam in w.cameras])
    ch = np.array([cam.height for cam in w.cameras])
    rays = np.stack([rng.integers(0, w.n_envs, n), c, (rng.random(n) * cw[c]).astype(np.int64),
                     (rng.random(n) * ch[c]).astype(np.int64)], 1).astype(np.int64)
    osc = oracle.OracleScene.from_workload(w)
    ref = osc.render(w.cameras, w.poses, 1, rays, w.sensor)
    o = np.asarray(offs)
    got = frames[1][rays[:, 0], o[rays[:, 1]] + rays[:, 3] * cw[rays[:, 1]] + rays[:, 2]]
    compare_depth(got, ref["depth"], ref["flags"], "batching full size")
    assert np.mean(ref["depth"] < 3.0) > 0.3


@pytest.mark.parametrize("n_envs,size", [(1, (3, 2)), (2, (13, 7)), (40, (9, 5))])
def test_per_sm_queues_with_fewer_tiles_than_queues(cuda, rpl_lib, n_envs, size):
    """Per-SM tile queues when most queues are empty (fewer tiles than SMs) or hold one or two tiles:
    every tile is still rendered once, giving the frames of the one-warp-per-tile launch."""
    torch = cuda
    w = W.config_small(n_steps=2, n_envs=n_envs)
    torso = w.cameras[0].mount_link
    w.cameras = [W.pinhole(size[0], size[1], 80.0, 50.0, torso, (0.10, 0.0, 0.30), 0.0, 45.0, 0.1, 3.0)]
    sen = W.Sensor(sigma_abs=0.01, p_drop=0.05, max_latency=1, seed=(5, 6))
    scene = rpl_lib.Scene.from_workload(w)
    view = rpl_lib.View(scene, w.n_envs, w.n_links)
    view.set_cameras(w.cameras)
    view.set_sensor(sen)
    poses = torch.from_numpy(w.poses).cuda()
    ref = [view.render(poses[s], s).clone() for s in range(2)]
    for tw in (8, 4, 16):
        rpl_lib.rpl_view_tuning_set(view.h, tile_w=tw, tile_h=32 // tw, persistent=2)
        view.reset(None, 0)
        for s in range(2):
            out = torch.full_like(ref[s], -1.0)
            view.render(poses[s], s, 0, out)
            assert torch.equal(out, ref[s]), (tw, s)
    view.sync()


def test_spatial_env_order_with_coincident_and_outside_envs(cuda, rpl_lib):
    """The spatial processing order buckets envs by position: envs that share one position (one
    bucket, arbitrary order inside it) and envs far outside the terrain (clamped to the edge cells)
    must render the same frames in env index order and in spatial order, contiguous or dealt in
    chunks."""
    torch = cuda
    w = W.config_small(n_steps=2, n_envs=12)
    poses = w.poses.copy()
    poses[:, 1:6, :, :2] += poses[:, :1, :1, :2] - poses[:, 1:6, :1, :2]      # envs 1-5 stand where env 0 does
    poses[:, 9:12, :, 0] += 1.0e4                                           # envs 9-11 far outside the terrain
    sen = W.Sensor(sigma_abs=0.01, p_drop=0.05, max_latency=1, seed=(7, 8))
    scene = rpl_lib.Scene.from_workload(w)
    view = rpl_lib.View(scene, w.n_envs, w.n_links)
    view.set_cameras(w.cameras)
    view.set_sensor(sen)
    pt = torch.from_numpy(poses).cuda()
    rpl_lib.rpl_view_tuning_set(view.h, tile_w=4, tile_h=8, persistent=2, env_order=0, chunk_envs=0)
    ref = [view.render(pt[s], s).clone() for s in range(2)]
    assert bool((ref[1][9:] == 3.0).any())                                  # the outside envs see nothing
    for order, chunk, pers in ((1, 0, 2), (1, 1, 2), (1, 5, 2), (1, 0, 0), (1, 0, 1)):
        rpl_lib.rpl_view_tuning_set(view.h, tile_w=4, tile_h=8, persistent=pers, env_order=order, chunk_envs=chunk)
        view.reset(None, 0)
        for s in range(2):
            assert torch.equal(view.render(pt[s], s), ref[s]), (order, chunk, pers, s)
    view.sync()
