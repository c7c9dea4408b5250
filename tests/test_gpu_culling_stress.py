"""GPU parity under randomised cameras: the per-camera and per-tile culling (view pyramids, entry
subtrees, oriented-box link tests) must never drop geometry a ray can reach.

Each case mounts three cameras on random links with random offsets and orientations (any roll),
fields of view from narrow to very wide, sizes from 3 px to 48 px (ragged tiles), principal points
moved up to 60 % of the image size (often off the image), ranges d_max from 0.4 m to 25 m, per-env
intrinsics jitter, z-depth or range depth, one of the three tile shapes and, from seed 7 on, one
camera ray cast at 2x or 3x and block-averaged; the frames are compared
with the FP64 oracle pixel by pixel.  (Seed 1 has a tile row one pixel tall: two corners of its
pyramid coincide, and an FP32 cross product of a corner ray with itself is not exactly zero.)
"""
import dataclasses

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from conftest import compare_depth
from paper_2602_03002_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TILES = [(4, 8), (8, 4), (16, 2)]


def _random_cameras(rng, seed, n_links):
    cams = []
    for k in range(3):
        width, height = int(rng.integers(3, 49)), int(rng.integers(2, 41))
        ds = 2 + seed % 2 if (k == 2 and seed > 6) else 1   # later seeds: one downsampled camera
        width, height = max(ds, width - width % ds), max(ds, height - height % ds)
        cam = W.pinhole(width, height, float(rng.uniform(20.0, 150.0)), float(rng.uniform(15.0, 120.0)),
                        int(rng.integers(0, n_links)), tuple(rng.uniform(-0.3, 0.3, 3)), 0.0, 0.0,
                        0.05, float(rng.choice([0.4, 1.5, 4.0, 25.0])))
        q = Rotation.random(random_state=1000 * seed + k).as_quat()   # x, y, z, w
        cams.append(dataclasses.replace(cam, offset_quat=tuple(float(v) for v in q),
                                        cx=cam.cx + float(rng.uniform(-0.6, 0.6)) * width,
                                        cy=cam.cy + float(rng.uniform(-0.6, 0.6)) * height, downsample=ds))
    return cams


@pytest.mark.parametrize("seed", list(range(1, 13)))
def test_random_cameras_match_oracle(cuda, rpl_lib, seed):
    torch = cuda
    rng = np.random.default_rng(seed)
    w = W.config_small(n_steps=1, n_envs=6)
    w.cameras = _random_cameras(rng, seed, w.n_links)
    intr = np.empty((w.n_envs, len(w.cameras), 4), np.float32)
    for c, cam in enumerate(w.cameras):
        intr[:, c, 0] = cam.fx * rng.uniform(0.95, 1.05, w.n_envs)
        intr[:, c, 1] = cam.fy * rng.uniform(0.95, 1.05, w.n_envs)
        intr[:, c, 2] = cam.cx + rng.uniform(-1.0, 1.0, w.n_envs)
        intr[:, c, 3] = cam.cy + rng.uniform(-1.0, 1.0, w.n_envs)
    sen = W.Sensor(depth_kind=int(seed % 2))
    scene = rpl_lib.Scene.from_workload(w)
    view = rpl_lib.View(scene, w.n_envs, w.n_links)
    view.set_cameras(w.cameras, intr)
    view.set_sensor(sen)
    tw, th = TILES[seed % 3]
    rpl_lib.rpl_view_tuning_set(view.h, tw, th, 0, seed % 2, 10)
    got = view.render(torch.from_numpy(w.poses[0]).cuda(), 0).cpu().numpy().copy()
    osc = oracle.OracleScene.from_workload(w)
    rays = oracle.all_rays(w.cameras, w.n_envs)
    ref = osc.render(w.cameras, w.poses, 0, rays, sen, per_env_intrinsics=intr)
    compare_depth(got, ref["depth"], ref["flags"], "random cameras, seed %d" % seed)
    # the frames see something: geometry within range on a good share of the pixels, and link
    # meshes on some of them (without the links those pixels see further; 63 to 2,083 of them)
    dmax = np.concatenate([np.full(c.out_width * c.out_height, c.d_max) for c in w.cameras])
    assert np.mean(ref["depth"].reshape(w.n_envs, -1) < dmax[None, :] - 1e-6) > 0.05
    bare = rpl_lib.Scene(w.terrain_verts, w.terrain_tris)
    bview = rpl_lib.View(bare, w.n_envs, w.n_links)
    bview.set_cameras(w.cameras, intr)
    bview.set_sensor(sen)
    far = bview.render(torch.from_numpy(w.poses[0]).cuda(), 0).cpu().numpy()
    assert np.count_nonzero(far.reshape(-1) > got.reshape(-1) + 1e-3) > 0
