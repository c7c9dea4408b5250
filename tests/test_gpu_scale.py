"""Parity at the full benchmark size: 4096 envs x 2 cameras x 64x48 px against the 20.48M-triangle
terrain and 30 links of 512 triangles, sensor on (sigma 0.01 m, 2 % dropout, latency 0-3), in the
launch configuration the benchmark times.  The oracle recomputes a sample of rays one by one
(uniform plus rays next to depth discontinuities); properties that hold at any size are checked on
every pixel."""
import math

import numpy as np
import pytest

import oracle
from conftest import compare_depth
from paper_2602_03002_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def scale(cuda, rpl_lib):
    torch = cuda
    w = W.config_scale(n_steps=4)
    scene = rpl_lib.Scene.from_workload(w)
    view = rpl_lib.View.from_workload(scene, w)
    poses = torch.from_numpy(w.poses).cuda()
    outs = [view.render(poses[s], s).cpu().numpy() for s in range(4)]
    again = view.render(poses[3], 3).cpu().numpy()
    view.sync()
    return w, scene, view, outs, again


def _sample(w, img, n_uniform, n_edge, rng):
    E, C, H, Wd = w.n_envs, len(w.cameras), w.cameras[0].height, w.cameras[0].width
    u = np.stack([rng.integers(0, E, n_uniform), rng.integers(0, C, n_uniform), rng.integers(0, Wd, n_uniform),
                  rng.integers(0, H, n_uniform)], 1)
    im = img.reshape(E, C, H, Wd)
    jump = np.zeros_like(im, bool)
    jump[..., :, 1:] |= np.abs(np.diff(im, axis=-1)) > 0.05
    jump[..., 1:, :] |= np.abs(np.diff(im, axis=-2)) > 0.05
    jump &= im > 0.0                                                   # not a dropped pixel
    idx = np.flatnonzero(jump)
    pick = rng.choice(idx, size=min(n_edge, idx.size), replace=False)
    e, c, y, x = np.unravel_index(pick, im.shape)
    return np.concatenate([u, np.stack([e, c, x, y], 1)]).astype(np.int64)


def test_scale_sampled_rays_match_oracle(scale):
    w, scene, view, outs, again = scale
    rng = np.random.default_rng(2602)
    osc = oracle.OracleScene.from_workload(w)
    rays = _sample(w, outs[3], 360, 120, rng)
    ref = osc.render(w.cameras, w.poses, 3, rays, w.sensor, s_first=np.zeros(w.n_envs, np.int64))
    P = w.pixels_per_env
    cam_w = w.cameras[0].width
    got = outs[3][rays[:, 0], rays[:, 1] * (P // len(w.cameras)) + rays[:, 3] * cam_w + rays[:, 2]]
    dropped = (ref["flags"] & oracle.FLAG_DROPPED) != 0
    assert np.array_equal(got == np.float32(w.sensor.fill), dropped)
    compare_depth(got, ref["depth"], ref["flags"], "scale step 3")
    assert np.mean(ref["raw"] < 3.0) > 0.5                               # the sample sees geometry


def test_scale_properties_every_pixel(scale):
    w, scene, view, outs, again = scale
    info = scene.info()
    assert info["terrain_tris"] == 20_480_000 and info["n_links"] == 30
    assert np.array_equal(outs[3], again)                                # re-rendering a step is deterministic
    sen = w.sensor
    cam = w.cameras[0]
    for s in range(4):
        z = outs[s].reshape(-1)
        dropped = z == np.float32(sen.fill)
        assert np.all((z[~dropped] >= np.float32(cam.d_min)) & (z[~dropped] <= np.float32(cam.d_max)))
        n = z.size
        assert abs(dropped.mean() - sen.p_drop) < 5 * math.sqrt(sen.p_drop * (1 - sen.p_drop) / n)
        assert 0.3 < np.mean(z[~dropped] < cam.d_max) < 0.999            # hits and misses both occur


@pytest.mark.slow
def test_many_envs_index_arithmetic(cuda, rpl_lib):
    """65,536 envs (100,663,296 rays, 786,432 blocks) on the small scene: the 64-bit tile, ring and
    output indexing stays right across the whole range -- sampled rays from the first and last envs
    and the middle match the oracle, and the frame matches re-rendering the last envs alone with
    their env_offset."""
    torch = cuda
    E = 65536
    w = W.config_small(n_steps=1, n_envs=E)
    sen = W.Sensor(sigma_abs=0.01, p_drop=0.02, max_latency=1, seed=(0x61, 0x62))
    scene = rpl_lib.Scene.from_workload(w)
    view = rpl_lib.View(scene, E, w.n_links)
    view.set_cameras(w.cameras)
    view.set_sensor(sen)
    poses = torch.from_numpy(w.poses[0]).cuda()
    out = view.render(poses, 0).cpu().numpy()
    view.sync()
    tail = 1000
    part = rpl_lib.View(scene, tail, w.n_links)
    part.set_cameras(w.cameras)
    part.set_sensor(sen)
    got_tail = part.render(poses[E - tail:].contiguous(), 0, E - tail).cpu().numpy()
    part.sync()
    assert np.array_equal(out[E - tail:], got_tail)
    rng = np.random.default_rng(65)
    envs = np.concatenate([np.arange(4), np.arange(E - 4, E), rng.integers(0, E, 8)])
    rays = []
    for e in envs:
        for c, cam in enumerate(w.cameras):
            for _ in range(8):
                rays.append([e, c, rng.integers(0, cam.width), rng.integers(0, cam.height)])
    rays = np.asarray(rays, np.int64)
    osc = oracle.OracleScene.from_workload(w)
    ref = osc.render(w.cameras, w.poses, 0, rays, sen, s_first=np.zeros(E, np.int64))
    offs = w.cam_offsets()
    cw = np.array([c.width for c in w.cameras])
    got = out[rays[:, 0], offs[rays[:, 1]] + rays[:, 3] * cw[rays[:, 1]] + rays[:, 2]]
    dropped = (ref["flags"] & oracle.FLAG_DROPPED) != 0
    assert np.array_equal(got == np.float32(sen.fill), dropped)
    compare_depth(got, ref["depth"], ref["flags"], "65536 envs")
