"""The steps next to the ray cast, on the GPU against the FP64 oracle: downsampled cameras (raw
image averaged over f x f blocks before the sensor model, Sec. 4.1), per-env camera mount and FOV
randomisation (Appendix A.2), and Random Side Masking (Sec. 3.2.4); then the paper's perception
configuration at full size (4096 envs x 2 cameras, 240x135 raw -> 48x27, 20.48M-triangle terrain)
on sampled output pixels and on properties of every pixel."""
import math

import numpy as np
import pytest

import oracle
from conftest import compare_depth
from paper_2602_03002_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _small_with(cams, n_steps=4, n_envs=6):
    w = W.config_small(n_steps=n_steps, n_envs=n_envs)
    torso = w.cameras[0].mount_link
    out = []
    for (wd, ht, f, yaw) in cams:
        c = W.pinhole(wd, ht, 101.0, 69.0, torso, (0.10 * math.cos(math.radians(yaw)), 0.10 * math.sin(math.radians(yaw)), 0.30),
                      yaw, 50.0, 0.1, 3.0)
        c.downsample = f
        out.append(c)
    w.cameras = out
    return w


def _gpu_frames(torch, rpl, w, sensor, steps, env_offset=0):
    scene = rpl.Scene.from_workload(w)
    view = rpl.View.from_workload(scene, w)
    view.set_sensor(sensor)
    poses = torch.from_numpy(w.poses).cuda()
    outs = [view.render(poses[s], s, env_offset).cpu().numpy().copy() for s in steps]
    view.sync()
    return outs, view


def _oracle_frames(w, sensor, steps, env_offset=0):
    osc = oracle.OracleScene.from_workload(w)
    rays = oracle.all_rays(w.cameras, w.n_envs)
    return [osc.render(w.cameras, w.poses, s, rays, sensor, s_first=np.zeros(w.n_envs, np.int64),
                       env_offset=env_offset, per_env_intrinsics=w.per_env_intrinsics, mount_dr=w.mount_delta,
                       rsm_mode=w.rsm_modes, rsm_cols=w.rsm_cols) for s in steps]


def test_downsampled_cameras_mixed_with_plain_ones(cuda, rpl_lib):
    """A 5x and a 2x downsampled camera beside a plain one with ragged tiles; latency, noise and
    dropout act on the downsampled image."""
    w = _small_with([(40, 30, 5, 0.0), (26, 18, 2, 180.0), (13, 9, 1, 90.0)])
    sen = W.Sensor(sigma_abs=0.01, sigma_rel=0.05, p_drop=0.05, max_latency=2, seed=(0xD0, 0x5A))
    outs, view = _gpu_frames(cuda, rpl_lib, w, sen, range(4), env_offset=11)
    offs, total = view.layout()
    assert list(offs) == [0, 48, 48 + 117, 48 + 117 + 117] and total == 282
    refs = _oracle_frames(w, sen, range(4), env_offset=11)
    for s in range(4):
        dropped = (refs[s]["flags"] & oracle.FLAG_DROPPED) != 0
        got = outs[s].reshape(-1)
        assert np.array_equal(got == np.float32(sen.fill), dropped)
        compare_depth(got, refs[s]["depth"], refs[s]["flags"], "downsample step %d" % s)
    assert np.mean(refs[3]["raw"] < 3.0) > 0.3


def test_randomised_mounts_and_fov(cuda, rpl_lib):
    w = _small_with([(32, 24, 1, 0.0), (40, 30, 5, 180.0)], n_envs=8)
    w.mount_delta, w.per_env_intrinsics = W.camera_randomization(w.n_envs, w.cameras, seed=4)
    outs, view = _gpu_frames(cuda, rpl_lib, w, W.Sensor(), range(2))
    refs = _oracle_frames(w, W.Sensor(), range(2))
    for s in range(2):
        compare_depth(outs[s], refs[s]["depth"], refs[s]["flags"], "camera DR step %d" % s)
    # clearing the randomisation restores the plain mounts
    view.randomize_cameras(None)
    import torch
    plain = view.render(torch.from_numpy(w.poses[1]).cuda(), 1).cpu().numpy()
    w2 = _small_with([(32, 24, 1, 0.0), (40, 30, 5, 180.0)], n_envs=8)
    w2.per_env_intrinsics = w.per_env_intrinsics
    ref2 = _oracle_frames(w2, W.Sensor(), [1])[0]
    compare_depth(plain, ref2["depth"], ref2["flags"], "camera DR cleared")
    assert np.abs(plain.reshape(-1) - outs[1].reshape(-1)).max() > 1e-3


def test_side_masking(cuda, rpl_lib):
    w = _small_with([(40, 30, 5, 0.0), (24, 16, 1, 180.0)], n_steps=5, n_envs=6)
    w.rsm_modes = np.array([0, 1, 2, 2, 1, 7], np.uint8)       # 7 counts as large
    w.rsm_cols = (0, 2, 3)
    sen = W.Sensor(sigma_rel=0.1, p_drop=0.05, max_latency=3, seed=(1, 2))
    outs, view = _gpu_frames(cuda, rpl_lib, w, sen, range(5), env_offset=3)
    refs = _oracle_frames(w, sen, range(5), env_offset=3)
    for s in range(5):
        masked = (refs[s]["flags"] & oracle.FLAG_MASKED) != 0
        got = outs[s].reshape(-1)
        assert masked.any()
        np.testing.assert_allclose(got[masked], refs[s]["depth"][masked], rtol=0, atol=1e-6)
        compare_depth(got, refs[s]["depth"], refs[s]["flags"], "side mask step %d" % s)
    # masking off again: identical to the unmasked oracle
    view.set_side_mask(env_mode=None)
    import torch
    got = view.render(torch.from_numpy(w.poses[4]).cuda(), 4, 3).cpu().numpy()   # a re-render of step 4
    w.rsm_modes = None
    ref = _oracle_frames(w, sen, [4], env_offset=3)[0]
    compare_depth(got, ref["depth"], ref["flags"], "side mask off")


def test_graph_replay_of_a_downsampled_view(cuda, rpl_lib):
    """The downsample launch is captured with the render: replays equal direct renders."""
    torch = cuda
    w = _small_with([(40, 30, 5, 0.0), (20, 10, 5, 180.0)], n_steps=4)
    w.rsm_modes, w.rsm_cols = np.array([0, 1, 2, 1, 0, 2], np.uint8), (0, 1, 2)
    sen = W.Sensor(sigma_abs=0.01, p_drop=0.05, max_latency=2, seed=(8, 9))
    scene = rpl_lib.Scene.from_workload(w)
    poses = torch.from_numpy(w.poses).cuda()
    a = rpl_lib.View.from_workload(scene, w)
    a.set_sensor(sen)
    ref = [a.render(poses[s], s).clone() for s in range(4)]
    b = rpl_lib.View.from_workload(scene, w)
    b.set_sensor(sen)
    stream = torch.cuda.Stream()
    pose_buf = torch.empty_like(poses[0])
    out = b.out_tensor()
    # the side stream waits for the default stream's pending work on memory the allocator may reuse
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        for s in range(4):
            pose_buf.copy_(poses[s])
            assert rpl_lib.rpl_render_graph(b.h, pose_buf, 0, out, stream) == s
            stream.synchronize()
            assert torch.equal(out, ref[s]), s
    b.sync()


def test_static_scratch_refuses_downsampled_cameras(cuda, rpl_lib):
    w = _small_with([(40, 30, 5, 0.0)])
    scene = rpl_lib.Scene.from_workload(w)
    rpl_lib.View.from_workload(scene, w)      # freezes the scene
    torch = cuda
    poses = torch.from_numpy(w.poses[0]).cuda()
    out = torch.empty(w.n_envs * 48, device="cuda")
    with pytest.raises(rpl_lib.RplError) as ei:
        rpl_lib.rpl_render_static_scratch(scene.h, w.cameras, w.n_envs, w.n_links, poses, out)
    assert ei.value.status == 1


# --------------------------------------------------------------------------------------------------
# the paper's perception configuration at full size
# --------------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def perception(cuda, rpl_lib):
    torch = cuda
    w = W.config_perception(n_steps=4)
    scene = rpl_lib.Scene.from_workload(w)
    view = rpl_lib.View.from_workload(scene, w)
    poses = torch.from_numpy(w.poses).cuda()
    outs = [view.render(poses[s], s).cpu().numpy() for s in range(4)]
    view.sync()
    return w, scene, view, outs


@pytest.mark.slow
def test_perception_scale_sampled_pixels(perception):
    w, scene, view, outs = perception
    rng = np.random.default_rng(7)
    E, C = w.n_envs, len(w.cameras)
    ow, oh = w.cameras[0].out_width, w.cameras[0].out_height
    n = 48
    rays = np.stack([rng.integers(0, E, n), rng.integers(0, C, n), rng.integers(0, ow, n), rng.integers(0, oh, n)], 1)
    # include masked columns of envs in the large mode
    large = np.flatnonzero(w.rsm_modes == 2)[:8]
    rays = np.concatenate([rays, np.stack([large, np.zeros_like(large), np.ones_like(large), np.full_like(large, 13)], 1)])
    rays = rays.astype(np.int64)
    osc = oracle.OracleScene.from_workload(w)
    ref = osc.render(w.cameras, w.poses, 3, rays, w.sensor, s_first=np.zeros(E, np.int64),
                     per_env_intrinsics=w.per_env_intrinsics, mount_dr=w.mount_delta, rsm_mode=w.rsm_modes,
                     rsm_cols=w.rsm_cols)
    got = outs[3][rays[:, 0], rays[:, 1] * (ow * oh) + rays[:, 3] * ow + rays[:, 2]]
    dropped = (ref["flags"] & oracle.FLAG_DROPPED) != 0
    masked = (ref["flags"] & oracle.FLAG_MASKED) != 0
    assert masked[-len(large):].all()
    assert np.array_equal((got == np.float32(w.sensor.fill)) & ~masked, dropped & ~masked)
    compare_depth(got, ref["depth"], ref["flags"], "perception step 3")
    assert np.mean(ref["raw"] < 3.0) > 0.5


@pytest.mark.slow
def test_perception_scale_every_pixel(perception):
    w, scene, view, outs = perception
    cam = w.cameras[0]
    assert view.layout()[1] == 2 * 48 * 27
    E, ow, oh = w.n_envs, cam.out_width, cam.out_height
    for s in range(4):
        img = outs[s].reshape(E, 2, oh, ow)
        z = img.reshape(-1)
        assert np.all((z == np.float32(w.sensor.fill)) | ((z >= np.float32(cam.d_min)) & (z <= np.float32(cam.d_max))))
        # envs without a mask have dropout at rate p in every column
        none = w.rsm_modes == 0
        d = img[none] == np.float32(w.sensor.fill)
        p = w.sensor.p_drop
        assert abs(d.mean() - p) < 5 * math.sqrt(p * (1 - p) / d.size)
        # large-mask envs: the outer 12 columns hold no dropout fill (they are masked after the sensor)
        large = img[w.rsm_modes == 2]
        assert not (large[..., :12] == np.float32(w.sensor.fill)).any()
        assert not (large[..., -12:] == np.float32(w.sensor.fill)).any()
