"""The sensor model alone (rpl_sensor_apply) on given pre-sensor depth.

It must reproduce the sensor stage of the fused render bit-exactly: the raw frames of a view with
the sensor off, fed through rpl_sensor_apply of a view with the sensor on, equal that view's own
renders step by step (latency ring, noise, clip, dropout and side masks included).  On a constant
input its statistics are those of the model: dropout at rate p, noise N(0, sigma^2) on hits,
misses (d_max) untouched, latency delays uniform over 0..Lmax."""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2602_03002_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SENSOR = W.Sensor(sigma_abs=0.01, sigma_rel=0.02, p_drop=0.05, max_latency=3, seed=(0xC0, 0xDE))


def test_sensor_stage_alone_equals_the_fused_render(cuda, rpl_lib):
    torch = cuda
    w = W.config_small(n_steps=6, n_envs=6)
    w.rsm_modes, w.rsm_cols = np.array([0, 1, 2, 0, 2, 1], np.uint8), (0, 3, 6)
    scene = rpl_lib.Scene.from_workload(w)
    poses = torch.from_numpy(w.poses).cuda()
    fused = rpl_lib.View.from_workload(scene, w)
    fused.set_sensor(SENSOR)
    raw_view = rpl_lib.View.from_workload(scene, w)
    raw_view.set_sensor(W.Sensor())
    raw_view.set_side_mask(env_mode=None)
    alone = rpl_lib.View.from_workload(scene, w)
    alone.set_sensor(SENSOR)
    for s in range(6):
        want = fused.render(poses[s], s, 11)
        raw = raw_view.render(poses[s], s, 11)
        assert bool((raw > np.float32(0.1)).all())     # no hit nearer than d_min: clamping kept raw depth
        got = alone.out_tensor()
        rpl_lib.rpl_sensor_apply(alone.h, raw, s, 11, got)
        torch.cuda.synchronize()
        assert torch.equal(got, want), s
    for v in (fused, raw_view, alone):
        v.sync()


def test_sensor_statistics_on_constant_depth(cuda, rpl_lib):
    torch = cuda
    w = W.config_small(n_steps=1, n_envs=64)
    cam = W.pinhole(64, 48, 80.0, 60.0, w.cameras[0].mount_link, (0.1, 0.0, 0.3), 0.0, 50.0, 0.1, 3.0)
    w.cameras = [cam]
    scene = rpl_lib.Scene.from_workload(w)
    view = rpl_lib.View(scene, w.n_envs, w.n_links)
    view.set_cameras([cam])
    sen = W.Sensor(sigma_abs=0.01, p_drop=0.05, max_latency=3, seed=(7, 8))
    view.set_sensor(sen)
    P = cam.width * cam.height
    raw = torch.full((w.n_envs, P), 2.0, device="cuda")
    raw[:, ::7] = cam.d_max                              # every seventh pixel is a miss
    miss = torch.zeros(P, dtype=torch.bool, device="cuda")
    miss[::7] = True
    outs = []
    for s in range(8):
        out = view.out_tensor()
        rpl_lib.rpl_sensor_apply(view.h, raw, s, 0, out)
        outs.append(out.cpu().numpy())
    view.sync()
    z = np.stack(outs)                                   # [S, E, P]
    m = miss.cpu().numpy()
    dropped = z == np.float32(sen.fill)
    n = dropped.size
    assert abs(dropped.mean() - sen.p_drop) < 5 * math.sqrt(sen.p_drop * (1 - sen.p_drop) / n)
    hits = z[:, :, ~m][~dropped[:, :, ~m]]
    noise = (hits.astype(np.float64) - 2.0) / sen.sigma_abs
    assert abs(noise.mean()) < 5 / math.sqrt(noise.size)
    assert abs(noise.var() - 1.0) < 5 * math.sqrt(2.0 / noise.size)
    assert stats.kstest(noise, "norm").pvalue > 1e-4
    misses = z[:, :, m][~dropped[:, :, m]]
    assert np.all(misses == np.float32(cam.d_max))       # no noise on misses
