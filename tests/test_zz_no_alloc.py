"""rpl_render_static_scratch: rendering without allocating.

This entry point is for callers that cannot allocate device memory where they render (a framework
whose caching allocator owns the device memory, a real-time loop where a cudaMalloc is not
acceptable).  Its scratch lives in the library's fixed device array, which keeps the previous call's
contents, so call after call it must give the oracle's depth and the same depth as rpl_render; a
smaller call after a larger one must not pick up the larger call's leftovers.  Faults its kernels
detect are read back by rpl_static_scratch_status.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest

import oracle
from conftest import DEPTH_TOL, compare_depth
from paper_2602_03002_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _side_camera(w):
    torso = w.cameras[0].mount_link
    return W.pinhole(21, 13, 80.0, 50.0, torso, (0.0, 0.12, 0.30), 90.0, 45.0, 0.1, 3.0)


def test_static_scratch_matches_oracle_and_rpl_render_large_then_small(cuda, rpl_lib):
    torch = cuda
    w = W.config_small(n_steps=6, n_envs=12)
    sen = W.Sensor(sigma_abs=0.01, p_drop=0.05, fill=0.0, max_latency=0, seed=(0x52504C31, 7))
    scene = rpl_lib.Scene.from_workload(w)
    poses = torch.from_numpy(w.poses).cuda()
    osc = oracle.OracleScene.from_workload(w)
    # (envs, cameras, env_offset, step): a large call, then a smaller one with fewer envs and cameras
    calls = [(12, w.cameras + [_side_camera(w)], 40, 4), (5, w.cameras, 3, 5)]
    for E, cams, off, s in calls:
        view = rpl_lib.View(scene, E, w.n_links)       # setup may allocate; the call below does not
        view.set_cameras(cams)
        view.set_sensor(sen)
        ref = view.render(poses[s, :E].contiguous(), s, off)
        out = torch.full_like(ref, -7.0)
        rpl_lib.rpl_render_static_scratch(scene.h, cams, E, w.n_links, poses[s, :E].contiguous(), out, sen, s, off)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(-1)
        assert bool((out >= 0).all())                   # every pixel was written
        # against rpl_render: same depth within the tolerance, same dropout decisions
        assert float((out - ref).abs().max()) <= DEPTH_TOL, (E, s)
        assert torch.equal(out == 0.0, ref == 0.0)
        # against the FP64 oracle
        o = osc.render(cams, w.poses[:, :E], s, oracle.all_rays(cams, E), sen, env_offset=off)
        dropped = (o["flags"] & oracle.FLAG_DROPPED) != 0
        assert np.array_equal(got == np.float32(sen.fill), dropped), (E, s)
        compare_depth(got, o["depth"], o["flags"], "no-allocation render, %d envs x %d cams" % (E, len(cams)))
        view.close()
    rpl_lib.rpl_static_scratch_status(scene.h)           # no kernel fault was recorded
    osc.close()


def test_static_scratch_rejects_oversize_latency_and_bad_arguments(cuda, rpl_lib):
    torch = cuda
    w = W.config_small(n_steps=1)
    scene = rpl_lib.Scene.from_workload(w)
    view = rpl_lib.View(scene, 1, w.n_links)
    view.set_cameras(w.cameras)
    big = (8 << 20) // (80 * (w.n_links + 2)) + 16          # just over the fixed array
    # full-size buffers, so the call would stay in bounds even if it did not refuse
    poses = torch.zeros((big, w.n_links, 7), device="cuda")
    poses[..., 6] = 1.0
    out = torch.zeros((big, w.pixels_per_env), device="cuda")
    with pytest.raises(rpl_lib.RplError) as ei:
        rpl_lib.rpl_render_static_scratch(scene.h, w.cameras, big, w.n_links, poses, out)
    assert ei.value.status == 5 and "scratch" in str(ei.value)
    with pytest.raises(rpl_lib.RplError) as ei:
        rpl_lib.rpl_render_static_scratch(scene.h, w.cameras, 1, w.n_links, poses, out, W.Sensor(max_latency=2))
    assert ei.value.status == 1
    # The checks below run with zero envs, where the call launches nothing even when it accepts.
    # 2^31 pixels per env (8 cameras of 16384 x 16384) would overflow the 32-bit pixel offsets
    huge = [W.pinhole(16384, 16384, 60.0, 60.0, 0, (0, 0, 0), 0.0, 30.0, 0.1, 3.0)] * 8
    with pytest.raises(rpl_lib.RplError) as ei:
        rpl_lib.rpl_render_static_scratch(scene.h, huge, 0, w.n_links, None, None)
    assert ei.value.status == 5 and "2^31" in str(ei.value)
    # non-finite intrinsics or range, as rpl_cameras_set refuses them
    for field, value in (("fx", float("inf")), ("cy", float("nan")), ("d_max", float("inf"))):
        cam = W.pinhole(32, 24, 87.0, 58.0, 0, (0, 0, 0), 0.0, 30.0, 0.1, 3.0)
        setattr(cam, field, value)
        with pytest.raises(rpl_lib.RplError) as ei:
            rpl_lib.rpl_render_static_scratch(scene.h, [cam], 0, w.n_links, None, None)
        assert ei.value.status == 1, field
    # misaligned poses or output
    raw = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(rpl_lib.RplError) as ei:
        rpl_lib.rpl_render_static_scratch(scene.h, w.cameras, 0, w.n_links, raw[1:], raw[4:])
    assert ei.value.status == 1 and "aligned" in str(ei.value)
    rpl_lib.rpl_static_scratch_status(scene.h)
