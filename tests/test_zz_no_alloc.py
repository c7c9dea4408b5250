"""rpl_render_static_scratch: rendering without allocating.

This entry point is for callers that cannot allocate device memory where they render (a framework
whose caching allocator owns the device memory, a real-time loop where a cudaMalloc is not
acceptable).  Its scratch lives in the library's fixed device array, so it must give the same
depth as rpl_render, call after call, while the array keeps the previous call's contents.
The file name makes pytest collect it last.
"""
import numpy as np
import pytest

from conftest import DEPTH_TOL
from paper_2602_03002_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_static_scratch_matches_rpl_render_on_consecutive_calls(cuda, rpl_lib):
    torch = cuda
    w = W.config_small(n_steps=2)
    sen = W.Sensor(sigma_abs=0.01, p_drop=0.05, fill=0.0, max_latency=0, seed=(0x52504C31, 0))
    scene = rpl_lib.Scene.from_workload(w)
    view = rpl_lib.View(scene, w.n_envs, w.n_links)        # freezes the scene (setup may allocate)
    view.set_cameras(w.cameras)
    view.set_sensor(sen)
    poses = torch.from_numpy(w.poses).cuda()
    for s in range(2):                                      # two calls in a row, different poses
        ref = view.render(poses[s], s, 5)
        out = torch.full_like(ref, -7.0)
        rpl_lib.rpl_render_static_scratch(scene.h, w.cameras, w.n_envs, w.n_links, poses[s], out, sen, s, 5)
        torch.cuda.synchronize()
        diff = (out - ref).abs().max().item()
        assert diff <= DEPTH_TOL, (s, diff)
        assert torch.equal(out == 0.0, ref == 0.0)          # the same dropout decisions
        assert bool((out >= 0).all())                       # every pixel was written


def test_static_scratch_rejects_oversize_and_latency(cuda, rpl_lib):
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
