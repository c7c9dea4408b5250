"""Precision variant: the eight-wide BVH with 8-bit quantised child boxes, and FP16 / unorm16 depth.

Quantised boxes only make culling coarser (they are rounded outward), and the triangle tests are
the same FP32 code, so with FP32 output the wide BVH must give bit-identical depth to the binary
BVH.  FP16 output adds at most half an FP16 ulp of the depth, unorm16 at most half a step of
d_max / 65535; both are checked against the FP64 oracle with that allowance on top of 1e-4 m.
"""
import numpy as np
import pytest

import oracle
from conftest import DEPTH_TOL, compare_depth
from paper_2602_03002_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _render(torch, rpl, w, scene, sensor, steps):
    view = rpl.View(scene, w.n_envs, w.n_links)
    view.set_cameras(w.cameras, w.per_env_intrinsics)
    view.set_sensor(sensor)
    poses = torch.from_numpy(w.poses).cuda()
    outs = [view.render(poses[s], s).cpu() for s in steps]
    view.sync()
    return outs


def _scene(rpl, w, kind):
    s = rpl.Scene(w.terrain_verts, w.terrain_tris, bvh_kind=kind)
    for l, (v, t) in enumerate(zip(w.link_verts, w.link_tris)):
        s.add_link(l, v, t)
    return s


def test_wide_bvh_matches_binary_bitexact(cuda, rpl_lib):
    w = W.config_small(n_steps=3)
    sen = W.Sensor(sigma_abs=0.01, p_drop=0.05, max_latency=2, seed=(3, 4))
    a = _render(cuda, rpl_lib, w, _scene(rpl_lib, w, rpl_lib.RPL_BVH2), sen, range(3))
    b = _render(cuda, rpl_lib, w, _scene(rpl_lib, w, rpl_lib.RPL_BVH8Q8), sen, range(3))
    for s in range(3):
        assert cuda.equal(a[s], b[s]), s
    info = _scene(rpl_lib, w, rpl_lib.RPL_BVH8Q8).info()
    assert info["terrain_tris"] == 3200 and info["terrain_bytes"] == info["terrain_nodes"] * 80 + 3200 * 48


@pytest.mark.parametrize("out_dtype", [1, 2])
def test_half_and_unorm16_output_vs_oracle(cuda, rpl_lib, out_dtype):
    w = W.config_small(n_steps=2)
    sen = W.Sensor(sigma_abs=0.01, p_drop=0.05, fill=0.0, max_latency=1, seed=(8, 9), out_dtype=out_dtype)
    outs = _render(cuda, rpl_lib, w, _scene(rpl_lib, w, rpl_lib.RPL_BVH8Q8), sen, range(2))
    osc = oracle.OracleScene.from_workload(w)
    rays = oracle.all_rays(w.cameras, w.n_envs)
    d_max = np.float32(w.cameras[0].d_max)
    for s in range(2):
        ref = osc.render(w.cameras, w.poses, s, rays, sen, s_first=np.zeros(w.n_envs, np.int64))
        if out_dtype == 1:
            got = outs[s].float().numpy().reshape(-1).astype(np.float64)
            tol = DEPTH_TOL + np.spacing(np.abs(ref["depth"]).astype(np.float16)).astype(np.float64) / 2
        else:
            got = outs[s].numpy().astype(np.float64).reshape(-1) * (float(d_max) / 65535.0)
            tol = DEPTH_TOL + float(d_max) / 65535.0 / 2
        dropped = (ref["flags"] & oracle.FLAG_DROPPED) != 0
        assert np.array_equal(got == 0.0, dropped)
        diff = np.abs(got - ref["depth"])
        bad = (diff > tol) & ((ref["flags"] & oracle.FLAG_FP32_SENSITIVE) == 0)
        assert not bad.any(), (s, diff[bad].max())
        assert (diff > tol).sum() <= max(1, int(1e-4 * diff.size))


@pytest.mark.slow
def test_scale_wide_half_sampled(cuda, rpl_lib):
    """The precision configuration at full size: 4096 envs x 2 cams, 20.48M triangles, wide BVH, FP16."""
    torch = cuda
    w = W.config_scale(n_steps=2)
    sen = W.scale_sensor()
    sen.out_dtype = 1
    scene = _scene(rpl_lib, w, rpl_lib.RPL_BVH8Q8)
    outs = _render(torch, rpl_lib, w, scene, sen, range(2))
    rng = np.random.default_rng(44)
    n = 300
    rays = np.stack([rng.integers(0, w.n_envs, n), rng.integers(0, 2, n), rng.integers(0, 64, n),
                     rng.integers(0, 48, n)], 1).astype(np.int64)
    osc = oracle.OracleScene.from_workload(w)
    ref = osc.render(w.cameras, w.poses, 1, rays, sen, s_first=np.zeros(w.n_envs, np.int64))
    img = outs[1].float().numpy()
    got = img[rays[:, 0], rays[:, 1] * 3072 + rays[:, 3] * 64 + rays[:, 2]].astype(np.float64)
    tol = DEPTH_TOL + np.spacing(np.abs(ref["depth"]).astype(np.float16)).astype(np.float64) / 2
    diff = np.abs(got - ref["depth"])
    bad = (diff > tol) & ((ref["flags"] & oracle.FLAG_FP32_SENSITIVE) == 0)
    assert not bad.any(), diff[bad].max()
