"""Watertightness of the GPU ray/triangle test (Woop, Benthin, Wald 2013) on closed meshes.

A camera inside a closed surface must see the surface through every pixel: a ray that slipped
between two triangles sharing an edge, or through a vertex shared by a fan, would report the far
plane.  The meshes are a UV ellipsoid (pole fans of 32 triangles, shared edges everywhere) and a
closed box subdivided into a grid (edges and vertices hit exactly by the axis-aligned rays of the
centre pixels); depths are checked against the FP64 oracle as well."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from conftest import compare_depth
from paper_2602_03002_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _camera_inside(rpl, torch, verts, tris, quats, centre, width=64, height=48):
    """Renders one env per camera orientation from `centre` (no links hit: a tiny link far away)."""
    link_v, link_t = W.box_mesh((0.01, 0.01, 0.01), (500.0, 500.0, 500.0), subdiv=1)
    scene = rpl.Scene(verts, tris)
    scene.add_link(0, link_v, link_t)
    cam = W.pinhole(width, height, 100.0, 80.0, 0, (0.0, 0.0, 0.0), 0.0, 0.0, 0.01, 50.0)
    E = len(quats)
    poses = np.zeros((E, 1, 7), np.float32)
    poses[:, 0, :3] = centre
    poses[:, 0, 3:] = quats
    view = rpl.View(scene, E, 1)
    view.set_cameras([cam])
    view.set_sensor(W.Sensor())
    out = view.render(torch.from_numpy(poses).cuda(), 0).cpu().numpy()
    view.sync()
    return out, cam, poses, (link_v, link_t)


def _quats(n, seed):
    q = Rotation.random(n, random_state=seed).as_quat()
    axis = Rotation.from_euler("xyz", [[0, 0, 0], [90, 0, 0], [-90, 0, 0], [0, 90, 0], [0, -90, 0], [180, 0, 0]],
                               degrees=True).as_quat()
    return np.concatenate([axis, q]).astype(np.float32)


@pytest.mark.parametrize("slices,bands", [(32, 33), (7, 5)])
def test_no_ray_escapes_a_closed_ellipsoid(cuda, rpl_lib, slices, bands):
    v, t = W.ellipsoid_mesh((2.0, 1.5, 1.0), (0.3, -0.2, 0.1), slices=slices, bands=bands)
    quats = _quats(26, 5)
    out, cam, poses, link = _camera_inside(rpl_lib, cuda, v, t, quats, (0.3, -0.2, 0.1))
    assert out.size == len(quats) * cam.width * cam.height
    assert np.all(out < np.float32(cam.d_max)), "%d rays escaped" % int((out >= cam.d_max).sum())
    osc = oracle.OracleScene(v, t, [link[0]], [link[1]])
    ref = osc.render([cam], poses[None], 0, oracle.all_rays([cam], len(quats)), W.Sensor())
    compare_depth(out, ref["depth"], ref["flags"], "ellipsoid interior")


def test_no_ray_escapes_a_closed_gridded_box(cuda, rpl_lib):
    """Box faces split into 8x8 quads of 0.25 m: the axis-aligned views put the centre pixels' rays
    exactly on grid vertices and edges (the camera sits at the centre, integer-aligned)."""
    v, t = W.box_mesh((1.0, 1.0, 1.0), (0.0, 0.0, 0.0), subdiv=8)
    quats = _quats(40, 9)
    out, cam, poses, link = _camera_inside(rpl_lib, cuda, v, t, quats, (0.0, 0.0, 0.0), width=65, height=49)
    assert np.all(out < np.float32(cam.d_max)), "%d rays escaped" % int((out >= cam.d_max).sum())
    # the centre pixel of an axis-aligned view hits a face centre, a shared grid vertex, at depth 1
    c = (cam.height // 2) * cam.width + cam.width // 2
    for e in range(6):
        assert abs(out[e, c] - 1.0) < 1e-6
    osc = oracle.OracleScene(v, t, [link[0]], [link[1]])
    ref = osc.render([cam], poses[None], 0, oracle.all_rays([cam], len(quats)), W.Sensor())
    compare_depth(out, ref["depth"], ref["flags"], "box interior")
