"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test derives the expected depth by a different route than the oracle takes (the oracle:
quaternion -> matrix, unit ray direction, plane + inside test per triangle, m * t):
  * plane, slope and range closed forms from scipy rotations and the unnormalised pixel ray;
  * a stairs profile with vertical risers, solved step by step in the vertical plane;
  * a rotated box occluder by Kay-Kajiya slabs in the box frame;
  * random triangle soups by a vectorised Moller-Trumbore brute force;
  * invariance under a rigid motion of the whole scene;
  * Philox4x32-10 against the published known-answer vectors;
  * sensor statistics (dropout rate, noise moments and normality, latency histogram) and the exact
    latency identity out(s) = out_{no delay}(s').
"""
import math
import os

import numpy as np
import pytest
from scipy import stats
from scipy.spatial.transform import Rotation

import oracle
from paper_2602_03002_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------------------------------
# helpers: a camera on link 0, expected depths from the camera axes given by scipy
# --------------------------------------------------------------------------------------------------
def _cam(width, height, hfov, vfov, yaw, pitch, d_min=0.1, d_max=3.0, mount=0, pos=(0.0, 0.0, 0.0)):
    return W.pinhole(width, height, hfov, vfov, mount, pos, yaw, pitch, d_min, d_max)


def _pose(pos, quat=(0.0, 0.0, 0.0, 1.0)):
    return np.array([*pos, *quat], np.float32)


def _f32(v):
    """The inputs the oracle sees are float32: round through float32, then compute in float64."""
    return np.asarray(np.asarray(v, np.float64).astype(np.float32), np.float64)


def _axes_world(cam, link_quat):
    """World right/down/forward axes of the optical frame (scipy, independent of the oracle)."""
    Rl = Rotation.from_quat(_f32(link_quat)).as_matrix()
    Rm = Rotation.from_quat(_f32(cam.offset_quat)).as_matrix()
    R = Rl @ Rm
    return R[:, 0], R[:, 1], R[:, 2]


def _pixel_dirs(cam, right, down, fwd, fx=None, fy=None, cx=None, cy=None):
    """Unnormalised world direction D = r_x right + r_y down + fwd per pixel: depth = parameter along D."""
    fx = np.float64(np.float32(cam.fx if fx is None else fx))
    fy = np.float64(np.float32(cam.fy if fy is None else fy))
    cx = np.float64(np.float32(cam.cx if cx is None else cx))
    cy = np.float64(np.float32(cam.cy if cy is None else cy))
    y, x = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    rx = (x - cx) / fx
    ry = (y - cy) / fy
    D = rx[..., None] * right + ry[..., None] * down + fwd
    return D.reshape(-1, 3), np.sqrt(rx ** 2 + ry ** 2 + 1).reshape(-1)


def _plane_mesh(z=0.0, half=50.0):
    v = np.array([[-half, -half, z], [half, -half, z], [half, half, z], [-half, half, z]], np.float32)
    return v, np.array([[0, 1, 2], [0, 2, 3]], np.int32)


def _render(terrain, links, cams, poses, sensor=None, step=0, rays=None, **kw):
    sc = oracle.OracleScene(terrain[0], terrain[1], [l[0] for l in links], [l[1] for l in links])
    poses = np.asarray(poses, np.float32)
    if poses.ndim == 3:
        poses = poses[None]
    if rays is None:
        rays = oracle.all_rays(cams, poses.shape[1])
    return sc.render(cams, poses, step, rays, sensor if sensor is not None else W.Sensor(), **kw)


EMPTY = (np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32))


def _clipped(lam, cam):
    z = np.where(np.isfinite(lam) & (lam > 0) & (lam < cam.d_max), lam, cam.d_max)
    return np.clip(z, cam.d_min, cam.d_max)


# --------------------------------------------------------------------------------------------------
def test_philox_known_answers():
    n = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(t, 16) for t in line.split()]
            assert list(oracle.philox4x32_10(w[0:4], w[4:6])) == w[6:10]
            n += 1
    assert n == 3


@pytest.mark.parametrize("yaw,pitch,link_yaw", [(0.0, 35.0, 0.0), (20.0, 50.0, 30.0), (-70.0, 15.0, -110.0)])
def test_flat_plane_closed_form(yaw, pitch, link_yaw):
    h, Hc = 0.2, 1.45
    cam = _cam(9, 7, 70.0, 50.0, yaw, pitch)
    q = Rotation.from_euler("z", link_yaw, degrees=True).as_quat()
    pose = _pose((0.3, -0.2, Hc), q)
    out = _render(_plane_mesh(h), [EMPTY], [cam], pose[None, None])
    right, down, fwd = _axes_world(cam, q)
    D, _ = _pixel_dirs(cam, right, down, fwd)
    lam = np.where(D[:, 2] < 0, (_f32(h) - _f32(Hc)) / np.where(D[:, 2] < 0, D[:, 2], -1.0), np.inf)
    np.testing.assert_allclose(out["depth"], _clipped(lam, cam), rtol=0, atol=1e-9)
    # with no link yaw the depth of a flat plane depends on the image row only
    if link_yaw == 0.0 and yaw == 0.0:
        img = out["depth"].reshape(cam.height, cam.width)
        assert np.allclose(img, img[:, :1], atol=1e-12)


def test_slope_closed_form():
    alpha = math.radians(20.0)
    v = np.array([[x, y, x * math.tan(alpha)] for x, y in ((-40, -40), (40, -40), (40, 40), (-40, 40))], np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    cam = _cam(11, 9, 87.0, 58.0, 0.0, 40.0)
    o = np.array([0.4, 0.1, 1.6])
    out = _render((v, t), [EMPTY], [cam], _pose(o)[None, None])
    right, down, fwd = _axes_world(cam, (0, 0, 0, 1))
    D, _ = _pixel_dirs(cam, right, down, fwd)
    o = _f32(o)
    vv = np.asarray(v, np.float64)                       # the float32 plane, exactly as stored
    n = np.cross(vv[1] - vv[0], vv[2] - vv[0])
    n /= np.linalg.norm(n)
    p0 = vv[0]
    denom = D @ n
    lam = np.where(denom != 0, ((p0 - o) @ n) / np.where(denom != 0, denom, 1.0), np.inf)
    np.testing.assert_allclose(out["depth"], _clipped(lam, cam), rtol=0, atol=1e-7)
    assert np.mean(out["depth"] < 3.0) > 0.5


def _stairs_mesh(rise, run, n_steps, y_half=20.0, x0=-10.0, x_end=40.0):
    """Ascending stairs along +x with exact vertical risers; tread k at z = k*rise over [k*run, (k+1)*run]."""
    verts, tris = [], []

    def quad(a, b, c, d):
        i = len(verts)
        verts.extend([a, b, c, d])
        tris.extend([[i, i + 1, i + 2], [i, i + 2, i + 3]])

    quad((x0, -y_half, 0.0), (0.0, -y_half, 0.0), (0.0, y_half, 0.0), (x0, y_half, 0.0))
    for k in range(n_steps + 1):
        z = k * rise
        xa = k * run
        xb = (k + 1) * run if k < n_steps else x_end
        quad((xa, -y_half, z), (xb, -y_half, z), (xb, y_half, z), (xa, y_half, z))
        if k >= 1:
            quad((xa, -y_half, z - rise), (xa, y_half, z - rise), (xa, y_half, z), (xa, -y_half, z))
    return np.asarray(verts, np.float32), np.asarray(tris, np.int32)


def _stairs_depth(o, D, rise, run, n_steps, x0=-10.0, x_end=40.0):
    """First intersection with the stairs profile, step by step in the x-z plane.  Tread heights and
    riser positions are the float32 values the mesh stores."""
    f = lambda v: float(np.float32(v))
    best = np.inf
    cands = [(0.0, f(x0), 0.0)]                      # ground in front of the stairs
    for k in range(n_steps + 1):
        cands.append((f(k * rise), f(k * run), f((k + 1) * run) if k < n_steps else f(x_end)))
    for z, xa, xb in cands:
        if D[2] != 0:
            lam = (z - o[2]) / D[2]
            x = o[0] + lam * D[0]
            if lam > 0 and xa <= x <= xb:
                best = min(best, lam)
    for k in range(1, n_steps + 1):
        if D[0] != 0:
            lam = (f(k * run) - o[0]) / D[0]
            z = o[2] + lam * D[2]
            if lam > 0 and f((k - 1) * rise) <= z <= f(k * rise):
                best = min(best, lam)
    return best


@pytest.mark.parametrize("rise,run", [(0.15, 0.25), (0.20, 0.30)])
def test_stairs_riser_and_tread(rise, run):
    n_steps = 10
    mesh = _stairs_mesh(rise, run, n_steps)
    cam = _cam(15, 11, 80.0, 60.0, 0.0, 30.0, d_max=4.0)
    o = np.array([-0.6, 0.0, 1.1])
    out = _render(mesh, [EMPTY], [cam], _pose(o)[None, None], flags=True)
    right, down, fwd = _axes_world(cam, (0, 0, 0, 1))
    D, _ = _pixel_dirs(cam, right, down, fwd)
    o = _f32(o)
    exp = _clipped(np.array([_stairs_depth(o, d, rise, run, n_steps) for d in D]), cam)
    edge = (out["flags"] & oracle.FLAG_EDGE) != 0
    np.testing.assert_allclose(out["depth"][~edge], exp[~edge], rtol=0, atol=1e-7)
    assert len(np.unique(np.round(exp, 3))) > 10   # several treads and risers are seen


def test_rotated_box_occludes_plane():
    half = np.array([0.3, 0.2, 0.25])
    bv, bt = W.box_mesh(half, (0.0, 0.0, 0.0), subdiv=2)
    qb = Rotation.from_euler("zyx", [25.0, 10.0, -5.0], degrees=True).as_quat()
    tb = np.array([1.4, 0.15, 0.35])
    cam = _cam(21, 15, 87.0, 58.0, 0.0, 35.0)
    o = np.array([0.0, 0.0, 1.5])
    poses = np.stack([_pose(o), _pose(tb, qb)])[None, None]
    out = _render(_plane_mesh(0.0), [EMPTY, (bv, bt)], [cam], poses[0], flags=True)
    right, down, fwd = _axes_world(cam, (0, 0, 0, 1))
    D, _ = _pixel_dirs(cam, right, down, fwd)
    Rb = Rotation.from_quat(_f32(qb)).as_matrix()
    tb32 = _f32(tb)
    o = _f32(o)
    ob = Rb.T @ (o - tb32)
    lam = []
    for d in D:
        db = Rb.T @ d
        with np.errstate(divide="ignore", invalid="ignore"):
            t1 = (-half - ob) / db
            t2 = (half - ob) / db
        tn = np.max(np.minimum(t1, t2))
        tf = np.min(np.maximum(t1, t2))
        box = tn if (tn <= tf and tn > 0) else np.inf
        plane = -o[2] / d[2] if d[2] < 0 else np.inf
        lam.append(min(box, plane))
    exp = _clipped(np.array(lam), cam)
    edge = (out["flags"] & oracle.FLAG_EDGE) != 0
    np.testing.assert_allclose(out["depth"][~edge], exp[~edge], rtol=0, atol=1e-6)
    assert np.sum(np.array(lam) < -o[2] / np.minimum(D[:, 2], -1e-9) - 1e-6) > 10   # the box is in view


def test_miss_far_and_near_clip():
    cam_up = _cam(5, 5, 60.0, 40.0, 0.0, -60.0)                 # looks up: nothing to hit
    out = _render(_plane_mesh(0.0), [EMPTY], [cam_up], _pose((0, 0, 1.0))[None, None])
    assert np.all(out["depth"] == 3.0) and np.all(out["raw"] == 3.0)
    cam_dn = _cam(5, 5, 40.0, 30.0, 0.0, 89.0)
    far = _render(_plane_mesh(-5.0), [EMPTY], [cam_dn], _pose((0, 0, 1.0))[None, None])
    assert np.all(far["depth"] == 3.0)                          # a hit beyond d_max reads d_max
    near = _render(_plane_mesh(0.95), [EMPTY], [cam_dn], _pose((0, 0, 1.0))[None, None])
    d_min = float(np.float32(0.1))
    assert np.all(near["depth"] == d_min) and np.all(near["raw"] < d_min)   # nearer than d_min reads d_min


def test_range_depth_and_per_env_intrinsics():
    h, Hc = 0.0, 1.2
    cam = _cam(9, 7, 70.0, 50.0, 0.0, 45.0)
    poses = np.stack([_pose((0, 0, Hc)), _pose((2, 0, Hc))])[:, None][None]   # [1, E=2, L=1, 7]
    intr = np.array([[[cam.fx * 1.2, cam.fy * 0.9, cam.cx + 0.3, cam.cy - 0.2]],
                     [[cam.fx * 0.8, cam.fy * 1.1, cam.cx, cam.cy]]], np.float32)
    sen = W.Sensor(depth_kind=1)
    out = _render(_plane_mesh(h), [EMPTY], [cam], poses[0], sensor=sen, per_env_intrinsics=intr)
    right, down, fwd = _axes_world(cam, (0, 0, 0, 1))
    n = cam.width * cam.height
    for e in range(2):
        D, rn = _pixel_dirs(cam, right, down, fwd, *intr[e, 0])
        lam = np.where(D[:, 2] < 0, (h - _f32(Hc)) / np.minimum(D[:, 2], -1e-30), np.inf)
        np.testing.assert_allclose(out["depth"][e * n:(e + 1) * n], _clipped(lam * rn, cam), rtol=0, atol=1e-9)


def _moller_trumbore(o, D, tri):
    """Vectorised closest hit (parameter along D) of rays o + lam D against triangles [T,3,3]."""
    v0, v1, v2 = tri[:, 0], tri[:, 1], tri[:, 2]
    e1, e2 = v1 - v0, v2 - v0
    best = np.full(len(D), np.inf)
    for i, d in enumerate(D):
        p = np.cross(d, e2)
        det = np.einsum("ij,ij->i", e1, p)
        ok = np.abs(det) > 1e-14
        inv = np.where(ok, 1.0 / np.where(ok, det, 1.0), 0.0)
        s = o - v0
        u = np.einsum("ij,ij->i", s, p) * inv
        q = np.cross(s, e1)
        v = (q @ d) * inv
        t = np.einsum("ij,ij->i", e2, q) * inv
        hit = ok & (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 0)
        if hit.any():
            best[i] = t[hit].min()
    return best


def test_random_soups_match_moller_trumbore():
    rng = np.random.default_rng(42)
    for trial in range(3):
        tv = rng.uniform([-2, -2, -0.5], [2, 2, 0.5], size=(60, 3)).astype(np.float32)
        tt = rng.integers(0, 60, size=(50, 3)).astype(np.int32)
        links = []
        for _ in range(2):
            lv = rng.uniform(-0.3, 0.3, size=(8, 3)).astype(np.float32)
            lt = rng.integers(0, 8, size=(10, 3)).astype(np.int32)
            links.append((lv, lt))
        cam = _cam(13, 9, 90.0, 70.0, rng.uniform(-180, 180), 55.0, d_max=5.0, mount=0)
        qs = [Rotation.from_euler("z", rng.uniform(-180, 180), degrees=True).as_quat()]   # camera link: yaw only
        qs += [Rotation.random(random_state=trial * 7 + k).as_quat() for k in range(2)]
        o = np.array([0.0, 0.0, 1.5])
        poses = np.stack([_pose(o, qs[0]), _pose((0.4, 0.2, 0.6), qs[1]), _pose((-0.3, 0.5, 0.5), qs[2])])
        out = _render((tv, tt), [EMPTY] + links, [cam], poses[None, None], flags=True)
        # world triangles from scipy rotations of the float32 link vertices
        tris = [tv[tt].astype(np.float64)]
        for k, (lv, lt) in enumerate(links):
            R = Rotation.from_quat(np.asarray(np.float32(qs[k + 1]), np.float64)).as_matrix()
            t = np.asarray(poses[k + 1, :3], np.float64)
            tris.append(lv[lt].astype(np.float64) @ R.T + t)
        right, down, fwd = _axes_world(cam, np.float32(qs[0]))
        D, _ = _pixel_dirs(cam, right, down, fwd)
        lam = _moller_trumbore(np.asarray(poses[0, :3], np.float64), D, np.concatenate(tris))
        exp = _clipped(lam, cam)
        edge = (out["flags"] & oracle.FLAG_EDGE) != 0
        np.testing.assert_allclose(out["depth"][~edge], exp[~edge], rtol=0, atol=1e-8)
        assert np.mean(exp < cam.d_max) > 0.1


def test_rigid_motion_invariance():
    w = W.config_small(n_steps=1, n_envs=2)
    base = _render((w.terrain_verts, w.terrain_tris), list(zip(w.link_verts, w.link_tris)), w.cameras, w.poses[0],
                   flags=True)
    G = Rotation.from_euler("zyx", [37.0, 4.0, -3.0], degrees=True)
    T = np.array([3.0, -2.0, 0.5])
    tv = (G.apply(w.terrain_verts.astype(np.float64)) + T).astype(np.float32)
    poses = w.poses[0].astype(np.float64).copy()
    poses[..., :3] = G.apply(poses[..., :3].reshape(-1, 3)).reshape(poses[..., :3].shape) + T
    q = (G * Rotation.from_quat(poses[..., 3:].reshape(-1, 4))).as_quat()
    poses[..., 3:] = q.reshape(poses[..., 3:].shape)
    moved = _render((tv, w.terrain_tris), list(zip(w.link_verts, w.link_tris)), w.cameras,
                    poses.astype(np.float32), flags=True)
    edge = ((base["flags"] | moved["flags"]) & oracle.FLAG_EDGE) != 0
    diff = np.abs(base["depth"] - moved["depth"])
    assert diff[~edge].max() < 2e-4, diff[~edge].max()       # FP32 re-rounding of the moved inputs only
    assert np.mean(diff[~edge] < 1e-5) > 0.99


def test_edge_flag_marks_silhouette_rays():
    half = np.array([0.3, 0.3, 0.25])
    bv, bt = W.box_mesh(half, (0.3, 0.0, 0.5), subdiv=2)      # top face z = 0.75, x in [0, 0.6]
    down = W.Camera(1, 1, 1.0, 1.0, 0.0, 0.0, 0, (0.0, 0.0, 0.0), W.mount_quat(0.0, 90.0), 0.1, 3.0)
    on_edge = _render(_plane_mesh(0.0), [EMPTY, (bv, bt)], [down],
                      np.stack([_pose((0.0, 0.0, 1.5)), _pose((0, 0, 0))])[None, None], flags=True)
    centre = _render(_plane_mesh(0.0), [EMPTY, (bv, bt)], [down],
                     np.stack([_pose((0.3, 0.01, 1.5)), _pose((0, 0, 0))])[None, None], flags=True)
    far = _render(_plane_mesh(0.0), [EMPTY, (bv, bt)], [down],
                  np.stack([_pose((-0.5, 0.0, 1.5)), _pose((0, 0, 0))])[None, None], flags=True)
    assert on_edge["flags"][0] & oracle.FLAG_EDGE
    assert abs(on_edge["depth"][0] - 0.75) < 1e-9
    assert not centre["flags"][0] & oracle.FLAG_EDGE and abs(centre["depth"][0] - 0.75) < 1e-9
    assert not far["flags"][0] & oracle.FLAG_EDGE and abs(far["depth"][0] - 1.5) < 1e-9


def _one_ray_over_plane(height, pitch_deg, rx=0.0, d_max=3.0, depth_kind=0):
    """One pixel ray of a 1x1 camera at `height` above the plane z = 0, pitched down by pitch_deg;
    the pixel sits rx (in units of the focal length) to the right of the optical axis."""
    cam = W.Camera(1, 1, 1.0, 1.0, -rx, 0.0, 0, (0.0, 0.0, 0.0), W.mount_quat(0.0, pitch_deg), 0.1, d_max)
    out = _render(_plane_mesh(0.0, half=400.0), [EMPTY], [cam], _pose((0.0, 0.0, height))[None, None],
                  sensor=W.Sensor(depth_kind=depth_kind), flags=True)
    return int(out["flags"][0]), float(out["raw"][0])


@pytest.mark.parametrize("offset,flagged", [(-2e-4, False), (-1.1e-4, False), (-0.9e-4, True), (-5e-5, True),
                                            (5e-5, True), (0.9e-4, True), (1.1e-4, False), (2e-4, False)])
def test_far_flag_band(offset, flagged):
    """FLAG_FAR marks a ray whose unclipped depth lies within 1e-4 m of d_max on either side (there FP32
    may decide hit or miss differently, and only a hit gets noise).  The depth of the single ray is set
    by geometry: a camera looking straight down from height d_max + offset at a flat plane."""
    d_max = 3.0
    h = float(np.float32(d_max + offset))
    flags, raw = _one_ray_over_plane(h, 90.0, d_max=d_max)
    assert abs(min(h, d_max) - raw) < 1e-9                  # the straight-down depth is the height
    assert bool(flags & oracle.FLAG_FAR) == flagged, (offset, flags)


def test_far_flag_not_on_misses_or_far_from_the_band():
    flags, raw = _one_ray_over_plane(1.0, -30.0)             # looking up: nothing is hit
    assert raw == 3.0 and not flags & oracle.FLAG_FAR
    flags, _ = _one_ray_over_plane(1.0, 90.0)                # hit at 1 m, far from d_max
    assert not flags & oracle.FLAG_FAR


def _grazing_u(height, pitch_rad, rx):
    """The depth change that a 2^-22 rad error of the ray direction causes, from the geometry alone: a
    ray rx to the right of an optical axis pitched down by p meets the plane at elevation a with
    sin a = sin p cos phi (tan phi = rx, the right axis is horizontal), after t = height / sin a; the
    incidence angle to the plane's normal is 90 deg - a, so tan(incidence) = cot a; z-depth = t cos phi,
    and the offset of the hit along the ray grows with the distance from the camera plus 1 m."""
    phi = math.atan(rx)
    a = math.asin(math.sin(pitch_rad) * math.cos(phi))
    t = height / math.sin(a)
    return math.cos(phi) * (t + 1.0) * 2.0 ** -22 / math.tan(a)


@pytest.mark.parametrize("rx", [0.0, 0.6])
@pytest.mark.parametrize("ratio", [0.5, 0.95, 1.05, 2.0])
def test_grazing_flag_threshold(rx, ratio):
    """FLAG_GRAZING marks a hit whose depth moves by more than 2.5e-5 m (a quarter of the tolerance) when
    the unit direction is off by 2^-22 rad (FP32 rounding).  The pitch is solved so that this amount,
    computed from the angle and the distance, is `ratio` times the threshold."""
    from scipy.optimize import brentq
    height, thr = 0.5, 2.5e-5
    p = brentq(lambda p: _grazing_u(height, p, rx) - ratio * thr, math.radians(0.5), math.radians(60.0))
    flags, raw = _one_ray_over_plane(height, math.degrees(p), rx=rx, d_max=40.0)
    phi = math.atan(rx)
    assert abs(raw - height / (math.sin(p) * math.cos(phi)) * math.cos(phi)) < 1e-4   # the plane was hit
    assert bool(flags & oracle.FLAG_GRAZING) == (ratio > 1.0), (rx, ratio, flags)


def test_grazing_flag_not_on_steep_hits_or_misses():
    flags, _ = _one_ray_over_plane(1.0, 90.0)                # normal incidence
    assert not flags & oracle.FLAG_GRAZING
    flags, _ = _one_ray_over_plane(1.0, -10.0, d_max=40.0)   # a miss is never grazing
    assert not flags & oracle.FLAG_GRAZING


# --------------------------------------------------------------------------------------------------
# sensor model
# --------------------------------------------------------------------------------------------------
def _plane_frames(sensor, n_envs=4, n_steps=6, step=None, s_first=None, env_offset=0):
    cam = _cam(48, 36, 80.0, 60.0, 0.0, 50.0)
    poses = np.stack([np.stack([_pose((e * 3.0, 0, 1.2))]) for e in range(n_envs)])   # [E, 1, 7]
    poses = np.repeat(poses[None], n_steps, axis=0)
    for s in range(n_steps):                                  # a different height per step
        poses[s, :, 0, 2] = 1.2 + 0.05 * s
    sc = oracle.OracleScene(*_plane_mesh(0.0), [EMPTY[0]], [EMPTY[1]])
    rays = oracle.all_rays([cam], n_envs)
    steps = range(n_steps) if step is None else [step]
    return cam, [sc.render([cam], poses, s, rays, sensor, s_first=s_first, env_offset=env_offset) for s in steps]


def test_dropout_rate_and_fill():
    p = 0.05
    sen = W.Sensor(p_drop=p, fill=0.0, seed=(3, 4))
    cam, frames = _plane_frames(sen)
    dropped = np.concatenate([(f["flags"] & oracle.FLAG_DROPPED) != 0 for f in frames])
    depth = np.concatenate([f["depth"] for f in frames])
    n = dropped.size
    assert abs(dropped.mean() - p) < 5 * math.sqrt(p * (1 - p) / n)
    assert np.all(depth[dropped] == 0.0)                       # fill survives the [0.1, 3] clip
    assert np.all(depth[~dropped] >= 0.1)
    assert not _plane_frames(W.Sensor(p_drop=0.0))[1][0]["flags"].any()
    one = _plane_frames(W.Sensor(p_drop=1.0, fill=-1.0))[1][0]
    assert np.all(one["depth"] == -1.0)


@pytest.mark.parametrize("sigma_abs,sigma_rel", [(0.01, 0.0), (0.0, 0.1), (0.005, 0.02)])
def test_noise_is_standard_normal_scaled(sigma_abs, sigma_rel):
    sen = W.Sensor(sigma_abs=sigma_abs, sigma_rel=sigma_rel, seed=(11, 22))
    cam, frames = _plane_frames(sen, n_envs=6)
    z = np.concatenate([f["depth"] for f in frames])
    raw = np.concatenate([f["raw"] for f in frames])
    hit = raw < cam.d_max
    sig = sigma_abs + sigma_rel * raw[hit]
    n = (z[hit] - raw[hit]) / sig
    # samples that no noise value can clip (|n| <= sqrt(-2 ln 2^-32) < 6.7), chosen on raw alone so
    # the selection does not depend on the noise
    inside = (raw[hit] - 6.7 * sig > cam.d_min) & (raw[hit] + 6.7 * sig < cam.d_max)
    n = n[inside]
    assert n.size > 5000
    assert abs(n.mean()) < 5 / math.sqrt(n.size)
    assert abs(n.var() - 1.0) < 5 * math.sqrt(2.0 / n.size)
    assert stats.kstest(n, "norm").pvalue > 1e-4
    assert np.all(z[~hit] == cam.d_max)                        # misses get no noise


def test_latency_histogram_uniform():
    sen = W.Sensor(max_latency=3, seed=(5, 6))
    ks = []
    sc = oracle.OracleScene(*_plane_mesh(0.0), [EMPTY[0]], [EMPTY[1]])
    cam = _cam(2, 2, 60.0, 40.0, 0.0, 45.0)
    E = 64
    poses = np.repeat(np.stack([_pose((0, 0, 1.0))] * E)[None, :, None], 40, axis=0)
    rays = np.array([[e, 0, 0, 0] for e in range(E)])
    for s in range(4, 40):
        ks.append(sc.render([cam], poses, s, rays, sen, flags=False)["k"])
    ks = np.concatenate(ks)
    counts = np.bincount(ks, minlength=4)
    assert counts.size == 4
    assert stats.chisquare(counts).pvalue > 1e-4


def test_latency_identity_exact():
    """out(s) with latency equals the undelayed output of the source step s' = max(s - k, s_first)."""
    delayed = W.Sensor(sigma_abs=0.01, p_drop=0.1, max_latency=3, seed=(9, 10))
    nodelay = W.Sensor(sigma_abs=0.01, p_drop=0.1, max_latency=0, seed=(9, 10))
    n_envs, n_steps = 4, 8
    s_first = np.array([0, 0, 5, 0], np.int64)
    cam, _ = _plane_frames(delayed, n_envs=1, n_steps=1)
    npx = cam.width * cam.height
    for s in range(5, 8):
        _, (fd,) = _plane_frames(delayed, n_envs, n_steps, step=s, s_first=s_first, env_offset=3)
        for e in range(n_envs):
            k = int(fd["k"][e * npx])
            src = max(s - k, int(s_first[e]))
            _, (fs,) = _plane_frames(nodelay, n_envs, n_steps, step=src, env_offset=3)
            sl = slice(e * npx, (e + 1) * npx)
            assert np.array_equal(fd["depth"][sl], fs["depth"][sl]), (s, e, k)
            assert np.all(fd["k"][sl] == k)                    # one draw per (env, camera, step)


# --------------------------------------------------------------------------------------------------
# adjacent steps: downsampling, randomised camera mounts, side masking
# --------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("f", [2, 5])
def test_downsample_is_the_block_mean_of_the_raw_closed_form(f):
    """A camera rendered at W x H and downsampled by f: every output pixel is the mean of its f x f
    raw block.  Expected values: the plane closed form per raw pixel, reshaped and averaged by numpy
    (a transposed block index or a dropped row of the block fails this: the image is yawed and
    partly beyond the far plane, so depth varies along both axes and includes misses)."""
    h, Hc = 0.0, 1.3
    cam = _cam(8 * f, 5 * f, 90.0, 60.0, 25.0, 30.0)
    cam.downsample = f
    q = Rotation.from_euler("z", 40.0, degrees=True).as_quat()
    out = _render(_plane_mesh(h), [EMPTY], [cam], _pose((0.2, 0.1, Hc), q)[None, None])
    right, down, fwd = _axes_world(cam, q)
    D, _ = _pixel_dirs(cam, right, down, fwd)
    lam = np.where(D[:, 2] < 0, (_f32(h) - _f32(Hc)) / np.where(D[:, 2] < 0, D[:, 2], -1.0), np.inf)
    raw = np.where(np.isfinite(lam) & (lam > 0) & (lam < cam.d_max), lam, cam.d_max).reshape(cam.height, cam.width)
    want = raw.reshape(cam.height // f, f, cam.width // f, f).mean(axis=(1, 3))
    want = np.clip(want, cam.d_min, cam.d_max)
    assert out["depth"].shape == (cam.out_width * cam.out_height,)
    np.testing.assert_allclose(out["depth"], want.reshape(-1), rtol=0, atol=1e-9)
    assert (want < cam.d_max).any() and (want == cam.d_max).any() and (raw[:, 0] != raw[:, -1]).any()


def test_downsample_factor_must_divide_the_image():
    cam = _cam(10, 6, 90.0, 60.0, 0.0, 30.0)
    cam.downsample = 4
    with pytest.raises(ValueError):
        _render(_plane_mesh(0.0), [EMPTY], [cam], _pose((0, 0, 1.0))[None, None], rays=np.zeros((1, 4), np.int64))


def test_randomised_mounts_plane_closed_form():
    """Per-env mount perturbation (dp, dq): camera at t_l + R_l (p_off + dp) with rotation
    R_l R_off R_dq (dq about the camera's own axes), checked against the plane closed form with the
    rotations composed by scipy."""
    rng = np.random.default_rng(3)
    h, E = 0.1, 5
    cam = _cam(12, 9, 80.0, 55.0, 10.0, 40.0, pos=(0.1, 0.0, 0.3))
    euler = np.stack([rng.uniform(-2.5, 2.5, E), rng.uniform(-3.0, 3.0, E), rng.uniform(-2.5, 2.5, E)], 1)
    dq = Rotation.from_euler("xyz", euler, degrees=True).as_quat()
    dp = rng.uniform(-0.025, 0.025, (E, 3))
    mount_dr = np.concatenate([dp, dq], 1).astype(np.float32)[:, None, :]        # [E, C=1, 7]
    link_q = Rotation.from_euler("z", rng.uniform(-180, 180, (E, 1)), degrees=True).as_quat()
    poses = np.stack([_pose((3.0 * e, 0.5, 1.2), link_q[e]) for e in range(E)])[:, None, :]
    out = _render(_plane_mesh(h, half=60.0), [EMPTY], [cam], poses, mount_dr=mount_dr)
    npx = cam.width * cam.height
    for e in range(E):
        Rl = Rotation.from_quat(_f32(link_q[e])).as_matrix()
        R = Rl @ Rotation.from_quat(_f32(cam.offset_quat)).as_matrix() @ Rotation.from_quat(_f32(dq[e])).as_matrix()
        o = _f32((3.0 * e, 0.5, 1.2)) + Rl @ (_f32(cam.offset_pos) + _f32(dp[e]))
        D, _ = _pixel_dirs(cam, R[:, 0], R[:, 1], R[:, 2])
        lam = np.where(D[:, 2] < 0, (_f32(h) - o[2]) / np.where(D[:, 2] < 0, D[:, 2], -1.0), np.inf)
        np.testing.assert_allclose(out["depth"][e * npx:(e + 1) * npx], _clipped(lam, cam), rtol=0, atol=1e-9)
    # the perturbation matters: without it the depths differ
    plain = _render(_plane_mesh(h, half=60.0), [EMPTY], [cam], poses)
    assert np.abs(plain["depth"] - out["depth"]).max() > 1e-3


def test_side_masking_columns_values_and_key():
    """Modes 0/1/2 mask 0/n1/n2 columns on both sides; the rest of the image is untouched; a masked
    value is d_min + (d_max - d_min)(w3 + 1/2) 2^-32 from the keyed stream of the current step (not
    the latency's source step); the values are uniform on [d_min, d_max]."""
    sen = W.Sensor(sigma_abs=0.01, p_drop=0.05, max_latency=3, seed=(21, 22))
    cam = _cam(24, 10, 80.0, 60.0, 0.0, 50.0)
    E, S, step, env_offset = 4, 6, 5, 7
    modes = np.array([0, 1, 2, 1], np.uint8)
    cols = (0, 3, 7)
    poses = np.stack([np.stack([_pose((e * 3.0, 0, 1.2 + 0.03 * e))]) for e in range(E)])
    poses = np.repeat(poses[None], S, axis=0)
    for s in range(S):
        poses[s, :, 0, 2] += 0.04 * s
    sc = oracle.OracleScene(*_plane_mesh(0.0), [EMPTY[0]], [EMPTY[1]])
    rays = oracle.all_rays([cam], E)
    base = sc.render([cam], poses, step, rays, sen, env_offset=env_offset)
    m = sc.render([cam], poses, step, rays, sen, env_offset=env_offset, rsm_mode=modes, rsm_cols=cols)
    assert (base["k"] > 0).any()                                # some sources are earlier steps
    x = rays[:, 2]
    n = np.asarray(cols)[modes[rays[:, 0]]]
    masked = (x < n) | (x >= cam.width - n)
    assert np.array_equal((m["flags"] & oracle.FLAG_MASKED) != 0, masked)
    assert np.array_equal(m["depth"][~masked], base["depth"][~masked])
    for i in np.flatnonzero(masked)[::5]:
        e, c, xx, yy = rays[i]
        w = oracle.philox4x32_10([env_offset + e, c, yy * cam.width + xx, step], [sen.seed[0], sen.seed[1]])
        want = np.float64(np.float32(cam.d_min)) + (np.float64(np.float32(cam.d_max)) - np.float64(np.float32(cam.d_min))) \
            * ((float(w[3]) + 0.5) / 2.0 ** 32)
        assert m["depth"][i] == want
    # uniformity of the fill over many masked pixels
    big = _cam(64, 48, 80.0, 60.0, 0.0, 50.0)
    r = oracle.all_rays([big], E)
    mm = sc.render([big], poses, step, r, sen, rsm_mode=np.full(E, 2, np.uint8), rsm_cols=(0, 0, 32), flags=False)
    u = (mm["depth"] - np.float32(big.d_min)) / (np.float32(big.d_max) - np.float32(big.d_min))
    assert stats.kstest(u, "uniform").pvalue > 1e-4


def test_mirrored_scene_gives_the_mirrored_image():
    """Reflecting the whole small workload in the plane y = 0 (terrain, link meshes in their frames,
    link poses, camera mounts) mirrors every image left-right: with the principal point at the image
    centre, pixel x of the mirrored render equals pixel W-1-x of the original.  Link poses reflect as
    q -> (-qx, qy, -qz, qw); a mount rotation as R -> M R F with F flipping the optical x axis."""
    w = W.config_small(n_steps=1, n_envs=3)
    base = _render((w.terrain_verts, w.terrain_tris), list(zip(w.link_verts, w.link_tris)), w.cameras, w.poses[0])
    M = np.diag([1.0, -1.0, 1.0])
    F = np.diag([-1.0, 1.0, 1.0])
    tv = (w.terrain_verts.astype(np.float64) @ M).astype(np.float32)
    lv = [(v.astype(np.float64) @ M).astype(np.float32) for v in w.link_verts]
    poses = w.poses[0].copy()
    poses[..., 1] = -poses[..., 1]
    poses[..., 3] = -poses[..., 3]
    poses[..., 5] = -poses[..., 5]
    cams = []
    for c in w.cameras:
        R = Rotation.from_quat(_f32(c.offset_quat)).as_matrix()
        q = Rotation.from_matrix(M @ R @ F).as_quat()
        cams.append(W.Camera(c.width, c.height, c.fx, c.fy, c.cx, c.cy, c.mount_link,
                             (c.offset_pos[0], -c.offset_pos[1], c.offset_pos[2]), tuple(q), c.d_min, c.d_max))
    mir = _render((tv, w.terrain_tris), list(zip(lv, w.link_tris)), cams, poses)
    n = 0
    for e in range(w.n_envs):
        for k, c in enumerate(w.cameras):
            off = e * sum(x.width * x.height for x in w.cameras) + sum(x.width * x.height for x in w.cameras[:k])
            sl = slice(off, off + c.width * c.height)
            a = base["depth"][sl].reshape(c.height, c.width)
            b = mir["depth"][sl].reshape(c.height, c.width)[:, ::-1]
            fa = base["flags"][sl].reshape(c.height, c.width)
            fb = mir["flags"][sl].reshape(c.height, c.width)[:, ::-1]
            edge = ((fa | fb) & oracle.FLAG_EDGE) != 0
            d = np.abs(a - b)[~edge]
            assert d.max() < 2e-6, d.max()             # float32 rounding of the reflected mount only
            n += d.size
            assert not np.array_equal(a, a[:, ::-1])   # the images are not symmetric themselves
    assert n > 0.99 * base["depth"].size
