"""Seeded synthetic inputs for multi-depth ray casting (Sec. 3.2.2, Algorithm 1).

This module builds the *inputs* of the method and nothing else: terrain heightfield meshes in the
paper's terrain families (20 deg slopes, stairs with 0.22/0.25/0.30 m runs, 0.25 m stepping stones
with 0.6 m gaps; Sec. 1, Sec. 3.1.1, Sec. 4.1), humanoid link meshes in their own link frames, a
kinematic chain that places the links in each environment, pinhole camera mounts and sensor
settings (Appendix A.2, Table "Domain randomization").  It contains none of the method's arithmetic
(no ray generation, intersection, min-merge or sensor model), so both the CUDA path and the CPU
oracle may take their inputs from it.

Conventions shared by both sides (documented in the C header as well):
  * link poses are float32 ``[S, E, L, 7]`` = (px, py, pz, qx, qy, qz, qw), world frame;
  * camera mounts are (link id, offset position, offset quaternion xyzw) and map the OpenCV optical
    frame (x right, y down, z forward) into the link frame;
  * pinhole intrinsics use integer pixel indices with the principal point at ((W-1)/2, (H-1)/2) and
    focal lengths that make the field of view span the image edges.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np
from scipy.spatial.transform import Rotation

__all__ = [
    "Camera", "Sensor", "Workload", "pinhole", "mount_quat",
    "box_mesh", "ellipsoid_mesh", "heightfield_mesh",
    "config_small", "config_scale", "config_uneven", "make_workload",
]


# --------------------------------------------------------------------------------------------------
# Plain records
# --------------------------------------------------------------------------------------------------
@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    mount_link: int
    offset_pos: Tuple[float, float, float]
    offset_quat: Tuple[float, float, float, float]  # xyzw, optical frame -> link frame
    d_min: float
    d_max: float
    downsample: int = 1   # f: rendered at width x height, output (width / f) x (height / f)

    @property
    def out_width(self) -> int:
        return self.width // max(1, self.downsample)

    @property
    def out_height(self) -> int:
        return self.height // max(1, self.downsample)


@dataclasses.dataclass
class Sensor:
    sigma_abs: float = 0.0
    sigma_rel: float = 0.0
    p_drop: float = 0.0
    fill: float = 0.0
    max_latency: int = 0
    seed: Tuple[int, int] = (0, 0)
    depth_kind: int = 0  # 0 = z-depth along the optical axis, 1 = range along the ray
    out_dtype: int = 0   # 0 = float32, 1 = float16, 2 = unorm16 over [0, d_max]

    @property
    def enabled(self) -> bool:
        return self.sigma_abs != 0 or self.sigma_rel != 0 or self.p_drop != 0 or self.max_latency != 0


@dataclasses.dataclass
class Workload:
    name: str
    terrain_verts: np.ndarray            # [V,3] float32, world frame
    terrain_tris: np.ndarray             # [T,3] int32
    link_verts: List[np.ndarray]         # per link [v,3] float32, link frame
    link_tris: List[np.ndarray]          # per link [t,3] int32
    cameras: List[Camera]
    poses: np.ndarray                    # [S,E,L,7] float32
    sensor: Sensor
    step0: int = 0                       # step number of poses[0]
    per_env_intrinsics: Optional[np.ndarray] = None  # [E,C,4] float32 (fx,fy,cx,cy) or None
    mount_delta: Optional[np.ndarray] = None         # [E,C,7] float32 (dp xyz, dq xyzw) or None
    rsm_modes: Optional[np.ndarray] = None           # [E] uint8 side-mask modes or None
    rsm_cols: Tuple[int, int, int] = (0, 0, 0)       # columns masked per side for modes 0, 1, 2

    @property
    def n_steps(self) -> int:
        return int(self.poses.shape[0])

    @property
    def n_envs(self) -> int:
        return int(self.poses.shape[1])

    @property
    def n_links(self) -> int:
        return int(self.poses.shape[2])

    @property
    def pixels_per_env(self) -> int:
        """Output pixels per env (downsampled images count at their output size)."""
        return int(sum(c.out_width * c.out_height for c in self.cameras))

    @property
    def raw_pixels_per_env(self) -> int:
        """Ray-cast pixels per env (downsampled cameras count at their raw size)."""
        return int(sum(c.width * c.height for c in self.cameras))

    @property
    def rays_per_step(self) -> int:
        return self.n_envs * self.raw_pixels_per_env

    def cam_offsets(self) -> np.ndarray:
        """Start of each camera's pixels inside one env's packed output row."""
        off = [0]
        for c in self.cameras:
            off.append(off[-1] + c.out_width * c.out_height)
        return np.asarray(off, dtype=np.int64)

    def link_arrays(self):
        """Concatenated link meshes: verts, vert offsets [L+1], tris (link-local ids), tri offsets."""
        vo, to = [0], [0]
        for v, t in zip(self.link_verts, self.link_tris):
            vo.append(vo[-1] + len(v))
            to.append(to[-1] + len(t))
        lv = np.concatenate(self.link_verts).astype(np.float32) if self.link_verts else np.zeros((0, 3), np.float32)
        lt = np.concatenate(self.link_tris).astype(np.int32) if self.link_tris else np.zeros((0, 3), np.int32)
        return lv, np.asarray(vo, np.int64), lt, np.asarray(to, np.int64)


# --------------------------------------------------------------------------------------------------
# Cameras
# --------------------------------------------------------------------------------------------------
def mount_quat(yaw_deg: float, pitch_down_deg: float) -> Tuple[float, float, float, float]:
    """Quaternion (xyzw) of an optical frame looking along yaw, tilted down by pitch, in the link frame."""
    y, p = math.radians(yaw_deg), math.radians(pitch_down_deg)
    z_axis = np.array([math.cos(p) * math.cos(y), math.cos(p) * math.sin(y), -math.sin(p)])
    x_axis = np.array([math.sin(y), -math.cos(y), 0.0])
    y_axis = np.cross(z_axis, x_axis)
    m = np.stack([x_axis, y_axis, z_axis], axis=1)
    q = Rotation.from_matrix(m).as_quat()
    return tuple(float(v) for v in q)


def pinhole(width: int, height: int, hfov_deg: float, vfov_deg: float, mount_link: int,
            offset_pos, yaw_deg: float, pitch_down_deg: float, d_min: float, d_max: float) -> Camera:
    fx = (width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)
    fy = (height / 2.0) / math.tan(math.radians(vfov_deg) / 2.0)
    return Camera(width, height, float(np.float32(fx)), float(np.float32(fy)),
                  (width - 1) / 2.0, (height - 1) / 2.0, mount_link,
                  tuple(float(v) for v in offset_pos), mount_quat(yaw_deg, pitch_down_deg),
                  float(d_min), float(d_max))


# --------------------------------------------------------------------------------------------------
# Meshes (welded, outward counter-clockwise winding)
# --------------------------------------------------------------------------------------------------
def box_mesh(half, center=(0.0, 0.0, 0.0), subdiv: int = 2):
    """Axis-aligned box, each face split into subdiv x subdiv quads (2 triangles each); welded."""
    n = subdiv
    idx = {}
    verts = []

    def vid(i, j, k):
        key = (i, j, k)
        if key not in idx:
            idx[key] = len(verts)
            verts.append([center[0] + half[0] * (2.0 * i / n - 1.0),
                          center[1] + half[1] * (2.0 * j / n - 1.0),
                          center[2] + half[2] * (2.0 * k / n - 1.0)])
        return idx[key]

    tris = []
    # (fixed axis, fixed value, u axis, v axis) chosen so that u x v points outward
    faces = [(0, n, 1, 2), (0, 0, 2, 1), (1, n, 2, 0), (1, 0, 0, 2), (2, n, 0, 1), (2, 0, 1, 0)]
    for ax, val, ua, va in faces:
        for a in range(n):
            for b in range(n):
                def p(du, dv):
                    c = [0, 0, 0]
                    c[ax] = val
                    c[ua] = a + du
                    c[va] = b + dv
                    return vid(*c)
                v00, v10, v11, v01 = p(0, 0), p(1, 0), p(1, 1), p(0, 1)
                tris.append([v00, v10, v11])
                tris.append([v00, v11, v01])
    return np.asarray(verts, np.float32), np.asarray(tris, np.int32)


def ellipsoid_mesh(radii, center=(0.0, 0.0, 0.0), slices: int = 16, bands: int = 17):
    """UV ellipsoid: two pole fans plus (bands-2) quad bands; slices*2*(bands-1) triangles (512 at 16/17)."""
    verts = [[center[0], center[1], center[2] + radii[2]]]
    for r in range(1, bands):
        th = math.pi * r / bands
        for s in range(slices):
            ph = 2.0 * math.pi * s / slices
            verts.append([center[0] + radii[0] * math.sin(th) * math.cos(ph),
                          center[1] + radii[1] * math.sin(th) * math.sin(ph),
                          center[2] + radii[2] * math.cos(th)])
    verts.append([center[0], center[1], center[2] - radii[2]])
    south = len(verts) - 1

    def ring(r, s):
        return 1 + (r - 1) * slices + (s % slices)

    tris = []
    for s in range(slices):
        tris.append([0, ring(1, s), ring(1, s + 1)])
    for r in range(1, bands - 1):
        for s in range(slices):
            a, b, c, d = ring(r, s), ring(r + 1, s), ring(r + 1, s + 1), ring(r, s + 1)
            tris.append([a, b, c])
            tris.append([a, c, d])
    for s in range(slices):
        tris.append([south, ring(bands - 1, s + 1), ring(bands - 1, s)])
    return np.asarray(verts, np.float32), np.asarray(tris, np.int32)


def heightfield_mesh(heights: np.ndarray, x0: float, y0: float, cell: float):
    """Grid mesh over heights[ny+1, nx+1] (row = y), two triangles per cell, counter-clockwise from above."""
    ny1, nx1 = heights.shape
    xs = x0 + cell * np.arange(nx1, dtype=np.float64)
    ys = y0 + cell * np.arange(ny1, dtype=np.float64)
    verts = np.empty((ny1 * nx1, 3), np.float32)
    verts[:, 0] = np.broadcast_to(xs[None, :], (ny1, nx1)).reshape(-1)
    verts[:, 1] = np.broadcast_to(ys[:, None], (ny1, nx1)).reshape(-1)
    verts[:, 2] = heights.reshape(-1)
    j, i = np.meshgrid(np.arange(ny1 - 1, dtype=np.int32), np.arange(nx1 - 1, dtype=np.int32), indexing="ij")
    v00 = (j * nx1 + i).reshape(-1)
    v10 = v00 + 1
    v01 = v00 + nx1
    v11 = v01 + 1
    tris = np.empty((2 * v00.size, 3), np.int32)
    tris[0::2, 0], tris[0::2, 1], tris[0::2, 2] = v00, v10, v11
    tris[1::2, 0], tris[1::2, 1], tris[1::2, 2] = v00, v11, v01
    return verts, tris


# --------------------------------------------------------------------------------------------------
# Terrain height functions (the paper's terrain families)
# --------------------------------------------------------------------------------------------------
def _edge_dist(lx, ly, size):
    return np.minimum(np.minimum(lx, size - lx), np.minimum(ly, size - ly))


def _stairs(d, rise, run, n_max):
    return rise * np.minimum(np.floor(d / run), n_max)


def _small_terrain_heights(xs, ys):
    """8 x 8 m tile centred at 0: x<0 pyramid staircase (rise 0.15, run 0.25), x>=0 a 20 deg ramp."""
    X, Y = np.meshgrid(xs, ys)
    d = np.minimum(np.minimum(X + 4.0, -X), np.minimum(Y + 4.0, 4.0 - Y))
    stairs = _stairs(np.maximum(d, 0.0), 0.15, 0.25, 1e9)
    ramp = np.maximum(X, 0.0) * math.tan(math.radians(20.0))
    return np.where(X < 0.0, stairs, ramp)


_TILE = 8.0


def _scale_tile_heights(lx, ly, kind):
    d = _edge_dist(lx, ly, _TILE)
    if kind in (0, 1, 2):                      # stairs, run 0.22 / 0.25 / 0.30, rise 0.20
        run = (0.22, 0.25, 0.30)[kind]
        return _stairs(d, 0.20, run, 8)
    if kind == 3:                              # 20 deg pyramid slope with a flat top
        return math.tan(math.radians(20.0)) * np.minimum(d, 2.5)
    # stepping stones: 0.25 m squares at a 0.85 m pitch (0.6 m gaps) over a 1 m pit, 1 m rim
    inner = (lx > 1.0) & (lx < 7.0) & (ly > 1.0) & (ly < 7.0)
    su = np.mod(lx - 1.0, 0.85)
    sv = np.mod(ly - 1.0, 0.85)
    stone = (su >= 0.30) & (su < 0.55) & (sv >= 0.30) & (sv < 0.55)
    return np.where(inner & ~stone, -1.0, 0.0)


def scale_terrain_height(x, y, tiles: int):
    """Analytic height of the tiled terrain at world (x, y) (terrain centred at the origin)."""
    half = tiles * _TILE / 2.0
    gx, gy = np.asarray(x, np.float64) + half, np.asarray(y, np.float64) + half
    ti = np.clip(np.floor(gx / _TILE).astype(np.int64), 0, tiles - 1)
    tj = np.clip(np.floor(gy / _TILE).astype(np.int64), 0, tiles - 1)
    lx, ly = gx - ti * _TILE, gy - tj * _TILE
    kind = (ti + tj) % 5
    out = np.zeros(np.broadcast(lx, ly).shape)
    for k in range(5):
        m = kind == k
        if np.any(m):
            out[m] = _scale_tile_heights(lx[m], ly[m], k)
    return out


def _scale_terrain(tiles: int, cell: float):
    n = int(round(tiles * _TILE / cell))
    half = tiles * _TILE / 2.0
    coords = -half + cell * np.arange(n + 1, dtype=np.float64)
    heights = np.empty((n + 1, n + 1), np.float32)
    chunk = 256
    for r0 in range(0, n + 1, chunk):
        ys = coords[r0:r0 + chunk]
        X, Y = np.meshgrid(coords, ys)
        heights[r0:r0 + chunk] = scale_terrain_height(X, Y, tiles)
    return heightfield_mesh(heights, -half, -half, cell)


# --------------------------------------------------------------------------------------------------
# Humanoid kinematic chain (G1-like proportions), link meshes in link frames
# --------------------------------------------------------------------------------------------------
# (name, parent, joint offset in parent frame, joint axis or None, standing angle,
#  mesh half extents, mesh centre in the link frame)
_LEG = [
    ("hip_pitch", None, (0.0, 0.10, -0.05), "y", -0.20, (0.04, 0.04, 0.04), (0.0, 0.0, 0.0)),
    ("hip_roll", "hip_pitch", (0.0, 0.0, 0.0), "x", 0.0, (0.035, 0.035, 0.035), (0.0, 0.0, -0.02)),
    ("hip_yaw", "hip_roll", (0.0, 0.0, -0.04), "z", 0.0, (0.06, 0.06, 0.15), (0.0, 0.0, -0.16)),
    ("knee", "hip_yaw", (0.0, 0.0, -0.31), "y", 0.40, (0.05, 0.05, 0.16), (0.0, 0.0, -0.17)),
    ("ankle_pitch", "knee", (0.0, 0.0, -0.34), "y", -0.20, (0.03, 0.03, 0.03), (0.0, 0.0, 0.0)),
    ("ankle_roll", "ankle_pitch", (0.0, 0.0, 0.0), "x", 0.0, (0.11, 0.045, 0.02), (0.03, 0.0, -0.03)),
]
_ARM3 = [
    ("shoulder_pitch", None, (0.0, 0.20, 0.27), "y", 0.20, (0.04, 0.04, 0.04), (0.0, 0.0, 0.0)),
    ("shoulder_roll", "shoulder_pitch", (0.0, 0.0, 0.0), "x", 0.15, (0.04, 0.04, 0.12), (0.0, 0.0, -0.12)),
    ("elbow", "shoulder_roll", (0.0, 0.0, -0.25), "y", -0.60, (0.035, 0.035, 0.11), (0.0, 0.0, -0.12)),
]
_ARM7 = [
    ("shoulder_pitch", None, (0.0, 0.20, 0.27), "y", 0.20, (0.04, 0.04, 0.04), (0.0, 0.0, 0.0)),
    ("shoulder_roll", "shoulder_pitch", (0.0, 0.0, 0.0), "x", 0.15, (0.035, 0.035, 0.035), (0.0, 0.0, 0.0)),
    ("shoulder_yaw", "shoulder_roll", (0.0, 0.0, -0.02), "z", 0.0, (0.04, 0.04, 0.11), (0.0, 0.0, -0.11)),
    ("elbow", "shoulder_yaw", (0.0, 0.0, -0.23), "y", -0.60, (0.035, 0.035, 0.035), (0.0, 0.0, 0.0)),
    ("wrist_roll", "elbow", (0.0, 0.0, -0.03), "z", 0.0, (0.032, 0.032, 0.08), (0.0, 0.0, -0.08)),
    ("wrist_pitch", "wrist_roll", (0.0, 0.0, -0.17), "y", 0.0, (0.025, 0.025, 0.025), (0.0, 0.0, 0.0)),
    ("wrist_yaw", "wrist_pitch", (0.0, 0.0, 0.0), "z", 0.0, (0.03, 0.05, 0.06), (0.0, 0.0, -0.05)),
]


def _robot(n_links: int):
    """Kinematic tree with 20 links (pelvis, torso, 2x6 legs, 2x3 arms) or 30 links
    (pelvis, waist yaw, waist roll, torso, 2x6 legs, 2x7 arms). Index of the torso link is returned."""
    links = [("pelvis", -1, (0.0, 0.0, 0.0), None, 0.0, (0.07, 0.12, 0.06), (0.0, 0.0, 0.0))]
    if n_links == 20:
        links.append(("torso", 0, (0.0, 0.0, 0.08), "z", 0.0, (0.07, 0.11, 0.13), (0.0, 0.0, 0.16)))
        torso, arm = 1, _ARM3
    elif n_links == 30:
        links.append(("waist_yaw", 0, (0.0, 0.0, 0.06), "z", 0.0, (0.04, 0.04, 0.03), (0.0, 0.0, 0.0)))
        links.append(("waist_roll", 1, (0.0, 0.0, 0.03), "x", 0.0, (0.04, 0.05, 0.03), (0.0, 0.0, 0.0)))
        links.append(("torso", 2, (0.0, 0.0, 0.02), "y", 0.0, (0.07, 0.11, 0.13), (0.0, 0.0, 0.16)))
        torso, arm = 3, _ARM7
    else:
        raise ValueError("robot has 20 or 30 links")
    for side in (1.0, -1.0):
        base = len(links)
        for k, (name, par, off, ax, q0, half, ctr) in enumerate(_LEG):
            parent = 0 if par is None else base + [r[0] for r in _LEG].index(par)
            links.append((name, parent, (off[0], side * off[1], off[2]), ax, q0, half, ctr))
    for side in (1.0, -1.0):
        base = len(links)
        for k, (name, par, off, ax, q0, half, ctr) in enumerate(arm):
            parent = torso if par is None else base + [r[0] for r in arm].index(par)
            links.append((name, parent, (off[0], side * off[1], off[2]), ax, q0, half, ctr))
    assert len(links) == n_links
    return links, torso


def _axis_rot(axis: Optional[str], ang: np.ndarray) -> np.ndarray:
    n = ang.shape[0]
    r = np.tile(np.eye(3), (n, 1, 1))
    if axis is None:
        return r
    c, s = np.cos(ang), np.sin(ang)
    i = "xyz".index(axis)
    a, b = [(1, 2), (2, 0), (0, 1)][i]
    r[:, a, a], r[:, a, b], r[:, b, a], r[:, b, b] = c, -s, s, c
    return r


def _link_poses(links, root_pos, root_yaw, angles):
    """Forward kinematics for one step: root [E,3], yaw [E], angles [E,L] -> poses [E,L,7] float32."""
    E = root_pos.shape[0]
    L = len(links)
    Rw = np.zeros((L, E, 3, 3))
    tw = np.zeros((L, E, 3))
    for l, (name, parent, off, ax, q0, half, ctr) in enumerate(links):
        if parent < 0:
            Rw[l] = _axis_rot("z", root_yaw)
            tw[l] = root_pos
        else:
            Rw[l] = Rw[parent] @ _axis_rot(ax, angles[:, l])
            tw[l] = tw[parent] + np.einsum("eij,j->ei", Rw[parent], np.asarray(off))
    q = Rotation.from_matrix(Rw.transpose(1, 0, 2, 3).reshape(-1, 3, 3)).as_quat().reshape(E, L, 4)
    out = np.empty((E, L, 7), np.float32)
    out[..., :3] = tw.transpose(1, 0, 2)
    out[..., 3:] = q
    return out


def _pose_sequence(links, root_pos, root_yaw, n_steps, rng, amp=0.3):
    L = len(links)
    E = root_pos.shape[0]
    stand = np.array([lk[4] for lk in links])
    seq = np.empty((n_steps, E, L, 7), np.float32)
    for s in range(n_steps):
        ang = stand[None, :] + rng.uniform(-amp, amp, size=(E, L))
        seq[s] = _link_poses(links, root_pos, root_yaw, ang)
    return seq


def _link_meshes(links, kind: str):
    lv, lt = [], []
    for (name, parent, off, ax, q0, half, ctr) in links:
        if kind == "box":
            v, t = box_mesh(half, ctr, subdiv=2)
        else:
            v, t = ellipsoid_mesh(half, ctr, slices=16, bands=17)
        lv.append(v)
        lt.append(t)
    return lv, lt


def _torso_cameras(torso: int, sizes, hfov=87.0, vfov=58.0, d_min=0.1, d_max=3.0):
    """Front/back cameras on the torso (+-0.10 m x, +0.30 m z, pitched 50 deg down), and for four
    cameras left/right ones (+-0.12 m y)."""
    mounts = [((0.10, 0.0, 0.30), 0.0), ((-0.10, 0.0, 0.30), 180.0),
              ((0.0, 0.12, 0.30), 90.0), ((0.0, -0.12, 0.30), -90.0)]
    cams = []
    for k, (w, h) in enumerate(sizes):
        pos, yaw = mounts[k]
        cams.append(pinhole(w, h, hfov, vfov, torso, pos, yaw, 50.0, d_min, d_max))
    return cams


# --------------------------------------------------------------------------------------------------
# The workloads
# --------------------------------------------------------------------------------------------------
def config_small(n_steps: int = 4, n_envs: int = 8, width: int = 32, height: int = 24,
                 sensor: Optional[Sensor] = None) -> Workload:
    """8 envs x 2 cameras x 32x24 px; 8x8 m terrain at 0.2 m (3,200 tris: stairs rise 0.15 / run
    0.25 and a 20 deg ramp); 20 links of 48-triangle boxes; joints +-0.3 rad around a standing pose."""
    cell = 0.2
    n = 40
    coords = -4.0 + cell * np.arange(n + 1, dtype=np.float64)
    heights = _small_terrain_heights(coords, coords).astype(np.float32)
    tv, tt = heightfield_mesh(heights, -4.0, -4.0, cell)
    links, torso = _robot(20)
    lv, lt = _link_meshes(links, "box")
    rng_root = np.random.default_rng(2)
    xy = rng_root.uniform(-3.0, 3.0, size=(n_envs, 2))
    yaw = rng_root.uniform(-math.pi, math.pi, size=n_envs)
    h = np.array([_small_terrain_heights(np.array([x]), np.array([y]))[0, 0] for x, y in xy])
    root = np.stack([xy[:, 0], xy[:, 1], h + 0.75], axis=1)
    poses = _pose_sequence(links, root, yaw, n_steps, np.random.default_rng(1))
    cams = _torso_cameras(torso, [(width, height)] * 2)
    return Workload("small: %d envs x 2 cams x %dx%d px, 3,200-tri terrain, 20 x 48-tri links"
                    % (n_envs, width, height), tv, tt, lv, lt, cams, poses,
                    sensor if sensor is not None else Sensor())


def scale_sensor() -> Sensor:
    return Sensor(sigma_abs=0.01, sigma_rel=0.0, p_drop=0.02, fill=0.0, max_latency=3,
                  seed=(0x52504C31, 0))


def config_scale(n_steps: int = 4, n_envs: int = 4096, tiles: int = 20, cell: float = 0.05,
                 cam_sizes: Sequence[Tuple[int, int]] = ((64, 48), (64, 48)),
                 sensor: Optional[Sensor] = None, seed: int = 0) -> Workload:
    """4096 envs x 2 cameras x 64x48 px; 20x20 tiles of 8x8 m at 0.05 m (20.48M tris; stairs 0.22 /
    0.25 / 0.30 m run at 0.20 m rise, 20 deg slopes, stepping stones); 30 links of 512-triangle
    ellipsoids; sensor sigma 0.01 m, 2 % dropout, latency 0-3 steps."""
    tv, tt = _scale_terrain(tiles, cell)
    links, torso = _robot(30)
    lv, lt = _link_meshes(links, "ellipsoid")
    poses, cams = scale_envs(n_envs, n_steps, tiles, cam_sizes, seed)
    return Workload("scale: %d envs x %d cams, %d-tri terrain (%dx%d tiles at %.2f m), 30 x 512-tri links"
                    % (n_envs, len(cams), len(tt), tiles, tiles, cell), tv, tt, lv, lt, cams, poses,
                    sensor if sensor is not None else scale_sensor())


def scale_envs(n_envs: int, n_steps: int, tiles: int = 20,
               cam_sizes: Sequence[Tuple[int, int]] = ((64, 48), (64, 48)), seed: int = 0):
    """Poses [S, E, 30, 7] of envs spread over the tiled terrain (env e on tile e mod tiles^2, uniform in
    its inner 5x5 m, 0.75 m above the ground, uniform yaw) and the torso cameras; no mesh is built."""
    links, torso = _robot(30)
    rng = np.random.default_rng(seed + 2)
    tile = np.arange(n_envs) % (tiles * tiles)
    ti, tj = tile // tiles, tile % tiles
    half = tiles * _TILE / 2.0
    x = -half + ti * _TILE + rng.uniform(1.5, 6.5, size=n_envs)
    y = -half + tj * _TILE + rng.uniform(1.5, 6.5, size=n_envs)
    yaw = rng.uniform(-math.pi, math.pi, size=n_envs)
    h = scale_terrain_height(x, y, tiles)
    root = np.stack([x, y, h + 0.75], axis=1)
    poses = _pose_sequence(links, root, yaw, n_steps, np.random.default_rng(seed + 1))
    return poses, _torso_cameras(torso, list(cam_sizes))


def config_uneven(n_steps: int = 4, n_envs: int = 4096, tiles: int = 20, cell: float = 0.05,
                  seed: int = 0) -> Workload:
    """4096 envs x 4 uneven cameras (front/back 80x60, left/right 48x36), FP32 depth, no sensor."""
    return config_scale(n_steps, n_envs, tiles, cell, ((80, 60), (80, 60), (48, 36), (48, 36)),
                        sensor=Sensor(), seed=seed)


# --------------------------------------------------------------------------------------------------
# The paper's perception settings (Sec. 4.1) and randomisation (Appendix A.2; Sec. 3.2.4)
# --------------------------------------------------------------------------------------------------
def _quat_axis(axis: int, ang: np.ndarray) -> np.ndarray:
    """Quaternions (x, y, z, w) of rotations by `ang` radians about coordinate axis 0, 1 or 2."""
    q = np.zeros(ang.shape + (4,))
    q[..., axis] = np.sin(ang / 2.0)
    q[..., 3] = np.cos(ang / 2.0)
    return q


def _quat_mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Hamilton product a * b of (x, y, z, w) quaternions (rotation b first, then a)."""
    ax, ay, az, aw = np.moveaxis(a, -1, 0)
    bx, by, bz, bw = np.moveaxis(b, -1, 0)
    return np.stack([aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw,
                     aw * bw - ax * bx - ay * by - az * bz], axis=-1)


def camera_randomization(n_envs: int, cams: Sequence[Camera], seed: int = 0, dpos: float = 0.025,
                         euler_deg: Tuple[float, float, float] = (2.5, 3.0, 2.5), dfov_deg: float = 2.0):
    """Per-env camera draws of the perception randomisation (Appendix A.2): mount translation
    U(+-dpos) per axis; rotation by Euler angles (roll, pitch, yaw) U(+-2.5, +-3.0, +-2.5) deg about
    the camera's optical axis z, right axis x and down axis y, composed as R_z(roll) R_x(pitch)
    R_y(yaw); FOV change dFOV U(+-2) deg added to the horizontal FOV, both focal lengths scaled by
    the same factor (square pixels kept).  Returns (mount_delta [E,C,7], per_env_intrinsics [E,C,4])."""
    rng = np.random.default_rng(seed + 17)
    C = len(cams)
    dp = rng.uniform(-dpos, dpos, size=(n_envs, C, 3))
    ang = np.radians(np.stack([rng.uniform(-a, a, size=(n_envs, C)) for a in euler_deg], axis=-1))
    dq = _quat_mul(_quat_mul(_quat_axis(2, ang[..., 0]), _quat_axis(0, ang[..., 1])), _quat_axis(1, ang[..., 2]))
    dfov = np.radians(rng.uniform(-dfov_deg, dfov_deg, size=(n_envs, C)))
    intr = np.zeros((n_envs, C, 4), np.float32)
    for c, cam in enumerate(cams):
        hfov = 2.0 * np.arctan(cam.width / (2.0 * cam.fx))
        scale = np.tan(hfov / 2.0) / np.tan((hfov + dfov[:, c]) / 2.0)
        intr[:, c, 0] = cam.fx * scale
        intr[:, c, 1] = cam.fy * scale
        intr[:, c, 2] = cam.cx
        intr[:, c, 3] = cam.cy
    return np.concatenate([dp, dq], axis=-1).astype(np.float32), intr


# Side-mask mode probabilities (none, small, large) per terrain kind: larger masks on continuous
# terrain (stairs, slopes), smaller ones on stepping stones (Sec. 3.2.4 gives the ordering only).
RSM_PROBS = {"continuous": (0.4, 0.2, 0.4), "stones": (0.5, 0.4, 0.1)}


def side_mask_modes(n_envs: int, tiles: int = 20, seed: int = 0) -> np.ndarray:
    """Mode per env (0 none, 1 small, 2 large) drawn from RSM_PROBS by the kind of the env's tile
    (env e stands on tile e mod tiles^2, as scale_envs places it)."""
    rng = np.random.default_rng(seed + 23)
    tile = np.arange(n_envs) % (tiles * tiles)
    kind = (tile // tiles + tile % tiles) % 5
    u = rng.uniform(size=n_envs)
    modes = np.zeros(n_envs, np.uint8)
    for stones, probs in ((False, RSM_PROBS["continuous"]), (True, RSM_PROBS["stones"])):
        m = (kind == 4) == stones
        modes[m] = np.where(u[m] < probs[0], 0, np.where(u[m] < probs[0] + probs[1], 1, 2))
    return modes


def perception_sensor() -> Sensor:
    """The paper's depth randomisation preset: sigma = 0.1 depth, 5 % dropout; latency 0-3 steps."""
    return Sensor(sigma_abs=0.0, sigma_rel=0.1, p_drop=0.05, fill=0.0, max_latency=3, seed=(0x52504C31, 1))


def perception_cameras(torso: int, n_cams: int = 2, raw=(240, 135), downsample: int = 5):
    """Torso cameras with the paper's perception settings (Sec. 4.1): FOV 101 x 69 deg, raw 240x135
    rendered and downsampled to 48x27; front/back, then left/right for four cameras."""
    cams = _torso_cameras(torso, [raw] * n_cams, hfov=101.0, vfov=69.0)
    for c in cams:
        c.downsample = downsample
    return cams


def config_perception(n_steps: int = 4, n_envs: int = 4096, tiles: int = 20, cell: float = 0.05, n_cams: int = 2,
                      seed: int = 0, rsm_cols: Tuple[int, int, int] = (0, 6, 12)) -> Workload:
    """The scale terrain and robot with the paper's cameras: 240x135 raw downsampled to 48x27 (101 x 69
    deg), per-env camera pose and FOV randomisation, side masking by terrain kind, sensor preset."""
    tv, tt = _scale_terrain(tiles, cell)
    links, torso = _robot(30)
    lv, lt = _link_meshes(links, "ellipsoid")
    poses, _ = scale_envs(n_envs, n_steps, tiles, seed=seed)
    cams = perception_cameras(torso, n_cams)
    md, intr = camera_randomization(n_envs, cams, seed)
    return Workload("perception: %d envs x %d cams 240x135 -> 48x27, %d-tri terrain, camera DR, side masking"
                    % (n_envs, n_cams, len(tt)), tv, tt, lv, lt, cams, poses, perception_sensor(),
                    per_env_intrinsics=intr, mount_delta=md, rsm_modes=side_mask_modes(n_envs, tiles, seed),
                    rsm_cols=rsm_cols)


def make_workload(name: str, **kw) -> Workload:
    return {"small": config_small, "scale": config_scale, "uneven": config_uneven,
            "perception": config_perception}[name](**kw)
