"""FP64 brute-force CPU oracle (test infrastructure).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg import this package.
It wraps ``oracle.c`` (plain C, OpenMP over rays) through ctypes.  It shares no code with the CUDA
path: the only common module is the seeded workload generator, which holds none of the method's
arithmetic.  See ``oracle.c`` for what is computed and the passages it follows (Sec. 3.2.2,
Algorithm 1, Appendix A.2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

FLAG_EDGE = 1
FLAG_EDGE_1E6 = 2
FLAG_FAR = 4
FLAG_DROPPED = 8
FLAG_GRAZING = 16
FLAG_MASKED = 32
# rays on which FP32 arithmetic may legitimately decide differently from the FP64 oracle
FLAG_FP32_SENSITIVE = 1 | 4 | 16

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, FP64, no contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fno-fast-math",
               "-fopenmp", "-fPIC", "-shared", "-fvisibility=hidden", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        L.oracle_philox4x32_10.argtypes = [P, P, P]
        L.oracle_philox4x32_10.restype = None
        L.oracle_scene_create.argtypes = [P, ctypes.c_int64, P, ctypes.c_int64, P, P, P, P, ctypes.c_int32]
        L.oracle_scene_create.restype = ctypes.c_void_p
        L.oracle_scene_destroy.argtypes = [P]
        L.oracle_scene_destroy.restype = None
        L.oracle_render.argtypes = [P, P, P, ctypes.c_int32, P, P, ctypes.c_int64, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_int64, P, P, ctypes.c_int32, P,
                                    ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, P, P, P, P, P, P, P,
                                    ctypes.c_int32]
        L.oracle_render.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(counter: Sequence[int], key: Sequence[int]) -> np.ndarray:
    c = np.asarray(counter, np.uint32)
    k = np.asarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


class _Sensor(ctypes.Structure):
    _fields_ = [("sigma_abs", ctypes.c_float), ("sigma_rel", ctypes.c_float),
                ("p_drop", ctypes.c_float), ("fill", ctypes.c_float),
                ("max_latency", ctypes.c_int32), ("seed", ctypes.c_uint32 * 2),
                ("depth_kind", ctypes.c_int32)]


class OracleScene:
    """Terrain + link meshes held by the oracle (silhouette edges are classified once here)."""

    def __init__(self, terrain_verts, terrain_tris, link_verts: Sequence[np.ndarray],
                 link_tris: Sequence[np.ndarray]):
        self._keep = []
        tv = np.ascontiguousarray(terrain_verts, np.float32).reshape(-1, 3)
        tt = np.ascontiguousarray(terrain_tris, np.int32).reshape(-1, 3)
        vo, to = [0], [0]
        for v, t in zip(link_verts, link_tris):
            vo.append(vo[-1] + len(v))
            to.append(to[-1] + len(t))
        lv = (np.ascontiguousarray(np.concatenate([np.asarray(v, np.float32).reshape(-1, 3) for v in link_verts]))
              if len(link_verts) else np.zeros((1, 3), np.float32))
        lt = (np.ascontiguousarray(np.concatenate([np.asarray(t, np.int32).reshape(-1, 3) for t in link_tris]))
              if len(link_tris) else np.zeros((1, 3), np.int32))
        vo = np.asarray(vo, np.int64)
        to = np.asarray(to, np.int64)
        self._keep = [tv, tt, lv, lt, vo, to]
        self.n_links = len(link_verts)
        h = lib().oracle_scene_create(_ptr(tv), len(tv), _ptr(tt), len(tt), _ptr(lv), _ptr(vo), _ptr(lt),
                                      _ptr(to), self.n_links)
        if not h:
            raise ValueError("oracle_scene_create failed (bad indices or out of memory)")
        self._h = h

    @classmethod
    def from_workload(cls, w) -> "OracleScene":
        return cls(w.terrain_verts, w.terrain_tris, w.link_verts, w.link_tris)

    def close(self):
        if getattr(self, "_h", None):
            lib().oracle_scene_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def render(self, cameras, poses: np.ndarray, step: int, rays: np.ndarray, sensor=None, step0: int = 0,
               s_first: Optional[np.ndarray] = None, env_offset: int = 0,
               per_env_intrinsics: Optional[np.ndarray] = None, flags: bool = True, threads: int = 0,
               mount_dr: Optional[np.ndarray] = None, rsm_mode: Optional[np.ndarray] = None,
               rsm_cols: Sequence[int] = (0, 0, 0)):
        """Depth of the rays [N,4] = (env, cam, x, y) at `step`; poses [S,E,L,7] start at step0.
        (x, y) index the output image ((width, height) / downsample).  mount_dr [E,C,7] perturbs each
        env's camera mounts (dp xyz, dq xyzw); rsm_mode [E] (0 none, 1 small, 2 large) with rsm_cols
        masks that many columns on both sides of every image.

        Returns dict(depth=[N] f64, raw=[N] f64, k=[N] i32, flags=[N] i32)."""
        poses = np.ascontiguousarray(poses, np.float32)
        S, E, L, _ = poses.shape
        cam_i = np.ascontiguousarray([[c.width, c.height, c.mount_link, getattr(c, "downsample", 1)]
                                      for c in cameras], np.int32)
        cam_f = np.ascontiguousarray([[c.fx, c.fy, c.cx, c.cy, *c.offset_pos, *c.offset_quat, c.d_min, c.d_max]
                                      for c in cameras], np.float32)
        rays = np.ascontiguousarray(rays, np.int64).reshape(-1, 4)
        n = len(rays)
        sen = _Sensor()
        if sensor is not None:
            sen.sigma_abs, sen.sigma_rel, sen.p_drop, sen.fill = (sensor.sigma_abs, sensor.sigma_rel,
                                                                  sensor.p_drop, sensor.fill)
            sen.max_latency = sensor.max_latency
            sen.seed[0], sen.seed[1] = int(sensor.seed[0]) & 0xFFFFFFFF, int(sensor.seed[1]) & 0xFFFFFFFF
            sen.depth_kind = sensor.depth_kind
        sf = None if s_first is None else np.ascontiguousarray(s_first, np.int64)
        intr = None if per_env_intrinsics is None else np.ascontiguousarray(per_env_intrinsics, np.float32)
        mdr = None if mount_dr is None else np.ascontiguousarray(mount_dr, np.float32).reshape(E, len(cameras), 7)
        rsm = None if rsm_mode is None else np.ascontiguousarray(rsm_mode, np.uint8).reshape(E)
        cols = np.ascontiguousarray(rsm_cols, np.int32).reshape(3)
        depth = np.zeros(n, np.float64)
        raw = np.zeros(n, np.float64)
        k = np.zeros(n, np.int32)
        fl = np.zeros(n, np.int32)
        rc = lib().oracle_render(self._h, _ptr(cam_i), _ptr(cam_f), len(cameras), _ptr(intr), _ptr(poses), S, E, L,
                                 int(step0), _ptr(sf), ctypes.byref(sen), int(env_offset), _ptr(rays), n,
                                 int(step), int(bool(flags)), _ptr(mdr), _ptr(rsm), _ptr(cols), _ptr(depth),
                                 _ptr(raw), _ptr(k), _ptr(fl), int(threads))
        if rc != 0:
            raise ValueError("oracle_render: bad argument (ray index, step outside the pose window, s_first, "
                         "a downsample factor that does not divide the image)")
        return {"depth": depth, "raw": raw, "k": k, "flags": fl}


def all_rays(cameras, n_envs: int) -> np.ndarray:
    """Every (env, cam, x, y) of the output images in the packed order [E][cam][y][x]."""
    out = []
    for e in range(n_envs):
        for c, cam in enumerate(cameras):
            f = getattr(cam, "downsample", 1)
            y, x = np.meshgrid(np.arange(cam.height // f), np.arange(cam.width // f), indexing="ij")
            n = x.size
            out.append(np.stack([np.full(n, e), np.full(n, c), x.reshape(-1), y.reshape(-1)], axis=1))
    return np.concatenate(out).astype(np.int64)
