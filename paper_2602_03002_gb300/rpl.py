"""Thin ctypes binding of librpl.so (include/rpl.h).

The module-level functions carry the C names and only marshal arguments; ``Scene`` and ``View`` are
small owners of the C handles on top of them.  PyTorch provides device memory and streams; every
step of the path runs in the library's CUDA kernels.  If librpl.so has not been built the import of
this module fails loudly instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# RPL_CHECKED=1 selects the bounds-checked build (librpl_checked.so, built by build.build(checked=True))
LIB_PATH = os.path.join(_HERE, "librpl_checked.so" if os.environ.get("RPL_CHECKED") == "1" else "librpl.so")

RPL_OK = 0
RPL_ERR_TIMEOUT = 6
_STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OUT_OF_MEMORY", 3: "CUDA", 4: "NOT_FOUND", 5: "CAPACITY",
           6: "TIMEOUT", 7: "DEVICE_FAULT"}
RPL_MAX_CAMERAS = 8
RPL_MAX_LINKS = 64
RPL_DEPTH_Z, RPL_DEPTH_RANGE = 0, 1
RPL_BVH2, RPL_BVH8Q8, RPL_BVH4 = 0, 1, 2
RPL_OUT_F32, RPL_OUT_F16, RPL_OUT_U16 = 0, 1, 2


class RplError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class rpl_scene_opts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("bvh_kind", ctypes.c_int32), ("max_leaf_size", ctypes.c_int32),
                ("build_threads", ctypes.c_int32), ("sah_node_cost", ctypes.c_float)]


class rpl_camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("mount_link", ctypes.c_int32), ("offset_pos", ctypes.c_float * 3),
                ("offset_quat_xyzw", ctypes.c_float * 4), ("d_min", ctypes.c_float), ("d_max", ctypes.c_float),
                ("downsample", ctypes.c_int32)]


class rpl_sensor_params(ctypes.Structure):
    _fields_ = [("sigma_abs", ctypes.c_float), ("sigma_rel", ctypes.c_float), ("p_drop", ctypes.c_float),
                ("fill", ctypes.c_float), ("max_latency", ctypes.c_int32), ("seed", ctypes.c_uint32 * 2),
                ("depth_kind", ctypes.c_int32), ("out_dtype", ctypes.c_int32)]


class rpl_scene_info(ctypes.Structure):
    _fields_ = [("terrain_tris", ctypes.c_int64), ("terrain_nodes", ctypes.c_int64),
                ("terrain_bytes", ctypes.c_int64), ("terrain_depth", ctypes.c_int32), ("n_links", ctypes.c_int32),
                ("link_tris", ctypes.c_int64), ("link_nodes", ctypes.c_int64), ("link_bytes", ctypes.c_int64),
                ("link_depth", ctypes.c_int32), ("frozen", ctypes.c_int32)]


class rpl_tuning(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("terrain_first", ctypes.c_int32), ("min_blocks", ctypes.c_int32), ("env_order", ctypes.c_int32),
                ("chunk_envs", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class rpl_server_opts(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int32), ("n_streams", ctypes.c_int32), ("staging_bytes", ctypes.c_int64),
                ("min_blocks", ctypes.c_int32), ("persistent", ctypes.c_int32)]


class rpl_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "completed", "failed", "cancelled", "batches",
                                                "fused_requests")] + \
               [("staging_peak_bytes", ctypes.c_int64), ("max_batch_seen", ctypes.c_int32),
                ("max_inflight_batches_seen", ctypes.c_int32)]


class rpl_counters(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("rays", "terrain_nodes", "terrain_tris", "link_boxes",
                                                "link_nodes", "link_tris")]


EXPORTS = ["rpl_bvh_build_host", "rpl_bvh8_build_host", "rpl_scene_create", "rpl_link_mesh_add", "rpl_scene_info_get", "rpl_scene_destroy", "rpl_view_create",
           "rpl_cameras_set", "rpl_cameras_randomize", "rpl_side_mask_set", "rpl_sensor_set", "rpl_view_state_size",
           "rpl_view_state_get", "rpl_view_state_set", "rpl_view_layout", "rpl_render", "rpl_view_reset", "rpl_sync",
           "rpl_render_counters", "rpl_view_timing", "rpl_view_host_async", "rpl_sensor_apply", "rpl_view_kernel_ms", "rpl_view_destroy", "rpl_last_error",
           "rpl_version", "rpl_render_static_scratch", "rpl_static_scratch_status", "rpl_view_tuning_set", "rpl_view_tuning_get",
           "rpl_view_autotune", "rpl_render_graph", "rpl_server_create", "rpl_server_submit", "rpl_server_wait",
           "rpl_server_cancel", "rpl_server_stats_get", "rpl_server_destroy"]

_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("librpl.so is not built (%s); run paper_2602_03002_gb300.build.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "rpl_bvh_build_host": ([P, I64, P, I64, I32, I32, P, I64, P, P, P], I32),
        "rpl_bvh8_build_host": ([P, I64, P, I64, I32, I32, P, I64, P, P, P], I32),
        "rpl_scene_create": ([P, I64, P, I64, P, P], I32),
        "rpl_link_mesh_add": ([P, I32, P, I64, P, I64], I32),
        "rpl_scene_info_get": ([P, P], I32),
        "rpl_scene_destroy": ([P], None),
        "rpl_view_create": ([P, I32, I32, P], I32),
        "rpl_cameras_set": ([P, P, I32, P], I32),
        "rpl_cameras_randomize": ([P, P], I32),
        "rpl_side_mask_set": ([P, P, P], I32),
        "rpl_sensor_set": ([P, P], I32),
        "rpl_view_layout": ([P, P, P], I32),
        "rpl_render": ([P, P, I64, I64, P, P], I32),
        "rpl_view_reset": ([P, P, I64, P], I32),
        "rpl_view_state_size": ([P, P], I32),
        "rpl_view_state_get": ([P, P, I64], I32),
        "rpl_view_state_set": ([P, P, I64], I32),
        "rpl_sync": ([P], I32),
        "rpl_render_counters": ([P, P, I64, I64, P, P, P], I32),
        "rpl_view_timing": ([P, I32], I32),
        "rpl_view_host_async": ([P, I32], I32),
        "rpl_sensor_apply": ([P, P, I64, I64, P, P], I32),
        "rpl_view_kernel_ms": ([P, P, I32, P], I32),
        "rpl_view_destroy": ([P], None),
        "rpl_last_error": ([], ctypes.c_char_p),
        "rpl_version": ([], I32),
        "rpl_render_static_scratch": ([P, P, I32, I32, I32, P, P, I64, I64, P, P], I32),
        "rpl_static_scratch_status": ([P, P], I32),
        "rpl_view_tuning_set": ([P, P], I32),
        "rpl_view_tuning_get": ([P, P], I32),
        "rpl_view_autotune": ([P, P, I64, I64, P, P, I32, P, P], I32),
        "rpl_render_graph": ([P, P, I64, P, P, P], I32),
        "rpl_server_create": ([P, P, P], I32),
        "rpl_server_submit": ([P, P, P, I64, I64, P, P], I32),
        "rpl_server_wait": ([P, ctypes.c_uint64, I32, P], I32),
        "rpl_server_cancel": ([P, ctypes.c_uint64], I32),
        "rpl_server_stats_get": ([P, P], I32),
        "rpl_server_destroy": ([P], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(status: int):
    if status != RPL_OK:
        raise RplError(status, lib().rpl_last_error().decode(errors="replace"))


def _ptr(a) -> Optional[int]:
    """Address of a numpy array or torch tensor (host or device), or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# --------------------------------------------------------------------------------------------------
# Same names as the C ABI (argument marshalling only)
# --------------------------------------------------------------------------------------------------
NODE_DTYPE = np.dtype([("c0x", "<f4", 2), ("c0y", "<f4", 2), ("c1x", "<f4", 2), ("c1y", "<f4", 2),
                       ("c0z", "<f4", 2), ("c1z", "<f4", 2), ("child", "<i4", 2), ("count", "<i4", 2)])
TRI_DTYPE = np.dtype([("v0", "<f4", 3), ("id", "<i4"), ("v1", "<f4", 3), ("pad1", "<f4"), ("v2", "<f4", 3),
                      ("pad2", "<f4")])


def rpl_bvh_build_host(verts, tris, max_leaf: int = 0, threads: int = 0):
    """Host BVH build (no GPU): returns (nodes structured array, leaf-ordered tris, depth)."""
    v = np.ascontiguousarray(verts, np.float32).reshape(-1, 3)
    t = np.ascontiguousarray(tris, np.int32).reshape(-1, 3)
    n = ctypes.c_int64()
    d = ctypes.c_int32()
    _check(lib().rpl_bvh_build_host(_ptr(v), len(v), _ptr(t), len(t), max_leaf, threads, None, 0, None,
                                    ctypes.byref(n), ctypes.byref(d)))
    nodes = np.zeros(n.value, NODE_DTYPE)
    out_t = np.zeros(len(t), TRI_DTYPE)
    _check(lib().rpl_bvh_build_host(_ptr(v), len(v), _ptr(t), len(t), max_leaf, threads, _ptr(nodes), n.value,
                                    _ptr(out_t) if len(t) else None, ctypes.byref(n), ctypes.byref(d)))
    return nodes, out_t, d.value


def rpl_bvh8_build_host(verts, tris, max_leaf: int = 0, threads: int = 0):
    """Host eight-wide quantised BVH build (no GPU): returns (nodes [N, 20] uint32, leaf-ordered tris, depth)."""
    v = np.ascontiguousarray(verts, np.float32).reshape(-1, 3)
    t = np.ascontiguousarray(tris, np.int32).reshape(-1, 3)
    n = ctypes.c_int64()
    d = ctypes.c_int32()
    _check(lib().rpl_bvh8_build_host(_ptr(v), len(v), _ptr(t), len(t), max_leaf, threads, None, 0, None,
                                     ctypes.byref(n), ctypes.byref(d)))
    nodes = np.zeros((n.value, 20), np.uint32)
    out_t = np.zeros(len(t), TRI_DTYPE)
    _check(lib().rpl_bvh8_build_host(_ptr(v), len(v), _ptr(t), len(t), max_leaf, threads, _ptr(nodes), n.value,
                                     _ptr(out_t) if len(t) else None, ctypes.byref(n), ctypes.byref(d)))
    return nodes, out_t, d.value


def rpl_scene_create(verts, tris, device: int = 0, max_leaf_size: int = 0, build_threads: int = 0,
                     sah_node_cost: float = 0.0, bvh_kind: int = 0) -> int:
    v = np.ascontiguousarray(verts, np.float32).reshape(-1, 3) if isinstance(verts, np.ndarray) else verts
    t = np.ascontiguousarray(tris, np.int32).reshape(-1, 3) if isinstance(tris, np.ndarray) else tris
    opts = rpl_scene_opts(device, bvh_kind, max_leaf_size, build_threads, sah_node_cost)
    h = ctypes.c_void_p()
    _check(lib().rpl_scene_create(_ptr(v), int(v.shape[0]), _ptr(t), int(t.shape[0]), ctypes.byref(opts),
                                  ctypes.byref(h)))
    return h.value


def rpl_link_mesh_add(scene: int, link_id: int, verts, tris):
    v = np.ascontiguousarray(verts, np.float32).reshape(-1, 3) if isinstance(verts, np.ndarray) else verts
    t = np.ascontiguousarray(tris, np.int32).reshape(-1, 3) if isinstance(tris, np.ndarray) else tris
    _check(lib().rpl_link_mesh_add(scene, int(link_id), _ptr(v), int(v.shape[0]), _ptr(t), int(t.shape[0])))


def rpl_scene_info_get(scene: int) -> dict:
    info = rpl_scene_info()
    _check(lib().rpl_scene_info_get(scene, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in rpl_scene_info._fields_}


def rpl_view_create(scene: int, n_envs: int, n_links: int) -> int:
    h = ctypes.c_void_p()
    _check(lib().rpl_view_create(scene, int(n_envs), int(n_links), ctypes.byref(h)))
    return h.value


def _camera_struct(c) -> rpl_camera:
    g = (lambda k, d=None: c.get(k, d)) if isinstance(c, dict) else (lambda k, d=None: getattr(c, k, d))
    return rpl_camera(int(g("width")), int(g("height")), g("fx"), g("fy"), g("cx"), g("cy"), int(g("mount_link")),
                      (ctypes.c_float * 3)(*g("offset_pos")), (ctypes.c_float * 4)(*g("offset_quat")),
                      g("d_min"), g("d_max"), int(g("downsample", 1)))


def rpl_cameras_set(view: int, cams: Sequence, per_env_intrinsics=None):
    arr = (rpl_camera * len(cams))(*[_camera_struct(c) for c in cams])
    intr = per_env_intrinsics
    if isinstance(intr, np.ndarray):
        intr = np.ascontiguousarray(intr, np.float32)
    _check(lib().rpl_cameras_set(view, arr, len(cams), _ptr(intr)))


def rpl_view_state_size(view: int) -> int:
    n = ctypes.c_int64()
    _check(lib().rpl_view_state_size(view, ctypes.byref(n)))
    return int(n.value)


def rpl_view_state_get(view: int, buf=None):
    """Sensor-state checkpoint into `buf` (numpy uint8 or torch tensor); a new host array when None."""
    n = rpl_view_state_size(view)
    if buf is None:
        buf = np.empty(n, np.uint8)
    nbytes = buf.nbytes if isinstance(buf, np.ndarray) else buf.numel() * buf.element_size()
    _check(lib().rpl_view_state_get(view, _ptr(buf), nbytes))
    return buf


def rpl_view_state_set(view: int, buf):
    nbytes = buf.nbytes if isinstance(buf, np.ndarray) else buf.numel() * buf.element_size()
    _check(lib().rpl_view_state_set(view, _ptr(buf), nbytes))


def rpl_cameras_randomize(view: int, mount_delta=None):
    """mount_delta: None or [E, C, 7] (dp xyz, dq xyzw), numpy or torch (host or device)."""
    if isinstance(mount_delta, np.ndarray):
        mount_delta = np.ascontiguousarray(mount_delta, np.float32)
    _check(lib().rpl_cameras_randomize(view, _ptr(mount_delta)))


def rpl_side_mask_set(view: int, cols=(0, 0, 0), env_mode=None):
    """env_mode: None (off) or [E] uint8 modes 0/1/2; cols: columns masked per side for each mode."""
    if isinstance(env_mode, np.ndarray):
        env_mode = np.ascontiguousarray(env_mode, np.uint8)
    c = (ctypes.c_int32 * 3)(*[int(v) for v in cols])
    _check(lib().rpl_side_mask_set(view, c, _ptr(env_mode)))


def _sensor_struct(s) -> rpl_sensor_params:
    g = (lambda k, d=0: s.get(k, d)) if isinstance(s, dict) else (lambda k, d=0: getattr(s, k, d))
    seed = g("seed", (0, 0))
    return rpl_sensor_params(g("sigma_abs"), g("sigma_rel"), g("p_drop"), g("fill"), int(g("max_latency")),
                             (ctypes.c_uint32 * 2)(int(seed[0]) & 0xFFFFFFFF, int(seed[1]) & 0xFFFFFFFF),
                             int(g("depth_kind")), int(g("out_dtype")))


def rpl_sensor_set(view: int, sensor):
    _check(lib().rpl_sensor_set(view, ctypes.byref(_sensor_struct(sensor))))


def rpl_view_layout(view: int, n_cams: int):
    off = (ctypes.c_int64 * (n_cams + 1))()
    total = ctypes.c_int64()
    _check(lib().rpl_view_layout(view, off, ctypes.byref(total)))
    return list(off), total.value


def rpl_render(view: int, poses, step: int, env_offset: int, out, stream=None):
    _check(lib().rpl_render(view, _ptr(poses), int(step), int(env_offset), _ptr(out), _stream_handle(stream)))


def rpl_sensor_apply(view: int, depth_in, step: int, env_offset: int, out, stream=None):
    _check(lib().rpl_sensor_apply(view, _ptr(depth_in), int(step), int(env_offset), _ptr(out), _stream_handle(stream)))


def rpl_render_counters(view: int, poses, step: int, env_offset: int, out, stream=None) -> dict:
    c = rpl_counters()
    _check(lib().rpl_render_counters(view, _ptr(poses), int(step), int(env_offset), _ptr(out),
                                     _stream_handle(stream), ctypes.byref(c)))
    return {f: int(getattr(c, f)) for f, _ in rpl_counters._fields_}


def rpl_view_reset(view: int, env_mask, step: int, stream=None):
    m = env_mask
    if isinstance(m, np.ndarray):
        m = np.ascontiguousarray(m, np.uint8)
    _check(lib().rpl_view_reset(view, _ptr(m), int(step), _stream_handle(stream)))


def rpl_sync(view: int):
    _check(lib().rpl_sync(view))


def rpl_view_timing(view: int, enable: bool):
    _check(lib().rpl_view_timing(view, int(bool(enable))))


def rpl_view_host_async(view: int, enable: bool):
    _check(lib().rpl_view_host_async(view, int(bool(enable))))


def rpl_view_kernel_ms(view: int, max_n: int = 256):
    buf = (ctypes.c_float * max_n)()
    n = ctypes.c_int32()
    _check(lib().rpl_view_kernel_ms(view, buf, int(max_n), ctypes.byref(n)))
    return [buf[i] for i in range(n.value)]


def rpl_render_static_scratch(scene: int, cams: Sequence, n_envs: int, n_links: int, poses, out, sensor=None,
                              step: int = 0, env_offset: int = 0, stream=None):
    """Render into `out` without allocating (scratch in the library's fixed device array)."""
    arr = (rpl_camera * len(cams))(*[_camera_struct(c) for c in cams])
    sen = None if sensor is None else ctypes.byref(_sensor_struct(sensor))
    _check(lib().rpl_render_static_scratch(scene, arr, len(cams), int(n_envs), int(n_links), _ptr(poses), sen,
                                           int(step), int(env_offset), _ptr(out), _stream_handle(stream)))


def rpl_static_scratch_status(scene: int, stream=None):
    """Waits for `stream`, then raises DEVICE_FAULT if a no-allocation render on the scene's device
    recorded a kernel fault since the last query (the word is cleared by the query)."""
    _check(lib().rpl_static_scratch_status(scene, _stream_handle(stream)))


def rpl_view_tuning_set(view: int, tile_w: int = 4, tile_h: int = 8, persistent: int = 2, terrain_first: int = 0,
                        min_blocks: int = 8, env_order: int = 1, chunk_envs: int = 1):
    t = rpl_tuning(tile_w, tile_h, persistent, terrain_first, min_blocks, env_order, chunk_envs)
    _check(lib().rpl_view_tuning_set(view, ctypes.byref(t)))


def rpl_view_tuning_get(view: int) -> dict:
    t = rpl_tuning()
    _check(lib().rpl_view_tuning_get(view, ctypes.byref(t)))
    return t.as_dict()


def rpl_view_autotune(view: int, poses, step: int, env_offset: int, out, stream=None, reps: int = 3):
    """Times the 192 launch shapes, keeps the fastest on the view; returns (tuning dict, ms per render)."""
    t = rpl_tuning()
    ms = ctypes.c_float()
    _check(lib().rpl_view_autotune(view, _ptr(poses), int(step), int(env_offset), _ptr(out), _stream_handle(stream),
                                   int(reps), ctypes.byref(t), ctypes.byref(ms)))
    return t.as_dict(), float(ms.value)


def rpl_render_graph(view: int, poses, env_offset: int, out, stream=None) -> int:
    """Replays the captured graph of the whole path for the next step; returns that step."""
    s = ctypes.c_int64()
    _check(lib().rpl_render_graph(view, _ptr(poses), int(env_offset), _ptr(out), _stream_handle(stream),
                                  ctypes.byref(s)))
    return int(s.value)


def rpl_view_destroy(view: int):
    lib().rpl_view_destroy(view)


def rpl_scene_destroy(scene: int):
    lib().rpl_scene_destroy(scene)


# --------------------------------------------------------------------------------------------------
# Handle owners
# --------------------------------------------------------------------------------------------------
class Scene:
    """Terrain BVH (built once) plus link BVHs in their own frames."""

    def __init__(self, terrain_verts, terrain_tris, device: int = 0, max_leaf_size: int = 0, build_threads: int = 0,
                 sah_node_cost: float = 0.0, bvh_kind: int = 0):
        self.device = device
        self.h = rpl_scene_create(terrain_verts, terrain_tris, device, max_leaf_size, build_threads, sah_node_cost,
                                  bvh_kind)

    @classmethod
    def from_workload(cls, w, device: int = 0, **kw) -> "Scene":
        s = cls(w.terrain_verts, w.terrain_tris, device, **kw)
        for l, (v, t) in enumerate(zip(w.link_verts, w.link_tris)):
            s.add_link(l, v, t)
        return s

    def add_link(self, link_id: int, verts, tris):
        rpl_link_mesh_add(self.h, link_id, verts, tris)

    def info(self) -> dict:
        return rpl_scene_info_get(self.h)

    def close(self):
        if getattr(self, "h", None):
            rpl_scene_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class View:
    """One trainer's envs: cameras, sensor model, per-env state; renders [E, pixels per env] depth."""

    def __init__(self, scene: Scene, n_envs: int, n_links: int):
        self.scene = scene
        self.n_envs, self.n_links = n_envs, n_links
        self.h = rpl_view_create(scene.h, n_envs, n_links)
        self.cams = []
        self.out_dtype = RPL_OUT_F32

    @classmethod
    def from_workload(cls, scene: Scene, w, n_envs: Optional[int] = None) -> "View":
        v = cls(scene, w.n_envs if n_envs is None else n_envs, w.n_links)
        v.set_cameras(w.cameras, w.per_env_intrinsics)
        if getattr(w, "mount_delta", None) is not None:
            v.randomize_cameras(w.mount_delta)
        if getattr(w, "rsm_modes", None) is not None:
            v.set_side_mask(w.rsm_cols, w.rsm_modes)
        v.set_sensor(w.sensor)
        return v

    def set_cameras(self, cams, per_env_intrinsics=None):
        rpl_cameras_set(self.h, cams, per_env_intrinsics)
        self.cams = list(cams)

    def save_state(self, buf=None):
        """Checkpoint of the sensor state (latency ring, first steps, last step); see rpl_view_state_get."""
        return rpl_view_state_get(self.h, buf)

    def load_state(self, buf):
        rpl_view_state_set(self.h, buf)

    def randomize_cameras(self, mount_delta=None):
        """Per-env camera mount perturbation [E, C, 7] (dp xyz, dq xyzw), or None to clear."""
        rpl_cameras_randomize(self.h, mount_delta)

    def set_side_mask(self, cols=(0, 0, 0), env_mode=None):
        """Random Side Masking: env_mode [E] (0 none, 1 small, 2 large), cols per mode; None = off."""
        rpl_side_mask_set(self.h, cols, env_mode)

    def set_sensor(self, sensor):
        rpl_sensor_set(self.h, sensor)
        self.out_dtype = int(sensor.get("out_dtype", 0) if isinstance(sensor, dict) else getattr(sensor, "out_dtype", 0))

    def layout(self):
        return rpl_view_layout(self.h, len(self.cams))

    def out_tensor(self, device=None):
        import torch
        _, total = self.layout()
        dev = torch.device("cuda", self.scene.device) if device is None else device
        dt = {RPL_OUT_F32: torch.float32, RPL_OUT_F16: torch.float16, RPL_OUT_U16: torch.uint16}[self.out_dtype]
        return torch.empty((self.n_envs, total), dtype=dt, device=dev)

    def render(self, poses, step: int, env_offset: int = 0, out=None, stream=None):
        if out is None:
            out = self.out_tensor(poses.device if hasattr(poses, "device") and poses.device.type == "cuda" else "cpu")
        rpl_render(self.h, poses, step, env_offset, out, stream)
        return out

    def render_counters(self, poses, step: int, env_offset: int = 0, out=None, stream=None) -> dict:
        if out is None:
            out = self.out_tensor()
        return rpl_render_counters(self.h, poses, step, env_offset, out, stream)

    def reset(self, env_mask=None, step: int = 0, stream=None):
        rpl_view_reset(self.h, env_mask, step, stream)

    def sync(self):
        rpl_sync(self.h)

    def close(self):
        if getattr(self, "h", None):
            rpl_view_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------------------------------
# Render server (continuous batching across trainers)
# --------------------------------------------------------------------------------------------------
def rpl_server_create(scene: int, max_batch: int = 0, n_streams: int = 0, staging_bytes: int = 0, min_blocks: int = 0,
                      persistent: int = 0) -> int:
    o = rpl_server_opts(max_batch, n_streams, staging_bytes, min_blocks, persistent)
    h = ctypes.c_void_p()
    _check(lib().rpl_server_create(scene, ctypes.byref(o), ctypes.byref(h)))
    return h.value


def rpl_server_submit(server: int, view: int, poses, step: int, env_offset: int, out) -> int:
    t = ctypes.c_uint64()
    _check(lib().rpl_server_submit(server, view, _ptr(poses), int(step), int(env_offset), _ptr(out), ctypes.byref(t)))
    return int(t.value)


def rpl_server_wait(server: int, ticket: int, timeout_ms: int = -1) -> float:
    """Waits for a request; returns its latency in seconds (raises RplError, TIMEOUT when still pending)."""
    lat = ctypes.c_double()
    _check(lib().rpl_server_wait(server, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(lat)))
    return float(lat.value)


def rpl_server_cancel(server: int, ticket: int):
    _check(lib().rpl_server_cancel(server, ctypes.c_uint64(ticket)))


def rpl_server_stats_get(server: int) -> dict:
    s = rpl_server_stats()
    _check(lib().rpl_server_stats_get(server, ctypes.byref(s)))
    return {f: int(getattr(s, f)) for f, _ in rpl_server_stats._fields_}


def rpl_server_destroy(server: int):
    lib().rpl_server_destroy(server)


class Server:
    """Owner of a render server for views of `scene` (see rpl_server_create)."""

    def __init__(self, scene: Scene, **opts):
        self.scene = scene
        self._held = {}      # ticket -> (view, poses, out): kept alive until the request completes
        self._cancelled = []
        self.h = rpl_server_create(scene.h, **opts)

    def submit(self, view: View, poses, step: int, out, env_offset: int = 0) -> int:
        ticket = rpl_server_submit(self.h, view.h, poses, step, env_offset, out)
        self._held[ticket] = (view, poses, out)
        return ticket

    def wait(self, ticket: int, timeout_ms: int = -1) -> float:
        try:
            dt = rpl_server_wait(self.h, ticket, timeout_ms)
        except RplError as e:
            if e.status != RPL_ERR_TIMEOUT:
                self._held.pop(ticket, None)
            raise
        self._held.pop(ticket, None)
        return dt

    def cancel(self, ticket: int):
        rpl_server_cancel(self.h, ticket)
        held = self._held.pop(ticket, None)
        if held is not None:
            self._cancelled.append(held)   # it may still render: released when the server is closed

    def stats(self) -> dict:
        return rpl_server_stats_get(self.h)

    def close(self):
        if getattr(self, "h", None):
            rpl_server_destroy(self.h)
            self.h = None
        self._held = {}
        self._cancelled = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
