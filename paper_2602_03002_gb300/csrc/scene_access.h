// scene_access.h -- what entry points outside rpl_api.cpp (the no-allocation render, the render
// server) may use of scenes and views, without depending on their layout.
#pragma once
#include <cuda_runtime.h>

#include "../../include/rpl.h"
#include "render.h"

namespace rpl {

struct SceneInputs {
    int device;
    int bvh_kind;   // rpl_bvh_kind of the terrain BVH
    const float4 *tnodes, *ttris, *lnodes, *ltris, *link_root;
    int64_t n_tnodes, n_ttris, n_lnodes, n_ltris;   // element counts of the four arrays
    int32_t lroot[RPL_MAX_LINKS];
};

// Fills `out` from a scene whose link meshes have been uploaded (frozen by rpl_view_create).
// Returns false for a null or unfrozen scene.
bool scene_inputs(const rpl_scene *s, SceneInputs *out);

// Records the message returned by rpl_last_error() and returns `st`.
rpl_status set_error(rpl_status st, const char *msg);

// Checks camera c of a camera set for n_links links (size, downsample factor, finite intrinsics with
// fx, fy != 0, mount link, finite 0 < d_max >= d_min, finite mount offset, nonzero quaternion);
// on failure records a message naming `who` and returns INVALID_ARG.
rpl_status check_camera(const rpl_camera &k, int c, int32_t n_links, const char *who);

// Views, for the render server (server.cpp).  view_prepare launches the sensor-state reset (when
// due) and the prep kernel on `st` and fills the render parameters; warps = tiles of the request.
rpl_status view_validate(rpl_view *v, const float *poses, int64_t env_offset, void *out);
bool view_step_allowed(const rpl_view *v, int64_t step);
rpl_status view_prepare(rpl_view *v, const float *poses_dev, int64_t step, int64_t env_offset, void *out_dev,
                        cudaStream_t st, RenderParams *rp, int64_t *warps);
// Records that `step` is the view's last rendered step (its work enqueued on `st`).
void view_commit(rpl_view *v, int64_t step, cudaStream_t st);
// Marks the end of the view's enqueued work on `st` (recorded after the render that uses it).
void view_mark_done(rpl_view *v, cudaStream_t st);
size_t view_pose_bytes(const rpl_view *v);
size_t view_out_bytes(const rpl_view *v);
int32_t view_envs(const rpl_view *v);
rpl_scene *view_scene(const rpl_view *v);
Tuning view_tuning(const rpl_view *v);
int scene_device_of(const rpl_scene *s);
int scene_bvh_kind(const rpl_scene *s);
bool pointer_on_device(const void *p, int device);
// A server keeps its scene alive: rpl_scene_destroy is deferred until the last server (and view) goes.
void scene_add_server(rpl_scene *s);
void scene_remove_server(rpl_scene *s);

}  // namespace rpl
