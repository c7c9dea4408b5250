/*
 * rpl.h -- C ABI of the GB300 multi-depth ray-casting library (librpl.so).
 *
 * The library renders, for many simulated environments at once, the depth images of several
 * cameras mounted on a robot by casting one ray per pixel against one shared static terrain
 * triangle mesh and against that environment's own posed robot-link meshes, then applies a depth
 * sensor model (latency ring buffer, additive noise, pixel dropout, range clipping).
 * It follows Sec. 3.2.2 ("Efficient Multi-Depth System Simulation") and Algorithm 1 of
 * "RPL: Learning Robust Humanoid Perceptive Locomotion on Challenging Terrains" (arXiv 2602.03002),
 * and the perception rows of its domain-randomisation table (Appendix A.2).
 *
 * Conventions used by every call
 *  - Status: every call returns rpl_status; nothing throws or aborts across the ABI.  The text of
 *    the last failure on the calling thread is available from rpl_last_error().
 *  - Pointers: arguments documented as "host or device" may point to host memory (pageable or
 *    pinned) or to device memory of the scene's GPU; the library detects which.  Everything else
 *    is host memory.
 *  - Ownership: input arrays are copied or only read during the call; the caller keeps them.
 *    Scenes and views own their device memory (BVHs, per-env transforms, ring buffers) and free
 *    it in rpl_*_destroy.  Output buffers belong to the caller.
 *  - Frames: link poses are float32 [E, L, 7] = (px, py, pz, qx, qy, qz, qw) in the world frame;
 *    quaternions need not be normalised (they are normalised in FP32).  Camera mounts map the
 *    OpenCV optical frame (x right, y down, z forward) into the mounting link's frame.
 *  - Concurrency: a scene may be shared by many views and threads once its link meshes are added;
 *    a view is used by one thread at a time.
 */
#ifndef RPL_H
#define RPL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define RPL_API __attribute__((visibility("default")))
#else
#define RPL_API
#endif

typedef enum {
    RPL_OK = 0,
    RPL_ERR_INVALID_ARG = 1,    /* a null handle, bad size, index out of range, step out of order */
    RPL_ERR_OUT_OF_MEMORY = 2,  /* host or device allocation failed */
    RPL_ERR_CUDA = 3,           /* a CUDA runtime call or a kernel launch failed */
    RPL_ERR_NOT_FOUND = 4,      /* no CUDA device with the requested ordinal */
    RPL_ERR_CAPACITY = 5,       /* more cameras/links than the library supports, BVH too deep */
    RPL_ERR_TIMEOUT = 6,        /* reserved for bounded device waits */
    RPL_ERR_DEVICE_FAULT = 7    /* a kernel recorded an error (see rpl_last_error); sticky per view */
} rpl_status;

typedef struct rpl_scene *rpl_scene_t;   /* terrain + link BVHs, read-only once frozen */
typedef struct rpl_view *rpl_view_t;     /* cameras, env count, sensor, per-env state */

#define RPL_MAX_CAMERAS 8
#define RPL_MAX_LINKS 64

/* Terrain acceleration structure.  RPL_BVH2: binary BVH with FP32 child boxes (64-byte nodes).
 * RPL_BVH8Q8: eight-wide BVH whose child boxes are quantised to 8 bits per bound on a per-node
 * power-of-two grid and rounded outward (80-byte nodes); traversal and triangle tests stay FP32,
 * so the depth is the same, only the culling is coarser.  RPL_BVH4: the binary tree collapsed to
 * four children per node with FP32 boxes (128-byte nodes, half the depth, the same triangles);
 * exact like RPL_BVH2.  Link meshes always use RPL_BVH2. */
typedef enum { RPL_BVH2 = 0, RPL_BVH8Q8 = 1, RPL_BVH4 = 2 } rpl_bvh_kind;
typedef enum { RPL_DEPTH_Z = 0, RPL_DEPTH_RANGE = 1 } rpl_depth_kind;
/* Output element type.  F32: float.  F16: IEEE half, round to nearest (max error 1/2 ulp of half:
 * 0.98 mm in [2, 4) m).  U16: unsigned normalised over [0, d_max], q = rint(z / d_max * 65535)
 * clamped to [0, 65535] (step d_max / 65535).  The latency ring buffer always holds FP32. */
typedef enum { RPL_OUT_F32 = 0, RPL_OUT_F16 = 1, RPL_OUT_U16 = 2 } rpl_out_dtype;

/* Scene options.  device: CUDA ordinal; bvh_kind: rpl_bvh_kind; max_leaf_size: triangles per BVH
 * leaf (1..8, 0 = default 4); build_threads: host threads for the BVH build (0 = all cores);
 * sah_node_cost: surface-area-heuristic cost of visiting a node relative to testing a triangle
 * (0 = default 1; larger values give fewer, bigger leaves). */
typedef struct {
    int32_t device;
    int32_t bvh_kind;
    int32_t max_leaf_size;
    int32_t build_threads;
    float sah_node_cost;
} rpl_scene_opts;

/* Pinhole camera.  Pixel (x, y), 0 <= x < width, 0 <= y < height, has the camera-frame ray
 * r = ((x - cx)/fx, (y - cy)/fy, 1) (Sec. 3.2.2: r_c = K^-1 [x, y, 1]^T).  The camera pose is the
 * pose of link `mount_link` composed with (offset_pos, offset_quat_xyzw).  Depths are clipped to
 * [d_min, d_max]; a ray that hits nothing closer than d_max reports d_max (the far plane).
 * downsample f (0 or 1: none; else 2..16 dividing width and height): the camera is ray cast at
 * width x height and its output image is (width/f) x (height/f), each pixel the mean of its f x f
 * block of raw depths (misses count as d_max), taken before the sensor model (Sec. 4.1: raw
 * 240x135 downsampled to 48x27).  The intrinsics are those of the raw image. */
typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    int32_t mount_link;
    float offset_pos[3];
    float offset_quat_xyzw[4];
    float d_min, d_max;
    int32_t downsample;
} rpl_camera;

/* Depth-sensor model (Appendix A.2: process delay, noise, dropout).  For output step s, pixel p
 * of camera c in global env g:
 *   k  = (w0(g, c, 0xFFFFFFFF, s) * (max_latency + 1)) >> 32          latency in steps
 *   s' = max(s - k, first step of the env since its reset)            source step
 *   z  = raw depth of step s' (far plane d_max when nothing is hit)
 *   if z < d_max: z += (sigma_abs + sigma_rel z) sqrt(-2 ln u1) cos(2 pi u2),
 *                 u1 = (w1 + 1) 2^-32, u2 = w2 2^-32                     (Box-Muller)
 *   z = min(max(z, d_min), d_max)
 *   if w0 < floor(p_drop 2^32): z = fill                               dropout
 * where (w0, w1, w2, w3) = Philox4x32-10(counter = (g, c, p, s' mod 2^32),
 * key = (seed[0] ^ (s' >> 32), seed[1])) for the noise and dropout words, and likewise with s for
 * the latency word.  All zeros (the default) turns the model off except for the clip. */
typedef struct {
    float sigma_abs, sigma_rel, p_drop, fill;
    int32_t max_latency;          /* 0..15 */
    uint32_t seed[2];
    int32_t depth_kind;           /* rpl_depth_kind: z-depth along the optical axis (default) or range */
    int32_t out_dtype;            /* rpl_out_dtype */
} rpl_sensor_params;

/* Statistics of a built scene (sizes in bytes on the device). */
typedef struct {
    int64_t terrain_tris, terrain_nodes, terrain_bytes;
    int32_t terrain_depth, n_links;
    int64_t link_tris, link_nodes, link_bytes;
    int32_t link_depth, frozen;
} rpl_scene_info;

/* Traversal counters of one render (see rpl_render_counters). */
typedef struct {
    uint64_t rays;
    uint64_t terrain_nodes, terrain_tris;   /* BVH nodes fetched, triangles tested */
    uint64_t link_boxes, link_nodes, link_tris;
} rpl_counters;

/* ---------------------------------------------------------------------------------------------
 * Scene
 * ------------------------------------------------------------------------------------------- */

/* Build the BVH of the static terrain (world frame) once and upload it (Sec. 3.2.2: the terrain is
 * one shared static mesh).  verts: [n_verts, 3] float32, tris: [n_tris, 3] int32 vertex indices,
 * both host or device.  n_tris may be 0 (nothing but links is hit).  opts may be NULL.
 * Errors: INVALID_ARG (index out of range, negative size), NOT_FOUND, OUT_OF_MEMORY, CUDA. */
RPL_API rpl_status rpl_scene_create(const float *verts, int64_t n_verts, const int32_t *tris,
                                    int64_t n_tris, const rpl_scene_opts *opts, rpl_scene_t *out);

/* Add the mesh of link `link_id` (0 <= link_id < RPL_MAX_LINKS) in its own frame and build its BVH
 * once (Sec. 3.2.2: body meshes stay canonical in their local frames, rays are moved instead, so
 * nothing is refitted per frame).  Links without a mesh are never hit.  verts/tris as in
 * rpl_scene_create, host or device.  Must come before the first rpl_view_create on the scene,
 * which freezes it (INVALID_ARG afterwards). */
RPL_API rpl_status rpl_link_mesh_add(rpl_scene_t scene, int32_t link_id, const float *verts,
                                     int64_t n_verts, const int32_t *tris, int64_t n_tris);

RPL_API rpl_status rpl_scene_info_get(rpl_scene_t scene, rpl_scene_info *info);

/* Host-only BVH build with the same builder the scene uses (no GPU needed), for inspection and tests.
 * Writes the nodes (64-byte records: child-0 box x lo/hi, y lo/hi; child-1 box x lo/hi, y lo/hi;
 * child-0 z lo/hi, child-1 z lo/hi; int32 child0, child1, count0, count1 -- a child >= 0 is an inner
 * node, < 0 a leaf whose first triangle is ~child) and the leaf-ordered triangles (48-byte records:
 * v0 xyz + original index as int32 bits, v1 xyz + 0, v2 xyz + 0).  Call with nodes_out = NULL to
 * learn *n_nodes first; tris_out must hold n_tris records or be NULL.  Errors: INVALID_ARG,
 * CAPACITY (nodes_cap too small), OUT_OF_MEMORY. */
RPL_API rpl_status rpl_bvh_build_host(const float *verts, int64_t n_verts, const int32_t *tris,
                                      int64_t n_tris, int32_t max_leaf, int32_t threads, void *nodes_out,
                                      int64_t nodes_cap, void *tris_out, int64_t *n_nodes, int32_t *depth);

/* The same for the eight-wide quantised BVH (RPL_BVH8Q8): 80-byte nodes in the layout described at
 * rpl_bvh_kind and leaf-ordered triangles; max_leaf 0..4. */
RPL_API rpl_status rpl_bvh8_build_host(const float *verts, int64_t n_verts, const int32_t *tris,
                                       int64_t n_tris, int32_t max_leaf, int32_t threads, void *nodes_out,
                                       int64_t nodes_cap, void *tris_out, int64_t *n_nodes, int32_t *depth);

/* Frees the scene's device memory.  While views or servers of the scene still exist the scene
 * stays alive and is freed when the last of them is destroyed (so destruction order, e.g. in a
 * garbage-collected binding, never matters); it must not be used for new views meanwhile. */
RPL_API void rpl_scene_destroy(rpl_scene_t scene);

/* ---------------------------------------------------------------------------------------------
 * View: one trainer's environments
 * ------------------------------------------------------------------------------------------- */

/* A view of n_envs environments with n_links links each (poses are [n_envs, n_links, 7]).
 * Freezes the scene.  n_envs may be 0.  Errors: INVALID_ARG, CAPACITY (n_links > RPL_MAX_LINKS),
 * OUT_OF_MEMORY, CUDA. */
RPL_API rpl_status rpl_view_create(rpl_scene_t scene, int32_t n_envs, int32_t n_links, rpl_view_t *out);

/* Set the cameras (1..RPL_MAX_CAMERAS; they may differ in size).  per_env_intrinsics, host or
 * device, is NULL or [n_envs, n_cams, 4] float32 (fx, fy, cx, cy) overriding each camera's
 * intrinsics per env (Sec. 3.2.2: batched inverse intrinsics for per-env FOV randomisation).
 * Allocates the raw-depth buffer of downsampled cameras ([n_envs, raw pixels per env] float32)
 * and clears the mount randomisation.  Restarts the sensor state (as rpl_view_reset with no
 * mask).  Errors: INVALID_ARG (size <= 0, fx or fy == 0, mount_link out of range, d_min > d_max,
 * a downsample factor outside 0..16 or not dividing the size), CAPACITY, OUT_OF_MEMORY. */
RPL_API rpl_status rpl_cameras_set(rpl_view_t view, const rpl_camera *cams, int32_t n_cams,
                                   const float *per_env_intrinsics);

/* Per-env camera mount randomisation (Appendix A.2, perception rows: camera translation and
 * rotation).  mount_delta, host or device, is [n_envs, n_cams, 7] float32 (dp_x, dp_y, dp_z, dq_x,
 * dq_y, dq_z, dq_w): camera c of env e is mounted at offset_pos + dp (link frame) with rotation
 * R(offset_quat) R(dq), i.e. dq turns the camera about its own axes; dq is normalised.  The values
 * are copied (call again to re-draw them, e.g. at episode resets); NULL restores the plain mounts.
 * FOV randomisation is the per-env intrinsics of rpl_cameras_set.  Call after rpl_cameras_set
 * (which clears them).  Does not restart the sensor state.  Errors: INVALID_ARG (no cameras set,
 * a zero or non-finite quaternion), OUT_OF_MEMORY, CUDA. */
RPL_API rpl_status rpl_cameras_randomize(rpl_view_t view, const float *mount_delta);

/* Random Side Masking (Sec. 3.2.4).  env_mode, host or device, is NULL (masking off) or [n_envs]
 * uint8: 0 none, 1 small, 2 large (larger values count as 2); cols[m] is the number of output
 * columns masked on each side of every image of an env in mode m (0 <= cols[m], 2 cols[m] may
 * cover the whole width).  A masked pixel of camera c in global env g at step s is replaced, after
 * the rest of the sensor model, by d_min + (d_max - d_min) (w3(g, c, p, s) + 1/2) 2^-32, a uniform
 * value in [d_min, d_max] keyed by the current step (not the latency's source step).  The modes are
 * copied; call again when they change.  Errors: INVALID_ARG (negative cols, cols NULL with env_mode
 * set), OUT_OF_MEMORY, CUDA. */
RPL_API rpl_status rpl_side_mask_set(rpl_view_t view, const int32_t cols[3], const uint8_t *env_mode);

/* Set the sensor model (see rpl_sensor_params).  Allocates the latency ring buffer,
 * [n_envs, max_latency + 1, pixels per env] float32, and restarts the sensor state.
 * Errors: INVALID_ARG (max_latency outside 0..15, p_drop outside [0, 1], negative sigma),
 * OUT_OF_MEMORY. */
RPL_API rpl_status rpl_sensor_set(rpl_view_t view, const rpl_sensor_params *params);

/* Layout of one render's output: env-major, cameras packed per env, row-major pixels; camera c
 * of env e starts at e * total_per_env + cam_offsets[c].  cam_offsets has room for n_cams + 1
 * entries (the last one is total_per_env); either pointer may be NULL. */
RPL_API rpl_status rpl_view_layout(rpl_view_t view, int64_t *cam_offsets, int64_t *total_per_env);

/* Render step `step` (Algorithm 1 plus the sensor model).
 *   link_poses  host or device, [n_envs, n_links, 7] float32 (see conventions)
 *   step        render-step counter: the first call after rpl_view_create / rpl_cameras_set /
 *               rpl_sensor_set / a full rpl_view_reset may use any value; afterwards each call
 *               uses the previous step (re-render) or the previous step + 1 (INVALID_ARG else)
 *   env_offset  global id of env 0 of this view (keys the random streams, so that a range of envs
 *               rendered by another GPU or process draws the same numbers); env_offset + n_envs
 *               must not exceed 2^32
 *   depth_out   host or device, n_envs * total_per_env elements of the view's output type
 *               (float32, or 16-bit for RPL_OUT_F16 / RPL_OUT_U16; see rpl_view_layout)
 *   stream      cudaStream_t to run on (NULL = the legacy default stream)
 * With device buffers the call only enqueues work and returns; it does not allocate or
 * synchronise, so it can be captured into a CUDA graph (a captured graph replays the step it was
 * captured with).  Host buffers are staged through view-owned device memory (allocated on the
 * first such call): with a host depth_out the call returns after the depth is in depth_out; with
 * host poses and a device depth_out it returns after enqueuing, and pinned host poses are read
 * asynchronously, so they must stay unchanged until the stream has passed this render.
 * Errors: INVALID_ARG, CUDA, DEVICE_FAULT (an earlier launch on this view recorded a kernel
 * error; call rpl_sync to read it and clear it). */
RPL_API rpl_status rpl_render(rpl_view_t view, const float *link_poses, int64_t step,
                              int64_t env_offset, void *depth_out, void *stream);

/* The sensor model alone (Appendix A.2; Sec. 3.2.4 side mask) on caller-provided pre-sensor depth:
 * depth_in, device, [n_envs, total_per_env] float32 in the view's output layout (rpl_view_layout),
 * is taken as the raw depth of `step` (what the ray cast would give: the closest hit's z-depth, or
 * d_max for a miss) and goes through the same ring buffer, latency, noise, clip, dropout and side
 * mask as rpl_render, with the same step rules, into depth_out (device, the view's output type).
 * For depth from another renderer, and to test the sensor model without ray casting.  Views with
 * downsampled cameras are refused.  Asynchronous on `stream`.  Errors: INVALID_ARG, CUDA,
 * DEVICE_FAULT. */
RPL_API rpl_status rpl_sensor_apply(rpl_view_t view, const float *depth_in, int64_t step, int64_t env_offset,
                                    void *depth_out, void *stream);

/* Asynchronous host output.  When enabled, rpl_render with a host depth_out returns after
 * enqueuing: the depth is staged in one of two view-owned device buffers (used in turn) and copied
 * to depth_out on a view-owned stream, overlapped with the next render; depth_out holds the result
 * after rpl_sync (which waits for the copy), and must be pinned memory for the copy to overlap.
 * Disabling waits for the view's work.  Errors: INVALID_ARG, CUDA. */
RPL_API rpl_status rpl_view_host_async(rpl_view_t view, int32_t enable);

/* Launch shape of the render kernel.  tile_w x tile_h = 32 rays per warp (4x8, 8x4 or 16x2
 * pixels of one camera); persistent: 0 = one warp per tile; 1 = launch only as many blocks as fit
 * on the GPU at once and let warps stride over the tiles; 2 = as many blocks, the tiles split into
 * one contiguous queue per SM from which the SM's warps take tiles one at a time (then from the
 * fullest other queue), so an SM works on neighbouring tiles and no warp waits for the rest of its
 * block (a view renders on one stream at a time: its queue counters are shared by its renders);
 * terrain_first: query the terrain before the links (Alg. 1 queries
 * the bodies first; the depth is the same either way); min_blocks: 8 (up to 64 registers per
 * thread), 9 (up to 56), 10 (up to 48) or 12 (up to 40) resident blocks of 128 threads per SM.  The
 * shape never changes the result, only the speed.  Default: 4x8, persistent 2 (per-SM queues), links
 * first, 8, env_order 1, chunk_envs 1. */
typedef struct {
    int32_t tile_w, tile_h;
    int32_t persistent;
    int32_t terrain_first;
    int32_t min_blocks;
    int32_t env_order;     /* 1: render the envs in the order of their positions (link 0's position on a
                              64 x 64 grid over the terrain, sorted on the GPU each render), so that
                              tiles in flight together share terrain in L2; 0: in env index order */
    int32_t chunk_envs;    /* persistent 2 only: 0 = one contiguous range of tiles per SM queue; > 0 =
                              the tiles dealt to the queues in chunks of this many envs (up to 2^20) */
} rpl_tuning;

RPL_API rpl_status rpl_view_tuning_set(rpl_view_t view, const rpl_tuning *tuning);
RPL_API rpl_status rpl_view_tuning_get(rpl_view_t view, rpl_tuning *tuning);

/* Autotuner: renders `step` (same step rules as rpl_render; device buffers only) `reps` times
 * with each of 192 launch shapes (tile 8x4 / 4x8 / 16x2; persistent 0 / 1 / 2, each in env index
 * or spatial order, the per-SM queues contiguous or dealt one env at a time; links or terrain
 * first; 8, 9, 10 or 12 blocks per SM), times them with CUDA events on `stream`, keeps the fastest on the
 * view and returns it with its mean time per render.  Synchronises; for setup, not the hot loop. */
RPL_API rpl_status rpl_view_autotune(rpl_view_t view, const float *link_poses, int64_t step,
                                     int64_t env_offset, void *depth_out, void *stream, int32_t reps,
                                     rpl_tuning *best, float *best_ms);

/* Render the next step by replaying a CUDA graph of the whole path (Sec. 3.2.2: the pipeline is
 * captured into a CUDA graph for low-overhead replay).  The first call, and any call after the
 * buffers, env_offset, cameras, sensor or tuning changed, captures prep + tile prep + render + a
 * step-advance kernel into a graph (on a view-owned stream) and instantiates it; every call then launches it on
 * `stream`.  The kernels read the step from a view-owned device counter that the graph advances,
 * so replays continue the sensor history: the step rendered is the previous step + 1 (0 for a new
 * view, or the step given to a full rpl_view_reset) and is returned in *step_out (may be NULL).
 * link_poses and depth_out must be device memory; their contents are read/written at replay
 * time.  Mixing with rpl_render is allowed (the counter is resynchronised with a tiny kernel).
 * Errors: INVALID_ARG, CUDA, DEVICE_FAULT. */
RPL_API rpl_status rpl_render_graph(rpl_view_t view, const float *link_poses, int64_t env_offset,
                                    void *depth_out, void *stream, int64_t *step_out);

/* ---------------------------------------------------------------------------------------------
 * Render server: continuous batching of requests from many trainers (not part of the paper's
 * method; it serves the renderer to several training processes or threads at once).
 * ------------------------------------------------------------------------------------------- */
typedef struct rpl_server *rpl_server_t;

/* max_batch: requests fused into one render launch (1..64, 0 = 32); n_streams: batches that may be
 * on the GPU at once (1..8, 0 = 2); staging_bytes: device memory budget for the pose and depth
 * staging of requests made with host buffers (0 = 256 MiB) -- a request is admitted only when its
 * staging fits; min_blocks, persistent: launch shape of the fused launch (see rpl_tuning; 0 = 8,
 * not persistent). */
typedef struct {
    int32_t max_batch;
    int32_t n_streams;
    int64_t staging_bytes;
    int32_t min_blocks;
    int32_t persistent;
} rpl_server_opts;

typedef struct {
    uint64_t submitted, completed, failed, cancelled, batches, fused_requests;
    int64_t staging_peak_bytes;
    int32_t max_batch_seen, max_inflight_batches_seen;
} rpl_server_stats;

/* A server for views of `scene`, with a worker thread that, while requests are waiting, admits them
 * in arrival order as stream slots and staging memory free up (at most one request per view on the
 * GPU at a time, since a view's ring buffer and scratch are stateful), fuses the admitted ones into
 * one launch (a prep and a tile-prep launch per request, one render launch over the tiles of all
 * of them) on a
 * free stream, and completes them when that launch's event has passed; batches on different
 * streams overlap on the device.  A request's result is the same as rpl_render of the same view
 * and step alone.  The scene must be frozen (a view created).  Errors: INVALID_ARG, CUDA,
 * OUT_OF_MEMORY. */
RPL_API rpl_status rpl_server_create(rpl_scene_t scene, const rpl_server_opts *opts, rpl_server_t *out);

/* Queue a render of `view` at `step` (the view's previous submitted step or that + 1, or any step
 * for its first request) into depth_out; link_poses and depth_out are host (staged through the
 * server's budget) or device memory; they and the view must stay valid (not destroyed) until the
 * request completes: rpl_server_wait returned for it, or, for a cancelled request, the server was
 * destroyed.  While a view has requests in a server it must not be rendered by other calls.  The
 * request runs after all work queued on the legacy default stream (cudaStreamLegacy, PyTorch's
 * default stream) before this call: the server records an event there and its launch waits for it.
 * Work on other streams that writes the poses or still uses depth_out's memory must be finished (or
 * ordered before that stream point) by the caller.  *ticket identifies the request.  Errors:
 * INVALID_ARG, CAPACITY (the request's staging exceeds the whole budget), CUDA (the event could not
 * be recorded, e.g. during a global-mode stream capture). */
RPL_API rpl_status rpl_server_submit(rpl_server_t server, rpl_view_t view, const float *link_poses, int64_t step,
                                     int64_t env_offset, void *depth_out, uint64_t *ticket);

/* Wait up to timeout_ms (< 0: forever) for a request; on completion returns its status, sets
 * *latency_s (submit to completion, host clock; may be NULL) and forgets the ticket.  Returns
 * RPL_ERR_TIMEOUT when it is still pending (the ticket stays valid), INVALID_ARG for an unknown
 * ticket, for a ticket another thread is already waiting on, or when another thread cancels the
 * request during the wait. */
RPL_API rpl_status rpl_server_wait(rpl_server_t server, uint64_t ticket, int32_t timeout_ms, double *latency_s);

/* Give up on a request: it still renders (so the view's step sequence stays whole) and is forgotten
 * when it completes; waiting on the ticket afterwards returns INVALID_ARG.  For callers that stop
 * waiting, e.g. a trainer that is shutting down. */
RPL_API rpl_status rpl_server_cancel(rpl_server_t server, uint64_t ticket);

RPL_API rpl_status rpl_server_stats_get(rpl_server_t server, rpl_server_stats *stats);

/* Stops admitting, waits for the batches on the GPU, fails requests still queued, frees. */
RPL_API void rpl_server_destroy(rpl_server_t server);

/* Restart the sensor history at `step` for the envs whose byte in env_mask (host or device,
 * [n_envs] uint8) is non-zero, or for all envs when env_mask is NULL: from then on the source step
 * of those envs is never older than `step`.  With a mask, `step` must be the next step to render
 * (last rendered step + 1); with no mask the next render must use `step`.  Asynchronous on
 * `stream`.  Errors: INVALID_ARG, CUDA. */
RPL_API rpl_status rpl_view_reset(rpl_view_t view, const uint8_t *env_mask, int64_t step, void *stream);

/* Checkpoint of the sensor state, so that a trainer resumes bit-exact (the paper does not describe
 * checkpointing; this serves callers of the library).  The state is the last rendered step, each
 * env's first step since its reset, and the latency ring ([n_envs, max_latency + 1, pixels per
 * env] float32, absent when max_latency is 0): a 64-byte header (magic "RPLS", version, n_envs,
 * pixels per env, ring span, flags, last step), then n_envs int64 first steps, then the ring.
 * rpl_view_state_size gives the byte count; rpl_view_state_get waits for the view's work and
 * copies the state into buf (host or device, `bytes` >= the size); rpl_view_state_set loads it
 * into a view with the same n_envs, pixels per env and max_latency (cameras, sensor and mounts
 * are configuration, set by their own calls), after which rendering continues from the saved step.
 * Errors: INVALID_ARG (NULL, too small, a header that does not match the view), CUDA. */
RPL_API rpl_status rpl_view_state_size(rpl_view_t view, int64_t *bytes);
RPL_API rpl_status rpl_view_state_get(rpl_view_t view, void *buf, int64_t bytes);
RPL_API rpl_status rpl_view_state_set(rpl_view_t view, const void *buf, int64_t bytes);

/* Wait until the view's most recently enqueued work (render, reset, graph replay or a server's
 * batch) has finished, on whichever stream it went (the stream may since have been destroyed),
 * then report and clear a recorded kernel error (DEVICE_FAULT), or a CUDA error. */
RPL_API rpl_status rpl_sync(rpl_view_t view);

/* Render like rpl_render (device buffers only) with the counting kernel variant, synchronise, and
 * return how many BVH nodes and triangles the traversal touched.  Does not advance the sensor
 * state check (it re-renders `step`).  For measurement only. */
RPL_API rpl_status rpl_render_counters(rpl_view_t view, const float *link_poses, int64_t step,
                                       int64_t env_offset, void *depth_out, void *stream,
                                       rpl_counters *counters);

/* Measurement aid: when enabled, each following render records a CUDA event pair on its stream
 * around the traversal kernel (a ring of the last 256 launches).  rpl_view_kernel_ms waits for and
 * returns the durations in milliseconds of the last min(max_n, recorded) launches, oldest first. */
RPL_API rpl_status rpl_view_timing(rpl_view_t view, int32_t enable);
RPL_API rpl_status rpl_view_kernel_ms(rpl_view_t view, float *ms, int32_t max_n, int32_t *n_out);

RPL_API void rpl_view_destroy(rpl_view_t view);

/* ---------------------------------------------------------------------------------------------
 * Rendering without allocating (the paper has no counterpart: this serves callers of the library)
 * ------------------------------------------------------------------------------------------- */

/* Size of the library's fixed device scratch array used by rpl_render_static_scratch. */
#define RPL_STATIC_SCRATCH_BYTES (8 << 20)

/* Render like rpl_render, but without allocating anything, for callers that cannot call cudaMalloc
 * where they render: for example code running under a framework whose caching allocator owns the
 * device memory, or a real-time loop where an allocation (which may synchronise the device) is not
 * acceptable.  The per-call scratch (per-env link transforms and boxes, per-env camera poses) lives
 * in one fixed __device__ array of RPL_STATIC_SCRATCH_BYTES inside the library, which every GPU
 * that loads the library keeps until the process exits; a call needs
 * 80 * n_envs * (n_links + n_cams) bytes of it and returns CAPACITY when that exceeds the array
 * (about 3,270 envs with 30 links and 2 cameras).
 *   scene       a frozen scene (rpl_view_create has been called on it once), read only
 *   cams        host array of n_cams cameras (1..RPL_MAX_CAMERAS), as for rpl_cameras_set
 *   link_poses  device, [n_envs, n_links, 7] float32, 4-byte aligned
 *   sensor      NULL (clip only) or a sensor with max_latency == 0: noise, clip and dropout are
 *               applied, keyed by (env_offset + env, camera, pixel, step); latency needs a view
 *   depth_out   device, n_envs * (sum of camera pixels) float32, cameras packed per env, 4-byte
 *               aligned
 *   stream      cudaStream_t (NULL = legacy default stream)
 * The first call on a device looks up the device addresses of the array and of a fixed error word
 * (cudaGetSymbolAddress) with that device current; make that first call before any stream capture.
 * Every call shares the array and it keeps the last call's contents: each call rewrites all of it
 * that it reads, but calls whose work overlaps on the GPU (other streams, other threads) race on it
 * and must be serialised by the caller.  The call only enqueues work.  A fault the kernels detect
 * (traversal stack overflow; index out of range in the bounds-checked build) is not returned by
 * this call: it is OR-ed into the fixed error word, which keeps it until rpl_static_scratch_status
 * reports it.
 * Errors: INVALID_ARG (unfrozen scene, bad counts, cameras or sensor, max_latency != 0, a camera
 * with downsample > 1, whose raw image needs a view's buffer, unaligned buffers), CAPACITY (scratch
 * beyond the array, 2^31 or more pixels per env), CUDA. */
RPL_API rpl_status rpl_render_static_scratch(rpl_scene_t scene, const rpl_camera *cams, int32_t n_cams,
                                             int32_t n_envs, int32_t n_links, const float *link_poses,
                                             const rpl_sensor_params *sensor, int64_t step,
                                             int64_t env_offset, float *depth_out, void *stream);

/* Reports the kernel-detected faults of rpl_render_static_scratch calls on the scene's device: waits
 * for `stream` (so give the stream the renders ran on, or synchronise first), reads the fixed error
 * word, clears it and returns DEVICE_FAULT when it was set (bit 1: traversal stack overflow, bit 4:
 * node or triangle index out of range, bounds-checked build only), else OK.  The word collects the
 * faults of every call since the last query.  Like the render call it allocates nothing.
 * Errors: INVALID_ARG (unfrozen scene), CUDA, DEVICE_FAULT. */
RPL_API rpl_status rpl_static_scratch_status(rpl_scene_t scene, void *stream);

/* Message of the last failed call on this thread ("" if none). */
RPL_API const char *rpl_last_error(void);

/* Library version, for the Python binding's compatibility check. */
RPL_API int32_t rpl_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RPL_H */
