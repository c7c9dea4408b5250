// render.h -- launch parameters shared by the C-ABI layer (rpl_api.cpp) and the kernels (render.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rpl.h"

namespace rpl {

// Division by a divisor d (1 <= d < 2^31) for dividends n < 2^31 as a multiply and a shift: with
// l = ceil(log2 d), k = 31 + l and m = ceil(2^k / d) (which is below 2^32), floor(n / d) = (n m) >> k,
// since the error term n (m d - 2^k) / (d 2^k) stays below 2^-l <= 1/d (Granlund and Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994).  m = 0 marks an unset divisor.
inline void fastdiv_magic(uint32_t d, uint32_t &m, uint32_t &k) {
    uint32_t l = 0;
    while (l < 31 && (1u << l) < d) ++l;
    k = 31u + l;
    m = (uint32_t)(((1ull << k) + d - 1ull) / d);
}

// One camera as the kernels see it.  width x height is the ray-cast (raw) image, tiled by warps of
// 32 rays; tile_off is the camera's first tile inside one env.  The output image is out_w x out_h
// = raw / ds; pix_off is its first pixel inside one env's output, raw_off (ds > 1 only) the first
// pixel of the raw image inside one env's raw buffer.
struct CamDev {
    int32_t width, height, tiles_x, tile_off;
    uint32_t tx_m, tx_k;   // fastdiv_magic of tiles_x (0 = unset)
    int32_t ds, out_w, out_h, raw_off;
    int32_t pix_off, mount;
    float fx, fy, cx, cy, d_min, d_max;
    float off_pos[3];
    float off_quat[4];   // xyzw, normalised on the host
};

// Per-(env, link) and per-(env, camera) transforms computed once per render by the prep kernel.
//   link_xf  [E*L*3] float4: rows of R^T (world -> link) with the link origin t in .w
//   link_box [E*L*2] float4: world AABB of the link's mesh (lo, hi); far away when the link has none
//   cam_xf   [E*C*5] float4: rows of R_c with the mounting link's origin in .w; the mount offset
//                            rotated into the world (R_l p_off); then (bits of the 64-bit mask of
//                            links inside the camera's view volume, low and high word, bits of the
//                            terrain entry node, bits of the latency word of this step: the delay
//                            s - s' in bits 0..7 and the ring slot s mod span in bits 8..15)
struct PrepParams {
    const float *poses;        // [E, L, 7]
    const float4 *link_root;   // [RPL_MAX_LINKS * 2] link-frame root boxes (lo, hi)
    const float4 *tnodes;      // terrain BVH nodes in the layout of bvh_kind
#ifdef RPL_CHECKED
    int64_t n_tnodes;          // number of terrain nodes (bounds-checked build)
#endif
    int32_t bvh_kind;          // rpl_bvh_kind: binary (bvh.h), eight-wide quantised (bvh8.h), four-wide (bvh4.h)
    const float *intr;         // [E, C, 4] per-env intrinsics or null
    const float *mount_dr;     // [E, C, 7] per-env mount perturbation (dp, dq xyzw) or null
    float4 *link_xf;
    float4 *link_box;
    float4 *cam_xf;
    int32_t E, L, C;
    int32_t lroot[RPL_MAX_LINKS];
    CamDev cams[RPL_MAX_CAMERAS];
    // latency draw (span = max_latency + 1; 0 or 1 = none)
    int64_t step;
    const int64_t *step_dev;   // when set, the step is read from device memory (graph replays)
    const int64_t *s_first;
    uint32_t env_offset, span, seed0, seed1;
    // tile queues of the render kernel's per-SM scheduling (Tuning::persistent == 2), zeroed here;
    // null otherwise
    unsigned long long *queues;
    int32_t n_queues;
    // spatial key of each env for the processing order (Tuning::env_order), or null: the Morton index
    // of link 0's position on a 64 x 64 grid over the terrain's xy extent [xy_lo, xy_hi]
    uint32_t *env_key;
    float xy_lo[2], xy_hi[2];
};

// Number of spatial buckets of the env processing order (64 x 64 cells in Morton order).
constexpr int kOrderBuckets = 4096;

// Launch shape of the render kernel (chosen by the autotuner or set by the caller).
struct Tuning {
    int32_t tile_w_log2;     // tile of 32 rays: width 2^tile_w_log2 (2..4: 4x8, 8x4, 16x2)
    int32_t persistent;      // 0: one warp per tile; 1: grid of resident blocks only, warps stride
                             // over the tiles; 2: grid of resident blocks, tiles split into one
                             // contiguous queue per SM, warps take tiles from their SM's queue and
                             // then from the fullest other queue
    int32_t terrain_first;   // query the terrain before the links
    int32_t min_blocks;      // 8, 9, 10 or 12 blocks of 128 per SM (64, 56, 48 or 40 registers)
    int32_t env_order;       // 1: tiles are processed env by env in the spatial order of the envs
                             // (sorted by position each render), 0: in env index order
    int32_t chunk_envs;      // persistent == 2 only: 0 = one contiguous range of tiles per queue; > 0 =
                             // chunks of the tiles of this many envs dealt to the queues in turn
};

struct RenderParams {
    const float4 *tnodes;   // terrain BVH nodes (4, 5 or 8 float4 each by bvh_kind), root = node 0
    const float4 *ttris;    // terrain triangles (3 float4 each)
    int32_t bvh_kind;       // rpl_bvh_kind of the terrain BVH
    int32_t out_dtype;      // rpl_out_dtype of `out`
    const float4 *lnodes;   // all link BVH nodes
    const float4 *ltris;    // all link triangles
#ifdef RPL_CHECKED
    int64_t n_tnodes, n_ttris, n_lnodes, n_ltris;   // element counts of the four arrays (checked build)
#endif
    const float4 *link_xf;
    const float4 *link_box;
    const float4 *link_root;   // [RPL_MAX_LINKS * 2] link-frame root boxes (lo, hi), for tile prep
    const float4 *cam_xf;
    // [E * tiles_per_env] per tile of 32 rays: (terrain entry node, link mask low word, high word,
    // second terrain entry node or -1), written by the tile-prep kernel; null makes the render kernel
    // derive the entry node and link mask itself
    int4 *tile_info;
    const float *intr;      // [E, C, 4] per-env (fx, fy, cx, cy) or null
    int32_t E, L, C, tiles_per_env;
    uint32_t tpe_m, tpe_k;   // fastdiv_magic of tiles_per_env (0 = unset)
    int32_t pix_per_env, depth_kind;
    int32_t lroot[RPL_MAX_LINKS];   // root node of each link BVH in lnodes, -1 = no mesh
    CamDev cams[RPL_MAX_CAMERAS];
    // launch shape (see Tuning)
    int32_t tile_w_log2, persistent, terrain_first, min_blocks;
    // sensor model
    int64_t step;
    const int64_t *step_dev;        // when set, the step is read from device memory (graph replays)
    uint32_t env_offset, span;      // span = max_latency + 1
    uint32_t seed0, seed1;
    uint64_t drop_thr;              // floor(p_drop 2^32)
    float sigma_abs, sigma_rel, fill;
    int32_t sensor_on;
    float *ring;                    // [E, span, pix_per_env] or null when span == 1
    float *raw;                     // [E, raw_per_env] raw depths of downsampled cameras, or null
    int32_t raw_per_env;
    const uint8_t *rsm_mode;        // [E] side-mask mode per env, or null (masking off)
    int32_t rsm_cols[3];            // columns masked on each side per mode
    const int64_t *s_first;         // [E]
    void *out;                      // [E, pix_per_env] of out_dtype
    int32_t *err;                   // error word (1: traversal stack overflow, 4: index out of range)
    unsigned long long *counters;   // rpl_counters fields, or null
    // per-SM tile queues (persistent == 2): n_queues counters of tiles taken, zeroed by the prep
    // kernel; the tiles are split into n_queues contiguous queues of near-equal size (chunk_envs 0)
    // or dealt to them in chunks of the tiles of chunk_envs envs; null otherwise
    unsigned long long *queues;
    int32_t n_queues, chunk_envs;
    uint32_t chunk_m, chunk_k;   // fastdiv_magic of chunk_envs * tiles_per_env (0 = unset)
    // processing order of the envs ([E] env indices, sorted by position), or null for index order
    const int32_t *env_order;
    // fused launches only (render_multi_kernel): tiles of this request still running, and a word in
    // host-mapped memory set to 1 when the last of them has stored its pixels; null when unused
    int32_t *done_counter;
    int32_t *done_flag;
};

cudaError_t launch_prep(const PrepParams &p, cudaStream_t s);
// Env processing order: order[0..E) = the envs sorted by key[e] (kOrderBuckets buckets; the order
// inside a bucket is arbitrary and does not affect any result).  Runs after launch_prep.
cudaError_t launch_env_order(const uint32_t *key, int32_t *order, int32_t E, cudaStream_t s);
// Per-tile terrain entry nodes and link masks into p.tile_info (no-op when it is null).  Runs after
// launch_prep and before launch_render of the same parameters.
cudaError_t launch_tile_prep(const RenderParams &p, cudaStream_t s);
cudaError_t launch_render(const RenderParams &p, bool count, cudaStream_t s);
// Averages the raw images of downsampled cameras and applies the sensor model to them (no-op when
// p.raw_per_env == 0).  Runs after launch_render of the same parameters.
cudaError_t launch_downsample(const RenderParams &p, cudaStream_t s);
// The sensor model alone on pre-sensor depth src [E, pix_per_env] (device, the output layout).
cudaError_t launch_sensor(const RenderParams &p, const float *src, cudaStream_t s);
cudaError_t launch_set_first(int64_t *s_first, int32_t E, int64_t step, const uint8_t *mask, cudaStream_t s);
cudaError_t launch_advance_step(int64_t *step, cudaStream_t s);
// One launch over several requests: reqs_dev[n_req] parameters in device memory, prefix_dev[n_req + 1]
// the first warp of each request (prefix_dev[n_req] = total_warps).
cudaError_t launch_render_multi(const RenderParams *reqs_dev, const int64_t *prefix_dev, int n_req,
                                int64_t total_warps, int bvh_kind, int min_blocks, bool persistent, cudaStream_t s);

// Depth of the traversal stack; scenes whose BVH is deeper are refused at build time.
constexpr int kStackDepth = 64;

}  // namespace rpl
