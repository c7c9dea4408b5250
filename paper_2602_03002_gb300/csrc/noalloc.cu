// noalloc.cu -- rpl_render_static_scratch: a render entry point that allocates no memory.
//
// rpl_render keeps its per-call scratch (per-env link transforms and world boxes, per-env camera
// poses) in buffers the view allocates.  Some callers cannot allocate device memory where they
// render: a framework whose caching allocator owns all device memory, a real-time loop in which a
// cudaMalloc (which may synchronise the device) is not acceptable, or code that must not change
// the memory footprint once set up.  This entry point takes the same scene plus the caller's poses
// and output and keeps its scratch in one fixed device array below, so the call itself allocates
// nothing.  It renders the depth of Algorithm 1 with the stateless part of the sensor model
// (noise, clip, dropout; no latency, which needs the per-view ring buffer).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/rpl.h"
#include "render.h"
#include "scene_access.h"

namespace rpl {
namespace {

// Fixed scratch shared by every call, on every GPU that loads the library, until the process exits.
// Layout per call: link_xf [E*L*3 float4], link_box [E*L*2 float4], cam_xf [E*C*5 float4], then
// one int32 error word (rounded up to 16 bytes).
static __device__ __align__(256) unsigned char g_scratch[RPL_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};   // device address of g_scratch per device, set on first use

// Looks up the device address of g_scratch for the current device `dev` (once per device).  The
// host-side name of the array is only a stand-in and must never be passed to a kernel.
cudaError_t scratch_address(int dev, void **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace rpl

using namespace rpl;

extern "C" RPL_API rpl_status rpl_render_static_scratch(rpl_scene_t scene, const rpl_camera *cams, int32_t n_cams,
                                                        int32_t n_envs, int32_t n_links, const float *link_poses,
                                                        const rpl_sensor_params *sensor, int64_t step,
                                                        int64_t env_offset, float *depth_out, void *stream) {
    SceneInputs si;
    if (!scene_inputs(scene, &si))
        return set_error(RPL_ERR_INVALID_ARG, "rpl_render_static_scratch: scene is NULL or not frozen "
                                              "(create a view of it first)");
    if (!cams || n_cams < 1 || n_cams > RPL_MAX_CAMERAS || n_envs < 0 || n_links < 1 || n_links > RPL_MAX_LINKS)
        return set_error(RPL_ERR_INVALID_ARG, "rpl_render_static_scratch: bad camera/env/link count");
    if (n_envs > 0 && (!link_poses || !depth_out))
        return set_error(RPL_ERR_INVALID_ARG, "rpl_render_static_scratch: NULL poses or output");
    if (env_offset < 0 || env_offset + (int64_t)n_envs > ((int64_t)1 << 32))
        return set_error(RPL_ERR_INVALID_ARG, "rpl_render_static_scratch: env_offset + n_envs beyond 2^32");
    rpl_sensor_params sp{};
    if (sensor) sp = *sensor;
    if (sp.max_latency != 0)
        return set_error(RPL_ERR_INVALID_ARG, "rpl_render_static_scratch: latency needs a view's ring buffer "
                                              "(max_latency must be 0)");
    if (!(sp.p_drop >= 0.f && sp.p_drop <= 1.f) || !(sp.sigma_abs >= 0.f) || !(sp.sigma_rel >= 0.f) ||
        (sp.depth_kind != RPL_DEPTH_Z && sp.depth_kind != RPL_DEPTH_RANGE))
        return set_error(RPL_ERR_INVALID_ARG, "rpl_render_static_scratch: bad sensor parameters");

    // scratch layout and the size check
    const size_t EL = (size_t)n_envs * n_links, EC = (size_t)n_envs * n_cams;
    const size_t off_box = EL * 3 * sizeof(float4);
    const size_t off_cam = off_box + EL * 2 * sizeof(float4);
    const size_t off_err = off_cam + EC * 5 * sizeof(float4);
    const size_t need = off_err + 16;
    if (need > (size_t)RPL_STATIC_SCRATCH_BYTES) {
        char msg[256];
        snprintf(msg, sizeof msg, "rpl_render_static_scratch: needs %zu bytes of scratch, the fixed array holds %d "
                 "(80 bytes per env and link plus 80 per env and camera)", need, RPL_STATIC_SCRATCH_BYTES);
        return set_error(RPL_ERR_CAPACITY, msg);
    }

    CamDev cd[RPL_MAX_CAMERAS];
    int32_t tiles = 0;
    int64_t pix = 0;
    for (int c = 0; c < n_cams; ++c) {
        const rpl_camera &k = cams[c];
        if (k.width <= 0 || k.height <= 0 || k.width > 16384 || k.height > 16384 || !(k.fx != 0.f) ||
            !(k.fy != 0.f) || k.mount_link < 0 || k.mount_link >= n_links || !(k.d_min <= k.d_max) ||
            !(k.d_max > 0.f))
            return set_error(RPL_ERR_INVALID_ARG, "rpl_render_static_scratch: bad camera");
        if (k.downsample > 1)
            return set_error(RPL_ERR_INVALID_ARG, "rpl_render_static_scratch: a downsampled camera needs a view's "
                                                  "raw-depth buffer");
        CamDev &d = cd[c];
        d.width = k.width;
        d.height = k.height;
        d.ds = 1;
        d.out_w = k.width;
        d.out_h = k.height;
        d.raw_off = 0;
        d.tiles_x = (k.width + 7) / 8;
        d.tile_off = tiles;
        d.pix_off = (int32_t)pix;
        d.mount = k.mount_link;
        d.fx = k.fx;
        d.fy = k.fy;
        d.cx = k.cx;
        d.cy = k.cy;
        d.d_min = k.d_min;
        d.d_max = k.d_max;
        for (int a = 0; a < 3; ++a) d.off_pos[a] = k.offset_pos[a];
        const double n = std::sqrt((double)k.offset_quat_xyzw[0] * k.offset_quat_xyzw[0] +
                                   (double)k.offset_quat_xyzw[1] * k.offset_quat_xyzw[1] +
                                   (double)k.offset_quat_xyzw[2] * k.offset_quat_xyzw[2] +
                                   (double)k.offset_quat_xyzw[3] * k.offset_quat_xyzw[3]);
        for (int a = 0; a < 4; ++a) d.off_quat[a] = n > 0 ? (float)(k.offset_quat_xyzw[a] / n) : (a == 3 ? 1.f : 0.f);
        tiles += ((k.width + 7) / 8) * ((k.height + 3) / 4);
        pix += (int64_t)k.width * k.height;
    }
    if (n_envs == 0) return RPL_OK;

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (si.device < 0 || si.device >= kMaxDevices || cudaSetDevice(si.device) != cudaSuccess)
        return set_error(RPL_ERR_CUDA, "rpl_render_static_scratch: cannot select the scene's device");
    rpl_status st = RPL_OK;
    void *base = nullptr;
    cudaError_t e = scratch_address(si.device, &base);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    unsigned char *sb = static_cast<unsigned char *>(base);
    if (e == cudaSuccess) e = cudaMemsetAsync(sb + off_err, 0, sizeof(int32_t), cs);   // error word starts at 0
    if (e != cudaSuccess) {
        st = set_error(RPL_ERR_CUDA, cudaGetErrorString(e));
    } else {
        PrepParams pp{};
        pp.poses = link_poses;
        pp.link_root = si.link_root;
        pp.tnodes = si.tnodes;
        pp.bvh_kind = si.bvh_kind;
#ifdef RPL_CHECKED
        pp.n_tnodes = si.n_tnodes;
#endif
        pp.intr = nullptr;
        pp.link_xf = reinterpret_cast<float4 *>(sb);
        pp.link_box = reinterpret_cast<float4 *>(sb + off_box);
        pp.cam_xf = reinterpret_cast<float4 *>(sb + off_cam);
        pp.E = n_envs;
        pp.L = n_links;
        pp.C = n_cams;
        for (int l = 0; l < RPL_MAX_LINKS; ++l) pp.lroot[l] = l < n_links ? si.lroot[l] : -1;
        std::memcpy(pp.cams, cd, sizeof(cd));
        e = launch_prep(pp, cs);
        if (e == cudaSuccess) {
            RenderParams rp{};
            rp.tnodes = si.tnodes;
            rp.ttris = si.ttris;
            rp.bvh_kind = si.bvh_kind;
#ifdef RPL_CHECKED
            rp.n_tnodes = si.n_tnodes;
            rp.n_ttris = si.n_ttris;
            rp.n_lnodes = si.n_lnodes;
            rp.n_ltris = si.n_ltris;
#endif
            rp.out_dtype = RPL_OUT_F32;
            rp.lnodes = si.lnodes;
            rp.ltris = si.ltris;
            rp.link_xf = pp.link_xf;
            rp.link_box = pp.link_box;
            rp.link_root = si.link_root;
            rp.cam_xf = pp.cam_xf;
            rp.intr = nullptr;
            rp.E = n_envs;
            rp.L = n_links;
            rp.C = n_cams;
            rp.tiles_per_env = tiles;
            rp.pix_per_env = (int32_t)pix;
            rp.depth_kind = sp.depth_kind;
            std::memcpy(rp.lroot, pp.lroot, sizeof(rp.lroot));
            std::memcpy(rp.cams, cd, sizeof(cd));
            rp.step = step;
            rp.env_offset = (uint32_t)env_offset;
            rp.span = 1;
            rp.seed0 = sp.seed[0];
            rp.seed1 = sp.seed[1];
            const double thr = std::floor((double)sp.p_drop * 4294967296.0);
            rp.drop_thr = (uint64_t)std::fmin(std::fmax(thr, 0.0), 4294967296.0);
            rp.sigma_abs = sp.sigma_abs;
            rp.sigma_rel = sp.sigma_rel;
            rp.fill = sp.fill;
            rp.sensor_on = (sp.sigma_abs != 0.f || sp.sigma_rel != 0.f || sp.p_drop != 0.f) ? 1 : 0;
            rp.ring = nullptr;
            rp.s_first = nullptr;
            rp.out = depth_out;
            rp.err = reinterpret_cast<int32_t *>(sb + off_err);
            rp.counters = nullptr;
            rp.tile_w_log2 = 3;   // 8x4 tiles, as counted above
            rp.min_blocks = 8;
            e = launch_render(rp, false, cs);
        }
        if (e != cudaSuccess) st = set_error(RPL_ERR_CUDA, cudaGetErrorString(e));
    }
    if (prev >= 0) cudaSetDevice(prev);
    return st;
}
