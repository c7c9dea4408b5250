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
//
// Kernel-detected errors (a traversal stack overflow; an index out of range in the bounds-checked
// build) go to a second fixed word, g_static_err, which no render call clears: they stay recorded
// until rpl_static_scratch_status reads and clears them.
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
// Layout per call: link_xf [E*L*3 float4], link_box [E*L*2 float4], cam_xf [E*C*5 float4].
static __device__ __align__(256) unsigned char g_scratch[RPL_STATIC_SCRATCH_BYTES];
// Error bits OR-ed by the render kernels of every call on this device (1: traversal stack
// overflow, 4: index out of range in the bounds-checked build), until read by the status query.
static __device__ int32_t g_static_err;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct Addrs {
    void *scratch = nullptr;   // device address of g_scratch on this device
    int32_t *err = nullptr;    // device address of g_static_err on this device
};
Addrs g_addr[kMaxDevices];     // set on first use of each device

// Looks up the device addresses of g_scratch and g_static_err for the current device `dev` (once per
// device).  The host-side names of these variables are only stand-ins and must never be passed to a
// kernel.
cudaError_t fixed_addresses(int dev, Addrs *out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev].scratch) {
        void *p = nullptr, *q = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        e = cudaGetSymbolAddress(&q, g_static_err);
        if (e != cudaSuccess) return e;
        g_addr[dev].scratch = p;
        g_addr[dev].err = static_cast<int32_t *>(q);
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
    if (((uintptr_t)link_poses & 3) || ((uintptr_t)depth_out & 3))
        return set_error(RPL_ERR_INVALID_ARG, "rpl_render_static_scratch: poses and output must be 4-byte aligned");
    if (env_offset < 0 || env_offset + (int64_t)n_envs > ((int64_t)1 << 32))
        return set_error(RPL_ERR_INVALID_ARG, "rpl_render_static_scratch: env_offset + n_envs beyond 2^32");
    rpl_sensor_params sp{};
    if (sensor) sp = *sensor;
    if (sp.max_latency != 0)
        return set_error(RPL_ERR_INVALID_ARG, "rpl_render_static_scratch: latency needs a view's ring buffer "
                                              "(max_latency must be 0)");
    if (!(sp.p_drop >= 0.f && sp.p_drop <= 1.f) || !(sp.sigma_abs >= 0.f) || !(sp.sigma_rel >= 0.f) ||
        !std::isfinite(sp.sigma_abs) || !std::isfinite(sp.sigma_rel) || !std::isfinite(sp.fill) ||
        (sp.depth_kind != RPL_DEPTH_Z && sp.depth_kind != RPL_DEPTH_RANGE))
        return set_error(RPL_ERR_INVALID_ARG, "rpl_render_static_scratch: bad sensor parameters");

    // scratch layout and the size check
    const size_t EL = (size_t)n_envs * n_links, EC = (size_t)n_envs * n_cams;
    const size_t off_box = EL * 3 * sizeof(float4);
    const size_t off_cam = off_box + EL * 2 * sizeof(float4);
    const size_t need = off_cam + EC * 5 * sizeof(float4);
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
        const rpl_status cst = check_camera(k, c, n_links, "rpl_render_static_scratch");
        if (cst != RPL_OK) return cst;
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
        fastdiv_magic((uint32_t)d.tiles_x, d.tx_m, d.tx_k);
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
        if (pix >= (int64_t)1 << 31)   // pixel offsets inside an env are 32-bit in the kernels
            return set_error(RPL_ERR_CAPACITY, "rpl_render_static_scratch: 2^31 or more pixels per env");
    }
    if (n_envs == 0) return RPL_OK;

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (si.device < 0 || si.device >= kMaxDevices || cudaSetDevice(si.device) != cudaSuccess)
        return set_error(RPL_ERR_CUDA, "rpl_render_static_scratch: cannot select the scene's device");
    rpl_status st = RPL_OK;
    Addrs ad;
    cudaError_t e = fixed_addresses(si.device, &ad);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    unsigned char *sb = static_cast<unsigned char *>(ad.scratch);
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
            if (tiles > 0) fastdiv_magic((uint32_t)tiles, rp.tpe_m, rp.tpe_k);
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
            rp.err = ad.err;
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

extern "C" RPL_API rpl_status rpl_static_scratch_status(rpl_scene_t scene, void *stream) {
    SceneInputs si;
    if (!scene_inputs(scene, &si))
        return set_error(RPL_ERR_INVALID_ARG, "rpl_static_scratch_status: scene is NULL or not frozen");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (si.device < 0 || si.device >= kMaxDevices || cudaSetDevice(si.device) != cudaSuccess)
        return set_error(RPL_ERR_CUDA, "rpl_static_scratch_status: cannot select the scene's device");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    Addrs ad;
    int32_t word = 0;
    static const int32_t zero = 0;
    cudaError_t e = fixed_addresses(si.device, &ad);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&word, ad.err, sizeof word, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e == cudaSuccess && word != 0) {
        e = cudaMemcpyAsync(ad.err, &zero, sizeof zero, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    }
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return set_error(RPL_ERR_CUDA, cudaGetErrorString(e));
    if (word != 0) {
        char msg[200];
        snprintf(msg, sizeof msg, "rpl_render_static_scratch: a render kernel recorded error 0x%x (1: traversal "
                 "stack overflow, 4: node or triangle index out of range)", word);
        return set_error(RPL_ERR_DEVICE_FAULT, msg);
    }
    return RPL_OK;
}
