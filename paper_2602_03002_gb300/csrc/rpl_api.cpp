// rpl_api.cpp -- the C ABI (include/rpl.h): scenes, views, argument checks, device memory,
// host/device pointer handling and kernel launches.  No torch types cross this boundary.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/rpl.h"
#include "bvh.h"
#include "bvh4.h"
#include "bvh8.h"
#include "render.h"
#include "scene_access.h"

using namespace rpl;

namespace {

thread_local std::string g_err;

rpl_status fail(rpl_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

rpl_status cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? RPL_ERR_OUT_OF_MEMORY : RPL_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

// An NVTX range around one library call, so profiler timelines show the calls (free when no tool
// is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Makes `dev` current for the lifetime of the guard and restores the caller's device after.
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        err = cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t alloc(size_t n) {
        release();
        if (n == 0) n = 16;
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        bytes = n;
        return cudaSuccess;
    }
    template <class T>
    T *as() const {
        return reinterpret_cast<T *>(p);
    }
};

enum PtrKind { PTR_HOST, PTR_DEVICE, PTR_OTHER_DEVICE };

PtrKind pointer_kind(const void *ptr, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return PTR_HOST;
    }
    if (a.type == cudaMemoryTypeDevice) return a.device == device ? PTR_DEVICE : PTR_OTHER_DEVICE;
    if (a.type == cudaMemoryTypeManaged) return PTR_DEVICE;
    return PTR_HOST;
}

// Copies a host-or-device array to host memory.
rpl_status to_host(const void *src, size_t bytes, int device, std::vector<char> &dst) {
    dst.resize(bytes);
    if (bytes == 0) return RPL_OK;
    PtrKind k = pointer_kind(src, device);
    if (k == PTR_HOST) {
        std::memcpy(dst.data(), src, bytes);
        return RPL_OK;
    }
    cudaError_t e = cudaMemcpy(dst.data(), src, bytes, cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_fail(e, "copying an input array to the host");
    return RPL_OK;
}

// The binary layout as the kernels read it: a leaf child carries its final reference
// ~((first << 3) | (count - 1)) and an empty child a zero-size box at 1e30, which no ray with a
// finite bound meets, so the traversal decodes nothing per child.  (The host layout, which the
// collapses and rpl_bvh_build_host use, keeps ~first and the count.)
void encode_for_device(std::vector<BvhNode> &nodes) {
    for (BvhNode &n : nodes) {
        if (n.child0 < 0) {
            if (n.cnt0 == 0) {
                n.c0lox = n.c0hix = n.c0loy = n.c0hiy = n.c0loz = n.c0hiz = 1e30f;
                n.child0 = -1;
            } else {
                n.child0 = ~((~n.child0 << 3) | (n.cnt0 - 1));
            }
        }
        if (n.child1 < 0) {
            if (n.cnt1 == 0) {
                n.c1lox = n.c1hix = n.c1loy = n.c1hiy = n.c1loz = n.c1hiz = 1e30f;
                n.child1 = -1;
            } else {
                n.child1 = ~((~n.child1 << 3) | (n.cnt1 - 1));
            }
        }
    }
}

// Two-triangle leaves whose triangles share an edge (a grid cell split along its diagonal, a quad
// face of a link mesh) are stored so that the first triangle is (A, B, C) and the second (A, C, D),
// each a cyclic rotation of its input triangle (so its orientation is kept), and the first
// triangle's v1.w (otherwise 0) is set to 1.  The binary traversal then tests the pair from four
// vertices (the shared edge's function is the first triangle's negated, exactly); every other
// reader tests the rotated triangles one by one.  nodes: host layout (leaf child ~first, count).
// Returns the number of pairs.
int64_t pair_quad_leaves(const std::vector<BvhNode> &nodes, std::vector<BvhTri> &tris) {
    auto vert = [](const BvhTri &t, int k, float out[3]) {
        const float *p = &t.v0x + 4 * k;
        out[0] = p[0];
        out[1] = p[1];
        out[2] = p[2];
    };
    auto same = [](const float a[3], const float b[3]) { return a[0] == b[0] && a[1] == b[1] && a[2] == b[2]; };
    auto put = [](BvhTri &t, int k, const float v[3]) {
        float *p = &t.v0x + 4 * k;
        p[0] = v[0];
        p[1] = v[1];
        p[2] = v[2];
    };
    int64_t pairs = 0;
    for (const BvhNode &n : nodes) {
        const int32_t ch[2] = {n.child0, n.child1}, cn[2] = {n.cnt0, n.cnt1};
        for (int k = 0; k < 2; ++k) {
            if (ch[k] >= 0 || cn[k] != 2) continue;
            const int64_t first = ~(int64_t)ch[k];
            if (first < 0 || first + 1 >= (int64_t)tris.size()) continue;
            BvhTri &t0 = tris[(size_t)first], &t1 = tris[(size_t)first + 1];
            float p[3][3], q[3][3];
            for (int i = 0; i < 3; ++i) {
                vert(t0, i, p[i]);
                vert(t1, i, q[i]);
            }
            // the vertex of each triangle that the other does not have
            int u = -1, w = -1, shared = 0;
            for (int i = 0; i < 3; ++i) {
                bool in_q = false, in_p = false;
                for (int j = 0; j < 3; ++j) {
                    in_q |= same(p[i], q[j]);
                    in_p |= same(q[i], p[j]);
                }
                if (in_q) ++shared;
                else u = i;
                if (!in_p) w = i;
            }
            if (shared != 2 || u < 0 || w < 0) continue;
            // first triangle: (A, B, C) with B its own vertex; second: (A, C, D) with D its own vertex
            const int s0 = (u + 2) % 3, s1 = (w + 1) % 3;
            float A[3], B[3], C[3], A1[3], C1[3], D[3];
            for (int a = 0; a < 3; ++a) {
                A[a] = p[s0][a];
                B[a] = p[(s0 + 1) % 3][a];
                C[a] = p[(s0 + 2) % 3][a];
                A1[a] = q[s1][a];
                C1[a] = q[(s1 + 1) % 3][a];
                D[a] = q[(s1 + 2) % 3][a];
            }
            if (!same(A, A1) || !same(C, C1)) continue;   // the two are not oriented alike
            put(t0, 0, A);
            put(t0, 1, B);
            put(t0, 2, C);
            put(t1, 0, A1);
            put(t1, 1, C1);
            put(t1, 2, D);
            t0.pad1 = 1.0f;
            t1.pad1 = 0.0f;
            ++pairs;
        }
    }
    return pairs;
}

void quat_normalise(const float in[4], float out[4]) {
    double n = std::sqrt((double)in[0] * in[0] + (double)in[1] * in[1] + (double)in[2] * in[2] +
                         (double)in[3] * in[3]);
    for (int k = 0; k < 4; ++k) out[k] = n > 0 ? (float)(in[k] / n) : (k == 3 ? 1.f : 0.f);
}

}  // namespace

struct rpl_scene {
    int device = 0;
    rpl_scene_opts opts{};
    DevBuf t_nodes, t_tris;
    int64_t t_n_nodes = 0, t_n_tris = 0;
    int32_t t_depth = 0;
    std::vector<HostBvh> links;      // indexed by link id
    std::vector<bool> has_link;
    DevBuf l_nodes, l_tris, l_roots;
    float xy_lo[2] = {0.f, 0.f}, xy_hi[2] = {1.f, 1.f};   // xy extent of the terrain's vertices
    int32_t l_root[RPL_MAX_LINKS];
    int64_t l_n_nodes = 0, l_n_tris = 0;
    int32_t l_depth = 0;
    bool frozen = false;
    int views = 0;                  // views and servers still using the scene
    int servers = 0;
    bool destroy_pending = false;   // rpl_scene_destroy came while they existed
    std::mutex mu;
};

struct rpl_view {
    rpl_scene *scene = nullptr;
    int32_t E = 0, L = 0, C = 0;
    rpl_camera cams[RPL_MAX_CAMERAS];
    int64_t cam_off[RPL_MAX_CAMERAS + 1];
    int32_t tile_off[RPL_MAX_CAMERAS + 1];
    int64_t P = 0;
    bool cams_set = false;
    rpl_sensor_params sensor{};
    DevBuf link_xf, link_box, cam_xf, intr, ring, s_first, mask_stage, pose_stage, out_stage;
    // asynchronous host output (rpl_view_host_async): a second staging buffer, the copy stream and
    // per-buffer events (render finished writing / copy finished reading)
    bool host_async = false;
    DevBuf out_stage2;
    int stage_next = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t rendered[2] = {}, copied[2] = {};
    // downsampled cameras: raw depths [E, raw_per_env]; camera c's raw image starts at raw_off[c]
    DevBuf raw;
    int64_t raw_per_env = 0;
    // per-tile terrain entry node and link mask [E, tiles per env] int4, sized for the tile shape
    // with the most tiles
    DevBuf tile_info;
    // per-SM tile queues of the render kernel (launch shape persistent == 2): one counter per SM
    DevBuf queues;
    int32_t n_queues = 0;
    // spatial processing order of the envs (launch shape env_order == 1): key and order [E]
    DevBuf env_key, env_order;
    int64_t raw_off[RPL_MAX_CAMERAS] = {};
    DevBuf mount_dr;                 // [E, C, 7] per-env mount perturbation (rpl_cameras_randomize)
    DevBuf rsm_mode;                 // [E] side-mask modes (rpl_side_mask_set)
    int32_t rsm_cols[3] = {0, 0, 0};
    bool rsm_on = false;
    int32_t *err_host = nullptr;   // mapped pinned word written by the kernels
    int32_t *err_dev = nullptr;
    bool has_last = false;
    int64_t last_step = 0;
    bool need_first = true;        // s_first must be set by the next render
    // recorded on the stream of every enqueued render or reset: rpl_sync and rpl_view_destroy wait on
    // it, which stays valid after the caller (or a server) has destroyed that stream
    cudaEvent_t done = nullptr;
    bool has_done = false;
    // optional timing of the traversal kernel: event pairs recorded around each launch
    static constexpr int kTimingSlots = 256;
    bool timing = false;
    cudaEvent_t ev[2 * kTimingSlots] = {};
    int64_t n_timed = 0;
    // launch shape of the render kernel: 4x8 tiles, per-SM tile queues dealt one env at a time in the
    // spatial order of the envs, links first, 8 blocks per SM (the fastest shape of the autotuner's
    // sweep on the 4096-env scale workload)
    Tuning tune{2, 2, 0, 8, 1, 1};
    // graph replay (rpl_render_graph): device step counter, captured graph and what it was captured for
    DevBuf d_step;
    int64_t dev_step_next = INT64_MIN; // value the device counter holds before the next replay
    int64_t gen = 0, g_gen = -1;       // bumped by rpl_cameras_set / rpl_sensor_set
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap_stream = nullptr;
    const void *g_poses = nullptr, *g_out = nullptr;
    Tuning g_tune{};
    int64_t g_env_offset = -1;
};

extern "C" {

RPL_API int32_t rpl_version(void) { return 1; }

RPL_API const char *rpl_last_error(void) { return g_err.c_str(); }

RPL_API rpl_status rpl_scene_create(const float *verts, int64_t n_verts, const int32_t *tris, int64_t n_tris,
                                    const rpl_scene_opts *opts, rpl_scene_t *out) {
    NvtxRange range("rpl_scene_create");
    if (!out) return fail(RPL_ERR_INVALID_ARG, "rpl_scene_create: out is NULL");
    *out = nullptr;
    if (n_verts < 0 || n_tris < 0) return fail(RPL_ERR_INVALID_ARG, "rpl_scene_create: negative size");
    if (n_tris > 0 && (!verts || !tris)) return fail(RPL_ERR_INVALID_ARG, "rpl_scene_create: NULL mesh array");
    // leaf references carry (first triangle << 3) in 31 bits during traversal
    if (n_tris >= (int64_t)0x0FFFFFFF) return fail(RPL_ERR_CAPACITY, "rpl_scene_create: too many triangles");
    rpl_scene_opts o{};
    if (opts) o = *opts;
    if (o.bvh_kind != RPL_BVH2 && o.bvh_kind != RPL_BVH8Q8 && o.bvh_kind != RPL_BVH4)
        return fail(RPL_ERR_INVALID_ARG, "rpl_scene_create: unknown bvh_kind %d", o.bvh_kind);
    if (o.max_leaf_size < 0 || o.max_leaf_size > 8)
        return fail(RPL_ERR_INVALID_ARG, "rpl_scene_create: max_leaf_size must be 0..8");
    if (o.bvh_kind == RPL_BVH8Q8 && o.max_leaf_size > 4)
        return fail(RPL_ERR_INVALID_ARG, "rpl_scene_create: the wide BVH holds at most 4 triangles per leaf");
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || o.device < 0 || o.device >= n_dev) {
        cudaGetLastError();
        return fail(RPL_ERR_NOT_FOUND, "rpl_scene_create: no CUDA device %d", o.device);
    }
    DeviceGuard g(o.device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "rpl_scene_create: cudaSetDevice");

    std::vector<char> hv, ht;
    rpl_status st = to_host(verts, (size_t)n_verts * 3 * sizeof(float), o.device, hv);
    if (st != RPL_OK) return st;
    st = to_host(tris, (size_t)n_tris * 3 * sizeof(int32_t), o.device, ht);
    if (st != RPL_OK) return st;

    rpl_scene *s = new (std::nothrow) rpl_scene();
    if (!s) return fail(RPL_ERR_OUT_OF_MEMORY, "rpl_scene_create: host allocation");
    s->device = o.device;
    s->opts = o;
    {
        // xy extent of the terrain (for the spatial order of the envs)
        const float *vp = reinterpret_cast<const float *>(hv.data());
        bool any = false;
        for (int64_t i = 0; i < n_verts; ++i)
            for (int a = 0; a < 2; ++a) {
                const float x = vp[3 * i + a];
                if (!std::isfinite(x)) continue;
                if (!any || x < s->xy_lo[a]) s->xy_lo[a] = x;
                if (!any || x > s->xy_hi[a]) s->xy_hi[a] = x;
                if (a == 1) any = true;
            }
    }
    s->links.resize(RPL_MAX_LINKS);
    s->has_link.assign(RPL_MAX_LINKS, false);
    for (int l = 0; l < RPL_MAX_LINKS; ++l) s->l_root[l] = -1;
    {
        HostBvh bvh;
        int rc = build_bvh2(reinterpret_cast<const float *>(hv.data()), n_verts,
                            reinterpret_cast<const int32_t *>(ht.data()), n_tris, o.max_leaf_size, o.build_threads,
                            &bvh, o.sah_node_cost);
        if (rc == -1) {
            delete s;
            return fail(RPL_ERR_INVALID_ARG, "rpl_scene_create: vertex index out of range");
        }
        if (rc != 0) {
            delete s;
            return fail(RPL_ERR_OUT_OF_MEMORY, "rpl_scene_create: host allocation during the BVH build");
        }
        if (bvh.depth >= kStackDepth) {
            delete s;
            return fail(RPL_ERR_CAPACITY, "rpl_scene_create: BVH depth %d exceeds %d", bvh.depth, kStackDepth);
        }
        pair_quad_leaves(bvh.nodes, bvh.tris);   // before any collapse: every layout tests the same triangles
        const void *node_src = bvh.nodes.data();
        size_t node_bytes = bvh.nodes.size() * sizeof(BvhNode);
        const std::vector<BvhTri> *tri_src = &bvh.tris;
        HostBvh8 wide;
        HostBvh4 four;
        s->t_n_nodes = (int64_t)bvh.nodes.size();
        s->t_depth = bvh.depth;
        if (o.bvh_kind == RPL_BVH4) {
            collapse_bvh4(bvh, &four);
            // a four-wide node pushes at most three children
            if (3 * four.depth > kStackDepth) {
                delete s;
                return fail(RPL_ERR_CAPACITY, "rpl_scene_create: four-wide BVH depth %d exceeds %d", four.depth,
                            kStackDepth / 3);
            }
            bvh.nodes.clear();
            bvh.nodes.shrink_to_fit();
            node_src = four.nodes.data();
            node_bytes = four.nodes.size() * sizeof(Bvh4Node);
            s->t_n_nodes = (int64_t)four.nodes.size();
            s->t_depth = four.depth;
        }
        if (o.bvh_kind == RPL_BVH8Q8) {
            if (collapse_bvh8(bvh, &wide) != 0) {
                delete s;
                return fail(RPL_ERR_INVALID_ARG, "rpl_scene_create: a leaf holds more than 4 triangles");
            }
            bvh.nodes.clear();
            bvh.nodes.shrink_to_fit();
            node_src = wide.nodes.data();
            node_bytes = wide.nodes.size() * sizeof(Bvh8Node);
            tri_src = &wide.tris;
            s->t_n_nodes = (int64_t)wide.nodes.size();
            s->t_depth = wide.depth;
        }
        s->t_n_tris = (int64_t)tri_src->size();
        if (o.bvh_kind == RPL_BVH2) encode_for_device(bvh.nodes);
        cudaError_t e = s->t_nodes.alloc(node_bytes);
        if (e == cudaSuccess) e = s->t_tris.alloc(std::max<size_t>(tri_src->size(), 1) * sizeof(BvhTri));
        if (e == cudaSuccess) e = cudaMemcpy(s->t_nodes.p, node_src, node_bytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !tri_src->empty())
            e = cudaMemcpy(s->t_tris.p, tri_src->data(), tri_src->size() * sizeof(BvhTri), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            delete s;
            return cuda_fail(e, "rpl_scene_create: uploading the terrain BVH");
        }
    }
    *out = s;
    return RPL_OK;
}

RPL_API rpl_status rpl_link_mesh_add(rpl_scene_t s, int32_t link_id, const float *verts, int64_t n_verts,
                                     const int32_t *tris, int64_t n_tris) {
    if (!s) return fail(RPL_ERR_INVALID_ARG, "rpl_link_mesh_add: scene is NULL");
    if (link_id < 0 || link_id >= RPL_MAX_LINKS)
        return fail(RPL_ERR_INVALID_ARG, "rpl_link_mesh_add: link_id %d outside 0..%d", link_id, RPL_MAX_LINKS - 1);
    if (n_verts < 0 || n_tris < 0) return fail(RPL_ERR_INVALID_ARG, "rpl_link_mesh_add: negative size");
    if (n_tris > 0 && (!verts || !tris)) return fail(RPL_ERR_INVALID_ARG, "rpl_link_mesh_add: NULL mesh array");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->frozen) return fail(RPL_ERR_INVALID_ARG, "rpl_link_mesh_add: scene is frozen by rpl_view_create");
    DeviceGuard g(s->device);
    std::vector<char> hv, ht;
    rpl_status st = to_host(verts, (size_t)n_verts * 3 * sizeof(float), s->device, hv);
    if (st != RPL_OK) return st;
    st = to_host(tris, (size_t)n_tris * 3 * sizeof(int32_t), s->device, ht);
    if (st != RPL_OK) return st;
    HostBvh bvh;
    int rc = build_bvh2(reinterpret_cast<const float *>(hv.data()), n_verts,
                        reinterpret_cast<const int32_t *>(ht.data()), n_tris, s->opts.max_leaf_size, 1, &bvh,
                        s->opts.sah_node_cost);
    if (rc == -1) return fail(RPL_ERR_INVALID_ARG, "rpl_link_mesh_add: vertex index out of range");
    if (rc != 0) return fail(RPL_ERR_OUT_OF_MEMORY, "rpl_link_mesh_add: host allocation");
    if (bvh.depth >= kStackDepth) return fail(RPL_ERR_CAPACITY, "rpl_link_mesh_add: BVH too deep");
    s->links[link_id] = std::move(bvh);
    s->has_link[link_id] = n_tris > 0;
    return RPL_OK;
}

static rpl_status freeze(rpl_scene *s) {
    if (s->frozen) return RPL_OK;
    std::vector<BvhNode> nodes;
    std::vector<BvhTri> tris;
    std::vector<float> roots(RPL_MAX_LINKS * 8, 0.f);
    int32_t depth = 0;
    for (int l = 0; l < RPL_MAX_LINKS; ++l) {
        float *r = roots.data() + 8 * l;
        if (!s->has_link[l]) {
            s->l_root[l] = -1;
            r[0] = r[1] = r[2] = 1.f;   // inverted: lo > hi marks "no mesh"
            r[4] = r[5] = r[6] = -1.f;
            continue;
        }
        const HostBvh &b = s->links[l];
        const int32_t nb = (int32_t)nodes.size(), tb = (int32_t)tris.size();
        for (BvhNode n : b.nodes) {
            n.child0 = n.child0 >= 0 ? n.child0 + nb : ~(~n.child0 + tb);
            n.child1 = n.child1 >= 0 ? n.child1 + nb : ~(~n.child1 + tb);
            nodes.push_back(n);
        }
        tris.insert(tris.end(), b.tris.begin(), b.tris.end());
        s->l_root[l] = nb;
        depth = std::max(depth, b.depth);
        for (int a = 0; a < 3; ++a) {
            r[a] = b.root_lo[a];
            r[4 + a] = b.root_hi[a];
        }
    }
    // leaf references carry (first triangle << 3) in 31 bits during traversal
    if (tris.size() >= (size_t)0x0FFFFFFF) return fail(RPL_ERR_CAPACITY, "the link meshes hold too many triangles");
    pair_quad_leaves(nodes, tris);
    encode_for_device(nodes);
    if (nodes.empty()) nodes.push_back(BvhNode{});
    if (tris.empty()) tris.push_back(BvhTri{});
    cudaError_t e = s->l_nodes.alloc(nodes.size() * sizeof(BvhNode));
    if (e == cudaSuccess) e = s->l_tris.alloc(tris.size() * sizeof(BvhTri));
    if (e == cudaSuccess) e = s->l_roots.alloc(roots.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(s->l_nodes.p, nodes.data(), nodes.size() * sizeof(BvhNode), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->l_tris.p, tris.data(), tris.size() * sizeof(BvhTri), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->l_roots.p, roots.data(), roots.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "uploading the link BVHs");
    s->l_n_nodes = 0;
    s->l_n_tris = 0;
    for (int l = 0; l < RPL_MAX_LINKS; ++l)
        if (s->has_link[l]) {
            s->l_n_nodes += (int64_t)s->links[l].nodes.size();
            s->l_n_tris += (int64_t)s->links[l].tris.size();
        }
    s->l_depth = depth;
    s->links.clear();
    s->links.shrink_to_fit();
    s->frozen = true;
    return RPL_OK;
}

RPL_API rpl_status rpl_scene_info_get(rpl_scene_t s, rpl_scene_info *info) {
    if (!s || !info) return fail(RPL_ERR_INVALID_ARG, "rpl_scene_info_get: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    info->terrain_tris = s->t_n_tris;
    info->terrain_nodes = s->t_n_nodes;
    info->terrain_bytes = s->t_n_nodes * (int64_t)(s->opts.bvh_kind == RPL_BVH8Q8 ? sizeof(Bvh8Node)
                                                   : s->opts.bvh_kind == RPL_BVH4 ? sizeof(Bvh4Node) : sizeof(BvhNode)) +
                          s->t_n_tris * (int64_t)sizeof(BvhTri);
    info->terrain_depth = s->t_depth;
    int n = 0;
    int64_t ln = 0, lt = 0;
    int32_t ld = 0;
    for (int l = 0; l < RPL_MAX_LINKS; ++l)
        if (s->has_link[l]) {
            ++n;
            if (!s->frozen) {
                ln += (int64_t)s->links[l].nodes.size();
                lt += (int64_t)s->links[l].tris.size();
                ld = std::max(ld, s->links[l].depth);
            }
        }
    if (s->frozen) {
        ln = s->l_n_nodes;
        lt = s->l_n_tris;
        ld = s->l_depth;
    }
    info->n_links = n;
    info->link_tris = lt;
    info->link_nodes = ln;
    info->link_bytes = ln * (int64_t)sizeof(BvhNode) + lt * (int64_t)sizeof(BvhTri);
    info->link_depth = ld;
    info->frozen = s->frozen ? 1 : 0;
    return RPL_OK;
}

RPL_API rpl_status rpl_bvh_build_host(const float *verts, int64_t n_verts, const int32_t *tris, int64_t n_tris,
                                      int32_t max_leaf, int32_t threads, void *nodes_out, int64_t nodes_cap,
                                      void *tris_out, int64_t *n_nodes, int32_t *depth) {
    if (n_verts < 0 || n_tris < 0 || !n_nodes || !depth || (n_tris > 0 && (!verts || !tris)))
        return fail(RPL_ERR_INVALID_ARG, "rpl_bvh_build_host: bad argument");
    if (max_leaf < 0 || max_leaf > 8) return fail(RPL_ERR_INVALID_ARG, "rpl_bvh_build_host: max_leaf 0..8");
    HostBvh b;
    int rc = build_bvh2(verts, n_verts, tris, n_tris, max_leaf, threads, &b);
    if (rc == -1) return fail(RPL_ERR_INVALID_ARG, "rpl_bvh_build_host: vertex index out of range");
    if (rc != 0) return fail(RPL_ERR_OUT_OF_MEMORY, "rpl_bvh_build_host: host allocation");
    *n_nodes = (int64_t)b.nodes.size();
    *depth = b.depth;
    if (nodes_out) {
        if (nodes_cap < (int64_t)b.nodes.size()) return fail(RPL_ERR_CAPACITY, "rpl_bvh_build_host: nodes_cap too small");
        std::memcpy(nodes_out, b.nodes.data(), b.nodes.size() * sizeof(BvhNode));
    }
    if (tris_out && n_tris > 0) std::memcpy(tris_out, b.tris.data(), b.tris.size() * sizeof(BvhTri));
    return RPL_OK;
}

RPL_API rpl_status rpl_bvh8_build_host(const float *verts, int64_t n_verts, const int32_t *tris, int64_t n_tris,
                                       int32_t max_leaf, int32_t threads, void *nodes_out, int64_t nodes_cap,
                                       void *tris_out, int64_t *n_nodes, int32_t *depth) {
    if (n_verts < 0 || n_tris < 0 || !n_nodes || !depth || (n_tris > 0 && (!verts || !tris)))
        return fail(RPL_ERR_INVALID_ARG, "rpl_bvh8_build_host: bad argument");
    if (max_leaf < 0 || max_leaf > 4) return fail(RPL_ERR_INVALID_ARG, "rpl_bvh8_build_host: max_leaf 0..4");
    HostBvh b;
    int rc = build_bvh2(verts, n_verts, tris, n_tris, max_leaf, threads, &b);
    if (rc == -1) return fail(RPL_ERR_INVALID_ARG, "rpl_bvh8_build_host: vertex index out of range");
    if (rc != 0) return fail(RPL_ERR_OUT_OF_MEMORY, "rpl_bvh8_build_host: host allocation");
    HostBvh8 w;
    if (collapse_bvh8(b, &w) != 0) return fail(RPL_ERR_INVALID_ARG, "rpl_bvh8_build_host: leaf too large");
    *n_nodes = (int64_t)w.nodes.size();
    *depth = w.depth;
    if (nodes_out) {
        if (nodes_cap < (int64_t)w.nodes.size()) return fail(RPL_ERR_CAPACITY, "rpl_bvh8_build_host: nodes_cap too small");
        std::memcpy(nodes_out, w.nodes.data(), w.nodes.size() * sizeof(Bvh8Node));
    }
    if (tris_out && n_tris > 0) std::memcpy(tris_out, w.tris.data(), w.tris.size() * sizeof(BvhTri));
    return RPL_OK;
}

RPL_API void rpl_scene_destroy(rpl_scene_t s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->views > 0 || s->servers > 0) {
            s->destroy_pending = true;   // freed by the last view or server that goes
            return;
        }
    }
    DeviceGuard g(s->device);
    delete s;
}

// Drops one user of the scene (a view or a server) and frees the scene if it was destroyed while
// in use and this was its last user.
static void scene_release(rpl_scene *s, bool server) {
    bool free_now;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (server)
            s->servers--;
        else
            s->views--;
        free_now = s->destroy_pending && s->views == 0 && s->servers == 0;
    }
    if (free_now) {
        DeviceGuard g(s->device);
        delete s;
    }
}

RPL_API rpl_status rpl_view_create(rpl_scene_t s, int32_t n_envs, int32_t n_links, rpl_view_t *out) {
    if (!out) return fail(RPL_ERR_INVALID_ARG, "rpl_view_create: out is NULL");
    *out = nullptr;
    if (!s) return fail(RPL_ERR_INVALID_ARG, "rpl_view_create: scene is NULL");
    if (n_envs < 0 || n_links < 1) return fail(RPL_ERR_INVALID_ARG, "rpl_view_create: n_envs >= 0 and n_links >= 1");
    if (n_links > RPL_MAX_LINKS) return fail(RPL_ERR_CAPACITY, "rpl_view_create: n_links > %d", RPL_MAX_LINKS);
    std::lock_guard<std::mutex> lk(s->mu);
    DeviceGuard g(s->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "rpl_view_create: cudaSetDevice");
    rpl_status st = freeze(s);
    if (st != RPL_OK) return st;
    rpl_view *v = new (std::nothrow) rpl_view();
    if (!v) return fail(RPL_ERR_OUT_OF_MEMORY, "rpl_view_create: host allocation");
    v->scene = s;
    v->E = n_envs;
    v->L = n_links;
    const size_t EL = (size_t)n_envs * n_links;
    cudaError_t e = v->link_xf.alloc(EL * 3 * sizeof(float4));
    if (e == cudaSuccess) e = v->link_box.alloc(EL * 2 * sizeof(float4));
    if (e == cudaSuccess) e = v->s_first.alloc((size_t)n_envs * sizeof(int64_t));
    if (e == cudaSuccess) e = v->mask_stage.alloc((size_t)n_envs);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&v->err_host, sizeof(int32_t), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        *v->err_host = 0;
        e = cudaHostGetDevicePointer((void **)&v->err_dev, v->err_host, 0);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&v->n_queues, cudaDevAttrMultiProcessorCount, s->device);
    if (e == cudaSuccess) {
        v->n_queues = std::max(1, v->n_queues);
        e = v->queues.alloc((size_t)v->n_queues * sizeof(unsigned long long));
    }
    if (e == cudaSuccess) e = v->env_key.alloc(std::max<size_t>((size_t)n_envs, 1) * sizeof(uint32_t));
    if (e == cudaSuccess) e = v->env_order.alloc(std::max<size_t>((size_t)n_envs, 1) * sizeof(int32_t));
    if (e != cudaSuccess) {
        if (v->err_host) cudaFreeHost(v->err_host);
        if (v->done) cudaEventDestroy(v->done);
        delete v;
        return cuda_fail(e, "rpl_view_create: allocating per-env state");
    }
    v->sensor.out_dtype = RPL_OUT_F32;
    s->views++;
    *out = v;
    return RPL_OK;
}

static rpl_status alloc_ring(rpl_view *v) {
    const int64_t span = (int64_t)v->sensor.max_latency + 1;
    if (!v->cams_set || span <= 1) {
        v->ring.release();
        return RPL_OK;
    }
    cudaError_t e = v->ring.alloc((size_t)v->E * span * v->P * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(e, "allocating the latency ring buffer");
    return RPL_OK;
}

RPL_API rpl_status rpl_cameras_set(rpl_view_t v, const rpl_camera *cams, int32_t n_cams, const float *per_env_intr) {
    if (!v || !cams) return fail(RPL_ERR_INVALID_ARG, "rpl_cameras_set: NULL argument");
    if (n_cams < 1) return fail(RPL_ERR_INVALID_ARG, "rpl_cameras_set: need at least one camera");
    if (n_cams > RPL_MAX_CAMERAS) return fail(RPL_ERR_CAPACITY, "rpl_cameras_set: more than %d cameras", RPL_MAX_CAMERAS);
    int64_t off = 0, raw = 0;
    int64_t raw_off[RPL_MAX_CAMERAS] = {};
    int32_t toff = 0;
    for (int c = 0; c < n_cams; ++c) {
        const rpl_camera &k = cams[c];
        const rpl_status cst = check_camera(k, c, v->L, "rpl_cameras_set");
        if (cst != RPL_OK) return cst;
        const int32_t ds = k.downsample <= 1 ? 1 : k.downsample;
        v->cam_off[c] = off;
        v->tile_off[c] = toff;
        off += (int64_t)(k.width / ds) * (k.height / ds);
        toff += ((k.width + 7) / 8) * ((k.height + 3) / 4);
        if (ds > 1) {
            raw_off[c] = raw;
            raw += (int64_t)k.width * k.height;
        }
    }
    if (off >= (int64_t)1 << 31 || raw >= (int64_t)1 << 31)
        return fail(RPL_ERR_CAPACITY, "rpl_cameras_set: too many pixels per env");
    DeviceGuard g(v->scene->device);
    for (int c = 0; c < n_cams; ++c) v->cams[c] = cams[c];
    v->cam_off[n_cams] = off;
    v->tile_off[n_cams] = toff;
    v->C = n_cams;
    v->P = off;
    v->cams_set = true;
    v->gen++;
    cudaError_t e = v->cam_xf.alloc((size_t)v->E * n_cams * 5 * sizeof(float4));
    if (e != cudaSuccess) return cuda_fail(e, "rpl_cameras_set: allocating camera transforms");
    int64_t max_tiles = 0;
    for (int lw = 2; lw <= 4; ++lw) {
        const int tw = 1 << lw, th = 32 / tw;
        int64_t tiles = 0;
        for (int c = 0; c < n_cams; ++c) tiles += (int64_t)((cams[c].width + tw - 1) / tw) * ((cams[c].height + th - 1) / th);
        max_tiles = std::max(max_tiles, tiles);
    }
    e = v->tile_info.alloc((size_t)v->E * max_tiles * sizeof(int4));
    if (e != cudaSuccess) return cuda_fail(e, "rpl_cameras_set: allocating the per-tile entry nodes");
    v->raw_per_env = raw;
    for (int c = 0; c < n_cams; ++c) v->raw_off[c] = raw_off[c];
    if (raw > 0) {
        e = v->raw.alloc((size_t)v->E * raw * sizeof(float));
        if (e != cudaSuccess) return cuda_fail(e, "rpl_cameras_set: allocating the raw-depth buffer");
    } else {
        v->raw.release();
    }
    v->mount_dr.release();
    if (per_env_intr) {
        const size_t bytes = (size_t)v->E * n_cams * 4 * sizeof(float);
        std::vector<char> h;
        rpl_status st = to_host(per_env_intr, bytes, v->scene->device, h);
        if (st != RPL_OK) return st;
        e = v->intr.alloc(bytes);
        if (e == cudaSuccess && bytes) e = cudaMemcpy(v->intr.p, h.data(), bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "rpl_cameras_set: per-env intrinsics");
        const float *k = reinterpret_cast<const float *>(h.data());
        for (size_t i = 0; i < (size_t)v->E * n_cams; ++i)
            if (!(k[4 * i] != 0.f) || !(k[4 * i + 1] != 0.f))
                return fail(RPL_ERR_INVALID_ARG, "rpl_cameras_set: per-env intrinsics have fx or fy 0");
    } else {
        v->intr.release();
    }
    v->out_stage.release();
    v->has_last = false;
    v->need_first = true;
    return alloc_ring(v);
}

RPL_API rpl_status rpl_cameras_randomize(rpl_view_t v, const float *mount_delta) {
    if (!v) return fail(RPL_ERR_INVALID_ARG, "rpl_cameras_randomize: view is NULL");
    if (!v->cams_set) return fail(RPL_ERR_INVALID_ARG, "rpl_cameras_randomize: cameras not set");
    DeviceGuard g(v->scene->device);
    v->gen++;   // a captured graph holds the buffer's address
    if (!mount_delta) {
        v->mount_dr.release();
        return RPL_OK;
    }
    const size_t n = (size_t)v->E * v->C;
    std::vector<char> h;
    rpl_status st = to_host(mount_delta, n * 7 * sizeof(float), v->scene->device, h);
    if (st != RPL_OK) return st;
    float *d = reinterpret_cast<float *>(h.data());
    for (size_t i = 0; i < n; ++i) {
        float *q = d + 7 * i + 3;
        const double nq = std::sqrt((double)q[0] * q[0] + (double)q[1] * q[1] + (double)q[2] * q[2] + (double)q[3] * q[3]);
        if (!(nq > 0) || !std::isfinite(nq) || !std::isfinite(d[7 * i]) || !std::isfinite(d[7 * i + 1]) ||
            !std::isfinite(d[7 * i + 2]))
            return fail(RPL_ERR_INVALID_ARG, "rpl_cameras_randomize: entry %zu has a zero or non-finite value", i);
        for (int k = 0; k < 4; ++k) q[k] = (float)(q[k] / nq);
    }
    if (v->has_done) cudaEventSynchronize(v->done);   // an enqueued render may still read the old values
    cudaError_t e = v->mount_dr.bytes >= std::max<size_t>(n * 7 * sizeof(float), 16) ? cudaSuccess
                                                                                       : v->mount_dr.alloc(n * 7 * sizeof(float));
    if (e == cudaSuccess && n) e = cudaMemcpy(v->mount_dr.p, h.data(), n * 7 * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "rpl_cameras_randomize: uploading the mount perturbations");
    return RPL_OK;
}

RPL_API rpl_status rpl_side_mask_set(rpl_view_t v, const int32_t cols[3], const uint8_t *env_mode) {
    if (!v) return fail(RPL_ERR_INVALID_ARG, "rpl_side_mask_set: view is NULL");
    DeviceGuard g(v->scene->device);
    v->gen++;
    if (!env_mode) {
        v->rsm_on = false;
        return RPL_OK;
    }
    if (!cols || cols[0] < 0 || cols[1] < 0 || cols[2] < 0)
        return fail(RPL_ERR_INVALID_ARG, "rpl_side_mask_set: cols must be three values >= 0");
    std::vector<char> h;
    rpl_status st = to_host(env_mode, (size_t)v->E, v->scene->device, h);
    if (st != RPL_OK) return st;
    if (v->has_done) cudaEventSynchronize(v->done);   // an enqueued render may still read the old modes
    cudaError_t e = v->rsm_mode.bytes >= std::max<size_t>((size_t)v->E, 16) ? cudaSuccess : v->rsm_mode.alloc((size_t)v->E);
    if (e == cudaSuccess && v->E) e = cudaMemcpy(v->rsm_mode.p, h.data(), (size_t)v->E, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "rpl_side_mask_set: uploading the modes");
    for (int k = 0; k < 3; ++k) v->rsm_cols[k] = cols[k];
    v->rsm_on = true;
    return RPL_OK;
}

RPL_API rpl_status rpl_sensor_set(rpl_view_t v, const rpl_sensor_params *prm) {
    if (!v || !prm) return fail(RPL_ERR_INVALID_ARG, "rpl_sensor_set: NULL argument");
    if (prm->max_latency < 0 || prm->max_latency > 15)
        return fail(RPL_ERR_INVALID_ARG, "rpl_sensor_set: max_latency must be 0..15");
    if (!(prm->p_drop >= 0.f && prm->p_drop <= 1.f))
        return fail(RPL_ERR_INVALID_ARG, "rpl_sensor_set: p_drop must be in [0, 1]");
    if (!(prm->sigma_abs >= 0.f) || !(prm->sigma_rel >= 0.f) || !std::isfinite(prm->sigma_abs) ||
        !std::isfinite(prm->sigma_rel) || !std::isfinite(prm->fill))
        return fail(RPL_ERR_INVALID_ARG, "rpl_sensor_set: sigmas must be finite and >= 0, fill finite");
    if (prm->depth_kind != RPL_DEPTH_Z && prm->depth_kind != RPL_DEPTH_RANGE)
        return fail(RPL_ERR_INVALID_ARG, "rpl_sensor_set: unknown depth_kind");
    if (prm->out_dtype != RPL_OUT_F32 && prm->out_dtype != RPL_OUT_F16 && prm->out_dtype != RPL_OUT_U16)
        return fail(RPL_ERR_INVALID_ARG, "rpl_sensor_set: unknown out_dtype");
    DeviceGuard g(v->scene->device);
    v->sensor = *prm;
    v->gen++;
    v->has_last = false;
    v->need_first = true;
    return alloc_ring(v);
}

RPL_API rpl_status rpl_view_layout(rpl_view_t v, int64_t *cam_offsets, int64_t *total) {
    if (!v) return fail(RPL_ERR_INVALID_ARG, "rpl_view_layout: view is NULL");
    if (!v->cams_set) return fail(RPL_ERR_INVALID_ARG, "rpl_view_layout: cameras not set");
    if (cam_offsets)
        for (int c = 0; c <= v->C; ++c) cam_offsets[c] = v->cam_off[c];
    if (total) *total = v->P;
    return RPL_OK;
}

// Kernel view of the cameras for the view's tile shape; returns the tiles per env.
static int32_t fill_cams(const rpl_view *v, CamDev *out) {
    const int tw = 1 << v->tune.tile_w_log2, th = 32 / tw;
    int32_t toff = 0;
    for (int c = 0; c < v->C; ++c) {
        const rpl_camera &k = v->cams[c];
        CamDev &d = out[c];
        d.width = k.width;
        d.height = k.height;
        d.tiles_x = (k.width + tw - 1) / tw;
        fastdiv_magic((uint32_t)d.tiles_x, d.tx_m, d.tx_k);
        d.tile_off = toff;
        toff += d.tiles_x * ((k.height + th - 1) / th);
        d.ds = k.downsample <= 1 ? 1 : k.downsample;
        d.out_w = k.width / d.ds;
        d.out_h = k.height / d.ds;
        d.raw_off = (int32_t)v->raw_off[c];
        d.pix_off = (int32_t)v->cam_off[c];
        d.mount = k.mount_link;
        d.fx = k.fx;
        d.fy = k.fy;
        d.cx = k.cx;
        d.cy = k.cy;
        d.d_min = k.d_min;
        d.d_max = k.d_max;
        for (int a = 0; a < 3; ++a) d.off_pos[a] = k.offset_pos[a];
        quat_normalise(k.offset_quat_xyzw, d.off_quat);
    }
    return toff;
}

static size_t out_elem_bytes(const rpl_view *v) { return v->sensor.out_dtype == RPL_OUT_F32 ? 4 : 2; }

// Terrain nodes held by the device array, in units of the scene's node layout.
static int64_t terrain_node_count(const rpl_scene *s) {
    const size_t node = s->opts.bvh_kind == RPL_BVH8Q8 ? sizeof(Bvh8Node)
                        : s->opts.bvh_kind == RPL_BVH4 ? sizeof(Bvh4Node) : sizeof(BvhNode);
    return (int64_t)(s->t_nodes.bytes / node);
}

// Marks the end of the work just enqueued for `v` on `st`.
static void mark_done(rpl_view *v, cudaStream_t st) {
    if (cudaEventRecord(v->done, st) == cudaSuccess) v->has_done = true;
}

// Prep and render parameters of one render of view v (device buffers); launches the sensor-state
// reset on `st` first when the view needs one.  step_dev (graph capture only) makes both kernels
// read the step from device memory instead of `step`.
static rpl_status build_params(rpl_view *v, const float *poses_dev, int64_t step, int64_t env_offset, void *out_dev,
                               cudaStream_t st, unsigned long long *counters_dev, const int64_t *step_dev,
                               PrepParams &pp, RenderParams &rp) {
    rpl_scene *s = v->scene;
    cudaError_t e;
    if (v->need_first && !step_dev) {
        e = launch_set_first(v->s_first.as<int64_t>(), v->E, step, nullptr, st);
        if (e != cudaSuccess) return cuda_fail(e, "rpl_render: launching the sensor-state reset");
        v->need_first = false;
    }
    pp = PrepParams{};
    pp.poses = poses_dev;
    pp.link_root = s->l_roots.as<const float4>();
    pp.tnodes = s->t_nodes.as<const float4>();
    pp.bvh_kind = s->opts.bvh_kind;
#ifdef RPL_CHECKED
    pp.n_tnodes = terrain_node_count(s);
#endif
    pp.intr = v->intr.p ? v->intr.as<const float>() : nullptr;
    pp.mount_dr = v->mount_dr.p ? v->mount_dr.as<const float>() : nullptr;
    for (int l = 0; l < RPL_MAX_LINKS; ++l) pp.lroot[l] = l < v->L ? s->l_root[l] : -1;
    pp.link_xf = v->link_xf.as<float4>();
    pp.link_box = v->link_box.as<float4>();
    pp.cam_xf = v->cam_xf.as<float4>();
    pp.E = v->E;
    pp.L = v->L;
    pp.C = v->C;
    const int32_t tiles_per_env = fill_cams(v, pp.cams);
    pp.step = step;
    pp.step_dev = step_dev;
    pp.s_first = v->s_first.as<const int64_t>();
    pp.env_offset = (uint32_t)env_offset;
    pp.span = (uint32_t)v->sensor.max_latency + 1u;
    pp.seed0 = v->sensor.seed[0];
    pp.seed1 = v->sensor.seed[1];
    const bool queued = v->tune.persistent == 2;
    pp.queues = queued ? v->queues.as<unsigned long long>() : nullptr;
    pp.n_queues = v->n_queues;
    pp.env_key = v->tune.env_order ? v->env_key.as<uint32_t>() : nullptr;
    for (int a = 0; a < 2; ++a) {
        pp.xy_lo[a] = s->xy_lo[a];
        pp.xy_hi[a] = s->xy_hi[a];
    }

    rp = RenderParams{};
    rp.tnodes = s->t_nodes.as<const float4>();
    rp.ttris = s->t_tris.as<const float4>();
    rp.bvh_kind = pp.bvh_kind;
    rp.out_dtype = v->sensor.out_dtype;
    rp.lnodes = s->l_nodes.as<const float4>();
    rp.ltris = s->l_tris.as<const float4>();
#ifdef RPL_CHECKED
    rp.n_tnodes = terrain_node_count(s);
    rp.n_ttris = (int64_t)(s->t_tris.bytes / sizeof(BvhTri));
    rp.n_lnodes = (int64_t)(s->l_nodes.bytes / sizeof(BvhNode));
    rp.n_ltris = (int64_t)(s->l_tris.bytes / sizeof(BvhTri));
#endif
    rp.link_xf = v->link_xf.as<const float4>();
    rp.link_box = v->link_box.as<const float4>();
    rp.link_root = s->l_roots.as<const float4>();
    rp.cam_xf = v->cam_xf.as<const float4>();
    rp.tile_info = v->tile_info.as<int4>();
    rp.intr = v->intr.p ? v->intr.as<const float>() : nullptr;
    rp.E = v->E;
    rp.L = v->L;
    rp.C = v->C;
    rp.tiles_per_env = tiles_per_env;
    if (tiles_per_env > 0) fastdiv_magic((uint32_t)tiles_per_env, rp.tpe_m, rp.tpe_k);
    rp.tile_w_log2 = v->tune.tile_w_log2;
    rp.persistent = v->tune.persistent;
    rp.terrain_first = v->tune.terrain_first;
    rp.min_blocks = v->tune.min_blocks;
    rp.step_dev = step_dev;
    rp.pix_per_env = (int32_t)v->P;
    rp.depth_kind = v->sensor.depth_kind;
    for (int l = 0; l < RPL_MAX_LINKS; ++l) rp.lroot[l] = l < v->L ? s->l_root[l] : -1;
    std::memcpy(rp.cams, pp.cams, sizeof(pp.cams));
    const rpl_sensor_params &sp = v->sensor;
    rp.step = step;
    rp.env_offset = (uint32_t)env_offset;
    rp.span = (uint32_t)sp.max_latency + 1u;
    rp.seed0 = sp.seed[0];
    rp.seed1 = sp.seed[1];
    double thr = std::floor((double)sp.p_drop * 4294967296.0);
    rp.drop_thr = (uint64_t)std::min(std::max(thr, 0.0), 4294967296.0);
    rp.sigma_abs = sp.sigma_abs;
    rp.sigma_rel = sp.sigma_rel;
    rp.fill = sp.fill;
    rp.sensor_on = (sp.sigma_abs != 0.f || sp.sigma_rel != 0.f || sp.p_drop != 0.f || sp.max_latency != 0) ? 1 : 0;
    rp.ring = rp.span > 1 ? v->ring.as<float>() : nullptr;
    rp.raw = v->raw_per_env > 0 ? v->raw.as<float>() : nullptr;
    rp.raw_per_env = (int32_t)v->raw_per_env;
    rp.rsm_mode = v->rsm_on ? v->rsm_mode.as<const uint8_t>() : nullptr;
    for (int k = 0; k < 3; ++k) rp.rsm_cols[k] = v->rsm_cols[k];
    rp.s_first = v->s_first.as<const int64_t>();
    rp.out = out_dev;
    rp.err = v->err_dev;
    rp.counters = counters_dev;
    rp.queues = pp.queues;
    rp.n_queues = pp.n_queues;
    rp.chunk_envs = v->tune.chunk_envs;
    const int64_t chunk = (int64_t)rp.chunk_envs * tiles_per_env;
    if (chunk > 0 && chunk < 0x7FFFFFFFll) fastdiv_magic((uint32_t)chunk, rp.chunk_m, rp.chunk_k);
    rp.env_order = v->tune.env_order ? v->env_order.as<const int32_t>() : nullptr;
    return RPL_OK;
}

// Enqueues prep + render of view v on `st`.
static rpl_status enqueue(rpl_view *v, const float *poses_dev, int64_t step, int64_t env_offset, void *out_dev,
                          cudaStream_t st, bool count, unsigned long long *counters_dev,
                          const int64_t *step_dev = nullptr) {
    PrepParams pp;
    RenderParams rp;
    rpl_status stt = build_params(v, poses_dev, step, env_offset, out_dev, st, counters_dev, step_dev, pp, rp);
    if (stt != RPL_OK) return stt;
    cudaError_t e = launch_prep(pp, st);
    if (e != cudaSuccess) return cuda_fail(e, "rpl_render: launching the prep kernel");
    if (pp.env_key) {
        e = launch_env_order(pp.env_key, v->env_order.as<int32_t>(), v->E, st);
        if (e != cudaSuccess) return cuda_fail(e, "rpl_render: launching the env-order kernel");
    }
    e = launch_tile_prep(rp, st);
    if (e != cudaSuccess) return cuda_fail(e, "rpl_render: launching the tile-prep kernel");
    const int slot = (int)(v->n_timed % rpl_view::kTimingSlots);
    const bool timed = v->timing && !step_dev;   // no event records inside a graph capture
    if (timed) cudaEventRecord(v->ev[2 * slot], st);
    e = launch_render(rp, count, st);
    if (e != cudaSuccess) return cuda_fail(e, "rpl_render: launching the render kernel");
    if (timed) {
        cudaEventRecord(v->ev[2 * slot + 1], st);
        v->n_timed++;
    }
    e = launch_downsample(rp, st);
    if (e != cudaSuccess) return cuda_fail(e, "rpl_render: launching the downsample kernel");
    if (!step_dev) mark_done(v, st);   // a captured render is marked by rpl_render_graph's launch
    return RPL_OK;
}

static rpl_status check_render_args(rpl_view *v, const float *poses, int64_t env_offset, void *out) {
    if (!v) return fail(RPL_ERR_INVALID_ARG, "rpl_render: view is NULL");
    if (!v->cams_set) return fail(RPL_ERR_INVALID_ARG, "rpl_render: cameras not set");
    if (v->E > 0 && (!poses || !out)) return fail(RPL_ERR_INVALID_ARG, "rpl_render: NULL poses or output");
    if (env_offset < 0 || env_offset + (int64_t)v->E > ((int64_t)1 << 32))
        return fail(RPL_ERR_INVALID_ARG, "rpl_render: env_offset + n_envs must lie in [0, 2^32]");
    if (((uintptr_t)poses & 3) || ((uintptr_t)out & 3))
        return fail(RPL_ERR_INVALID_ARG, "rpl_render: poses and output must be 4-byte aligned");
    if (*v->err_host != 0)
        return fail(RPL_ERR_DEVICE_FAULT, "rpl_render: an earlier kernel on this view recorded error 0x%x "
                    "(1: stack overflow, 4: index out of range); call rpl_sync", *v->err_host);
    return RPL_OK;
}

RPL_API rpl_status rpl_render(rpl_view_t v, const float *poses, int64_t step, int64_t env_offset, void *out,
                              void *stream) {
    NvtxRange range("rpl_render");
    rpl_status st = check_render_args(v, poses, env_offset, out);
    if (st != RPL_OK) return st;
    if (v->has_last && step != v->last_step && step != v->last_step + 1)
        return fail(RPL_ERR_INVALID_ARG, "rpl_render: step %lld after %lld; steps must advance by 0 or 1 "
                    "(rpl_view_reset restarts)", (long long)step, (long long)v->last_step);
    if (v->E == 0) {
        v->has_last = true;
        v->last_step = step;
        return RPL_OK;
    }
    rpl_scene *s = v->scene;
    DeviceGuard g(s->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "rpl_render: cudaSetDevice");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    const size_t pose_bytes = (size_t)v->E * v->L * 7 * sizeof(float);
    const size_t out_bytes = (size_t)v->E * v->P * out_elem_bytes(v);
    // While the stream is being captured into a graph the buffers must be device memory: no
    // pointer queries are issued then.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(cs, &cap) != cudaSuccess) {
        cudaGetLastError();
        cap = cudaStreamCaptureStatusNone;
    }
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    const PtrKind pk = capturing ? PTR_DEVICE : pointer_kind(poses, s->device);
    const PtrKind ok = capturing ? PTR_DEVICE : pointer_kind(out, s->device);
    if (pk == PTR_OTHER_DEVICE || ok == PTR_OTHER_DEVICE)
        return fail(RPL_ERR_INVALID_ARG, "rpl_render: a buffer lives on another GPU than the scene");
    const float *pd = poses;
    void *od = out;
    cudaError_t e;
    if (pk == PTR_HOST) {
        if (v->pose_stage.bytes < pose_bytes) {
            e = v->pose_stage.alloc(pose_bytes);
            if (e != cudaSuccess) return cuda_fail(e, "rpl_render: allocating the pose staging buffer");
        }
        e = cudaMemcpyAsync(v->pose_stage.p, poses, pose_bytes, cudaMemcpyHostToDevice, cs);
        if (e != cudaSuccess) return cuda_fail(e, "rpl_render: copying poses to the device");
        pd = v->pose_stage.as<const float>();
    }
    const bool async_out = ok == PTR_HOST && v->host_async;
    const int k = v->stage_next;
    if (ok == PTR_HOST) {
        DevBuf &stage = async_out && k == 1 ? v->out_stage2 : v->out_stage;
        if (stage.bytes < out_bytes) {
            if (async_out) cudaEventSynchronize(v->copied[k]);   // the buffer may still be copied from
            e = stage.alloc(out_bytes);
            if (e != cudaSuccess) return cuda_fail(e, "rpl_render: allocating the output staging buffer");
        }
        od = stage.p;
        // the render may overwrite this staging buffer only after its previous copy to the host
        if (async_out) cudaStreamWaitEvent(cs, v->copied[k], 0);
    }
    st = enqueue(v, pd, step, env_offset, od, cs, false, nullptr);
    if (st != RPL_OK) return st;
    v->has_last = true;
    v->last_step = step;
    if (async_out) {
        // the copy to the host runs on the view's copy stream, overlapped with the next render
        e = cudaEventRecord(v->rendered[k], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(v->copy_stream, v->rendered[k], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, od, out_bytes, cudaMemcpyDeviceToHost, v->copy_stream);
        if (e == cudaSuccess) e = cudaEventRecord(v->copied[k], v->copy_stream);
        if (e != cudaSuccess) return cuda_fail(e, "rpl_render: enqueuing the copy of depth to the host");
        mark_done(v, v->copy_stream);   // rpl_sync waits for the copy (which waited for the render)
        v->stage_next = 1 - k;
    } else if (ok == PTR_HOST) {
        e = cudaMemcpyAsync(out, od, out_bytes, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) return cuda_fail(e, "rpl_render: copying depth to the host");
    }
    return RPL_OK;
}

RPL_API rpl_status rpl_sensor_apply(rpl_view_t v, const float *depth_in, int64_t step, int64_t env_offset, void *out,
                                    void *stream) {
    NvtxRange range("rpl_sensor_apply");
    rpl_status st = check_render_args(v, depth_in, env_offset, out);
    if (st != RPL_OK) return st;
    if (v->raw_per_env > 0)
        return fail(RPL_ERR_INVALID_ARG, "rpl_sensor_apply: the view has downsampled cameras (give their averaged "
                                         "depth to a view without downsampling)");
    if (v->has_last && step != v->last_step && step != v->last_step + 1)
        return fail(RPL_ERR_INVALID_ARG, "rpl_sensor_apply: step %lld after %lld; steps must advance by 0 or 1",
                    (long long)step, (long long)v->last_step);
    if (v->E == 0) {
        v->has_last = true;
        v->last_step = step;
        return RPL_OK;
    }
    rpl_scene *s = v->scene;
    DeviceGuard g(s->device);
    if (pointer_kind(depth_in, s->device) != PTR_DEVICE || pointer_kind(out, s->device) != PTR_DEVICE)
        return fail(RPL_ERR_INVALID_ARG, "rpl_sensor_apply: input and output must be device memory");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    PrepParams pp;
    RenderParams rp;
    st = build_params(v, nullptr, step, env_offset, out, cs, nullptr, nullptr, pp, rp);
    if (st != RPL_OK) return st;
    cudaError_t e = launch_sensor(rp, depth_in, cs);
    if (e != cudaSuccess) return cuda_fail(e, "rpl_sensor_apply: launch");
    v->has_last = true;
    v->last_step = step;
    mark_done(v, cs);
    return RPL_OK;
}

RPL_API rpl_status rpl_render_counters(rpl_view_t v, const float *poses, int64_t step, int64_t env_offset,
                                       void *out, void *stream, rpl_counters *counters) {
    rpl_status st = check_render_args(v, poses, env_offset, out);
    if (st != RPL_OK) return st;
    if (!counters) return fail(RPL_ERR_INVALID_ARG, "rpl_render_counters: counters is NULL");
    std::memset(counters, 0, sizeof(*counters));
    if (v->E == 0) return RPL_OK;
    rpl_scene *s = v->scene;
    DeviceGuard g(s->device);
    if (pointer_kind(poses, s->device) != PTR_DEVICE || pointer_kind(out, s->device) != PTR_DEVICE)
        return fail(RPL_ERR_INVALID_ARG, "rpl_render_counters: poses and output must be device memory");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    DevBuf cnt;
    cudaError_t e = cnt.alloc(6 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt.p, 0, 6 * sizeof(unsigned long long), cs);
    if (e != cudaSuccess) return cuda_fail(e, "rpl_render_counters: counter buffer");
    st = enqueue(v, poses, step, env_offset, out, cs, true, cnt.as<unsigned long long>());
    if (st != RPL_OK) return st;
    unsigned long long h[6];
    e = cudaMemcpyAsync(h, cnt.p, sizeof h, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return cuda_fail(e, "rpl_render_counters: reading counters");
    counters->rays = h[0];
    counters->terrain_nodes = h[1];
    counters->terrain_tris = h[2];
    counters->link_boxes = h[3];
    counters->link_nodes = h[4];
    counters->link_tris = h[5];
    return RPL_OK;
}

RPL_API rpl_status rpl_view_reset(rpl_view_t v, const uint8_t *mask, int64_t step, void *stream) {
    if (!v) return fail(RPL_ERR_INVALID_ARG, "rpl_view_reset: view is NULL");
    if (mask == nullptr) {
        v->has_last = true;
        v->last_step = step - 1;
        v->need_first = true;   // the next render (at `step`) sets every env's first step
        return RPL_OK;
    }
    if (!v->has_last || step != v->last_step + 1)
        return fail(RPL_ERR_INVALID_ARG, "rpl_view_reset: with a mask, step must be the next step to render");
    if (v->need_first) return RPL_OK;   // the next render restarts every env at `step` anyway
    if (v->E == 0) return RPL_OK;
    DeviceGuard g(v->scene->device);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    const uint8_t *md = mask;
    cudaError_t e;
    if (pointer_kind(mask, v->scene->device) == PTR_HOST) {
        e = cudaMemcpyAsync(v->mask_stage.p, mask, (size_t)v->E, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) return cuda_fail(e, "rpl_view_reset: copying the mask");
        md = v->mask_stage.as<const uint8_t>();
    }
    e = launch_set_first(v->s_first.as<int64_t>(), v->E, step, md, cs);
    if (e != cudaSuccess) return cuda_fail(e, "rpl_view_reset: launch");
    mark_done(v, cs);
    return RPL_OK;
}

namespace {

struct StateHeader {
    char magic[4];           // "RPLS"
    int32_t version;         // 1
    int32_t E, P, span;
    int32_t flags;           // bit 0 has_last, bit 1 need_first
    int64_t last_step;
    int64_t reserved[4];
};
static_assert(sizeof(StateHeader) == 64, "state header is 64 bytes");

int64_t state_bytes(const rpl_view *v) {
    const int64_t span = (int64_t)v->sensor.max_latency + 1;
    const int64_t ring = span > 1 && v->cams_set ? (int64_t)v->E * span * v->P * (int64_t)sizeof(float) : 0;
    return (int64_t)sizeof(StateHeader) + (int64_t)v->E * (int64_t)sizeof(int64_t) + ring;
}

}  // namespace

RPL_API rpl_status rpl_view_state_size(rpl_view_t v, int64_t *bytes) {
    if (!v || !bytes) return fail(RPL_ERR_INVALID_ARG, "rpl_view_state_size: NULL argument");
    if (!v->cams_set) return fail(RPL_ERR_INVALID_ARG, "rpl_view_state_size: cameras not set");
    *bytes = state_bytes(v);
    return RPL_OK;
}

RPL_API rpl_status rpl_view_state_get(rpl_view_t v, void *buf, int64_t bytes) {
    if (!v || !buf) return fail(RPL_ERR_INVALID_ARG, "rpl_view_state_get: NULL argument");
    if (!v->cams_set) return fail(RPL_ERR_INVALID_ARG, "rpl_view_state_get: cameras not set");
    const int64_t need = state_bytes(v);
    if (bytes < need) return fail(RPL_ERR_INVALID_ARG, "rpl_view_state_get: buffer of %lld bytes, need %lld",
                                  (long long)bytes, (long long)need);
    DeviceGuard g(v->scene->device);
    if (v->has_done) cudaEventSynchronize(v->done);
    StateHeader h{};
    std::memcpy(h.magic, "RPLS", 4);
    h.version = 1;
    h.E = v->E;
    h.P = (int32_t)v->P;
    h.span = v->sensor.max_latency + 1;
    h.flags = (v->has_last ? 1 : 0) | (v->need_first ? 2 : 0);
    h.last_step = v->last_step;
    char *dst = static_cast<char *>(buf);
    cudaError_t e = cudaMemcpy(dst, &h, sizeof h, cudaMemcpyDefault);
    const size_t sf = (size_t)v->E * sizeof(int64_t);
    if (e == cudaSuccess && sf) e = cudaMemcpy(dst + sizeof h, v->s_first.p, sf, cudaMemcpyDefault);
    const size_t ring = (size_t)(need - (int64_t)sizeof h - (int64_t)sf);
    if (e == cudaSuccess && ring) e = cudaMemcpy(dst + sizeof h + sf, v->ring.p, ring, cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_fail(e, "rpl_view_state_get: copying the state");
    return RPL_OK;
}

RPL_API rpl_status rpl_view_state_set(rpl_view_t v, const void *buf, int64_t bytes) {
    if (!v || !buf) return fail(RPL_ERR_INVALID_ARG, "rpl_view_state_set: NULL argument");
    if (!v->cams_set) return fail(RPL_ERR_INVALID_ARG, "rpl_view_state_set: cameras not set");
    const int64_t need = state_bytes(v);
    if (bytes < need) return fail(RPL_ERR_INVALID_ARG, "rpl_view_state_set: %lld bytes, the state has %lld",
                                  (long long)bytes, (long long)need);
    DeviceGuard g(v->scene->device);
    StateHeader h{};
    const char *src = static_cast<const char *>(buf);
    cudaError_t e = cudaMemcpy(&h, src, sizeof h, cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_fail(e, "rpl_view_state_set: reading the header");
    if (std::memcmp(h.magic, "RPLS", 4) != 0 || h.version != 1 || h.E != v->E || h.P != (int32_t)v->P ||
        h.span != v->sensor.max_latency + 1)
        return fail(RPL_ERR_INVALID_ARG, "rpl_view_state_set: the state was saved from a view with other envs, "
                                         "pixels or latency span");
    if (v->has_done) cudaEventSynchronize(v->done);   // an enqueued render may still use the ring
    const size_t sf = (size_t)v->E * sizeof(int64_t);
    if (sf) e = cudaMemcpy(v->s_first.p, src + sizeof h, sf, cudaMemcpyDefault);
    const size_t ring = (size_t)(need - (int64_t)sizeof h - (int64_t)sf);
    if (e == cudaSuccess && ring) e = cudaMemcpy(v->ring.p, src + sizeof h + sf, ring, cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_fail(e, "rpl_view_state_set: copying the state");
    v->has_last = (h.flags & 1) != 0;
    v->need_first = (h.flags & 2) != 0;
    v->last_step = h.last_step;
    v->dev_step_next = INT64_MIN;   // a graph replay resets its device step counter
    return RPL_OK;
}

RPL_API rpl_status rpl_sync(rpl_view_t v) {
    if (!v) return fail(RPL_ERR_INVALID_ARG, "rpl_sync: view is NULL");
    DeviceGuard g(v->scene->device);
    cudaError_t e = v->has_done ? cudaEventSynchronize(v->done) : cudaSuccess;
    if (e != cudaSuccess) return cuda_fail(e, "rpl_sync");
    int32_t w = *(volatile int32_t *)v->err_host;
    if (w != 0) {
        *v->err_host = 0;
        return fail(RPL_ERR_DEVICE_FAULT, "rpl_sync: a render kernel recorded error 0x%x (1: traversal stack overflow, "
                    "4: node or triangle index out of range)", w);
    }
    return RPL_OK;
}

RPL_API rpl_status rpl_view_host_async(rpl_view_t v, int32_t enable) {
    if (!v) return fail(RPL_ERR_INVALID_ARG, "rpl_view_host_async: view is NULL");
    DeviceGuard g(v->scene->device);
    if (enable && !v->copy_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&v->copy_stream, cudaStreamNonBlocking);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
            e = cudaEventCreateWithFlags(&v->rendered[k], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v->copied[k], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_fail(e, "rpl_view_host_async: creating the copy stream");
    }
    if (!enable && v->host_async && v->has_done) cudaEventSynchronize(v->done);
    v->host_async = enable != 0;
    return RPL_OK;
}

RPL_API rpl_status rpl_view_timing(rpl_view_t v, int32_t enable) {
    if (!v) return fail(RPL_ERR_INVALID_ARG, "rpl_view_timing: view is NULL");
    DeviceGuard g(v->scene->device);
    if (enable && !v->ev[0]) {
        for (int i = 0; i < 2 * rpl_view::kTimingSlots; ++i) {
            cudaError_t e = cudaEventCreate(&v->ev[i]);
            if (e != cudaSuccess) return cuda_fail(e, "rpl_view_timing: cudaEventCreate");
        }
    }
    v->timing = enable != 0;
    v->n_timed = 0;
    return RPL_OK;
}

RPL_API rpl_status rpl_view_kernel_ms(rpl_view_t v, float *ms, int32_t max_n, int32_t *n_out) {
    if (!v || !ms || !n_out || max_n < 0) return fail(RPL_ERR_INVALID_ARG, "rpl_view_kernel_ms: bad argument");
    DeviceGuard g(v->scene->device);
    const int64_t avail = std::min<int64_t>(v->n_timed, rpl_view::kTimingSlots);
    const int64_t n = std::min<int64_t>(avail, max_n);
    for (int64_t i = 0; i < n; ++i) {
        const int slot = (int)((v->n_timed - n + i) % rpl_view::kTimingSlots);
        cudaError_t e = cudaEventSynchronize(v->ev[2 * slot + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[i], v->ev[2 * slot], v->ev[2 * slot + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "rpl_view_kernel_ms");
    }
    *n_out = (int32_t)n;
    return RPL_OK;
}

static bool tuning_from(const rpl_tuning *t, Tuning *out) {
    const int lg = t->tile_w == 4 ? 2 : t->tile_w == 8 ? 3 : t->tile_w == 16 ? 4 : -1;
    if (lg < 0 || t->tile_w * t->tile_h != 32 ||
        (t->min_blocks != 8 && t->min_blocks != 9 && t->min_blocks != 10 && t->min_blocks != 12))
        return false;
    out->tile_w_log2 = lg;
    if (t->persistent < 0 || t->persistent > 2 || t->env_order < 0 || t->env_order > 1 || t->chunk_envs < 0 ||
        t->chunk_envs > (1 << 20))
        return false;
    out->persistent = t->persistent;
    out->env_order = t->env_order;
    out->chunk_envs = t->chunk_envs;
    out->terrain_first = t->terrain_first ? 1 : 0;
    out->min_blocks = t->min_blocks;
    return true;
}

static void tuning_to(const Tuning &t, rpl_tuning *out) {
    out->tile_w = 1 << t.tile_w_log2;
    out->tile_h = 32 >> t.tile_w_log2;
    out->persistent = t.persistent;
    out->terrain_first = t.terrain_first;
    out->min_blocks = t.min_blocks;
    out->env_order = t.env_order;
    out->chunk_envs = t.chunk_envs;
}

RPL_API rpl_status rpl_view_tuning_set(rpl_view_t v, const rpl_tuning *t) {
    if (!v || !t) return fail(RPL_ERR_INVALID_ARG, "rpl_view_tuning_set: NULL argument");
    Tuning n;
    if (!tuning_from(t, &n))
        return fail(RPL_ERR_INVALID_ARG, "rpl_view_tuning_set: tile must be 4x8, 8x4 or 16x2, persistent 0, 1 or 2, "
                    "min_blocks 8, 9, 10 or 12, env_order 0 or 1 and chunk_envs 0..2^20");
    v->tune = n;
    return RPL_OK;
}

RPL_API rpl_status rpl_view_tuning_get(rpl_view_t v, rpl_tuning *t) {
    if (!v || !t) return fail(RPL_ERR_INVALID_ARG, "rpl_view_tuning_get: NULL argument");
    tuning_to(v->tune, t);
    return RPL_OK;
}

RPL_API rpl_status rpl_view_autotune(rpl_view_t v, const float *poses, int64_t step, int64_t env_offset, void *out,
                                     void *stream, int32_t reps, rpl_tuning *best, float *best_ms) {
    NvtxRange range("rpl_view_autotune");
    rpl_status st = check_render_args(v, poses, env_offset, out);
    if (st != RPL_OK) return st;
    if (reps < 1) return fail(RPL_ERR_INVALID_ARG, "rpl_view_autotune: reps must be >= 1");
    if (v->has_last && step != v->last_step && step != v->last_step + 1)
        return fail(RPL_ERR_INVALID_ARG, "rpl_view_autotune: step must be the previous step or the next one");
    if (v->E == 0) {
        if (best) tuning_to(v->tune, best);
        if (best_ms) *best_ms = 0.f;
        return RPL_OK;
    }
    rpl_scene *s = v->scene;
    DeviceGuard g(s->device);
    if (pointer_kind(poses, s->device) != PTR_DEVICE || pointer_kind(out, s->device) != PTR_DEVICE)
        return fail(RPL_ERR_INVALID_ARG, "rpl_view_autotune: poses and output must be device memory");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return cuda_fail(e, "rpl_view_autotune: cudaEventCreate");
    }
    const Tuning saved = v->tune;
    const bool saved_timing = v->timing;
    v->timing = false;
    Tuning best_t = saved;
    float best_v = INFINITY;
    const int tiles[3] = {3, 2, 4};
    // (persistent, env_order, chunk_envs): index order or spatial order for each scheduling, and the
    // per-SM queues as contiguous ranges or dealt one env at a time
    const int sched[8][3] = {{0, 0, 0}, {0, 1, 0}, {1, 0, 0}, {1, 1, 0}, {2, 0, 0}, {2, 1, 0}, {2, 0, 1}, {2, 1, 1}};
    for (int ti = 0; ti < 3 && st == RPL_OK; ++ti)
        for (int sc = 0; sc < 8 && st == RPL_OK; ++sc)
            for (int tf = 0; tf < 2 && st == RPL_OK; ++tf)
                for (int mi = 0; mi < 4 && st == RPL_OK; ++mi) {
                    const int mbs[4] = {8, 9, 10, 12};
                    v->tune = Tuning{tiles[ti], sched[sc][0], tf, mbs[mi], sched[sc][1], sched[sc][2]};
                    st = enqueue(v, poses, step, env_offset, out, cs, false, nullptr);   // warm-up
                    if (st != RPL_OK) break;
                    cudaEventRecord(a, cs);
                    for (int r = 0; r < reps && st == RPL_OK; ++r)
                        st = enqueue(v, poses, step, env_offset, out, cs, false, nullptr);
                    cudaEventRecord(b, cs);
                    e = cudaEventSynchronize(b);
                    float ms = 0.f;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
                    if (e != cudaSuccess) st = cuda_fail(e, "rpl_view_autotune: timing");
                    ms /= (float)reps;
                    if (st == RPL_OK && ms < best_v) {
                        best_v = ms;
                        best_t = v->tune;
                    }
                }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    v->timing = saved_timing;
    v->tune = st == RPL_OK ? best_t : saved;
    if (st != RPL_OK) return st;
    v->has_last = true;
    v->last_step = step;
    if (best) tuning_to(best_t, best);
    if (best_ms) *best_ms = best_v;
    return RPL_OK;
}

static void graph_release(rpl_view *v) {
    if (v->gexec) cudaGraphExecDestroy(v->gexec);
    v->gexec = nullptr;
}

RPL_API rpl_status rpl_render_graph(rpl_view_t v, const float *poses, int64_t env_offset, void *out, void *stream,
                                    int64_t *step_out) {
    NvtxRange range("rpl_render_graph");
    rpl_status st = check_render_args(v, poses, env_offset, out);
    if (st != RPL_OK) return st;
    const int64_t next = v->has_last ? v->last_step + 1 : 0;
    if (step_out) *step_out = next;
    if (v->E == 0) {
        v->has_last = true;
        v->last_step = next;
        return RPL_OK;
    }
    rpl_scene *s = v->scene;
    DeviceGuard g(s->device);
    if (pointer_kind(poses, s->device) != PTR_DEVICE || pointer_kind(out, s->device) != PTR_DEVICE)
        return fail(RPL_ERR_INVALID_ARG, "rpl_render_graph: poses and output must be device memory");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (!v->d_step.p) e = v->d_step.alloc(sizeof(int64_t));
    if (e == cudaSuccess && !v->cap_stream) e = cudaStreamCreateWithFlags(&v->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "rpl_render_graph: setting up");
    if (v->need_first) {
        e = launch_set_first(v->s_first.as<int64_t>(), v->E, next, nullptr, cs);
        if (e != cudaSuccess) return cuda_fail(e, "rpl_render_graph: launching the sensor-state reset");
        v->need_first = false;
    }
    const bool same = v->gexec && v->g_poses == poses && v->g_out == out && v->g_env_offset == env_offset &&
                      v->g_gen == v->gen && std::memcmp(&v->g_tune, &v->tune, sizeof(Tuning)) == 0;
    if (!same) {
        graph_release(v);
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(v->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "rpl_render_graph: cudaStreamBeginCapture");
        st = enqueue(v, poses, next, env_offset, out, v->cap_stream, false, nullptr, v->d_step.as<const int64_t>());
        if (st == RPL_OK) {
            e = launch_advance_step(v->d_step.as<int64_t>(), v->cap_stream);
            if (e != cudaSuccess) st = cuda_fail(e, "rpl_render_graph: capturing the step advance");
        }
        const cudaError_t ec = cudaStreamEndCapture(v->cap_stream, &graph);
        if (st == RPL_OK && ec != cudaSuccess) st = cuda_fail(ec, "rpl_render_graph: cudaStreamEndCapture");
        if (st == RPL_OK) {
            e = cudaGraphInstantiate(&v->gexec, graph, 0);
            if (e != cudaSuccess) {
                v->gexec = nullptr;
                st = cuda_fail(e, "rpl_render_graph: cudaGraphInstantiate");
            }
        }
        if (graph) cudaGraphDestroy(graph);
        if (st != RPL_OK) return st;
        v->g_poses = poses;
        v->g_out = out;
        v->g_env_offset = env_offset;
        v->g_gen = v->gen;
        v->g_tune = v->tune;
    }
    if (v->dev_step_next != next) {
        // the counter is out of step (first replay, or rpl_render ran in between): set it in stream order
        e = launch_set_first(v->d_step.as<int64_t>(), 1, next, nullptr, cs);
        if (e != cudaSuccess) return cuda_fail(e, "rpl_render_graph: setting the step counter");
    }
    e = cudaGraphLaunch(v->gexec, cs);
    if (e != cudaSuccess) return cuda_fail(e, "rpl_render_graph: cudaGraphLaunch");
    v->dev_step_next = next + 1;
    v->has_last = true;
    v->last_step = next;
    mark_done(v, cs);
    return RPL_OK;
}

RPL_API void rpl_view_destroy(rpl_view_t v) {
    if (!v) return;
    {
        DeviceGuard g(v->scene->device);
        if (v->has_done) cudaEventSynchronize(v->done);
        if (v->done) cudaEventDestroy(v->done);
        if (v->err_host) cudaFreeHost(v->err_host);
        for (int i = 0; i < 2 * rpl_view::kTimingSlots; ++i)
            if (v->ev[i]) cudaEventDestroy(v->ev[i]);
        graph_release(v);
        if (v->cap_stream) cudaStreamDestroy(v->cap_stream);
        for (int k = 0; k < 2; ++k) {
            if (v->rendered[k]) cudaEventDestroy(v->rendered[k]);
            if (v->copied[k]) cudaEventDestroy(v->copied[k]);
        }
        if (v->copy_stream) cudaStreamDestroy(v->copy_stream);
    }
    rpl_scene *s = v->scene;
    delete v;
    scene_release(s, false);
}

}  // extern "C"

namespace rpl {

rpl_status check_camera(const rpl_camera &k, int c, int32_t n_links, const char *who) {
    if (k.width <= 0 || k.height <= 0 || k.width > 16384 || k.height > 16384)
        return fail(RPL_ERR_INVALID_ARG, "%s: camera %d size %dx%d", who, c, k.width, k.height);
    const int32_t ds = k.downsample <= 1 ? 1 : k.downsample;
    if (k.downsample < 0 || k.downsample > 16 || k.width % ds != 0 || k.height % ds != 0)
        return fail(RPL_ERR_INVALID_ARG, "%s: camera %d downsample %d must be 0..16 and divide %dx%d", who, c,
                    k.downsample, k.width, k.height);
    if (!(k.fx != 0.f) || !(k.fy != 0.f) || !std::isfinite(k.fx) || !std::isfinite(k.fy) || !std::isfinite(k.cx) ||
        !std::isfinite(k.cy))
        return fail(RPL_ERR_INVALID_ARG, "%s: camera %d needs finite intrinsics with fx, fy != 0", who, c);
    if (k.mount_link < 0 || k.mount_link >= n_links)
        return fail(RPL_ERR_INVALID_ARG, "%s: camera %d mount_link %d outside 0..%d", who, c, k.mount_link,
                    n_links - 1);
    if (!(k.d_min <= k.d_max) || !(k.d_max > 0.f) || !std::isfinite(k.d_max) || !std::isfinite(k.d_min))
        return fail(RPL_ERR_INVALID_ARG, "%s: camera %d needs finite 0 < d_max, d_min <= d_max", who, c);
    double qn = 0.0;
    for (int a = 0; a < 4; ++a) qn += (double)k.offset_quat_xyzw[a] * k.offset_quat_xyzw[a];
    if (!std::isfinite(k.offset_pos[0]) || !std::isfinite(k.offset_pos[1]) || !std::isfinite(k.offset_pos[2]) ||
        !(qn > 0.0) || !std::isfinite(qn))
        return fail(RPL_ERR_INVALID_ARG, "%s: camera %d needs a finite mount offset and a nonzero quaternion", who, c);
    return RPL_OK;
}

bool scene_inputs(const rpl_scene *s, SceneInputs *out) {
    if (!s) return false;
    std::lock_guard<std::mutex> lk(const_cast<rpl_scene *>(s)->mu);
    if (!s->frozen) return false;
    out->device = s->device;
    out->bvh_kind = s->opts.bvh_kind;
    out->tnodes = s->t_nodes.as<const float4>();
    out->n_tnodes = terrain_node_count(s);
    out->n_ttris = (int64_t)(s->t_tris.bytes / sizeof(BvhTri));
    out->n_lnodes = (int64_t)(s->l_nodes.bytes / sizeof(BvhNode));
    out->n_ltris = (int64_t)(s->l_tris.bytes / sizeof(BvhTri));
    out->ttris = s->t_tris.as<const float4>();
    out->lnodes = s->l_nodes.as<const float4>();
    out->ltris = s->l_tris.as<const float4>();
    out->link_root = s->l_roots.as<const float4>();
    for (int l = 0; l < RPL_MAX_LINKS; ++l) out->lroot[l] = s->l_root[l];
    return true;
}

rpl_status set_error(rpl_status st, const char *msg) { return fail(st, "%s", msg); }

rpl_status view_validate(rpl_view *v, const float *poses, int64_t env_offset, void *out) {
    return check_render_args(v, poses, env_offset, out);
}

bool view_step_allowed(const rpl_view *v, int64_t step) {
    return !v->has_last || step == v->last_step || step == v->last_step + 1;
}

rpl_status view_prepare(rpl_view *v, const float *poses_dev, int64_t step, int64_t env_offset, void *out_dev,
                        cudaStream_t st, RenderParams *rp, int64_t *warps) {
    PrepParams pp;
    rpl_status s = build_params(v, poses_dev, step, env_offset, out_dev, st, nullptr, nullptr, pp, *rp);
    if (s != RPL_OK) return s;
    pp.queues = rp->queues = nullptr;   // the fused launch schedules its own tiles
    pp.env_key = nullptr;
    rp->env_order = nullptr;
    cudaError_t e = launch_prep(pp, st);
    if (e != cudaSuccess) return cuda_fail(e, "launching the prep kernel");
    e = launch_tile_prep(*rp, st);
    if (e != cudaSuccess) return cuda_fail(e, "launching the tile-prep kernel");
    *warps = (int64_t)rp->E * rp->tiles_per_env;
    return RPL_OK;
}

void view_commit(rpl_view *v, int64_t step, cudaStream_t st) {
    (void)st;
    v->has_last = true;
    v->last_step = step;
}

void view_mark_done(rpl_view *v, cudaStream_t st) { mark_done(v, st); }

size_t view_pose_bytes(const rpl_view *v) { return (size_t)v->E * v->L * 7 * sizeof(float); }
size_t view_out_bytes(const rpl_view *v) { return (size_t)v->E * v->P * out_elem_bytes(v); }
int32_t view_envs(const rpl_view *v) { return v->E; }
rpl_scene *view_scene(const rpl_view *v) { return v->scene; }
Tuning view_tuning(const rpl_view *v) { return v->tune; }
int scene_device_of(const rpl_scene *s) { return s->device; }
int scene_bvh_kind(const rpl_scene *s) { return s->opts.bvh_kind; }
bool pointer_on_device(const void *p, int device) { return pointer_kind(p, device) == PTR_DEVICE; }

void scene_add_server(rpl_scene *s) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->servers++;
}

void scene_remove_server(rpl_scene *s) { scene_release(s, true); }

}  // namespace rpl
