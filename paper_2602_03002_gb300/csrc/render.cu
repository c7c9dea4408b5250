// render.cu -- sm_103a kernels of the multi-depth ray-casting path (Sec. 3.2.2, Algorithm 1) and of
// the depth-sensor model (Appendix A.2).
//
//   prep_kernel    one thread per (env, link): normalised link rotation, world->link transform and
//                  the link's world AABB; four threads per (env, camera): camera pose = link pose
//                  composed with the (optionally per-env randomised) mount offset, the links in the
//                  camera's view volume, its terrain entry node and latency word.
//   tile_prep_kernel  one thread per 32-pixel tile: terrain entry subtrees and link mask of the tile.
//   render_kernel  one thread per pixel ray, one warp per 32-pixel tile of one (env, camera):
//                  BuildDepthRay -> links whose world AABB the ray meets within the running bound
//                  (ray moved into the link frame, link BVH traversed, bound shrinks on each hit)
//                  -> terrain BVH traversal with the bound (the order of the two queries is a
//                  launch-shape option; links first, Alg. 1's order, by default) -> far-plane clip
//                  -> fused sensor model
//                  (ring-buffer write, latency select, noise, clip, dropout, side mask) -> store;
//                  rays of a downsampled camera store their raw depth instead.
//   downsample_kernel  one thread per output pixel of a downsampled camera: mean of its raw block
//                  -> the same sensor epilogue -> store.
//
// The path is pointer chasing, not a dense contraction, so it runs on the SIMT pipes: node and
// triangle fetches are 16-byte read-only vector loads, the per-ray stack is short, rays of a warp
// are a compact pixel tile so their fetches coalesce and hit the same cache lines.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <climits>

#include "render.h"

namespace rpl {
namespace {

// Bounds-checked build (RPL_CHECKED, librpl_checked.so): every node and triangle index is tested
// against the length of its array before it is read; a violation sets bit 4 of the view's error
// word and ends that ray's walk instead of reading.  In the normal build the macros below expand to
// nothing, so its kernels are exactly the unchecked code.
#ifdef RPL_CHECKED
__device__ __forceinline__ bool in_range(int64_t i, int64_t n) { return (uint64_t)i < (uint64_t)n; }
constexpr uint32_t kErrBounds = 4;
#define RPL_CK_PARAMS , int64_t ck_nodes, int64_t ck_tris, uint32_t &ck_err
#define RPL_CK_ARGS(n, t, e) , (n), (t), (e)
#define RPL_CK_NODE(i, on_fail)                                                                        \
    if (!in_range((i), ck_nodes)) {                                                                  \
        ck_err |= kErrBounds;                                                                        \
        on_fail;                                                                                     \
    }
#define RPL_CK_DESCEND_PARAMS , int64_t ck_nodes
#define RPL_CK_DESCEND_ARGS(n) , (n)
#define RPL_CK_PUSH(sp, on_fail)                                                                       \
    if ((sp) >= kStackDepth) {                                                                       \
        ck_err |= kErrBounds;                                                                        \
        on_fail;                                                                                     \
    }
#else
#define RPL_CK_PARAMS
#define RPL_CK_ARGS(n, t, e)
#define RPL_CK_NODE(i, on_fail)
#define RPL_CK_DESCEND_PARAMS
#define RPL_CK_DESCEND_ARGS(n)
#define RPL_CK_PUSH(sp, on_fail)
#endif

// ---------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
// the key advanced by the Weyl constants between rounds.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 sensor_words(uint32_t env, uint32_t cam, uint32_t pix, int64_t step,
                                              uint32_t seed0, uint32_t seed1) {
    const uint64_t s = (uint64_t)step;
    return philox10(make_uint4(env, cam, pix, (uint32_t)s), seed0 ^ (uint32_t)(s >> 32), seed1);
}

// Latency word of (env, camera, step): the delay k = (w0 (Lmax + 1)) >> 32 drawn from the word with
// pixel field 0xFFFFFFFF, the source step s' = max(s - k, first step since reset) stored as s - s' in
// bits 0..7, and the ring slot s mod span in bits 8..15 (span = Lmax + 1 <= 16), so that the
// per-pixel sensor code needs no 64-bit division.  0 when latency is off.
__device__ __forceinline__ uint32_t latency_word(uint32_t env, uint32_t cam, int64_t step, int64_t first,
                                                 uint32_t span, uint32_t seed0, uint32_t seed1) {
    if (span <= 1) return 0u;
    const uint4 wl = sensor_words(env, cam, 0xFFFFFFFFu, step, seed0, seed1);
    int64_t src = step - (int64_t)__umulhi(wl.x, span);
    if (src < first) src = first;
    if (src > step) src = step;
    int64_t slot = step % (int64_t)span;
    if (slot < 0) slot += span;
    return (uint32_t)(step - src) | ((uint32_t)slot << 8);
}

// Rotation matrix (row-major) of a quaternion (x, y, z, w), normalised in FP32.
__device__ __forceinline__ void quat_rot(float x, float y, float z, float w, float R[9]) {
    const float inv = 1.0f / sqrtf(x * x + y * y + z * z + w * w);
    x *= inv; y *= inv; z *= inv; w *= inv;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - z * w);       R[2] = 2.f * (x * z + y * w);
    R[3] = 2.f * (x * y + z * w);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - x * w);
    R[6] = 2.f * (x * z - y * w);       R[7] = 2.f * (y * z + x * w);       R[8] = 1.f - 2.f * (x * x + y * y);
}

__device__ __forceinline__ float pad_lo(float v) { return v - (fabsf(v) * 0x1p-18f + 1e-5f); }
__device__ __forceinline__ float pad_hi(float v) { return v + (fabsf(v) * 0x1p-18f + 1e-5f); }

// World AABB of link l of env e (the link-frame root box moved by the link pose), padded outward.
// Returns false for a link without a mesh.
__device__ __forceinline__ bool link_world_box(const PrepParams &p, int64_t el, int l, const float R[9],
                                               float lo_out[3], float hi_out[3]) {
    const float *q = p.poses + 7 * el;
    const float4 lo = p.link_root[2 * l], hi = p.link_root[2 * l + 1];
    if (!(lo.x <= hi.x)) return false;
    const float cx = 0.5f * (lo.x + hi.x), cy = 0.5f * (lo.y + hi.y), cz = 0.5f * (lo.z + hi.z);
    const float hx = 0.5f * (hi.x - lo.x), hy = 0.5f * (hi.y - lo.y), hz = 0.5f * (hi.z - lo.z);
    const float w[3] = {R[0] * cx + R[1] * cy + R[2] * cz + q[0], R[3] * cx + R[4] * cy + R[5] * cz + q[1],
                        R[6] * cx + R[7] * cy + R[8] * cz + q[2]};
    // slack covers the rounding of the centre/extent arithmetic above
    const float ext[3] = {fabsf(R[0]) * hx + fabsf(R[1]) * hy + fabsf(R[2]) * hz + 1e-6f,
                          fabsf(R[3]) * hx + fabsf(R[4]) * hy + fabsf(R[5]) * hz + 1e-6f,
                          fabsf(R[6]) * hx + fabsf(R[7]) * hy + fabsf(R[8]) * hz + 1e-6f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo_out[a] = pad_lo(w[a] - ext[a]);
        hi_out[a] = pad_hi(w[a] + ext[a]);
    }
    return true;
}

__device__ __forceinline__ bool boxes_overlap(float alx, float ahx, float aly, float ahy, float alz, float ahz,
                                              const float blo[3], const float bhi[3]) {
    return alx <= bhi[0] && blo[0] <= ahx && aly <= bhi[1] && blo[1] <= ahy && alz <= bhi[2] && blo[2] <= ahz;
}

// The view pyramid of a rectangle of pixels: apex o (the camera origin) and far face at z-depth d_max
// through the rectangle's corner pixels.  Every ray segment of those pixels lies inside it, for
// z-depth and for range depth (a range segment of length d_max ends at z-depth
// d_max / |(r_x, r_y, 1)| <= d_max), since the pixel directions R_c (r_x, r_y, 1) are affine in the
// pixel coordinates.  Holds the padded AABB, the four side planes' unit normals oriented inward
// (towards the mean corner direction, which lies inside the pyramid even when the optical axis does
// not) and the optical axis for the far plane.
struct Pyramid {
    float o[3], V[4][3], N[4][3], tol[4], axis[3], d_max;
    float lo[3], hi[3];
};

// B: far corners o + d_max R_c (r_x, r_y, 1) in ring order around the rectangle.
__device__ __forceinline__ void make_pyramid(Pyramid &P, const float o[3], const float B[4][3], const float axis[3],
                                             float d_max) {
    float mean[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        P.o[a] = o[a];
#pragma unroll
        for (int k = 0; k < 4; ++k) P.V[k][a] = B[k][a];
        P.axis[a] = axis[a];
        float lo = fminf(fminf(o[a], fminf(B[0][a], B[1][a])), fminf(B[2][a], B[3][a]));
        float hi = fmaxf(fmaxf(o[a], fmaxf(B[0][a], B[1][a])), fmaxf(B[2][a], B[3][a]));
        const float slack = 1e-3f + 1e-5f * fmaxf(fabsf(lo), fabsf(hi));
        P.lo[a] = lo - slack;
        P.hi[a] = hi + slack;
        mean[a] = (B[0][a] - o[a]) + (B[1][a] - o[a]) + (B[2][a] - o[a]) + (B[3][a] - o[a]);
    }
    P.d_max = d_max;
    // reach of the pyramid (its farthest points are the far corners) and size of the apex coordinates
    float reach = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        reach = fmaxf(reach, sqrtf((B[k][0] - o[0]) * (B[k][0] - o[0]) + (B[k][1] - o[1]) * (B[k][1] - o[1]) +
                                   (B[k][2] - o[2]) * (B[k][2] - o[2])));
    const float omag = fmaxf(fmaxf(fabsf(o[0]), fabsf(o[1])), fabsf(o[2]));
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const float *a = B[s], *b = B[(s + 1) & 3];
        const float u[3] = {a[0] - o[0], a[1] - o[1], a[2] - o[2]}, v[3] = {b[0] - o[0], b[1] - o[1], b[2] - o[2]};
        const float n[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
        const float lu = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        const float lv = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        const float ln = sqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        // sine of the angle between the side's two corner rays.  Where they are (nearly) parallel --
        // a rectangle one pixel wide repeats a corner -- the FP32 cross product is rounding noise
        // (not zero: the compiler may contract it into FMAs), so the side culls nothing.
        const float sin_t = lu > 0.f && lv > 0.f ? ln / (lu * lv) : 0.f;
        if (!(sin_t >= 1e-5f)) {
            P.N[s][0] = P.N[s][1] = P.N[s][2] = 0.f;
            P.tol[s] = 0.f;
            continue;
        }
        // unit normal, oriented inward.  Its direction is off by at most delta (radians): the
        // rounding of the corner directions (relative to the apex coordinates and the reach) and of
        // the cross product, divided by sin_t; a point of the pyramid then lies up to reach * delta
        // behind the computed plane, which the tolerance adds to the 1 mm padding.
        const float delta = (1e-6f + 2e-7f * (omag + reach) / fminf(lu, lv)) / sin_t;
        P.tol[s] = 1e-3f + reach * delta;
        float inv = 1.0f / ln;
        if (n[0] * mean[0] + n[1] * mean[1] + n[2] * mean[2] < 0.f) inv = -inv;
        P.N[s][0] = n[0] * inv; P.N[s][1] = n[1] * inv; P.N[s][2] = n[2] * inv;
    }
}

// The plane part of pyramid_meets_box (the box is already known to meet the pyramid's AABB).
__device__ __forceinline__ bool pyramid_planes_meet_box(const Pyramid &P, const float lo[3], const float hi[3]) {
    bool inside = true;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        // the box corner farthest along the inward normal must not be behind the plane
        const float *n = P.N[s];
        const float d = n[0] * ((n[0] >= 0.f ? hi[0] : lo[0]) - P.o[0]) + n[1] * ((n[1] >= 0.f ? hi[1] : lo[1]) - P.o[1]) +
                        n[2] * ((n[2] >= 0.f ? hi[2] : lo[2]) - P.o[2]);
        inside &= d >= -P.tol[s];
    }
    // far plane: the box corner nearest along the optical axis must lie within d_max
    const float *ax = P.axis;
    const float zn = ax[0] * ((ax[0] >= 0.f ? lo[0] : hi[0]) - P.o[0]) + ax[1] * ((ax[1] >= 0.f ? lo[1] : hi[1]) - P.o[1]) +
                     ax[2] * ((ax[2] >= 0.f ? lo[2] : hi[2]) - P.o[2]);
    return inside && zn <= P.d_max + 1e-3f;
}

// Conservative test of a world box against the pyramid: false only when the box lies outside the
// padded AABB, behind a side plane by more than that side's tolerance or beyond the far plane by
// more than 1 mm.
__device__ __forceinline__ bool pyramid_meets_box(const Pyramid &P, const float lo[3], const float hi[3]) {
    return boxes_overlap(lo[0], hi[0], lo[1], hi[1], lo[2], hi[2], P.lo, P.hi) && pyramid_planes_meet_box(P, lo, hi);
}

// Conservative separating-axis test of the pyramid against an oriented box: centre c, unit axes
// A[i] (world), half extents h[i].  The box is kept unless one of the pyramid's four side planes or
// its far plane, or one of the box's three face axes, separates the two by more than the side's
// tolerance (1 mm for the far plane and the box axes).  (The
// edge-cross-product axes are left out: without them the test can only keep more, never less.)
__device__ __forceinline__ bool pyramid_meets_obb(const Pyramid &P, const float c[3], const float A[3][3],
                                                  const float h[3]) {
    const float co[3] = {c[0] - P.o[0], c[1] - P.o[1], c[2] - P.o[2]};
    bool inside = true;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        // support of the box along the inward normal must reach the plane
        const float *n = P.N[s];
        const float r = h[0] * fabsf(n[0] * A[0][0] + n[1] * A[0][1] + n[2] * A[0][2]) +
                        h[1] * fabsf(n[0] * A[1][0] + n[1] * A[1][1] + n[2] * A[1][2]) +
                        h[2] * fabsf(n[0] * A[2][0] + n[1] * A[2][1] + n[2] * A[2][2]);
        inside &= n[0] * co[0] + n[1] * co[1] + n[2] * co[2] + r >= -P.tol[s];
    }
    {
        const float *ax = P.axis;
        const float r = h[0] * fabsf(ax[0] * A[0][0] + ax[1] * A[0][1] + ax[2] * A[0][2]) +
                        h[1] * fabsf(ax[0] * A[1][0] + ax[1] * A[1][1] + ax[2] * A[1][2]) +
                        h[2] * fabsf(ax[0] * A[2][0] + ax[1] * A[2][1] + ax[2] * A[2][2]);
        inside &= ax[0] * co[0] + ax[1] * co[1] + ax[2] * co[2] - r <= P.d_max + 1e-3f;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        // the pyramid's vertices projected on the box axis must overlap [-h, h] around the centre
        const float *a = A[i];
        float lo = -(a[0] * co[0] + a[1] * co[1] + a[2] * co[2]), hi = lo;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float q = a[0] * (P.V[k][0] - c[0]) + a[1] * (P.V[k][1] - c[1]) + a[2] * (P.V[k][2] - c[2]);
            lo = fminf(lo, q);
            hi = fmaxf(hi, q);
        }
        inside &= lo <= h[i] + 1e-3f && hi >= -h[i] - 1e-3f;
    }
    return inside;
}

// Deepest binary node below `node` that holds everything inside the AABB [lo, hi]: descend while
// exactly one child's box meets the AABB and that child is an inner node.
__device__ __forceinline__ int descend_binary(const float4 *__restrict__ nodes, int node, const float lo[3],
                                              const float hi[3] RPL_CK_DESCEND_PARAMS) {
#pragma unroll 1
    for (int depth = 0; depth < kStackDepth; ++depth) {
        const float4 *n = nodes + 4 * node;
        const float4 n0 = __ldg(n), n1 = __ldg(n + 1), n2 = __ldg(n + 2);
        const int4 n3 = __ldg(reinterpret_cast<const int4 *>(n + 3));
        const bool h0 = !(n3.x < 0 && n3.z == 0) && boxes_overlap(n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, lo, hi);
        const bool h1 = !(n3.y < 0 && n3.w == 0) && boxes_overlap(n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, lo, hi);
        int next = -1;
        if (h0 && !h1 && n3.x >= 0) next = n3.x;
        if (h1 && !h0 && n3.y >= 0) next = n3.y;
        if (next < 0) break;
#ifdef RPL_CHECKED
        if (!in_range(next, ck_nodes)) break;
#endif
        node = next;
    }
    return node;
}

// Descent of the binary layout against a tile's view pyramid: from `node`, step into the one child
// whose box meets the pyramid while that child is an inner node.  Returns the node where it stops;
// when it stops because both children meet the pyramid and both are inner nodes, they are returned
// in ca, cb (else -1).  The pyramid test is conservative, so no ray of the tile reaches a triangle
// outside the subtree of the returned node.  The plane tests run only where both children meet the
// pyramid's AABB: where one child alone does, stepping into it is safe whether or not the pyramid
// itself meets it (if it does not, no ray reaches anything below this node at all).
// One step of that descent on the fetched node n0..n3: the child to step into, or -1 where the
// descent stops (then ca, cb receive both children when both meet the pyramid and are inner nodes).
__device__ __forceinline__ int pyramid_step(const float4 &n0, const float4 &n1, const float4 &n2, const int4 &n3,
                                            const Pyramid &P, int &ca, int &cb) {
    // empty children of the device layout sit at 1e30 and meet no pyramid
    const float lo0[3] = {n0.x, n0.z, n2.x}, hi0[3] = {n0.y, n0.w, n2.y};
    const float lo1[3] = {n1.x, n1.z, n2.z}, hi1[3] = {n1.y, n1.w, n2.w};
    bool h0 = boxes_overlap(lo0[0], hi0[0], lo0[1], hi0[1], lo0[2], hi0[2], P.lo, P.hi);
    bool h1 = boxes_overlap(lo1[0], hi1[0], lo1[1], hi1[1], lo1[2], hi1[2], P.lo, P.hi);
    if (h0 && h1) {
        h0 = pyramid_planes_meet_box(P, lo0, hi0);
        h1 = pyramid_planes_meet_box(P, lo1, hi1);
    }
    if (h0 && h1) {
        if (n3.x >= 0 && n3.y >= 0) {
            ca = n3.x;
            cb = n3.y;
        }
        return -1;
    }
    return h0 ? n3.x : (h1 ? n3.y : -1);
}

__device__ __forceinline__ int descend_binary_pyramid(const float4 *__restrict__ nodes, int node, const Pyramid &P,
                                                      int &ca, int &cb RPL_CK_DESCEND_PARAMS) {
    ca = cb = -1;
#pragma unroll 1
    for (int depth = 0; depth < kStackDepth; ++depth) {
        const float4 *n = nodes + 4 * node;
        const float4 n0 = __ldg(n), n1 = __ldg(n + 1), n2 = __ldg(n + 2);
        const int4 n3 = __ldg(reinterpret_cast<const int4 *>(n + 3));
        const int next = pyramid_step(n0, n1, n2, n3, P, ca, cb);
        if (next < 0) break;
#ifdef RPL_CHECKED
        if (!in_range(next, ck_nodes)) break;
#endif
        node = next;
    }
    return node;
}

// The same descent from two nodes at once (the two children of a node the pyramid splits), so that
// the two chains of dependent node fetches overlap; a, b become the nodes where each one stops.
__device__ __forceinline__ void descend_binary_pyramid2(const float4 *__restrict__ nodes, int &a, int &b,
                                                        const Pyramid &P RPL_CK_DESCEND_PARAMS) {
    bool go_a = true, go_b = true;
    int xa, xb;
#pragma unroll 1
    for (int depth = 0; depth < kStackDepth && (go_a || go_b); ++depth) {
        const float4 *na = nodes + 4 * a, *nb = nodes + 4 * b;
        float4 a0, a1, a2, b0, b1, b2;
        int4 a3, b3;
        if (go_a) {
            a0 = __ldg(na); a1 = __ldg(na + 1); a2 = __ldg(na + 2);
            a3 = __ldg(reinterpret_cast<const int4 *>(na + 3));
        }
        if (go_b) {
            b0 = __ldg(nb); b1 = __ldg(nb + 1); b2 = __ldg(nb + 2);
            b3 = __ldg(reinterpret_cast<const int4 *>(nb + 3));
        }
        if (go_a) {
            const int next = pyramid_step(a0, a1, a2, a3, P, xa, xb);
#ifdef RPL_CHECKED
            go_a = next >= 0 && in_range(next, ck_nodes);
#else
            go_a = next >= 0;
#endif
            if (go_a) a = next;
        }
        if (go_b) {
            const int next = pyramid_step(b0, b1, b2, b3, P, xa, xb);
#ifdef RPL_CHECKED
            go_b = next >= 0 && in_range(next, ck_nodes);
#else
            go_b = next >= 0;
#endif
            if (go_b) b = next;
        }
    }
}

// Squared distance from point o to the box [lo, hi].
__device__ __forceinline__ float box_dist2(const float o[3], const float lo[3], const float hi[3]) {
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float d = fmaxf(fmaxf(lo[a] - o[a], o[a] - hi[a]), 0.f);
        s += d * d;
    }
    return s;
}

// The same for the eight-wide layout (defined with the wide traversal below).
__device__ __forceinline__ int descend_wide(const float4 *__restrict__ nodes, int node, const float lo[3],
                                            const float hi[3] RPL_CK_DESCEND_PARAMS);
__device__ __forceinline__ int descend4(const float4 *__restrict__ nodes, int node, const float lo[3],
                                        const float hi[3] RPL_CK_DESCEND_PARAMS);

// Entry node of the terrain walk for the layout `kind` (rpl_bvh_kind).
__device__ __forceinline__ int descend_any(int kind, const float4 *__restrict__ nodes, int node, const float lo[3],
                                           const float hi[3] RPL_CK_DESCEND_PARAMS) {
#ifdef RPL_CHECKED
    if (!in_range(node, ck_nodes)) node = 0;
#endif
    if (kind == RPL_BVH8Q8) return descend_wide(nodes, node, lo, hi RPL_CK_DESCEND_ARGS(ck_nodes));
    if (kind == RPL_BVH4) return descend4(nodes, node, lo, hi RPL_CK_DESCEND_ARGS(ck_nodes));
    return descend_binary(nodes, node, lo, hi RPL_CK_DESCEND_ARGS(ck_nodes));
}

__global__ void __launch_bounds__(256) prep_kernel(const __grid_constant__ PrepParams p) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p.queues)   // the render kernel's tile queues start empty
        for (int64_t k = i; k < p.n_queues; k += (int64_t)gridDim.x * blockDim.x) p.queues[k] = 0ull;
    const int64_t n_link = (int64_t)p.E * p.L;
    if (i < n_link) {
        const int l = (int)(i % p.L);
        const float *q = p.poses + 7 * i;
        if (l == 0 && p.env_key) {
            // spatial key of the env: Morton index of link 0's cell on a 64 x 64 grid over the terrain
            uint32_t cell[2];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const float span = p.xy_hi[a] - p.xy_lo[a];
                const float u = span > 0.f ? (q[a] - p.xy_lo[a]) / span * 64.f : 0.f;
                cell[a] = u >= 0.f ? (uint32_t)fminf(u, 63.f) : 0u;   // NaN and below the grid -> 0
            }
            uint32_t m = 0;
#pragma unroll
            for (int b = 0; b < 6; ++b) m |= (((cell[0] >> b) & 1u) << (2 * b)) | (((cell[1] >> b) & 1u) << (2 * b + 1));
            p.env_key[i / p.L] = m;
        }
        float R[9];
        quat_rot(q[3], q[4], q[5], q[6], R);
        p.link_xf[3 * i + 0] = make_float4(R[0], R[3], R[6], q[0]);
        p.link_xf[3 * i + 1] = make_float4(R[1], R[4], R[7], q[1]);
        p.link_xf[3 * i + 2] = make_float4(R[2], R[5], R[8], q[2]);
        float lo[3], hi[3];
        if (!link_world_box(p, i, l, R, lo, hi)) {
            lo[0] = lo[1] = lo[2] = hi[0] = hi[1] = hi[2] = 1e30f;
        }
        p.link_box[2 * i + 0] = make_float4(lo[0], lo[1], lo[2], 0.f);
        p.link_box[2 * i + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
        return;
    }
    // four consecutive threads per (env, camera), from the first warp boundary after the link threads
    // on: each tests a quarter of the links against the view volume, so that the camera's chain of
    // work is a quarter as long
    const int64_t cam0 = (n_link + 31) & ~(int64_t)31;
    if (i < cam0) return;
    const int64_t j = (i - cam0) >> 2;
    const int sub = (int)((i - cam0) & 3);
    if (j >= (int64_t)p.E * p.C) return;
    const int e = (int)(j / p.C), c = (int)(j % p.C);
    const CamDev &cam = p.cams[c];
    const float *q = p.poses + 7 * ((int64_t)e * p.L + cam.mount);
    float Rl[9], Ro[9];
    quat_rot(q[3], q[4], q[5], q[6], Rl);
    quat_rot(cam.off_quat[0], cam.off_quat[1], cam.off_quat[2], cam.off_quat[3], Ro);
    float op[3] = {cam.off_pos[0], cam.off_pos[1], cam.off_pos[2]};
    if (p.mount_dr) {
        // randomised mount of this env: offset + dp, rotation R_off R(dq) (dq about the camera's axes)
        const float *dr = p.mount_dr + 7 * j;
        float Rd[9], Rm[9];
        quat_rot(dr[3], dr[4], dr[5], dr[6], Rd);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                Rm[3 * r + k] = Ro[3 * r + 0] * Rd[k] + Ro[3 * r + 1] * Rd[3 + k] + Ro[3 * r + 2] * Rd[6 + k];
#pragma unroll
        for (int k = 0; k < 9; ++k) Ro[k] = Rm[k];
        op[0] += dr[0];
        op[1] += dr[1];
        op[2] += dr[2];
    }
    float Rc[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            Rc[3 * r + k] = Rl[3 * r + 0] * Ro[k] + Rl[3 * r + 1] * Ro[3 + k] + Rl[3 * r + 2] * Ro[6 + k];
    const float ox = Rl[0] * op[0] + Rl[1] * op[1] + Rl[2] * op[2];
    const float oy = Rl[3] * op[0] + Rl[4] * op[1] + Rl[5] * op[2];
    const float oz = Rl[6] * op[0] + Rl[7] * op[1] + Rl[8] * op[2];
    if (sub == 0) {
        p.cam_xf[5 * j + 0] = make_float4(Rc[0], Rc[1], Rc[2], q[0]);
        p.cam_xf[5 * j + 1] = make_float4(Rc[3], Rc[4], Rc[5], q[1]);
        p.cam_xf[5 * j + 2] = make_float4(Rc[6], Rc[7], Rc[8], q[2]);
        p.cam_xf[5 * j + 3] = make_float4(ox, oy, oz, 0.f);
    }

    // The camera's view volume: apex o, far face at z-depth d_max through the four corner pixels.
    // Every pixel ray segment of this camera (z-depth or range) lies inside it.
    float fx = cam.fx, fy = cam.fy, pcx = cam.cx, pcy = cam.cy;
    if (p.intr) {
        const float4 k = reinterpret_cast<const float4 *>(p.intr)[(int64_t)e * p.C + c];
        fx = k.x; fy = k.y; pcx = k.z; pcy = k.w;
    }
    const float o[3] = {q[0] + ox, q[1] + oy, q[2] + oz};
    float B[4][3];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        // ring order: (0, 0), (w - 1, 0), (w - 1, h - 1), (0, h - 1)
        const float rx = ((k == 1 || k == 2) ? (float)(cam.width - 1) - pcx : -pcx) / fx;
        const float ry = (k >= 2 ? (float)(cam.height - 1) - pcy : -pcy) / fy;
#pragma unroll
        for (int a = 0; a < 3; ++a) B[k][a] = o[a] + cam.d_max * (Rc[3 * a] * rx + Rc[3 * a + 1] * ry + Rc[3 * a + 2]);
    }
    Pyramid V;
    const float axis[3] = {Rc[2], Rc[5], Rc[8]};
    make_pyramid(V, o, B, axis, cam.d_max);

    // 1) links whose world AABB meets the view pyramid: links sub, sub + 4, ... by each of the four
    //    threads, the masks OR-ed across them (the four are consecutive lanes of one warp)
    uint64_t mask = 0;
    for (int l = sub; l < p.L; l += 4) {
        if (p.lroot[l] < 0) continue;
        const int64_t el = (int64_t)e * p.L + l;
        const float *ql = p.poses + 7 * el;
        float R[9], lo[3], hi[3];
        quat_rot(ql[3], ql[4], ql[5], ql[6], R);
        if (!link_world_box(p, el, l, R, lo, hi)) continue;
        if (pyramid_meets_box(V, lo, hi)) mask |= 1ull << l;
    }
    {
        const unsigned group = 0xFu << (threadIdx.x & 28);
        mask |= __shfl_xor_sync(group, mask, 1);
        mask |= __shfl_xor_sync(group, mask, 2);
    }
    if (sub != 0) return;

    // 2) terrain entry node: descend while exactly one child's box meets the view volume's AABB and
    //    that child is an inner node; nothing in the other subtrees can be hit by this camera's rays
    const int node = descend_any(p.bvh_kind, p.tnodes, 0, V.lo, V.hi RPL_CK_DESCEND_ARGS(p.n_tnodes));
    // 3) latency word of this (env, camera, step)
    uint32_t lat = 0;
    if (p.span > 1) {
        const int64_t step = p.step_dev ? *p.step_dev : p.step;
        lat = latency_word(p.env_offset + (uint32_t)e, (uint32_t)c, step, p.s_first[e], p.span, p.seed0, p.seed1);
    }
    p.cam_xf[5 * j + 4] = make_float4(__uint_as_float((uint32_t)mask), __uint_as_float((uint32_t)(mask >> 32)),
                                      __int_as_float(node), __uint_as_float(lat));
}

// ---------------------------------------------------------------------------------------------
// Ray state for one mesh query.  Box tests use the rounded origin `o` with 1/d; the triangle test
// uses the origin as base + off (both FP32), so vertex - origin keeps the precision of the small
// difference even 80 m away from the world origin.  (One rounded FP32 origin was 2.6 % faster but
// let near-grazing hits amplify its 3.8e-6 m rounding past the 1e-4 m depth tolerance.)
// ---------------------------------------------------------------------------------------------
struct Ray {
    float3 invd, oinv;    // 1/d and o/d for the slab test
    float3 base, off;     // triangle-test origin = base + off
    float Sx, Sy, Sz;     // watertight shear constants
    int kz;               // dominant axis of d
};

// Correctly rounded reciprocal (the same value as 1.0f / v, with fewer instructions than a division).
__device__ __forceinline__ float safe_rcp(float v) {
    return __frcp_rn(fabsf(v) > 1e-20f ? v : copysignf(1e-20f, v));
}

__device__ __forceinline__ float comp(const float3 &v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

__device__ __forceinline__ void make_ray(Ray &r, float3 base, float3 off, float3 d) {
    const float3 o = make_float3(base.x + off.x, base.y + off.y, base.z + off.z);
    r.invd = make_float3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    r.oinv = make_float3(o.x * r.invd.x, o.y * r.invd.y, o.z * r.invd.z);
    r.base = base;
    r.off = off;
    const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    r.kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    const int kx = r.kz == 2 ? 0 : r.kz + 1;
    const int ky = kx == 2 ? 0 : kx + 1;
    // the shear only has to be the same for every triangle of this ray (watertightness), not the
    // correctly rounded quotient: an approximate reciprocal (2 ulp) and products with it
    r.Sz = __fdividef(1.0f, comp(d, r.kz));
    r.Sx = comp(d, kx) * r.Sz;
    r.Sy = comp(d, ky) * r.Sz;
}

// Slab test of one child box against (0, tmax]; returns the entry distance or +inf.
__device__ __forceinline__ float slab(const Ray &r, float lox, float hix, float loy, float hiy, float loz,
                                      float hiz, float tmax) {
    const float x0 = fmaf(lox, r.invd.x, -r.oinv.x), x1 = fmaf(hix, r.invd.x, -r.oinv.x);
    const float y0 = fmaf(loy, r.invd.y, -r.oinv.y), y1 = fmaf(hiy, r.invd.y, -r.oinv.y);
    const float z0 = fmaf(loz, r.invd.z, -r.oinv.z), z1 = fmaf(hiz, r.invd.z, -r.oinv.z);
    const float tin = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), 0.0f));
    const float tout = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fminf(fmaxf(z0, z1), tmax));
    return tin <= tout ? tin : CUDART_INF_F;
}

// Two FP32 fused multiply-adds in one packed instruction (fma.rn.f32x2, sm_100 and later): each lane is
// an ordinary round-to-nearest fma, so the results equal two fmaf calls.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

// Three-input minimum and maximum (min.f32 / max.f32 with three sources, sm_100 and later): the same
// value as two nested fminf / fmaxf, in one instruction.
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Slab tests of the two child boxes of a binary node (n0: child 0's x and y lo/hi, n1: child 1's, n2:
// both z lo/hi) against (0, tmax]: the (lo, hi) plane distances of each axis come from one packed fma
// on the adjacent pair, the same arithmetic as slab().  Returns the entry distances and whether the
// ray meets each child within (0, tmax].
__device__ __forceinline__ void slab_pair(const float2 &ix, const float2 &iy, const float2 &iz, const float2 &ox,
                                          const float2 &oy, const float2 &oz, const float4 &n0, const float4 &n1,
                                          const float4 &n2, float tmax, float &t0, float &t1, bool &h0, bool &h1) {
    const float2 x0 = fma2(make_float2(n0.x, n0.y), ix, ox), y0 = fma2(make_float2(n0.z, n0.w), iy, oy);
    const float2 z0 = fma2(make_float2(n2.x, n2.y), iz, oz);
    const float2 x1 = fma2(make_float2(n1.x, n1.y), ix, ox), y1 = fma2(make_float2(n1.z, n1.w), iy, oy);
    const float2 z1 = fma2(make_float2(n2.z, n2.w), iz, oz);
    const float in0 = fmax3(fminf(x0.x, x0.y), fminf(y0.x, y0.y), fmaxf(fminf(z0.x, z0.y), 0.0f));
    const float out0 = fmin3(fmaxf(x0.x, x0.y), fmaxf(y0.x, y0.y), fminf(fmaxf(z0.x, z0.y), tmax));
    const float in1 = fmax3(fminf(x1.x, x1.y), fminf(y1.x, y1.y), fmaxf(fminf(z1.x, z1.y), 0.0f));
    const float out1 = fmin3(fmaxf(x1.x, x1.y), fmaxf(y1.x, y1.y), fminf(fmaxf(z1.x, z1.y), tmax));
    t0 = in0;
    t1 = in1;
    h0 = in0 <= out0;
    h1 = in1 <= out1;
}

// Vertex relative to the ray origin, permuted so the dominant axis comes last, then sheared so that
// the ray becomes the +z axis (Woop, Benthin, Wald 2013, "Watertight Ray/Triangle Intersection").
template <bool kSplit>
__device__ __forceinline__ float3 shear_vertex(const Ray &r, float vx, float vy, float vz) {
    float ax = vx - r.base.x, ay = vy - r.base.y, az = vz - r.base.z;
    if (kSplit) {
        ax -= r.off.x;
        ay -= r.off.y;
        az -= r.off.z;
    }
    const float3 a = make_float3(ax, ay, az);
    const int kx = r.kz == 2 ? 0 : r.kz + 1;
    const int ky = kx == 2 ? 0 : kx + 1;
    const float pz = comp(a, r.kz);
    return make_float3(fmaf(-r.Sx, pz, comp(a, kx)), fmaf(-r.Sy, pz, comp(a, ky)), r.Sz * pz);
}

// The rest of the watertight test once the edge functions U, V, W of the sheared triangle are known
// (az, bz, cz: its sheared vertices' z): inside test (closed, two-sided), determinant, hit
// distance.  The arithmetic is spelled out with round-to-nearest intrinsics, so every caller gets
// the same bits for the same inputs.
__device__ __forceinline__ bool tri_finish(float U, float V, float W, float az, float bz, float cz, float &tmax) {
    const bool has_neg = fmin3(U, V, W) < 0.f;
    const bool has_pos = fmax3(U, V, W) > 0.f;
    if (has_neg && has_pos) return false;
    const float det = __fadd_rn(__fadd_rn(U, V), W);
    if (det == 0.f) return false;
    const float T = __fmaf_rn(W, cz, __fmaf_rn(V, bz, __fmul_rn(U, az)));
    const float td = __fmul_rn(tmax, det);
    if (det > 0.f ? (T <= 0.f || T > td) : (T >= 0.f || T < td)) return false;
    const float t = __fdiv_rn(T, det);
    if (!(t > 0.f && t < tmax)) return false;
    tmax = t;
    return true;
}

// 2D edge function of the sheared vertices P, Q, evaluated without contraction.
__device__ __forceinline__ float edge_fn(const float3 &P, const float3 &Q) {
    return __fsub_rn(__fmul_rn(P.x, Q.y), __fmul_rn(P.y, Q.x));
}

// Two-sided, closed watertight test.  The 2D edge functions are evaluated without contraction, so a
// shared edge yields exactly negated values in its two triangles and no ray slips between them.
template <bool kSplit>
__device__ __forceinline__ bool tri_hit(const Ray &r, const float4 &v0, const float4 &v1, const float4 &v2,
                                        float &tmax) {
    const float3 A = shear_vertex<kSplit>(r, v0.x, v0.y, v0.z);
    const float3 B = shear_vertex<kSplit>(r, v1.x, v1.y, v1.z);
    const float3 C = shear_vertex<kSplit>(r, v2.x, v2.y, v2.z);
    return tri_finish(edge_fn(C, B), edge_fn(A, C), edge_fn(B, A), A.z, B.z, C.z, tmax);
}

// The pair (A, B, C), (A, C, D) of a quad leaf: four vertices sheared instead of six.  The second
// triangle's edge function of C-A is edge_fn(C, A), which equals -edge_fn(A, C) exactly (the same
// two rounded products, subtracted the other way round; only the sign of a zero can differ, and it
// changes no decision).  So this gives the bits of tri_hit on each triangle in turn.
template <bool kSplit>
__device__ __forceinline__ bool quad_hit(const Ray &r, const float4 &v0, const float4 &v1, const float4 &v2,
                                         const float4 &v3, float &tmax) {
    const float3 A = shear_vertex<kSplit>(r, v0.x, v0.y, v0.z);
    const float3 B = shear_vertex<kSplit>(r, v1.x, v1.y, v1.z);
    const float3 C = shear_vertex<kSplit>(r, v2.x, v2.y, v2.z);
    const float3 D = shear_vertex<kSplit>(r, v3.x, v3.y, v3.z);
    const float eAC = edge_fn(A, C);
    bool h = tri_finish(edge_fn(C, B), eAC, edge_fn(B, A), A.z, B.z, C.z, tmax);
    h |= tri_finish(edge_fn(D, C), edge_fn(A, D), -eAC, A.z, C.z, D.z, tmax);
    return h;
}

struct Counts {
    uint32_t nodes = 0, tris = 0;
};

template <bool kSplit, bool kCount>
__device__ __forceinline__ void leaf(const float4 *__restrict__ tris, int first, int count, const Ray &r,
                                     float &tmax, bool &hit, Counts &cnt RPL_CK_PARAMS) {
#ifdef RPL_CHECKED
    if (first < 0 || !in_range((int64_t)first + count - 1, ck_tris)) {
        ck_err |= kErrBounds;
        return;
    }
#endif
    int i = first;
    if (count == 2) {
        // the second triangle's last vertex is loaded with the first triangle, so that a quad's four
        // vertices arrive together instead of after the quad flag in b.w
        const float4 a = __ldg(tris + 3 * i), b = __ldg(tris + 3 * i + 1), c = __ldg(tris + 3 * i + 2);
        const float4 d = __ldg(tris + 3 * i + 5);
        if (b.w != 0.f) {
            // a quad: the second triangle is (a, c, d)
            if (kCount) cnt.tris += 2;
            hit |= quad_hit<kSplit>(r, a, b, c, d, tmax);
            return;
        }
        if (kCount) ++cnt.tris;
        hit |= tri_hit<kSplit>(r, a, b, c, tmax);
        ++i;
    }
#pragma unroll 1
    for (; i < first + count; ++i) {
        const float4 a = __ldg(tris + 3 * i), b = __ldg(tris + 3 * i + 1), c = __ldg(tris + 3 * i + 2);
        if (kCount) ++cnt.tris;
        hit |= tri_hit<kSplit>(r, a, b, c, tmax);
    }
}

// During traversal a leaf child is carried as ~((first << 3) | (count - 1)) (always negative, since
// scenes hold fewer than 2^28 - 1 triangles and leaves at most 8); kDone marks an exhausted stack.
constexpr int kDone = INT_MIN;

// The traversal's leaf reference of a four-wide child (whose node stores ~first and the count apart).
__device__ __forceinline__ int leaf_ref(int child, int count) { return ~((~child << 3) | (count - 1)); }

__device__ __forceinline__ int stack_pop(const int *stack, int &sp) { return sp > 0 ? stack[--sp] : kDone; }

// Closest hit below tmax in one BVH, searched from node `root` and, when root2 >= 0, then from node
// root2 (two disjoint subtrees); tmax shrinks to the hit distance.  The stack holds at most one
// entry per level of the current path plus root2, so it cannot overflow for the scenes accepted at
// build time (BVH depth < kStackDepth); the bounds-checked build verifies every push.  Returns true.
//
// Inner nodes and leaves are handled in two phases (Aila and Laine, "Understanding the Efficiency of
// Ray Traversal on GPUs", HPG 2009): a lane that meets a leaf postpones it and keeps descending
// while any lane of the warp has not found a leaf yet, then the warp tests its leaves together, so
// triangle tests run with most lanes active instead of one lane at a time.  The stack (in local
// memory, cached in L1) holds node references only: culling popped entries by their entry distance
// cost more than the node fetches it saves, which mostly hit in cache.  (Measured alternatives that
// were slower on the scale workload: a shared-memory short stack, whose carve-out takes L1 capacity
// the node fetches depend on; one traversal loop shared by links and terrain; and compacting the
// warp's (ray, link) pairs so that link BVHs are traversed with full warps.)
template <bool kSplit, bool kCount>
__device__ __forceinline__ bool traverse(const float4 *__restrict__ nodes, const float4 *__restrict__ tris, int root,
                                         int root2, const Ray &r, float &tmax, bool &hit, Counts &cnt RPL_CK_PARAMS) {
    int stack_node[kStackDepth];
    int sp = 0;
    if (root2 >= 0) stack_node[sp++] = root2;
    int cur = root;      // >= 0 inner node, < 0 leaf reference, kDone nothing left
    int pending = 0;     // postponed leaf reference, 0 = none
    auto pop = [&]() -> int { return stack_pop(stack_node, sp); };
    // the ray's 1/d and -o/d per axis, twice, for the packed slab tests
    const float2 ix = make_float2(r.invd.x, r.invd.x), iy = make_float2(r.invd.y, r.invd.y),
                 iz = make_float2(r.invd.z, r.invd.z);
    const float2 ox = make_float2(-r.oinv.x, -r.oinv.x), oy = make_float2(-r.oinv.y, -r.oinv.y),
                 oz = make_float2(-r.oinv.z, -r.oinv.z);
#pragma unroll 1
    for (;;) {
#pragma unroll 1
        while (cur >= 0) {
            RPL_CK_NODE(cur, cur = kDone; break)
            const float4 *n = nodes + 4 * cur;
            const float4 n0 = __ldg(n), n1 = __ldg(n + 1), n2 = __ldg(n + 2);
            const int4 n3 = __ldg(reinterpret_cast<const int4 *>(n + 3));
            if (kCount) ++cnt.nodes;
            float t0, t1;
            bool h0, h1;
            slab_pair(ix, iy, iz, ox, oy, oz, n0, n1, n2, tmax, t0, t1, h0, h1);
            // leaf children arrive encoded and empty ones never hit (device layout, see rpl_api.cpp)
            const int e0 = n3.x, e1 = n3.y;
            // nearer hit child next (child 0 on a tie), the other one pushed; branch-free selects
            const bool sw = h1 && (!h0 || t1 < t0);
            const int near = sw ? e1 : e0, far = sw ? e0 : e1;
            if (h0 && h1) {
                RPL_CK_PUSH(sp, cur = kDone; break)
                stack_node[sp++] = far;
            }
            cur = (h0 || h1) ? near : pop();
            if (cur < 0 && cur != kDone && pending == 0) {
                pending = cur;
                cur = pop();
            }
            if (!__any_sync(__activemask(), pending == 0 && cur >= 0)) break;
        }
#pragma unroll 1
        while (pending < 0) {
            const int ref = ~pending;
            leaf<kSplit, kCount>(tris, ref >> 3, (ref & 7) + 1, r, tmax, hit, cnt RPL_CK_ARGS(ck_nodes, ck_tris, ck_err));
            pending = 0;
            if (cur < 0 && cur != kDone) {
                pending = cur;
                cur = pop();
            }
        }
        if (cur == kDone) return true;
    }
}

// ---------------------------------------------------------------------------------------------
// Four-wide BVH with FP32 boxes (layout in bvh4.h)
// ---------------------------------------------------------------------------------------------
struct Node4 {
    float4 lx, hx, ly, hy, lz, hz;
    int4 ch, cn;
};

__device__ __forceinline__ Node4 load4(const float4 *__restrict__ nodes, int i) {
    const float4 *n = nodes + 8 * (int64_t)i;
    return Node4{__ldg(n), __ldg(n + 1), __ldg(n + 2), __ldg(n + 3), __ldg(n + 4), __ldg(n + 5),
                 __ldg(reinterpret_cast<const int4 *>(n + 6)), __ldg(reinterpret_cast<const int4 *>(n + 7))};
}

// Deepest four-wide node below `node` that holds everything inside the AABB [lo, hi]: descend while
// exactly one child box meets the AABB and that child is an inner node (unused slots sit at 1e30).
__device__ __forceinline__ int descend4(const float4 *__restrict__ nodes, int node, const float lo[3],
                                        const float hi[3] RPL_CK_DESCEND_PARAMS) {
#pragma unroll 1
    for (int depth = 0; depth < kStackDepth; ++depth) {
        const Node4 n = load4(nodes, node);
        const bool o0 = boxes_overlap(n.lx.x, n.hx.x, n.ly.x, n.hy.x, n.lz.x, n.hz.x, lo, hi);
        const bool o1 = boxes_overlap(n.lx.y, n.hx.y, n.ly.y, n.hy.y, n.lz.y, n.hz.y, lo, hi);
        const bool o2 = boxes_overlap(n.lx.z, n.hx.z, n.ly.z, n.hy.z, n.lz.z, n.hz.z, lo, hi);
        const bool o3 = boxes_overlap(n.lx.w, n.hx.w, n.ly.w, n.hy.w, n.lz.w, n.hz.w, lo, hi);
        if ((int)o0 + (int)o1 + (int)o2 + (int)o3 != 1) break;
        const int c = o0 ? n.ch.x : (o1 ? n.ch.y : (o2 ? n.ch.z : n.ch.w));
        if (c < 0) break;
#ifdef RPL_CHECKED
        if (!in_range(c, ck_nodes)) break;
#endif
        node = c;
    }
    return node;
}

// Compare-exchange of (distance, reference) pairs, ascending by distance.
__device__ __forceinline__ void cmp_swap(float &ta, int &ea, float &tb, int &eb) {
    const bool sw = tb < ta;
    const float t = sw ? tb : ta;
    const int e = sw ? eb : ea;
    tb = sw ? ta : tb;
    eb = sw ? ea : eb;
    ta = t;
    ea = e;
}

// Closest hit in the four-wide terrain BVH, with the same two-phase leaf handling as the binary
// traversal: the four child boxes of a node are tested from one 128-byte fetch, the hit children
// are sorted by entry distance, the nearest is visited next and the others pushed far to near.
template <bool kCount>
__device__ __forceinline__ bool traverse4(const float4 *__restrict__ nodes, const float4 *__restrict__ tris, int root,
                                          const Ray &r, float &tmax, bool &hit, Counts &cnt RPL_CK_PARAMS) {
    int stack_node[kStackDepth];
    int sp = 0;
    bool ok = true;
    int cur = root;
    int pending = 0;
    auto pop = [&]() -> int { return stack_pop(stack_node, sp); };
#pragma unroll 1
    for (;;) {
#pragma unroll 1
        while (cur >= 0) {
            RPL_CK_NODE(cur, cur = kDone; break)
            const Node4 n = load4(nodes, cur);
            if (kCount) ++cnt.nodes;
            float t0 = slab(r, n.lx.x, n.hx.x, n.ly.x, n.hy.x, n.lz.x, n.hz.x, tmax);
            float t1 = slab(r, n.lx.y, n.hx.y, n.ly.y, n.hy.y, n.lz.y, n.hz.y, tmax);
            float t2 = slab(r, n.lx.z, n.hx.z, n.ly.z, n.hy.z, n.lz.z, n.hz.z, tmax);
            float t3 = slab(r, n.lx.w, n.hx.w, n.ly.w, n.hy.w, n.lz.w, n.hz.w, tmax);
            int e0 = n.ch.x >= 0 ? n.ch.x : leaf_ref(n.ch.x, n.cn.x);
            int e1 = n.ch.y >= 0 ? n.ch.y : leaf_ref(n.ch.y, n.cn.y);
            int e2 = n.ch.z >= 0 ? n.ch.z : leaf_ref(n.ch.z, n.cn.z);
            int e3 = n.ch.w >= 0 ? n.ch.w : leaf_ref(n.ch.w, n.cn.w);
            cmp_swap(t0, e0, t1, e1);
            cmp_swap(t2, e2, t3, e3);
            cmp_swap(t0, e0, t2, e2);
            cmp_swap(t1, e1, t3, e3);
            cmp_swap(t1, e1, t2, e2);
            const int nh = (int)(t0 != CUDART_INF_F) + (int)(t1 != CUDART_INF_F) + (int)(t2 != CUDART_INF_F) +
                           (int)(t3 != CUDART_INF_F);
            if (nh == 0) {
                cur = pop();
            } else {
                if (sp + nh - 1 > kStackDepth) {
                    ok = false;
                    cur = kDone;
                    break;
                }
                if (nh > 3) stack_node[sp++] = e3;
                if (nh > 2) stack_node[sp++] = e2;
                if (nh > 1) stack_node[sp++] = e1;
                cur = e0;
            }
            if (cur < 0 && cur != kDone && pending == 0) {
                pending = cur;
                cur = pop();
            }
            if (!__any_sync(__activemask(), pending == 0 && cur >= 0)) break;
        }
#pragma unroll 1
        while (pending < 0) {
            const int ref = ~pending;
            leaf<true, kCount>(tris, ref >> 3, (ref & 7) + 1, r, tmax, hit, cnt RPL_CK_ARGS(ck_nodes, ck_tris, ck_err));
            pending = 0;
            if (cur < 0 && cur != kDone) {
                pending = cur;
                cur = pop();
            }
        }
        if (cur == kDone) return ok;
    }
}

// ---------------------------------------------------------------------------------------------
// Eight-wide quantised BVH (layout in bvh8.h)
// ---------------------------------------------------------------------------------------------
// Byte j of w as a float: the byte is placed into the mantissa of 2^23 and 2^23 subtracted (exact).
template <int j>
__device__ __forceinline__ float qbyte(uint32_t w) {
    return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7650 + j)) - 8388608.0f;
}

// Permutes an 8-bit slot mask into traversal order (bit i <- slot i ^ oct) and back.
__device__ __forceinline__ uint32_t oct_permute(uint32_t m, int oct) {
    if (oct & 1) m = ((m & 0x55u) << 1) | ((m & 0xAAu) >> 1);
    if (oct & 2) m = ((m & 0x33u) << 2) | ((m & 0xCCu) >> 2);
    if (oct & 4) m = ((m & 0x0Fu) << 4) | ((m & 0xF0u) >> 4);
    return m;
}

struct WideNode {
    uint4 a, b, c, d, f;
};

__device__ __forceinline__ WideNode load_wide(const float4 *__restrict__ nodes, int i) {
    const uint4 *n = reinterpret_cast<const uint4 *>(nodes) + 5 * (int64_t)i;
    return WideNode{__ldg(n), __ldg(n + 1), __ldg(n + 2), __ldg(n + 3), __ldg(n + 4)};
}

// Slab tests of the eight children of one wide node against (0, tmax]; returns the hit mask in slot
// order.  t(q) = q * step * (1/d) + (origin - o) * (1/d) per axis, near/far planes chosen by the
// sign of d, so an empty slot (q_lo 255, q_hi 0) never hits.
__device__ __forceinline__ uint32_t wide_hits(const WideNode &n, const Ray &r, float tmax) {
    const float ox = __uint_as_float(n.a.x), oy = __uint_as_float(n.a.y), oz = __uint_as_float(n.a.z);
    const float sx = __uint_as_float((n.a.w & 0xFFu) << 23), sy = __uint_as_float(((n.a.w >> 8) & 0xFFu) << 23),
                sz = __uint_as_float(((n.a.w >> 16) & 0xFFu) << 23);
    const float ax = sx * r.invd.x, ay = sy * r.invd.y, az = sz * r.invd.z;
    const float bx = fmaf(ox, r.invd.x, -r.oinv.x), by = fmaf(oy, r.invd.y, -r.oinv.y),
                bz = fmaf(oz, r.invd.z, -r.oinv.z);
    const bool px = r.invd.x >= 0.f, py = r.invd.y >= 0.f, pz = r.invd.z >= 0.f;
    // words: q_lo x (c.x, c.y), y (c.z, c.w), z (d.x, d.y); q_hi x (d.z, d.w), y (f.x, f.y), z (f.z, f.w)
    const uint32_t nx0 = px ? n.c.x : n.d.z, nx1 = px ? n.c.y : n.d.w, fx0 = px ? n.d.z : n.c.x, fx1 = px ? n.d.w : n.c.y;
    const uint32_t ny0 = py ? n.c.z : n.f.x, ny1 = py ? n.c.w : n.f.y, fy0 = py ? n.f.x : n.c.z, fy1 = py ? n.f.y : n.c.w;
    const uint32_t nz0 = pz ? n.d.x : n.f.z, nz1 = pz ? n.d.y : n.f.w, fz0 = pz ? n.f.z : n.d.x, fz1 = pz ? n.f.w : n.d.y;
    uint32_t hits = 0;
#define RPL_WIDE_SLOT(S, NX, NY, NZ, FX, FY, FZ, J)                                                          \
    {                                                                                                      \
        const float tin = fmaxf(fmaxf(fmaf(qbyte<J>(NX), ax, bx), fmaf(qbyte<J>(NY), ay, by)),             \
                                fmaxf(fmaf(qbyte<J>(NZ), az, bz), 0.0f));                                  \
        const float tout = fminf(fminf(fmaf(qbyte<J>(FX), ax, bx), fmaf(qbyte<J>(FY), ay, by)),            \
                                 fminf(fmaf(qbyte<J>(FZ), az, bz), tmax));                                 \
        hits |= (tin <= tout ? 1u : 0u) << (S);                                                            \
    }
    RPL_WIDE_SLOT(0, nx0, ny0, nz0, fx0, fy0, fz0, 0)
    RPL_WIDE_SLOT(1, nx0, ny0, nz0, fx0, fy0, fz0, 1)
    RPL_WIDE_SLOT(2, nx0, ny0, nz0, fx0, fy0, fz0, 2)
    RPL_WIDE_SLOT(3, nx0, ny0, nz0, fx0, fy0, fz0, 3)
    RPL_WIDE_SLOT(4, nx1, ny1, nz1, fx1, fy1, fz1, 0)
    RPL_WIDE_SLOT(5, nx1, ny1, nz1, fx1, fy1, fz1, 1)
    RPL_WIDE_SLOT(6, nx1, ny1, nz1, fx1, fy1, fz1, 2)
    RPL_WIDE_SLOT(7, nx1, ny1, nz1, fx1, fy1, fz1, 3)
#undef RPL_WIDE_SLOT
    return hits;
}

__device__ __forceinline__ uint32_t meta_byte(const WideNode &n, int s) {
    return ((s < 4 ? n.b.z : n.b.w) >> (8 * (s & 3))) & 0xFFu;
}

// Dequantised box of slot s (rounded outward by the padding of the caller's overlap test).
__device__ __forceinline__ void wide_child_box(const WideNode &n, int s, float lo[3], float hi[3]) {
    const uint32_t wl[3][2] = {{n.c.x, n.c.y}, {n.c.z, n.c.w}, {n.d.x, n.d.y}};
    const uint32_t wh[3][2] = {{n.d.z, n.d.w}, {n.f.x, n.f.y}, {n.f.z, n.f.w}};
    const uint32_t org[3] = {n.a.x, n.a.y, n.a.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float step = __uint_as_float(((n.a.w >> (8 * a)) & 0xFFu) << 23);
        const float o = __uint_as_float(org[a]);
        const float ql = (float)((wl[a][s >> 2] >> (8 * (s & 3))) & 0xFFu);
        const float qh = (float)((wh[a][s >> 2] >> (8 * (s & 3))) & 0xFFu);
        lo[a] = fmaf(ql, step, o);
        hi[a] = fmaf(qh, step, o);
    }
}

// Deepest wide node below `node` that holds everything inside the AABB [lo, hi]: descend while
// exactly one slot's box meets the AABB and that slot is an inner node.
__device__ __forceinline__ int descend_wide(const float4 *__restrict__ nodes, int node, const float lo[3],
                                            const float hi[3] RPL_CK_DESCEND_PARAMS) {
#pragma unroll 1
    for (int depth = 0; depth < kStackDepth; ++depth) {
        const WideNode n = load_wide(nodes, node);
        int n_hit = 0, slot = -1;
#pragma unroll 1
        for (int s = 0; s < 8; ++s) {
            if (meta_byte(n, s) == 0) continue;
            float bl[3], bh[3];
            wide_child_box(n, s, bl, bh);
            if (boxes_overlap(bl[0], bh[0], bl[1], bh[1], bl[2], bh[2], lo, hi)) {
                ++n_hit;
                slot = s;
            }
        }
        const uint32_t imask = n.a.w >> 24;
        if (n_hit != 1 || !((imask >> slot) & 1u)) break;
#ifdef RPL_CHECKED
        if (!in_range((int64_t)n.b.x + (meta_byte(n, slot) & 0x7Fu), ck_nodes)) break;
#endif
        node = (int)n.b.x + (int)(meta_byte(n, slot) & 0x7Fu);
    }
    return node;
}

// Closest hit in the wide terrain BVH.  The stack holds groups of inner children still to visit,
// (first child index, imask | remaining traversal-order mask << 8); children are taken in the order
// slot ^ octant(d), roughly front to back.  Leaf children of a node are tested when it is visited:
// postponing them as the binary traversal does was 40 % slower here, since the bound then shrinks
// late and the coarse octant order visits many more nodes before the first hit.
template <bool kCount>
__device__ __forceinline__ bool traverse8(const float4 *__restrict__ nodes, const float4 *__restrict__ tris, int root,
                                          const Ray &r, int oct, float &tmax, bool &hit, Counts &cnt RPL_CK_PARAMS) {
    uint2 stack[kStackDepth];
    int sp = 0;
    int node = root;
#pragma unroll 1
    for (;;) {
        RPL_CK_NODE(node, return true)
        const WideNode n = load_wide(nodes, node);
        if (kCount) ++cnt.nodes;
        const uint32_t hits = wide_hits(n, r, tmax);
        const uint32_t imask = n.a.w >> 24;
        // leaf children, nearest first
        uint32_t leaves = oct_permute(hits & ~imask & 0xFFu, oct);
#pragma unroll 1
        while (leaves) {
            const int s = (__ffs(leaves) - 1) ^ oct;
            leaves &= leaves - 1;
            const uint32_t m = meta_byte(n, s);
            leaf<true, kCount>(tris, (int)n.b.y + (int)((m >> 2) & 31u), (int)(m & 3u) + 1, r, tmax, hit,
                               cnt RPL_CK_ARGS(ck_nodes, ck_tris, ck_err));
        }
        uint32_t inner = oct_permute(hits & imask, oct);
        uint32_t base = n.b.x, im = imask;
        if (!inner) {
            // next group from the stack
            bool found = false;
            while (sp > 0) {
                const uint2 g = stack[--sp];
                if (g.y >> 8) {
                    base = g.x;
                    im = g.y & 0xFFu;
                    inner = g.y >> 8;
                    found = true;
                    break;
                }
            }
            if (!found) return true;
        }
        const int s = (__ffs(inner) - 1) ^ oct;
        inner &= inner - 1;
        if (inner) {
            if (sp == kStackDepth) return false;
            stack[sp++] = make_uint2(base, im | (inner << 8));
        }
        node = (int)base + __popc(im & ((1u << s) - 1u));
    }
}

// The sensor model and the store of output pixel (x, y) of camera c in env e, whose pre-sensor
// depth at this step is z: ring-buffer write, latency select (source step = step - delay, both from
// the latency word `lat` the prep kernel drew), noise on hits, clip, dropout, side mask (Appendix A.2;
// Sec. 3.2.4).
__device__ __forceinline__ void finish_pixel(const RenderParams &p, int e, int c, const CamDev &cam, int x, int y,
                                             float z, int64_t step, uint32_t lat) {
    const uint32_t pix = (uint32_t)(y * cam.out_w + x);
    const int64_t col = (int64_t)cam.pix_off + pix;
    const uint32_t ge = p.env_offset + (uint32_t)e;
    int64_t src = step;
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
    if (p.sensor_on) {
        const uint32_t span = p.span;
        if (span > 1) {
            // lat (latency_word): delay in bits 0..7, ring slot of this step in bits 8..15
            const uint32_t delta = lat & 0xFFu, slot = (lat >> 8) & 0xFFu;
            const int64_t row = (int64_t)e * span;
            p.ring[(row + slot) * p.pix_per_env + col] = z;
            src = step - (int64_t)delta;
            if (delta != 0u) {
                const uint32_t sslot = slot >= delta ? slot - delta : slot + span - delta;
                z = p.ring[(row + sslot) * p.pix_per_env + col];
            }
        }
        w = sensor_words(ge, (uint32_t)c, pix, src, p.seed0, p.seed1);
        if (z < cam.d_max) {
            const float u1 = ((float)w.y + 1.0f) * 0x1p-32f;
            const float u2 = (float)w.z * 0x1p-32f;
            // cos(2 pi u2) by the hardware cosine on [-pi, pi) (absolute error below 5e-7, i.e. below
            // 1e-6 m of depth for noise scales up to 1 m); the logarithm stays exact to an ulp, since
            // near u1 = 1 an absolute error of the fast one would reach the depth tolerance
            const float a = 6.2831853071795864f * (u2 >= 0.5f ? u2 - 1.0f : u2);
            const float n = sqrtf(-2.0f * logf(u1)) * __cosf(a);
            z = z + (p.sigma_abs + p.sigma_rel * z) * n;
        }
        z = fminf(fmaxf(z, cam.d_min), cam.d_max);
        if ((uint64_t)w.x < p.drop_thr) z = p.fill;
    } else {
        z = fminf(fmaxf(z, cam.d_min), cam.d_max);
    }
    if (p.rsm_mode) {
        const int n = p.rsm_cols[min((int)p.rsm_mode[e], 2)];
        if (x < n || x >= cam.out_w - n) {
            // uniform fill keyed by the current step; the words above belong to the source step
            if (!p.sensor_on || src != step) w = sensor_words(ge, (uint32_t)c, pix, step, p.seed0, p.seed1);
            z = cam.d_min + (cam.d_max - cam.d_min) * (((float)w.w + 0.5f) * 0x1p-32f);
        }
    }
    const int64_t o_idx = (int64_t)e * p.pix_per_env + col;
    if (p.out_dtype == RPL_OUT_F32) {
        static_cast<float *>(p.out)[o_idx] = z;
    } else if (p.out_dtype == RPL_OUT_F16) {
        static_cast<__half *>(p.out)[o_idx] = __float2half_rn(z);
    } else {
        const float q = rintf(fminf(fmaxf(z / cam.d_max, 0.f), 1.f) * 65535.f);
        static_cast<uint16_t *>(p.out)[o_idx] = (uint16_t)q;
    }
}

// floor(n / d) for 0 <= n < 2^31 from the multiplier m and shift k of the divisor d (fastdiv_magic in
// render.h): one wide multiply and a shift instead of a division.
__device__ __forceinline__ uint32_t fastdiv(uint32_t n, uint32_t m, uint32_t k) {
    return (uint32_t)(((uint64_t)n * m) >> k);
}

// Env and tile within the env of tile `warp`: multiply and shift when the host set the divisor's
// magic and the index fits in 31 bits, else a 32- or 64-bit division.
__device__ __forceinline__ void split_tile(int64_t warp, const RenderParams &p, int &e, int &r_tile) {
    const int32_t tpe = p.tiles_per_env;
    if ((uint64_t)warp < 0x80000000ull && p.tpe_m != 0u) {
        const uint32_t q = fastdiv((uint32_t)warp, p.tpe_m, p.tpe_k);
        e = (int)q;
        r_tile = (int)((uint32_t)warp - q * (uint32_t)tpe);
    } else if ((uint64_t)warp < 0x100000000ull) {
        const uint32_t w = (uint32_t)warp, q = w / (uint32_t)tpe;
        e = (int)q;
        r_tile = (int)(w - q * (uint32_t)tpe);
    } else {
        e = (int)(warp / tpe);
        r_tile = (int)(warp - (int64_t)e * tpe);
    }
}

// Row and column of tile t (0 <= t < 2^31) of a camera's tile grid.
__device__ __forceinline__ void tile_row_col(const CamDev &cam, int t, int &row, int &col) {
    row = cam.tx_m ? (int)fastdiv((uint32_t)t, cam.tx_m, cam.tx_k) : t / cam.tiles_x;
    col = t - row * cam.tiles_x;
}

// Terrain entry node and link mask of a tile, derived by its warp (when no tile-prep output is
// given): the AABB of the 32 ray segments from o3 along d3 to tmax, padded for FP32 rounding; the
// deepest terrain node below the camera's entry node that holds the AABB; and, one link of the
// camera's mask per lane (links 0..31, then 32..63), the links whose world box meets the AABB.
template <int kKind>
__device__ __forceinline__ void tile_reach_in_warp(const RenderParams &p, int e, int lane, const float o3[3],
                                                   const float d3[3], float tmax, int cam_entry, uint64_t cam_mask,
                                                   int &entry, uint64_t &link_mask) {
    float tlo[3], thi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float far = o3[a] + d3[a] * tmax;
        float lo = fminf(o3[a], far), hi = fmaxf(o3[a], far);
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, s));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, s));
        }
        const float slack = 1e-3f + 1e-5f * fmaxf(fabsf(lo), fabsf(hi));
        tlo[a] = lo - slack;
        thi[a] = hi + slack;
    }
    entry = descend_any(kKind, p.tnodes, cam_entry, tlo, thi RPL_CK_DESCEND_ARGS(p.n_tnodes));
    link_mask = 0;
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
        const int l = lane + 32 * half;
        bool keep = false;
        if ((cam_mask >> l) & 1ull) {
            const int64_t el = (int64_t)e * p.L + l;
            const float4 blo = __ldg(p.link_box + 2 * el), bhi = __ldg(p.link_box + 2 * el + 1);
            keep = boxes_overlap(blo.x, bhi.x, blo.y, bhi.y, blo.z, bhi.z, tlo, thi);
        }
        link_mask |= (uint64_t)__ballot_sync(0xffffffffu, keep) << (32 * half);
        if ((cam_mask >> 32) == 0) break;
    }
}

// Tile index (env * tiles_per_env + tile within the env) of the t-th tile in processing order: the
// envs in p.env_order's order when it is set, else in index order.
__device__ __forceinline__ int64_t tile_of(const RenderParams &p, int64_t t) {
    if (!p.env_order) return t;
    int e, r;
    split_tile(t, p, e, r);
    return (int64_t)__ldg(p.env_order + e) * p.tiles_per_env + r;
}

// One warp renders one tile of 32 pixel rays (tile_w x tile_h, tile_w = 2^tile_w_log2) of one
// (env, camera).  Called once per warp, or in a grid-stride loop by the persistent launch; `warp` is
// uniform across the warp so the warp-wide reductions below see all 32 lanes.  kTileInfo: the tile's
// entry node and link mask come from p.tile_info (else the warp derives them).
// (e, r_tile: the tile's env and its index inside the env, i.e. warp = e * tiles_per_env + r_tile.)
template <bool kCount, int kKind, bool kTileInfo>
__device__ __forceinline__ void render_tile(const RenderParams &p, int64_t warp, int e, int r_tile, int lane,
                                            int64_t step) {
    int c = 0;
    while (c + 1 < p.C && r_tile >= p.cams[c + 1].tile_off) ++c;
    const CamDev &cam = p.cams[c];
    const int tw_log2 = p.tile_w_log2, th = 32 >> tw_log2;
    int trow, tcol;
    tile_row_col(cam, r_tile - cam.tile_off, trow, tcol);
    const int x = tcol * (1 << tw_log2) + (lane & ((1 << tw_log2) - 1));
    const int y = trow * th + (lane >> tw_log2);
    // lanes outside a ragged tile still take part in the warp-wide reductions below
    const bool active = x < cam.width && y < cam.height;
    const int xs = min(x, cam.width - 1), ys = min(y, cam.height - 1);

    // BuildDepthRay: r = K^-1 [x, y, 1], d = R_c r / |r|, m = 1 / |r|
    float fx = cam.fx, fy = cam.fy, cx = cam.cx, cy = cam.cy;
    if (p.intr) {
        const float4 k = __ldg(reinterpret_cast<const float4 *>(p.intr) + (int64_t)e * p.C + c);
        fx = k.x; fy = k.y; cx = k.z; cy = k.w;
    }
    const float4 *cx4 = p.cam_xf + 5 * ((int64_t)e * p.C + c);
    const float4 R0 = __ldg(cx4), R1 = __ldg(cx4 + 1), R2 = __ldg(cx4 + 2), OF = __ldg(cx4 + 3);
    const float4 CV = __ldg(cx4 + 4);
    const uint64_t cam_mask = ((uint64_t)__float_as_uint(CV.y) << 32) | __float_as_uint(CV.x);
    // fast division and reciprocal square root (2 ulp each): they only move the ray by ~1e-7 rad
    const float rx = __fdividef((float)xs - cx, fx), ry = __fdividef((float)ys - cy, fy);
    const float inv_n = rsqrtf(rx * rx + ry * ry + 1.0f);
    const float ux = rx * inv_n, uy = ry * inv_n, uz = inv_n;
    const float3 d = make_float3(R0.x * ux + R0.y * uy + R0.z * uz, R1.x * ux + R1.y * uy + R1.z * uz,
                                 R2.x * ux + R2.y * uy + R2.z * uz);
    const float3 base = make_float3(R0.w, R1.w, R2.w);
    const float3 off = make_float3(OF.x, OF.y, OF.z);
    const float m = p.depth_kind == RPL_DEPTH_Z ? inv_n : 1.0f;
    float tmax = __fdividef(cam.d_max, m);
    bool hit = false;
    bool ok = true;
    Counts cnt_t, cnt_l;
    uint32_t n_boxes = 0;

    Ray ray;
    make_ray(ray, base, off, d);

    // The tile's terrain entry node and link mask (uniform across the warp): from the tile-prep
    // kernel, or else derived by the warp itself.
#ifdef RPL_CHECKED
    uint32_t ck_err = 0;
#endif
    int entry, entry2 = -1;
    uint64_t link_mask;
    if (kTileInfo) {
        const int4 ti = __ldg(p.tile_info + warp);
        entry = ti.x;
        entry2 = ti.w;
        link_mask = ((uint64_t)(uint32_t)ti.z << 32) | (uint32_t)ti.y;
    } else {
        const float o3[3] = {base.x + off.x, base.y + off.y, base.z + off.z};
        const float d3[3] = {d.x, d.y, d.z};
        tile_reach_in_warp<kKind>(p, e, lane, o3, d3, tmax, __float_as_int(CV.z), cam_mask, entry, link_mask);
    }
    if (!active) return;

    // Both queries shrink the shared bound tmax; the minimum does not depend on their order
    // (Alg. 1 queries the bodies first; terrain first makes the link queries shorter instead).
    // 1) dynamic robot bodies that the tile can reach: rays move into each link frame
    //    (o_b = R^T (o - t), d_b = R^T d)
    auto query_links = [&]() {
#pragma unroll 1
    for (uint64_t mk = link_mask; mk; mk &= mk - 1) {
        const int l = __ffsll((long long)mk) - 1;
        const int root = p.lroot[l];
        if (root < 0) continue;
        const int64_t el = (int64_t)e * p.L + l;
        const float4 blo = __ldg(p.link_box + 2 * el), bhi = __ldg(p.link_box + 2 * el + 1);
        if (kCount) ++n_boxes;
        if (slab(ray, blo.x, bhi.x, blo.y, bhi.y, blo.z, bhi.z, tmax) == CUDART_INF_F) continue;
        const float4 X0 = __ldg(p.link_xf + 3 * el), X1 = __ldg(p.link_xf + 3 * el + 1),
                     X2 = __ldg(p.link_xf + 3 * el + 2);
        const float3 rel = make_float3((base.x - X0.w) + off.x, (base.y - X1.w) + off.y, (base.z - X2.w) + off.z);
        const float3 ob = make_float3(X0.x * rel.x + X0.y * rel.y + X0.z * rel.z,
                                      X1.x * rel.x + X1.y * rel.y + X1.z * rel.z,
                                      X2.x * rel.x + X2.y * rel.y + X2.z * rel.z);
        const float3 db = make_float3(X0.x * d.x + X0.y * d.y + X0.z * d.z, X1.x * d.x + X1.y * d.y + X1.z * d.z,
                                      X2.x * d.x + X2.y * d.y + X2.z * d.z);
        Ray lr;
        make_ray(lr, ob, make_float3(0.f, 0.f, 0.f), db);
        ok &= traverse<false, kCount>(p.lnodes, p.ltris, root, -1, lr, tmax, hit, cnt_l RPL_CK_ARGS(p.n_lnodes, p.n_ltris, ck_err));
    }
    };
    // 2) static terrain, bounded by the closest hit so far
    auto query_terrain = [&]() {
        if (kKind == RPL_BVH8Q8) {
            const int oct = (d.x < 0.f ? 1 : 0) | (d.y < 0.f ? 2 : 0) | (d.z < 0.f ? 4 : 0);
            ok &= traverse8<kCount>(p.tnodes, p.ttris, entry, ray, oct, tmax, hit, cnt_t RPL_CK_ARGS(p.n_tnodes, p.n_ttris, ck_err));
        } else if (kKind == RPL_BVH4) {
            ok &= traverse4<kCount>(p.tnodes, p.ttris, entry, ray, tmax, hit, cnt_t RPL_CK_ARGS(p.n_tnodes, p.n_ttris, ck_err));
        } else {
            ok &= traverse<true, kCount>(p.tnodes, p.ttris, entry, entry2, ray, tmax, hit, cnt_t RPL_CK_ARGS(p.n_tnodes, p.n_ttris, ck_err));
        }
    };
    if (p.terrain_first) {
        query_terrain();
        query_links();
    } else {
        query_links();
        query_terrain();
    }
    if (!ok) atomicOr(p.err, 1);
#ifdef RPL_CHECKED
    if (ck_err) atomicOr(p.err, (int)ck_err);
#endif

    const float z = hit ? fminf(m * tmax, cam.d_max) : cam.d_max;
    if (cam.ds > 1) {
        // downsampled camera: keep the raw depth; downsample_kernel averages and finishes it
        p.raw[(int64_t)e * p.raw_per_env + cam.raw_off + (int64_t)y * cam.width + x] = z;
    } else {
        finish_pixel(p, e, c, cam, x, y, z, step, __float_as_uint(CV.w));
    }

    if (kCount) {
        const unsigned mask = __activemask();
        const unsigned v[6] = {1u, cnt_t.nodes, cnt_t.tris, n_boxes, cnt_l.nodes, cnt_l.tris};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const unsigned s = __reduce_add_sync(mask, v[k]);
            if (lane == __ffs(mask) - 1) atomicAdd(p.counters + k, (unsigned long long)s);
        }
    }
}

template <bool kCount, int kKind, bool kTileInfo>
__device__ __forceinline__ void render_tile(const RenderParams &p, int64_t warp, int lane, int64_t step) {
    int e, r_tile;
    split_tile(warp, p, e, r_tile);
    render_tile<kCount, kKind, kTileInfo>(p, warp, e, r_tile, lane, step);
}

// What a tile's rays need, derived from (env, tile within the env, lane): camera, pixel, ray,
// z-depth scale, initial bound, latency word, terrain entry nodes and link mask.  The same arithmetic
// as render_tile's setup, so the rays are bit-identical.
struct TileSetup {
    int c, x, y;
    bool active;
    float3 d, base, off;
    float m, tmax0;
    uint32_t lat;
    int entry, entry2;
    uint64_t link_mask;
};

__device__ __forceinline__ TileSetup tile_setup(const RenderParams &p, int64_t warp, int e, int r_tile, int lane) {
    TileSetup t;
    int c = 0;
    while (c + 1 < p.C && r_tile >= p.cams[c + 1].tile_off) ++c;
    const CamDev &cam = p.cams[c];
    const int tw_log2 = p.tile_w_log2, th = 32 >> tw_log2;
    int trow, tcol;
    tile_row_col(cam, r_tile - cam.tile_off, trow, tcol);
    t.c = c;
    t.x = tcol * (1 << tw_log2) + (lane & ((1 << tw_log2) - 1));
    t.y = trow * th + (lane >> tw_log2);
    t.active = t.x < cam.width && t.y < cam.height;
    const int xs = min(t.x, cam.width - 1), ys = min(t.y, cam.height - 1);
    float fx = cam.fx, fy = cam.fy, cx = cam.cx, cy = cam.cy;
    if (p.intr) {
        const float4 k = __ldg(reinterpret_cast<const float4 *>(p.intr) + (int64_t)e * p.C + c);
        fx = k.x; fy = k.y; cx = k.z; cy = k.w;
    }
    const float4 *cx4 = p.cam_xf + 5 * ((int64_t)e * p.C + c);
    const float4 R0 = __ldg(cx4), R1 = __ldg(cx4 + 1), R2 = __ldg(cx4 + 2), OF = __ldg(cx4 + 3);
    const float4 CV = __ldg(cx4 + 4);
    const float rx = __fdividef((float)xs - cx, fx), ry = __fdividef((float)ys - cy, fy);
    const float inv_n = rsqrtf(rx * rx + ry * ry + 1.0f);
    const float ux = rx * inv_n, uy = ry * inv_n, uz = inv_n;
    t.d = make_float3(R0.x * ux + R0.y * uy + R0.z * uz, R1.x * ux + R1.y * uy + R1.z * uz,
                      R2.x * ux + R2.y * uy + R2.z * uz);
    t.base = make_float3(R0.w, R1.w, R2.w);
    t.off = make_float3(OF.x, OF.y, OF.z);
    t.m = p.depth_kind == RPL_DEPTH_Z ? inv_n : 1.0f;
    t.tmax0 = __fdividef(cam.d_max, t.m);
    t.lat = __float_as_uint(CV.w);
    const int4 ti = __ldg(p.tile_info + warp);
    t.entry = ti.x;
    t.entry2 = ti.w;
    t.link_mask = ((uint64_t)(uint32_t)ti.z << 32) | (uint32_t)ti.y;
    return t;
}

// One tile with tile info, links queried first (Alg. 1's order), in the per-SM queued launch: the
// same results as render_tile, but for a tile with links to test the setup is derived again after
// the link queries (the compiler is kept from reusing it) instead of being held in registers
// through them, which lowers the register pressure of the whole kernel (the terrain traversal runs
// with fewer spills).
template <int kKind>
__device__ __forceinline__ void render_tile_links_first(const RenderParams &p, int64_t warp, int e, int r_tile,
                                                        int lane, int64_t step) {
    TileSetup t = tile_setup(p, warp, e, r_tile, lane);
    if (!t.active) return;
    float tmax = t.tmax0;
    bool hit = false, ok = true;
    Counts cnt;
#ifdef RPL_CHECKED
    uint32_t ck_err = 0;
#endif
    if (t.link_mask != 0) {
        // 1) the robot bodies the tile can reach: rays move into each link frame
        Ray ray;
        make_ray(ray, t.base, t.off, t.d);
        const float3 base = t.base, off = t.off, d = t.d;
        const uint64_t link_mask = t.link_mask;
#pragma unroll 1
        for (uint64_t mk = link_mask; mk; mk &= mk - 1) {
            const int l = __ffsll((long long)mk) - 1;
            const int root = p.lroot[l];
            if (root < 0) continue;
            const int64_t el = (int64_t)e * p.L + l;
            const float4 blo = __ldg(p.link_box + 2 * el), bhi = __ldg(p.link_box + 2 * el + 1);
            if (slab(ray, blo.x, bhi.x, blo.y, bhi.y, blo.z, bhi.z, tmax) == CUDART_INF_F) continue;
            const float4 X0 = __ldg(p.link_xf + 3 * el), X1 = __ldg(p.link_xf + 3 * el + 1),
                         X2 = __ldg(p.link_xf + 3 * el + 2);
            const float3 rel = make_float3((base.x - X0.w) + off.x, (base.y - X1.w) + off.y, (base.z - X2.w) + off.z);
            const float3 ob = make_float3(X0.x * rel.x + X0.y * rel.y + X0.z * rel.z,
                                          X1.x * rel.x + X1.y * rel.y + X1.z * rel.z,
                                          X2.x * rel.x + X2.y * rel.y + X2.z * rel.z);
            const float3 db = make_float3(X0.x * d.x + X0.y * d.y + X0.z * d.z, X1.x * d.x + X1.y * d.y + X1.z * d.z,
                                          X2.x * d.x + X2.y * d.y + X2.z * d.z);
            Ray lr;
            make_ray(lr, ob, make_float3(0.f, 0.f, 0.f), db);
            ok &= traverse<false, false>(p.lnodes, p.ltris, root, -1, lr, tmax, hit, cnt
                                         RPL_CK_ARGS(p.n_lnodes, p.n_ltris, ck_err));
        }
        // an empty asm that may change these inputs, as far as the compiler knows: the setup is
        // computed again from them rather than kept live through the link queries
        asm volatile("" : "+r"(r_tile), "+l"(warp), "+r"(e));
        t = tile_setup(p, warp, e, r_tile, lane);
    }
    // 2) the static terrain, bounded by the closest body hit
    Ray ray;
    make_ray(ray, t.base, t.off, t.d);
    if (kKind == RPL_BVH8Q8) {
        const int oct = (t.d.x < 0.f ? 1 : 0) | (t.d.y < 0.f ? 2 : 0) | (t.d.z < 0.f ? 4 : 0);
        ok &= traverse8<false>(p.tnodes, p.ttris, t.entry, ray, oct, tmax, hit, cnt
                               RPL_CK_ARGS(p.n_tnodes, p.n_ttris, ck_err));
    } else if (kKind == RPL_BVH4) {
        ok &= traverse4<false>(p.tnodes, p.ttris, t.entry, ray, tmax, hit, cnt RPL_CK_ARGS(p.n_tnodes, p.n_ttris, ck_err));
    } else {
        ok &= traverse<true, false>(p.tnodes, p.ttris, t.entry, t.entry2, ray, tmax, hit, cnt
                                    RPL_CK_ARGS(p.n_tnodes, p.n_ttris, ck_err));
    }
    if (!ok) atomicOr(p.err, 1);
#ifdef RPL_CHECKED
    if (ck_err) atomicOr(p.err, (int)ck_err);
#endif
    const CamDev &cam = p.cams[t.c];
    const float z = hit ? fminf(t.m * tmax, cam.d_max) : cam.d_max;
    if (cam.ds > 1) {
        // downsampled camera: keep the raw depth; downsample_kernel averages and finishes it
        p.raw[(int64_t)e * p.raw_per_env + cam.raw_off + (int64_t)t.y * cam.width + t.x] = z;
    } else {
        finish_pixel(p, e, t.c, cam, t.x, t.y, z, step, t.lat);
    }
}

// kMinBlocks caps registers so that many blocks of 128 threads stay resident per SM (8 -> 64
// registers, 9 -> 56, 10 -> 48, 12 -> 40).  With p.persistent the grid holds only as many blocks as fit on
// the device at once and each warp walks the tiles with a grid stride; otherwise one warp per tile.
// kQueued (p.queues set, same grid as persistent): warps take tiles from per-SM queues instead.
// kTileInfo = false serves callers that run no tile prep (p.tile_info null).
// First tile of queue q when `total` tiles are split into nq contiguous queues (the first total mod
// nq queues hold one tile more).
__device__ __forceinline__ int64_t queue_begin(int64_t total, int q, int nq) {
    const int64_t base = total / nq, rem = total - base * nq;
    return base * q + min((int64_t)q, rem);
}

// Tiles of queue q: a contiguous range (chunk == 0), or chunks q, q + nq, q + 2 nq, ... of `chunk`
// tiles each (the last chunk of all may be short).
__device__ __forceinline__ int64_t queue_size(int64_t total, int q, int nq, int64_t chunk) {
    if (chunk <= 0) return queue_begin(total, q + 1, nq) - queue_begin(total, q, nq);
    const int64_t nc = (total + chunk - 1) / chunk;
    if (q >= nc) return 0;
    const int64_t mine = (nc - 1 - q) / nq + 1;           // chunks of queue q
    const int64_t last = q + (mine - 1) * nq;
    return mine * chunk - (last == nc - 1 ? nc * chunk - total : 0);
}

// Processing-order position of the k-th tile of queue q (k < queue_size); b = queue_begin(total, q,
// nq) when chunk == 0.  32-bit division whenever the operands fit.
__device__ __forceinline__ int64_t queue_tile(int q, int nq, int64_t chunk, int64_t b, int64_t k) {
    if (chunk <= 0) return b + k;
    int64_t j;
    if ((uint64_t)k < 0x100000000ull && (uint64_t)chunk < 0x100000000ull)
        j = (int64_t)((uint32_t)k / (uint32_t)chunk);
    else
        j = k / chunk;
    return (q + j * nq) * chunk + (k - j * chunk);
}

// Per-SM scheduling (p.queues set): the tiles are split into p.n_queues contiguous queues, one per
// SM.  A warp takes the next tile of its SM's queue (one atomic per tile), so the SM's warps work on
// neighbouring tiles of the same images, whose terrain nodes they share in L1; a warp whose block
// siblings are still busy does not idle, since it takes tiles by itself.  When the SM's queue is
// empty the warp moves to the queue with the most tiles left, until every queue is empty.  Each
// warp that finds its queue empty reads every counter (bypassing L1), so it ends only when all
// queues were seen empty.
// kLinksFirst (with tile info, not counting): the tiles are rendered by render_tile_links_first.
template <bool kCount, int kKind, bool kTileInfo, bool kLinksFirst = false>
__device__ __forceinline__ void render_queued(const RenderParams &p, int lane, int64_t total, int64_t step) {
    const int nq = p.n_queues;
    const int64_t chunk = (int64_t)p.chunk_envs * p.tiles_per_env;
    uint32_t smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    int q = (int)(smid % (uint32_t)nq);
    int64_t qsize = queue_size(total, q, nq, chunk), qbegin = queue_begin(total, q, nq);
    // multiply-and-shift divisions whenever every tile position fits in 31 bits and the host set the
    // magics of the divisors
    const bool small = total < 0x7FFFFFFFll && p.tpe_m != 0u && (chunk <= 0 || p.chunk_m != 0u);
#pragma unroll 1
    for (;;) {
        unsigned long long k = 0ull;
        if (lane == 0) k = atomicAdd(p.queues + q, 1ull);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k < (unsigned long long)qsize) {
            // the tile's position in processing order, then its env (through the env order) and index
            int e, r;
            if (small) {
                uint32_t pos;
                if (chunk <= 0) {
                    pos = (uint32_t)(qbegin + (int64_t)k);
                } else {
                    const uint32_t j = fastdiv((uint32_t)k, p.chunk_m, p.chunk_k);
                    pos = (uint32_t)(q + j * nq) * (uint32_t)chunk + ((uint32_t)k - j * (uint32_t)chunk);
                }
                e = (int)fastdiv(pos, p.tpe_m, p.tpe_k);
                r = (int)(pos - (uint32_t)e * (uint32_t)p.tiles_per_env);
            } else {
                split_tile(queue_tile(q, nq, chunk, qbegin, (int64_t)k), p, e, r);
            }
            if (p.env_order) e = __ldg(p.env_order + e);
            if constexpr (kLinksFirst && kTileInfo && !kCount)
                render_tile_links_first<kKind>(p, (int64_t)e * p.tiles_per_env + r, e, r, lane, step);
            else
                render_tile<kCount, kKind, kTileInfo>(p, (int64_t)e * p.tiles_per_env + r, e, r, lane, step);
            continue;
        }
        // this queue is empty: the queue with the most tiles left (warp-wide argmax)
        int64_t best = 0;
        int best_q = -1;
        for (int j = lane; j < nq; j += 32) {
            const int64_t sz = queue_size(total, j, nq, chunk);
            const unsigned long long taken = __ldcg(p.queues + j);
            const int64_t left = taken < (unsigned long long)sz ? sz - (int64_t)taken : 0;
            if (left > best) {
                best = left;
                best_q = j;
            }
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            const int64_t ob = __shfl_xor_sync(0xffffffffu, best, s);
            const int oq = __shfl_xor_sync(0xffffffffu, best_q, s);
            if (ob > best || (ob == best && oq > best_q)) {
                best = ob;
                best_q = oq;
            }
        }
        if (best <= 0) return;
        q = best_q;
        qsize = queue_size(total, q, nq, chunk);
        qbegin = queue_begin(total, q, nq);
    }
}

template <bool kCount, int kKind, int kMinBlocks, bool kTileInfo = true, bool kQueued = false, bool kLinksFirst = false>
__global__ void __launch_bounds__(128, kMinBlocks) render_kernel(const __grid_constant__ RenderParams p) {
    const int lane = threadIdx.x & 31;
    const int64_t total = (int64_t)p.E * p.tiles_per_env;
    const int64_t step = p.step_dev ? *p.step_dev : p.step;
    if (kQueued) {
        render_queued<kCount, kKind, kTileInfo, kLinksFirst>(p, lane, total, step);
        return;
    }
    const int64_t stride = (int64_t)gridDim.x * (blockDim.x >> 5);
#pragma unroll 1
    for (int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); warp < total; warp += stride)
        render_tile<kCount, kKind, kTileInfo>(p, tile_of(p, warp), lane, step);
}

// Terrain entry node and link mask of every tile, one thread per tile of 32 rays (the same work done
// by the tile's warp would occupy 32 lanes): the view pyramid of the tile's pixel rectangle; the
// deepest terrain node below the camera's entry node that holds the pyramid's AABB; and the links of
// the camera's mask whose world box meets the pyramid.  The corner directions use the same
// arithmetic as the render kernel's rays; the padding of each test covers their FP32 rounding.
// At most 80 registers (3 blocks of 256 per SM): its time is mostly the latency of dependent node
// fetches, which more resident threads hide (measured: 3 blocks beat 2, 4 and 6).
__global__ void __launch_bounds__(256, 3) tile_prep_kernel(const __grid_constant__ RenderParams p) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)p.E * p.tiles_per_env) return;
    int e, r_tile;
    split_tile(i, p, e, r_tile);
    int c = 0;
    while (c + 1 < p.C && r_tile >= p.cams[c + 1].tile_off) ++c;
    const CamDev &cam = p.cams[c];
    const int tw = 1 << p.tile_w_log2, th = 32 >> p.tile_w_log2;
    int trow, tcol;
    tile_row_col(cam, r_tile - cam.tile_off, trow, tcol);
    const int x0 = tcol * tw, y0 = trow * th;
    const int x1 = min(x0 + tw, cam.width) - 1, y1 = min(y0 + th, cam.height) - 1;
    float fx = cam.fx, fy = cam.fy, cx = cam.cx, cy = cam.cy;
    if (p.intr) {
        const float4 k = __ldg(reinterpret_cast<const float4 *>(p.intr) + (int64_t)e * p.C + c);
        fx = k.x; fy = k.y; cx = k.z; cy = k.w;
    }
    const float4 *cx4 = p.cam_xf + 5 * ((int64_t)e * p.C + c);
    const float4 R0 = __ldg(cx4), R1 = __ldg(cx4 + 1), R2 = __ldg(cx4 + 2), OF = __ldg(cx4 + 3);
    const float4 CV = __ldg(cx4 + 4);
    const uint64_t cam_mask = ((uint64_t)__float_as_uint(CV.y) << 32) | __float_as_uint(CV.x);
    const float o[3] = {R0.w + OF.x, R1.w + OF.y, R2.w + OF.z};
    const float rxa = __fdividef((float)x0 - cx, fx), rxb = __fdividef((float)x1 - cx, fx);
    const float rya = __fdividef((float)y0 - cy, fy), ryb = __fdividef((float)y1 - cy, fy);
    float B[4][3];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        // ring order: (x0, y0), (x1, y0), (x1, y1), (x0, y1)
        const float rx = (k == 1 || k == 2) ? rxb : rxa, ry = k >= 2 ? ryb : rya;
        B[k][0] = o[0] + cam.d_max * (R0.x * rx + R0.y * ry + R0.z);
        B[k][1] = o[1] + cam.d_max * (R1.x * rx + R1.y * ry + R1.z);
        B[k][2] = o[2] + cam.d_max * (R2.x * rx + R2.y * ry + R2.z);
    }
    Pyramid V;
    const float axis[3] = {R0.z, R1.z, R2.z};
    make_pyramid(V, o, B, axis, cam.d_max);
    // terrain entry: for the binary layout, the pyramid descent, continued below a node where the
    // pyramid meets both children (two subtrees, the one nearer the camera first)
    int entry, entry2 = -1;
    if (p.bvh_kind == RPL_BVH2) {
        int ca, cb;
        entry = descend_binary_pyramid(p.tnodes, __float_as_int(CV.z), V, ca, cb RPL_CK_DESCEND_ARGS(p.n_tnodes));
        if (ca >= 0) {
            const float4 *n = p.tnodes + 4 * entry;
            const float4 n0 = __ldg(n), n1 = __ldg(n + 1), n2 = __ldg(n + 2);
            const float lo0[3] = {n0.x, n0.z, n2.x}, hi0[3] = {n0.y, n0.w, n2.y};
            const float lo1[3] = {n1.x, n1.z, n2.z}, hi1[3] = {n1.y, n1.w, n2.w};
            int ea = ca, eb = cb;
            descend_binary_pyramid2(p.tnodes, ea, eb, V RPL_CK_DESCEND_ARGS(p.n_tnodes));
            const bool a_first = box_dist2(o, lo0, hi0) <= box_dist2(o, lo1, hi1);
            entry = a_first ? ea : eb;
            entry2 = a_first ? eb : ea;
        }
    } else {
        entry = descend_any(p.bvh_kind, p.tnodes, __float_as_int(CV.z), V.lo, V.hi RPL_CK_DESCEND_ARGS(p.n_tnodes));
    }
    uint64_t mask = 0;
#pragma unroll 1
    for (uint64_t mk = cam_mask; mk; mk &= mk - 1) {
        const int l = __ffsll((long long)mk) - 1;
        const int64_t el = (int64_t)e * p.L + l;
        const float4 blo = __ldg(p.link_box + 2 * el), bhi = __ldg(p.link_box + 2 * el + 1);
        const float lo[3] = {blo.x, blo.y, blo.z}, hi[3] = {bhi.x, bhi.y, bhi.z};
        if (!pyramid_meets_box(V, lo, hi)) continue;
        // the link's oriented box: its link-frame root box under the link pose (rows of R^T are the
        // world directions of the link axes)
        const float4 X0 = __ldg(p.link_xf + 3 * el), X1 = __ldg(p.link_xf + 3 * el + 1),
                     X2 = __ldg(p.link_xf + 3 * el + 2);
        const float4 rl = __ldg(p.link_root + 2 * l), rh = __ldg(p.link_root + 2 * l + 1);
        const float A[3][3] = {{X0.x, X0.y, X0.z}, {X1.x, X1.y, X1.z}, {X2.x, X2.y, X2.z}};
        const float cl[3] = {0.5f * (rl.x + rh.x), 0.5f * (rl.y + rh.y), 0.5f * (rl.z + rh.z)};
        const float h[3] = {0.5f * (rh.x - rl.x), 0.5f * (rh.y - rl.y), 0.5f * (rh.z - rl.z)};
        const float cw[3] = {A[0][0] * cl[0] + A[1][0] * cl[1] + A[2][0] * cl[2] + X0.w,
                             A[0][1] * cl[0] + A[1][1] * cl[1] + A[2][1] * cl[2] + X1.w,
                             A[0][2] * cl[0] + A[1][2] * cl[1] + A[2][2] * cl[2] + X2.w};
        if (pyramid_meets_obb(V, cw, A, h)) mask |= 1ull << l;
    }
    p.tile_info[i] = make_int4(entry, (int)(uint32_t)mask, (int)(uint32_t)(mask >> 32), entry2);
}

// Several render requests (each with its own view, envs, cameras and sensor) in one launch: the
// tiles of request r occupy warps [prefix[r], prefix[r + 1]); each warp finds its request by binary
// search and renders one tile with that request's parameters (read from global memory).
template <int kKind, int kMinBlocks>
__global__ void __launch_bounds__(128, kMinBlocks)
    render_multi_kernel(const RenderParams *__restrict__ reqs, const int64_t *__restrict__ prefix, int n_req) {
    const int lane = threadIdx.x & 31;
    const int64_t total = prefix[n_req];
    const int64_t stride = (int64_t)gridDim.x * (blockDim.x >> 5);
#pragma unroll 1
    for (int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); warp < total; warp += stride) {
        int lo = 0, hi = n_req - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= warp) lo = mid;
            else hi = mid - 1;
        }
        const RenderParams &p = reqs[lo];
        const int64_t step = p.step_dev ? *p.step_dev : p.step;
        render_tile<false, kKind, true>(p, warp - prefix[lo], lane, step);
        if (p.done_counter) {
            // per-request completion inside the fused launch: every lane's stores are made visible,
            // then the warp counts its tile off; the warp that finishes the request's last tile
            // raises the request's flag in host-mapped memory (the last-block pattern)
            __threadfence();
            __syncwarp();
            if (lane == 0 && atomicSub(p.done_counter, 1) == 1) {
                __threadfence_system();
                *reinterpret_cast<volatile int32_t *>(p.done_flag) = 1;
            }
        }
    }
}

// Output pixels of downsampled cameras: one thread per output pixel of one env (grid-stride over
// E x pix_per_env); the mean of the f x f raw depths, summed row by row in FP32, then the sensor.
__global__ void __launch_bounds__(256) downsample_kernel(const __grid_constant__ RenderParams p) {
    const int64_t total = (int64_t)p.E * p.pix_per_env;
    const int64_t step = p.step_dev ? *p.step_dev : p.step;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(i / p.pix_per_env);
        const int col = (int)(i - (int64_t)e * p.pix_per_env);
        int c = 0;
        while (c + 1 < p.C && col >= p.cams[c + 1].pix_off) ++c;
        const CamDev &cam = p.cams[c];
        if (cam.ds <= 1) continue;
        const int pix = col - cam.pix_off;
        const int y = pix / cam.out_w, x = pix - y * cam.out_w;
        const float *src = p.raw + (int64_t)e * p.raw_per_env + cam.raw_off + (int64_t)(y * cam.ds) * cam.width + x * cam.ds;
        float sum = 0.f;
        for (int j = 0; j < cam.ds; ++j)
            for (int k = 0; k < cam.ds; ++k) sum += src[(int64_t)j * cam.width + k];
        const float z = __fdiv_rn(sum, (float)(cam.ds * cam.ds));
        const float4 CV = __ldg(p.cam_xf + 5 * ((int64_t)e * p.C + c) + 4);
        finish_pixel(p, e, c, cam, x, y, z, step, __float_as_uint(CV.w));
    }
}

// The sensor model alone on caller-provided pre-sensor depth `src` ([E, pix_per_env], the output
// layout): one thread per output pixel; the latency of (env, camera, step) is drawn here the way the
// prep kernel draws it.
__global__ void __launch_bounds__(256) sensor_kernel(const __grid_constant__ RenderParams p, const float *src) {
    const int64_t total = (int64_t)p.E * p.pix_per_env;
    const int64_t step = p.step;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(i / p.pix_per_env);
        const int col = (int)(i - (int64_t)e * p.pix_per_env);
        int c = 0;
        while (c + 1 < p.C && col >= p.cams[c + 1].pix_off) ++c;
        const CamDev &cam = p.cams[c];
        const int pix = col - cam.pix_off;
        const int y = pix / cam.out_w, x = pix - y * cam.out_w;
        const uint32_t lat = p.span > 1 ? latency_word(p.env_offset + (uint32_t)e, (uint32_t)c, step, p.s_first[e],
                                                       p.span, p.seed0, p.seed1)
                                        : 0u;
        finish_pixel(p, e, c, cam, x, y, src[i], step, lat);
    }
}

// Graph replays read the step from device memory; this advances it after each replayed render.
__global__ void advance_step_kernel(int64_t *step) { *step += 1; }

__global__ void set_first_kernel(int64_t *s_first, int32_t E, int64_t step, const uint8_t *mask) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < E && (mask == nullptr || mask[i] != 0)) s_first[i] = step;
}

// Counting sort of the envs by their spatial key in one block: histogram of the kOrderBuckets keys in
// shared memory, exclusive prefix sum, then each env's slot by an atomic increment of its bucket's
// offset (so the order inside a bucket is arbitrary).
__global__ void __launch_bounds__(1024) env_order_kernel(const uint32_t *__restrict__ key, int32_t *__restrict__ order,
                                                         int32_t E) {
    constexpr int kPer = kOrderBuckets / 1024;
    __shared__ uint32_t h[kOrderBuckets];
    __shared__ uint32_t warp_sum[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int i = t; i < kOrderBuckets; i += 1024) h[i] = 0u;
    __syncthreads();
    for (int64_t e = t; e < E; e += 1024) atomicAdd(&h[__ldg(key + e) & (kOrderBuckets - 1)], 1u);
    __syncthreads();
    // exclusive scan: each thread owns kPer consecutive buckets
    uint32_t v[kPer], sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        v[k] = h[t * kPer + k];
        sum += v[k];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, inc, s);
        if (lane >= s) inc += o;
    }
    if (lane == 31) warp_sum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = warp_sum[lane], wi = w;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, wi, s);
            if (lane >= s) wi += o;
        }
        warp_sum[lane] = wi - w;   // exclusive prefix of the warps
    }
    __syncthreads();
    uint32_t run = warp_sum[wid] + inc - sum;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        h[t * kPer + k] = run;
        run += v[k];
    }
    __syncthreads();
    for (int64_t e = t; e < E; e += 1024) order[atomicAdd(&h[__ldg(key + e) & (kOrderBuckets - 1)], 1u)] = (int32_t)e;
}

}  // namespace

cudaError_t launch_prep(const PrepParams &p, cudaStream_t s) {
    if ((int64_t)p.E * (p.L + p.C) == 0) return cudaSuccess;
    // one thread per (env, link), then (from a warp boundary) four per (env, camera)
    const int64_t n = (((int64_t)p.E * p.L + 31) & ~(int64_t)31) + 4 * (int64_t)p.E * p.C;
    (void)cudaGetLastError();   // report only this launch's error, not a stale one
    prep_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p);
    return cudaGetLastError();
}

namespace {

// The render kernel for one terrain layout; the counting variant runs with 8 blocks per SM.
template <int kKind>
void launch_kind(const RenderParams &p, bool count, int min_blocks, unsigned g, cudaStream_t s) {
    if (p.tile_info == nullptr)
        render_kernel<false, kKind, 8, false><<<g, 128, 0, s>>>(p);   // callers without tile prep (no counters)
    else if (count)
        render_kernel<true, kKind, 8><<<g, 128, 0, s>>>(p);
    else if (p.queues && !p.terrain_first && min_blocks == 12)
        render_kernel<false, kKind, 12, true, true, true><<<g, 128, 0, s>>>(p);
    else if (p.queues && !p.terrain_first && min_blocks == 10)
        render_kernel<false, kKind, 10, true, true, true><<<g, 128, 0, s>>>(p);
    else if (p.queues && !p.terrain_first && min_blocks == 9)
        render_kernel<false, kKind, 9, true, true, true><<<g, 128, 0, s>>>(p);
    else if (p.queues && !p.terrain_first)
        render_kernel<false, kKind, 8, true, true, true><<<g, 128, 0, s>>>(p);
    else if (p.queues && min_blocks == 12)
        render_kernel<false, kKind, 12, true, true><<<g, 128, 0, s>>>(p);
    else if (p.queues && min_blocks == 10)
        render_kernel<false, kKind, 10, true, true><<<g, 128, 0, s>>>(p);
    else if (p.queues && min_blocks == 9)
        render_kernel<false, kKind, 9, true, true><<<g, 128, 0, s>>>(p);
    else if (p.queues)
        render_kernel<false, kKind, 8, true, true><<<g, 128, 0, s>>>(p);
    else if (min_blocks == 12)
        render_kernel<false, kKind, 12><<<g, 128, 0, s>>>(p);
    else if (min_blocks == 10)
        render_kernel<false, kKind, 10><<<g, 128, 0, s>>>(p);
    else if (min_blocks == 9)
        render_kernel<false, kKind, 9><<<g, 128, 0, s>>>(p);
    else
        render_kernel<false, kKind, 8><<<g, 128, 0, s>>>(p);
}

template <int kKind>
void launch_multi_kind(const RenderParams *reqs_dev, const int64_t *prefix_dev, int n_req, int min_blocks, unsigned g,
                       cudaStream_t s) {
    if (min_blocks == 12)
        render_multi_kernel<kKind, 12><<<g, 128, 0, s>>>(reqs_dev, prefix_dev, n_req);
    else if (min_blocks == 10)
        render_multi_kernel<kKind, 10><<<g, 128, 0, s>>>(reqs_dev, prefix_dev, n_req);
    else
        render_multi_kernel<kKind, 8><<<g, 128, 0, s>>>(reqs_dev, prefix_dev, n_req);
}

}  // namespace

cudaError_t launch_tile_prep(const RenderParams &p, cudaStream_t s) {
    const int64_t n = (int64_t)p.E * p.tiles_per_env;
    if (n == 0 || p.tile_info == nullptr) return cudaSuccess;
    (void)cudaGetLastError();
    tile_prep_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_render(const RenderParams &p, bool count, cudaStream_t s) {
    const int64_t warps = (int64_t)p.E * p.tiles_per_env;
    if (warps == 0) return cudaSuccess;
    const int min_blocks = p.min_blocks == 12 ? 12 : p.min_blocks == 10 ? 10 : p.min_blocks == 9 ? 9 : 8;
    int64_t blocks = (warps + 3) / 4;
    if (p.persistent || (p.queues && p.tile_info && !count)) {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ==
                                                       cudaSuccess && sms > 0)
            blocks = std::min<int64_t>(blocks, (int64_t)sms * min_blocks);
    }
    (void)cudaGetLastError();
    const unsigned g = (unsigned)blocks;
    if (p.bvh_kind == RPL_BVH8Q8)
        launch_kind<RPL_BVH8Q8>(p, count, min_blocks, g, s);
    else if (p.bvh_kind == RPL_BVH4)
        launch_kind<RPL_BVH4>(p, count, min_blocks, g, s);
    else
        launch_kind<RPL_BVH2>(p, count, min_blocks, g, s);
    return cudaGetLastError();
}

cudaError_t launch_downsample(const RenderParams &p, cudaStream_t s) {
    const int64_t n = (int64_t)p.E * p.pix_per_env;
    if (p.raw_per_env == 0 || n == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    int64_t blocks = (n + 255) / 256;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ==
                                                   cudaSuccess && sms > 0)
        blocks = std::min<int64_t>(blocks, (int64_t)sms * 8);
    (void)cudaGetLastError();
    downsample_kernel<<<(unsigned)blocks, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_sensor(const RenderParams &p, const float *src, cudaStream_t s) {
    const int64_t n = (int64_t)p.E * p.pix_per_env;
    if (n == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    int64_t blocks = (n + 255) / 256;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ==
                                                   cudaSuccess && sms > 0)
        blocks = std::min<int64_t>(blocks, (int64_t)sms * 8);
    (void)cudaGetLastError();
    sensor_kernel<<<(unsigned)blocks, 256, 0, s>>>(p, src);
    return cudaGetLastError();
}

cudaError_t launch_render_multi(const RenderParams *reqs_dev, const int64_t *prefix_dev, int n_req,
                                int64_t total_warps, int bvh_kind, int min_blocks, bool persistent, cudaStream_t s) {
    if (total_warps <= 0 || n_req <= 0) return cudaSuccess;
    int64_t blocks = (total_warps + 3) / 4;
    const int mb = min_blocks == 12 ? 12 : (min_blocks == 10 ? 10 : 8);
    if (persistent) {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ==
                                                       cudaSuccess && sms > 0)
            blocks = std::min<int64_t>(blocks, (int64_t)sms * mb);
    }
    (void)cudaGetLastError();
    const unsigned g = (unsigned)blocks;
    if (bvh_kind == RPL_BVH8Q8)
        launch_multi_kind<RPL_BVH8Q8>(reqs_dev, prefix_dev, n_req, mb, g, s);
    else if (bvh_kind == RPL_BVH4)
        launch_multi_kind<RPL_BVH4>(reqs_dev, prefix_dev, n_req, mb, g, s);
    else
        launch_multi_kind<RPL_BVH2>(reqs_dev, prefix_dev, n_req, mb, g, s);
    return cudaGetLastError();
}

cudaError_t launch_env_order(const uint32_t *key, int32_t *order, int32_t E, cudaStream_t s) {
    if (E <= 0) return cudaSuccess;
    (void)cudaGetLastError();
    env_order_kernel<<<1, 1024, 0, s>>>(key, order, E);
    return cudaGetLastError();
}

cudaError_t launch_advance_step(int64_t *step, cudaStream_t s) {
    (void)cudaGetLastError();
    advance_step_kernel<<<1, 1, 0, s>>>(step);
    return cudaGetLastError();
}

cudaError_t launch_set_first(int64_t *s_first, int32_t E, int64_t step, const uint8_t *mask, cudaStream_t s) {
    if (E == 0) return cudaSuccess;
    (void)cudaGetLastError();
    set_first_kernel<<<(E + 255) / 256, 256, 0, s>>>(s_first, E, step, mask);
    return cudaGetLastError();
}

}  // namespace rpl
