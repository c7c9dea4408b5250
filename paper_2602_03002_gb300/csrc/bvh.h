// bvh.h -- in-memory layout of the BVHs shared by the host builder, the C-ABI layer and the kernels.
//
// Binary BVH ("BVH2") in the two-children-per-node layout: one 64-byte node holds the bounding
// boxes of both children, so one node fetch (four 16-byte vector loads) lets a ray decide which
// children to visit.  Triangles are stored leaf-ordered, 48 bytes each (three float4 = the three
// vertices), so that a leaf is one contiguous run of vector loads.  Shared vertices are duplicated
// bit-exactly, which the watertight triangle test relies on.
#pragma once
#include <cstdint>
#include <vector>

namespace rpl {

// 64-byte node.  Child encoding: c >= 0 is the index of an inner node; c < 0 is a leaf whose
// first triangle is ~c and whose triangle count is in cnt0/cnt1 (0 = empty child, never hit:
// its box is inverted).
struct alignas(16) BvhNode {
    float c0lox, c0hix, c0loy, c0hiy;   // float4 #0
    float c1lox, c1hix, c1loy, c1hiy;   // float4 #1
    float c0loz, c0hiz, c1loz, c1hiz;   // float4 #2
    int32_t child0, child1, cnt0, cnt1; // int4   #3
};
static_assert(sizeof(BvhNode) == 64, "node is 64 bytes");

struct alignas(16) BvhTri {
    float v0x, v0y, v0z, id;    // id: original triangle index (bit pattern of an int32)
    float v1x, v1y, v1z, pad1;  // pad1: 1 on the device when this triangle (A, B, C) and the next
                                // one (A, C, D) form a pair sharing the edge A-C (a quad), else 0
    float v2x, v2y, v2z, pad2;
};
static_assert(sizeof(BvhTri) == 48, "triangle is 48 bytes");

struct HostBvh {
    std::vector<BvhNode> nodes;   // node 0 is the root (always an inner node)
    std::vector<BvhTri> tris;     // leaf order
    float root_lo[3], root_hi[3]; // bounds of all triangles (unpadded); inverted when empty
    int32_t depth = 0;            // inner-node levels on the longest root-to-leaf path
};

// Builds the BVH with binned SAH splits (16 bins, all three axes).  Deterministic for a given input
// whatever the thread count.  Child boxes are padded outward by max(|x| 2^-20, 1e-6) per bound, so
// that FP32 slab tests stay conservative for rays whose origin carries FP32 rounding.
// Returns 0, or -1 on a bad vertex index, -2 on allocation failure.
// node_cost: SAH cost of visiting a node relative to testing one triangle (larger -> bigger leaves).
int build_bvh2(const float *verts, int64_t n_verts, const int32_t *tris, int64_t n_tris,
               int max_leaf, int n_threads, HostBvh *out, double node_cost = 1.0);

}  // namespace rpl
