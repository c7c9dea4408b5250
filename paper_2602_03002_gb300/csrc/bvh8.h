// bvh8.h -- eight-wide BVH with 8-bit quantised child boxes, collapsed from the binary SAH BVH.
//
// One node is 80 bytes (five 16-byte loads):
//   w0..w2   origin of the quantisation grid (float bits): the node box's low corner
//   w3       exponent bytes ex | ey << 8 | ez << 16 (grid step 2^(e-127) per axis) | imask << 24
//   w4       index of the first inner child (inner children are stored contiguously)
//   w5       index of the first triangle of the node's leaf children (stored contiguously)
//   w6, w7   meta byte per child slot: 0 empty; inner 0x80 | rank among inner children;
//            leaf 0x80 | (triangle offset << 2) | (count - 1), count 1..4
//   w8..w19  q_lo x[8], q_lo y[8], q_lo z[8], q_hi x[8], q_hi y[8], q_hi z[8] (bytes, slot order)
// Child box = origin + q * step, rounded outward (floor for lo, ceil for hi) from boxes that are
// already padded, so the dequantised box always contains the child.  Empty slots have q_lo = 255,
// q_hi = 0 on every axis, which no slab test with ordered near/far planes can hit.  A child in slot
// s whose bits are (sx, sy, sz) lies towards +x if sx, etc., so visiting slots in the order
// i ^ octant(ray direction) is roughly front to back.
#pragma once
#include <cstdint>
#include <vector>

#include "bvh.h"

namespace rpl {

struct alignas(16) Bvh8Node {
    uint32_t w[20];
};
static_assert(sizeof(Bvh8Node) == 80, "wide node is 80 bytes");

struct HostBvh8 {
    std::vector<Bvh8Node> nodes;   // node 0 is the root
    std::vector<BvhTri> tris;      // leaf order of the wide tree
    int32_t depth = 0;             // wide levels on the longest path
};

// Collapses a binary BVH (leaves of at most 4 triangles) into an 8-wide quantised BVH.
// Returns 0, or -1 when a leaf holds more than 4 triangles.
int collapse_bvh8(const HostBvh &b2, HostBvh8 *out);

}  // namespace rpl
