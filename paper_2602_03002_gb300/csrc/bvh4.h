// bvh4.h -- four-wide BVH with full-precision child boxes, collapsed from the binary SAH BVH.
//
// One node is 128 bytes (eight 16-byte loads): the four child boxes stored axis by axis (lo x[4],
// hi x[4], lo y[4], hi y[4], lo z[4], hi z[4]), then the four child references and the four leaf
// triangle counts.  Child encoding as in the binary layout: c >= 0 is an inner node of this tree;
// c < 0 is a leaf whose first triangle is ~c with count[k] triangles.  An unused slot has count 0
// and a zero-size box at +1e30 on every axis, which no ray with a finite bound can hit, so the
// traversal needs no per-slot test for it.  The triangles are those of the binary tree, in its leaf
// order (collapsing regroups nodes only).  Halving the depth halves the chain of dependent node
// fetches a ray waits on, at four box tests per fetch.
#pragma once
#include <cstdint>
#include <vector>

#include "bvh.h"

namespace rpl {

struct alignas(16) Bvh4Node {
    float lox[4], hix[4], loy[4], hiy[4], loz[4], hiz[4];
    int32_t child[4];
    int32_t count[4];
};
static_assert(sizeof(Bvh4Node) == 128, "four-wide node is 128 bytes");

struct HostBvh4 {
    std::vector<Bvh4Node> nodes;   // node 0 is the root
    int32_t depth = 0;             // four-wide levels on the longest path
};

// Collapses a binary BVH into a four-wide one: each node takes its binary node's two children and
// repeatedly opens the inner child with the largest surface area until it has four children or
// only leaves.  Nodes are emitted in depth-first order.  Returns 0 (it cannot fail on a valid tree).
int collapse_bvh4(const HostBvh &b2, HostBvh4 *out);

}  // namespace rpl
