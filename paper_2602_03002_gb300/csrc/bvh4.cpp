// bvh4.cpp -- collapse of the binary SAH BVH into the four-wide full-precision layout (bvh4.h).
#include "bvh4.h"

#include <algorithm>

namespace rpl {
namespace {

struct Slot {
    float lo[3], hi[3];
    int32_t child;   // binary inner node index, or a leaf reference (< 0)
    int32_t count;   // leaf triangle count
};

float half_area(const Slot &s) {
    const float dx = s.hi[0] - s.lo[0], dy = s.hi[1] - s.lo[1], dz = s.hi[2] - s.lo[2];
    return dx * dy + dy * dz + dz * dx;
}

// The non-empty children of binary node n.
int binary_children(const HostBvh &b, int32_t n, Slot out[2]) {
    const BvhNode &nd = b.nodes[(size_t)n];
    int k = 0;
    if (!(nd.child0 < 0 && nd.cnt0 == 0))
        out[k++] = Slot{{nd.c0lox, nd.c0loy, nd.c0loz}, {nd.c0hix, nd.c0hiy, nd.c0hiz}, nd.child0, nd.cnt0};
    if (!(nd.child1 < 0 && nd.cnt1 == 0))
        out[k++] = Slot{{nd.c1lox, nd.c1loy, nd.c1loz}, {nd.c1hix, nd.c1hiy, nd.c1hiz}, nd.child1, nd.cnt1};
    return k;
}

}  // namespace

int collapse_bvh4(const HostBvh &b2, HostBvh4 *out) {
    out->nodes.clear();
    out->depth = 0;
    out->nodes.reserve(b2.nodes.size() / 2 + 1);
    struct Item {
        int32_t b2, index, depth;
    };
    std::vector<Item> stack;
    out->nodes.push_back(Bvh4Node{});
    stack.push_back(Item{0, 0, 1});
    while (!stack.empty()) {
        const Item it = stack.back();
        stack.pop_back();
        out->depth = std::max(out->depth, it.depth);
        Slot slots[4];
        int n = binary_children(b2, it.b2, slots);
        // open the largest inner child until four slots are filled or only leaves remain
        while (n < 4) {
            int best = -1;
            float best_area = -1.0f;
            for (int k = 0; k < n; ++k)
                if (slots[k].child >= 0 && half_area(slots[k]) > best_area) {
                    best = k;
                    best_area = half_area(slots[k]);
                }
            if (best < 0) break;
            Slot kids[2];
            const int m = binary_children(b2, slots[best].child, kids);
            if (n - 1 + m > 4) break;
            slots[best] = slots[n - 1];
            --n;
            for (int k = 0; k < m; ++k) slots[n++] = kids[k];
        }
        Bvh4Node node{};
        for (int k = 0; k < 4; ++k) {
            if (k >= n) {
                node.lox[k] = node.hix[k] = node.loy[k] = node.hiy[k] = node.loz[k] = node.hiz[k] = 1e30f;
                node.child[k] = -1;
                node.count[k] = 0;
                continue;
            }
            const Slot &s = slots[k];
            node.lox[k] = s.lo[0];
            node.hix[k] = s.hi[0];
            node.loy[k] = s.lo[1];
            node.hiy[k] = s.hi[1];
            node.loz[k] = s.lo[2];
            node.hiz[k] = s.hi[2];
            node.count[k] = s.count;
            if (s.child >= 0) {
                const int32_t idx = (int32_t)out->nodes.size();
                out->nodes.push_back(Bvh4Node{});
                node.child[k] = idx;
                stack.push_back(Item{s.child, idx, it.depth + 1});
            } else {
                node.child[k] = s.child;
            }
        }
        out->nodes[(size_t)it.index] = node;
    }
    return 0;
}

}  // namespace rpl
