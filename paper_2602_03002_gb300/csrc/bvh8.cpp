// bvh8.cpp -- collapse of the binary SAH BVH into the eight-wide quantised layout of bvh8.h.
//
// Each wide node takes a binary node and repeatedly replaces its largest-area inner child by that
// child's two children until it has eight children or only leaves (a greedy surface-area collapse).
// Wide nodes are emitted breadth first, so the inner children of a node are contiguous.
#include "bvh8.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace rpl {
namespace {

struct Child {
    int32_t enc, count;   // binary encoding: >= 0 inner node, < 0 leaf ~first with count triangles
    float lo[3], hi[3];
};

void child_of(const BvhNode &n, int k, Child &c) {
    if (k == 0) {
        c.enc = n.child0; c.count = n.cnt0;
        c.lo[0] = n.c0lox; c.hi[0] = n.c0hix; c.lo[1] = n.c0loy; c.hi[1] = n.c0hiy; c.lo[2] = n.c0loz; c.hi[2] = n.c0hiz;
    } else {
        c.enc = n.child1; c.count = n.cnt1;
        c.lo[0] = n.c1lox; c.hi[0] = n.c1hix; c.lo[1] = n.c1loy; c.hi[1] = n.c1hiy; c.lo[2] = n.c1loz; c.hi[2] = n.c1hiz;
    }
}

double half_area(const Child &c) {
    double dx = (double)c.hi[0] - c.lo[0], dy = (double)c.hi[1] - c.lo[1], dz = (double)c.hi[2] - c.lo[2];
    return dx * dy + dy * dz + dz * dx;
}

void set_byte(uint32_t *w, int word0, int idx, uint32_t v) {
    uint32_t &x = w[word0 + idx / 4];
    const int sh = 8 * (idx % 4);
    x = (x & ~(0xFFu << sh)) | ((v & 0xFFu) << sh);
}

}  // namespace

int collapse_bvh8(const HostBvh &b2, HostBvh8 *out) {
    out->nodes.clear();
    out->tris.clear();
    out->depth = 0;
    std::vector<std::pair<int32_t, int32_t>> pending;   // (binary inner node, wide index)
    std::vector<int32_t> level;
    out->nodes.resize(1);
    pending.push_back({0, 0});
    level.push_back(1);
    for (size_t qi = 0; qi < pending.size(); ++qi) {
        const int32_t n2 = pending[qi].first, wi = pending[qi].second;
        out->depth = std::max(out->depth, level[qi]);
        // gather up to eight children
        std::vector<Child> kids;
        for (int k = 0; k < 2; ++k) {
            Child c;
            child_of(b2.nodes[n2], k, c);
            if (c.enc < 0 && c.count == 0) continue;
            kids.push_back(c);
        }
        while (kids.size() < 8) {
            int best = -1;
            double area = -1.0;
            for (size_t i = 0; i < kids.size(); ++i)
                if (kids[i].enc >= 0 && half_area(kids[i]) > area) {
                    area = half_area(kids[i]);
                    best = (int)i;
                }
            if (best < 0) break;
            const BvhNode &m = b2.nodes[kids[best].enc];
            kids.erase(kids.begin() + best);
            for (int k = 0; k < 2; ++k) {
                Child c;
                child_of(m, k, c);
                if (c.enc < 0 && c.count == 0) continue;
                kids.push_back(c);
            }
        }
        for (const Child &c : kids)
            if (c.enc < 0 && c.count > 4) return -1;

        Bvh8Node node;
        std::memset(&node, 0, sizeof node);
        // empty slots: q_lo = 255, q_hi = 0 on every axis
        for (int s = 0; s < 8; ++s)
            for (int a = 0; a < 3; ++a) {
                set_byte(node.w, 8 + 2 * a, s, 255);
                set_byte(node.w, 14 + 2 * a, s, 0);
            }
        if (kids.empty()) {
            for (int a = 0; a < 3; ++a) {
                float z = 0.f;
                std::memcpy(&node.w[a], &z, 4);
                set_byte(&node.w[3], 0, a, 127);
            }
            out->nodes[wi] = node;
            continue;
        }
        float lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = kids[0].lo[a];
            hi[a] = kids[0].hi[a];
            for (const Child &c : kids) {
                lo[a] = std::min(lo[a], c.lo[a]);
                hi[a] = std::max(hi[a], c.hi[a]);
            }
        }
        double step[3];
        for (int a = 0; a < 3; ++a) {
            const double ext = (double)hi[a] - (double)lo[a];
            int e = ext > 0 ? (int)std::ceil(std::log2(ext / 255.0)) : -126;
            e = std::max(e, -126);
            while (std::ldexp(1.0, e) * 255.0 < ext) ++e;
            step[a] = std::ldexp(1.0, e);
            set_byte(&node.w[3], 0, a, (uint32_t)(e + 127));
            std::memcpy(&node.w[a], &lo[a], 4);
        }
        // slot assignment: child towards +axis goes to a slot with that axis bit set (greedy)
        const int k = (int)kids.size();
        int slot_of[8];
        {
            struct Pair { double score; int c, s; };
            std::vector<Pair> pairs;
            for (int c = 0; c < k; ++c)
                for (int s = 0; s < 8; ++s) {
                    double sc = 0;
                    for (int a = 0; a < 3; ++a) {
                        const double ext = std::max((double)hi[a] - lo[a], 1e-12);
                        const double rel = (0.5 * ((double)kids[c].lo[a] + kids[c].hi[a]) - 0.5 * ((double)lo[a] + hi[a])) / ext;
                        sc += ((s >> a) & 1) ? rel : -rel;
                    }
                    pairs.push_back({sc, c, s});
                }
            std::stable_sort(pairs.begin(), pairs.end(), [](const Pair &x, const Pair &y) { return x.score > y.score; });
            bool cused[8] = {}, sused[8] = {};
            for (int c = 0; c < k; ++c) slot_of[c] = -1;
            for (const Pair &p : pairs)
                if (!cused[p.c] && !sused[p.s]) {
                    cused[p.c] = sused[p.s] = true;
                    slot_of[p.c] = p.s;
                }
        }
        int child_at[8];
        for (int s = 0; s < 8; ++s) child_at[s] = -1;
        for (int c = 0; c < k; ++c) child_at[slot_of[c]] = c;
        // children in slot order: inner ones contiguous from child_base, leaf triangles from tri_base
        uint32_t imask = 0;
        int n_inner = 0;
        for (int s = 0; s < 8; ++s)
            if (child_at[s] >= 0 && kids[child_at[s]].enc >= 0) ++n_inner;
        const uint32_t child_base = (uint32_t)out->nodes.size();
        const uint32_t tri_base = (uint32_t)out->tris.size();
        out->nodes.resize(out->nodes.size() + n_inner);
        int rank = 0;
        for (int s = 0; s < 8; ++s) {
            if (child_at[s] < 0) continue;
            const Child &c = kids[child_at[s]];
            for (int a = 0; a < 3; ++a) {
                double ql = std::floor(((double)c.lo[a] - (double)lo[a]) / step[a]);
                double qh = std::ceil(((double)c.hi[a] - (double)lo[a]) / step[a]);
                ql = std::min(std::max(ql, 0.0), 255.0);
                qh = std::min(std::max(qh, 0.0), 255.0);
                set_byte(node.w, 8 + 2 * a, s, (uint32_t)ql);
                set_byte(node.w, 14 + 2 * a, s, (uint32_t)qh);
            }
            if (c.enc >= 0) {
                imask |= 1u << s;
                set_byte(node.w, 6, s, 0x80u | (uint32_t)rank);
                pending.push_back({c.enc, (int32_t)(child_base + rank)});
                level.push_back(level[qi] + 1);
                ++rank;
            } else {
                const uint32_t off = (uint32_t)out->tris.size() - tri_base;
                for (int t = 0; t < c.count; ++t) out->tris.push_back(b2.tris[(size_t)(~c.enc) + t]);
                set_byte(node.w, 6, s, 0x80u | (off << 2) | (uint32_t)(c.count - 1));
            }
        }
        set_byte(&node.w[3], 0, 3, imask);
        node.w[4] = child_base;
        node.w[5] = tri_base;
        out->nodes[wi] = node;
    }
    return 0;
}

}  // namespace rpl
