// bvh_build.cpp -- one-time host build of the terrain and link BVHs (binned SAH, multithreaded).
//
// Sec. 3.2.2 keeps every mesh static in its own frame so that no acceleration structure is refitted
// per frame; the BVHs are therefore built once on the host, with care for quality (SAH), and
// uploaded.  The top levels are split on the calling thread (with the binning of large ranges
// spread over threads); the remaining subtrees are built by a pool of threads into private node
// arrays that are concatenated in a fixed order, so the result does not depend on the thread count.
#include "bvh.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <limits>
#include <thread>

namespace rpl {
namespace {

constexpr int kBins = 16;
constexpr int kMedianDepth = 32;        // below this depth splits become object medians
constexpr double kDefaultNodeCost = 1.0;  // SAH cost of visiting one node, relative to one triangle

struct Box {
    float lo[3], hi[3];
    void reset() {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::numeric_limits<float>::infinity();
            hi[a] = -std::numeric_limits<float>::infinity();
        }
    }
    void grow(const Box &b) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], b.lo[a]);
            hi[a] = std::max(hi[a], b.hi[a]);
        }
    }
    void grow(const float *p) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], p[a]);
            hi[a] = std::max(hi[a], p[a]);
        }
    }
    bool empty() const { return !(lo[0] <= hi[0]); }
    double half_area() const {
        if (empty()) return 0.0;
        double dx = (double)hi[0] - lo[0], dy = (double)hi[1] - lo[1], dz = (double)hi[2] - lo[2];
        return dx * dy + dy * dz + dz * dx;
    }
};

struct ChildRef {
    int32_t enc;    // inner node index (>= 0) or ~first triangle (leaf)
    int32_t count;  // triangles of a leaf, 0 for an inner node
    Box box;
};

struct Prims {
    const float *box;   // [T][6] lo xyz, hi xyz
    const float *cen;   // [T][3]
};

// Outward rounding of a padded bound to float.
float pad_lo(float v) {
    double x = (double)v - std::max(std::fabs((double)v) * 0x1p-20, 1e-6);
    float f = (float)x;
    if ((double)f > x) f = std::nextafter(f, -std::numeric_limits<float>::infinity());
    return f;
}
float pad_hi(float v) {
    double x = (double)v + std::max(std::fabs((double)v) * 0x1p-20, 1e-6);
    float f = (float)x;
    if ((double)f < x) f = std::nextafter(f, std::numeric_limits<float>::infinity());
    return f;
}

void write_child(BvhNode &n, int slot, const ChildRef &c) {
    float lo[3], hi[3];
    if (c.box.empty() || (c.enc < 0 && c.count == 0)) {
        for (int a = 0; a < 3; ++a) lo[a] = hi[a] = 1e30f;  // far away: never within a ray's reach
    } else {
        for (int a = 0; a < 3; ++a) {
            lo[a] = pad_lo(c.box.lo[a]);
            hi[a] = pad_hi(c.box.hi[a]);
        }
    }
    if (slot == 0) {
        n.c0lox = lo[0]; n.c0hix = hi[0]; n.c0loy = lo[1]; n.c0hiy = hi[1]; n.c0loz = lo[2]; n.c0hiz = hi[2];
        n.child0 = c.enc; n.cnt0 = c.count;
    } else {
        n.c1lox = lo[0]; n.c1hix = hi[0]; n.c1loy = lo[1]; n.c1hiy = hi[1]; n.c1loz = lo[2]; n.c1hiz = hi[2];
        n.child1 = c.enc; n.cnt1 = c.count;
    }
}

struct BinResult {
    int axis = -1, split = -1;   // split between bin `split` and `split + 1`
    double cost = std::numeric_limits<double>::infinity();
};

struct Bins {
    int count[3][kBins];
    Box box[3][kBins];
    void reset() {
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < kBins; ++b) {
                count[a][b] = 0;
                box[a][b].reset();
            }
    }
};

inline int bin_of(float c, float lo, float scale) {
    int b = (int)(((double)c - lo) * scale);
    return std::min(std::max(b, 0), kBins - 1);
}

void fill_bins(const Prims &P, const int32_t *ref, int64_t b0, int64_t b1, const Box &cb, Bins &bins) {
    bins.reset();
    double scale[3];
    for (int a = 0; a < 3; ++a) {
        double ext = (double)cb.hi[a] - cb.lo[a];
        scale[a] = ext > 0 ? kBins / ext * (1.0 - 1e-9) : 0.0;
    }
    for (int64_t i = b0; i < b1; ++i) {
        int32_t t = ref[i];
        const float *c = P.cen + 3 * (int64_t)t;
        Box pb;
        std::memcpy(pb.lo, P.box + 6 * (int64_t)t, 3 * sizeof(float));
        std::memcpy(pb.hi, P.box + 6 * (int64_t)t + 3, 3 * sizeof(float));
        for (int a = 0; a < 3; ++a) {
            int b = bin_of(c[a], cb.lo[a], (float)scale[a]);
            bins.count[a][b]++;
            bins.box[a][b].grow(pb);
        }
    }
}

BinResult best_split(const Bins &bins, const Box &cb) {
    BinResult r;
    for (int a = 0; a < 3; ++a) {
        if (!(cb.hi[a] > cb.lo[a])) continue;
        double right_area[kBins];
        int right_count[kBins];
        Box acc;
        acc.reset();
        int cnt = 0;
        for (int b = kBins - 1; b > 0; --b) {
            acc.grow(bins.box[a][b]);
            cnt += bins.count[a][b];
            right_area[b] = acc.half_area();
            right_count[b] = cnt;
        }
        acc.reset();
        cnt = 0;
        for (int b = 0; b < kBins - 1; ++b) {
            acc.grow(bins.box[a][b]);
            cnt += bins.count[a][b];
            if (cnt == 0 || right_count[b + 1] == 0) continue;
            double cost = acc.half_area() * cnt + right_area[b + 1] * right_count[b + 1];
            if (cost < r.cost) {
                r.cost = cost;
                r.axis = a;
                r.split = b;
            }
        }
    }
    return r;
}

struct Deferred {
    int64_t begin, end;
    int depth;
    Box box, cbox;
    int32_t parent;   // node in the top array
    int slot;
};

class Builder {
public:
    Builder(const Prims &P, int32_t *ref, int max_leaf, double node_cost)
        : P_(P), ref_(ref), max_leaf_(max_leaf), node_cost_(node_cost) {}

    // Top phase when defer_below > 0: ranges at or under the threshold are recorded, not built.
    ChildRef build(int64_t b0, int64_t b1, int depth, const Box &box, const Box &cbox,
                   int64_t defer_below, std::vector<Deferred> *deferred, int32_t parent, int slot,
                   int n_threads) {
        int64_t n = b1 - b0;
        max_depth_ = std::max(max_depth_, depth);
        if (deferred && n <= defer_below && n > max_leaf_) {
            deferred->push_back({b0, b1, depth, box, cbox, parent, slot});
            ChildRef c;
            c.enc = 0;
            c.count = -1;   // patched after the parallel phase
            c.box = box;
            return c;
        }
        // split decision
        int axis = -1;
        int64_t mid = -1;
        if (depth < kMedianDepth) {
            Bins bins;
            if (n > 262144 && n_threads > 1) {
                parallel_bins(b0, b1, cbox, bins, n_threads);
            } else {
                fill_bins(P_, ref_, b0, b1, cbox, bins);
            }
            BinResult r = best_split(bins, cbox);
            double leaf_cost = box.half_area() * (double)n;
            double split_cost = r.axis >= 0 ? node_cost_ * box.half_area() + r.cost
                                             : std::numeric_limits<double>::infinity();
            if (n <= max_leaf_ && leaf_cost <= split_cost) return leaf(b0, b1, box);
            if (r.axis >= 0) {
                axis = r.axis;
                double ext = (double)cbox.hi[axis] - cbox.lo[axis];
                float scale = (float)(kBins / ext * (1.0 - 1e-9));
                float lo = cbox.lo[axis];
                int split = r.split;
                int32_t *p = std::partition(ref_ + b0, ref_ + b1, [&](int32_t t) {
                    return bin_of(P_.cen[3 * (int64_t)t + axis], lo, scale) <= split;
                });
                mid = p - ref_;
                if (mid == b0 || mid == b1) mid = -1;
            }
        } else if (n <= max_leaf_) {
            return leaf(b0, b1, box);
        }
        if (mid < 0) {
            // object median along the widest centroid axis (or by index if all centroids coincide)
            int a = 0;
            for (int k = 1; k < 3; ++k)
                if ((double)cbox.hi[k] - cbox.lo[k] > (double)cbox.hi[a] - cbox.lo[a]) a = k;
            mid = b0 + n / 2;
            if (cbox.hi[a] > cbox.lo[a]) {
                std::nth_element(ref_ + b0, ref_ + mid, ref_ + b1, [&](int32_t x, int32_t y) {
                    float cx = P_.cen[3 * (int64_t)x + a], cy = P_.cen[3 * (int64_t)y + a];
                    return cx < cy || (cx == cy && x < y);
                });
            }
        }
        Box lb, lcb, rb, rcb;
        bounds(b0, mid, lb, lcb);
        bounds(mid, b1, rb, rcb);
        int32_t idx = (int32_t)nodes.size();
        nodes.push_back(BvhNode{});
        ChildRef l = build(b0, mid, depth + 1, lb, lcb, defer_below, deferred, idx, 0, n_threads);
        write_child(nodes[idx], 0, l);
        ChildRef r = build(mid, b1, depth + 1, rb, rcb, defer_below, deferred, idx, 1, n_threads);
        write_child(nodes[idx], 1, r);
        ChildRef c;
        c.enc = idx;
        c.count = 0;
        c.box = box;
        return c;
    }

    void bounds(int64_t b0, int64_t b1, Box &box, Box &cbox) const {
        box.reset();
        cbox.reset();
        for (int64_t i = b0; i < b1; ++i) {
            int32_t t = ref_[i];
            Box pb;
            std::memcpy(pb.lo, P_.box + 6 * (int64_t)t, 3 * sizeof(float));
            std::memcpy(pb.hi, P_.box + 6 * (int64_t)t + 3, 3 * sizeof(float));
            box.grow(pb);
            cbox.grow(P_.cen + 3 * (int64_t)t);
        }
    }

    std::vector<BvhNode> nodes;
    int max_depth_ = 0;

private:
    ChildRef leaf(int64_t b0, int64_t b1, const Box &box) {
        ChildRef c;
        c.enc = ~(int32_t)b0;
        c.count = (int32_t)(b1 - b0);
        c.box = box;
        return c;
    }

    void parallel_bins(int64_t b0, int64_t b1, const Box &cbox, Bins &out, int n_threads) {
        std::vector<Bins> part(n_threads);
        std::vector<std::thread> th;
        int64_t n = b1 - b0;
        for (int k = 0; k < n_threads; ++k) {
            int64_t s = b0 + n * k / n_threads, e = b0 + n * (k + 1) / n_threads;
            th.emplace_back([&, s, e, k]() { fill_bins(P_, ref_, s, e, cbox, part[k]); });
        }
        for (auto &t : th) t.join();
        out.reset();
        for (int k = 0; k < n_threads; ++k)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < kBins; ++b) {
                    out.count[a][b] += part[k].count[a][b];
                    out.box[a][b].grow(part[k].box[a][b]);
                }
    }

    const Prims &P_;
    int32_t *ref_;
    int max_leaf_;
    double node_cost_;
};

}  // namespace

int build_bvh2(const float *verts, int64_t n_verts, const int32_t *tris, int64_t n_tris, int max_leaf,
               int n_threads, HostBvh *out, double node_cost) {
    if (!(node_cost > 0.0)) node_cost = kDefaultNodeCost;
    if (max_leaf < 1) max_leaf = 4;
    if (max_leaf > 8) max_leaf = 8;
    if (n_threads <= 0) n_threads = (int)std::max(1u, std::thread::hardware_concurrency());
    out->nodes.clear();
    out->tris.clear();
    out->depth = 0;
    for (int a = 0; a < 3; ++a) {
        out->root_lo[a] = std::numeric_limits<float>::infinity();
        out->root_hi[a] = -std::numeric_limits<float>::infinity();
    }
    for (int64_t i = 0; i < 3 * n_tris; ++i)
        if (tris[i] < 0 || tris[i] >= n_verts) return -1;

    std::vector<float> pbox, pcen;
    std::vector<int32_t> ref;
    try {
        pbox.resize((size_t)n_tris * 6);
        pcen.resize((size_t)n_tris * 3);
        ref.resize((size_t)n_tris);
        out->tris.resize((size_t)n_tris);
    } catch (...) {
        return -2;
    }
    for (int64_t t = 0; t < n_tris; ++t) {
        const float *v[3];
        for (int k = 0; k < 3; ++k) v[k] = verts + 3 * (int64_t)tris[3 * t + k];
        for (int a = 0; a < 3; ++a) {
            float lo = std::min(v[0][a], std::min(v[1][a], v[2][a]));
            float hi = std::max(v[0][a], std::max(v[1][a], v[2][a]));
            pbox[6 * t + a] = lo;
            pbox[6 * t + 3 + a] = hi;
            pcen[3 * t + a] = (float)(0.5 * ((double)lo + (double)hi));
        }
        ref[t] = (int32_t)t;
    }
    Prims P{pbox.data(), pcen.data()};

    BvhNode root{};
    if (n_tris <= max_leaf) {
        // the root stays an inner node: child 0 holds every triangle, child 1 is empty
        Builder b(P, ref.data(), max_leaf, node_cost);
        Box box, cbox;
        b.bounds(0, n_tris, box, cbox);
        ChildRef l;
        l.enc = ~0;
        l.count = (int32_t)n_tris;
        l.box = box;
        ChildRef e;
        e.enc = ~0;
        e.count = 0;
        e.box.reset();
        write_child(root, 0, l);
        write_child(root, 1, e);
        out->nodes.push_back(root);
        out->depth = 1;
        for (int a = 0; a < 3; ++a) {
            out->root_lo[a] = box.lo[a];
            out->root_hi[a] = box.hi[a];
        }
    } else {
        Builder top(P, ref.data(), max_leaf, node_cost);
        Box box, cbox;
        top.bounds(0, n_tris, box, cbox);
        for (int a = 0; a < 3; ++a) {
            out->root_lo[a] = box.lo[a];
            out->root_hi[a] = box.hi[a];
        }
        std::vector<Deferred> deferred;
        const int64_t defer_below = std::max<int64_t>(n_tris / (8 * (int64_t)n_threads), 2048);
        // the root itself is never deferred: the parallel phase only builds proper subtrees
        const bool parallel = n_threads > 1 && n_tris > defer_below;
        ChildRef r = top.build(0, n_tris, 0, box, cbox, parallel ? defer_below : 0, parallel ? &deferred : nullptr,
                               -1, 0, n_threads);
        (void)r;   // the root is node 0 of the top array
        // parallel phase
        std::vector<Builder *> sub(deferred.size(), nullptr);
        std::vector<ChildRef> sub_root(deferred.size());
        std::atomic<size_t> next{0};
        auto worker = [&]() {
            for (;;) {
                size_t i = next.fetch_add(1);
                if (i >= deferred.size()) break;
                const Deferred &d = deferred[i];
                sub[i] = new Builder(P, ref.data(), max_leaf, node_cost);
                sub_root[i] = sub[i]->build(d.begin, d.end, d.depth, d.box, d.cbox, 0, nullptr, -1, 0, 1);
            }
        };
        std::vector<std::thread> th;
        for (int k = 0; k < n_threads && !deferred.empty(); ++k) th.emplace_back(worker);
        for (auto &t : th) t.join();
        // concatenate in task order and patch the parents' child slots
        out->nodes = std::move(top.nodes);
        int depth = top.max_depth_;
        for (size_t i = 0; i < deferred.size(); ++i) {
            int32_t base = (int32_t)out->nodes.size();
            for (BvhNode nd : sub[i]->nodes) {
                if (nd.child0 >= 0) nd.child0 += base;
                if (nd.child1 >= 0) nd.child1 += base;
                out->nodes.push_back(nd);
            }
            ChildRef c = sub_root[i];
            if (c.enc >= 0) c.enc += base;
            write_child(out->nodes[deferred[i].parent], deferred[i].slot, c);
            depth = std::max(depth, sub[i]->max_depth_);
            delete sub[i];
        }
        out->depth = depth + 1;
    }
    // leaf-ordered triangles
    for (int64_t i = 0; i < n_tris; ++i) {
        int32_t t = ref[i];
        BvhTri &o = out->tris[i];
        const float *v0 = verts + 3 * (int64_t)tris[3 * (int64_t)t + 0];
        const float *v1 = verts + 3 * (int64_t)tris[3 * (int64_t)t + 1];
        const float *v2 = verts + 3 * (int64_t)tris[3 * (int64_t)t + 2];
        o.v0x = v0[0]; o.v0y = v0[1]; o.v0z = v0[2];
        o.v1x = v1[0]; o.v1y = v1[1]; o.v1z = v1[2];
        o.v2x = v2[0]; o.v2y = v2[1]; o.v2z = v2[2];
        std::memcpy(&o.id, &t, sizeof(float));
        o.pad1 = o.pad2 = 0.0f;
    }
    if (out->nodes.empty()) {
        // no triangles: a root with two empty children
        ChildRef e;
        e.enc = ~0;
        e.count = 0;
        e.box.reset();
        write_child(root, 0, e);
        write_child(root, 1, e);
        out->nodes.push_back(root);
        out->depth = 1;
    }
    return 0;
}

}  // namespace rpl
