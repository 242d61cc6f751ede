// rich_bvh.cpp -- host builder of the triangle BVH used by the trace kernel.
//
// Binned surface-area-heuristic build of a binary tree (12 bins per axis over
// the triangle centroids, traversal cost 1, intersection cost 1 per
// triangle, at most 8 triangles per leaf), collapsed into four-wide nodes
// (each node takes its binary children and opens the largest inner ones
// until it holds four) of 128 bytes carrying the children's boxes, in
// breadth-first order so the top levels of the tree are contiguous.
// Triangles are re-ordered into leaf order.
//
// Triangles that share a surface id (one mirror segment, flat mirror or
// window face) get a subtree of their own: each surface is built
// separately, the triangles without a surface together, and a top level
// joins the subtrees by the same heuristic over their boxes. A photon
// leaving a surface then skips that surface's subtree at its root.
#include "rich_bvh.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <limits>
#include <numeric>

namespace rich {

namespace {

constexpr int kBins = 12;
constexpr int kMaxLeaf = 8;
constexpr float kTraversalCost = 1.0f;

struct Box {
    float lo[3], hi[3];
    Box() {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::numeric_limits<float>::infinity();
            hi[k] = -std::numeric_limits<float>::infinity();
        }
    }
    void grow(const Box &b) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], b.lo[k]);
            hi[k] = std::max(hi[k], b.hi[k]);
        }
    }
    void grow(const float *p) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], p[k]);
            hi[k] = std::max(hi[k], p[k]);
        }
    }
    float area() const {
        if (!(hi[0] >= lo[0])) return 0.0f;
        float dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        return 2.0f * (dx * dy + dy * dz + dz * dx);
    }
};

struct Node {
    Box box;
    int left = -1, right = -1;  // children (build indices) for inner nodes
    int first = 0, count = 0;   // leaf range in `order` when count > 0
};

struct Builder {
    const std::vector<Box> &tri_box;
    const std::vector<float> &cen;   // 3 per triangle
    std::vector<int> order;
    std::vector<Node> nodes;

    Builder(const std::vector<Box> &tb, const std::vector<float> &c) : tri_box(tb), cen(c) {}

    int build(int first, int count) {
        Node nd;
        Box cb;
        for (int i = first; i < first + count; ++i) {
            nd.box.grow(tri_box[order[i]]);
            cb.grow(&cen[3 * order[i]]);
        }
        const int id = (int)nodes.size();
        nodes.push_back(nd);
        if (count <= 2) return make_leaf(id, first, count);
        // binned SAH over all three axes
        float best_cost = std::numeric_limits<float>::infinity();
        int best_axis = -1, best_split = -1;
        for (int axis = 0; axis < 3; ++axis) {
            const float ext = cb.hi[axis] - cb.lo[axis];
            if (!(ext > 0.0f)) continue;
            Box bb[kBins];
            int bc[kBins] = {0};
            const float scale = kBins / ext;
            for (int i = first; i < first + count; ++i) {
                int b = (int)((cen[3 * order[i] + axis] - cb.lo[axis]) * scale);
                b = std::min(std::max(b, 0), kBins - 1);
                bc[b]++;
                bb[b].grow(tri_box[order[i]]);
            }
            float right_area[kBins];
            int right_count[kBins];
            Box acc;
            int n = 0;
            for (int b = kBins - 1; b > 0; --b) {
                acc.grow(bb[b]);
                n += bc[b];
                right_area[b] = acc.area();
                right_count[b] = n;
            }
            Box left;
            int nl = 0;
            for (int b = 0; b < kBins - 1; ++b) {
                left.grow(bb[b]);
                nl += bc[b];
                const int nr = right_count[b + 1];
                if (nl == 0 || nr == 0) continue;
                const float cost = left.area() * nl + right_area[b + 1] * nr;
                if (cost < best_cost) {
                    best_cost = cost;
                    best_axis = axis;
                    best_split = b;
                }
            }
        }
        const float parent_area = std::max(nodes[id].box.area(), 1e-30f);
        const float split_cost = kTraversalCost + best_cost / parent_area;
        int mid;
        if (best_axis < 0) {
            if (count <= kMaxLeaf) return make_leaf(id, first, count);
            mid = first + count / 2;   // coincident centroids: split by count
        } else {
            if (split_cost >= (float)count && count <= kMaxLeaf)
                return make_leaf(id, first, count);
            const float ext = cb.hi[best_axis] - cb.lo[best_axis];
            const float scale = kBins / ext;
            auto it = std::partition(
                order.begin() + first, order.begin() + first + count, [&](int t) {
                    int b = (int)((cen[3 * t + best_axis] - cb.lo[best_axis]) * scale);
                    b = std::min(std::max(b, 0), kBins - 1);
                    return b <= best_split;
                });
            mid = (int)(it - order.begin());
            if (mid == first || mid == first + count) mid = first + count / 2;
        }
        const int l = build(first, mid - first);
        const int r = build(mid, first + count - mid);
        nodes[id].left = l;
        nodes[id].right = r;
        return id;
    }

    int make_leaf(int id, int first, int count) {
        nodes[id].first = first;
        nodes[id].count = count;
        return id;
    }
};

// Centre and half extent of [lo, hi] in FP32, rounded outward: the
// differences are exact in double, and the half extent is rounded up and
// then widened by one more ulp, so [c - e, c + e] holds [lo, hi].
void centre_extent(float lo, float hi, float &c, float &e) {
    c = (float)(0.5 * ((double)lo + (double)hi));
    const double need = std::max((double)c - (double)lo, (double)hi - (double)c);
    float f = (float)need;
    if ((double)f < need) f = std::nextafter(f, std::numeric_limits<float>::infinity());
    e = std::nextafter(f, std::numeric_limits<float>::infinity());
}

void put_box(DevNode &d, int slot, const Box &b) {
    centre_extent(b.lo[0], b.hi[0], d.cx[slot], d.ex[slot]);
    centre_extent(b.lo[1], b.hi[1], d.cy[slot], d.ey[slot]);
    centre_extent(b.lo[2], b.hi[2], d.cz[slot], d.ez[slot]);
}

// An empty slot: a point box at 1e30 on every axis, which every ray's slab
// test misses (its entry distance is beyond any tmax or its exit before 0).
void clear_node(DevNode &d) {
    std::memset(&d, 0, sizeof d);
    for (int k = 0; k < 4; ++k) {
        d.cx[k] = d.cy[k] = d.cz[k] = 1e30f;
        d.ex[k] = d.ey[k] = d.ez[k] = 0.0f;
        d.child[k] = std::numeric_limits<int32_t>::min();
    }
}

// Top level over subtree roots `items` (indices into `all`), each weighted
// by its triangle count: at every level the split (along the axis and at
// the position over the sorted centroids) that minimises
// area(left) * n(left) + area(right) * n(right).
int build_top(std::vector<Node> &all, std::vector<int> &items, const std::vector<int> &weight,
              int first, int count) {
    if (count == 1) return items[first];
    float best = std::numeric_limits<float>::infinity();
    int best_axis = 0, best_k = count / 2;
    for (int axis = 0; axis < 3; ++axis) {
        std::sort(items.begin() + first, items.begin() + first + count, [&](int a, int b) {
            return all[a].box.lo[axis] + all[a].box.hi[axis] <
                   all[b].box.lo[axis] + all[b].box.hi[axis];
        });
        std::vector<float> left_cost(count);
        Box acc;
        int n = 0;
        for (int k = 0; k < count - 1; ++k) {
            acc.grow(all[items[first + k]].box);
            n += weight[items[first + k]];
            left_cost[k] = acc.area() * n;
        }
        Box racc;
        int nr = 0;
        for (int k = count - 1; k >= 1; --k) {
            racc.grow(all[items[first + k]].box);
            nr += weight[items[first + k]];
            const float c = left_cost[k - 1] + racc.area() * nr;
            if (c < best) {
                best = c;
                best_axis = axis;
                best_k = k;
            }
        }
    }
    std::sort(items.begin() + first, items.begin() + first + count, [&](int a, int b) {
        return all[a].box.lo[best_axis] + all[a].box.hi[best_axis] <
               all[b].box.lo[best_axis] + all[b].box.hi[best_axis];
    });
    Node nd;
    for (int k = first; k < first + count; ++k) nd.box.grow(all[items[k]].box);
    const int id = (int)all.size();
    all.push_back(nd);
    const int l = build_top(all, items, weight, first, best_k);
    const int r = build_top(all, items, weight, first + best_k, count - best_k);
    all[id].left = l;
    all[id].right = r;
    return id;
}

}  // namespace

bool build_bvh(const float *vertices, const int32_t *surface, int64_t n_tris, BvhResult &out,
               std::string &err) {
    out = BvhResult();
    if (n_tris <= 0) return true;
    if (n_tris >= (int64_t(1) << 27)) {
        err = "too many triangles for the BVH leaf encoding";
        return false;
    }
    std::vector<Box> tri_box((size_t)n_tris);
    std::vector<float> cen(3 * (size_t)n_tris);
    for (int64_t i = 0; i < n_tris; ++i) {
        const float *t = vertices + 9 * i;
        Box bx;
        bx.grow(t);
        bx.grow(t + 3);
        bx.grow(t + 6);
        for (int k = 0; k < 3; ++k) {
            if (!std::isfinite(t[k]) || !std::isfinite(t[3 + k]) || !std::isfinite(t[6 + k])) {
                err = "non-finite triangle vertex";
                return false;
            }
            cen[3 * i + k] = (t[k] + t[3 + k] + t[6 + k]) * (1.0f / 3.0f);
        }
        tri_box[i] = bx;
    }
    // ---- groups: one per surface id, one for the triangles without one
    std::map<int32_t, std::vector<int>> groups;
    for (int64_t i = 0; i < n_tris; ++i) {
        const int32_t sid = surface ? surface[i] : -1;
        if (sid < -1) {
            err = "triangle surface id below -1";
            return false;
        }
        groups[sid].push_back((int)i);
    }
    // ---- build each group, then join the subtrees
    std::vector<Node> all;
    std::vector<int> order_all;
    std::vector<int> items, weight;
    std::vector<std::pair<int32_t, int>> group_root;   // (surface id, root in all)
    all.reserve(2 * (size_t)n_tris + 2 * groups.size());
    for (auto &[sid, tris] : groups) {
        Builder b(tri_box, cen);
        b.order = tris;
        b.nodes.reserve(2 * tris.size());
        const int root = b.build(0, (int)tris.size());
        const int off = (int)all.size(), base = (int)order_all.size();
        for (Node n : b.nodes) {
            if (n.count > 0) {
                n.first += base;
            } else {
                n.left += off;
                n.right += off;
            }
            all.push_back(n);
        }
        order_all.insert(order_all.end(), b.order.begin(), b.order.end());
        items.push_back(root + off);
        group_root.push_back({sid, root + off});
    }
    weight.assign(all.size() + groups.size() + 1, 0);
    for (size_t g = 0; g < items.size(); ++g) {
        const int32_t sid = group_root[g].first;
        weight[items[g]] = (int)groups[sid].size();
    }
    std::vector<int> top_items = items;
    const int root = build_top(all, top_items, weight, 0, (int)top_items.size());

    out.leaf_order = order_all;
    auto leaf_code = [&](const Node &n) { return ~((n.first << 3) | (n.count - 1)); };
    // surface roots are never opened into their parent, so each surface
    // keeps one subtree (one node or one leaf) of its own
    std::vector<char> is_surface_root(all.size(), 0);
    for (auto &[sid, gr] : group_root)
        if (sid >= 0) is_surface_root[gr] = 1;
    // the up-to-four children of the four-wide node made from binary node n
    auto collapse = [&](int n) {
        std::vector<int> c = {all[n].left, all[n].right};
        while (c.size() < 4) {
            int best = -1;
            float best_area = -1.0f;
            for (size_t k = 0; k < c.size(); ++k) {
                const Node &x = all[c[k]];
                if (x.count > 0 || is_surface_root[c[k]]) continue;
                const float a = x.box.area();
                if (a > best_area) {
                    best_area = a;
                    best = (int)k;
                }
            }
            if (best < 0) break;
            const int x = c[best];
            c[best] = all[x].left;
            c.push_back(all[x].right);
        }
        return c;
    };
    std::vector<int> dev_index(all.size(), -1);
    if (all[root].count > 0) {
        // the whole tree is one leaf
        DevNode d;
        clear_node(d);
        put_box(d, 0, all[root].box);
        d.child[0] = leaf_code(all[root]);
        out.nodes.push_back(d);
        out.depth = 1;
    } else {
        // breadth-first flattening of the four-wide nodes
        std::deque<std::pair<int, int>> q;   // (binary node, depth)
        q.push_back({root, 1});
        std::vector<int> bfs;
        std::vector<std::vector<int>> kids;
        while (!q.empty()) {
            auto [n, depth] = q.front();
            q.pop_front();
            dev_index[n] = (int)bfs.size();
            bfs.push_back(n);
            out.depth = std::max(out.depth, depth);
            kids.push_back(collapse(n));
            for (int c : kids.back())
                if (all[c].count == 0) q.push_back({c, depth + 1});
        }
        out.nodes.resize(bfs.size());
        for (size_t i = 0; i < bfs.size(); ++i) {
            DevNode &d = out.nodes[i];
            clear_node(d);
            for (size_t k = 0; k < kids[i].size(); ++k) {
                const int c = kids[i][k];
                put_box(d, (int)k, all[c].box);
                d.child[k] = all[c].count > 0 ? leaf_code(all[c]) : dev_index[c];
            }
        }
    }
    // ---- the subtree reference of every triangle's surface
    out.surface_ref.assign((size_t)n_tris, kNoSurface);
    std::vector<int> pos_of((size_t)n_tris);
    for (size_t k = 0; k < order_all.size(); ++k) pos_of[order_all[k]] = (int)k;
    for (auto &[sid, gr] : group_root) {
        if (sid < 0) continue;
        const int ref = all[gr].count > 0 ? leaf_code(all[gr]) : dev_index[gr];
        for (int t : groups[sid]) out.surface_ref[pos_of[t]] = ref;
    }
    return true;
}

}  // namespace rich
