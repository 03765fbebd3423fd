// Host BVH builder: binned surface-area heuristic (16 bins on each axis),
// leaves of up to 8 triangles, depth capped so the device traversal stack
// cannot overflow.  Output in depth-first order in the 64-byte two-child node
// layout described in rp_internal.h.
#include "bvh_build.h"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>

#include "rp_internal.h"

namespace rp {

namespace {

struct Box {
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX};
    float hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
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
    bool empty() const { return lo[0] > hi[0]; }
    float area() const {
        if (empty()) return 0.f;
        float dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        return 2.f * (dx * dy + dy * dz + dz * dx);
    }
};

struct Prim {
    Box box;
    float c[3];
    int id;
};

struct TmpNode {
    Box box;
    int left = -1, right = -1;     // children (TmpNode indices), -1 for a leaf
    int first = 0, count = 0;      // leaf range in the ordered primitive list
};

struct Builder {
    std::vector<Prim> prims;
    std::vector<TmpNode> nodes;
    static constexpr int kBins = 16;
    static constexpr int kMaxLeaf = 8;

    int make_leaf(int first, int count, const Box &b) {
        TmpNode n;
        n.box = b;
        n.first = first;
        n.count = count;
        nodes.push_back(n);
        return (int)nodes.size() - 1;
    }

    int build(int first, int count, int depth) {
        Box b, cb;
        for (int i = first; i < first + count; ++i) {
            b.grow(prims[i].box);
            cb.grow(prims[i].c);
        }
        if (count <= 2 || depth >= kBvhMaxDepth) return make_leaf(first, count, b);
        // binned SAH over the three axes
        float best_cost = FLT_MAX;
        int best_axis = -1, best_split = -1;
        for (int a = 0; a < 3; ++a) {
            float ext = cb.hi[a] - cb.lo[a];
            if (!(ext > 0.f)) continue;
            Box bb[kBins];
            int bc[kBins] = {0};
            float k = kBins / ext;
            for (int i = first; i < first + count; ++i) {
                int bi = std::min(kBins - 1, (int)((prims[i].c[a] - cb.lo[a]) * k));
                bb[bi].grow(prims[i].box);
                ++bc[bi];
            }
            float la[kBins], ra[kBins];
            int lc[kBins], rc[kBins];
            Box acc;
            int n = 0;
            for (int i = 0; i < kBins; ++i) {
                acc.grow(bb[i]);
                n += bc[i];
                la[i] = acc.area();
                lc[i] = n;
            }
            acc = Box();
            n = 0;
            for (int i = kBins - 1; i >= 0; --i) {
                acc.grow(bb[i]);
                n += bc[i];
                ra[i] = acc.area();
                rc[i] = n;
            }
            for (int s = 0; s < kBins - 1; ++s) {
                if (lc[s] == 0 || rc[s + 1] == 0) continue;
                float cost = la[s] * lc[s] + ra[s + 1] * rc[s + 1];
                if (cost < best_cost) {
                    best_cost = cost;
                    best_axis = a;
                    best_split = s;
                }
            }
        }
        const float parent = b.area();
        const float leaf_cost = (float)count;
        const float split_cost = parent > 0.f ? 1.0f + best_cost / parent : FLT_MAX;
        int mid;
        if (best_axis < 0) {
            // all centroids coincide: split in half if too many for a leaf
            if (count <= kMaxLeaf) return make_leaf(first, count, b);
            mid = first + count / 2;
        } else {
            if (split_cost >= leaf_cost && count <= kMaxLeaf) return make_leaf(first, count, b);
            const int a = best_axis;
            const float ext = cb.hi[a] - cb.lo[a];
            const float k = kBins / ext;
            auto it = std::partition(prims.begin() + first, prims.begin() + first + count,
                                     [&](const Prim &p) {
                                         int bi = std::min(kBins - 1, (int)((p.c[a] - cb.lo[a]) * k));
                                         return bi <= best_split;
                                     });
            mid = (int)(it - prims.begin());
            if (mid == first || mid == first + count) mid = first + count / 2;
        }
        int self = (int)nodes.size();
        nodes.push_back(TmpNode());
        nodes[self].box = b;
        int l = build(first, mid - first, depth + 1);
        int r = build(mid, first + count - mid, depth + 1);
        nodes[self].left = l;
        nodes[self].right = r;
        return self;
    }
};

inline float4 f4(float x, float y, float z, float w) {
    float4 v;
    v.x = x; v.y = y; v.z = z; v.w = w;
    return v;
}

inline float ibits(int i) {
    float f;
    std::memcpy(&f, &i, 4);
    return f;
}

}  // namespace

BuiltBVH build_bvh(const float *verts, const uint32_t *tris, int n, int id_offset) {
    BuiltBVH out;
    if (n <= 0) return out;
    Builder B;
    B.prims.resize(n);
    for (int i = 0; i < n; ++i) {
        Prim &p = B.prims[i];
        for (int k = 0; k < 3; ++k) p.box.grow(verts + 3 * tris[3 * i + k]);
        for (int a = 0; a < 3; ++a) p.c[a] = 0.5f * (p.box.lo[a] + p.box.hi[a]);
        p.id = i;
    }
    B.nodes.reserve(2 * n);
    int root = B.build(0, n, 1);
    // ordered triangles
    out.tris.resize(3 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        const int id = B.prims[i].id;
        for (int k = 0; k < 3; ++k) {
            const float *v = verts + 3 * tris[3 * id + k];
            out.tris[3 * (size_t)i + k] = f4(v[0], v[1], v[2], k == 0 ? ibits(id + id_offset) : 0.f);
        }
    }
    // flatten inner nodes depth-first; a leaf root gets a dummy parent
    std::vector<int> map(B.nodes.size(), -1);
    std::vector<int> order;
    if (B.nodes[root].left < 0) {
        TmpNode dummy;
        dummy.box = B.nodes[root].box;
        dummy.left = root;
        dummy.right = -2;   // empty
        B.nodes.push_back(dummy);
        root = (int)B.nodes.size() - 1;
        map.push_back(-1);
    }
    std::vector<int> stack{root};
    while (!stack.empty()) {
        int i = stack.back();
        stack.pop_back();
        map[i] = (int)order.size();
        order.push_back(i);
        const TmpNode &t = B.nodes[i];
        if (t.right >= 0 && B.nodes[t.right].left >= 0) stack.push_back(t.right);
        if (t.left >= 0 && B.nodes[t.left].left >= 0) stack.push_back(t.left);
    }
    out.nodes.resize(4 * order.size());
    out.depth = 0;
    for (size_t o = 0; o < order.size(); ++o) {
        const TmpNode &t = B.nodes[order[o]];
        Box cbox[2];
        int child[2], cnt[2];
        for (int s = 0; s < 2; ++s) {
            int ci = s ? t.right : t.left;
            if (ci == -2) {                 // empty child: an inverted box, never hit
                child[s] = ~0;
                cnt[s] = 0;
                continue;
            }
            const TmpNode &c = B.nodes[ci];
            cbox[s] = c.box;
            if (c.left >= 0) {
                child[s] = map[ci];
                cnt[s] = 0;
            } else {
                child[s] = ~c.first;
                cnt[s] = c.count;
            }
        }
        out.nodes[4 * o + 0] = f4(cbox[0].lo[0], cbox[0].hi[0], cbox[0].lo[1], cbox[0].hi[1]);
        out.nodes[4 * o + 1] = f4(cbox[1].lo[0], cbox[1].hi[0], cbox[1].lo[1], cbox[1].hi[1]);
        out.nodes[4 * o + 2] = f4(cbox[0].lo[2], cbox[0].hi[2], cbox[1].lo[2], cbox[1].hi[2]);
        out.nodes[4 * o + 3] = f4(ibits(child[0]), ibits(child[1]), ibits(cnt[0]), ibits(cnt[1]));
    }
    // depth of the flattened tree (inner levels), for the stack bound
    std::vector<std::pair<int, int>> st{{0, 1}};
    while (!st.empty()) {
        auto [i, d] = st.back();
        st.pop_back();
        out.depth = std::max(out.depth, d);
        for (int s = 0; s < 2; ++s) {
            float cf = s ? out.nodes[4 * i + 3].y : out.nodes[4 * i + 3].x;
            int c;
            std::memcpy(&c, &cf, 4);
            if (c >= 0) st.push_back({c, d + 1});
        }
    }
    return out;
}

}  // namespace rp
