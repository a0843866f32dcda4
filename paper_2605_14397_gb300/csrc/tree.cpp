// Cluster tree over element centroids and block partition (host C++).
//
// The paper builds an H-matrix of E with dense near-field and low-rank far-field
// blocks (Sec. 3.1) and names no clustering rule.  Rules used here:
//   * a cluster of more than leaf_size elements is split along the longest axis of the
//     bounding box of its centroids, at the median: elements ordered by (coordinate,
//     user index), the first n/2 go to the left child;
//   * nodes are numbered in depth-first pre-order;
//   * cluster boxes bound the element vertices c +- a s1 +- b s2;
//   * (s, t) is admissible iff dist(B_s, B_t) > 0 and min(diam B_s, diam B_t) <=
//     eta dist(B_s, B_t) (Euclidean diagonal and gap);
//   * the block tree starts at (root, root); an admissible pair is a far block, a pair
//     of leaves a near block, otherwise the non-leaf members are split and the children
//     visited in the order (s0,t0), (s0,t1), (s1,t0), (s1,t1).
// This file is compiled with floating-point contraction disabled so that the box and
// admissibility arithmetic is the plain IEEE sequence written here.
#include "tree.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace hm {

namespace {

struct Builder {
    const hm_elements& el;
    Tree& T;
    std::vector<std::array<double, 3>> vlo, vhi;  // per-element vertex boxes

    Builder(const hm_elements& e, Tree& t) : el(e), T(t) {}

    void element_boxes() {
        const int64_t N = el.N;
        vlo.assign(N, {INFINITY, INFINITY, INFINITY});
        vhi.assign(N, {-INFINITY, -INFINITY, -INFINITY});
        for (int64_t i = 0; i < N; ++i) {
            for (int ia = 0; ia < 2; ++ia) {
                for (int ib = 0; ib < 2; ++ib) {
                    const double sa = ia ? 1.0 : -1.0, sb = ib ? 1.0 : -1.0;
                    const double fa = sa * el.a[i], fb = sb * el.b[i];
                    for (int k = 0; k < 3; ++k) {
                        double v = el.c[3 * i + k] + fa * el.s1[3 * i + k] + fb * el.s2[3 * i + k];
                        vlo[i][k] = std::min(vlo[i][k], v);
                        vhi[i][k] = std::max(vhi[i][k], v);
                    }
                }
            }
        }
    }

    int64_t make(int64_t b, int64_t e, int64_t lev) {
        const int64_t q = (int64_t)T.begin.size();
        T.begin.push_back(b);
        T.end.push_back(e);
        T.left.push_back(-1);
        T.right.push_back(-1);
        T.level.push_back(lev);
        std::array<double, 3> lo = {INFINITY, INFINITY, INFINITY}, hi = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t k = b; k < e; ++k) {
            const int64_t i = T.perm[k];
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], vlo[i][d]);
                hi[d] = std::max(hi[d], vhi[i][d]);
            }
        }
        T.lo.push_back(lo);
        T.hi.push_back(hi);
        T.depth = std::max<int>(T.depth, (int)lev);
        const int64_t n = e - b;
        if (n > T.leaf_size && n > 1) {
            double cmin[3] = {INFINITY, INFINITY, INFINITY}, cmax[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (int64_t k = b; k < e; ++k) {
                const int64_t i = T.perm[k];
                for (int d = 0; d < 3; ++d) {
                    cmin[d] = std::min(cmin[d], el.c[3 * i + d]);
                    cmax[d] = std::max(cmax[d], el.c[3 * i + d]);
                }
            }
            int axis = 0;
            double best = cmax[0] - cmin[0];
            for (int d = 1; d < 3; ++d) {
                const double ext = cmax[d] - cmin[d];
                if (ext > best) { best = ext; axis = d; }
            }
            const double* c = el.c;
            std::sort(T.perm.begin() + b, T.perm.begin() + e, [c, axis](int64_t x, int64_t y) {
                const double cx = c[3 * x + axis], cy = c[3 * y + axis];
                if (cx < cy) return true;
                if (cy < cx) return false;
                return x < y;
            });
            const int64_t m = b + n / 2;
            const int64_t l = make(b, m, lev + 1);
            T.left[q] = l;
            const int64_t r = make(m, e, lev + 1);
            T.right[q] = r;
        }
        return q;
    }
};

double box_diam(const std::array<double, 3>& lo, const std::array<double, 3>& hi) {
    const double d0 = hi[0] - lo[0], d1 = hi[1] - lo[1], d2 = hi[2] - lo[2];
    return std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
}

double box_dist(const std::array<double, 3>& lo1, const std::array<double, 3>& hi1,
                const std::array<double, 3>& lo2, const std::array<double, 3>& hi2) {
    double g[3];
    for (int k = 0; k < 3; ++k) g[k] = std::max(0.0, std::max(lo2[k] - hi1[k], lo1[k] - hi2[k]));
    return std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
}

}  // namespace

void build_tree(const hm_elements& el, int leaf_size, double eta, Tree& T) {
    if (el.N <= 0) fail(HM_EINVAL, "build_cluster_tree: N must be positive");
    if (leaf_size < 1) fail(HM_EINVAL, "build_cluster_tree: leaf_size must be >= 1");
    if (!(eta > 0.0)) fail(HM_EINVAL, "build_cluster_tree: eta must be positive");
    if (!el.c || !el.s1 || !el.s2 || !el.n || !el.a || !el.b) fail(HM_EINVAL, "build_cluster_tree: NULL geometry");
    for (int64_t i = 0; i < el.N; ++i) {
        if (!(el.a[i] > 0.0) || !(el.b[i] > 0.0)) fail(HM_EINVAL, "build_cluster_tree: half sides must be positive");
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(el.c[3 * i + k]) || !std::isfinite(el.n[3 * i + k]) ||
                !std::isfinite(el.s1[3 * i + k]) || !std::isfinite(el.s2[3 * i + k]))
                fail(HM_ENAN, "build_cluster_tree: non-finite geometry");
    }
    T = Tree();
    T.N = el.N;
    T.leaf_size = leaf_size;
    T.eta = eta;
    T.perm.resize(el.N);
    std::iota(T.perm.begin(), T.perm.end(), 0);
    Builder B(el, T);
    B.element_boxes();
    B.make(0, el.N, 0);

    const int64_t nn = (int64_t)T.begin.size();
    T.leaf_of_node.assign(nn, -1);
    for (int64_t q = 0; q < nn; ++q)
        if (T.left[q] < 0) {
            T.leaf_of_node[q] = (int64_t)T.leaves.size();
            T.leaves.push_back(q);
        }

    // block partition, depth-first with an explicit stack
    std::vector<std::array<int64_t, 2>> stack;
    stack.push_back({0, 0});
    while (!stack.empty()) {
        const auto st = stack.back();
        stack.pop_back();
        const int64_t s = st[0], t = st[1];
        const double ds = box_diam(T.lo[s], T.hi[s]);
        const double dt = box_diam(T.lo[t], T.hi[t]);
        const double dist = box_dist(T.lo[s], T.hi[s], T.lo[t], T.hi[t]);
        if (dist > 0.0 && std::min(ds, dt) <= eta * dist) {
            T.far.push_back({s, t});
            continue;
        }
        const bool ls = T.left[s] < 0, lt = T.left[t] < 0;
        if (ls && lt) {
            T.near.push_back({s, t});
            continue;
        }
        int64_t cs[2], ct[2];
        int ns = 0, nt = 0;
        if (ls) cs[ns++] = s; else { cs[ns++] = T.left[s]; cs[ns++] = T.right[s]; }
        if (lt) ct[nt++] = t; else { ct[nt++] = T.left[t]; ct[nt++] = T.right[t]; }
        // push in reverse so that they are visited in (s0,t0), (s0,t1), (s1,t0), (s1,t1) order
        for (int a = ns - 1; a >= 0; --a)
            for (int b = nt - 1; b >= 0; --b) stack.push_back({cs[a], ct[b]});
    }

    // element records in cluster order
    T.elems.resize(el.N);
    for (int64_t k = 0; k < el.N; ++k) {
        const int64_t i = T.perm[k];
        ElemRec r;
        for (int d = 0; d < 3; ++d) {
            r.c[d] = el.c[3 * i + d];
            r.s1[d] = el.s1[3 * i + d];
            r.s2[d] = el.s2[3 * i + d];
            r.n[d] = el.n[3 * i + d];
        }
        r.a = el.a[i];
        r.b = el.b[i];
        r.pad[0] = r.pad[1] = 0.0;
        T.elems[k] = r;
    }
}

}  // namespace hm
