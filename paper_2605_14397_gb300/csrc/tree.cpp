// Cluster tree over element centroids and block partition (host C++).
//
// The paper builds an H-matrix of E with dense near-field and low-rank far-field
// blocks (Sec. 3.1) and names no clustering rule.  Rules used here:
//   * a cluster of more than leaf_size elements is split along the longest axis of the
//     bounding box of its centroids, at the median: elements ordered by (coordinate,
//     user index), the first n/2 go to the left child;
//   * nodes are numbered in depth-first pre-order;
//   * cluster boxes bound the element vertices: c +- a s1 +- b s2 of a rectangle, the
//     three given vertices of a triangle;
//   * (s, t) is admissible iff dist(B_s, B_t) > 0 and min(diam B_s, diam B_t) <=
//     eta dist(B_s, B_t) (Euclidean diagonal and gap);
//   * the block tree starts at (root, root); an admissible pair is a far block, a pair
//     of leaves a near block, otherwise the non-leaf members are split and the children
//     visited in the order (s0,t0), (s0,t1), (s1,t0), (s1,t1).
// This file is compiled with floating-point contraction disabled so that the box and
// admissibility arithmetic is the plain IEEE sequence written here.
#include "tree.h"

#include <string>

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
            if (el.shape && el.shape[i] == HM_SHAPE_TRI) {
                for (int v = 0; v < 3; ++v)
                    for (int k = 0; k < 3; ++k) {
                        const double x = el.tri[9 * i + 3 * v + k];
                        vlo[i][k] = std::min(vlo[i][k], x);
                        vhi[i][k] = std::max(vhi[i][k], x);
                    }
                continue;
            }
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

void validate_elements(const hm_elements& el, const char* who) {
    const std::string w(who);
    if (el.N <= 0) fail(HM_EINVAL, w + ": N must be positive");
    if (!el.c || !el.s1 || !el.s2 || !el.n || !el.a || !el.b) fail(HM_EINVAL, w + ": NULL geometry");
    bool any_tri = false;
    for (int64_t i = 0; i < el.N; ++i) {
        const int sh = el.shape ? el.shape[i] : HM_SHAPE_RECT;
        if (sh != HM_SHAPE_RECT && sh != HM_SHAPE_TRI) fail(HM_EINVAL, w + ": unknown element shape");
        any_tri = any_tri || sh == HM_SHAPE_TRI;
        if (sh == HM_SHAPE_RECT && (!(el.a[i] > 0.0) || !(el.b[i] > 0.0)))
            fail(HM_EINVAL, w + ": half sides must be positive");
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(el.c[3 * i + k]) || !std::isfinite(el.n[3 * i + k]) ||
                !std::isfinite(el.s1[3 * i + k]) || !std::isfinite(el.s2[3 * i + k]))
                fail(HM_ENAN, w + ": non-finite geometry");
    }
    if (any_tri && !el.tri) fail(HM_EINVAL, w + ": triangles need their vertices (tri)");
    for (int64_t i = 0; any_tri && i < el.N; ++i) {
        if (el.shape[i] != HM_SHAPE_TRI) continue;
        const double* v = el.tri + 9 * i;
        for (int k = 0; k < 9; ++k)
            if (!std::isfinite(v[k])) fail(HM_ENAN, w + ": non-finite triangle vertex");
        const ElemRec r = make_elem_record(el, i);
        const double size = std::sqrt(r.area);
        if (!(r.area > 0.0)) fail(HM_EINVAL, w + ": degenerate triangle");
        for (int q = 0; q < 3; ++q) {
            double off = 0.0;
            for (int k = 0; k < 3; ++k) off += (v[3 * q + k] - el.c[3 * i + k]) * el.n[3 * i + k];
            if (std::fabs(off) > 1e-6 * size) fail(HM_EINVAL, w + ": a triangle vertex is off the plane of c and n");
        }
        // c inside: the three edge cross products have the orientation's sign
        const double o = (r.tv[2] - r.tv[0]) * (r.tv[5] - r.tv[1]) - (r.tv[3] - r.tv[1]) * (r.tv[4] - r.tv[0]);
        for (int e = 0; e < 3; ++e) {
            const double* P = r.tv + 2 * e;
            const double* Q = r.tv + 2 * ((e + 1) % 3);
            const double cr = (Q[0] - P[0]) * (0.0 - P[1]) - (Q[1] - P[1]) * (0.0 - P[0]);
            if (!(cr * o > 0.0)) fail(HM_EINVAL, w + ": the collocation point c lies outside its triangle");
        }
    }
}

ElemRec make_elem_record(const hm_elements& el, int64_t i) {
    ElemRec r;
    for (int d = 0; d < 3; ++d) {
        r.c[d] = el.c[3 * i + d];
        r.s1[d] = el.s1[3 * i + d];
        r.s2[d] = el.s2[3 * i + d];
        r.n[d] = el.n[3 * i + d];
    }
    for (double& t : r.tv) t = 0.0;
    if (el.shape && el.shape[i] == HM_SHAPE_TRI) {
        const double* v = el.tri + 9 * i;
        for (int q = 0; q < 3; ++q) {
            double x = 0.0, y = 0.0;
            for (int d = 0; d < 3; ++d) {
                const double dv = v[3 * q + d] - r.c[d];
                x += dv * r.s1[d];
                y += dv * r.s2[d];
            }
            r.tv[2 * q] = x;
            r.tv[2 * q + 1] = y;
        }
        r.area = 0.5 * std::fabs((r.tv[2] - r.tv[0]) * (r.tv[5] - r.tv[1]) - (r.tv[3] - r.tv[1]) * (r.tv[4] - r.tv[0]));
        r.a = r.b = 0.5 * std::sqrt(r.area);
        r.shape = HM_SHAPE_TRI;
    } else {
        r.a = el.a[i];
        r.b = el.b[i];
        r.area = 4.0 * r.a * r.b;
        r.shape = HM_SHAPE_RECT;
    }
    return r;
}

void build_tree(const hm_elements& el, int leaf_size, double eta, Tree& T) {
    if (el.N <= 0) fail(HM_EINVAL, "build_cluster_tree: N must be positive");
    if (leaf_size < 1) fail(HM_EINVAL, "build_cluster_tree: leaf_size must be >= 1");
    if (!(eta > 0.0)) fail(HM_EINVAL, "build_cluster_tree: eta must be positive");
    validate_elements(el, "build_cluster_tree");
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
        T.elems[k] = make_elem_record(el, i);
    }
}

}  // namespace hm
