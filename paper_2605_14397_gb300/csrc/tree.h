// Host-side cluster tree and block partition of the H-matrix.
#pragma once

#include <array>
#include <cstdint>
#include <vector>

#include "common.h"

namespace hm {

struct Tree {
    int64_t N = 0;
    int leaf_size = 64;
    double eta = 2.0;
    int depth = 0;
    std::vector<int64_t> perm;  // cluster position -> user element index
    std::vector<int64_t> begin, end, left, right, level;
    std::vector<std::array<double, 3>> lo, hi;  // element-vertex boxes
    std::vector<int64_t> leaves;                // leaf node ids in position order
    std::vector<int64_t> leaf_of_node;          // node -> leaf ordinal (-1 if inner)
    std::vector<std::array<int64_t, 2>> near, far;
    // element geometry copied in cluster order (host), for assembly
    std::vector<ElemRec> elems;
};

// Build the tree, the partition and the cluster-ordered element records.
void build_tree(const hm_elements& el, int leaf_size, double eta, Tree& T);

// Checks of the element description (shapes, finite values, half sides, triangles in
// their plane around their collocation point); who names the caller in the message.
void validate_elements(const hm_elements& el, const char* who);

// Device record of user element i (frame, shape, the triangle's vertices in its frame).
ElemRec make_elem_record(const hm_elements& el, int64_t i);

}  // namespace hm
