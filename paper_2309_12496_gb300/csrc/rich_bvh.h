// rich_bvh.h -- host BVH builder interface.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "rich_internal.h"

namespace rich {

struct BvhResult {
    std::vector<DevNode> nodes;   // breadth-first, node 0 is the root
    std::vector<int> leaf_order;  // leaf-order position -> input triangle
    int depth = 0;                // inner-node levels
};

struct Bvh8Result {
    std::vector<DevNode8> nodes;  // breadth-first, node 0 is the root
    std::vector<int> leaf_order;  // leaf-order position -> input triangle
    int depth = 0;                // node levels
};

// Build over n_tris triangles given as 9 floats each. Returns false and sets
// err for malformed input.
bool build_bvh(const float *vertices, int64_t n_tris, BvhResult &out,
               std::string &err);

// Eight-wide BVH: the binary SAH tree collapsed (largest-area inner child
// opened first) into nodes of up to eight children, children placed in
// octant slots, boxes quantised outwards to 8 bits.
bool build_bvh8(const float *vertices, int64_t n_tris, Bvh8Result &out,
                std::string &err);

}  // namespace rich
