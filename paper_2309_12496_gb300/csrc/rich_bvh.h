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

// Build over n_tris triangles given as 9 floats each. Returns false and sets
// err for malformed input.
bool build_bvh(const float *vertices, int64_t n_tris, BvhResult &out,
               std::string &err);

}  // namespace rich
