// rich_bvh.h -- host BVH builder interface.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "rich_internal.h"

namespace rich {

// Reference of "no surface" (never a node index or a leaf code).
constexpr int32_t kNoSurface = 0x7FFFFFFF;

struct BvhResult {
    std::vector<DevNode> nodes;   // breadth-first, node 0 is the root
    std::vector<int> leaf_order;  // leaf-order position -> input triangle
    std::vector<int32_t> surface_ref;  // per leaf-order position: the node
                                  // index or leaf code of the subtree holding
                                  // exactly its surface, or kNoSurface
    int depth = 0;                // inner-node levels
};

// Build over n_tris triangles given as 9 floats each; surface (may be null):
// per triangle a surface id >= 0 shared by the triangles of one surface, or
// -1. Returns false and sets err for malformed input.
bool build_bvh(const float *vertices, const int32_t *surface, int64_t n_tris, BvhResult &out,
               std::string &err);

}  // namespace rich
