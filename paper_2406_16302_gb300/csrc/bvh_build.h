// Host SAH BVH builder (see bvh_build.cpp).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace rp {

struct BuiltBVH {
    std::vector<float4> nodes;   // 4 float4 per inner node
    std::vector<float4> tris;    // 3 float4 per triangle in leaf order
    int depth = 0;               // inner-node levels
};

// verts: [*][3] float, tris: [n][3] vertex indices; triangle i gets the
// global id id_offset + i
BuiltBVH build_bvh(const float *verts, const uint32_t *tris, int n, int id_offset);

}  // namespace rp
