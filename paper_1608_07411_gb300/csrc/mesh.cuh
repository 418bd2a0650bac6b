// Launchers of the marching-cubes extraction of the zero level set (mesh.cu).
#pragma once

#include "ofu_internal.cuh"

namespace ofu {

// The field on a dense grid of the 8^D voxel centres (grid, x-major), then per
// voxel the mask of its crossed +x/+y/+z edges (cm) and packed counts (cnt:
// vertices low 32 bits, triangles of the cube at that voxel high 32 bits).
cudaError_t launch_mesh_count(View v, const float* u, float* grid, uint8_t* cm, uint64_t* cnt,
                              cudaStream_t s);

// Vertices (float32 [V][3], world coordinates) and triangles (int32 [T][3])
// at the exclusive scan `off` of the packed counts (8^D + 1 entries).
cudaError_t launch_mesh_emit(int D, const float* grid, const uint8_t* cm, const uint64_t* off,
                             const double origin[3], double spacing, float* verts, int32_t* tris,
                             cudaStream_t s);

}  // namespace ofu
