// Launchers of the per-frame TSDF octree build (frames.cu).
#pragma once

#include "ofu_internal.cuh"

namespace ofu {

// Entries of the per-frame pyramid (levels 0 .. D-1): (8^D - 1) / 7.
size_t frame_pyramid_nodes(int D);

// One frame's pyramid (count, float64 sum, min, max of the observed Eq. 1
// samples below each node, levels 0 .. D-1) and, per finest voxel (Morton
// order), the flag "first voxel of a tree leaf".  `range` and `cam` are that
// frame's range map and camera.
cudaError_t launch_frame_tree_flags(const float* range, const Cam* cam, int H, int W, Geo g,
                                    double tau, uint32_t* pcnt, double* ptot, float* plo,
                                    float* phi, uint32_t* flags, cudaStream_t s);

// The tree leaves of that frame at the scanned positions `pos` of the flags:
// key, level, observed count and float64 sum of f.
cudaError_t launch_frame_tree_emit(const uint32_t* flags, const uint32_t* pos, const uint32_t* pcnt,
                                   const double* ptot, const float* plo, const float* phi,
                                   double tau, const float* range, const Cam* cam, int H, int W,
                                   Geo g, uint64_t* key, uint8_t* level, uint64_t* cnt, double* tot,
                                   cudaStream_t s);

}  // namespace ofu
