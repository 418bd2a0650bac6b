// Zero level set of the fused field as a triangle mesh (Sec. 3.3: the result
// is meshed by marching cubes).
//
// The leaf field is sampled at every finest-voxel centre (a voxel takes the
// value of the leaf containing it, found through the voxel -> leaf map).  A
// cube has eight neighbouring voxel centres as corners; u < 0 is inside,
// u >= 0 outside.  Every grid edge between centres of opposite sign carries
// one vertex, placed by linear interpolation; vertices are shared by the
// cubes around their edge.  Each cube's triangles are derived from its six
// faces instead of a stored case table: on a face (corners counter-clockwise
// seen from outside) every crossing where the boundary walk passes from
// outside to inside starts a contour segment that ends at the next crossing
// of the walk, which keeps the outside on the segment's left and separates
// the inside corners of a face with four crossings.  A face is seen the same
// way by both cubes that share it, so the surface is closed.  Every crossing
// starts one segment and ends one, so the segments form loops; loops are
// taken in the order their first segment was found (faces in the order
// -x, +x, -y, +y, -z, +z; crossings in walk order) and fanned from that
// segment's start.
//
// Three launches over the 8^D voxels in x-major order (index (x n + y) n + z):
// the field on a dense grid, per-voxel counts (vertices on the voxel's +x,
// +y, +z edges; triangles of the cube whose lowest corner it is), an
// exclusive scan of the packed counts, and the emission of positions and
// triangles at the scanned offsets.  The output order is therefore fixed:
// vertices by (voxel, axis), triangles by cube, then loop, then fan.
#include "mesh.cuh"

namespace ofu {

namespace {

// Corner c of a cube sits at offset (c & 1, c >> 1 & 1, c >> 2 & 1) from the
// cube's lowest voxel.  Faces -x, +x, -y, +y, -z, +z, each as its corners in
// counter-clockwise order seen from outside the cube, starting from the
// corner where the outward normal check put it (the walk order matters: it
// fixes which loop is found first).
__constant__ int8_t kFaceRing[6][4] = {{4, 6, 2, 0}, {1, 3, 7, 5}, {0, 1, 5, 4},
                                       {6, 7, 3, 2}, {2, 3, 1, 0}, {4, 5, 7, 6}};

struct Grid {
  const float* g;  // value at voxel (x, y, z), index (x n + y) n + z
  uint32_t n;
};

__device__ __forceinline__ size_t lin(uint32_t n, uint32_t x, uint32_t y, uint32_t z) {
  return (size_t(x) * n + y) * n + z;
}

// Cube edge between corners i and j (one bit apart): code lo * 8 + hi.
__device__ __forceinline__ int edge_code(int i, int j) { return i < j ? i * 8 + j : j * 8 + i; }

// Triangles of a cube with the given inside flags; emit(k, a, b, c) gets the
// k-th triangle as three edge codes.  Returns the triangle count.
template <typename Emit>
__device__ int cube_triangles(const bool inside[8], Emit emit) {
  int8_t nxt[64];
#pragma unroll
  for (int k = 0; k < 64; ++k) nxt[k] = -1;
  int8_t starts[12];
  int ns = 0;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    int cr[4];
    int nc = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = kFaceRing[f][k], j = kFaceRing[f][(k + 1) & 3];
      if (inside[i] != inside[j]) cr[nc++] = k;
    }
    for (int s = 0; s < nc; ++s) {
      const int k = cr[s];
      const int i = kFaceRing[f][k], j = kFaceRing[f][(k + 1) & 3];
      if (!inside[i] && inside[j] && ns < 12) {
        const int k2 = cr[s + 1 < nc ? s + 1 : 0];
        const int i2 = kFaceRing[f][k2], j2 = kFaceRing[f][(k2 + 1) & 3];
        const int from = edge_code(i, j);
        nxt[from] = int8_t(edge_code(i2, j2));
        starts[ns++] = int8_t(from);
      }
    }
  }
  uint64_t seen = 0;
  int nt = 0;
  for (int si = 0; si < ns; ++si) {
    const int st = starts[si];
    if (seen >> st & 1ull) continue;
    seen |= 1ull << st;
    // a loop has at most 12 vertices (one per cube edge); the bound and the
    // -1 checks only guard the walk, every listed edge has a successor
    int a = nxt[st];
    for (int guard = 0; guard < 12 && a >= 0 && a != st; ++guard) {
      seen |= 1ull << a;
      const int b = nxt[a];
      if (b < 0 || b == st) break;
      emit(nt, st, a, b);
      ++nt;
      a = b;
    }
  }
  return nt;
}

__global__ void k_mesh_field(View v, const float* __restrict__ u, float* __restrict__ g) {
  const uint32_t n = 1u << v.D;
  const size_t nv = size_t(n) * n * n;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nv;
       i += size_t(gridDim.x) * blockDim.x) {
    const uint32_t z = uint32_t(i % n), y = uint32_t((i / n) % n), x = uint32_t(i / (size_t(n) * n));
    g[i] = u[v.map[morton(x, y, z)]];
  }
}

__device__ __forceinline__ void corners(const Grid& G, uint32_t x, uint32_t y, uint32_t z,
                                        bool inside[8]) {
#pragma unroll
  for (int c = 0; c < 8; ++c)
    inside[c] = G.g[lin(G.n, x + (c & 1), y + ((c >> 1) & 1), z + ((c >> 2) & 1))] < 0.0f;
}

// Per voxel: bits of its crossed +x/+y/+z edges (cm) and packed counts
// (vertices low 32 bits, triangles of its cube high 32 bits).
__global__ void k_mesh_count(Grid G, uint8_t* __restrict__ cm, uint64_t* __restrict__ cnt) {
  const uint32_t n = G.n;
  const size_t nv = size_t(n) * n * n;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nv;
       i += size_t(gridDim.x) * blockDim.x) {
    const uint32_t z = uint32_t(i % n), y = uint32_t((i / n) % n), x = uint32_t(i / (size_t(n) * n));
    const bool in0 = G.g[i] < 0.0f;
    uint32_t m = 0;
    if (x + 1 < n && (G.g[lin(n, x + 1, y, z)] < 0.0f) != in0) m |= 1;
    if (y + 1 < n && (G.g[lin(n, x, y + 1, z)] < 0.0f) != in0) m |= 2;
    if (z + 1 < n && (G.g[lin(n, x, y, z + 1)] < 0.0f) != in0) m |= 4;
    uint32_t nt = 0;
    if (x + 1 < n && y + 1 < n && z + 1 < n) {
      bool inside[8];
      corners(G, x, y, z, inside);
      int k = 0;
#pragma unroll
      for (int c = 0; c < 8; ++c) k += inside[c];
      if (k > 0 && k < 8) nt = uint32_t(cube_triangles(inside, [](int, int, int, int) {}));
    }
    cm[i] = uint8_t(m);
    cnt[i] = uint64_t(__popc(m)) | (uint64_t(nt) << 32);
  }
}

// Vertex index of the grid edge of cube-edge code `code` of the cube at
// (x, y, z): the edge's lower voxel and axis, then that voxel's offset plus
// the rank of the axis among its crossed edges.
__device__ __forceinline__ int32_t vertex_id(const Grid& G, const uint8_t* __restrict__ cm,
                                             const uint64_t* __restrict__ off, uint32_t x,
                                             uint32_t y, uint32_t z, int code) {
  const int lo = code >> 3, hi = code & 7;
  const int axis = __ffs(lo ^ hi) - 1;
  const size_t j = lin(G.n, x + (lo & 1), y + ((lo >> 1) & 1), z + ((lo >> 2) & 1));
  return int32_t(uint32_t(off[j]) + __popc(uint32_t(cm[j]) & ((1u << axis) - 1)));
}

__global__ void k_mesh_emit(Grid G, const uint8_t* __restrict__ cm, const uint64_t* __restrict__ off,
                            double ox, double oy, double oz, double spacing,
                            float* __restrict__ verts, int32_t* __restrict__ tris) {
  const uint32_t n = G.n;
  const size_t nv = size_t(n) * n * n;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nv;
       i += size_t(gridDim.x) * blockDim.x) {
    const uint32_t z = uint32_t(i % n), y = uint32_t((i / n) % n), x = uint32_t(i / (size_t(n) * n));
    const uint32_t m = cm[i];
    const uint64_t o = off[i];
    if (m) {
      // t = a / (a - b) along the edge from this voxel; position
      // origin + ((corner + t e_axis) + 1/2) spacing, all in float64 with one
      // rounding per operation
      const double a = double(G.g[i]);
      uint32_t r = uint32_t(o);
      const uint32_t c[3] = {x, y, z};
      const double org[3] = {ox, oy, oz};
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        if (!(m >> ax & 1u)) continue;
        const size_t j = lin(n, x + (ax == 0), y + (ax == 1), z + (ax == 2));
        const double b = double(G.g[j]);
        const double t = __ddiv_rn(a, __dsub_rn(a, b));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const double pos = k == ax ? __dadd_rn(double(c[k]), t) : double(c[k]);
          verts[3 * size_t(r) + k] = float(__dadd_rn(org[k], __dmul_rn(__dadd_rn(pos, 0.5), spacing)));
        }
        ++r;
      }
    }
    if (uint32_t(o >> 32) != uint32_t(off[i + 1] >> 32)) {
      bool inside[8];
      corners(G, x, y, z, inside);
      int32_t* out = tris + 3 * size_t(o >> 32);
      cube_triangles(inside, [&](int k, int ea, int eb, int ec) {
        out[3 * k + 0] = vertex_id(G, cm, off, x, y, z, ea);
        out[3 * k + 1] = vertex_id(G, cm, off, x, y, z, eb);
        out[3 * k + 2] = vertex_id(G, cm, off, x, y, z, ec);
      });
    }
  }
}

constexpr int kMeshThreads = 256;

inline unsigned grid_for(size_t n) {
  const size_t b = (n + kMeshThreads - 1) / kMeshThreads;
  return unsigned(b < 152 * 64 ? b : 152 * 64);   // grid-stride beyond 64 blocks per SM
}

}  // namespace

cudaError_t launch_mesh_count(View v, const float* u, float* grid, uint8_t* cm, uint64_t* cnt,
                              cudaStream_t s) {
  const uint32_t n = 1u << v.D;
  const size_t nv = size_t(n) * n * n;
  k_mesh_field<<<grid_for(nv), kMeshThreads, 0, s>>>(v, u, grid);
  count_launches(1);
  k_mesh_count<<<grid_for(nv), kMeshThreads, 0, s>>>(Grid{grid, n}, cm, cnt);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mesh_emit(int D, const float* grid, const uint8_t* cm, const uint64_t* off,
                             const double origin[3], double spacing, float* verts, int32_t* tris,
                             cudaStream_t s) {
  const uint32_t n = 1u << D;
  const size_t nv = size_t(n) * n * n;
  k_mesh_emit<<<grid_for(nv), kMeshThreads, 0, s>>>(Grid{grid, n}, cm, off, origin[0], origin[1],
                                                   origin[2], spacing, verts, tris);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace ofu
