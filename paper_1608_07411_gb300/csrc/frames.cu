// Per-frame TSDF octrees f_i* as the data-term source (Sec. 3.1 "Octree
// construction", Sec. 3.2 "Optimization on the Octree", Fig. 4, Table 1).
//
// Each frame's field (Eq. 1 at every finest-voxel centre, unobserved where
// w_i = 0) becomes an octree built top-down: a node is split while its
// voxels do not all share one weight, or while they are all observed and the
// spread of f over them (Eq. 2) exceeds tau; every node keeps the mean of the
// observed f below it, and its weight is 1 when any voxel below it is
// observed.  The data term of an iterate leaf n at level L reads the deepest
// node of the tree on the path to n at a level no finer than L (Fig. 4: the
// node at n's level when the tree has one, else the tree leaf containing n).
//
// Layout in HBM: per frame, its tree leaves sorted by Morton key (key, level,
// observed count, float64 sum of f), concatenated over frames, with float64
// and integer exclusive prefix sums of the sums and counts over the
// concatenation.  A lookup is one binary search for the tree leaf holding
// n's first voxel; when that leaf is finer than n, the node at n's level is an
// inner node whose leaves are the contiguous key range of n, found by a
// second binary search, and its mean is a difference of prefix sums.
//
// Build, frame by frame on one stream: level D-1 of a count / sum / min / max
// pyramid from the voxels (8 Eq. 1 evaluations per node), the levels above
// from their children (children summed in Morton order), per finest voxel the
// level of its tree leaf by descending the split rule, a scan of "first voxel
// of a tree leaf" flags, and the emission of the leaves.
#include "frames.cuh"

#include <math_constants.h>

namespace ofu {

namespace {

__host__ __device__ inline int64_t lev_off_f(int L) { return ((int64_t(1) << (3 * L)) - 1) / 7; }

__device__ __forceinline__ bool voxel_sample(const Cam& k, const float* range, int H, int W,
                                             const Geo& g, uint64_t m, float* f) {
  const float x = centre_coord(g.org[0], compact3(m), 1, g.vox);
  const float y = centre_coord(g.org[1], compact3(m >> 1), 1, g.vox);
  const float z = centre_coord(g.org[2], compact3(m >> 2), 1, g.vox);
  return eq1_sample(k, range, H, W, x, y, z, g.delta, g.eta, f);
}

// Level D-1 of the pyramid of frame `cam`: observed count, sum (children in
// order 0..7), min and max of f over the node's 8 voxels.
__global__ void k_ft_base(const float* __restrict__ range, const Cam* __restrict__ cam, int H,
                          int W, Geo g, int64_t nn, uint32_t* __restrict__ cnt,
                          double* __restrict__ tot, float* __restrict__ lo, float* __restrict__ hi) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= nn) return;
  const Cam k = *cam;
  uint32_t c = 0;
  double s = 0.0;
  float a = CUDART_INF_F, b = -CUDART_INF_F;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float f;
    if (voxel_sample(k, range, H, W, g, uint64_t(8 * j + q), &f)) {
      ++c;
      s += double(f);
      a = fminf(a, f);
      b = fmaxf(b, f);
    }
  }
  cnt[j] = c;
  tot[j] = s;
  lo[j] = a;
  hi[j] = b;
}

__global__ void k_ft_up(const uint32_t* __restrict__ ccnt, const double* __restrict__ ctot,
                        const float* __restrict__ clo, const float* __restrict__ chi, int64_t nn,
                        uint32_t* __restrict__ cnt, double* __restrict__ tot, float* __restrict__ lo,
                        float* __restrict__ hi) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= nn) return;
  uint32_t c = 0;
  double s = 0.0;
  float a = CUDART_INF_F, b = -CUDART_INF_F;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    c += ccnt[8 * j + q];
    s += ctot[8 * j + q];
    a = fminf(a, clo[8 * j + q]);
    b = fmaxf(b, chi[8 * j + q]);
  }
  cnt[j] = c;
  tot[j] = s;
  lo[j] = a;
  hi[j] = b;
}

struct Pyr {
  const uint32_t* cnt;
  const double* tot;
  const float* lo;
  const float* hi;
};

// Level of the tree leaf holding finest voxel m: descend while the node
// splits (mixed weights, or fully observed with spread > tau).
__device__ __forceinline__ int tree_level(uint64_t m, const Pyr& p, int D, double tau) {
  int L = 0;
  while (L < D) {
    const int64_t o = lev_off_f(L) + int64_t(m >> (3 * (D - L)));
    const uint32_t c = p.cnt[o];
    const uint32_t full = 1u << (3 * (D - L));
    const bool mixed = c > 0 && c < full;
    const bool wide = c == full && double(p.hi[o]) - double(p.lo[o]) > tau;
    if (!(mixed || wide)) break;
    ++L;
  }
  return L;
}

__global__ void k_ft_flags(Pyr p, int D, double tau, int64_t nvox, uint32_t* __restrict__ flags) {
  const int64_t m = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (m >= nvox) return;
  const int L = tree_level(uint64_t(m), p, D, tau);
  const uint64_t mask = (uint64_t(1) << (3 * (D - L))) - 1;
  flags[m] = (uint64_t(m) & mask) == 0 ? 1u : 0u;
}

// Emits the tree leaves of one frame at out + pos[m] (count and sum of a
// finest leaf from its own voxel).
__global__ void k_ft_emit(const uint32_t* __restrict__ flags, const uint32_t* __restrict__ pos, Pyr p,
                          int D, double tau, int64_t nvox, const float* __restrict__ range,
                          const Cam* __restrict__ cam, int H, int W, Geo g,
                          uint64_t* __restrict__ key, uint8_t* __restrict__ level,
                          uint64_t* __restrict__ cnt, double* __restrict__ tot) {
  const int64_t m = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (m >= nvox || !flags[m]) return;
  const uint32_t j = pos[m];
  const int L = tree_level(uint64_t(m), p, D, tau);
  key[j] = uint64_t(m);
  level[j] = uint8_t(L);
  if (L < D) {
    const int64_t o = lev_off_f(L) + int64_t(uint64_t(m) >> (3 * (D - L)));
    cnt[j] = p.cnt[o];
    tot[j] = p.tot[o];
  } else {
    float f;
    const bool w = voxel_sample(*cam, range, H, W, g, uint64_t(m), &f);
    cnt[j] = w ? 1u : 0u;
    tot[j] = w ? double(f) : 0.0;
  }
}

constexpr int kT = 256;
inline unsigned nblk(int64_t n) { return unsigned((n + kT - 1) / kT); }

}  // namespace

size_t frame_pyramid_nodes(int D) { return size_t(lev_off_f(D)); }

cudaError_t launch_frame_tree_flags(const float* range, const Cam* cam, int H, int W, Geo g,
                                    double tau, uint32_t* pcnt, double* ptot, float* plo,
                                    float* phi, uint32_t* flags, cudaStream_t s) {
  const int D = g.D;
  const int64_t nvox = int64_t(1) << (3 * D);
  // level L occupies [lev_off(L), lev_off(L + 1)) of the pyramid arrays
  const int64_t nb = int64_t(1) << (3 * (D - 1));
  const int64_t ob = lev_off_f(D - 1);
  k_ft_base<<<nblk(nb), kT, 0, s>>>(range, cam, H, W, g, nb, pcnt + ob, ptot + ob, plo + ob, phi + ob);
  count_launches(1);
  for (int L = D - 2; L >= 0; --L) {
    const int64_t nn = int64_t(1) << (3 * L);
    const int64_t o = lev_off_f(L), oc = lev_off_f(L + 1);
    k_ft_up<<<nblk(nn), kT, 0, s>>>(pcnt + oc, ptot + oc, plo + oc, phi + oc, nn, pcnt + o, ptot + o,
                                    plo + o, phi + o);
    count_launches(1);
  }
  k_ft_flags<<<nblk(nvox), kT, 0, s>>>(Pyr{pcnt, ptot, plo, phi}, D, tau, nvox, flags);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_frame_tree_emit(const uint32_t* flags, const uint32_t* pos, const uint32_t* pcnt,
                                   const double* ptot, const float* plo, const float* phi,
                                   double tau, const float* range, const Cam* cam, int H, int W,
                                   Geo g, uint64_t* key, uint8_t* level, uint64_t* cnt, double* tot,
                                   cudaStream_t s) {
  const int64_t nvox = int64_t(1) << (3 * g.D);
  k_ft_emit<<<nblk(nvox), kT, 0, s>>>(flags, pos, Pyr{pcnt, ptot, plo, phi}, g.D, tau, nvox, range,
                                      cam, H, W, g, key, level, cnt, tot);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace ofu
