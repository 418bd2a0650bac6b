// Structure kernels: prefix sums, Eq. 1 integration, Eq. 2 construction,
// face neighbours, step sizes and the split/join pass (Sec. 3.1-3.2).
#include <math_constants.h>

#include "ofu_internal.cuh"

namespace ofu {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// ---------------------------------------------------------------------------
// Prefix sums: tiles of kTile items.  One pass writes the tile totals; a
// second pass scans each tile in shared memory and adds its tile offset,
// which each block sums itself from the totals before it when there are at
// most kSelfOffsetTiles tiles (two launches in all), else takes from a
// recursive exclusive scan of the totals.

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kTile = kScanThreads * kScanItems;
constexpr int kSelfOffsetTiles = 2048;

// Shared-memory slot of tile item i: one pad slot every 32 (4-byte) or 16
// (8-byte) items keeps both the coalesced-order and the thread-order
// accesses free of bank conflicts.
template <typename T>
__device__ __forceinline__ int tile_slot(int i) {
  return i + (i >> (sizeof(T) == 8 ? 4 : 5));
}
constexpr int kTileSlots = kTile + kTile / 16;

template <typename T>
__device__ T warp_inclusive(T v) {
  const int lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan of one value per thread across the block; *total gets the sum.
template <typename T>
__device__ T block_exclusive(T v, T* total) {
  __shared__ T warp_sums[32];
  const int lane = lane_id(), wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T inc = warp_inclusive(v);
  if (lane == 31) warp_sums[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T w = lane < nw ? warp_sums[lane] : T(0);
    T wi = warp_inclusive(w);
    warp_sums[lane] = wi - w;
    if (lane == 31) warp_sums[31] = wi;  // nw <= 31 leaves slot 31 for the total
  }
  __syncthreads();
  T res = warp_sums[wid] + inc - v;
  *total = warp_sums[31];
  __syncthreads();
  return res;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_tile_sums(const T* __restrict__ in, int64_t n,
                                                            T* __restrict__ sums) {
  const int64_t base = int64_t(blockIdx.x) * kTile;
  T acc = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + int64_t(k) * kScanThreads + threadIdx.x;
    if (i < n) acc += in[i];
  }
  T tot;
  block_exclusive(acc, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// offs == nullptr: a single tile.  self_offset: offs holds the tile totals
// and the block adds those of the tiles before it; else offs[b] is the
// tile's offset.
template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_tile_scan(const T* in, T* out, int64_t n,
                                                            const T* __restrict__ offs,
                                                            int self_offset) {
  __shared__ T tile[kTileSlots];
  const int64_t base = int64_t(blockIdx.x) * kTile;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int idx = k * kScanThreads + threadIdx.x;
    const int64_t i = base + idx;
    tile[tile_slot<T>(idx)] = i < n ? in[i] : T(0);
  }
  T off = 0;
  if (offs && self_offset) {
    T acc = 0;
    for (int b = threadIdx.x; b < int(blockIdx.x); b += kScanThreads) acc += offs[b];
    block_exclusive(acc, &off);  // synchronises the block, so the tile is loaded
  } else {
    if (offs) off = offs[blockIdx.x];
    __syncthreads();
  }
  T loc[kScanItems];
  T s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    loc[k] = tile[tile_slot<T>(threadIdx.x * kScanItems + k)];
    s += loc[k];
  }
  T tot;
  T run = block_exclusive(s, &tot) + off;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    tile[tile_slot<T>(threadIdx.x * kScanItems + k)] = run;
    run += loc[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int idx = k * kScanThreads + threadIdx.x;
    const int64_t i = base + idx;
    if (i < n) out[i] = tile[tile_slot<T>(idx)];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = off + tot;
}

// ---------------------------------------------------------------------------
// Warp-cooperative bitonic sort of P floats in shared memory (P power of 2).
template <int P>
__device__ __forceinline__ void warp_bitonic(float* a) {
  const int lane = lane_id();
#pragma unroll 1
  for (int k = 2; k <= P; k <<= 1) {
#pragma unroll 1
    for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
      for (int i = lane; i < P; i += 32) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const float ai = a[i], aj = a[ixj];
          const bool up = (i & k) == 0;
          if ((ai > aj) == up) {
            a[i] = aj;
            a[ixj] = ai;
          }
        }
      }
      __syncwarp();
    }
  }
}

__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ float warp_min_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}
__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// Median of the W smallest entries of the sorted array a (float64 result):
// the middle one for odd W, (a + b) * 0.5 of the two middle ones for even W,
// -1 when W = 0.
__device__ __forceinline__ double sorted_median(const float* a, int W) {
  if (W == 0) return -1.0;
  if (W & 1) return double(a[(W - 1) / 2]);
  return (double(a[W / 2 - 1]) + double(a[W / 2])) * 0.5;
}

constexpr int kWarpsPerBlock = 8;

// Stage the cameras of all frames in shared memory.
__device__ __forceinline__ void stage_cams(Cam* sc, const Cam* cams, int F) {
  const int words = F * int(sizeof(Cam) / 4);
  const float* src = reinterpret_cast<const float*>(cams);
  float* dst = reinterpret_cast<float*>(sc);
  for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// Samples of one point by one warp into a[0..P) (+inf where unobserved);
// sample(i, &f) gives frame i's sample and whether it is observed.  Returns W
// and the min / max of the observed samples.
template <int P, typename Src>
__device__ __forceinline__ int warp_samples_of(Src sample, int F, float* a, float* mn, float* mx) {
  const int lane = lane_id();
  int cnt = 0;
  float lo = CUDART_INF_F, hi = -CUDART_INF_F;
#pragma unroll 4
  for (int i = lane; i < P; i += 32) {
    float f = CUDART_INF_F;
    if (i < F) {
      float t;
      if (sample(i, &t)) {
        f = t;
        ++cnt;
        lo = fminf(lo, t);
        hi = fmaxf(hi, t);
      }
    }
    a[i] = f;
  }
  *mn = warp_min_f(lo);
  *mx = warp_max_f(hi);
  return warp_sum_i(cnt);
}

// Eq. 1 samples of the point (x, y, z) by one warp (see warp_samples_of).
template <int P>
__device__ __forceinline__ int warp_samples(const Cam* sc, const float* depth, int F, int H, int W,
                                            float x, float y, float z, float delta, float eta,
                                            float* a, float* mn, float* mx) {
  return warp_samples_of<P>(
      [&](int i, float* t) {
        return eq1_sample(sc[i], depth + size_t(i) * H * W, H, W, x, y, z, delta, eta, t);
      },
      F, a, mn, mx);
}

// ---------------------------------------------------------------------------
// Frame classification of a box of voxel centres.  A warp of the median scan
// holds 32 Morton-consecutive finest voxels, a 4 x 4 x 2 box of centres.  For
// most frames the whole box either sees one value or is unobserved: it lies
// in front of the surface by more than delta (every Eq. 1 sample is +1), or
// behind it by more than eta, outside the image or behind the camera (no
// sample).  The test bounds the box's projection by its 8 corners (the
// projection of a convex box in front of the camera is the hull of the
// corners'), the ranges under it by the range pyramid, and the distances by
// the nearest point and the farthest corner.  Every bound is widened by a
// margin far above float32 rounding (relative 1e-5 against errors near 1e-6),
// so a frame classified this way gives every voxel exactly what Eq. 1 in
// float32 gives it; any other frame is "mixed" and evaluated per voxel.
constexpr int kObsMixed = 0, kObsOne = 1, kObsNone = 2;

// Min and max of the valid ranges over the pixel rectangle [px0, px1] x
// [py0, py1] (inside the image) of frame f, from the smallest pyramid level
// at which the rectangle touches at most 2 x 2 texels (a superset of it).
__device__ __forceinline__ float2 range_bounds(const RangePyr& rp, const int* lv, const float* range,
                                               int f, int H, int W, int px0, int px1, int py0,
                                               int py1) {
  int k = 0;
  while (k < rp.nl && ((px1 >> k) - (px0 >> k) > 1 || (py1 >> k) - (py0 >> k) > 1)) ++k;
  float lo = CUDART_INF_F, hi = -CUDART_INF_F;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int x = (a ? px1 : px0) >> k, y = (b ? py1 : py0) >> k;
      float2 t;
      if (k == 0) {
        const float r = range[size_t(f) * H * W + size_t(y) * W + x];
        t.x = t.y = r > 0.0f ? r : -CUDART_INF_F;
      } else {
        const int wk = lv[k], hk = lv[kMaxRangeLevels + 1 + k], ok = lv[2 * (kMaxRangeLevels + 1) + k];
        t = rp.tex[f * rp.frame_texels + ok + int64_t(min(y, hk - 1)) * wk + min(x, wk - 1)];
      }
      lo = fminf(lo, t.x);
      hi = fmaxf(hi, t.y);
    }
  return make_float2(lo, hi);
}

// Class of frame f for every voxel centre in the box with centre (bx, by, bz)
// and half extents (hx, hy, hz); lv holds the pyramid's level widths,
// heights and offsets.
__device__ __forceinline__ int classify_box(const Cam& k, const float* range, const RangePyr& rp,
                                            const int* lv, int f, int H, int W, float bx, float by,
                                            float bz, float hx, float hy, float hz, float delta,
                                            float eta) {
  const float dx = bx - k.c[0], dy = by - k.c[1], dz = bz - k.c[2];
  const float xc = k.r[0] * dx + k.r[3] * dy + k.r[6] * dz;
  const float yc = k.r[1] * dx + k.r[4] * dy + k.r[7] * dz;
  const float zc = k.r[2] * dx + k.r[5] * dy + k.r[8] * dz;
  const float mz = 1e-5f * (fabsf(dx) + fabsf(dy) + fabsf(dz) + hx + hy + hz);
  const float ez = fabsf(k.r[2]) * hx + fabsf(k.r[5]) * hy + fabsf(k.r[8]) * hz;
  if (zc + ez < -mz) return kObsNone;   // the whole box behind the camera
  if (!(zc - ez > mz)) return kObsMixed;
  float u0 = CUDART_INF_F, u1 = -CUDART_INF_F, v0 = CUDART_INF_F, v1 = -CUDART_INF_F;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float sx = c & 1 ? hx : -hx, sy = c & 2 ? hy : -hy, sz = c & 4 ? hz : -hz;
    const float X = xc + k.r[0] * sx + k.r[3] * sy + k.r[6] * sz;
    const float Y = yc + k.r[1] * sx + k.r[4] * sy + k.r[7] * sz;
    const float iz = __frcp_rn(zc + k.r[2] * sx + k.r[5] * sy + k.r[8] * sz);
    const float u = k.fx * (X * iz) + k.cx, v = k.fy * (Y * iz) + k.cy;
    u0 = fminf(u0, u);
    u1 = fmaxf(u1, u);
    v0 = fminf(v0, v);
    v1 = fmaxf(v1, v);
  }
  const float mu = 1e-4f * (fmaxf(fabsf(u0), fabsf(u1)) + fabsf(k.cx)) + 1e-3f;
  const float mv = 1e-4f * (fmaxf(fabsf(v0), fabsf(v1)) + fabsf(k.cy)) + 1e-3f;
  const float ua = u0 - mu, ub = u1 + mu, va = v0 - mv, vb = v1 + mv;
  if (ub < 0.0f || ua >= float(W) || vb < 0.0f || va >= float(H)) return kObsNone;
  if (!(ua >= 0.0f && ub < float(W) && va >= 0.0f && vb < float(H))) return kObsMixed;
  const float2 r = range_bounds(rp, lv, range, f, H, W, int(floorf(ua)), int(floorf(ub)),
                                int(floorf(va)), int(floorf(vb)));
  const float nx = fmaxf(fabsf(dx) - hx, 0.0f), ny = fmaxf(fabsf(dy) - hy, 0.0f),
              nz = fmaxf(fabsf(dz) - hz, 0.0f);
  const float fx = fabsf(dx) + hx, fy = fabsf(dy) + hy, fz = fabsf(dz) + hz;
  const float dmin = sqrtf(nx * nx + ny * ny + nz * nz), dmax = sqrtf(fx * fx + fy * fy + fz * fz);
  const float md = 1e-5f * dmax;
  // every pixel valid and every phi >= delta: all samples +1
  if (r.x > 0.0f && r.x - (dmax + md) >= delta + 1e-5f * (r.x + dmax)) return kObsOne;
  // every pixel invalid or every phi < -eta: unobserved (r.y = -inf: all invalid)
  if (r.y - (dmin - md) < -eta - 1e-5f * (fabsf(r.y) + dmax)) return kObsNone;
  return kObsMixed;
}

// Median field, first pass: a thread per finest voxel walks the frames and
// keeps W, min and max of the observed Eq. 1 samples.  The median is final
// where W = 0 (-1) or every observed sample is the same value; the other
// voxels (near a surface) are queued for the warp sort of k_dense_u0.
// Warps stride over the voxels together, so every lane reaches the ballots.
// A full warp first classifies the frames against its box of centres (lane
// i the frames i, i + 32, ...); only the mixed frames are evaluated per voxel.
__global__ void __launch_bounds__(256) k_dense_scan(const float* __restrict__ depth,
                                                    const Cam* __restrict__ cams, int F, int H,
                                                    int W, Geo g, RangePyr rp, int64_t nvox,
                                                    double* __restrict__ u0,
                                                    uint32_t* __restrict__ queue,
                                                    unsigned long long* __restrict__ nqueue) {
  extern __shared__ float4 smem_dyn[];
  __shared__ int lv[3 * (kMaxRangeLevels + 1)];
  Cam* sc = reinterpret_cast<Cam*>(smem_dyn);
  for (int i = threadIdx.x; i <= kMaxRangeLevels; i += blockDim.x) {
    lv[i] = rp.w[i];
    lv[kMaxRangeLevels + 1 + i] = rp.h[i];
    lv[2 * (kMaxRangeLevels + 1) + i] = rp.off[i];
  }
  stage_cams(sc, cams, F);
  const int lane = lane_id();
  for (int64_t m0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) & ~int64_t(31); m0 < nvox;
       m0 += int64_t(gridDim.x) * blockDim.x) {
    const int64_t m = m0 + lane;
    const uint32_t ix = compact3(uint64_t(m)), iy = compact3(uint64_t(m) >> 1),
                   iz = compact3(uint64_t(m) >> 2);
    const float x = centre_coord(g.org[0], ix, 1, g.vox);
    const float y = centre_coord(g.org[1], iy, 1, g.vox);
    const float z = centre_coord(g.org[2], iz, 1, g.vox);
    int cnt = 0;
    float lo = CUDART_INF_F, hi = -CUDART_INF_F;
    auto eval = [&](int i) {
      float t;
      if (eq1_sample(sc[i], depth + size_t(i) * H * W, H, W, x, y, z, g.delta, g.eta, &t)) {
        ++cnt;
        lo = fminf(lo, t);
        hi = fmaxf(hi, t);
      }
    };
    if (m0 + 32 <= nvox) {
      // the warp's box: x over 4 voxels, y over 4, z over 2 (Morton bits
      // x0 y0 z0 x1 y1 below the warp's base)
      const uint32_t bx0 = compact3(uint64_t(m0)), by0 = compact3(uint64_t(m0) >> 1),
                     bz0 = compact3(uint64_t(m0) >> 2);
      const float xa = centre_coord(g.org[0], bx0, 1, g.vox), xb = centre_coord(g.org[0], bx0 + 3, 1, g.vox);
      const float ya = centre_coord(g.org[1], by0, 1, g.vox), yb = centre_coord(g.org[1], by0 + 3, 1, g.vox);
      const float za = centre_coord(g.org[2], bz0, 1, g.vox), zb = centre_coord(g.org[2], bz0 + 1, 1, g.vox);
      int ones = 0;
      for (int c0 = 0; c0 < F; c0 += 32) {
        const int f = c0 + lane;
        const int cls = f < F ? classify_box(sc[f], depth, rp, lv, f, H, W, 0.5f * (xa + xb),
                                             0.5f * (ya + yb), 0.5f * (za + zb), 0.5f * (xb - xa),
                                             0.5f * (yb - ya), 0.5f * (zb - za), g.delta, g.eta)
                              : kObsNone;
        ones += __popc(__ballot_sync(kFull, cls == kObsOne));
        for (unsigned mixed = __ballot_sync(kFull, cls == kObsMixed); mixed; mixed &= mixed - 1)
          eval(c0 + __ffs(mixed) - 1);
      }
      if (ones) {
        cnt += ones;
        lo = fminf(lo, 1.0f);
        hi = fmaxf(hi, 1.0f);
      }
    } else if (m < nvox) {
      for (int i = 0; i < F; ++i) eval(i);
    }
    const bool sort = m < nvox && cnt > 0 && lo != hi;
    if (m < nvox && !sort) u0[m] = cnt == 0 ? -1.0 : double(lo);
    const unsigned bal = __ballot_sync(kFull, sort);
    if (bal) {
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(nqueue, static_cast<unsigned long long>(__popc(bal)));
      base = __shfl_sync(kFull, base, 0);
      if (sort) queue[base + __popc(bal & ((1u << lane) - 1))] = uint32_t(m);
    }
  }
}

// Pyramid level 1 from the range maps, then each level from the one below.
__global__ void k_rpyr_base(const float* __restrict__ range, int F, int H, int W, RangePyr rp,
                            float2* __restrict__ tex) {
  const int w1 = rp.w[1], h1 = rp.h[1];
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= int64_t(F) * w1 * h1) return;
  const int f = int(i / (int64_t(w1) * h1));
  const int r = int(i - int64_t(f) * w1 * h1);
  const int ty = r / w1, tx = r - ty * w1;
  float lo = CUDART_INF_F, hi = -CUDART_INF_F;
  for (int y = 2 * ty; y < min(2 * ty + 2, H); ++y)
    for (int x = 2 * tx; x < min(2 * tx + 2, W); ++x) {
      const float v = range[size_t(f) * H * W + size_t(y) * W + x];
      const float c = v > 0.0f ? v : -CUDART_INF_F;
      lo = fminf(lo, c);
      hi = fmaxf(hi, c);
    }
  tex[f * rp.frame_texels + rp.off[1] + r] = make_float2(lo, hi);
}

__global__ void k_rpyr_up(int F, int k, RangePyr rp, float2* __restrict__ tex) {
  const int wk = rp.w[k], hk = rp.h[k], wb = rp.w[k - 1], hb = rp.h[k - 1];
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= int64_t(F) * wk * hk) return;
  const int f = int(i / (int64_t(wk) * hk));
  const int r = int(i - int64_t(f) * wk * hk);
  const int ty = r / wk, tx = r - ty * wk;
  const float2* below = tex + f * rp.frame_texels + rp.off[k - 1];
  float lo = CUDART_INF_F, hi = -CUDART_INF_F;
  for (int y = 2 * ty; y < min(2 * ty + 2, hb); ++y)
    for (int x = 2 * tx; x < min(2 * tx + 2, wb); ++x) {
      const float2 t = below[y * wb + x];
      lo = fminf(lo, t.x);
      hi = fmaxf(hi, t.y);
    }
  tex[f * rp.frame_texels + rp.off[k] + r] = make_float2(lo, hi);
}

// Median field, second pass: a warp per queued voxel (one frame per lane)
// sorts the samples in shared memory and takes the median.
template <int P>
__global__ void __launch_bounds__(256) k_dense_u0(const float* __restrict__ depth,
                                                  const Cam* __restrict__ cams, int F, int H,
                                                  int W, Geo g, const uint32_t* __restrict__ queue,
                                                  const unsigned long long* __restrict__ nqueue,
                                                  double* __restrict__ u0) {
  extern __shared__ float4 smem_dyn[];
  Cam* sc = reinterpret_cast<Cam*>(smem_dyn);
  float* bufs = reinterpret_cast<float*>(sc + F);
  stage_cams(sc, cams, F);
  const int warp = threadIdx.x >> 5;
  float* a = bufs + warp * P;
  const int64_t nq = int64_t(*nqueue);
  for (int64_t j = int64_t(blockIdx.x) * kWarpsPerBlock + warp; j < nq;
       j += int64_t(gridDim.x) * kWarpsPerBlock) {
    const int64_t m = queue[j];
    const uint32_t ix = compact3(uint64_t(m)), iy = compact3(uint64_t(m) >> 1),
                   iz = compact3(uint64_t(m) >> 2);
    const float x = centre_coord(g.org[0], ix, 1, g.vox);
    const float y = centre_coord(g.org[1], iy, 1, g.vox);
    const float z = centre_coord(g.org[2], iz, 1, g.vox);
    float mn, mx;
    const int cnt = warp_samples<P>(sc, depth, F, H, W, x, y, z, g.delta, g.eta, a, &mn, &mx);
    double med;
    if (cnt == 0) {
      med = -1.0;
    } else if (mn == mx) {
      med = double(mn);
    } else {
      __syncwarp();
      warp_bitonic<P>(a);
      med = sorted_median(a, cnt);
    }
    if (lane_id() == 0) u0[m] = med;
    __syncwarp();
  }
}

__global__ void k_range_map(float* __restrict__ depth, const Cam* __restrict__ cams, int F, int H,
                            int W) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t per = int64_t(H) * W;
  if (i >= per * F) return;
  const int f = int(i / per);
  const int64_t r = i - int64_t(f) * per;
  const int py = int(r / W), px = int(r - int64_t(py) * W);
  depth[i] = pixel_range(cams[f], depth[i], px, py);
}

// ---------------------------------------------------------------------------
// Eq. 2 pyramid: per node the min and max of u0 over its finest voxels.
// Level L occupies [(8^L - 1)/7, (8^(L+1) - 1)/7) of mn / mx.

__host__ __device__ inline int64_t lev_off(int L) { return ((int64_t(1) << (3 * L)) - 1) / 7; }

__global__ void k_pyr_base(const double* __restrict__ u0, int64_t nn, double* __restrict__ mn,
                           double* __restrict__ mx) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= nn) return;
  double lo = u0[8 * j], hi = lo;
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    const double v = u0[8 * j + k];
    lo = fmin(lo, v);
    hi = fmax(hi, v);
  }
  mn[j] = lo;
  mx[j] = hi;
}

__global__ void k_pyr_up(const double* __restrict__ cmn, const double* __restrict__ cmx,
                         int64_t nn, double* __restrict__ mn, double* __restrict__ mx) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= nn) return;
  double lo = cmn[8 * j], hi = cmx[8 * j];
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    lo = fmin(lo, cmn[8 * j + k]);
    hi = fmax(hi, cmx[8 * j + k]);
  }
  mn[j] = lo;
  mx[j] = hi;
}

// Level of the leaf containing finest voxel m: descend while the node's
// spread exceeds tau (Eq. 2).
__device__ __forceinline__ int constructed_level(uint64_t m, const double* mn, const double* mx,
                                                 int D, double tau) {
  int L = 0;
  while (L < D) {
    const int64_t node = int64_t(m >> (3 * (D - L)));
    const int64_t o = lev_off(L) + node;
    if (!(mx[o] - mn[o] > tau)) break;
    ++L;
  }
  return L;
}

__global__ void k_leaf_flags(const double* __restrict__ mn, const double* __restrict__ mx, int D,
                             double tau, int64_t nvox, uint32_t* __restrict__ flags) {
  const int64_t m = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (m >= nvox) return;
  const int L = constructed_level(uint64_t(m), mn, mx, D, tau);
  const uint64_t mask = (uint64_t(1) << (3 * (D - L))) - 1;
  flags[m] = (uint64_t(m) & mask) == 0 ? 1u : 0u;
}

__global__ void k_emit_constructed(const uint32_t* __restrict__ flags,
                                   const uint32_t* __restrict__ pos, const double* __restrict__ mn,
                                   const double* __restrict__ mx, int D, double tau, int64_t nvox,
                                   uint64_t* __restrict__ key, uint8_t* __restrict__ level) {
  const int64_t m = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (m >= nvox || !flags[m]) return;
  const uint32_t j = pos[m];
  key[j] = uint64_t(m);
  level[j] = uint8_t(constructed_level(uint64_t(m), mn, mx, D, tau));
}

// ---------------------------------------------------------------------------
// Eq. 1 samples at leaf centres.

__device__ __forceinline__ void leaf_centre(uint64_t key, int level, const Geo& g, float* x,
                                            float* y, float* z) {
  const uint32_t h = 1u << (g.D - level);
  *x = centre_coord(g.org[0], compact3(key), h, g.vox);
  *y = centre_coord(g.org[1], compact3(key >> 1), h, g.vox);
  *z = centre_coord(g.org[2], compact3(key >> 2), h, g.vox);
}

__global__ void __launch_bounds__(256) k_leaf_count(const uint64_t* __restrict__ key,
                                                    const uint8_t* __restrict__ level,
                                                    const uint32_t* __restrict__ list,
                                                    const unsigned long long* __restrict__ nlist,
                                                    int64_t n,
                                                    const float* __restrict__ depth,
                                                    const Cam* __restrict__ cams, int F, int H,
                                                    int W, Geo g, FrameTrees tr,
                                                    uint32_t* __restrict__ count) {
  extern __shared__ float4 smem_dyn[];
  Cam* sc = reinterpret_cast<Cam*>(smem_dyn);
  stage_cams(sc, cams, F);
  if (nlist) n = int64_t(*nlist);
  const int warp = threadIdx.x >> 5, lane = lane_id();
  for (int64_t j = int64_t(blockIdx.x) * kWarpsPerBlock + warp; j < n;
       j += int64_t(gridDim.x) * kWarpsPerBlock) {
    const int64_t l = list ? int64_t(list[j]) : j;
    const uint64_t kl = key[l];
    const int lv = level[l];
    float x, y, z;
    leaf_centre(kl, lv, g, &x, &y, &z);
    int cnt = 0;
    for (int i = lane; i < F; i += 32) {
      float t;
      cnt += tr.key ? tree_sample(tr, i, kl, lv, g.D, &t)
                    : eq1_sample(sc[i], depth + size_t(i) * H * W, H, W, x, y, z, g.delta, g.eta, &t);
    }
    cnt = warp_sum_i(cnt);
    if (lane == 0) count[l] = uint32_t(cnt);
  }
}

template <int P, typename T>
__global__ void __launch_bounds__(256) k_leaf_fill(
    const uint64_t* __restrict__ key, const uint8_t* __restrict__ level,
    const uint32_t* __restrict__ list, const unsigned long long* __restrict__ nlist, int64_t n,
    const float* __restrict__ depth,
    const Cam* __restrict__ cams, int F, int H, int W, Geo g, FrameTrees tr,
    const uint32_t* __restrict__ soff, T* __restrict__ samp, float* __restrict__ u,
    float* __restrict__ ubar) {
  extern __shared__ float4 smem_dyn[];
  Cam* sc = reinterpret_cast<Cam*>(smem_dyn);
  float* bufs = reinterpret_cast<float*>(sc + F);
  stage_cams(sc, cams, F);
  if (nlist) n = int64_t(*nlist);
  const int warp = threadIdx.x >> 5, lane = lane_id();
  float* a = bufs + warp * P;
  for (int64_t j = int64_t(blockIdx.x) * kWarpsPerBlock + warp; j < n;
       j += int64_t(gridDim.x) * kWarpsPerBlock) {
    const int64_t l = list ? int64_t(list[j]) : j;
    const uint64_t kl = key[l];
    const int lv = level[l];
    float x, y, z;
    leaf_centre(kl, lv, g, &x, &y, &z);
    float mn, mx;
    const int cnt = warp_samples_of<P>(
        [&](int i, float* t) {
          return tr.key ? tree_sample(tr, i, kl, lv, g.D, t)
                        : eq1_sample(sc[i], depth + size_t(i) * H * W, H, W, x, y, z, g.delta,
                                     g.eta, t);
        },
        F, a, &mn, &mx);
    __syncwarp();
    // equal observed samples (e.g. all saturated) need no sort; the others are
    // sorted with the unobserved (+inf) entries last
    const bool flat = cnt > 0 && mn == mx;
    if (!flat && cnt > 1) warp_bitonic<P>(a);
    const uint32_t o = soff[l];
    for (int k = lane; k < cnt; k += 32) {
      const float fv = flat ? mn : a[k];
      if constexpr (sizeof(T) == 2)
        samp[o + k] = __float2half_rn(fv);
      else
        samp[o + k] = fv;
    }
    if (u != nullptr && lane == 0) {
      float lo = 0.0f, hi = 0.0f;
      if (cnt > 0) {
        lo = flat ? mn : a[(cnt - 1) / 2];
        hi = flat ? mn : a[cnt / 2];
      }
      if constexpr (sizeof(T) == 2) {
        // median of the stored (rounded) samples
        lo = __half2float(__float2half_rn(lo));
        hi = __half2float(__float2half_rn(hi));
      }
      const double med = cnt == 0 ? -1.0 : (cnt & 1 ? double(lo) : (double(lo) + double(hi)) * 0.5);
      u[l] = float(med);
      ubar[l] = float(med);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Voxel map: for every finest voxel (Morton order) the index of the leaf that
// contains it.  Leaves cover contiguous key ranges [key, key + h^3), so the
// map turns "which leaf holds this point" into one load.  Small leaves are
// written by one thread each, larger ones by a block each.

constexpr uint32_t kSmallFill = 64;

// Leaves of more voxels than this are written by the whole grid together
// (a few coarse leaves can hold a third of the map).
constexpr uint64_t kHugeFill = uint64_t(1) << 18;

// nbig[0] counts the queued big leaves (from the front of `big`), nbig[1]
// the huge ones (from the back).
__global__ void k_map_small(const uint64_t* __restrict__ key, const uint8_t* __restrict__ level,
                            int64_t n, int D, uint32_t* __restrict__ map, uint32_t* __restrict__ big,
                            unsigned long long* __restrict__ nbig) {
  const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l >= n) return;
  const uint64_t k = key[l];
  const uint64_t h3 = uint64_t(1) << (3 * (D - level[l]));
  if (h3 <= kSmallFill) {
    if (h3 >= 4) {
      const uint4 w = make_uint4(uint32_t(l), uint32_t(l), uint32_t(l), uint32_t(l));
      uint4* m4 = reinterpret_cast<uint4*>(map + k);
      for (uint64_t j = 0; j < h3 / 4; ++j) m4[j] = w;
    } else {
      map[k] = uint32_t(l);
    }
  } else if (h3 > kHugeFill) {
    big[n - 1 - int64_t(atomicAdd(nbig + 1, 1ull))] = uint32_t(l);
  } else {
    big[atomicAdd(nbig, 1ull)] = uint32_t(l);
  }
}

// The huge leaves, each striped over every thread of the grid.
__global__ void k_map_huge(const uint64_t* __restrict__ key, const uint8_t* __restrict__ level,
                           const uint32_t* __restrict__ big, int64_t n,
                           const unsigned long long* __restrict__ nbig, int D,
                           uint32_t* __restrict__ map) {
  const unsigned long long nh = nbig[1];
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (unsigned long long b = 0; b < nh; ++b) {
    const uint32_t l = big[n - 1 - int64_t(b)];
    const uint64_t h34 = (uint64_t(1) << (3 * (D - level[l]))) / 4;
    const uint4 w = make_uint4(l, l, l, l);
    uint4* m4 = reinterpret_cast<uint4*>(map + key[l]);
    for (uint64_t j = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < h34; j += stride) m4[j] = w;
  }
}

__global__ void k_map_big(const uint64_t* __restrict__ key, const uint8_t* __restrict__ level,
                          const uint32_t* __restrict__ big, const unsigned long long* __restrict__ nbig,
                          int D, uint32_t* __restrict__ map) {
  // blockIdx.y walks the queued leaves, blockIdx.x the 4096-voxel chunks of one
  const unsigned long long nb = *nbig;
  for (unsigned long long b = blockIdx.y; b < nb; b += gridDim.y) {
    const uint32_t l = big[b];
    const uint64_t k = key[l];
    const uint64_t h34 = (uint64_t(1) << (3 * (D - level[l]))) / 4;
    const uint4 w = make_uint4(l, l, l, l);
    uint4* m4 = reinterpret_cast<uint4*>(map + k);
    for (uint64_t c = uint64_t(blockIdx.x) * 1024; c < h34; c += uint64_t(gridDim.x) * 1024)
      for (uint64_t j = c + threadIdx.x; j < c + 1024 && j < h34; j += blockDim.x) m4[j] = w;
  }
}

struct FaceHit {
  int kind;  // 0 empty, 1 single, 2 finer list
  uint32_t m;
  int mlev;
};

__device__ __forceinline__ FaceHit face_query(const View& v, int64_t l, int face) {
  FaceHit r;
  r.kind = 0;
  const uint64_t k = v.key[l];
  const int lev = v.level[l];
  const int64_t h = int64_t(1) << (v.D - lev);
  const int64_t n1 = int64_t(1) << v.D;
  int64_t c[3] = {int64_t(compact3(k)), int64_t(compact3(k >> 1)), int64_t(compact3(k >> 2))};
  const int axis = face % 3;
  c[axis] += face < 3 ? h : -h;
  if (c[axis] < 0 || c[axis] >= n1) return r;
  r.m = v.map[morton(uint32_t(c[0]), uint32_t(c[1]), uint32_t(c[2]))];
  r.mlev = v.level[r.m];
  r.kind = r.mlev <= lev ? 1 : 2;
  return r;
}

// Finer neighbours across a face.  The finest voxels just outside the face
// form an h x h square; leaf m touching the face is listed once, at the face
// voxel matching m's corner in the two tangential axes.  Enumerating the
// square in 2-D Morton order of the tangential coordinates (lower axis index
// = lower bit) yields the leaves in ascending key order: along the path to
// every such leaf the bit of the face axis is the same at each level (all on
// one side of the neighbour cube), so keys compare by the tangential bits.
struct FaceSquare {
  int t1, t2;          // tangential axes, t1 < t2
  uint32_t c1, c2;     // corner of the square on t1, t2
  uint32_t cax;        // the face voxels' coordinate on the face axis
  int axis;
  uint32_t h;          // square edge
};

__device__ __forceinline__ FaceSquare face_square(const View& v, int64_t l, int face) {
  FaceSquare q;
  const uint64_t k = v.key[l];
  const uint32_t c[3] = {compact3(k), compact3(k >> 1), compact3(k >> 2)};
  q.h = 1u << (v.D - v.level[l]);
  q.axis = face % 3;
  q.t1 = q.axis == 0 ? 1 : 0;
  q.t2 = q.axis == 2 ? 1 : 2;
  q.c1 = c[q.t1];
  q.c2 = c[q.t2];
  q.cax = face < 3 ? c[q.axis] + q.h : c[q.axis] - 1;
  return q;
}

__device__ __forceinline__ uint32_t even_bits(uint32_t x) {
  x &= 0x55555555u;
  x = (x | (x >> 1)) & 0x33333333u;
  x = (x | (x >> 2)) & 0x0f0f0f0fu;
  x = (x | (x >> 4)) & 0x00ff00ffu;
  x = (x | (x >> 8)) & 0x0000ffffu;
  return x;
}

// Leaf listed at face voxel i (2-D Morton index), or -1.  For a square of
// edge 2 the (subdivided) neighbour cube's children are finest voxels, so
// every face voxel is its own leaf and no key check is needed.
__device__ __forceinline__ int64_t face_rep(const View& v, const FaceSquare& q, uint32_t i) {
  const uint32_t a = q.c1 + even_bits(i), b = q.c2 + even_bits(i >> 1);
  uint32_t c[3];
  c[q.axis] = q.cax;
  c[q.t1] = a;
  c[q.t2] = b;
  const uint32_t m = v.map[morton(c[0], c[1], c[2])];
  if (q.h == 2) return int64_t(m);
  const uint64_t km = v.key[m];
  return (compact3(km >> q.t1) == a && compact3(km >> q.t2) == b) ? int64_t(m) : -1;
}

// Lists of squares up to kThreadSquare voxels are walked by one thread;
// larger ones by a block (k_nbr_long_*).
constexpr uint32_t kThreadSquare = 16;

// Entry of a face whose finer-neighbour list is not yet written, and of one
// whose list is carried over from the structure before a split/join pass.
constexpr int32_t kListPending = int32_t(0x80000000u | 0x7ffffffeu);
constexpr int32_t kCarryPending = int32_t(0x80000000u | 0x7ffffffdu);
// Queue bit of a long list that may be carried; aux values of such a list
// when it is not carried (searched again) or no longer a list.
constexpr uint32_t kCarryBit = 0x80000000u;
constexpr uint32_t kSearch = 0xffffffffu;
constexpr uint32_t kNotList = 0xfffffffeu;

// Face `face` of leaf l (t = face * n + l): an entry carried from the old
// structure, a single neighbour or a boundary is final here; a finer list is
// counted (a small square or a short carried list by this thread, larger ones
// queued for a block) and marked pending for the fill pass.  With a carry,
// cy.full[t] = 1 when the face was carried here.  Returns whether the entry
// is pending.
__device__ __forceinline__ bool count_face(const View& v, const Carry& cy, int64_t t,
                                           int32_t* __restrict__ nbr,
                                           uint32_t* __restrict__ ovf_count,
                                           uint32_t* __restrict__ longq,
                                           unsigned long long* __restrict__ nlong) {
  const int face = int(t / v.n);
  const int64_t l = t - int64_t(face) * v.n;
  const int64_t slot = int64_t(face) * v.stride + l;
  if (cy.nbr) {
    const int32_t s = cy.src[l];
    uint8_t carried = 0;
    if (s >= 0) {
      const int32_t eo = cy.nbr[int64_t(face) * cy.stride + s];
      if (eo == kEmpty) {  // the domain boundary does not move
        nbr[slot] = kEmpty;
        ovf_count[t] = 0;
        carried = 1;
      } else if (is_single(eo)) {
        const int32_t m = cy.fwd[entry_idx(eo)];
        if (m >= 0) {
          nbr[slot] = make_single(uint32_t(m), entry_level(eo));
          ovf_count[t] = 0;
          carried = 1;
        }
      } else {
        const uint32_t so = list_start(eo);
        const uint32_t c = uint32_t(cy.ovf[so]);
        if (c > kThreadSquare) {
          nbr[slot] = kListPending;
          ovf_count[t] = 1;  // k_nbr_long_count decides
          longq[atomicAdd(nlong, 1ull)] = uint32_t(t) | kCarryBit;
          cy.full[t] = 0;
          return true;
        }
        bool all = true;
        for (uint32_t k = 0; k < c; ++k) all &= cy.fwd[entry_idx(cy.ovf[so + 1 + k])] >= 0;
        if (all) {
          nbr[slot] = kCarryPending;
          cy.aux[t] = so;
          ovf_count[t] = 1 + c;
          cy.full[t] = 1;
          return true;
        }
      }
    }
    cy.full[t] = carried;
    if (carried) return false;
  }
  const FaceHit f = face_query(v, l, face);
  int32_t e = kEmpty;
  uint32_t cnt = 0;
  if (f.kind == 1) {
    e = make_single(f.m, f.mlev);
  } else if (f.kind == 2) {
    e = kListPending;
    const FaceSquare q = face_square(v, l, face);
    cnt = 1;
    if (q.h * q.h > kThreadSquare) {
      longq[atomicAdd(nlong, 1ull)] = uint32_t(t);   // k_nbr_long_count adds the leaves
    } else {
#pragma unroll 4
      for (uint32_t i = 0; i < q.h * q.h; ++i) cnt += face_rep(v, q, i) >= 0;
    }
  }
  nbr[slot] = e;
  ovf_count[t] = cnt;
  return f.kind == 2;
}

// One thread per (leaf, face) (count_face); the pending slots are appended to
// pendq, one atomic per warp (every lane reaches the ballot: the grid is whole
// warps and nothing returns early), so the fill pass visits only them.
__global__ void k_nbr_count(View v, Carry cy, int32_t* __restrict__ nbr,
                            uint32_t* __restrict__ ovf_count, uint32_t* __restrict__ longq,
                            unsigned long long* __restrict__ nlong, uint32_t* __restrict__ pendq,
                            unsigned long long* __restrict__ npend) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool pend = t < 6 * v.n && count_face(v, cy, t, nbr, ovf_count, longq, nlong);
  const unsigned bal = __ballot_sync(kFull, pend);
  if (bal) {
    const int lane = lane_id();
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(npend, static_cast<unsigned long long>(__popc(bal)));
    base = __shfl_sync(kFull, base, 0);
    if (pend) pendq[base + __popc(bal & ((1u << lane) - 1))] = uint32_t(t);
  }
}

// Pending slots only: writes the finer-neighbour lists of small squares and
// short carried lists and points each pending entry at its list (a long list
// gets only its pointer here; a long carry candidate that turned out single
// is no longer pending and is skipped).
__global__ void k_nbr_fill(View v, Carry cy, const uint32_t* __restrict__ ovf_off,
                           int32_t* __restrict__ nbr, int32_t* __restrict__ ovf,
                           const uint32_t* __restrict__ pendq,
                           const unsigned long long* __restrict__ npend) {
  const int64_t np = int64_t(*npend);
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < np;
       j += int64_t(gridDim.x) * blockDim.x) {
    const int64_t t = pendq[j];
    const int face = int(t / v.n);
    const int64_t l = t - int64_t(face) * v.n;
    const int64_t slot = int64_t(face) * v.stride + l;
    const int32_t e = nbr[slot];
    if (e != kListPending && e != kCarryPending) continue;
    const uint32_t st = ovf_off[t];
    if (e == kCarryPending) {
      const uint32_t so = cy.aux[t];
      const int32_t c = cy.ovf[so];
      for (int32_t k = 0; k < c; ++k) {
        const int32_t eo = cy.ovf[so + 1 + k];
        ovf[st + 1 + k] = make_single(uint32_t(cy.fwd[entry_idx(eo)]), entry_level(eo));
      }
      ovf[st] = c;
    } else {
      const FaceSquare q = face_square(v, l, face);
      if (q.h * q.h <= kThreadSquare) {
        uint32_t c = 0;
#pragma unroll 4
        for (uint32_t i = 0; i < q.h * q.h; ++i) {
          const int64_t m = face_rep(v, q, i);
          if (m >= 0) ovf[st + 1 + c++] = make_single(uint32_t(m), v.level[m]);
        }
        ovf[st] = int32_t(c);
      }
    }
    nbr[slot] = make_list(st);
  }
}

// Block-wide ordered walk of a face square: calls emit(position, leaf) for
// each listed leaf in ascending order; returns the count in every thread.
template <typename Emit>
__device__ uint32_t block_face_walk(const View& v, const FaceSquare& q, Emit emit) {
  __shared__ uint32_t wsum[8];
  uint32_t base = 0;
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  const uint32_t n = q.h * q.h;
  for (uint32_t i0 = 0; i0 < n; i0 += blockDim.x) {
    const uint32_t i = i0 + threadIdx.x;
    const int64_t m = i < n ? face_rep(v, q, i) : -1;
    const unsigned bal = __ballot_sync(kFull, m >= 0);
    if (lane == 0) wsum[wid] = __popc(bal);
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) {
      before += w < wid ? wsum[w] : 0;
      total += wsum[w];
    }
    if (m >= 0) emit(base + before + __popc(bal & ((1u << lane) - 1)), m);
    base += total;
    __syncthreads();
  }
  return base;
}

// Long lists, a block each.  A carry candidate (a kept leaf whose old entry
// was a long list) keeps its list when every listed leaf was kept; else the
// face is searched again, and if it no longer has finer neighbours its entry
// is written here and its aux slot set to kNotList.
__global__ void k_nbr_long_count(View v, Carry cy, const uint32_t* __restrict__ longq,
                                 const unsigned long long* __restrict__ nlong,
                                 int32_t* __restrict__ nbr, uint32_t* __restrict__ ovf_count) {
  __shared__ int kind_s;
  __shared__ int32_t single_s;
  const unsigned long long nq = *nlong;
  for (unsigned long long j = blockIdx.x; j < nq; j += gridDim.x) {
    const uint32_t qv = longq[j];
    const uint32_t t = qv & ~kCarryBit;
    const int face = int(int64_t(t) / v.n);
    const int64_t l = int64_t(t) - int64_t(face) * v.n;
    if (qv & kCarryBit) {
      const int32_t eo = cy.nbr[int64_t(face) * cy.stride + cy.src[l]];
      const uint32_t so = list_start(eo);
      const uint32_t c = uint32_t(cy.ovf[so]);
      int ok = 1;
      for (uint32_t k = threadIdx.x; k < c; k += blockDim.x)
        ok &= cy.fwd[entry_idx(cy.ovf[so + 1 + k])] >= 0;
      if (__syncthreads_and(ok)) {
        if (threadIdx.x == 0) {
          ovf_count[t] = 1 + c;
          cy.aux[t] = so;
        }
        continue;
      }
      if (threadIdx.x == 0) {
        const FaceHit f = face_query(v, l, face);
        kind_s = f.kind;
        single_s = f.kind == 1 ? make_single(f.m, f.mlev) : kEmpty;
      }
      __syncthreads();
      const int kind = kind_s;
      const int32_t single = single_s;
      __syncthreads();
      if (kind != 2) {
        if (threadIdx.x == 0) {
          nbr[int64_t(face) * v.stride + l] = single;
          ovf_count[t] = 0;
          cy.aux[t] = kNotList;
        }
        continue;
      }
      if (threadIdx.x == 0) cy.aux[t] = kSearch;
    }
    const FaceSquare q = face_square(v, l, face);
    const uint32_t cnt = block_face_walk(v, q, [](uint32_t, int64_t) {});
    if (threadIdx.x == 0) ovf_count[t] = 1 + cnt;
  }
}

__global__ void k_nbr_long_fill(View v, Carry cy, const uint32_t* __restrict__ longq,
                                const unsigned long long* __restrict__ nlong,
                                const uint32_t* __restrict__ ovf_off, int32_t* __restrict__ ovf) {
  const unsigned long long nq = *nlong;
  for (unsigned long long j = blockIdx.x; j < nq; j += gridDim.x) {
    const uint32_t qv = longq[j];
    const uint32_t t = qv & ~kCarryBit;
    const int face = int(int64_t(t) / v.n);
    const int64_t l = int64_t(t) - int64_t(face) * v.n;
    const uint32_t st = ovf_off[t];
    int32_t* out = ovf + st + 1;
    if (qv & kCarryBit) {
      const uint32_t so = cy.aux[t];
      if (so == kNotList) continue;
      if (so != kSearch) {
        const int32_t c = cy.ovf[so];
        for (int32_t k = threadIdx.x; k < c; k += blockDim.x) {
          const int32_t eo = cy.ovf[so + 1 + k];
          out[k] = make_single(uint32_t(cy.fwd[entry_idx(eo)]), entry_level(eo));
        }
        if (threadIdx.x == 0) ovf[st] = c;
        continue;
      }
    }
    const FaceSquare q = face_square(v, l, face);
    const uint32_t cnt = block_face_walk(v, q, [&](uint32_t pos, int64_t m) {
      out[pos] = make_single(uint32_t(m), v.level[m]);
    });
    if (threadIdx.x == 0) ovf[st] = int32_t(cnt);
  }
}

// 2^e as float for -126 <= e <= 127 (exact).
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// sqrt(8^k) = 2^(3k/2): exact for even k, otherwise the float sqrt(2) scaled.
__device__ __forceinline__ float sqrt_pow8f(int k) {
  const int e = 3 * k;
  const float b = pow2f(e >> 1);
  return (e & 1) ? b * 1.41421356237309505f : b;
}

// Diagonal preconditioning (Pock & Chambolle 2011, alpha = 1) of the
// volume-weighted operator: sigma_l = 1 / max over non-empty rows d of
// sum_j |K~_(l,d),j|, tau_l = 1 / sum over rows of |K~_row,l|, where
// K~ = W_p^1/2 K W_u^-1/2.  Entries of K: alpha / Delta with face share
// alpha = min(1, (h_m / h_l)^2) and centre distance Delta = (h_l + h_m) / 2.
// Per-face contribution of one list entry (neighbour level ml) of leaf
// level lev: for +faces the row and diagonal terms, for -faces the column term.
__device__ __forceinline__ void precond_terms(int face, int lev, int ml, float hl, int D,
                                              float* row, float* diag, float* col) {
  const float hm = pow2f(D - ml);
  const float inv_d = 2.0f / (hl + hm);
  if (face < 3) {
    // alpha_lm = min(1, (h_m/h_l)^2); scale sqrt(h_l^3 / h_m^3)
    const float w = (ml > lev ? pow2f(2 * (lev - ml)) : 1.0f) * inv_d;
    *row += w * sqrt_pow8f(ml - lev);
    *diag += w;
  } else {
    // alpha_nl = min(1, (h_l/h_n)^2); scale sqrt(h_n^3 / h_l^3)
    const float w = (ml < lev ? pow2f(2 * (ml - lev)) : 1.0f) * inv_d;
    *col += w * sqrt_pow8f(lev - ml);
  }
}

__device__ __forceinline__ float block_sum_f(float x, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  __syncthreads();
  if (lane_id() == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  float t = 0.0f;
  for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// Diagonal preconditioning (Pock & Chambolle 2011, alpha = 1) of the
// volume-weighted operator: sigma_l = 1 / max over non-empty rows d of
// sum_j |K~_(l,d),j|, tau_l = 1 / sum over rows of |K~_row,l|, where
// K~ = W_p^1/2 K W_u^-1/2.  Entries of K: alpha / Delta with face share
// alpha = min(1, (h_m / h_l)^2) and centre distance Delta = (h_l + h_m) / 2.
// Leaves with a list longer than kHeavy get a block each (the first
// n_heavy blocks); the others a thread.
__global__ void k_precond(View v, Carry cy, float* __restrict__ tau, float* __restrict__ sigma,
                          const uint32_t* __restrict__ heavy, int n_heavy) {
  if (int(blockIdx.x) < n_heavy) {
    __shared__ float red[8];
    const int64_t l = heavy[blockIdx.x];
    const int lev = v.level[l];
    const float hl = pow2f(v.D - lev);
    float rowmax = 0.0f, col = 0.0f;
    for (int face = 0; face < 6; ++face) {
      const int32_t e = v.nbr[int64_t(face) * v.stride + l];
      if (e == kEmpty) continue;
      float row = 0.0f, diag = 0.0f, cl = 0.0f;
      if (is_list(e)) {
        const uint32_t st = list_start(e);
        const int cnt = v.ovf[st];
        for (int k = threadIdx.x; k < cnt; k += blockDim.x)
          precond_terms(face, lev, entry_level(v.ovf[st + 1 + k]), hl, v.D, &row, &diag, &cl);
      } else if (threadIdx.x == 0) {
        precond_terms(face, lev, entry_level(e), hl, v.D, &row, &diag, &cl);
      }
      if (face < 3) {
        const float r = block_sum_f(row, red);
        const float dg = block_sum_f(diag, red);
        rowmax = fmaxf(rowmax, r + dg);
        col += dg;
      } else {
        col += block_sum_f(cl, red);
      }
    }
    if (threadIdx.x == 0) {
      sigma[l] = rowmax > 0.0f ? 1.0f / rowmax : 0.0f;
      tau[l] = col > 0.0f ? 1.0f / col : 1.0f;
    }
    return;
  }
  const int64_t l = int64_t(blockIdx.x - n_heavy) * blockDim.x + threadIdx.x;
  if (l >= v.n) return;
  if (cy.nbr && cy.full[l] & cy.full[v.n + l] & cy.full[2 * v.n + l] & cy.full[3 * v.n + l] &
                    cy.full[4 * v.n + l] & cy.full[5 * v.n + l]) {
    // every face carried: same neighbours and levels as before the pass
    const int32_t s = cy.src[l];
    tau[l] = cy.tau[s];
    sigma[l] = cy.sigma[s];
    return;
  }
  int32_t es[6];
#pragma unroll
  for (int face = 0; face < 6; ++face) es[face] = v.nbr[int64_t(face) * v.stride + l];
  const int lev = v.level[l];
  const float hl = pow2f(v.D - lev);
  float rowmax = 0.0f, col = 0.0f;
#pragma unroll
  for (int face = 0; face < 6; ++face) {
    const int32_t e = es[face];
    if (e == kEmpty) continue;
    float row = 0.0f, diag = 0.0f;
    if (is_list(e)) {
      const uint32_t st = list_start(e);
      const int cnt = v.ovf[st];
      if (cnt > kHeavy) return;   // a heavy block computes this leaf
      for (int k = 0; k < cnt; ++k)
        precond_terms(face, lev, entry_level(v.ovf[st + 1 + k]), hl, v.D, &row, &diag, &col);
    } else {
      precond_terms(face, lev, entry_level(e), hl, v.D, &row, &diag, &col);
    }
    if (face < 3) {
      rowmax = fmaxf(rowmax, row + diag);
      col += diag;
    }
  }
  sigma[l] = rowmax > 0.0f ? 1.0f / rowmax : 0.0f;
  tau[l] = col > 0.0f ? 1.0f / col : 1.0f;
}

// Leaf classes from the list counts of the neighbour pass (1 + list length
// per list face, 0 otherwise), before those counts are scanned: packed flags
// per leaf (bit 0 dual, bit 32 primal) for heavy leaves and for list leaves,
// scanned, then emitted in leaf order, so the sets do not depend on
// scheduling.
__global__ void k_class_flags(View v, const uint32_t* __restrict__ ovf_count,
                              uint64_t* __restrict__ hflags, uint64_t* __restrict__ lflags) {
  const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l >= v.n) return;
  bool hd = false, hp = false, ld = false, lp = false;
  for (int face = 0; face < 6; ++face) {
    const uint32_t c = ovf_count[int64_t(face) * v.n + l];
    if (c > uint32_t(kHeavy) + 1) {
      hp = true;
      if (face < 3) hd = true;
    } else if (c > 0) {
      lp = true;
      if (face < 3) ld = true;
    }
  }
  ld &= !hd;
  lp &= !hp;
  hflags[l] = (hd ? 1ull : 0ull) | (hp ? (1ull << 32) : 0ull);
  lflags[l] = (ld ? 1ull : 0ull) | (lp ? (1ull << 32) : 0ull);
}

__global__ void k_class_emit(int64_t n, const uint64_t* __restrict__ hscan,
                             const uint64_t* __restrict__ lscan, uint32_t* __restrict__ sets,
                             int64_t cap) {
  const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l >= n) return;
  const uint64_t* sc[2] = {hscan, lscan};
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const uint64_t a = sc[k][l], b = sc[k][l + 1];
    if ((b & 0xffffffffull) != (a & 0xffffffffull)) sets[(2 * k) * cap + (a & 0xffffffffull)] = uint32_t(l);
    if ((b >> 32) != (a >> 32)) sets[(2 * k + 1) * cap + (a >> 32)] = uint32_t(l);
  }
}

__global__ void k_check_tiling(const uint64_t* __restrict__ key, const uint8_t* __restrict__ level,
                               int64_t n, int D, uint32_t* __restrict__ bad) {
  const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l >= n) return;
  const int lev = level[l];
  bool ok = lev <= D;
  if (ok) {
    const uint64_t sz = uint64_t(1) << (3 * (D - lev));
    const uint64_t end = l + 1 < n ? key[l + 1] : (uint64_t(1) << (3 * D));
    ok = (key[l] & (sz - 1)) == 0 && key[l] + sz == end && (l > 0 || key[0] == 0);
  }
  if (!ok) atomicAdd(bad, 1u);
}

// ---------------------------------------------------------------------------
// Split / join.

// Packed class counter: bit 32 counts |u| > tau_j positive, bit 0 negative.
__global__ void k_classify(const float* __restrict__ u, int64_t n, double tau_j,
                           uint64_t* __restrict__ cls) {
  const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l >= n) return;
  const double x = double(u[l]);
  cls[l] = (x > tau_j ? (uint64_t(1) << 32) : 0) | (x < -tau_j ? 1u : 0u);
}

// Marks: a leaf joins into the coarsest ancestor whose leaves all carry its
// class (checked finest-first: once an ancestor fails, every coarser one
// fails too), else splits to the finest level when |u| < tau_s, else stays.
// out_count is the number of new leaves it emits (join: 1 for the group's
// first leaf, 0 for the others).
__global__ void k_mark(View v, const float* __restrict__ u, const uint64_t* __restrict__ cscan,
                       double tau_s, double tau_j, uint64_t* __restrict__ out_count,
                       int8_t* __restrict__ join_level, unsigned long long* __restrict__ counters) {
  const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l >= v.n) return;
  const int lev = v.level[l];
  const double x = double(u[l]);
  const int cls = x > tau_j ? 1 : (x < -tau_j ? -1 : 0);
  int jl = -1;
  int64_t jlo = 0;
  if (cls != 0) {
    for (int L = lev - 1; L >= 0; --L) {
      const uint64_t sz = uint64_t(1) << (3 * (v.D - L));
      const uint64_t a = v.key[l] & ~(sz - 1);
      const int64_t lo = v.map[a];
      const int64_t hi = int64_t(v.map[a + sz - 1]) + 1;
      const uint64_t d = cscan[hi] - cscan[lo];
      const uint64_t want = uint64_t(hi - lo);
      const bool ok = cls > 0 ? (d >> 32) == want : (d & 0xffffffffull) == want;
      if (!ok) break;
      jl = L;
      jlo = lo;
    }
  }
  uint64_t oc;
  if (jl >= 0) {
    oc = (jlo == l) ? 1 : 0;
    if (jlo == l) atomicAdd(&counters[1], 1ull);
  } else if (lev < v.D && fabs(x) < tau_s) {
    oc = uint64_t(1) << (3 * (v.D - lev));
    atomicAdd(&counters[0], 1ull);
  } else {
    oc = 1;
  }
  out_count[l] = oc;
  join_level[l] = int8_t(jl);
}

constexpr uint64_t kSmallEmit = 64;
// Joins of more leaves than this are summed by a block (a thread's serial
// FP64 sum over up to kSmallEmit leaves made the pass wait on one thread).
constexpr uint64_t kSmallJoin = 8;

// One thread per old leaf writes the new leaves it produces at its offset:
// kept leaves copy themselves (and record their new index in fwd; -1 for
// every other old leaf), small splits write their finest children
// (inheriting u and p), small joins write the volume-weighted means.  Splits
// of more than kSmallEmit leaves and joins of more than kSmallJoin leaves are
// queued for k_emit_big.
__global__ void k_emit(View v, const float* __restrict__ u, const float* __restrict__ p,
                       const uint64_t* __restrict__ off, const int8_t* __restrict__ join_level,
                       uint64_t* __restrict__ nkey, uint8_t* __restrict__ nlevel,
                       float* __restrict__ nu, float* __restrict__ nubar, float* __restrict__ np_,
                       int64_t nstride, int32_t* __restrict__ src, int32_t* __restrict__ fwd,
                       uint32_t* __restrict__ big, unsigned long long* __restrict__ nbig) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const uint64_t o = off[i];
  const uint64_t oc = off[i + 1] - o;
  const int jl = join_level[i];
  fwd[i] = (oc == 1 && jl < 0) ? int32_t(o) : -1;
  if (oc == 0) return;
  const float ui = u[i];
  const float p0 = p[i], p1 = p[v.stride + i], p2 = p[2 * v.stride + i];
  if (jl >= 0) {
    const uint64_t sz = uint64_t(1) << (3 * (v.D - jl));
    const uint64_t a = v.key[i] & ~(sz - 1);
    const int64_t e = int64_t(v.map[a + sz - 1]) + 1;
    if (uint64_t(e - i) > kSmallJoin) {
      big[atomicAdd(nbig, 1ull)] = uint32_t(i);
      return;
    }
    double su = 0.0, s0 = 0.0, s1 = 0.0, s2 = 0.0, sw = 0.0;
    for (int64_t k = i; k < e; ++k) {
      const double w = double(uint64_t(1) << (3 * (v.D - v.level[k])));
      su += w * double(u[k]);
      s0 += w * double(p[k]);
      s1 += w * double(p[v.stride + k]);
      s2 += w * double(p[2 * v.stride + k]);
      sw += w;
    }
    nkey[o] = a;
    nlevel[o] = uint8_t(jl);
    nu[o] = float(su / sw);
    nubar[o] = float(su / sw);
    np_[o] = float(s0 / sw);
    np_[nstride + o] = float(s1 / sw);
    np_[2 * nstride + o] = float(s2 / sw);
    src[o] = -1;
    return;
  }
  if (oc == 1) {
    nkey[o] = v.key[i];
    nlevel[o] = v.level[i];
    nu[o] = ui;
    nubar[o] = ui;
    np_[o] = p0;
    np_[nstride + o] = p1;
    np_[2 * nstride + o] = p2;
    src[o] = int32_t(i);
    return;
  }
  if (oc > kSmallEmit) {
    big[atomicAdd(nbig, 1ull)] = uint32_t(i);
    return;
  }
  const uint64_t k0 = v.key[i];
  for (uint64_t c = 0; c < oc; ++c) {
    nkey[o + c] = k0 + c;
    nlevel[o + c] = uint8_t(v.D);
    nu[o + c] = ui;
    nubar[o + c] = ui;
    np_[o + c] = p0;
    np_[nstride + o + c] = p1;
    np_[2 * nstride + o + c] = p2;
    src[o + c] = -1;
  }
}

// Block per queued large split or join.
__global__ void k_emit_big(View v, const float* __restrict__ u, const float* __restrict__ p,
                           const uint64_t* __restrict__ off, const int8_t* __restrict__ join_level,
                           uint64_t* __restrict__ nkey, uint8_t* __restrict__ nlevel,
                           float* __restrict__ nu, float* __restrict__ nubar,
                           float* __restrict__ np_, int64_t nstride, int32_t* __restrict__ src,
                           const uint32_t* __restrict__ big,
                           const unsigned long long* __restrict__ nbig) {
  __shared__ double red[5][32];
  const unsigned long long nb = *nbig;
  for (unsigned long long b = blockIdx.x; b < nb; b += gridDim.x) {
    const int64_t i = big[b];
    const uint64_t o = off[i];
    const int jl = join_level[i];
    if (jl >= 0) {
      const uint64_t sz = uint64_t(1) << (3 * (v.D - jl));
      const uint64_t a = v.key[i] & ~(sz - 1);
      const int64_t e = int64_t(v.map[a + sz - 1]) + 1;
      double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      for (int64_t k = i + threadIdx.x; k < e; k += blockDim.x) {
        const double w = double(uint64_t(1) << (3 * (v.D - v.level[k])));
        acc[0] += w * double(u[k]);
        acc[1] += w * double(p[k]);
        acc[2] += w * double(p[v.stride + k]);
        acc[3] += w * double(p[2 * v.stride + k]);
        acc[4] += w;
      }
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        for (int s = 16; s > 0; s >>= 1) acc[q] += __shfl_xor_sync(kFull, acc[q], s);
        if (lane_id() == 0) red[q][threadIdx.x >> 5] = acc[q];
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double t[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < int(blockDim.x >> 5); ++w)
          for (int q = 0; q < 5; ++q) t[q] += red[q][w];
        nkey[o] = a;
        nlevel[o] = uint8_t(jl);
        nu[o] = float(t[0] / t[4]);
        nubar[o] = float(t[0] / t[4]);
        np_[o] = float(t[1] / t[4]);
        np_[nstride + o] = float(t[2] / t[4]);
        np_[2 * nstride + o] = float(t[3] / t[4]);
        src[o] = -1;
      }
      __syncthreads();
    } else {
      const uint64_t oc = off[i + 1] - o;
      const uint64_t k0 = v.key[i];
      const float ui = u[i];
      const float p0 = p[i], p1 = p[v.stride + i], p2 = p[2 * v.stride + i];
      for (uint64_t c = threadIdx.x; c < oc; c += blockDim.x) {
        nkey[o + c] = k0 + c;
        nlevel[o + c] = uint8_t(v.D);
        nu[o + c] = ui;
        nubar[o + c] = ui;
        np_[o + c] = p0;
        np_[nstride + o + c] = p1;
        np_[2 * nstride + o + c] = p2;
        src[o + c] = -1;
      }
    }
  }
}

__global__ void k_new_list(const int32_t* __restrict__ src, int64_t n, uint32_t* __restrict__ list,
                           unsigned long long* __restrict__ cnt) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n || src[j] >= 0) return;
  const unsigned long long k = atomicAdd(cnt, 1ull);
  list[k] = uint32_t(j);
}

__global__ void k_kept_counts(const int32_t* __restrict__ src, const uint32_t* __restrict__ old_soff,
                              int64_t n, uint32_t* __restrict__ count) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int32_t s = src[j];
  if (s >= 0) count[j] = old_soff[s + 1] - old_soff[s];
}

// Samples of kept leaves into the new CSR.  A warp takes 32 consecutive new
// leaves; when they are 32 kept leaves with consecutive sources (the common
// case) their samples are one contiguous run in both arrays and are copied
// coalesced, otherwise each lane copies its own leaf's samples.
template <typename T>
__global__ void k_copy_kept(const int32_t* __restrict__ src, int64_t n,
                            const uint32_t* __restrict__ old_soff, const T* __restrict__ old_samp,
                            const uint32_t* __restrict__ new_soff, T* __restrict__ new_samp) {
  const int warp = threadIdx.x >> 5, lane = lane_id();
  for (int64_t j0 = (int64_t(blockIdx.x) * kWarpsPerBlock + warp) * 32; j0 < n;
       j0 += int64_t(gridDim.x) * kWarpsPerBlock * 32) {
    const int64_t j = j0 + lane;
    const int32_t sj = j < n ? src[j] : -1;
    const int32_t s0 = __shfl_sync(kFull, sj, 0);
    const bool run = __all_sync(kFull, j < n && s0 >= 0 && sj == s0 + lane);
    // four loads in flight before their stores (a store waits for its load)
    if (run) {
      const uint32_t a = old_soff[s0], c = old_soff[s0 + 32] - a, b = new_soff[j0];
      for (uint32_t k0 = lane; k0 < c; k0 += 128) {
        T x[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t k = k0 + 32u * q;
          if (k < c) x[q] = old_samp[a + k];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t k = k0 + 32u * q;
          if (k < c) new_samp[b + k] = x[q];
        }
      }
    } else if (sj >= 0) {
      const uint32_t a = old_soff[sj], c = old_soff[sj + 1] - a, b = new_soff[j];
      for (uint32_t k0 = 0; k0 < c; k0 += 4) {
        T x[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (k0 + q < c) x[q] = old_samp[a + k0 + q];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (k0 + q < c) new_samp[b + k0 + q] = x[q];
      }
    }
  }
}

__global__ void k_widen(const __half* __restrict__ in, int64_t n, float* __restrict__ out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] = __half2float(in[i]);
}

__global__ void k_w_from_soff(const uint32_t* __restrict__ soff, int64_t n, int32_t* __restrict__ out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] = int32_t(soff[i + 1] - soff[i]);
}

inline unsigned blocks_for(int64_t n, int threads) {
  return unsigned((n + threads - 1) / threads);
}

// Grid of warp-per-item kernels: enough blocks to fill the machine, grid-stride beyond.
inline unsigned warp_grid(int64_t items) {
  const int64_t want = (items + kWarpsPerBlock - 1) / kWarpsPerBlock;
  const int64_t cap = int64_t(sm_count()) * 16;
  return unsigned(want < 1 ? 1 : (want < cap ? want : cap));
}

int pad_frames(int F) {
  int P = 32;
  while (P < F) P <<= 1;
  return P;
}

}  // namespace

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// ---------------------------------------------------------------------------
// launchers

template <typename T>
size_t scan_tmp_items(int64_t n) {
  size_t t = 0;
  int64_t m = n;
  while (m > kTile) {
    m = (m + kTile - 1) / kTile;
    t += size_t(m) + 1;
  }
  return t + 1;
}

template <typename T>
cudaError_t scan_exclusive(const T* in, T* out, int64_t n, T* tmp, cudaStream_t s) {
  if (n <= kTile) {
    k_tile_scan<T><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, 0);
    count_launches(1);
    return cudaGetLastError();
  }
  const int64_t nb = (n + kTile - 1) / kTile;
  k_tile_sums<T><<<unsigned(nb), kScanThreads, 0, s>>>(in, n, tmp);
  count_launches(1);
  const int self = nb <= kSelfOffsetTiles;
  if (!self) {
    cudaError_t e = scan_exclusive<T>(tmp, tmp, nb, tmp + nb + 1, s);
    if (e != cudaSuccess) return e;
  }
  k_tile_scan<T><<<unsigned(nb), kScanThreads, 0, s>>>(in, out, n, tmp, self);
  count_launches(1);
  return cudaGetLastError();
}

template size_t scan_tmp_items<uint32_t>(int64_t);
template size_t scan_tmp_items<uint64_t>(int64_t);
template cudaError_t scan_exclusive<uint32_t>(const uint32_t*, uint32_t*, int64_t, uint32_t*, cudaStream_t);
template cudaError_t scan_exclusive<uint64_t>(const uint64_t*, uint64_t*, int64_t, uint64_t*, cudaStream_t);
template size_t scan_tmp_items<double>(int64_t);
template cudaError_t scan_exclusive<double>(const double*, double*, int64_t, double*, cudaStream_t);

template <int P>
static cudaError_t dense_u0_p(const float* depth, const Cam* cams, int F, int H, int W, Geo g,
                              RangePyr rp, double* u0, uint32_t* queue,
                              unsigned long long* nqueue, cudaStream_t s) {
  const int64_t nvox = int64_t(1) << (3 * g.D);
  cudaError_t e = cudaMemsetAsync(nqueue, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const size_t sm0 = size_t(F) * sizeof(Cam);
  if (sm0 > 48 * 1024) cudaFuncSetAttribute(k_dense_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm0));
  const int64_t want = (nvox + 255) / 256, cap = int64_t(sm_count()) * 16;
  k_dense_scan<<<unsigned(want < cap ? want : cap), 256, sm0, s>>>(depth, cams, F, H, W, g, rp, nvox,
                                                                 u0, queue, nqueue);
  count_launches(1);
  const size_t sm = sm0 + size_t(kWarpsPerBlock) * P * sizeof(float);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_dense_u0<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  k_dense_u0<P><<<warp_grid(nvox), 32 * kWarpsPerBlock, sm, s>>>(depth, cams, F, H, W, g, queue,
                                                                 nqueue, u0);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_dense_u0(const float* depth, const Cam* cams, int F, int H, int W, Geo g,
                            RangePyr rp, double* u0, uint32_t* queue, unsigned long long* nqueue,
                            cudaStream_t s) {
  switch (pad_frames(F)) {
    case 32: return dense_u0_p<32>(depth, cams, F, H, W, g, rp, u0, queue, nqueue, s);
    case 64: return dense_u0_p<64>(depth, cams, F, H, W, g, rp, u0, queue, nqueue, s);
    case 128: return dense_u0_p<128>(depth, cams, F, H, W, g, rp, u0, queue, nqueue, s);
    case 256: return dense_u0_p<256>(depth, cams, F, H, W, g, rp, u0, queue, nqueue, s);
    case 512: return dense_u0_p<512>(depth, cams, F, H, W, g, rp, u0, queue, nqueue, s);
    default: return cudaErrorInvalidValue;
  }
}

RangePyr range_pyr_dims(int H, int W) {
  RangePyr rp{};
  int w = W, h = H, off = 0, k = 0;
  rp.w[0] = W;
  rp.h[0] = H;
  while ((w > 1 || h > 1) && k < kMaxRangeLevels) {
    ++k;
    w = (w + 1) / 2;
    h = (h + 1) / 2;
    rp.w[k] = w;
    rp.h[k] = h;
    rp.off[k] = off;
    off += w * h;
  }
  rp.nl = k;
  rp.frame_texels = off;
  return rp;
}

cudaError_t launch_range_pyr(const float* range, int F, int H, int W, RangePyr rp, float2* tex,
                             cudaStream_t s) {
  if (rp.nl < 1) return cudaSuccess;
  k_rpyr_base<<<blocks_for(int64_t(F) * rp.w[1] * rp.h[1], 256), 256, 0, s>>>(range, F, H, W, rp, tex);
  count_launches(1);
  for (int k = 2; k <= rp.nl; ++k) {
    k_rpyr_up<<<blocks_for(int64_t(F) * rp.w[k] * rp.h[k], 256), 256, 0, s>>>(F, k, rp, tex);
    count_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_range_map(float* depth, const Cam* cams, int F, int H, int W, cudaStream_t s) {
  const int64_t n = int64_t(F) * H * W;
  k_range_map<<<blocks_for(n, 256), 256, 0, s>>>(depth, cams, F, H, W);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_pyramid(const double* u0, int D, double* mn, double* mx, cudaStream_t s) {
  // level D-1 from the voxels, then upwards
  int64_t nn = int64_t(1) << (3 * (D - 1));
  k_pyr_base<<<blocks_for(nn, 256), 256, 0, s>>>(u0, nn, mn + lev_off(D - 1), mx + lev_off(D - 1));
  count_launches(1);
  for (int L = D - 2; L >= 0; --L) {
    nn = int64_t(1) << (3 * L);
    k_pyr_up<<<blocks_for(nn, 256), 256, 0, s>>>(mn + lev_off(L + 1), mx + lev_off(L + 1), nn,
                                                  mn + lev_off(L), mx + lev_off(L));
    count_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_leaf_flags(const double* mn, const double* mx, int D, double spread_tau,
                              uint32_t* flags, cudaStream_t s) {
  const int64_t nvox = int64_t(1) << (3 * D);
  k_leaf_flags<<<blocks_for(nvox, 256), 256, 0, s>>>(mn, mx, D, spread_tau, nvox, flags);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_emit_constructed(const uint32_t* flags, const uint32_t* pos, const double* mn,
                                    const double* mx, int D, double spread_tau, uint64_t* key,
                                    uint8_t* level, cudaStream_t s) {
  const int64_t nvox = int64_t(1) << (3 * D);
  k_emit_constructed<<<blocks_for(nvox, 256), 256, 0, s>>>(flags, pos, mn, mx, D, spread_tau,
                                                           nvox, key, level);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_leaf_count(const uint64_t* key, const uint8_t* level, const uint32_t* list,
                              const unsigned long long* nlist, int64_t n, const float* depth,
                              const Cam* cams, int F, int H, int W, Geo g, FrameTrees tr,
                              uint32_t* count, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t sm = size_t(F) * sizeof(Cam);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_leaf_count, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  k_leaf_count<<<warp_grid(n), 32 * kWarpsPerBlock, sm, s>>>(key, level, list, nlist, n, depth,
                                                              cams, F, H, W, g, tr, count);
  count_launches(1);
  return cudaGetLastError();
}

template <int P, typename T>
static cudaError_t leaf_fill_p(const uint64_t* key, const uint8_t* level, const uint32_t* list,
                               const unsigned long long* nlist, int64_t n, const float* depth,
                               const Cam* cams, int F, int H, int W, Geo g, FrameTrees tr,
                               const uint32_t* soff, void* samp, float* u, float* ubar,
                               cudaStream_t s) {
  const size_t sm = size_t(F) * sizeof(Cam) + size_t(kWarpsPerBlock) * P * sizeof(float);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_leaf_fill<P, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  k_leaf_fill<P, T><<<warp_grid(n), 32 * kWarpsPerBlock, sm, s>>>(
      key, level, list, nlist, n, depth, cams, F, H, W, g, tr, soff, reinterpret_cast<T*>(samp), u, ubar);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t leaf_fill_t(const uint64_t* key, const uint8_t* level, const uint32_t* list,
                               const unsigned long long* nlist, int64_t n, const float* depth,
                               const Cam* cams, int F, int H, int W, Geo g, FrameTrees tr,
                               const uint32_t* soff, void* samp, float* u, float* ubar,
                               cudaStream_t s) {
  switch (pad_frames(F)) {
    case 32: return leaf_fill_p<32, T>(key, level, list, nlist, n, depth, cams, F, H, W, g, tr, soff, samp, u, ubar, s);
    case 64: return leaf_fill_p<64, T>(key, level, list, nlist, n, depth, cams, F, H, W, g, tr, soff, samp, u, ubar, s);
    case 128: return leaf_fill_p<128, T>(key, level, list, nlist, n, depth, cams, F, H, W, g, tr, soff, samp, u, ubar, s);
    case 256: return leaf_fill_p<256, T>(key, level, list, nlist, n, depth, cams, F, H, W, g, tr, soff, samp, u, ubar, s);
    case 512: return leaf_fill_p<512, T>(key, level, list, nlist, n, depth, cams, F, H, W, g, tr, soff, samp, u, ubar, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_leaf_fill(const uint64_t* key, const uint8_t* level, const uint32_t* list,
                             const unsigned long long* nlist, int64_t n, const float* depth,
                             const Cam* cams, int F, int H, int W, Geo g, FrameTrees tr,
                             const uint32_t* soff, void* samp, bool fp16, float* u, float* ubar,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  return fp16 ? leaf_fill_t<__half>(key, level, list, nlist, n, depth, cams, F, H, W, g, tr, soff, samp, u, ubar, s)
              : leaf_fill_t<float>(key, level, list, nlist, n, depth, cams, F, H, W, g, tr, soff, samp, u, ubar, s);
}

cudaError_t launch_nbr_count(View v, Carry cy, int32_t* nbr, uint32_t* ovf_count, uint32_t* longq,
                             unsigned long long* nlong, uint32_t* pendq, unsigned long long* npend,
                             cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(nlong, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(npend, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_nbr_count<<<blocks_for(6 * v.n, 256), 256, 0, s>>>(v, cy, nbr, ovf_count, longq, nlong, pendq,
                                                       npend);
  count_launches(1);
  k_nbr_long_count<<<unsigned(sm_count() * 8), 256, 0, s>>>(v, cy, longq, nlong, nbr, ovf_count);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_nbr_fill(View v, Carry cy, const uint32_t* ovf_off, int32_t* nbr, int32_t* ovf,
                            const uint32_t* longq, const unsigned long long* nlong,
                            const uint32_t* pendq, const unsigned long long* npend,
                            cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  const int64_t want = blocks_for(6 * v.n, 256), cap = int64_t(sm_count()) * 8;
  k_nbr_fill<<<unsigned(want < cap ? want : cap), 256, 0, s>>>(v, cy, ovf_off, nbr, ovf, pendq, npend);
  count_launches(1);
  k_nbr_long_fill<<<unsigned(sm_count() * 8), 256, 0, s>>>(v, cy, longq, nlong, ovf_off, ovf);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_precond(View v, Carry cy, float* tau, float* sigma, const uint32_t* heavy,
                           int n_heavy, cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  k_precond<<<blocks_for(v.n, 256) + n_heavy, 256, 0, s>>>(v, cy, tau, sigma, heavy, n_heavy);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_leaf_sets(View v, const uint32_t* ovf_count, uint64_t* hflags,
                             uint64_t* lflags, uint64_t* tmp, uint32_t* sets, int64_t cap,
                             cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  k_class_flags<<<blocks_for(v.n, 256), 256, 0, s>>>(v, ovf_count, hflags, lflags);
  count_launches(1);
  cudaError_t e = scan_exclusive<uint64_t>(hflags, hflags, v.n, tmp, s);
  if (e == cudaSuccess) e = scan_exclusive<uint64_t>(lflags, lflags, v.n, tmp, s);
  if (e != cudaSuccess) return e;
  k_class_emit<<<blocks_for(v.n, 256), 256, 0, s>>>(v.n, hflags, lflags, sets, cap);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_check_tiling(const uint64_t* key, const uint8_t* level, int64_t n, int D,
                                uint32_t* bad, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_check_tiling<<<blocks_for(n, 256), 256, 0, s>>>(key, level, n, D, bad);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_classify(const float* u, int64_t n, double tau_j, uint64_t* cls,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_classify<<<blocks_for(n, 256), 256, 0, s>>>(u, n, tau_j, cls);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mark(View v, const float* u, const uint64_t* cls_scan, double tau_s,
                        double tau_j, uint64_t* out_count, int8_t* join_level,
                        unsigned long long* counters, cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  k_mark<<<blocks_for(v.n, 256), 256, 0, s>>>(v, u, cls_scan, tau_s, tau_j, out_count, join_level,
                                               counters);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_emit(View v, const float* u, const float* p, const uint64_t* out_off,
                        const int8_t* join_level, uint64_t* nkey, uint8_t* nlevel, float* nu,
                        float* nubar, float* np_, int64_t nstride, int32_t* src, int32_t* fwd,
                        uint32_t* big, unsigned long long* nbig, cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(nbig, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_emit<<<blocks_for(v.n, 256), 256, 0, s>>>(v, u, p, out_off, join_level, nkey, nlevel, nu, nubar,
                                              np_, nstride, src, fwd, big, nbig);
  count_launches(1);
  k_emit_big<<<unsigned(sm_count() * 2), 256, 0, s>>>(v, u, p, out_off, join_level, nkey, nlevel,
                                                      nu, nubar, np_, nstride, src, big, nbig);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_map(const uint64_t* key, const uint8_t* level, int64_t n, int D, uint32_t* map,
                       uint32_t* big, unsigned long long* nbig, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(nbig, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_map_small<<<blocks_for(n, 256), 256, 0, s>>>(key, level, n, D, map, big, nbig);
  count_launches(1);
  k_map_big<<<dim3(16, unsigned(sm_count() * 2)), 256, 0, s>>>(key, level, big, nbig, D, map);
  count_launches(1);
  k_map_huge<<<unsigned(sm_count() * 4), 256, 0, s>>>(key, level, big, n, nbig, D, map);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_new_list(const int32_t* src, int64_t n, uint32_t* list,
                            unsigned long long* cnt, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_new_list<<<blocks_for(n, 256), 256, 0, s>>>(src, n, list, cnt);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_kept_counts(const int32_t* src, const uint32_t* old_soff, int64_t n,
                               uint32_t* count, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_kept_counts<<<blocks_for(n, 256), 256, 0, s>>>(src, old_soff, n, count);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_copy_kept_samples(const int32_t* src, int64_t n, const uint32_t* old_soff,
                                     const void* old_samp, const uint32_t* new_soff,
                                     void* new_samp, bool fp16, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (fp16)
    k_copy_kept<__half><<<warp_grid((n + 31) / 32), 32 * kWarpsPerBlock, 0, s>>>(
        src, n, old_soff, reinterpret_cast<const __half*>(old_samp), new_soff,
        reinterpret_cast<__half*>(new_samp));
  else
    k_copy_kept<float><<<warp_grid((n + 31) / 32), 32 * kWarpsPerBlock, 0, s>>>(
        src, n, old_soff, reinterpret_cast<const float*>(old_samp), new_soff,
        reinterpret_cast<float*>(new_samp));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_widen_samples(const void* samp, bool fp16, int64_t n, float* out,
                                 cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (!fp16) return cudaMemcpyAsync(out, samp, size_t(n) * 4, cudaMemcpyDefault, s);
  k_widen<<<blocks_for(n, 256), 256, 0, s>>>(reinterpret_cast<const __half*>(samp), n, out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_w_from_soff(const uint32_t* soff, int64_t n, int32_t* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_w_from_soff<<<blocks_for(n, 256), 256, 0, s>>>(soff, n, out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace ofu
