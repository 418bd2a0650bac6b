// Structure kernels: prefix sums, Eq. 1 integration, Eq. 2 construction,
// face neighbours, step sizes and the split/join pass (Sec. 3.1-3.2).
#include <math_constants.h>

#include "ofu_internal.cuh"

namespace ofu {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// ---------------------------------------------------------------------------
// Prefix sums: tiles of kTile items; one pass of tile totals, a recursive
// exclusive scan of the totals, then a pass that scans each tile in shared
// memory and adds its tile offset.

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kTile = kScanThreads * kScanItems;

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

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_tile_scan(const T* in, T* out, int64_t n,
                                                            const T* __restrict__ offs) {
  __shared__ T tile[kTile];
  const int64_t base = int64_t(blockIdx.x) * kTile;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int idx = k * kScanThreads + threadIdx.x;
    const int64_t i = base + idx;
    tile[idx] = i < n ? in[i] : T(0);
  }
  __syncthreads();
  T loc[kScanItems];
  T s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    loc[k] = tile[threadIdx.x * kScanItems + k];
    s += loc[k];
  }
  T tot;
  T run = block_exclusive(s, &tot);
  const T off = offs ? offs[blockIdx.x] : T(0);
  run += off;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    tile[threadIdx.x * kScanItems + k] = run;
    run += loc[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int idx = k * kScanThreads + threadIdx.x;
    const int64_t i = base + idx;
    if (i < n) out[i] = tile[idx];
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
// returns W and the min / max of the observed samples.
template <int P>
__device__ __forceinline__ int warp_samples(const Cam* sc, const float* depth, int F, int H, int W,
                                            float x, float y, float z, float delta, float eta,
                                            float* a, float* mn, float* mx) {
  const int lane = lane_id();
  int cnt = 0;
  float lo = CUDART_INF_F, hi = -CUDART_INF_F;
#pragma unroll 4
  for (int i = lane; i < P; i += 32) {
    float f = CUDART_INF_F;
    if (i < F) {
      float t;
      if (eq1_sample(sc[i], depth + size_t(i) * H * W, H, W, x, y, z, delta, eta, &t)) {
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

template <int P>
__global__ void __launch_bounds__(256) k_dense_u0(const float* __restrict__ depth,
                                                  const Cam* __restrict__ cams, int F, int H,
                                                  int W, Geo g, int64_t nvox,
                                                  double* __restrict__ u0) {
  extern __shared__ float4 smem_dyn[];
  Cam* sc = reinterpret_cast<Cam*>(smem_dyn);
  float* bufs = reinterpret_cast<float*>(sc + F);
  stage_cams(sc, cams, F);
  const int warp = threadIdx.x >> 5;
  float* a = bufs + warp * P;
  for (int64_t m = int64_t(blockIdx.x) * kWarpsPerBlock + warp; m < nvox;
       m += int64_t(gridDim.x) * kWarpsPerBlock) {
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
                                                    const uint32_t* __restrict__ list, int64_t n,
                                                    const float* __restrict__ depth,
                                                    const Cam* __restrict__ cams, int F, int H,
                                                    int W, Geo g, uint32_t* __restrict__ count) {
  extern __shared__ float4 smem_dyn[];
  Cam* sc = reinterpret_cast<Cam*>(smem_dyn);
  stage_cams(sc, cams, F);
  const int warp = threadIdx.x >> 5, lane = lane_id();
  for (int64_t j = int64_t(blockIdx.x) * kWarpsPerBlock + warp; j < n;
       j += int64_t(gridDim.x) * kWarpsPerBlock) {
    const int64_t l = list ? int64_t(list[j]) : j;
    float x, y, z;
    leaf_centre(key[l], level[l], g, &x, &y, &z);
    int cnt = 0;
    for (int i = lane; i < F; i += 32) {
      float t;
      cnt += eq1_sample(sc[i], depth + size_t(i) * H * W, H, W, x, y, z, g.delta, g.eta, &t);
    }
    cnt = warp_sum_i(cnt);
    if (lane == 0) count[l] = uint32_t(cnt);
  }
}

template <int P, typename T>
__global__ void __launch_bounds__(256) k_leaf_fill(
    const uint64_t* __restrict__ key, const uint8_t* __restrict__ level,
    const uint32_t* __restrict__ list, int64_t n, const float* __restrict__ depth,
    const Cam* __restrict__ cams, int F, int H, int W, Geo g, const uint32_t* __restrict__ soff,
    T* __restrict__ samp, float* __restrict__ u, float* __restrict__ ubar) {
  extern __shared__ float4 smem_dyn[];
  Cam* sc = reinterpret_cast<Cam*>(smem_dyn);
  float* bufs = reinterpret_cast<float*>(sc + F);
  stage_cams(sc, cams, F);
  const int warp = threadIdx.x >> 5, lane = lane_id();
  float* a = bufs + warp * P;
  for (int64_t j = int64_t(blockIdx.x) * kWarpsPerBlock + warp; j < n;
       j += int64_t(gridDim.x) * kWarpsPerBlock) {
    const int64_t l = list ? int64_t(list[j]) : j;
    float x, y, z;
    leaf_centre(key[l], level[l], g, &x, &y, &z);
    float mn, mx;
    const int cnt = warp_samples<P>(sc, depth, F, H, W, x, y, z, g.delta, g.eta, a, &mn, &mx);
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
// Search in the sorted key array: largest i with key[i] <= q, galloping from
// `hint` (neighbours are usually close in Morton order).  key[0] == 0 <= q.

__device__ __forceinline__ int64_t locate(const uint64_t* __restrict__ key, int64_t n, uint64_t q,
                                          int64_t hint) {
  int64_t lo, hi;
  if (key[hint] <= q) {
    lo = hint;
    int64_t step = 1;
    for (;;) {
      const int64_t t = lo + step;
      if (t >= n) { hi = n; break; }
      if (key[t] <= q) { lo = t; step <<= 1; } else { hi = t; break; }
    }
  } else {
    hi = hint;
    int64_t step = 1;
    for (;;) {
      int64_t t = hi - step;
      if (t <= 0) { lo = 0; break; }
      if (key[t] <= q) { lo = t; break; }
      hi = t;
      step <<= 1;
    }
  }
  while (hi - lo > 1) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (key[mid] <= q) lo = mid; else hi = mid;
  }
  return lo;
}

// Finer neighbours across a face, in ascending key order: depth-first walk of
// the same-size neighbour cube restricted to the octants on the face.
// `side` is the bit the face octants have on `axis` (0: the cube's low side).
template <bool WRITE>
__device__ uint32_t finer_face_list(const View& v, uint64_t cube_key, int cube_level, int axis,
                                    int side, int64_t hint, int32_t* out) {
  uint64_t sk[64];
  int8_t sl[64];
  int sp = 0;
  auto push_children = [&](uint64_t k, int L) {
    const uint64_t csz = uint64_t(1) << (3 * (v.D - L - 1));
    for (int c = 7; c >= 0; --c) {
      if (((c >> axis) & 1) != side) continue;
      if (sp < 64) {
        sk[sp] = k + uint64_t(c) * csz;
        sl[sp] = int8_t(L + 1);
        ++sp;
      }
    }
  };
  push_children(cube_key, cube_level);
  uint32_t cnt = 0;
  while (sp > 0) {
    --sp;
    const uint64_t k = sk[sp];
    const int L = sl[sp];
    const int64_t i = locate(v.key, v.n, k, hint);
    hint = i;
    const int li = v.level[i];
    if (li <= L || L >= v.D || sp > 60) {
      if (WRITE) out[cnt] = make_single(uint32_t(i), li);
      ++cnt;
    } else {
      push_children(k, L);
    }
  }
  return cnt;
}

struct FaceHit {
  int kind;  // 0 empty, 1 single, 2 finer list
  int64_t m;
  int mlev;
  uint64_t cube;
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
  const uint64_t q = morton(uint32_t(c[0]), uint32_t(c[1]), uint32_t(c[2]));
  const int64_t m = locate(v.key, v.n, q, l);
  r.m = m;
  r.mlev = v.level[m];
  r.cube = q;
  r.kind = r.mlev <= lev ? 1 : 2;
  return r;
}

__global__ void k_nbr_count(View v, uint32_t* __restrict__ ovf_count) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= 6 * v.n) return;
  const int face = int(t / v.n);
  const int64_t l = t - int64_t(face) * v.n;
  const FaceHit f = face_query(v, l, face);
  uint32_t c = 0;
  if (f.kind == 2)
    c = 1 + finer_face_list<false>(v, f.cube, v.level[l], face % 3, face < 3 ? 0 : 1, f.m, nullptr);
  ovf_count[t] = c;
}

__global__ void k_nbr_fill(View v, const uint32_t* __restrict__ ovf_off, int32_t* __restrict__ nbr,
                           int32_t* __restrict__ ovf) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= 6 * v.n) return;
  const int face = int(t / v.n);
  const int64_t l = t - int64_t(face) * v.n;
  const FaceHit f = face_query(v, l, face);
  int32_t e = kEmpty;
  if (f.kind == 1) {
    e = make_single(uint32_t(f.m), f.mlev);
  } else if (f.kind == 2) {
    const uint32_t st = ovf_off[t];
    const uint32_t cnt = finer_face_list<true>(v, f.cube, v.level[l], face % 3, face < 3 ? 0 : 1,
                                               f.m, ovf + st + 1);
    ovf[st] = int32_t(cnt);
    e = make_list(st);
  }
  nbr[int64_t(face) * v.stride + l] = e;
}

// sqrt(2^(3k)) for integer k, exact up to the rounding of sqrt(2).
__device__ __forceinline__ double sqrt_pow8(int k) {
  const int e = 3 * k;
  const double base = ldexp(1.0, e >> 1);  // floor(e / 2) also for negative e
  return (e & 1) ? base * 1.4142135623730951 : base;
}

// Diagonal preconditioning (Pock & Chambolle 2011, alpha = 1) of the
// volume-weighted operator: sigma_l = 1 / max over non-empty rows d of
// sum_j |K~_(l,d),j|, tau_l = 1 / sum over rows of |K~_row,l|.
__global__ void k_precond(View v, float* __restrict__ tau, float* __restrict__ sigma) {
  const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l >= v.n) return;
  const int lev = v.level[l];
  const double hl = double(int64_t(1) << (v.D - lev));
  double rowmax = 0.0, col = 0.0;
  for (int face = 0; face < 6; ++face) {
    const int32_t e = v.nbr[int64_t(face) * v.stride + l];
    if (e == kEmpty) continue;
    uint32_t cnt = 1;
    const int32_t* lst = &e;
    if (is_list(e)) {
      cnt = uint32_t(v.ovf[list_start(e)]);
      lst = v.ovf + list_start(e) + 1;
    }
    double row = 0.0, diag = 0.0;
    for (uint32_t k = 0; k < cnt; ++k) {
      const int ml = entry_level(lst[k]);
      const double hm = double(int64_t(1) << (v.D - ml));
      const double w = face < 3 ? fmin(1.0, (hm / hl) * (hm / hl)) / ((hl + hm) * 0.5)
                                : fmin(1.0, (hl / hm) * (hl / hm)) / ((hl + hm) * 0.5);
      if (face < 3) {
        row += w * sqrt_pow8(ml - lev);   // sqrt(h_l^3 / h_m^3)
        diag += w;
      } else {
        col += w * sqrt_pow8(lev - ml);   // sqrt(h_n^3 / h_l^3)
      }
    }
    if (face < 3) {
      rowmax = fmax(rowmax, row + diag);
      col += diag;
    }
  }
  sigma[l] = rowmax > 0.0 ? float(1.0 / rowmax) : 0.0f;
  tau[l] = col > 0.0 ? float(1.0 / col) : 1.0f;
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
    // finest ancestor first; a node that fails makes every coarser one fail
    for (int L = lev - 1; L >= 0; --L) {
      const uint64_t sz = uint64_t(1) << (3 * (v.D - L));
      const uint64_t a = v.key[l] & ~(sz - 1);
      const int64_t lo = locate(v.key, v.n, a, l);
      const int64_t hi = locate(v.key, v.n, a + sz - 1, l) + 1;
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

// One thread per new leaf: find its source leaf in the exclusive scan of the
// output counts (the last leaf whose offset is <= j).
__global__ void k_emit(View v, const float* __restrict__ u, const float* __restrict__ p,
                       const uint64_t* __restrict__ off, const int8_t* __restrict__ join_level,
                       int64_t n_new, uint64_t* __restrict__ nkey, uint8_t* __restrict__ nlevel,
                       float* __restrict__ nu, float* __restrict__ nubar, float* __restrict__ np_,
                       int64_t nstride, int32_t* __restrict__ src) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n_new) return;
  int64_t lo = 0, hi = v.n;  // off[lo] <= j < off[hi]
  while (hi - lo > 1) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (off[mid] <= uint64_t(j)) lo = mid; else hi = mid;
  }
  const int64_t i = lo;
  const int jl = join_level[i];
  const int lev = v.level[i];
  if (jl >= 0) {
    const uint64_t sz = uint64_t(1) << (3 * (v.D - jl));
    const uint64_t a = v.key[i] & ~(sz - 1);
    const int64_t e = locate(v.key, v.n, a + sz - 1, i) + 1;
    double su = 0.0, sp[3] = {0.0, 0.0, 0.0}, sw = 0.0;
    for (int64_t k = i; k < e; ++k) {
      const double w = double(uint64_t(1) << (3 * (v.D - v.level[k])));
      su += w * double(u[k]);
      for (int d = 0; d < 3; ++d) sp[d] += w * double(p[int64_t(d) * v.stride + k]);
      sw += w;
    }
    nkey[j] = a;
    nlevel[j] = uint8_t(jl);
    nu[j] = float(su / sw);
    nubar[j] = float(su / sw);
    for (int d = 0; d < 3; ++d) np_[int64_t(d) * nstride + j] = float(sp[d] / sw);
    src[j] = -1;
  } else {
    // a split leaf emits 8^(D - level) > 1 children; a kept one emits 1
    const uint64_t cnt = off[i + 1] - off[i];
    if (cnt > 1) {
      nkey[j] = v.key[i] + (uint64_t(j) - off[i]);
      nlevel[j] = uint8_t(v.D);
      src[j] = -1;
    } else {
      nkey[j] = v.key[i];
      nlevel[j] = uint8_t(lev);
      src[j] = int32_t(i);
    }
    nu[j] = u[i];
    nubar[j] = u[i];
    for (int d = 0; d < 3; ++d) np_[int64_t(d) * nstride + j] = p[int64_t(d) * v.stride + i];
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

template <typename T>
__global__ void k_copy_kept(const int32_t* __restrict__ src, int64_t n,
                            const uint32_t* __restrict__ old_soff, const T* __restrict__ old_samp,
                            const uint32_t* __restrict__ new_soff, T* __restrict__ new_samp) {
  const int warp = threadIdx.x >> 5, lane = lane_id();
  for (int64_t j = int64_t(blockIdx.x) * kWarpsPerBlock + warp; j < n;
       j += int64_t(gridDim.x) * kWarpsPerBlock) {
    const int32_t s = src[j];
    if (s < 0) continue;
    const uint32_t a = old_soff[s], c = old_soff[s + 1] - a, b = new_soff[j];
    for (uint32_t k = lane; k < c; k += 32) new_samp[b + k] = old_samp[a + k];
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
    k_tile_scan<T><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
    count_launches(1);
    return cudaGetLastError();
  }
  const int64_t nb = (n + kTile - 1) / kTile;
  k_tile_sums<T><<<unsigned(nb), kScanThreads, 0, s>>>(in, n, tmp);
  count_launches(1);
  cudaError_t e = scan_exclusive<T>(tmp, tmp, nb, tmp + nb + 1, s);
  if (e != cudaSuccess) return e;
  k_tile_scan<T><<<unsigned(nb), kScanThreads, 0, s>>>(in, out, n, tmp);
  count_launches(1);
  return cudaGetLastError();
}

template size_t scan_tmp_items<uint32_t>(int64_t);
template size_t scan_tmp_items<uint64_t>(int64_t);
template cudaError_t scan_exclusive<uint32_t>(const uint32_t*, uint32_t*, int64_t, uint32_t*, cudaStream_t);
template cudaError_t scan_exclusive<uint64_t>(const uint64_t*, uint64_t*, int64_t, uint64_t*, cudaStream_t);

template <int P>
static cudaError_t dense_u0_p(const float* depth, const Cam* cams, int F, int H, int W, Geo g,
                              double* u0, cudaStream_t s) {
  const int64_t nvox = int64_t(1) << (3 * g.D);
  const size_t sm = size_t(F) * sizeof(Cam) + size_t(kWarpsPerBlock) * P * sizeof(float);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_dense_u0<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  k_dense_u0<P><<<warp_grid(nvox), 32 * kWarpsPerBlock, sm, s>>>(depth, cams, F, H, W, g, nvox, u0);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_dense_u0(const float* depth, const Cam* cams, int F, int H, int W, Geo g,
                            double* u0, cudaStream_t s) {
  switch (pad_frames(F)) {
    case 32: return dense_u0_p<32>(depth, cams, F, H, W, g, u0, s);
    case 64: return dense_u0_p<64>(depth, cams, F, H, W, g, u0, s);
    case 128: return dense_u0_p<128>(depth, cams, F, H, W, g, u0, s);
    case 256: return dense_u0_p<256>(depth, cams, F, H, W, g, u0, s);
    case 512: return dense_u0_p<512>(depth, cams, F, H, W, g, u0, s);
    default: return cudaErrorInvalidValue;
  }
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
                              int64_t n, const float* depth, const Cam* cams, int F, int H, int W,
                              Geo g, uint32_t* count, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t sm = size_t(F) * sizeof(Cam);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_leaf_count, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  k_leaf_count<<<warp_grid(n), 32 * kWarpsPerBlock, sm, s>>>(key, level, list, n, depth, cams, F,
                                                              H, W, g, count);
  count_launches(1);
  return cudaGetLastError();
}

template <int P, typename T>
static cudaError_t leaf_fill_p(const uint64_t* key, const uint8_t* level, const uint32_t* list,
                               int64_t n, const float* depth, const Cam* cams, int F, int H, int W,
                               Geo g, const uint32_t* soff, void* samp, float* u, float* ubar,
                               cudaStream_t s) {
  const size_t sm = size_t(F) * sizeof(Cam) + size_t(kWarpsPerBlock) * P * sizeof(float);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_leaf_fill<P, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  k_leaf_fill<P, T><<<warp_grid(n), 32 * kWarpsPerBlock, sm, s>>>(
      key, level, list, n, depth, cams, F, H, W, g, soff, reinterpret_cast<T*>(samp), u, ubar);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t leaf_fill_t(const uint64_t* key, const uint8_t* level, const uint32_t* list,
                               int64_t n, const float* depth, const Cam* cams, int F, int H, int W,
                               Geo g, const uint32_t* soff, void* samp, float* u, float* ubar,
                               cudaStream_t s) {
  switch (pad_frames(F)) {
    case 32: return leaf_fill_p<32, T>(key, level, list, n, depth, cams, F, H, W, g, soff, samp, u, ubar, s);
    case 64: return leaf_fill_p<64, T>(key, level, list, n, depth, cams, F, H, W, g, soff, samp, u, ubar, s);
    case 128: return leaf_fill_p<128, T>(key, level, list, n, depth, cams, F, H, W, g, soff, samp, u, ubar, s);
    case 256: return leaf_fill_p<256, T>(key, level, list, n, depth, cams, F, H, W, g, soff, samp, u, ubar, s);
    case 512: return leaf_fill_p<512, T>(key, level, list, n, depth, cams, F, H, W, g, soff, samp, u, ubar, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_leaf_fill(const uint64_t* key, const uint8_t* level, const uint32_t* list,
                             int64_t n, const float* depth, const Cam* cams, int F, int H, int W,
                             Geo g, const uint32_t* soff, void* samp, bool fp16, float* u,
                             float* ubar, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  return fp16 ? leaf_fill_t<__half>(key, level, list, n, depth, cams, F, H, W, g, soff, samp, u, ubar, s)
              : leaf_fill_t<float>(key, level, list, n, depth, cams, F, H, W, g, soff, samp, u, ubar, s);
}

cudaError_t launch_nbr_count(View v, uint32_t* ovf_count, cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  k_nbr_count<<<blocks_for(6 * v.n, 256), 256, 0, s>>>(v, ovf_count);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_nbr_fill(View v, const uint32_t* ovf_off, int32_t* nbr, int32_t* ovf,
                            cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  k_nbr_fill<<<blocks_for(6 * v.n, 256), 256, 0, s>>>(v, ovf_off, nbr, ovf);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_precond(View v, float* tau, float* sigma, cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  k_precond<<<blocks_for(v.n, 256), 256, 0, s>>>(v, tau, sigma);
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
                        const int8_t* join_level, int64_t n_new, uint64_t* nkey, uint8_t* nlevel,
                        float* nu, float* nubar, float* np_, int64_t nstride, int32_t* src,
                        cudaStream_t s) {
  if (n_new <= 0) return cudaSuccess;
  k_emit<<<blocks_for(n_new, 256), 256, 0, s>>>(v, u, p, out_off, join_level, n_new, nkey, nlevel,
                                                 nu, nubar, np_, nstride, src);
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
    k_copy_kept<__half><<<warp_grid(n), 32 * kWarpsPerBlock, 0, s>>>(
        src, n, old_soff, reinterpret_cast<const __half*>(old_samp), new_soff,
        reinterpret_cast<__half*>(new_samp));
  else
    k_copy_kept<float><<<warp_grid(n), 32 * kWarpsPerBlock, 0, s>>>(
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
