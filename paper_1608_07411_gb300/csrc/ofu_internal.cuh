// Internal declarations of the octfuse CUDA library (not part of the C ABI).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/octfuse.h"

namespace ofu {

// ---------------------------------------------------------------------------
// Face-neighbour entries.  Each leaf has one int32 entry per face:
//   kEmpty (-1)                     domain boundary
//   bit31 = 0                       one neighbour of the same or a coarser
//                                   level: bits 0..26 index, 27..30 level
//   bit31 = 1, not kEmpty           list of finer neighbours starting at
//                                   ovf[bits 0..30]: ovf[start] = count,
//                                   then count entries (index | level << 27)
// so the common case costs one 4-byte read and carries the neighbour's level.
constexpr int32_t kEmpty = -1;
constexpr uint32_t kIdxMask = (1u << 27) - 1;
constexpr int kMaxDepth = 15;
constexpr int64_t kMaxLeaves = int64_t(1) << 27;
// Warm-start network: 39 inputs, two hidden layers of 64, one output.
constexpr int kMlpIn = 39;
constexpr int kMlpHid = 64;
constexpr int kMlpParams = kMlpHid * kMlpIn + kMlpHid + kMlpHid * kMlpHid + kMlpHid + kMlpHid + 1;

// Face lists longer than this make a leaf "heavy": its iteration updates run
// as one block per leaf instead of one thread.
constexpr int kHeavy = 16;

__host__ __device__ inline int32_t make_single(uint32_t idx, int level) {
  return int32_t(idx | (uint32_t(level) << 27));
}
__host__ __device__ inline int32_t make_list(uint32_t start) { return int32_t(0x80000000u | start); }
__host__ __device__ inline bool is_single(int32_t e) { return e >= 0; }
__host__ __device__ inline bool is_list(int32_t e) { return e < 0 && e != kEmpty; }
__host__ __device__ inline uint32_t entry_idx(int32_t e) { return uint32_t(e) & kIdxMask; }
__host__ __device__ inline int entry_level(int32_t e) { return int((uint32_t(e) >> 27) & 15u); }
__host__ __device__ inline uint32_t list_start(int32_t e) { return uint32_t(e) & 0x7fffffffu; }

// ---------------------------------------------------------------------------
// Morton keys: bit k of x -> bit 3k, y -> 3k+1, z -> 3k+2.

__host__ __device__ inline uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | x << 32) & 0x1f00000000ffffull;
  x = (x | x << 16) & 0x1f0000ff0000ffull;
  x = (x | x << 8) & 0x100f00f00f00f00full;
  x = (x | x << 4) & 0x10c30c30c30c30c3ull;
  x = (x | x << 2) & 0x1249249249249249ull;
  return x;
}
__host__ __device__ inline uint32_t compact3(uint64_t x) {
  x &= 0x1249249249249249ull;
  x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
  x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
  x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
  x = (x ^ (x >> 32)) & 0x1fffffull;
  return uint32_t(x);
}
__host__ __device__ inline uint64_t morton(uint32_t x, uint32_t y, uint32_t z) {
  return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

// ---------------------------------------------------------------------------
// One frame's camera in float32 (Eq. 1 is evaluated in float32).
struct Cam {
  float r[9];  // camera-to-world rotation, row-major
  float c[3];  // centre C_i
  float fx, fy, cx, cy;
};

// Geometry shared by the Eq. 1 kernels.
struct Geo {
  float org[3];  // domain minimum corner
  float vox;     // finest voxel edge = extent / 2^D
  float delta, eta;
  int D;
};

// Range along the ray of pixel (px, py): D * |K^-1 (px + 0.5, py + 0.5, 1)|,
// float32, one rounding per operation.  Depends on the pixel only, so it is
// precomputed once per frame set (the "range map"); 0, negative or NaN depth
// stays non-positive or NaN, +inf stays +inf.
__device__ __forceinline__ float pixel_range(const Cam& k, float d, int px, int py) {
  const float a = __fdiv_rn(__fsub_rn(__fadd_rn(float(px), 0.5f), k.cx), k.fx);
  const float b = __fdiv_rn(__fsub_rn(__fadd_rn(float(py), 0.5f), k.cy), k.fy);
  const float rl = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b)), 1.0f));
  return __fmul_rn(d, rl);
}

// Eq. 1 for one point and one frame, float32 with one rounding per
// operation in a fixed order (no contraction into fused multiply-adds).
// `range` is the frame's range map.  Returns false when the frame does not
// observe the point (w = 0).
__device__ __forceinline__ bool eq1_sample(const Cam& k, const float* __restrict__ range, int H,
                                           int W, float x, float y, float z, float delta, float eta,
                                           float* f) {
  const float dx = __fsub_rn(x, k.c[0]);
  const float dy = __fsub_rn(y, k.c[1]);
  const float dz = __fsub_rn(z, k.c[2]);
  const float xc = __fadd_rn(__fadd_rn(__fmul_rn(k.r[0], dx), __fmul_rn(k.r[3], dy)), __fmul_rn(k.r[6], dz));
  const float yc = __fadd_rn(__fadd_rn(__fmul_rn(k.r[1], dx), __fmul_rn(k.r[4], dy)), __fmul_rn(k.r[7], dz));
  const float zc = __fadd_rn(__fadd_rn(__fmul_rn(k.r[2], dx), __fmul_rn(k.r[5], dy)), __fmul_rn(k.r[8], dz));
  if (!(zc > 0.0f)) return false;
  const float u = __fadd_rn(__fmul_rn(k.fx, __fdiv_rn(xc, zc)), k.cx);
  const float v = __fadd_rn(__fmul_rn(k.fy, __fdiv_rn(yc, zc)), k.cy);
  if (!(u >= 0.0f && u < float(W) && v >= 0.0f && v < float(H))) return false;
  const int px = int(floorf(u));
  const int py = int(floorf(v));
  const float rng = __ldg(range + size_t(py) * W + px);
  if (!(rng > 0.0f)) return false;   // depth 0, negative or NaN
  const float dist = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)));
  const float phi = __fsub_rn(rng, dist);
  if (!(phi >= -eta)) return false;
  // Outside the band |phi| < delta the rounded quotient is already beyond
  // +-1 (rounding is monotone and 1 is exact), so the clamp decides alone.
  *f = phi >= delta ? 1.0f
                    : (phi <= -delta ? -1.0f : fminf(fmaxf(__fdiv_rn(phi, delta), -1.0f), 1.0f));
  return true;
}

// Per-frame TSDF octrees (Fig. 4 data term; built by frames.cu): the tree
// leaves of every frame sorted by key, frame i at [start[i], start[i + 1]),
// with observed counts and float64 sums of f, and exclusive prefix sums of
// both over the concatenation.  key == nullptr: Eq. 1 at leaf centres.
struct FrameTrees {
  const int64_t* start = nullptr;   // [F + 1]
  const uint64_t* key = nullptr;
  const uint8_t* level = nullptr;
  const uint64_t* cnt = nullptr;
  const double* tot = nullptr;
  const uint64_t* pcnt = nullptr;   // [total + 1]
  const double* ptot = nullptr;     // [total + 1]
};

// f_i* for the iterate leaf (key k, level L) by the Fig. 4 rule: the deepest
// node of frame i's tree on the path to the leaf at a level <= L, its mean
// when any voxel below it is observed.  Returns false when it is not
// observed (w = 0).
__device__ __forceinline__ bool tree_sample(const FrameTrees& t, int i, uint64_t k, int L, int D,
                                            float* f) {
  int64_t lo = t.start[i], hi = t.start[i + 1];
  const int64_t end0 = hi;
  while (lo < hi) {   // first tree leaf with key > k
    const int64_t mid = (lo + hi) >> 1;
    if (t.key[mid] <= k) lo = mid + 1; else hi = mid;
  }
  const int64_t j = lo - 1;   // the tree leaf holding voxel k (the first leaf has key 0)
  uint64_t c;
  double s;
  if (t.level[j] <= L) {
    c = t.cnt[j];
    s = t.tot[j];
  } else {
    // the node at level L is an inner node: its leaves are the keys [k, k + 8^(D-L))
    const uint64_t kend = k + (uint64_t(1) << (3 * (D - L)));
    lo = j;
    hi = end0;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (t.key[mid] < kend) lo = mid + 1; else hi = mid;
    }
    c = t.pcnt[lo] - t.pcnt[j];
    s = t.ptot[lo] - t.ptot[j];
  }
  if (c == 0) return false;
  *f = float(s / double(c));
  return true;
}

// Leaf centre in float32: origin + (corner + h/2) * voxel.
__device__ __forceinline__ float centre_coord(float org, uint32_t corner, uint32_t h, float vox) {
  const float mid = __fadd_rn(float(corner), __fmul_rn(0.5f, float(h)));
  return __fadd_rn(org, __fmul_rn(mid, vox));
}

// ---------------------------------------------------------------------------
// Device buffers of one copy of the leaf arrays.
struct Leaves {
  int64_t cap = 0;
  uint64_t* key = nullptr;
  uint8_t* level = nullptr;
  float* u = nullptr;
  float* ubar = nullptr;
  float* p = nullptr;      // [3][cap]
  float* tau = nullptr;
  float* sigma = nullptr;
  int32_t* nbr = nullptr;  // [6][cap]
  uint32_t* soff = nullptr;  // [cap + 1]
  uint16_t* khint = nullptr;  // rank k* of the last prox of each leaf (a search hint only)
  int32_t* ovf = nullptr;  // finer-neighbour lists of nbr
  int64_t ovf_cap = 0;
};

// Raw view of the current structure handed to kernels.
struct View {
  int64_t n;
  int D;
  const uint64_t* key;
  const uint8_t* level;
  const int32_t* nbr;  // [6][stride]
  const int32_t* ovf;
  int64_t stride;      // leaf capacity (row pitch of nbr and p)
  const uint32_t* map; // finest voxel (Morton order) -> index of its leaf
};

// Leaves an iteration launch treats apart from the thread-per-leaf path:
// heavy leaves (a face list longer than kHeavy, one block each) and list
// leaves (finer neighbours on some face, none heavy; a thread each over this
// compacted list so that their list walks share warps only with each other).
struct LeafSets {
  const uint32_t* heavy = nullptr;
  int n_heavy = 0;
  const uint32_t* list = nullptr;
  int n_list = 0;
};

// Neighbour records of the heavy and list leaves, rebuilt with the leaf
// classes (solve.cu): the operator entries of those leaves as flat lists, so
// the iteration kernels read them before griddepcontrol.wait instead of
// walking the face lists after it.  Group position g runs over the heavy
// set, then the list set.  Its neighbours are the records start[g] ..
// start[g + 1] - 1, rec = neighbour index | axis << 28 and w = the weight:
//   dual step (gradient)     +face neighbours, alpha / Delta;
//   primal step (divergence) -face neighbours, (h_n^3 / h^3) alpha_nl / Delta,
//                            and cp[3 g + d], the sum of alpha / Delta over
//                            the neighbours across the +d face.
struct NbrRecs {
  const uint32_t* start = nullptr;
  const uint32_t* rec = nullptr;
  const float* w = nullptr;
  const float* cp = nullptr;
};

// The structure before a split/join pass, handed to the neighbour build of
// the new one: a kept leaf (same key, same level) whose neighbours across a
// face were all kept has the same neighbours afterwards, so its entry is
// carried over with the indices renumbered instead of being searched again.
// Kept leaves keep their relative order, so carried lists stay ascending.
struct Carry {
  const int32_t* nbr = nullptr;  // old [6][stride]; nullptr: build from scratch
  const int32_t* ovf = nullptr;  // old lists
  int64_t stride = 0;
  const int32_t* src = nullptr;  // new leaf -> old index if kept, else -1
  const int32_t* fwd = nullptr;  // old leaf -> new index if kept, else -1
  uint32_t* aux = nullptr;       // [6 n]: old list start of a carried list
  uint8_t* full = nullptr;       // [6 n]: the face was carried
  const float* tau = nullptr;    // old step sizes (copied for fully carried leaves)
  const float* sigma = nullptr;
};

}  // namespace ofu

// ---------------------------------------------------------------------------
// The warm-start network object (opaque to callers).
struct ofu_mlp {
  cudaStream_t stream = nullptr;
  std::string err;
  bool poisoned = false;
  float* params = nullptr;   // kMlpParams
  float* m = nullptr;        // Adam first moments
  float* v = nullptr;        // Adam second moments
  float* grad = nullptr;
  float* partial = nullptr;  // per-block gradients
  int64_t partial_blocks = 0;
  double* sums = nullptr;    // per-block loss sums, then [loss, sum w]
  int64_t step = 0;
  void* pinned = nullptr;
};

// ---------------------------------------------------------------------------
// The context (opaque to callers).
struct ofu_ctx {
  ofu_params prm{};
  cudaStream_t stream = nullptr;
  int device = 0;

  // device memory: the caller's allocator (ofu_create_octree_ex) or cudaMalloc;
  // live blocks with their sizes (the free callback is given the size)
  ofu_alloc_fn alloc_fn = nullptr;
  ofu_free_fn free_fn = nullptr;
  void* alloc_user = nullptr;
  std::unordered_map<void*, size_t> live;
  std::string err;
  bool poisoned = false;

  // frames (copied in by ofu_integrate_frames)
  int F = 0, H = 0, W = 0;
  float* depth = nullptr;      // range maps after ofu_integrate_frames (pixel_range)
  ofu::Cam* cams = nullptr;
  bool have_frames = false;

  // leaves: two copies, swapped by restructuring
  ofu::Leaves L[2];
  int cur = 0;
  int64_t n = 0;

  // samples (sorted CSR), double buffered like the leaves
  void* samp[2] = {nullptr, nullptr};
  int64_t samp_cap[2] = {0, 0};
  int64_t n_samples = 0;

  // finest voxel -> leaf index of the current structure (8^D entries)
  uint32_t* map = nullptr;

  // leaf classes of the current structure (see kHeavy, LeafSets): [4][cap]
  // heavy dual, heavy primal, list dual, list primal
  uint32_t* heavy = nullptr;
  int64_t heavy_cap = 0;
  int n_heavy_dual = 0, n_heavy_primal = 0;
  int n_list_dual = 0, n_list_primal = 0;

  // scratch (grown on demand)
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  void* pinned = nullptr;  // small host staging for scalar results

  // per-frame TSDF octrees (data_term = 1): see FrameTrees
  int64_t* ft_start = nullptr;       // device [F + 1]
  uint64_t* ft_key = nullptr;
  uint8_t* ft_level = nullptr;
  uint64_t* ft_cnt = nullptr;
  double* ft_tot = nullptr;
  uint64_t* ft_pcnt = nullptr;       // [cap + 1]
  double* ft_ptot = nullptr;         // [cap + 1]
  int64_t ft_cap = 0;
  std::vector<int64_t> ft_host_start;  // host copy of ft_start

  // per-launch timing of the iteration kernels (ofu_profile)
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;   // pool, 3 per iteration
  size_t prof_used = 0;
  double prof_bytes[2] = {0.0, 0.0};
  int64_t prof_launches[2] = {0, 0};
};

namespace ofu {

// Process-wide count of kernel launches made by this library.
void count_launches(int64_t k);
int64_t launches_so_far();

// ---------------------------------------------------------------------------
// Launchers (defined in build.cu / solve.cu).  All enqueue on `s`.

// Exclusive prefix sum of n items into out[0..n] (out[n] = total).  `in`
// and `out` may alias.  `tmp` needs scan_tmp_items<T>(n) elements.
template <typename T>
size_t scan_tmp_items(int64_t n);
template <typename T>
cudaError_t scan_exclusive(const T* in, T* out, int64_t n, T* tmp, cudaStream_t s);

// Depth maps -> range maps in place (see pixel_range).
cudaError_t launch_range_map(float* depth, const Cam* cams, int F, int H, int W, cudaStream_t s);

// Median field at finest-voxel centres (Morton order), then the Eq. 2 min/max
// pyramid and the per-voxel leaf flags.  launch_dense_u0 needs a queue of
// 8^D entries and a device counter as scratch.
// Min / max pyramid of the range maps, used by the median scan to classify a
// block of voxel centres against a whole frame at once.  Level k (1..nl) of a
// frame has w[k] x h[k] texels; texel (x, y) holds the min and the max, over
// the image's pixels in [x 2^k, (x + 1) 2^k) x [y 2^k, (y + 1) 2^k), of the
// range where it is valid (> 0) and -inf where it is not.  Level 0 is the
// range map itself.
constexpr int kMaxRangeLevels = 24;
struct RangePyr {
  const float2* tex;
  int64_t frame_texels;  // texels of one frame (levels 1..nl)
  int nl;
  int off[kMaxRangeLevels + 1], w[kMaxRangeLevels + 1], h[kMaxRangeLevels + 1];
};
// Level sizes and offsets for H x W maps (tex = nullptr).
RangePyr range_pyr_dims(int H, int W);
cudaError_t launch_range_pyr(const float* range, int F, int H, int W, RangePyr rp, float2* tex,
                             cudaStream_t s);
cudaError_t launch_dense_u0(const float* depth, const Cam* cams, int F, int H, int W, Geo g,
                            RangePyr rp, double* u0, uint32_t* queue, unsigned long long* nqueue,
                            cudaStream_t s);
cudaError_t launch_pyramid(const double* u0, int D, double* mn, double* mx, cudaStream_t s);
cudaError_t launch_leaf_flags(const double* mn, const double* mx, int D, double spread_tau,
                              uint32_t* flags, cudaStream_t s);
cudaError_t launch_emit_constructed(const uint32_t* flags, const uint32_t* pos,
                                    const double* mn, const double* mx, int D, double spread_tau,
                                    uint64_t* key, uint8_t* level, cudaStream_t s);

// Eq. 1 samples of leaves: counts (W) and the sorted CSR fill.  `list`
// selects leaves (nullptr = all n); with `nlist` (device) the number of listed
// leaves is read on the device and n is only the grid's upper bound.  fill
// also writes u = ubar = median when u is given.
cudaError_t launch_leaf_count(const uint64_t* key, const uint8_t* level, const uint32_t* list,
                              const unsigned long long* nlist, int64_t n, const float* depth,
                              const Cam* cams, int F, int H, int W, Geo g, FrameTrees tr,
                              uint32_t* count, cudaStream_t s);
cudaError_t launch_leaf_fill(const uint64_t* key, const uint8_t* level, const uint32_t* list,
                             const unsigned long long* nlist, int64_t n, const float* depth,
                             const Cam* cams, int F, int H, int W, Geo g, FrameTrees tr,
                             const uint32_t* soff, void* samp, bool fp16, float* u, float* ubar,
                             cudaStream_t s);

// Leaf classes of the iteration kernels, read from the unscanned
// neighbour-list counts and listed in leaf order: heavy (dual: a +face list
// longer than kHeavy; primal: any face list longer than kHeavy) and list
// leaves (dual: a +face list, none heavy; primal: any face list, none heavy).
// sets: [4][cap] = heavy dual, heavy primal, list dual, list primal.
// hflags, lflags: n + 1 scratch words each; hflags[n] and lflags[n] receive
// the packed totals (dual count low 32 bits, primal count high 32 bits);
// tmp: scan scratch for n.
cudaError_t launch_leaf_sets(View v, const uint32_t* ovf_count, uint64_t* hflags,
                             uint64_t* lflags, uint64_t* tmp, uint32_t* sets, int64_t cap,
                             cudaStream_t s);

// Face neighbours: count pass (long lists queued in longq and counted by a
// block each), then the fill.
cudaError_t launch_nbr_count(View v, Carry cy, int32_t* nbr, uint32_t* ovf_count, uint32_t* longq,
                             unsigned long long* nlong, uint32_t* pendq, unsigned long long* npend,
                             cudaStream_t s);
cudaError_t launch_nbr_fill(View v, Carry cy, const uint32_t* ovf_off, int32_t* nbr, int32_t* ovf,
                            const uint32_t* longq, const unsigned long long* nlong,
                            const uint32_t* pendq, const unsigned long long* npend,
                            cudaStream_t s);
cudaError_t launch_precond(View v, Carry cy, float* tau, float* sigma, const uint32_t* heavy,
                           int n_heavy, cudaStream_t s);
cudaError_t launch_check_tiling(const uint64_t* key, const uint8_t* level, int64_t n, int D,
                                uint32_t* bad, cudaStream_t s);

// Restructuring.
cudaError_t launch_classify(const float* u, int64_t n, double tau_j, uint64_t* cls,
                            cudaStream_t s);
cudaError_t launch_mark(View v, const float* u, const uint64_t* cls_scan, double tau_s,
                        double tau_j, uint64_t* out_count, int8_t* join_level,
                        unsigned long long* counters, cudaStream_t s);
cudaError_t launch_emit(View v, const float* u, const float* p, const uint64_t* out_off,
                        const int8_t* join_level, uint64_t* nkey, uint8_t* nlevel, float* nu,
                        float* nubar, float* np_, int64_t nstride, int32_t* src, int32_t* fwd,
                        uint32_t* big, unsigned long long* nbig, cudaStream_t s);
// Voxel -> leaf map of a structure (big: scratch of n entries, nbig: two
// counters, of the big and of the huge leaves).
cudaError_t launch_map(const uint64_t* key, const uint8_t* level, int64_t n, int D, uint32_t* map,
                       uint32_t* big, unsigned long long* nbig, cudaStream_t s);
cudaError_t launch_new_list(const int32_t* src, int64_t n, uint32_t* list,
                            unsigned long long* cnt, cudaStream_t s);
cudaError_t launch_kept_counts(const int32_t* src, const uint32_t* old_soff, int64_t n,
                               uint32_t* count, cudaStream_t s);
cudaError_t launch_copy_kept_samples(const int32_t* src, int64_t n, const uint32_t* old_soff,
                                     const void* old_samp, const uint32_t* new_soff,
                                     void* new_samp, bool fp16, cudaStream_t s);

// Solver kernels.  `ls` names the heavy leaves and the list leaves of the
// step (see LeafSets).
cudaError_t launch_dual(View v, const float* ubar, float* p, const float* sigma, float lambda,
                        LeafSets ls, NbrRecs gr, cudaStream_t s);
// p = lambda g / |g| where |g| >= g0 (g the gradient of u), else 0.
cudaError_t launch_dual_init(View v, const float* u, float* p, float lambda, float g0,
                             LeafSets ls, NbrRecs gr, cudaStream_t s);
cudaError_t launch_primal(View v, float* u, float* ubar, const float* p, const float* tau,
                          const uint32_t* soff, const void* samp, bool fp16, float gamma,
                          uint16_t* khint, LeafSets ls, NbrRecs dr, cudaStream_t s);
// Neighbour records of a leaf set (plus: the dual step's gradient records,
// else the primal step's divergence records with cp): counts per group
// position (cnt[0 .. n_heavy + n_list)), then, with start = their exclusive
// scan, the records.  rec / w need at least the scanned total, which is at
// most the list entries plus three per group leaf.
cudaError_t launch_recs_count(View v, LeafSets ls, bool plus, uint32_t* cnt, cudaStream_t s);
cudaError_t launch_recs_fill(View v, LeafSets ls, bool plus, const uint32_t* start, uint32_t* rec,
                             float* w, float* cp, cudaStream_t s);
// SMs of the current device (looked up once per process; build.cu).
int sm_count();
size_t energy_tmp_bytes(int64_t n);
cudaError_t launch_energy(View v, const float* u, const float* p, const uint32_t* soff,
                          const void* samp, bool fp16, double lambda, double gamma, LeafSets ls,
                          double* partial, double* out3, cudaStream_t s);

// Energy with its scratch in a file-scope device array (solve.cu).
int64_t energy_static_max_leaves();
cudaError_t energy_static_scratch(double** ptr);
cudaError_t launch_energy_static(View v, const float* u, const float* p, const uint32_t* soff,
                                 const void* samp, bool fp16, double lambda, double gamma,
                                 LeafSets ls, double* scratch, cudaStream_t s);
int energy_static_result_offset();

// Warm-start network (mlp.cu).
size_t mlp_tile_smem();
int64_t mlp_grad_blocks(int64_t B);
cudaError_t launch_features(View v, const float* u, const uint32_t* soff, const void* samp,
                            bool fp16, float* X, cudaStream_t s);
cudaError_t launch_mlp_forward(const float* params, const float* X, int64_t B, float* y,
                               cudaStream_t s);
cudaError_t launch_warm_start(View v, const float* u, const uint32_t* soff, const void* samp,
                              bool fp16, const float* params, float* out, cudaStream_t s);
cudaError_t launch_mlp_grad(const float* params, const float* X, const float* t, const float* w,
                            const int32_t* rows, int64_t B, float* partial, double* psums,
                            float* grad, double* loss2, cudaStream_t s);
cudaError_t launch_adam(float* params, float* m, float* v, const float* g, float lr, int64_t step,
                        cudaStream_t s);

// Export helpers.
cudaError_t launch_widen_samples(const void* samp, bool fp16, int64_t n, float* out,
                                 cudaStream_t s);
cudaError_t launch_w_from_soff(const uint32_t* soff, int64_t n, int32_t* out, cudaStream_t s);

}  // namespace ofu
