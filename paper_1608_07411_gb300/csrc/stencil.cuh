// Device helpers shared by the iteration kernels of the primal-dual solver
// (solve.cu) and of the eps-L1 gradient descent (descent.cu): the level-aware
// operator entries, the launch layout [heavy blocks][list blocks][light
// blocks] and the divergence gathers (Sec. 3.2, forward / backward
// differences across levels).
#pragma once

#include "ofu_internal.cuh"

namespace ofu {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;
// Resident blocks per SM the iteration kernels are compiled for.  Without a
// stated minimum the compiler caps them at 32 registers and spills (the heavy
// path's block reductions share the register budget); 6 blocks (<= 42
// registers) measured fastest over 4..8 on both the 256^3 and 512^3 workloads.
constexpr int kIterMinBlocks = 6;

// Programmatic dependent launch (a launch attribute on sm_90 and later): a
// kernel launched with it may start while the kernel before it in the stream
// is still running.  Before grid_dep_wait() it may read only data that no
// kernel of the last few launches writes (the octree's structure arrays);
// after it, everything the previous kernels wrote is visible.  Every block
// calls grid_dep_launch() only after its own wait, which lets the next kernel
// start: the next kernel's early reads then never overlap a kernel that is
// still waiting.  Without the attribute both are no-ops.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// 2^e as a float, -126 <= e <= 127 (built from the exponent field)
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

__device__ __forceinline__ float edge_f(int D, int level) { return pow2f(D - level); }

// 1 / Delta for leaves of edges h and hm: 2 / (h + hm), exact sum of powers of two.
__device__ __forceinline__ float inv_delta(float h, float hm) { return __fdividef(2.0f, h + hm); }

template <typename T>
__device__ __forceinline__ float load_sample(const T* s, uint32_t i) {
  if constexpr (sizeof(T) == 2)
    return __half2float(s[i]);
  else
    return s[i];
}

// Leaves with a face list longer than kHeavy are updated by one block each
// (the octree is not 2:1 balanced: a coarse leaf can face hundreds of finest
// leaves); the thread-per-leaf path leaves them alone.  A launch runs the
// heavy blocks first, then the per-leaf blocks.
constexpr int kHeavyThreads = kThreads;   // a heavy leaf's block is a full launch block

// Fixed-order block sum of one float per thread (kHeavyThreads threads).
__device__ __forceinline__ float block_sum(float x, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  float t = 0.0f;
#pragma unroll
  for (int w = 0; w < kHeavyThreads / 32; ++w) t += red[w];
  return t;
}

// Sum over one face's finer-neighbour list of w(level) * val(index), in list
// order.  The entries are loaded four at a time and their values gathered
// four at a time, so a list of c entries costs about 2 ceil(c / 4) dependent
// loads instead of 2 c.
template <typename WFn, typename VFn>
__device__ __forceinline__ float list_sum(const int32_t* __restrict__ lst, int cnt, WFn w, VFn val) {
  float acc = 0.0f;
  for (int k0 = 0; k0 < cnt; k0 += 4) {
    int32_t f[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) f[j] = k0 + j < cnt ? lst[k0 + j] : 0;
    float x[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = k0 + j < cnt ? val(entry_idx(f[j])) : 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (k0 + j < cnt) acc += w(entry_level(f[j])) * x[j];
  }
  return acc;
}

// Which leaf a thread of an iteration launch updates.  A launch is laid out as
// [heavy blocks][list blocks][light blocks]: heavy leaves (a face list longer
// than kHeavy) get a block each; "list" leaves (some face with finer
// neighbours, none longer than kHeavy) a thread each over their compacted
// index list, so their list walks do not hold up warps of plain leaves; every
// other leaf a thread of the light blocks, which skip list leaves.  Returns
// -1 for a thread with no leaf.
struct Segments {
  const uint32_t* heavy;
  int n_heavy;
  const uint32_t* list;
  int n_list;
};

__device__ __forceinline__ int64_t segment_leaf(const Segments& sg, int64_t n, bool* is_list_leaf) {
  const int lb = (sg.n_list + kThreads - 1) / kThreads;
  const int b = int(blockIdx.x) - sg.n_heavy;
  if (b < lb) {
    const int j = b * kThreads + int(threadIdx.x);
    *is_list_leaf = true;
    return j < sg.n_list ? int64_t(sg.list[j]) : -1;
  }
  *is_list_leaf = false;
  const int64_t l = int64_t(b - lb) * kThreads + threadIdx.x;
  return l < n ? l : -1;
}

// Divergence of the vector field p at a list leaf l (gathers only; face
// lists of at most kHeavy entries); q = p(l).
__device__ __forceinline__ float divergence(const View& v, const float* __restrict__ p, int64_t l,
                                            float h, const int32_t e[6], const float q[3]) {
  float dv = 0.0f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float coef = 0.0f;
    if (e[d] >= 0) {
      coef = inv_delta(h, edge_f(v.D, entry_level(e[d])));
    } else if (e[d] != kEmpty) {
      const uint32_t st = list_start(e[d]);
      const int32_t* lst = v.ovf + st + 1;
      const int cnt = v.ovf[st];
      for (int k = 0; k < cnt; ++k) {
        const float hm = edge_f(v.D, entry_level(lst[k]));
        const float r = hm / h;
        coef += r * r * inv_delta(h, hm);
      }
    }
    dv += coef * q[d];
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int32_t ed = e[3 + d];
    const float* pd = p + int64_t(d) * v.stride;
    if (ed >= 0) {
      // same or coarser n: (h_n^3 / h^3) (h / h_n)^2 / Delta = (h_n / h) / Delta
      const float hn = edge_f(v.D, entry_level(ed));
      dv -= (hn / h) * inv_delta(h, hn) * pd[entry_idx(ed)];
    } else if (ed != kEmpty) {
      // finer n: alpha = 1, weight (h_n / h)^3 / Delta
      const uint32_t st = list_start(ed);
      dv -= list_sum(
          v.ovf + st + 1, v.ovf[st],
          [&](int lev) {
            const float hn = edge_f(v.D, lev);
            const float r = hn / h;
            return r * r * r * inv_delta(h, hn);
          },
          [&](uint32_t m) { return pd[m]; });
    }
  }
  return dv;
}

// The same divergence by one block (kHeavyThreads threads) of a heavy leaf;
// the result is valid in every thread.
__device__ float divergence_block(const View& v, const float* __restrict__ p, int64_t l, float h,
                                  float* red) {
  float dv = 0.0f;
  for (int d = 0; d < 3; ++d) {
    const int32_t e = v.nbr[int64_t(d) * v.stride + l];
    float coef = 0.0f;
    if (e >= 0) {
      if (threadIdx.x == 0) coef = inv_delta(h, edge_f(v.D, entry_level(e)));
    } else if (e != kEmpty) {
      const uint32_t st = list_start(e);
      const int cnt = v.ovf[st];
      for (int k = threadIdx.x; k < cnt; k += kHeavyThreads) {
        const float hm = edge_f(v.D, entry_level(v.ovf[st + 1 + k]));
        const float r = hm / h;
        coef += r * r * inv_delta(h, hm);
      }
    }
    dv += block_sum(coef, red) * p[int64_t(d) * v.stride + l];
  }
  for (int d = 0; d < 3; ++d) {
    const int32_t e = v.nbr[int64_t(3 + d) * v.stride + l];
    float acc = 0.0f;
    if (e >= 0) {
      if (threadIdx.x == 0) {
        const float hn = edge_f(v.D, entry_level(e));
        acc = (hn / h) * inv_delta(h, hn) * p[int64_t(d) * v.stride + entry_idx(e)];
      }
    } else if (e != kEmpty) {
      const uint32_t st = list_start(e);
      const int cnt = v.ovf[st];
      for (int k = threadIdx.x; k < cnt; k += kHeavyThreads) {
        const int32_t f = v.ovf[st + 1 + k];
        const float hn = edge_f(v.D, entry_level(f));
        const float r = hn / h;
        acc += r * r * r * inv_delta(h, hn) * p[int64_t(d) * v.stride + entry_idx(f)];
      }
    }
    dv -= block_sum(acc, red);
  }
  return dv;
}

}  // namespace
}  // namespace ofu

namespace ofu {
namespace {

// Lanes per list leaf in the group layout of the primal-dual kernels: a
// list leaf's (face, entry) slots are spread over G consecutive lanes of one
// warp (G a power of two <= 32) and reduced by shuffles.

// Face entries of one leaf as a flat run of slots: face f holds len_f slots
// (0 on the domain boundary, 1 for a single neighbour, the list length for
// finer neighbours).  fn(f, entry) is called for the slots lane, lane + G,
// ...; every list count is loaded up front (all faces at once), so a leaf
// costs four dependent loads (entries, counts, list entries, values) however
// many faces carry lists, plus two per further round of B G slots.
template <int NF, int B = 4, typename Fn>
__device__ __forceinline__ void for_each_slot(const View& v, const int32_t* e, int lane, int G,
                                              Fn fn) {
  int pre[NF + 1];
  pre[0] = 0;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int len = e[f] >= 0 ? 1 : (e[f] == kEmpty ? 0 : v.ovf[list_start(e[f])]);
    pre[f + 1] = pre[f] + len;
  }
  // B slots per lane per round: their entries, then their values, are
  // loaded together (a heavy leaf's lists can hold hundreds of entries)
  for (int s0 = lane; s0 < pre[NF]; s0 += B * G) {
    int fs[B];
    int32_t ent[B];
#pragma unroll
    for (int r = 0; r < B; ++r) {
      const int s = s0 + r * G;
      int f = 0;
#pragma unroll
      for (int q = 1; q < NF; ++q) f += s >= pre[q];
      int32_t ef = e[0], pf = pre[0];
#pragma unroll
      for (int q = 1; q < NF; ++q)
        if (f == q) {
          ef = e[q];
          pf = pre[q];
        }
      fs[r] = s < pre[NF] ? f : -1;
      ent[r] = s >= pre[NF] ? 0 : (ef >= 0 ? ef : v.ovf[list_start(ef) + 1 + (s - pf)]);
    }
#pragma unroll
    for (int r = 0; r < B; ++r)
      if (fs[r] >= 0) fn(fs[r], ent[r]);
  }
}

// Sum over the G lanes of a group (groups aligned in the warp; every lane
// of the warp takes part).
template <int G>
__device__ __forceinline__ float group_sum(float x) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

// Leaf of a thread of the list segment in the group layout: the j-th list
// leaf for threads j * G .. j * G + G - 1.  Lanes past the end take the last
// list leaf and must not write (valid = false), since every lane of the warp
// joins the shuffles.
template <int G>
__device__ __forceinline__ int64_t list_group_leaf(const Segments& sg, int b, int* lane, bool* valid) {
  const int t = b * kThreads + int(threadIdx.x);
  const int j = t / G;
  *lane = t % G;
  *valid = j < sg.n_list;
  return int64_t(sg.list[*valid ? j : sg.n_list - 1]);
}

// alpha / Delta of a +face neighbour m (edge hm) of a leaf of edge h:
// alpha = min(1, (hm / h)^2) -- 1 for a single entry, the face share for a
// finer neighbour.
__device__ __forceinline__ float plus_weight(float h, float hm) {
  const float r = hm / h;
  return fminf(1.0f, r * r) * inv_delta(h, hm);
}

// (h_n^3 / h^3) alpha_nl / Delta of a -face neighbour n (edge hn):
// hn / h / Delta for a same or coarser n, (hn / h)^3 / Delta for a finer one.
__device__ __forceinline__ float minus_weight(float h, float hn) {
  const float r = hn / h;
  return (r >= 1.0f ? r : r * r * r) * inv_delta(h, hn);
}

}  // namespace
}  // namespace ofu
