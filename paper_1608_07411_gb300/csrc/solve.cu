// Primal-dual iteration kernels and the float64 energy / gap reduction
// (Sec. 3.2, Eq. 5; the primal-dual scheme is the one named in Sec. 5).
//
// Operators on the leaves (edges h in finest voxels, Delta = (h_l + h_m) / 2):
//   grad_d u(l) = sum over m across l's +d face of alpha_lm (u_m - u_l) / Delta
//                 with alpha_lm = min(1, (h_m / h_l)^2), 0 on the boundary;
//   div p(l)    = sum_d p_d(l) sum_{m in +d face} alpha_lm / Delta
//               - sum_d sum_{n in -d face} (h_n^3 / h_l^3) alpha_nl / Delta p_d(n),
// the negative adjoint of grad under volume-weighted inner products, so the
// divergence gathers from the -face lists and nothing is scattered.
#include <math_constants.h>

#include <algorithm>

#include "stencil.cuh"

namespace ofu {

namespace {

// p of a piecewise-ramp field: lambda g / |g| where |g| >= g0, else 0 (the
// optimal dual wherever the TV term is differentiable and the field has an
// edge); used to start the dual together with a warm-started u.
__device__ __forceinline__ void dual_init_write(float* __restrict__ p, int64_t stride, int64_t l,
                                                const float g[3], float lambda, float g0) {
  const float nrm = sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  const float sc = nrm >= g0 && nrm > 0.0f ? lambda / nrm : 0.0f;
  p[l] = sc * g[0];
  p[stride + l] = sc * g[1];
  p[2 * stride + l] = sc * g[2];
}

// Dual-step value of leaf l from its gradient g: the ascent and projection,
// or (INIT) the start lambda g / |g|.
template <bool INIT>
__device__ __forceinline__ void dual_finish(float* __restrict__ p, size_t st, int64_t l,
                                            const float q[3], float sl, const float g[3],
                                            float lambda, float g0) {
  if (INIT) {
    dual_init_write(p, int64_t(st), l, g, lambda, g0);
    return;
  }
  float r0 = q[0] + sl * g[0], r1 = q[1] + sl * g[1], r2 = q[2] + sl * g[2];
  const float nrm = sqrtf(r0 * r0 + r1 * r1 + r2 * r2);
  if (nrm > lambda) {
    const float sc = lambda / nrm;
    r0 *= sc;
    r1 *= sc;
    r2 *= sc;
  }
  p[l] = r0;
  p[st + l] = r1;
  p[2 * st + l] = r2;
}

// Lanes per list leaf of the dual and primal steps (measured over 1..16: 4
// and 2 fastest on the 256^3 and 512^3 workloads; the primal step has about
// twice as many list leaves, six faces and its prox).
constexpr int kDualListLanes = 4;
constexpr int kPrimalListLanes = 2;
// Lanes per heavy leaf (a face list longer than kHeavy): one warp.
constexpr int kHeavyLanes = 32;
// Leaves per thread of the dual step's light path.
constexpr int kDualLightLeaves = 2;

// Blocks of the heavy segment (kHeavyLanes lanes per heavy leaf).
__device__ __host__ __forceinline__ int heavy_blocks(const Segments& sg) {
  return (sg.n_heavy * kHeavyLanes + kThreads - 1) / kThreads;
}

// Records a lane loads before the wait (G lanes per leaf cover G times this
// many neighbours in the first round).
constexpr int kRecBatch = 4;

// A dual step of the leaves of a compacted set (heavy or list leaves), G
// lanes per leaf: the j-th leaf of `set` (group position g0 + j) for threads
// j G .. j G + G - 1 of the segment starting at block 0 + `b`.  The leaf's
// +face neighbours come from its gradient records (static between
// restructures, so read before the wait); after it the lanes gather ubar at
// the neighbours and the group sums each axis.  Lanes past the end take the
// last leaf and do not write (every lane of the warp joins the shuffles).
template <bool INIT, int G>
__device__ __forceinline__ void dual_group(const View& v, const float* __restrict__ ubar,
                                           float* __restrict__ p, const float* __restrict__ sigma,
                                           float lambda, float gth, const NbrRecs& gr,
                                           const uint32_t* __restrict__ set, int n_set, int g0,
                                           int b) {
  const size_t st = size_t(v.stride);
  const int t = b * kThreads + int(threadIdx.x);
  const int j = t / G, lane = t % G;
  const bool valid = j < n_set;
  const int jc = valid ? j : n_set - 1;
  const int64_t l = set[jc];
  const int g = g0 + jc;
  const uint32_t m0 = gr.start[g], m1 = gr.start[g + 1];
  const float sl = INIT ? 0.0f : sigma[l];
  uint32_t rec[kRecBatch];
  float w[kRecBatch];
#pragma unroll
  for (int r = 0; r < kRecBatch; ++r) {
    const uint32_t k = m0 + lane + r * G;
    rec[r] = k < m1 ? gr.rec[k] : 0u;
    w[r] = k < m1 ? gr.w[k] : 0.0f;
  }
  grid_dep_wait();
  grid_dep_launch();
  const float ul = ubar[l];
  float acc[3] = {0.0f, 0.0f, 0.0f};
  auto add = [&](uint32_t rk, float wk) {
    const float tk = wk * (ubar[rk & 0x0fffffffu] - ul);
    const uint32_t d = rk >> 28;
    acc[0] += d == 0 ? tk : 0.0f;
    acc[1] += d == 1 ? tk : 0.0f;
    acc[2] += d == 2 ? tk : 0.0f;
  };
#pragma unroll
  for (int r = 0; r < kRecBatch; ++r) add(rec[r], w[r]);
#pragma unroll 4
  for (uint32_t k = m0 + lane + kRecBatch * G; k < m1; k += G) add(gr.rec[k], gr.w[k]);
  float gv[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) gv[d] = group_sum<G>(acc[d]);
  if (lane != 0 || !valid) return;
  const float q[3] = {p[l], p[st + l], p[2 * st + l]};
  dual_finish<INIT>(p, st, l, q, sl, gv, lambda, gth);
}

// INIT = false: the dual step p <- proj(p + sigma grad ubar).
// INIT = true:  p <- dual_init_write(grad ubar) with threshold g0 (sigma unused).
// Launch layout [heavy blocks][list blocks][light blocks]: a heavy leaf's
// slots are spread over a warp, a list leaf's over kDualListLanes lanes, a
// light leaf (single entries only) has a thread.
template <bool INIT>
__global__ void __launch_bounds__(kThreads, kIterMinBlocks) k_dual(View v, const float* __restrict__ ubar,
                                                                   float* __restrict__ p,
                                                                   const float* __restrict__ sigma,
                                                                   float lambda, Segments sg, float g0,
                                                                   NbrRecs gr) {
  const size_t st = size_t(v.stride);
  const int hb = heavy_blocks(sg);
  const int lb = (sg.n_list * kDualListLanes + kThreads - 1) / kThreads;
  const int b = int(blockIdx.x);
  if (b < hb + lb) {
    if (b < hb)
      dual_group<INIT, kHeavyLanes>(v, ubar, p, sigma, lambda, g0, gr, sg.heavy, sg.n_heavy, 0, b);
    else
      dual_group<INIT, kDualListLanes>(v, ubar, p, sigma, lambda, g0, gr, sg.list, sg.n_list,
                                       sg.n_heavy, b - hb);
    return;
  }
  const int lbase = hb + lb;
  // light path: kDualLightLeaves leaves per thread (a block covers that many
  // runs of kThreads consecutive leaves), single entries only.  All loads of
  // all of them are issued before any gather, and all gathers before any
  // arithmetic, so a thread keeps several independent loads in flight.  A
  // thread past the end re-reads the last leaf and writes nothing; a list
  // leaf's lane gathers its own value (harmless) and writes nothing.
  constexpr int K = kDualLightLeaves;
  const int64_t base = int64_t(b - lbase) * (kThreads * K) + threadIdx.x;
  int64_t l[K];
  int32_t e[K][3];
  int lev[K];
  float ul[K], q[K][3], sl[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    l[j] = base + j * kThreads;
    const int64_t lc = l[j] < v.n ? l[j] : v.n - 1;
#pragma unroll
    for (int d = 0; d < 3; ++d) e[j][d] = v.nbr[d * st + lc];
    lev[j] = v.level[lc];
    sl[j] = INIT ? 0.0f : sigma[lc];
  }
  // the structure arrays above are read before the previous kernel ends;
  // ubar and p only after it
  grid_dep_wait();
  grid_dep_launch();
  float x[K][3];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int64_t lc = l[j] < v.n ? l[j] : v.n - 1;
    ul[j] = ubar[lc];
#pragma unroll
    for (int d = 0; d < 3; ++d) q[j][d] = p[d * st + lc];
#pragma unroll
    for (int d = 0; d < 3; ++d) x[j][d] = ubar[e[j][d] >= 0 ? entry_idx(e[j][d]) : 0u];
    if (l[j] >= v.n) l[j] = -1;
  }
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const float h = edge_f(v.D, lev[j]);
    float g[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float hm = edge_f(v.D, e[j][d] >= 0 ? entry_level(e[j][d]) : lev[j]);
      g[d] = e[j][d] >= 0 ? (x[j][d] - ul[j]) * inv_delta(h, hm) : 0.0f;
    }
    if (l[j] < 0 || is_list(e[j][0]) || is_list(e[j][1]) || is_list(e[j][2])) continue;
    dual_finish<INIT>(p, st, l[j], q[j], sl[j], g, lambda, g0);
  }
}

// Prox of the data term: argmin_x (x - v)^2 / (2 tau) + c sum_k |x - f_k| is
// the median of {f_k} and {v + t (W - 2k)}_{k=0..W}, t = tau c.  With the
// samples sorted it is clamp(b_k*, f_(k*-1), f_k*) (0-based f, f_-1 = -inf,
// f_W = +inf) where k* is the number of k with f_k < b_k = v + t (W - 2k).
// That predicate holds exactly for a prefix of k (f rises, b falls, and the
// rounded b_k still falls), so k* is the unique rank where it turns false,
// and any search that keeps [lo, hi] around it with f_(lo-1) (a rank that
// held) and f_hi (a rank that failed) ends with the same k* and the same
// two samples: the result does not depend on the search order.
//
// The prox from the search hint kh (the leaf's k* of the previous
// iteration): ranks kh - 1 and kh are tested first (two loads of adjacent
// samples, issued together), which settles k* at once whenever it has not
// moved -- nearly always once the field has settled -- and otherwise the
// side that remains is bisected.  Returns the prox (before the clamp to
// [-1, 1]) and k*.
template <typename T>
__device__ __forceinline__ float prox_hinted(const T* __restrict__ fs, int W, float x, float t, int kh,
                                             int* kstar) {
  int lo = 0, hi = W;
  float flo = -CUDART_INF_F, fhi = CUDART_INF_F;
  const float fa = kh > 0 ? load_sample(fs, kh - 1) : 0.0f;
  const float fb = kh < W ? load_sample(fs, kh) : 0.0f;
  if (kh > 0) {
    if (fa < __fmaf_rn(t, float(W - 2 * (kh - 1)), x)) {
      lo = kh;
      flo = fa;
    } else {
      hi = kh - 1;
      fhi = fa;
    }
  }
  if (kh < W && lo <= kh && kh < hi) {
    if (fb < __fmaf_rn(t, float(W - 2 * kh), x)) {
      lo = kh + 1;
      flo = fb;
    } else {
      hi = kh;
      fhi = fb;
    }
  }
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const float fm = load_sample(fs, mid);
    if (fm < __fmaf_rn(t, float(W - 2 * mid), x)) {
      lo = mid + 1;
      flo = fm;
    } else {
      hi = mid;
      fhi = fm;
    }
  }
  *kstar = lo;
  return fmaxf(flo, fminf(__fmaf_rn(t, float(W - 2 * lo), x), fhi));
}

// Primal step of the light path: a thread per leaf, single entries only, the
// prox by prox_hinted.  A thread past the end re-reads the last leaf and
// writes nothing; a list leaf's lane gathers its own p (harmless) and writes
// nothing.
template <typename T>
__device__ __forceinline__ void primal_light(const View& v, float* __restrict__ u,
                                             float* __restrict__ ubar, const float* __restrict__ p,
                                             const float* __restrict__ tau,
                                             const uint32_t* __restrict__ soff,
                                             const T* __restrict__ samp, float gamma,
                                             uint16_t* __restrict__ khint, int b) {
  const size_t st = size_t(v.stride);
  const int64_t l = int64_t(b) * kThreads + threadIdx.x;
  const int64_t lc = l < v.n ? l : v.n - 1;
  int32_t e[6];
#pragma unroll
  for (int f = 0; f < 6; ++f) e[f] = v.nbr[f * st + lc];
  const int lev = v.level[lc];
  const float tl = tau[lc];
  const uint32_t o = soff[lc];
  const int W = int(soff[lc + 1] - o);
  // the structure arrays above are read before the previous kernel ends;
  // u, p and the hint only after it
  grid_dep_wait();
  grid_dep_launch();
  const float ul = u[lc];
  float q[3], pn[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) q[d] = p[d * st + lc];
#pragma unroll
  for (int d = 0; d < 3; ++d) pn[d] = p[d * st + (e[3 + d] >= 0 ? entry_idx(e[3 + d]) : 0u)];
  const int kh = min(int(khint[lc]), W);
  const float h = edge_f(v.D, lev);
  float dv = 0.0f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float hm = edge_f(v.D, e[d] >= 0 ? entry_level(e[d]) : lev);
    dv += (e[d] >= 0 ? inv_delta(h, hm) : 0.0f) * q[d];
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    // same or coarser n: (h_n^3 / h^3) (h / h_n)^2 / Delta = (h_n / h) / Delta
    const float hn = edge_f(v.D, e[3 + d] >= 0 ? entry_level(e[3 + d]) : lev);
    dv -= e[3 + d] >= 0 ? (hn / h) * inv_delta(h, hn) * pn[d] : 0.0f;
  }
  bool skip = l >= v.n;
#pragma unroll
  for (int f = 0; f < 6; ++f) skip |= is_list(e[f]);
  const float x = ul + tl * dv;
  const float t = tl / (float(W) + gamma);
  int ks = 0;
  const float pr = skip ? 0.0f : prox_hinted(samp + o, W, x, t, kh, &ks);
  if (skip) return;
  const float un = fminf(fmaxf(pr, -1.0f), 1.0f);
  u[l] = un;
  ubar[l] = 2.0f * un - ul;
  khint[l] = uint16_t(ks);
}

// A primal step of the leaves of a compacted set (heavy or list leaves), G
// lanes per leaf: the j-th leaf of `set` (group position g0 + j) for threads
// j G .. j G + G - 1 of the segment starting at block 0 + `b`.  The leaf's
// -face neighbours come from its divergence records, static between
// restructures and so read before the wait together with the +face weight
// sums; after it the lanes gather p at the neighbours, the group sums, and
// lane 0 runs the prox search from the hint.  Lanes past the end take the
// last leaf and do not write (every lane of the warp joins the shuffles).
template <int G, typename T>
__device__ __forceinline__ void primal_group(const View& v, float* __restrict__ u,
                                             float* __restrict__ ubar, const float* __restrict__ p,
                                             const float* __restrict__ tau,
                                             const uint32_t* __restrict__ soff,
                                             const T* __restrict__ samp, float gamma,
                                             uint16_t* __restrict__ khint, const NbrRecs& dr,
                                             const uint32_t* __restrict__ set, int n_set, int g0,
                                             int b) {
  const size_t st = size_t(v.stride);
  const int t = b * kThreads + int(threadIdx.x);
  const int j = t / G, lane = t % G;
  const bool valid = j < n_set;
  const int jc = valid ? j : n_set - 1;
  const int64_t l = set[jc];
  const int g = g0 + jc;
  const uint32_t m0 = dr.start[g], m1 = dr.start[g + 1];
  float cp[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) cp[d] = dr.cp[3 * g + d];
  const float tl = tau[l];
  const uint32_t o = soff[l];
  const int W = int(soff[l + 1] - o);
  uint32_t rec[kRecBatch];
  float w[kRecBatch];
#pragma unroll
  for (int r = 0; r < kRecBatch; ++r) {
    const uint32_t k = m0 + lane + r * G;
    rec[r] = k < m1 ? dr.rec[k] : 0u;
    w[r] = k < m1 ? dr.w[k] : 0.0f;
  }
  grid_dep_wait();
  grid_dep_launch();
  float acc = 0.0f;
#pragma unroll
  for (int r = 0; r < kRecBatch; ++r)
    acc += w[r] * p[size_t(rec[r] >> 28) * st + (rec[r] & 0x0fffffffu)];
#pragma unroll 4
  for (uint32_t k = m0 + lane + kRecBatch * G; k < m1; k += G) {
    const uint32_t rk = dr.rec[k];
    acc += dr.w[k] * p[size_t(rk >> 28) * st + (rk & 0x0fffffffu)];
  }
  acc = group_sum<G>(acc);
  if (lane != 0 || !valid) return;
  const float ul = u[l];
  const float dv = cp[0] * p[l] + cp[1] * p[st + l] + cp[2] * p[2 * st + l] - acc;
  int ks;
  const float un = fminf(fmaxf(prox_hinted(samp + o, W, ul + tl * dv, tl / (float(W) + gamma),
                                           min(int(khint[l]), W), &ks),
                               -1.0f),
                         1.0f);
  u[l] = un;
  ubar[l] = 2.0f * un - ul;
  khint[l] = uint16_t(ks);
}

// Neighbour records (see NbrRecs) of a leaf set: PLUS the +face neighbours
// with alpha / Delta (gradient of the dual step), else the -face neighbours
// with (h_n^3 / h^3) alpha_nl / Delta and the +face weight sums (divergence
// of the primal step).  Counts first, then the records.
template <bool PLUS>
__global__ void k_recs_count(View v, LeafSets ls, uint32_t* __restrict__ cnt) {
  const int g = int(blockIdx.x) * blockDim.x + int(threadIdx.x);
  if (g >= ls.n_heavy + ls.n_list) return;
  const int64_t l = g < ls.n_heavy ? ls.heavy[g] : ls.list[g - ls.n_heavy];
  uint32_t c = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int32_t e = v.nbr[int64_t(PLUS ? d : 3 + d) * v.stride + l];
    c += e >= 0 ? 1u : (e == kEmpty ? 0u : uint32_t(v.ovf[list_start(e)]));
  }
  cnt[g] = c;
}

// A warp per group position: lanes share each face list (records written
// in list order, the +face weight sums reduced in a fixed order).
template <bool PLUS>
__global__ void k_recs_fill(View v, LeafSets ls, const uint32_t* __restrict__ start,
                            uint32_t* __restrict__ rec, float* __restrict__ w,
                            float* __restrict__ cp) {
  const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = int(threadIdx.x & 31);
  if (gw >= ls.n_heavy + ls.n_list) return;   // the whole warp
  const int g = int(gw);
  const int64_t l = g < ls.n_heavy ? ls.heavy[g] : ls.list[g - ls.n_heavy];
  const int32_t* __restrict__ ovf = v.ovf;
  const float h = edge_f(v.D, v.level[l]);
  if (!PLUS) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int32_t e = v.nbr[int64_t(d) * v.stride + l];
      float sum = 0.0f;
      if (e >= 0) {
        if (lane == 0) sum = plus_weight(h, edge_f(v.D, entry_level(e)));
      } else if (e != kEmpty) {
        const uint32_t s0 = list_start(e);
        const int c = ovf[s0];
        for (int k = lane; k < c; k += 32) sum += plus_weight(h, edge_f(v.D, entry_level(ovf[s0 + 1 + k])));
      }
      sum = group_sum<32>(sum);
      if (lane == 0) cp[3 * g + d] = sum;
    }
  }
  auto weight = [&](int32_t f) {
    const float hm = edge_f(v.D, entry_level(f));
    return PLUS ? plus_weight(h, hm) : minus_weight(h, hm);
  };
  uint32_t k0 = start[g];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int32_t e = v.nbr[int64_t(PLUS ? d : 3 + d) * v.stride + l];
    if (e >= 0) {
      if (lane == 0) {
        rec[k0] = entry_idx(e) | (uint32_t(d) << 28);
        w[k0] = weight(e);
      }
      k0 += 1;
    } else if (e != kEmpty) {
      const uint32_t s0 = list_start(e);
      const int c = ovf[s0];
      for (int i = lane; i < c; i += 32) {
        const int32_t f = ovf[s0 + 1 + i];
        rec[k0 + i] = entry_idx(f) | (uint32_t(d) << 28);
        w[k0 + i] = weight(f);
      }
      k0 += uint32_t(c);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads, kIterMinBlocks) k_primal(View v, float* __restrict__ u,
                                                                     float* __restrict__ ubar,
                                                                     const float* __restrict__ p,
                                                                     const float* __restrict__ tau,
                                                                     const uint32_t* __restrict__ soff,
                                                                     const T* __restrict__ samp,
                                                                     float gamma,
                                                                     uint16_t* __restrict__ khint,
                                                                     Segments sg, NbrRecs dr) {
  const int hb = heavy_blocks(sg);
  const int lb = (sg.n_list * kPrimalListLanes + kThreads - 1) / kThreads;
  const int b = int(blockIdx.x);
  if (b < hb + lb) {
    if (b < hb)
      primal_group<kHeavyLanes>(v, u, ubar, p, tau, soff, samp, gamma, khint, dr, sg.heavy,
                                sg.n_heavy, 0, b);
    else
      primal_group<kPrimalListLanes>(v, u, ubar, p, tau, soff, samp, gamma, khint, dr, sg.list,
                                     sg.n_list, sg.n_heavy, b - hb);
    return;
  }
  primal_light(v, u, ubar, p, tau, soff, samp, gamma, khint, b - (hb + lb));
}

// ---------------------------------------------------------------------------
// Energy.  Per leaf, with c = 1 / (W + gamma) and volume h^3:
//   primal  h^3 [c sum_k |u - f_k| + lambda |grad u|]
//   dual    h^3 min_{x in [-1,1]} [c sum_k |x - f_k| - x div p]
// The dual minimum of the convex piecewise-linear function sits where its
// slope c (2k - W) - div p turns non-negative: at f_k for the first such k,
// at -1 if already for k = 0, at +1 if never.
//
// Precision.  GB300 issues float64 at a small fraction of its float32 rate,
// so per-leaf float64 arithmetic (about a hundred operations a leaf) made this
// reduction compute-bound.  The per-leaf terms are therefore evaluated in
// float-float arithmetic: a value is an unevaluated sum hi + lo of two
// float32s, kept exact by the error-free transformations TwoSum (Knuth) and
// TwoProduct (Dekker, with a fused multiply-add), which carries about 44
// significant bits, near float64's 53 and far below the energy's tolerance.
// Each thread accumulates its leaves in float-float; the block partials and
// the final sum are float64 in a fixed order, so the result is reproducible.

// float-float value hi + lo with |lo| <= ulp(hi) (not necessarily rounded)
struct ff {
  float hi, lo;
};

// a + b = s + e exactly (Knuth's TwoSum, no ordering needed)
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// a + b = s + e exactly when |a| >= |b| or a = 0 (Dekker's FastTwoSum)
__device__ __forceinline__ ff ff_fast_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a b = p + e exactly (barring underflow) with one fused multiply-add
__device__ __forceinline__ ff ff_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff ff_add(ff x, ff y) {
  const ff s = ff_two_sum(x.hi, y.hi);
  return ff_fast_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ ff ff_neg(ff x) { return {-x.hi, -x.lo}; }

// x 2^k, exact (p2 a power of two, no overflow or underflow)
__device__ __forceinline__ ff ff_scale(ff x, float p2) { return {x.hi * p2, x.lo * p2}; }

__device__ __forceinline__ ff ff_mul_f(ff x, float b) {
  const ff p = ff_two_prod(x.hi, b);
  return ff_fast_sum(p.hi, __fmaf_rn(x.lo, b, p.lo));
}

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
  const ff p = ff_two_prod(x.hi, y.hi);
  return ff_fast_sum(p.hi, __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo)));
}

// sqrt(x) for x >= 0: s within a few ulps of sqrt(hi) (hi rsqrt(hi); the
// correctly rounded root below 2^-100, where the approximation loses
// precision), then one Newton correction (x - s^2) / (2 s), where hi - s^2
// is exact (the two are within a factor 2).
__device__ __forceinline__ ff ff_sqrt(ff x) {
  if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
  const float s = x.hi >= 0x1p-100f ? x.hi * rsqrtf(x.hi) : __fsqrt_rn(x.hi);
  const ff sq = ff_two_prod(s, s);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, sq.hi), sq.lo), x.lo);
  return ff_fast_sum(s, __fdividef(r, 2.0f * s));
}

// 1 / x for x > 0: r within a few ulps of 1 / hi, then r + r (1 - x r),
// where 1 - x r is formed from the exact product.
__device__ __forceinline__ ff ff_recip(ff x) {
  const float r = __fdividef(1.0f, x.hi);
  const ff xr = ff_mul_f(x, r);
  const float e = __fsub_rn(__fsub_rn(1.0f, xr.hi), xr.lo);
  return ff_fast_sum(r, __fmul_rn(r, e));
}

// d as a pair (host side: kernel arguments)
inline ff ff_split(double d) {
  const float hi = float(d);
  return {hi, float(d - double(hi))};
}

__device__ __forceinline__ double ff_double(ff x) { return double(x.hi) + double(x.lo); }


// 1 / (1 + 2^d), d = 0..15, split into a float pair: 1 / Delta for leaves of
// edges 2^a and 2^b is 2^(1 - min(a, b)) / (1 + 2^|a - b|).
constexpr double inv_one_plus_pow2(int d) { return 1.0 / (1.0 + double(1 << d)); }
constexpr float inv_hi(int d) { return float(inv_one_plus_pow2(d)); }
constexpr float inv_lo(int d) { return float(inv_one_plus_pow2(d) - double(inv_hi(d))); }
__constant__ float kInvHi[16] = {inv_hi(0),  inv_hi(1),  inv_hi(2),  inv_hi(3),  inv_hi(4),  inv_hi(5),
                                 inv_hi(6),  inv_hi(7),  inv_hi(8),  inv_hi(9),  inv_hi(10), inv_hi(11),
                                 inv_hi(12), inv_hi(13), inv_hi(14), inv_hi(15)};
__constant__ float kInvLo[16] = {inv_lo(0),  inv_lo(1),  inv_lo(2),  inv_lo(3),  inv_lo(4),  inv_lo(5),
                                 inv_lo(6),  inv_lo(7),  inv_lo(8),  inv_lo(9),  inv_lo(10), inv_lo(11),
                                 inv_lo(12), inv_lo(13), inv_lo(14), inv_lo(15)};

// alpha / Delta 2^extra for the ordered pair (row leaf of edge exponent a,
// neighbour of edge exponent b) with alpha = min(1, (2^b / 2^a)^2): a table
// pair scaled by a power of two, so exact to the pair's precision.
__device__ __forceinline__ ff face_weight(int a, int b, int extra) {
  const int lo = a < b ? a : b;
  const int d = a < b ? b - a : a - b;
  const float s = pow2f(1 - lo + (b < a ? 2 * (b - a) : 0) + extra);
  return {kInvHi[d] * s, kInvLo[d] * s};
}

// alpha / Delta 2^extra for a single face neighbour, which is never finer
// (b >= a, alpha = 1): the table pair times 2^(1 - a + extra).
__device__ __forceinline__ ff single_weight(int a, int b, int extra) {
  const float s = pow2f(1 - a + extra);
  return {kInvHi[b - a] * s, kInvLo[b - a] * s};
}

// +face term of neighbour value um: alpha / Delta (um - ul), and the weight
__device__ __forceinline__ ff grad_term(int a, int b, float um, float ul, ff* w) {
  *w = face_weight(a, b, 0);
  return ff_mul(*w, ff_two_sum(um, -ul));
}

// -face term of neighbour value pn: (h_n^3 / h^3) alpha_nl / Delta pn
__device__ __forceinline__ ff div_term(int a, int b, float pn) {
  return ff_mul_f(face_weight(b, a, 3 * (b - a)), pn);
}

// Primal and dual terms of leaf l (edge exponent a) from its gradient g, the
// +face weight sums c and the -face sums m of the divergence, and p(l).
template <typename T>
__device__ __forceinline__ void leaf_terms(const uint32_t* __restrict__ soff,
                                           const T* __restrict__ samp, int64_t l, int a, float ul,
                                           const ff g[3], const ff c[3], const ff m[3],
                                           const float pl[3], ff lambda, ff gamma, ff* sp, ff* sd) {
  const ff g2 = ff_add(ff_add(ff_mul(g[0], g[0]), ff_mul(g[1], g[1])), ff_mul(g[2], g[2]));
  ff dv = ff_add(ff_mul_f(c[0], pl[0]), ff_neg(m[0]));
  dv = ff_add(dv, ff_add(ff_mul_f(c[1], pl[1]), ff_neg(m[1])));
  dv = ff_add(dv, ff_add(ff_mul_f(c[2], pl[2]), ff_neg(m[2])));
  const uint32_t o = soff[l];
  const int W = int(soff[l + 1] - o);
  const float Wf = float(W);
  const ff wg = ff_add({Wf, 0.0f}, gamma);
  const ff rc = ff_recip(wg);
  // dual term: first k with slope c (2k - W) - dv >= 0, i.e. k >= (W + dv / c) / 2;
  // the minimiser is -1 before the first sample, +1 after the last, else f_(k-1).
  // ceil of the pair q = (W + dv (W + gamma)) / 2: ceil(q.hi), plus one when
  // q.hi is an integer and q.lo > 0 (|q.lo| is below the distance from a
  // non-integer q.hi to the next integer).
  const ff q = ff_scale(ff_add({Wf, 0.0f}, ff_mul(dv, wg)), 0.5f);
  float kk = ceilf(q.hi);
  if (kk == q.hi && q.lo > 0.0f) kk += 1.0f;
  const int mx = kk <= 0.0f ? 0 : (kk > Wf ? W : int(kk) - 1);
  const float xs = kk <= 0.0f ? -1.0f : (kk > Wf ? 1.0f : load_sample(samp, o + mx));
  // With the samples sorted, sum_k |x - f_k| = x (2 m - W) + sum_k f_k - 2 sum_{k<m} f_k for
  // any m splitting them into f_k <= x (k < m) and f_k >= x (k >= m).  One pass gives
  // the total and the two prefix sums (m = #{f_k < u} for the primal term, m = mx for
  // the dual term), each a TwoSum pair.
  float th = 0.0f, tl = 0.0f, uh = 0.0f, ulo = 0.0f, xh = 0.0f, xl = 0.0f;
  int mu = W;
  for (int k = 0; k < W; ++k) {
    const float f = load_sample(samp, o + k);
    if (mu == W && !(f < ul)) {
      mu = k;
      uh = th;
      ulo = tl;
    }
    if (k == mx) {
      xh = th;
      xl = tl;
    }
    const ff s = ff_two_sum(th, f);
    th = s.hi;
    tl = __fadd_rn(tl, s.lo);
  }
  if (mu == W) {
    uh = th;
    ulo = tl;
  }
  if (mx == W) {
    xh = th;
    xl = tl;
  }
  const ff tot = ff_two_sum(th, tl);
  const ff data = ff_add(ff_add(ff_two_prod(ul, float(2 * mu - W)), tot),
                         ff_scale(ff_two_sum(uh, ulo), -2.0f));
  const ff dd = ff_add(ff_add(ff_two_prod(xs, float(2 * mx - W)), tot),
                       ff_scale(ff_two_sum(xh, xl), -2.0f));
  const float vol = pow2f(3 * a);
  *sp = ff_add(*sp, ff_scale(ff_add(ff_mul(rc, data), ff_mul(lambda, ff_sqrt(g2))), vol));
  *sd = ff_add(*sd, ff_scale(ff_add(ff_mul(rc, dd), ff_neg(ff_mul_f(dv, xs))), vol));
}

// Sum over the G lanes of a group of one pair (groups aligned in the warp;
// every lane of the warp takes part; lane 0's sum is in a fixed order).
template <int G>
__device__ __forceinline__ ff group_sum_ff(ff x) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1)
    x = ff_add(x, ff{__shfl_xor_sync(kFull, x.hi, o), __shfl_xor_sync(kFull, x.lo, o)});
  return x;
}

// Block sum of one pair per thread: each warp's sum in float-float, then the
// warps' sums in float64 in a fixed order (the result is thread 0's).
__device__ __forceinline__ double block_sum_ff(ff x, double* red) {
  x = group_sum_ff<32>(x);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ff_double(x);
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
  return t;
}

// Energy terms of a light leaf l (single entries on every face): the six
// neighbour values are gathered first (an empty face gathers l's own, unused).
template <typename T>
__device__ __forceinline__ void light_energy(const View& v, const float* __restrict__ u,
                                             const float* __restrict__ p,
                                             const uint32_t* __restrict__ soff,
                                             const T* __restrict__ samp, ff lambda, ff gamma,
                                             int64_t l, const int32_t e[6], ff* sp, ff* sd) {
  const size_t st = size_t(v.stride);
  const int a = v.D - v.level[l];
  const float ul = u[l];
  const float pl[3] = {p[l], p[st + l], p[2 * st + l]};
  float x[6];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    x[d] = u[e[d] >= 0 ? entry_idx(e[d]) : uint32_t(l)];
    x[3 + d] = p[d * st + (e[3 + d] >= 0 ? entry_idx(e[3 + d]) : uint32_t(l))];
  }
  ff g[3], c[3], m[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const ff zero{0.0f, 0.0f};
    const int bp = e[d] >= 0 ? v.D - entry_level(e[d]) : a;
    const ff w = single_weight(a, bp, 0);
    g[d] = e[d] >= 0 ? ff_mul(w, ff_two_sum(x[d], -ul)) : zero;
    c[d] = e[d] >= 0 ? w : zero;
    // (h_n^3 / h^3) alpha_nl / Delta = (h_n / h) / Delta for a neighbour n
    // of the same size or coarser
    const int bn = e[3 + d] >= 0 ? v.D - entry_level(e[3 + d]) : a;
    m[d] = e[3 + d] >= 0 ? ff_mul_f(single_weight(a, bn, bn - a), x[3 + d]) : zero;
  }
  leaf_terms(soff, samp, l, a, ul, g, c, m, pl, lambda, gamma, sp, sd);
}

// Energy terms of leaf l, its slots spread over a group of G lanes: the
// gradient of u (+faces) and divergence of p (both sides), reduced over the
// group; lane 0 adds the leaf's primal and dual terms to sp, sd when `valid`.
template <int G, typename T>
__device__ __forceinline__ void group_energy(const View& v, const float* __restrict__ u,
                                             const float* __restrict__ p,
                                             const uint32_t* __restrict__ soff,
                                             const T* __restrict__ samp, ff lambda, ff gamma,
                                             int64_t l, int lane, bool valid, ff* sp, ff* sd) {
  int32_t e[6];
#pragma unroll
  for (int f = 0; f < 6; ++f) e[f] = v.nbr[int64_t(f) * v.stride + l];
  const int a = v.D - v.level[l];
  const float ul = u[l];
  const ff zero{0.0f, 0.0f};
  ff g[3] = {zero, zero, zero}, c[3] = {zero, zero, zero}, m[3] = {zero, zero, zero};
  // face by face (unrolled, so each sum is a register): this lane takes the
  // entries lane, lane + G, ... of the face's list, or the single entry on lane 0
  int cnt[6];
#pragma unroll
  for (int f = 0; f < 6; ++f)
    cnt[f] = e[f] >= 0 ? 1 : (e[f] == kEmpty ? 0 : v.ovf[list_start(e[f])]);
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int32_t* lst = e[f] >= 0 ? nullptr : v.ovf + list_start(e[f]) + 1;
    for (int k = lane; k < cnt[f]; k += G) {
      const int32_t ent = e[f] >= 0 ? e[f] : lst[k];
      const int b = v.D - entry_level(ent);
      if (f < 3) {
        ff w;
        const ff t = grad_term(a, b, u[entry_idx(ent)], ul, &w);
        g[f] = ff_add(g[f], t);
        c[f] = ff_add(c[f], w);
      } else {
        m[f - 3] = ff_add(m[f - 3], div_term(a, b, p[int64_t(f - 3) * v.stride + entry_idx(ent)]));
      }
    }
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    g[d] = group_sum_ff<G>(g[d]);
    c[d] = group_sum_ff<G>(c[d]);
    m[d] = group_sum_ff<G>(m[d]);
  }
  if (lane != 0 || !valid) return;
  const float pl[3] = {p[l], p[v.stride + l], p[2 * v.stride + l]};
  leaf_terms(soff, samp, l, a, ul, g, c, m, pl, lambda, gamma, sp, sd);
}

constexpr int kEnergyListLanes = 4;

// Launch layout: hb blocks of heavy leaves (a warp per leaf, strided over
// the heavy set), lb blocks of list leaves (kEnergyListLanes lanes per leaf,
// strided over the list set), then light leaves (a thread each, strided over
// all leaves, skipping those with a finer-neighbour list).  Each thread sums
// its leaves in float-float; each block writes its (primal, dual) partial in
// float64; all sums are in a fixed order.
template <typename T>
__global__ void __launch_bounds__(kThreads, 4) k_energy(View v, const float* __restrict__ u,
                                                        const float* __restrict__ p,
                                                        const uint32_t* __restrict__ soff,
                                                        const T* __restrict__ samp, ff lambda,
                                                        ff gamma, Segments sg, int hb, int lb,
                                                        double* __restrict__ partial) {
  __shared__ double red[kThreads / 32];
  ff sp{0.0f, 0.0f}, sd{0.0f, 0.0f};
  const int b = int(blockIdx.x);
  if (b < hb) {
    const int w = b * (kThreads / 32) + int(threadIdx.x >> 5), nw = hb * (kThreads / 32);
    for (int q = w; q < sg.n_heavy; q += nw)
      group_energy<32>(v, u, p, soff, samp, lambda, gamma, sg.heavy[q], int(threadIdx.x & 31), true,
                       &sp, &sd);
  } else if (b < hb + lb) {
    constexpr int G = kEnergyListLanes;
    const int t = (b - hb) * kThreads + int(threadIdx.x);
    const int gi = t / G, ng = lb * (kThreads / G);
    const int rounds = (sg.n_list + ng - 1) / ng;   // the same in every lane
    for (int r = 0; r < rounds; ++r) {
      const int q = gi + r * ng;
      const bool valid = q < sg.n_list;
      group_energy<G>(v, u, p, soff, samp, lambda, gamma, sg.list[valid ? q : sg.n_list - 1], t % G,
                      valid, &sp, &sd);
    }
  } else {
    const int nb = int(gridDim.x) - hb - lb;
    for (int64_t l = int64_t(b - hb - lb) * blockDim.x + threadIdx.x; l < v.n;
         l += int64_t(nb) * blockDim.x) {
      int32_t e[6];
      bool listed = false;
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        e[f] = v.nbr[int64_t(f) * v.stride + l];
        listed |= is_list(e[f]);
      }
      if (listed) continue;   // summed by a heavy or list group
      light_energy(v, u, p, soff, samp, lambda, gamma, l, e, &sp, &sd);
    }
  }
  // block partial in a fixed order
  const double bp = block_sum_ff(sp, red);
  const double bd = block_sum_ff(sd, red);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = bp;
    partial[2 * blockIdx.x + 1] = bd;
  }
}

// Fixed-order sum of nb partial pairs by one block of kFinalThreads threads:
// thread t adds partials t, t + kFinalThreads, ...; then a tree over threads.
constexpr int kFinalThreads = 256;

__global__ void __launch_bounds__(kFinalThreads) k_energy_final(const double* __restrict__ partial,
                                                                int nb, double* __restrict__ out3) {
  __shared__ double ra[kFinalThreads], rb[kFinalThreads];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nb; i += kFinalThreads) {
    a += partial[2 * i];
    b += partial[2 * i + 1];
  }
  ra[threadIdx.x] = a;
  rb[threadIdx.x] = b;
  __syncthreads();
  for (int s = kFinalThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      ra[threadIdx.x] += ra[threadIdx.x + s];
      rb[threadIdx.x] += rb[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out3[0] = ra[0];
    out3[1] = rb[0];
    out3[2] = ra[0] - rb[0];
  }
}

constexpr int kEnergyBlocks = 8192;

inline unsigned blocks_for(int64_t n, int threads) { return unsigned((n + threads - 1) / threads); }

}  // namespace

// The iteration kernels are launched with programmatic dependent launch
// (see grid_dep_wait): a kernel's launch, block start-up and structure reads
// overlap the tail of the kernel before it.
constexpr bool kIterPDL = true;

template <typename... KArgs, typename... Args>
cudaError_t launch_iter(void (*kernel)(KArgs...), unsigned grid, cudaStream_t s, Args... args) {
  if (!kIterPDL) {
    kernel<<<grid, kThreads, 0, s>>>(args...);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

inline unsigned grid_of(int64_t n, const Segments& sg, int list_lanes, int light_leaves) {
  return blocks_for(n, kThreads * light_leaves) +
         blocks_for(int64_t(sg.n_list) * list_lanes, kThreads) + unsigned(heavy_blocks(sg));
}

cudaError_t launch_dual(View v, const float* ubar, float* p, const float* sigma, float lambda,
                        LeafSets ls, NbrRecs gr, cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  const Segments sg{ls.heavy, ls.n_heavy, ls.list, ls.n_list};
  const cudaError_t e = launch_iter(k_dual<false>, grid_of(v.n, sg, kDualListLanes, kDualLightLeaves),
                                    s, v, ubar, p, sigma, lambda, sg, 0.0f, gr);
  count_launches(1);
  return e;
}

cudaError_t launch_dual_init(View v, const float* u, float* p, float lambda, float g0, LeafSets ls,
                             NbrRecs gr, cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  const Segments sg{ls.heavy, ls.n_heavy, ls.list, ls.n_list};
  k_dual<true><<<grid_of(v.n, sg, kDualListLanes, kDualLightLeaves), kThreads, 0, s>>>(v, u, p, nullptr,
                                                                                        lambda, sg, g0, gr);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_primal(View v, float* u, float* ubar, const float* p, const float* tau,
                          const uint32_t* soff, const void* samp, bool fp16, float gamma,
                          uint16_t* khint, LeafSets ls, NbrRecs dr, cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  const Segments sg{ls.heavy, ls.n_heavy, ls.list, ls.n_list};
  const unsigned nb = grid_of(v.n, sg, kPrimalListLanes, 1);
  const cudaError_t e =
      fp16 ? launch_iter(k_primal<__half>, nb, s, v, u, ubar, p, tau, soff,
                         reinterpret_cast<const __half*>(samp), gamma, khint, sg, dr)
           : launch_iter(k_primal<float>, nb, s, v, u, ubar, p, tau, soff,
                         reinterpret_cast<const float*>(samp), gamma, khint, sg, dr);
  count_launches(1);
  return e;
}

cudaError_t launch_recs_count(View v, LeafSets ls, bool plus, uint32_t* cnt, cudaStream_t s) {
  const int ng = ls.n_heavy + ls.n_list;
  if (ng == 0) return cudaSuccess;
  if (plus)
    k_recs_count<true><<<blocks_for(ng, kThreads), kThreads, 0, s>>>(v, ls, cnt);
  else
    k_recs_count<false><<<blocks_for(ng, kThreads), kThreads, 0, s>>>(v, ls, cnt);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_recs_fill(View v, LeafSets ls, bool plus, const uint32_t* start, uint32_t* rec,
                             float* w, float* cp, cudaStream_t s) {
  const int ng = ls.n_heavy + ls.n_list;
  if (ng == 0) return cudaSuccess;
  const unsigned nb = blocks_for(int64_t(ng) * 32, kThreads);
  if (plus)
    k_recs_fill<true><<<nb, kThreads, 0, s>>>(v, ls, start, rec, w, cp);
  else
    k_recs_fill<false><<<nb, kThreads, 0, s>>>(v, ls, start, rec, w, cp);
  count_launches(1);
  return cudaGetLastError();
}

size_t energy_tmp_bytes(int64_t) { return size_t(2 * kEnergyBlocks) * sizeof(double); }

// Grid of k_energy: at most 128 blocks of heavy warps and 1024 of list
// groups (both strided over their sets), then light blocks of up to
// `per_light_block` leaves each (strided), max_blocks in all.
struct EnergyLayout {
  int hb, lb, nb;
};

inline EnergyLayout energy_layout(int64_t n, const Segments& sg, int64_t per_light_block,
                                  int max_blocks) {
  EnergyLayout g;
  g.hb = int(std::min<int64_t>((int64_t(sg.n_heavy) * 32 + kThreads - 1) / kThreads, 128));
  g.lb = int(std::min<int64_t>((int64_t(sg.n_list) * kEnergyListLanes + kThreads - 1) / kThreads, 1024));
  const int64_t want = (n + per_light_block - 1) / per_light_block;
  const int64_t room = max_blocks - g.hb - g.lb;
  g.nb = g.hb + g.lb + int(std::max<int64_t>(1, std::min<int64_t>(want, room)));
  return g;
}

template <typename T>
void energy_launch(EnergyLayout g, View v, const float* u, const float* p, const uint32_t* soff,
                   const void* samp, double lambda, double gamma, Segments sg, double* partial,
                   cudaStream_t s) {
  k_energy<T><<<g.nb, kThreads, 0, s>>>(v, u, p, soff, reinterpret_cast<const T*>(samp),
                                        ff_split(lambda), ff_split(gamma), sg, g.hb, g.lb, partial);
}

cudaError_t launch_energy(View v, const float* u, const float* p, const uint32_t* soff,
                          const void* samp, bool fp16, double lambda, double gamma, LeafSets ls,
                          double* partial, double* out3, cudaStream_t s) {
  const Segments sg{ls.heavy, ls.n_heavy, ls.list, ls.n_list};
  // light blocks: one wave of resident blocks (4 per SM), strided over the leaves
  const int64_t wave = int64_t(sm_count()) * 4;
  const int64_t per = std::max<int64_t>(kThreads, (v.n + wave - 1) / wave);
  const EnergyLayout g = energy_layout(v.n, sg, per, kEnergyBlocks);
  if (fp16)
    energy_launch<__half>(g, v, u, p, soff, samp, lambda, gamma, sg, partial, s);
  else
    energy_launch<float>(g, v, u, p, soff, samp, lambda, gamma, sg, partial, s);
  count_launches(1);
  k_energy_final<<<1, kFinalThreads, 0, s>>>(partial, g.nb, out3);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Energy without allocation: the same per-leaf energy kernel, its block
// partials and the three results kept in a file-scope device array instead of
// context memory.  Each block covers up to kStaticLeavesPerBlock leaves, so
// the array bounds the leaf count.

namespace {
constexpr int kStaticEnergyBlocks = 8192;
constexpr int64_t kStaticLeavesPerBlock = int64_t(kThreads) * 8;
}  // namespace

// [2 * kStaticEnergyBlocks] block partials, then [3] primal, dual, gap.
// Shared by every call in the process; each call overwrites what it reads.
static __device__ __align__(256) double g_energy_scratch[2 * kStaticEnergyBlocks + 3];

int64_t energy_static_max_leaves() { return int64_t(kStaticEnergyBlocks) * kStaticLeavesPerBlock; }

cudaError_t energy_static_scratch(double** ptr) {
  // Host code cannot use the array's name as a device address: look the
  // address up with the device current.  The lookup is repeated on every call
  // (it allocates nothing) so that a module reloaded after cudaDeviceReset is
  // never written through a stale address.
  void* a = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&a, g_energy_scratch);
  if (e != cudaSuccess) return e;
  *ptr = static_cast<double*>(a);
  return cudaSuccess;
}

cudaError_t launch_energy_static(View v, const float* u, const float* p, const uint32_t* soff,
                                 const void* samp, bool fp16, double lambda, double gamma,
                                 LeafSets ls, double* scratch, cudaStream_t s) {
  const int64_t want = (v.n + kStaticLeavesPerBlock - 1) / kStaticLeavesPerBlock;
  if (want > kStaticEnergyBlocks) return cudaErrorInvalidValue;
  const Segments sg{ls.heavy, ls.n_heavy, ls.list, ls.n_list};
  const EnergyLayout g = energy_layout(v.n, sg, kStaticLeavesPerBlock, kStaticEnergyBlocks);
  if (fp16)
    energy_launch<__half>(g, v, u, p, soff, samp, lambda, gamma, sg, scratch, s);
  else
    energy_launch<float>(g, v, u, p, soff, samp, lambda, gamma, sg, scratch, s);
  count_launches(1);
  k_energy_final<<<1, kFinalThreads, 0, s>>>(scratch, g.nb, scratch + 2 * kStaticEnergyBlocks);
  count_launches(1);
  return cudaGetLastError();
}

int energy_static_result_offset() { return 2 * kStaticEnergyBlocks; }

}  // namespace ofu
