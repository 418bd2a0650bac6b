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

// Gradient of ubar at leaf l over its +face slots, this lane's share of a
// group of G lanes (every neighbour term alpha (ubar_m - ubar_l) / Delta).
__device__ __forceinline__ void grad_share(const View& v, const float* __restrict__ ubar, int64_t l,
                                           const int32_t e[3], float h, float ul, int lane, int G,
                                           float acc[3]) {
  acc[0] = acc[1] = acc[2] = 0.0f;
  for_each_slot<3>(v, e, lane, G, [&](int f, int32_t ent) {
    const float t = plus_weight(h, edge_f(v.D, entry_level(ent))) * (ubar[entry_idx(ent)] - ul);
    acc[0] += f == 0 ? t : 0.0f;
    acc[1] += f == 1 ? t : 0.0f;
    acc[2] += f == 2 ? t : 0.0f;
  });
}

// Lanes per list leaf of the dual and primal steps (measured over 1..16: 4
// and 2 fastest on the 256^3 and 512^3 workloads; the primal step has about
// twice as many list leaves, six faces and its prox).
constexpr int kDualListLanes = 4;
constexpr int kPrimalListLanes = 2;
// Lanes per heavy leaf (a face list longer than kHeavy): one warp.
constexpr int kHeavyLanes = 32;
// Slots a lane of the primal step loads per round (registers allow 2 there).
constexpr int kPrimalSlotBatch = 2;

// Blocks of the heavy segment (kHeavyLanes lanes per heavy leaf).
__device__ __host__ __forceinline__ int heavy_blocks(const Segments& sg) {
  return (sg.n_heavy * kHeavyLanes + kThreads - 1) / kThreads;
}

// A dual step of the leaves of a compacted set (heavy or list leaves), G
// lanes per leaf: the j-th leaf of `set` for threads j G .. j G + G - 1 of
// the segment starting at block 0 + `b`.  Lanes past the end take the last
// leaf and do not write (every lane of the warp joins the shuffles).
template <bool INIT, int G>
__device__ __forceinline__ void dual_group(const View& v, const float* __restrict__ ubar,
                                           float* __restrict__ p, const float* __restrict__ sigma,
                                           float lambda, float g0, const uint32_t* __restrict__ set,
                                           int n_set, int b) {
  const size_t st = size_t(v.stride);
  const int t = b * kThreads + int(threadIdx.x);
  const int j = t / G, lane = t % G;
  const bool valid = j < n_set;
  const int64_t l = set[valid ? j : n_set - 1];
  const int32_t e[3] = {v.nbr[l], v.nbr[st + l], v.nbr[2 * st + l]};
  const float h = edge_f(v.D, v.level[l]);
  const float ul = ubar[l];
  float acc[3];
  grad_share(v, ubar, l, e, h, ul, lane, G, acc);
  float g[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) g[d] = group_sum<G>(acc[d]);
  if (lane != 0 || !valid) return;
  const float q[3] = {p[l], p[st + l], p[2 * st + l]};
  dual_finish<INIT>(p, st, l, q, INIT ? 0.0f : sigma[l], g, lambda, g0);
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
                                                                   float lambda, Segments sg, float g0) {
  const size_t st = size_t(v.stride);
  const int hb = heavy_blocks(sg);
  const int lb = (sg.n_list * kDualListLanes + kThreads - 1) / kThreads;
  const int b = int(blockIdx.x);
  if (b < hb + lb) {
    if (b < hb)
      dual_group<INIT, kHeavyLanes>(v, ubar, p, sigma, lambda, g0, sg.heavy, sg.n_heavy, b);
    else
      dual_group<INIT, kDualListLanes>(v, ubar, p, sigma, lambda, g0, sg.list, sg.n_list, b - hb);
    return;
  }
  const int lbase = hb + lb;
  // light path: one leaf per thread, single entries only; every load that does
  // not depend on another is issued before any branch
  const int64_t l = int64_t(b - lbase) * kThreads + threadIdx.x;
  if (l >= v.n) return;
  const int32_t e[3] = {v.nbr[l], v.nbr[st + l], v.nbr[2 * st + l]};
  const int lev = v.level[l];
  const float h = edge_f(v.D, lev);
  const float ul = ubar[l];
  const float q[3] = {p[l], p[st + l], p[2 * st + l]};
  const float sl = INIT ? 0.0f : sigma[l];
  // a list leaf's lane gathers its own value (harmless) and writes nothing
  float x[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) x[d] = ubar[e[d] >= 0 ? entry_idx(e[d]) : uint32_t(l)];
  float g[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float hm = edge_f(v.D, e[d] >= 0 ? entry_level(e[d]) : lev);
    g[d] = e[d] >= 0 ? (x[d] - ul) * inv_delta(h, hm) : 0.0f;
  }
  if (is_list(e[0]) || is_list(e[1]) || is_list(e[2])) return;
  dual_finish<INIT>(p, st, l, q, sl, g, lambda, g0);
}

// Prox of the data term: argmin_x (x - v)^2 / (2 tau) + c sum_k |x - f_k| is
// the median of {f_k} and {v + t (W - 2k)}_{k=0..W}, t = tau c.  With the
// samples sorted it is clamp(b_k*, f_(k*-1), f_k*) (0-based f, f_-1 = -inf,
// f_W = +inf) where k* is the number of k with f_k < b_k = v + t (W - 2k).
// That predicate holds exactly for a prefix of k (f rises, b falls, and the
// rounded b_k still falls), so k* is found by bisection in ceil(log2(W + 1))
// probes.  The last probe that held is f_(k*-1), the last that failed is
// f_k*, so no sample is loaded twice.
template <typename T>
__device__ __forceinline__ float prox_l1(const T* __restrict__ f, int W, float v, float t) {
  int lo = 0, hi = W;
  float flo = -CUDART_INF_F, fhi = CUDART_INF_F;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const float fm = load_sample(f, mid);
    if (fm < __fmaf_rn(t, float(W - 2 * mid), v)) {
      lo = mid + 1;
      flo = fm;
    } else {
      hi = mid;
      fhi = fm;
    }
  }
  const float b = __fmaf_rn(t, float(W - 2 * lo), v);
  return fmaxf(flo, fminf(b, fhi));
}

// Divergence of p at leaf l over its six faces' slots, this lane's share of
// a group of G lanes: +faces weigh p(l) by alpha / Delta per neighbour,
// -faces subtract (h_n^3 / h^3) alpha_nl / Delta p(n).
__device__ __forceinline__ float div_share(const View& v, const float* __restrict__ p, int64_t l,
                                           const int32_t e[6], float h, const float q[3], int lane,
                                           int G) {
  float acc = 0.0f;
  for_each_slot<6, kPrimalSlotBatch>(v, e, lane, G, [&](int f, int32_t ent) {
    const float hm = edge_f(v.D, entry_level(ent));
    if (f < 3) {
      acc += plus_weight(h, hm) * (f == 0 ? q[0] : (f == 1 ? q[1] : q[2]));
    } else {
      acc -= minus_weight(h, hm) * p[int64_t(f - 3) * v.stride + entry_idx(ent)];
    }
  });
  return acc;
}

// The prox of prox_l1 found by a group of G lanes: each round the lanes test
// G evenly spaced ranks of [lo, hi) and the count of those that hold (a prefix,
// the predicate being monotone) narrows the range, so a leaf of W samples
// takes about log_G(W) rounds of independent loads.  k* is the same as the
// bisection's, hence so is the result, in every lane.  The count is a warp
// ballot (every lane of the warp takes part in every round).
template <int G, typename T>
__device__ __forceinline__ float prox_l1_group(const T* __restrict__ f, int W, float v, float t,
                                               int lane) {
  static_assert(G >= 1 && G <= 32 && (G & (G - 1)) == 0, "G lanes of one warp");
  constexpr unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
  const unsigned gshift = (threadIdx.x & 31u) & ~unsigned(G - 1);
  int lo = 0, hi = W;
  for (;;) {
    const bool active = lo < hi;
    if (!__any_sync(kFull, active)) break;
    const int step = active ? (hi - lo + G - 1) / G : 0;
    const int q = lo + lane * step;
    const bool ok = active && q < hi && load_sample(f, q) < __fmaf_rn(t, float(W - 2 * q), v);
    const int c = __popc((__ballot_sync(kFull, ok) >> gshift) & gmask);
    if (active) {
      if (c == 0) {
        hi = lo;
      } else {
        const int last = lo + (c - 1) * step;   // the last rank that holds
        hi = min(hi, lo + c * step);             // the first that fails, if tested
        lo = last + 1;
      }
    }
  }
  const float flo = lo > 0 ? load_sample(f, lo - 1) : -CUDART_INF_F;
  const float fhi = lo < W ? load_sample(f, lo) : CUDART_INF_F;
  const float b = __fmaf_rn(t, float(W - 2 * lo), v);
  return fmaxf(flo, fminf(b, fhi));
}

template <typename T>
__device__ __forceinline__ void primal_finish(float* __restrict__ u, float* __restrict__ ubar,
                                              int64_t l, float ul, float tl, float dv, uint32_t o,
                                              int W, const T* __restrict__ samp, float gamma) {
  const float x = ul + tl * dv;
  const float t = tl / (float(W) + gamma);
  const float un = fminf(fmaxf(prox_l1(samp + o, W, x, t), -1.0f), 1.0f);
  u[l] = un;
  ubar[l] = 2.0f * un - ul;
}

// A primal step of the leaves of a compacted set, G lanes per leaf (layout
// as dual_group): the divergence over the slots and the prox by group search.
template <int G, typename T>
__device__ __forceinline__ void primal_group(const View& v, float* __restrict__ u,
                                             float* __restrict__ ubar, const float* __restrict__ p,
                                             const float* __restrict__ tau,
                                             const uint32_t* __restrict__ soff,
                                             const T* __restrict__ samp, float gamma,
                                             const uint32_t* __restrict__ set, int n_set, int b) {
  const int t = b * kThreads + int(threadIdx.x);
  const int j = t / G, lane = t % G;
  const bool valid = j < n_set;
  const int64_t l = set[valid ? j : n_set - 1];
  int32_t e[6];
#pragma unroll
  for (int f = 0; f < 6; ++f) e[f] = v.nbr[int64_t(f) * v.stride + l];
  const float h = edge_f(v.D, v.level[l]);
  float q[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) q[d] = p[int64_t(d) * v.stride + l];
  const uint32_t o = soff[l];
  const int W = int(soff[l + 1] - o);
  const float ul = u[l];
  const float tl = tau[l];
  const float dv = group_sum<G>(div_share(v, p, l, e, h, q, lane, G));
  float un = prox_l1_group<G>(samp + o, W, ul + tl * dv, tl / (float(W) + gamma), lane);
  if (lane != 0 || !valid) return;
  un = fminf(fmaxf(un, -1.0f), 1.0f);
  u[l] = un;
  ubar[l] = 2.0f * un - ul;
}

template <typename T>
__global__ void __launch_bounds__(kThreads, kIterMinBlocks) k_primal(View v, float* __restrict__ u,
                                                                     float* __restrict__ ubar,
                                                                     const float* __restrict__ p,
                                                                     const float* __restrict__ tau,
                                                                     const uint32_t* __restrict__ soff,
                                                                     const T* __restrict__ samp,
                                                                     float gamma, Segments sg) {
  const int hb = heavy_blocks(sg);
  const int lb = (sg.n_list * kPrimalListLanes + kThreads - 1) / kThreads;
  const int b = int(blockIdx.x);
  if (b < hb + lb) {
    if (b < hb)
      primal_group<kHeavyLanes>(v, u, ubar, p, tau, soff, samp, gamma, sg.heavy, sg.n_heavy, b);
    else
      primal_group<kPrimalListLanes>(v, u, ubar, p, tau, soff, samp, gamma, sg.list, sg.n_list,
                                     b - hb);
    return;
  }
  const int lbase = hb + lb;
  // light path: one leaf per thread, single entries only; every load that does
  // not depend on another is issued before any branch
  const int64_t l = int64_t(b - lbase) * kThreads + threadIdx.x;
  if (l >= v.n) return;
  int32_t e[6];
#pragma unroll
  for (int f = 0; f < 6; ++f) e[f] = v.nbr[int64_t(f) * v.stride + l];
  const int lev = v.level[l];
  const float h = edge_f(v.D, lev);
  float q[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) q[d] = p[int64_t(d) * v.stride + l];
  const float tl = tau[l];
  const float ul = u[l];
  const uint32_t o = soff[l];
  const int W = int(soff[l + 1] - o);
  // a list leaf's lane gathers its own p (harmless) and writes nothing
  float pn[3];
#pragma unroll
  for (int d = 0; d < 3; ++d)
    pn[d] = p[int64_t(d) * v.stride + (e[3 + d] >= 0 ? entry_idx(e[3 + d]) : uint32_t(l))];
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
  bool any = false;
#pragma unroll
  for (int f = 0; f < 6; ++f) any |= is_list(e[f]);
  if (any) return;
  primal_finish(u, ubar, l, ul, tl, dv, o, W, samp, gamma);
}

// ---------------------------------------------------------------------------
// Energy (float64).  Per leaf, with c = 1 / (W + gamma) and volume h^3:
//   primal  h^3 [c sum_k |u - f_k| + lambda |grad u|]
//   dual    h^3 min_{x in [-1,1]} [c sum_k |x - f_k| - x div p]
// The dual minimum of the convex piecewise-linear function sits where its
// slope c (2k - W) - div p turns non-negative: at f_k for the first such k,
// at -1 if already for k = 0, at +1 if never.  1 / Delta comes from a table
// (no division in the neighbour loops); partial sums are per block, then
// summed by one block in a fixed order, so the result is reproducible.

// 1 / (1 + 2^d), d = 0..15: 1 / Delta = 2^(1 - min(a, b)) / (1 + 2^|a - b|)
// for leaves of edges 2^a and 2^b.
__constant__ double kInvOnePlusPow2[16] = {
    1.0 / 2.0,     1.0 / 3.0,     1.0 / 5.0,     1.0 / 9.0,     1.0 / 17.0,    1.0 / 33.0,
    1.0 / 65.0,    1.0 / 129.0,   1.0 / 257.0,   1.0 / 513.0,   1.0 / 1025.0,  1.0 / 2049.0,
    1.0 / 4097.0,  1.0 / 8193.0,  1.0 / 16385.0, 1.0 / 32769.0};

__device__ __forceinline__ double pow2d(int e) {
  return __longlong_as_double(static_cast<long long>(1023 + e) << 52);   // 2^e, |e| < 1000
}

// alpha / Delta for the ordered pair (row leaf of edge exponent a, neighbour
// of edge exponent b) with alpha = min(1, (2^b / 2^a)^2); exact scalings of a
// table entry by powers of two.
__device__ __forceinline__ double face_weight(int a, int b) {
  const int lo = a < b ? a : b;
  const int d = a < b ? b - a : a - b;
  const double inv_delta = kInvOnePlusPow2[d] * pow2d(1 - lo);
  return b < a ? inv_delta * pow2d(2 * (b - a)) : inv_delta;
}

// Primal and dual terms of leaf l from its gradient (g2 = |g|^2) and div p.
template <typename T>
__device__ __forceinline__ void leaf_terms(const uint32_t* __restrict__ soff,
                                           const T* __restrict__ samp, int64_t l, int a, double ul,
                                           double g2, double dv, double lambda, double gamma,
                                           double* sp, double* sd) {
  const double vol = pow2d(3 * a);
  const uint32_t o = soff[l];
  const int W = int(soff[l + 1] - o);
  const double rc = 1.0 / (double(W) + gamma);
  // dual term: first k with slope c (2k - W) - dv >= 0, i.e. k >= (W + dv / c) / 2;
  // the minimiser is -1 before the first sample, +1 after the last, else f_(k-1)
  const double kk = ceil((double(W) + dv * (double(W) + gamma)) * 0.5);
  const int mx = kk <= 0.0 ? 0 : (kk > double(W) ? W : int(kk) - 1);
  const double xs = kk <= 0.0 ? -1.0 : (kk > double(W) ? 1.0 : double(load_sample(samp, o + mx)));
  // With the samples sorted, sum_k |x - f_k| = x (2 m - W) + sum_k f_k - 2 sum_{k<m} f_k for
  // any m splitting them into f_k <= x (k < m) and f_k >= x (k >= m).  One pass gives
  // the total and the two prefix sums (m = #{f_k < u} for the primal term, m = mx for the
  // dual term).  The running sum is a float32 pair (hi, lo) updated by Knuth's
  // error-free TwoSum, so it carries about 48 bits: on GB300's narrow FP64 pipe
  // this keeps the per-sample work off it, and the prefix sums reach float64 with
  // a relative error near 2^-48, far below the energy's tolerance.
  const float ulf = float(ul);
  float th = 0.0f, tl = 0.0f, uh = 0.0f, ulo = 0.0f, xh = 0.0f, xl = 0.0f;
  int mu = W;
  for (int k = 0; k < W; ++k) {
    const float f = load_sample(samp, o + k);
    if (mu == W && !(f < ulf)) {
      mu = k;
      uh = th;
      ulo = tl;
    }
    if (k == mx) {
      xh = th;
      xl = tl;
    }
    const float sum = __fadd_rn(th, f);
    const float bv = __fsub_rn(sum, th);
    const float err = __fadd_rn(__fsub_rn(th, __fsub_rn(sum, bv)), __fsub_rn(f, bv));
    th = sum;
    tl = __fadd_rn(tl, err);
  }
  if (mu == W) {
    uh = th;
    ulo = tl;
  }
  if (mx == W) {
    xh = th;
    xl = tl;
  }
  const double tot = double(th) + double(tl);
  const double su = double(uh) + double(ulo);
  const double sx = double(xh) + double(xl);
  const double data = ul * double(2 * mu - W) + tot - 2.0 * su;
  const double dd = xs * double(2 * mx - W) + tot - 2.0 * sx;
  *sp += vol * (rc * data + lambda * sqrt(g2));
  *sd += vol * (rc * dd - xs * dv);
}

__device__ __forceinline__ double block_sum_d(double x, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < kThreads / 32; ++w) t += red[w];
  return t;
}

// Sum over the G lanes of a group of one double (groups aligned in the warp;
// every lane of the warp takes part).
template <int G>
__device__ __forceinline__ double group_sum_d(double x) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

// Energy terms of leaf l, its slots spread over a group of G lanes: the
// float64 gradient of u (+faces) and divergence of p (both sides), reduced
// over the group; lane 0 adds the leaf's primal and dual terms to sp, sd
// when `valid`.
template <int G, typename T>
__device__ __forceinline__ void leaf_energy(const View& v, const float* __restrict__ u,
                                            const float* __restrict__ p,
                                            const uint32_t* __restrict__ soff,
                                            const T* __restrict__ samp, double lambda, double gamma,
                                            int64_t l, int lane, bool valid, double* sp, double* sd) {
  int32_t e[6];
#pragma unroll
  for (int f = 0; f < 6; ++f) e[f] = v.nbr[int64_t(f) * v.stride + l];
  const int a = v.D - v.level[l];
  const double ul = double(u[l]);
  double g0 = 0.0, g1 = 0.0, g2 = 0.0, c0 = 0.0, c1 = 0.0, c2 = 0.0, m0 = 0.0, m1 = 0.0, m2 = 0.0;
  for_each_slot<6, 2>(v, e, lane, G, [&](int f, int32_t ent) {
    const int b = v.D - entry_level(ent);
    if (f < 3) {
      const double w = face_weight(a, b);
      const double t = w * (double(u[entry_idx(ent)]) - ul);
      g0 += f == 0 ? t : 0.0;
      g1 += f == 1 ? t : 0.0;
      g2 += f == 2 ? t : 0.0;
      c0 += f == 0 ? w : 0.0;
      c1 += f == 1 ? w : 0.0;
      c2 += f == 2 ? w : 0.0;
    } else {
      // (h_n^3 / h^3) alpha_nl / Delta
      const double w = face_weight(b, a) * pow2d(3 * (b - a));
      const double t = w * double(p[int64_t(f - 3) * v.stride + entry_idx(ent)]);
      m0 += f == 3 ? t : 0.0;
      m1 += f == 4 ? t : 0.0;
      m2 += f == 5 ? t : 0.0;
    }
  });
  g0 = group_sum_d<G>(g0);
  g1 = group_sum_d<G>(g1);
  g2 = group_sum_d<G>(g2);
  c0 = group_sum_d<G>(c0);
  c1 = group_sum_d<G>(c1);
  c2 = group_sum_d<G>(c2);
  m0 = group_sum_d<G>(m0);
  m1 = group_sum_d<G>(m1);
  m2 = group_sum_d<G>(m2);
  if (lane != 0 || !valid) return;
  const double dv = (c0 * double(p[l]) - m0) + (c1 * double(p[v.stride + l]) - m1) +
                    (c2 * double(p[2 * v.stride + l]) - m2);
  leaf_terms(soff, samp, l, a, ul, g0 * g0 + g1 * g1 + g2 * g2, dv, lambda, gamma, sp, sd);
}

constexpr int kEnergyListLanes = 4;

// Launch layout: hb blocks of heavy leaves (a warp per leaf, strided over
// the heavy set), lb blocks of list leaves (kEnergyListLanes lanes per leaf,
// strided over the list set), then light leaves (a thread each, strided over
// all leaves, skipping those with a finer-neighbour list).  Each block writes
// its (primal, dual) partial; all sums are in a fixed order.
template <typename T>
__global__ void __launch_bounds__(kThreads, 4) k_energy(View v, const float* __restrict__ u,
                                                        const float* __restrict__ p,
                                                        const uint32_t* __restrict__ soff,
                                                        const T* __restrict__ samp, double lambda,
                                                        double gamma, Segments sg, int hb, int lb,
                                                        double* __restrict__ partial) {
  __shared__ double red[kThreads / 32];
  double sp = 0.0, sd = 0.0;
  const int b = int(blockIdx.x);
  if (b < hb) {
    const int w = b * (kThreads / 32) + int(threadIdx.x >> 5), nw = hb * (kThreads / 32);
    for (int q = w; q < sg.n_heavy; q += nw)
      leaf_energy<32>(v, u, p, soff, samp, lambda, gamma, sg.heavy[q], int(threadIdx.x & 31), true,
                      &sp, &sd);
  } else if (b < hb + lb) {
    constexpr int G = kEnergyListLanes;
    const int t = (b - hb) * kThreads + int(threadIdx.x);
    const int gi = t / G, ng = lb * (kThreads / G);
    const int rounds = (sg.n_list + ng - 1) / ng;   // the same in every lane
    for (int r = 0; r < rounds; ++r) {
      const int q = gi + r * ng;
      const bool valid = q < sg.n_list;
      leaf_energy<G>(v, u, p, soff, samp, lambda, gamma, sg.list[valid ? q : sg.n_list - 1], t % G,
                     valid, &sp, &sd);
    }
  } else {
    const int nb = int(gridDim.x) - hb - lb;
    for (int64_t l = int64_t(b - hb - lb) * blockDim.x + threadIdx.x; l < v.n;
         l += int64_t(nb) * blockDim.x) {
      bool listed = false;
#pragma unroll
      for (int f = 0; f < 6; ++f) listed |= is_list(v.nbr[int64_t(f) * v.stride + l]);
      if (listed) continue;   // summed by a heavy or list group
      leaf_energy<1>(v, u, p, soff, samp, lambda, gamma, l, 0, true, &sp, &sd);
    }
  }
  // block partial in a fixed order
  const double bp = block_sum_d(sp, red);
  const double bd = block_sum_d(sd, red);
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

inline unsigned grid_of(int64_t n, const Segments& sg, int list_lanes) {
  return blocks_for(n, kThreads) + blocks_for(int64_t(sg.n_list) * list_lanes, kThreads) +
         unsigned(heavy_blocks(sg));
}

cudaError_t launch_dual(View v, const float* ubar, float* p, const float* sigma, float lambda,
                        LeafSets ls, cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  const Segments sg{ls.heavy, ls.n_heavy, ls.list, ls.n_list};
  k_dual<false><<<grid_of(v.n, sg, kDualListLanes), kThreads, 0, s>>>(v, ubar, p, sigma, lambda, sg, 0.0f);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_dual_init(View v, const float* u, float* p, float lambda, float g0, LeafSets ls,
                             cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  const Segments sg{ls.heavy, ls.n_heavy, ls.list, ls.n_list};
  k_dual<true><<<grid_of(v.n, sg, kDualListLanes), kThreads, 0, s>>>(v, u, p, nullptr, lambda, sg, g0);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_primal(View v, float* u, float* ubar, const float* p, const float* tau,
                          const uint32_t* soff, const void* samp, bool fp16, float gamma,
                          LeafSets ls, cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  const Segments sg{ls.heavy, ls.n_heavy, ls.list, ls.n_list};
  const unsigned nb = grid_of(v.n, sg, kPrimalListLanes);
  if (fp16)
    k_primal<__half><<<nb, kThreads, 0, s>>>(v, u, ubar, p, tau, soff,
                                             reinterpret_cast<const __half*>(samp), gamma, sg);
  else
    k_primal<float><<<nb, kThreads, 0, s>>>(v, u, ubar, p, tau, soff,
                                            reinterpret_cast<const float*>(samp), gamma, sg);
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
  k_energy<T><<<g.nb, kThreads, 0, s>>>(v, u, p, soff, reinterpret_cast<const T*>(samp), lambda,
                                        gamma, sg, g.hb, g.lb, partial);
}

cudaError_t launch_energy(View v, const float* u, const float* p, const uint32_t* soff,
                          const void* samp, bool fp16, double lambda, double gamma, LeafSets ls,
                          double* partial, double* out3, cudaStream_t s) {
  const Segments sg{ls.heavy, ls.n_heavy, ls.list, ls.n_list};
  const EnergyLayout g = energy_layout(v.n, sg, kThreads, kEnergyBlocks);
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
