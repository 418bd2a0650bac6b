// The paper's own solver (Eq. 4-6, Sec. 4): gradient descent on the
// eps-L1-smoothed normalised energy
//   E_eps(u) = sum_l h_l^3 [c_l sum_k Gamma(u_l - f_k) + lambda Gamma(|g(l)|)],
//   Gamma(x) = sqrt(x^2 + eps^2),  c_l = 1 / (W_l + gamma),  g = K u,
// on the same leaves, face entries and level-aware operators as the
// primal-dual kernels.  Its gradient in the volume-weighted metric is
//   G(u)_l = c_l sum_k (u_l - f_k) / Gamma(u_l - f_k) - lambda div(g / Gamma(|g|))(l)
// (Eq. 6 with the sign flipped), and an iteration is u <- u - xi_t G(u).
// Pass 1 (k_descent_q) forms q = g / Gamma(|g|) from the +face lists; pass 2
// (k_descent_u) gathers div q from the -face lists, adds the data term over
// the leaf's samples and updates u in place (it reads only its own u).  Both
// passes use the leaf classes of the primal-dual kernels: heavy leaves (a list
// longer than 16) get a block with fixed-order reductions, list leaves a
// thread of their own segment, the rest a thread each.
#include "descent.cuh"
#include "stencil.cuh"

namespace ofu {

namespace {

// Sum over the leaf's samples of (u - f_k) / Gamma(u - f_k), Gamma(x) =
// sqrt(x^2 + eps^2), four samples per step.
template <typename T>
__device__ __forceinline__ float data_slope(const T* __restrict__ f, int W, float ul, float e2) {
  float acc = 0.0f;
  int k = 0;
  for (; k + 4 <= W; k += 4) {
    float r[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) r[j] = ul - load_sample(f, k + j);
#pragma unroll
    for (int j = 0; j < 4; ++j) acc += r[j] / sqrtf(r[j] * r[j] + e2);
  }
  for (; k < W; ++k) {
    const float r = ul - load_sample(f, k);
    acc += r / sqrtf(r * r + e2);
  }
  return acc;
}

// Pass 1: q = g / Gamma(|g|) with g = K u from the +face lists.  Launch
// layout and leaf classes as the dual step (heavy, list, light).
__global__ void __launch_bounds__(kThreads, kIterMinBlocks) k_descent_q(View v, const float* __restrict__ u,
                                                                        float eps, float* __restrict__ q,
                                                                        Segments sg) {
  float g[3];
  int64_t l;
  if (int(blockIdx.x) < sg.n_heavy) {
    __shared__ float red[kHeavyThreads / 32];
    l = sg.heavy[blockIdx.x];
    const float h = edge_f(v.D, v.level[l]);
    const float ul = u[l];
    for (int d = 0; d < 3; ++d) {
      const int32_t e = v.nbr[int64_t(d) * v.stride + l];
      float acc = 0.0f;
      if (e >= 0) {
        if (threadIdx.x == 0) acc = (u[entry_idx(e)] - ul) * inv_delta(h, edge_f(v.D, entry_level(e)));
      } else if (e != kEmpty) {
        const uint32_t st = list_start(e);
        const int cnt = v.ovf[st];
        for (int k = threadIdx.x; k < cnt; k += kHeavyThreads) {
          const int32_t f = v.ovf[st + 1 + k];
          const float hm = edge_f(v.D, entry_level(f));
          const float r = hm / h;
          acc += r * r * (u[entry_idx(f)] - ul) * inv_delta(h, hm);
        }
      }
      g[d] = block_sum(acc, red);
    }
    if (threadIdx.x != 0) return;
  } else {
    bool listed;
    l = segment_leaf(sg, v.n, &listed);
    if (l < 0) return;
    const size_t st = size_t(v.stride);
    const int32_t e[3] = {v.nbr[l], v.nbr[st + l], v.nbr[2 * st + l]};
    const int lev = v.level[l];
    const float h = edge_f(v.D, lev);
    const float ul = u[l];
    if (!listed) {
      float x[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) x[d] = u[e[d] >= 0 ? entry_idx(e[d]) : uint32_t(l)];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float hm = edge_f(v.D, e[d] >= 0 ? entry_level(e[d]) : lev);
        g[d] = e[d] >= 0 ? (x[d] - ul) * inv_delta(h, hm) : 0.0f;
      }
      if (is_list(e[0]) || is_list(e[1]) || is_list(e[2])) return;   // a list thread's
    } else {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        float acc = 0.0f;
        if (e[d] >= 0) {
          acc = (u[entry_idx(e[d])] - ul) * inv_delta(h, edge_f(v.D, entry_level(e[d])));
        } else if (e[d] != kEmpty) {
          const uint32_t s0 = list_start(e[d]);
          acc = list_sum(
              v.ovf + s0 + 1, v.ovf[s0],
              [&](int lv) {
                const float hm = edge_f(v.D, lv);
                const float r = hm / h;
                return r * r * inv_delta(h, hm);
              },
              [&](uint32_t m) { return u[m] - ul; });
        }
        g[d] = acc;
      }
    }
  }
  const float inv = 1.0f / sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2] + eps * eps);
#pragma unroll
  for (int d = 0; d < 3; ++d) q[int64_t(d) * v.stride + l] = g[d] * inv;
}

// Pass 2: u <- u - xi [c sum_k (u - f_k) / Gamma(u - f_k) - lambda div q];
// reads only its own u.  Layout and classes as the primal step.
template <typename T>
__global__ void __launch_bounds__(kThreads, kIterMinBlocks) k_descent_u(
    View v, float* __restrict__ u, float* __restrict__ ubar, const float* __restrict__ q,
    const uint32_t* __restrict__ soff, const T* __restrict__ samp, float eps, float xi,
    float lambda, float gamma, Segments sg) {
  const float e2 = eps * eps;
  if (int(blockIdx.x) < sg.n_heavy) {
    __shared__ float red[kHeavyThreads / 32];
    const int64_t l = sg.heavy[blockIdx.x];
    const float h = edge_f(v.D, v.level[l]);
    const float dv = divergence_block(v, q, l, h, red);
    const uint32_t o = soff[l];
    const int W = int(soff[l + 1] - o);
    const float ul = u[l];
    float part = 0.0f;
    for (int k = threadIdx.x; k < W; k += kHeavyThreads) {
      const float r = ul - load_sample(samp + o, k);
      part += r / sqrtf(r * r + e2);
    }
    const float data = block_sum(part, red);
    if (threadIdx.x == 0) {
      const float un = ul - xi * (data / (float(W) + gamma) - lambda * dv);
      u[l] = un;
      ubar[l] = un;
    }
    return;
  }
  bool listed;
  const int64_t l = segment_leaf(sg, v.n, &listed);
  if (l < 0) return;
  int32_t e[6];
#pragma unroll
  for (int f = 0; f < 6; ++f) e[f] = v.nbr[int64_t(f) * v.stride + l];
  const int lev = v.level[l];
  const float h = edge_f(v.D, lev);
  float qq[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) qq[d] = q[int64_t(d) * v.stride + l];
  const float ul = u[l];
  const uint32_t o = soff[l];
  const int W = int(soff[l + 1] - o);
  float dv;
  if (!listed) {
    float qn[3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
      qn[d] = q[int64_t(d) * v.stride + (e[3 + d] >= 0 ? entry_idx(e[3 + d]) : uint32_t(l))];
    dv = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float hm = edge_f(v.D, e[d] >= 0 ? entry_level(e[d]) : lev);
      dv += (e[d] >= 0 ? inv_delta(h, hm) : 0.0f) * qq[d];
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float hn = edge_f(v.D, e[3 + d] >= 0 ? entry_level(e[3 + d]) : lev);
      dv -= e[3 + d] >= 0 ? (hn / h) * inv_delta(h, hn) * qn[d] : 0.0f;
    }
    bool any = false;
#pragma unroll
    for (int f = 0; f < 6; ++f) any |= is_list(e[f]);
    if (any) return;   // a list thread's
  } else {
    dv = divergence(v, q, l, h, e, qq);
  }
  const float data = data_slope(samp + o, W, ul, e2);
  const float un = ul - xi * (data / (float(W) + gamma) - lambda * dv);
  u[l] = un;
  ubar[l] = un;
}

unsigned grid_of(int64_t n, const Segments& sg) {
  return unsigned((n + kThreads - 1) / kThreads) + unsigned((sg.n_list + kThreads - 1) / kThreads) +
         unsigned(sg.n_heavy);
}

}  // namespace

cudaError_t launch_descent_step(View v, float* u, float* ubar, float* q, const uint32_t* soff,
                                const void* samp, bool fp16, float eps, float xi, float lambda,
                                float gamma, LeafSets dual_sets, LeafSets primal_sets,
                                cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  const Segments sq{dual_sets.heavy, dual_sets.n_heavy, dual_sets.list, dual_sets.n_list};
  const Segments su{primal_sets.heavy, primal_sets.n_heavy, primal_sets.list, primal_sets.n_list};
  k_descent_q<<<grid_of(v.n, sq), kThreads, 0, s>>>(v, u, eps, q, sq);
  if (fp16)
    k_descent_u<__half><<<grid_of(v.n, su), kThreads, 0, s>>>(
        v, u, ubar, q, soff, reinterpret_cast<const __half*>(samp), eps, xi, lambda, gamma, su);
  else
    k_descent_u<float><<<grid_of(v.n, su), kThreads, 0, s>>>(
        v, u, ubar, q, soff, reinterpret_cast<const float*>(samp), eps, xi, lambda, gamma, su);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace ofu
