// The paper's own solver (Eq. 4-6, Sec. 4): gradient descent on the
// eps-L1-smoothed normalised energy
//   E_eps(u) = sum_l h_l^3 [c_l sum_k Gamma(u_l - f_k) + lambda Gamma(|g(l)|)],
//   Gamma(x) = sqrt(x^2 + eps^2),  c_l = 1 / (W_l + gamma),  g = K u,
// on the same leaves, face entries and level-aware operators as the
// primal-dual kernels.  Its gradient in the volume-weighted metric is
//   G(u)_l = c_l sum_k (u_l - f_k) / Gamma(u_l - f_k) - lambda div(g / Gamma(|g|))(l)
// (Eq. 6 with the sign flipped), and an iteration is u <- u - xi_t G(u).
// Pass 1 (k_descent_q, thread per leaf) forms q = g / Gamma(|g|) from the +face
// lists; pass 2 (k_descent_u) gathers div q from the -face lists, adds the data
// term over the leaf's samples and updates u in place (it reads only its own
// u).  A thread walks every list, however long.
#include "descent.cuh"

namespace ofu {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float edge_f(int D, int level) { return float(1u << (D - level)); }

// 1 / Delta for leaves of edges h and hm: 2 / (h + hm)
__device__ __forceinline__ float inv_delta(float h, float hm) { return __fdividef(2.0f, h + hm); }

template <typename T>
__device__ __forceinline__ float sample_at(const T* s, uint32_t i) {
  if constexpr (sizeof(T) == 2)
    return __half2float(s[i]);
  else
    return s[i];
}

__global__ void __launch_bounds__(kThreads) k_descent_q(View v, const float* __restrict__ u,
                                                        float eps, float* __restrict__ q) {
  const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l >= v.n) return;
  const float h = edge_f(v.D, v.level[l]);
  const float ul = u[l];
  float g[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int32_t e = v.nbr[int64_t(d) * v.stride + l];
    float acc = 0.0f;
    if (e >= 0) {
      // same or coarser neighbour: alpha = 1
      acc = (u[entry_idx(e)] - ul) * inv_delta(h, edge_f(v.D, entry_level(e)));
    } else if (e != kEmpty) {
      // finer neighbours: alpha = (h_m / h)^2
      const uint32_t st = list_start(e);
      const int cnt = v.ovf[st];
      for (int k = 0; k < cnt; ++k) {
        const int32_t f = v.ovf[st + 1 + k];
        const float hm = edge_f(v.D, entry_level(f));
        const float r = hm / h;
        acc += r * r * (u[entry_idx(f)] - ul) * inv_delta(h, hm);
      }
    }
    g[d] = acc;
  }
  const float inv = 1.0f / sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2] + eps * eps);
#pragma unroll
  for (int d = 0; d < 3; ++d) q[int64_t(d) * v.stride + l] = g[d] * inv;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_descent_u(View v, float* __restrict__ u,
                                                        float* __restrict__ ubar,
                                                        const float* __restrict__ q,
                                                        const uint32_t* __restrict__ soff,
                                                        const T* __restrict__ samp, float eps,
                                                        float xi, float lambda, float gamma) {
  const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l >= v.n) return;
  const float h = edge_f(v.D, v.level[l]);
  // div q: + faces weigh q(l) by sum alpha / Delta, - faces gather the
  // neighbours' q with weight (h_n^3 / h^3) alpha_nl / Delta
  float dv = 0.0f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int32_t e = v.nbr[int64_t(d) * v.stride + l];
    float coef = 0.0f;
    if (e >= 0) {
      coef = inv_delta(h, edge_f(v.D, entry_level(e)));
    } else if (e != kEmpty) {
      const uint32_t st = list_start(e);
      const int cnt = v.ovf[st];
      for (int k = 0; k < cnt; ++k) {
        const float hm = edge_f(v.D, entry_level(v.ovf[st + 1 + k]));
        const float r = hm / h;
        coef += r * r * inv_delta(h, hm);
      }
    }
    dv += coef * q[int64_t(d) * v.stride + l];
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int32_t e = v.nbr[int64_t(3 + d) * v.stride + l];
    if (e >= 0) {
      // same or coarser n: (h_n / h) / Delta
      const float hn = edge_f(v.D, entry_level(e));
      dv -= (hn / h) * inv_delta(h, hn) * q[int64_t(d) * v.stride + entry_idx(e)];
    } else if (e != kEmpty) {
      // finer n: (h_n / h)^3 / Delta
      const uint32_t st = list_start(e);
      const int cnt = v.ovf[st];
      for (int k = 0; k < cnt; ++k) {
        const int32_t f = v.ovf[st + 1 + k];
        const float hn = edge_f(v.D, entry_level(f));
        const float r = hn / h;
        dv -= r * r * r * inv_delta(h, hn) * q[int64_t(d) * v.stride + entry_idx(f)];
      }
    }
  }
  const uint32_t o = soff[l];
  const int W = int(soff[l + 1] - o);
  const float ul = u[l];
  const float e2 = eps * eps;
  float data = 0.0f;
  for (int k = 0; k < W; ++k) {
    const float r = ul - sample_at(samp + o, k);
    data += r / sqrtf(r * r + e2);
  }
  const float un = ul - xi * (data / (float(W) + gamma) - lambda * dv);
  u[l] = un;
  ubar[l] = un;
}

unsigned blocks_for(int64_t n) { return unsigned((n + kThreads - 1) / kThreads); }

}  // namespace

cudaError_t launch_descent_step(View v, float* u, float* ubar, float* q, const uint32_t* soff,
                                const void* samp, bool fp16, float eps, float xi, float lambda,
                                float gamma, cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  const unsigned nb = blocks_for(v.n);
  k_descent_q<<<nb, kThreads, 0, s>>>(v, u, eps, q);
  if (fp16)
    k_descent_u<__half><<<nb, kThreads, 0, s>>>(v, u, ubar, q, soff,
                                                reinterpret_cast<const __half*>(samp), eps, xi,
                                                lambda, gamma);
  else
    k_descent_u<float><<<nb, kThreads, 0, s>>>(v, u, ubar, q, soff,
                                               reinterpret_cast<const float*>(samp), eps, xi,
                                               lambda, gamma);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace ofu
