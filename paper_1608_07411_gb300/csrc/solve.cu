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

#include <mutex>

#include "ofu_internal.cuh"

namespace ofu {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;

__device__ __forceinline__ float edge_f(int D, int level) { return float(1u << (D - level)); }

// 1 / Delta for leaves of edges h and hm: 2 / (h + hm), exact sum of powers of two.
__device__ __forceinline__ float inv_delta(float h, float hm) { return __fdividef(2.0f, h + hm); }

template <typename T>
__device__ __forceinline__ float load_sample(const T* s, uint32_t i) {
  if constexpr (sizeof(T) == 2)
    return __half2float(s[i]);
  else
    return s[i];
}

__global__ void __launch_bounds__(kThreads) k_dual(View v, const float* __restrict__ ubar,
                                                   float* __restrict__ p,
                                                   const float* __restrict__ sigma, float lambda) {
  const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l >= v.n) return;
  const float h = edge_f(v.D, v.level[l]);
  const float ul = ubar[l];
  float g[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int32_t e = v.nbr[int64_t(d) * v.stride + l];
    float acc = 0.0f;
    if (e >= 0) {
      // same or coarser neighbour: alpha = 1
      const float hm = edge_f(v.D, entry_level(e));
      acc = (ubar[entry_idx(e)] - ul) * inv_delta(h, hm);
    } else if (e != kEmpty) {
      const uint32_t st = list_start(e);
      const int cnt = v.ovf[st];
      for (int k = 0; k < cnt; ++k) {
        const int32_t f = v.ovf[st + 1 + k];
        const float hm = edge_f(v.D, entry_level(f));
        const float r = hm / h;
        acc += r * r * (ubar[entry_idx(f)] - ul) * inv_delta(h, hm);
      }
    }
    g[d] = acc;
  }
  const float s = sigma[l];
  float q0 = p[l] + s * g[0];
  float q1 = p[v.stride + l] + s * g[1];
  float q2 = p[2 * v.stride + l] + s * g[2];
  const float nrm = sqrtf(q0 * q0 + q1 * q1 + q2 * q2);
  if (nrm > lambda) {
    const float sc = lambda / nrm;
    q0 *= sc;
    q1 *= sc;
    q2 *= sc;
  }
  p[l] = q0;
  p[v.stride + l] = q1;
  p[2 * v.stride + l] = q2;
}

// Divergence of p at leaf l (gathers only).
__device__ __forceinline__ float divergence(const View& v, const float* __restrict__ p, int64_t l,
                                            float h) {
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
    dv += coef * p[int64_t(d) * v.stride + l];
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int32_t e = v.nbr[int64_t(3 + d) * v.stride + l];
    if (e >= 0) {
      // same or coarser n: (h_n^3 / h^3) (h / h_n)^2 / Delta = (h_n / h) / Delta
      const float hn = edge_f(v.D, entry_level(e));
      dv -= (hn / h) * inv_delta(h, hn) * p[int64_t(d) * v.stride + entry_idx(e)];
    } else if (e != kEmpty) {
      // finer n: alpha = 1, weight (h_n / h)^3 / Delta
      const uint32_t st = list_start(e);
      const int cnt = v.ovf[st];
      for (int k = 0; k < cnt; ++k) {
        const int32_t f = v.ovf[st + 1 + k];
        const float hn = edge_f(v.D, entry_level(f));
        const float r = hn / h;
        dv -= r * r * r * inv_delta(h, hn) * p[int64_t(d) * v.stride + entry_idx(f)];
      }
    }
  }
  return dv;
}

// Prox of the data term: argmin_x (x - v)^2 / (2 tau) + c sum_k |x - f_k| is
// the median of {f_k} and {v + t (W - 2k)}_{k=0..W}, t = tau c.  With the
// samples sorted, it is clamp(b_k, f_k, f_(k+1)) for the smallest k with
// f_(k+1) >= b_k = v + t (W - 2k) (f_0 = -inf, f_(W+1) = +inf), found by
// bisection because the predicate is monotone in k.
template <typename T>
__device__ __forceinline__ float prox_l1(const T* __restrict__ f, int W, float v, float t) {
  int lo = 0, hi = W;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const float b = v + t * float(W - 2 * mid);
    if (load_sample(f, mid) >= b) hi = mid; else lo = mid + 1;
  }
  const int k = lo;
  float x = v + t * float(W - 2 * k);
  if (k < W) x = fminf(x, load_sample(f, k));
  if (k > 0) x = fmaxf(x, load_sample(f, k - 1));
  return x;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_primal(View v, float* __restrict__ u,
                                                     float* __restrict__ ubar,
                                                     const float* __restrict__ p,
                                                     const float* __restrict__ tau,
                                                     const uint32_t* __restrict__ soff,
                                                     const T* __restrict__ samp, float gamma) {
  const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l >= v.n) return;
  const float h = edge_f(v.D, v.level[l]);
  const float tl = tau[l];
  const float ul = u[l];
  const float x = ul + tl * divergence(v, p, l, h);
  const uint32_t o = soff[l];
  const int W = int(soff[l + 1] - o);
  const float t = tl / (float(W) + gamma);
  const float un = fminf(fmaxf(prox_l1(samp + o, W, x, t), -1.0f), 1.0f);
  u[l] = un;
  ubar[l] = 2.0f * un - ul;
}

// ---------------------------------------------------------------------------
// Energy (float64).  Per leaf, with c = 1 / (W + gamma) and volume h^3:
//   primal  h^3 [c sum_k |u - f_k| + lambda |grad u|]
//   dual    h^3 min_{x in [-1,1]} [c sum_k |x - f_k| - x div p]
// The dual minimum of the convex piecewise-linear function sits where its
// slope c (2k - W) - div p turns non-negative: at f_k for the first such k,
// at -1 if already for k = 0, at +1 if never.

constexpr int kEnergyBlocks = 1024;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_energy(View v, const float* __restrict__ u,
                                                     const float* __restrict__ p,
                                                     const uint32_t* __restrict__ soff,
                                                     const T* __restrict__ samp, double lambda,
                                                     double gamma, double* __restrict__ partial) {
  double sp = 0.0, sd = 0.0;
  for (int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; l < v.n;
       l += int64_t(gridDim.x) * blockDim.x) {
    const int lev = v.level[l];
    const double h = double(int64_t(1) << (v.D - lev));
    const double vol = h * h * h;
    const double ul = double(u[l]);
    double g2 = 0.0, dv = 0.0;
    for (int d = 0; d < 3; ++d) {
      const int32_t e = v.nbr[int64_t(d) * v.stride + l];
      double g = 0.0, coef = 0.0;
      if (e != kEmpty) {
        const int32_t* lst = &e;
        int cnt = 1;
        if (e < 0) {
          cnt = v.ovf[list_start(e)];
          lst = v.ovf + list_start(e) + 1;
        }
        for (int k = 0; k < cnt; ++k) {
          const double hm = double(int64_t(1) << (v.D - entry_level(lst[k])));
          const double w = fmin(1.0, (hm / h) * (hm / h)) / ((h + hm) * 0.5);
          g += w * (double(u[entry_idx(lst[k])]) - ul);
          coef += w;
        }
      }
      g2 += g * g;
      dv += coef * double(p[int64_t(d) * v.stride + l]);
      const int32_t e2 = v.nbr[int64_t(3 + d) * v.stride + l];
      if (e2 != kEmpty) {
        const int32_t* lst = &e2;
        int cnt = 1;
        if (e2 < 0) {
          cnt = v.ovf[list_start(e2)];
          lst = v.ovf + list_start(e2) + 1;
        }
        for (int k = 0; k < cnt; ++k) {
          const double hn = double(int64_t(1) << (v.D - entry_level(lst[k])));
          const double w = fmin(1.0, (h / hn) * (h / hn)) / ((h + hn) * 0.5);
          dv -= (hn * hn * hn) / vol * w * double(p[int64_t(d) * v.stride + entry_idx(lst[k])]);
        }
      }
    }
    const uint32_t o = soff[l];
    const int W = int(soff[l + 1] - o);
    const double c = 1.0 / (double(W) + gamma);
    double data = 0.0;
    for (int k = 0; k < W; ++k) data += fabs(ul - double(load_sample(samp, o + k)));
    sp += vol * (c * data + lambda * sqrt(g2));
    // dual term
    double xs;
    const double kk = ceil((double(W) + dv / c) * 0.5);
    if (kk <= 0.0) xs = -1.0;
    else if (kk > double(W)) xs = 1.0;
    else xs = double(load_sample(samp, o + int(kk) - 1));
    xs = fmin(1.0, fmax(-1.0, xs));
    double dd = 0.0;
    for (int k = 0; k < W; ++k) dd += fabs(xs - double(load_sample(samp, o + k)));
    sd += vol * (c * dd - xs * dv);
  }
  // block reduction in a fixed order
  __shared__ double rp[kThreads / 32], rd[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sp += __shfl_xor_sync(kFull, sp, o);
    sd += __shfl_xor_sync(kFull, sd, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    rp[wid] = sp;
    rd[wid] = sd;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) {
      a += rp[w];
      b += rd[w];
    }
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = b;
  }
}

__global__ void k_energy_final(const double* __restrict__ partial, int nb, double* __restrict__ out3) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < nb; ++i) {
    a += partial[2 * i];
    b += partial[2 * i + 1];
  }
  out3[0] = a;
  out3[1] = b;
  out3[2] = a - b;
}

inline unsigned blocks_for(int64_t n, int threads) { return unsigned((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_dual(View v, const float* ubar, float* p, const float* sigma, float lambda,
                        cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  k_dual<<<blocks_for(v.n, kThreads), kThreads, 0, s>>>(v, ubar, p, sigma, lambda);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_primal(View v, float* u, float* ubar, const float* p, const float* tau,
                          const uint32_t* soff, const void* samp, bool fp16, float gamma,
                          cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  if (fp16)
    k_primal<__half><<<blocks_for(v.n, kThreads), kThreads, 0, s>>>(
        v, u, ubar, p, tau, soff, reinterpret_cast<const __half*>(samp), gamma);
  else
    k_primal<float><<<blocks_for(v.n, kThreads), kThreads, 0, s>>>(
        v, u, ubar, p, tau, soff, reinterpret_cast<const float*>(samp), gamma);
  count_launches(1);
  return cudaGetLastError();
}

size_t energy_tmp_bytes(int64_t) { return size_t(2 * kEnergyBlocks) * sizeof(double); }

cudaError_t launch_energy(View v, const float* u, const float* p, const uint32_t* soff,
                          const void* samp, bool fp16, double lambda, double gamma,
                          double* partial, double* out3, cudaStream_t s) {
  const int nb = kEnergyBlocks;
  if (fp16)
    k_energy<__half><<<nb, kThreads, 0, s>>>(v, u, p, soff, reinterpret_cast<const __half*>(samp),
                                             lambda, gamma, partial);
  else
    k_energy<float><<<nb, kThreads, 0, s>>>(v, u, p, soff, reinterpret_cast<const float*>(samp),
                                            lambda, gamma, partial);
  count_launches(1);
  k_energy_final<<<1, 32, 0, s>>>(partial, nb, out3);
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
  // address up once per device, with that device current.
  static std::mutex mu;
  static double* addr[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* a = nullptr;
    e = cudaGetSymbolAddress(&a, g_energy_scratch);
    if (e != cudaSuccess) return e;
    addr[dev] = static_cast<double*>(a);
  }
  *ptr = addr[dev];
  return cudaSuccess;
}

cudaError_t launch_energy_static(View v, const float* u, const float* p, const uint32_t* soff,
                                 const void* samp, bool fp16, double lambda, double gamma,
                                 double* scratch, cudaStream_t s) {
  const int64_t want = (v.n + kStaticLeavesPerBlock - 1) / kStaticLeavesPerBlock;
  if (want > kStaticEnergyBlocks) return cudaErrorInvalidValue;
  const int nb = want < 1 ? 1 : int(want);
  if (fp16)
    k_energy<__half><<<nb, kThreads, 0, s>>>(v, u, p, soff, reinterpret_cast<const __half*>(samp),
                                             lambda, gamma, scratch);
  else
    k_energy<float><<<nb, kThreads, 0, s>>>(v, u, p, soff, reinterpret_cast<const float*>(samp),
                                            lambda, gamma, scratch);
  count_launches(1);
  k_energy_final<<<1, 32, 0, s>>>(scratch, nb, scratch + 2 * kStaticEnergyBlocks);
  count_launches(1);
  return cudaGetLastError();
}

int energy_static_result_offset() { return 2 * kStaticEnergyBlocks; }

}  // namespace ofu
