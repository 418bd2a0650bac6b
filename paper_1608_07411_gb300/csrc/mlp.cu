// Warm-start network: per-leaf features, forward pass, gradient (per-block
// partials summed in a fixed order) and Adam.  Not in the paper: it replaces
// the median initialisation of observed leaves by a learned value.
//
// Features (39): nearest-rank quantiles f_(r_j), r_j = ceil((2j - 1) W / 64),
// j = 1..32, of the leaf's sorted samples (0 if W = 0); level / D_max; per face
// (+x, +y, +z, -x, -y, -z) the neighbours' u weighted by the share of the face
// each covers, min(1, (h_m / h_l)^2), or the leaf's own u on the boundary.
// Network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = tanh(w3 . h2 + b3),
// W1 [64 x 39], W2 [64 x 64]; parameters packed W1, b1, W2, b2, w3, b3.
#include <math_constants.h>

#include <cmath>

#include "ofu_internal.cuh"

namespace ofu {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kIn = kMlpIn, kHid = kMlpHid;
constexpr int oW1 = 0, oB1 = oW1 + kHid * kIn, oW2 = oB1 + kHid, oB2 = oW2 + kHid * kHid,
              oW3 = oB2 + kHid, oB3 = oW3 + kHid, kN = oB3 + 1;
static_assert(kN == kMlpParams, "parameter layout");

template <typename T>
__device__ __forceinline__ float samp_at(const T* s, uint32_t i) {
  if constexpr (sizeof(T) == 2)
    return __half2float(s[i]);
  else
    return s[i];
}

template <typename T>
__device__ __forceinline__ void leaf_features(const View& v, const float* __restrict__ u,
                              const uint32_t* __restrict__ soff, const T* __restrict__ samp,
                              int64_t l, float* x) {
  const uint32_t o = soff[l];
  const int W = int(soff[l + 1] - o);
#pragma unroll
  for (int j = 1; j <= 32; ++j) {
    const int r = ((2 * j - 1) * W + 63) / 64;
    x[j - 1] = W > 0 ? samp_at(samp, o + r - 1) : 0.0f;
  }
  const int lev = v.level[l];
  x[32] = float(lev) / float(v.D);
  const float ul = u[l];
  const float h = float(1u << (v.D - lev));
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int32_t e = v.nbr[int64_t(f) * v.stride + l];
    float val = ul;
    if (e >= 0) {
      val = u[entry_idx(e)];
    } else if (e != kEmpty) {
      const uint32_t st = list_start(e);
      const int cnt = v.ovf[st];
      float num = 0.0f, den = 0.0f;
      for (int k = 0; k < cnt; ++k) {
        const int32_t g = v.ovf[st + 1 + k];
        const float r = float(1u << (v.D - entry_level(g))) / h;
        num += r * r * u[entry_idx(g)];
        den += r * r;
      }
      val = den > 0.0f ? num / den : ul;
    }
    x[33 + f] = val;
  }
}

__device__ __forceinline__ void load_params(const float* __restrict__ params, float* sp) {
  for (int i = threadIdx.x; i < kN; i += blockDim.x) sp[i] = params[i];
  __syncthreads();
}

__device__ __forceinline__ float mlp_row(const float* sp, const float* x) {
  float h1[kHid];
#pragma unroll
  for (int k = 0; k < kHid; ++k) {
    float a = sp[oB1 + k];
#pragma unroll
    for (int i = 0; i < kIn; ++i) a += sp[oW1 + k * kIn + i] * x[i];
    h1[k] = fmaxf(a, 0.0f);
  }
  float y = sp[oB3];
  for (int j = 0; j < kHid; ++j) {
    float a = sp[oB2 + j];
#pragma unroll
    for (int k = 0; k < kHid; ++k) a += sp[oW2 + j * kHid + k] * h1[k];
    y += sp[oW3 + j] * fmaxf(a, 0.0f);
  }
  return tanhf(y);
}

constexpr int kFwdThreads = 128;

template <typename T>
__global__ void __launch_bounds__(kFwdThreads) k_features(View v, const float* __restrict__ u,
                                                          const uint32_t* __restrict__ soff,
                                                          const T* __restrict__ samp,
                                                          float* __restrict__ X) {
  const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l >= v.n) return;
  float x[kIn];
  leaf_features(v, u, soff, samp, l, x);
#pragma unroll
  for (int i = 0; i < kIn; ++i) X[l * kIn + i] = x[i];
}

__global__ void __launch_bounds__(kFwdThreads) k_forward(const float* __restrict__ params,
                                                         const float* __restrict__ X, int64_t B,
                                                         float* __restrict__ y) {
  __shared__ float sp[kN];
  load_params(params, sp);
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= B) return;
  float x[kIn];
#pragma unroll
  for (int i = 0; i < kIn; ++i) x[i] = X[r * kIn + i];
  y[r] = mlp_row(sp, x);
}

// Warm start: features from the median-initialised u, network output into
// `out` (a buffer this kernel does not read) where W > 0 and the output is
// finite, the median elsewhere.
template <typename T>
__global__ void __launch_bounds__(kFwdThreads) k_warm_start(View v, const float* __restrict__ u,
                                                            const uint32_t* __restrict__ soff,
                                                            const T* __restrict__ samp,
                                                            const float* __restrict__ params,
                                                            float* __restrict__ out) {
  __shared__ float sp[kN];
  load_params(params, sp);
  const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l >= v.n) return;
  const int W = int(soff[l + 1] - soff[l]);
  float y = u[l];
  if (W > 0) {
    float x[kIn];
    leaf_features(v, u, soff, samp, l, x);
    const float m = mlp_row(sp, x);
    if (isfinite(m)) y = m;
  }
  out[l] = y;
}

// Gradient of L = sum_i w_i (y_i - t_i)^2 / sum_i w_i over a batch: each block
// takes kTile rows, keeps their activations in shared memory and writes the
// unnormalised gradient of its rows (and its sums of w (y - t)^2 and w) to
// partial[block]; k_grad_reduce adds the blocks in order and divides by sum w.
constexpr int kTile = 128;
constexpr int kLd = kHid + 1;   // padded row stride against bank conflicts

__global__ void __launch_bounds__(kTile) k_grad_tile(const float* __restrict__ params,
                                                     const float* __restrict__ X,
                                                     const float* __restrict__ t,
                                                     const float* __restrict__ w,
                                                     const int32_t* __restrict__ rows, int64_t B,
                                                     float* __restrict__ partial,
                                                     double* __restrict__ psums) {
  extern __shared__ float sm[];
  float* sp = sm;                       // kN
  float* xs = sp + kN;                  // kTile x kIn
  float* h1 = xs + kTile * kIn;         // kTile x kLd
  float* h2 = h1 + kTile * kLd;
  float* d2 = h2 + kTile * kLd;
  float* d1 = d2 + kTile * kLd;
  float* d3 = d1 + kTile * kLd;         // kTile
  load_params(params, sp);
  const int r = threadIdx.x;
  const int64_t gi = int64_t(blockIdx.x) * kTile + r;
  const bool live = gi < B;
  const int64_t row = live ? (rows ? int64_t(rows[gi]) : gi) : 0;
  for (int i = 0; i < kIn; ++i) xs[r * kIn + i] = live ? X[row * kIn + i] : 0.0f;
  // forward, keeping activations
  for (int k = 0; k < kHid; ++k) {
    float a = sp[oB1 + k];
    for (int i = 0; i < kIn; ++i) a += sp[oW1 + k * kIn + i] * xs[r * kIn + i];
    h1[r * kLd + k] = fmaxf(a, 0.0f);
  }
  float ya = sp[oB3];
  for (int j = 0; j < kHid; ++j) {
    float a = sp[oB2 + j];
    for (int k = 0; k < kHid; ++k) a += sp[oW2 + j * kHid + k] * h1[r * kLd + k];
    const float hj = fmaxf(a, 0.0f);
    h2[r * kLd + j] = hj;
    ya += sp[oW3 + j] * hj;
  }
  const float y = tanhf(ya);
  const float wi = live ? w[row] : 0.0f;
  const float e = live ? y - t[row] : 0.0f;
  const float g3 = 2.0f * wi * e * (1.0f - y * y);   // times 1 / sum w later
  d3[r] = g3;
  for (int j = 0; j < kHid; ++j) d2[r * kLd + j] = h2[r * kLd + j] > 0.0f ? g3 * sp[oW3 + j] : 0.0f;
  for (int k = 0; k < kHid; ++k) {
    float a = 0.0f;
    for (int j = 0; j < kHid; ++j) a += sp[oW2 + j * kHid + k] * d2[r * kLd + j];
    d1[r * kLd + k] = h1[r * kLd + k] > 0.0f ? a : 0.0f;
  }
  // loss sums of the tile (fixed order: warp shuffles, then warps in order)
  double sl = double(wi) * double(e) * double(e), sw = double(wi);
  for (int o = 16; o > 0; o >>= 1) {
    sl += __shfl_xor_sync(kFull, sl, o);
    sw += __shfl_xor_sync(kFull, sw, o);
  }
  __shared__ double red[2][kTile / 32];
  if ((r & 31) == 0) {
    red[0][r >> 5] = sl;
    red[1][r >> 5] = sw;
  }
  __syncthreads();
  if (r == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < kTile / 32; ++q) {
      a += red[0][q];
      b += red[1][q];
    }
    psums[2 * blockIdx.x] = a;
    psums[2 * blockIdx.x + 1] = b;
  }
  // per-parameter sums over the tile's rows
  float* out = partial + size_t(blockIdx.x) * kN;
  for (int p = r; p < kN; p += kTile) {
    float g = 0.0f;
    if (p < oB1) {
      const int k = p / kIn, i = p % kIn;
      for (int q = 0; q < kTile; ++q) g += d1[q * kLd + k] * xs[q * kIn + i];
    } else if (p < oW2) {
      const int k = p - oB1;
      for (int q = 0; q < kTile; ++q) g += d1[q * kLd + k];
    } else if (p < oB2) {
      const int j = (p - oW2) / kHid, k = (p - oW2) % kHid;
      for (int q = 0; q < kTile; ++q) g += d2[q * kLd + j] * h1[q * kLd + k];
    } else if (p < oW3) {
      const int j = p - oB2;
      for (int q = 0; q < kTile; ++q) g += d2[q * kLd + j];
    } else if (p < oB3) {
      const int j = p - oW3;
      for (int q = 0; q < kTile; ++q) g += d3[q] * h2[q * kLd + j];
    } else {
      for (int q = 0; q < kTile; ++q) g += d3[q];
    }
    out[p] = g;
  }
}

__global__ void k_grad_reduce(const float* __restrict__ partial, const double* __restrict__ psums,
                              int nb, float* __restrict__ grad, double* __restrict__ loss2) {
  __shared__ double inv;
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < nb; ++q) {
      a += psums[2 * q];
      b += psums[2 * q + 1];
    }
    inv = b > 0.0 ? 1.0 / b : 0.0;
    if (blockIdx.x == 0) {
      loss2[0] = a * inv;
      loss2[1] = b;
    }
  }
  __syncthreads();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kN) return;
  double g = 0.0;
  for (int q = 0; q < nb; ++q) g += double(partial[size_t(q) * kN + p]);
  grad[p] = float(g * inv);
}

__global__ void k_adam(float* __restrict__ params, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kN) return;
  const float gp = g[p];
  const float mp = 0.9f * m[p] + 0.1f * gp;
  const float vp = 0.999f * v[p] + 0.001f * gp * gp;
  m[p] = mp;
  v[p] = vp;
  // c1 = 1 / (1 - beta1^k), c2 = 1 / (1 - beta2^k)
  params[p] -= lr * (mp * c1) / (sqrtf(vp * c2) + 1e-8f);
}

inline unsigned blocks_for(int64_t n, int t) { return unsigned((n + t - 1) / t); }

}  // namespace

size_t mlp_tile_smem() {
  return (size_t(kN) + size_t(kTile) * kIn + 4 * size_t(kTile) * kLd + kTile) * sizeof(float);
}
int64_t mlp_grad_blocks(int64_t B) { return (B + kTile - 1) / kTile; }

cudaError_t launch_features(View v, const float* u, const uint32_t* soff, const void* samp,
                            bool fp16, float* X, cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  if (fp16)
    k_features<__half><<<blocks_for(v.n, kFwdThreads), kFwdThreads, 0, s>>>(
        v, u, soff, reinterpret_cast<const __half*>(samp), X);
  else
    k_features<float><<<blocks_for(v.n, kFwdThreads), kFwdThreads, 0, s>>>(
        v, u, soff, reinterpret_cast<const float*>(samp), X);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float* params, const float* X, int64_t B, float* y,
                               cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  k_forward<<<blocks_for(B, kFwdThreads), kFwdThreads, 0, s>>>(params, X, B, y);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_warm_start(View v, const float* u, const uint32_t* soff, const void* samp,
                              bool fp16, const float* params, float* out, cudaStream_t s) {
  if (v.n <= 0) return cudaSuccess;
  if (fp16)
    k_warm_start<__half><<<blocks_for(v.n, kFwdThreads), kFwdThreads, 0, s>>>(
        v, u, soff, reinterpret_cast<const __half*>(samp), params, out);
  else
    k_warm_start<float><<<blocks_for(v.n, kFwdThreads), kFwdThreads, 0, s>>>(
        v, u, soff, reinterpret_cast<const float*>(samp), params, out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const float* params, const float* X, const float* t, const float* w,
                            const int32_t* rows, int64_t B, float* partial, double* psums,
                            float* grad, double* loss2, cudaStream_t s) {
  const int64_t nb = mlp_grad_blocks(B);
  if (nb <= 0) return cudaErrorInvalidValue;
  const size_t sm = mlp_tile_smem();
  cudaError_t e = cudaFuncSetAttribute(k_grad_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  if (e != cudaSuccess) return e;
  k_grad_tile<<<unsigned(nb), kTile, sm, s>>>(params, X, t, w, rows, B, partial, psums);
  count_launches(1);
  k_grad_reduce<<<blocks_for(kN, 256), 256, 0, s>>>(partial, psums, int(nb), grad, loss2);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* params, float* m, float* v, const float* g, float lr, int64_t step,
                        cudaStream_t s) {
  const float c1 = float(1.0 / (1.0 - std::pow(0.9, double(step))));
  const float c2 = float(1.0 / (1.0 - std::pow(0.999, double(step))));
  k_adam<<<blocks_for(kN, 256), 256, 0, s>>>(params, m, v, g, lr, c1, c2);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace ofu
