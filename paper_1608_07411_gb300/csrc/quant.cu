// Eq. 7: quantisation error between a field on the finest voxels (a fully
// refined run) and the leaves of an octree,
//   err = sum over leaves n of | u(n) - (1 / |n|) integral over n of u_fine |.
// A leaf covers the contiguous Morton range [key, key + h^3) of finest voxels,
// so its mean is a difference of two float64 prefix sums of the fine field;
// the per-leaf terms are summed by the same fixed-order scan.
#include "quant.cuh"

namespace ofu {

namespace {

constexpr int kThreads = 256;

unsigned blocks_for(int64_t n) { return unsigned((n + kThreads - 1) / kThreads); }

__global__ void k_widen_f64(const float* __restrict__ in, int64_t n, double* __restrict__ out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] = double(in[i]);
}

__global__ void k_quant_terms(View v, const float* __restrict__ u, const double* __restrict__ cfine,
                              double* __restrict__ terms) {
  const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l >= v.n) return;
  const int64_t k = int64_t(v.key[l]);
  const int64_t h3 = int64_t(1) << (3 * (v.D - v.level[l]));
  const double mean = (cfine[k + h3] - cfine[k]) / double(h3);
  terms[l] = fabs(double(u[l]) - mean);
}

}  // namespace

cudaError_t launch_quant_error(View v, const float* u, const float* fine, double* cfine,
                               double* terms, double* tmp, cudaStream_t s) {
  const int64_t nf = int64_t(1) << (3 * v.D);
  k_widen_f64<<<blocks_for(nf), kThreads, 0, s>>>(fine, nf, cfine);
  count_launches(1);
  cudaError_t e = scan_exclusive<double>(cfine, cfine, nf, tmp, s);   // cfine[nf] = total
  if (e != cudaSuccess) return e;
  if (v.n > 0) {
    k_quant_terms<<<blocks_for(v.n), kThreads, 0, s>>>(v, u, cfine, terms);
    count_launches(1);
  }
  e = scan_exclusive<double>(terms, terms, v.n, tmp, s);              // terms[n] = the sum
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace ofu
