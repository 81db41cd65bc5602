// quantiles.cu -- confidence bounds from the gPC surrogate (Sec. 2.4 step 7:
// confidence intervals from the expansion coefficients; Sec. 4 profile
// bands).  For each requested cell a block evaluates the surrogate
// sum_a c_a(x) Phi_a(s_m) at the M input samples into shared memory, sorts
// them with a bitonic network and writes the k-th smallest values.
#include <cuda_runtime.h>
#include <math.h>

#include "sclbm_internal.h"

namespace sclbm {
namespace {

constexpr int kQuantThreads = 256;

// coef [P][ncell] (FP64), phi [M][P], cells [n_cells], kidx [nq] (1-based
// ranks); out [nq][n_cells].  Dynamic shared memory: P + Mp doubles, Mp the
// power of two >= M (the tail padded with +inf).
__global__ void __launch_bounds__(kQuantThreads) gpc_quantile_kernel(
    const double* __restrict__ coef, long long ncell, int P, const int32_t* __restrict__ cells,
    int n_cells, const double* __restrict__ phi, int M, int Mp, const int32_t* __restrict__ kidx, int nq,
    double* __restrict__ out) {
  extern __shared__ double sh[];
  double* cs = sh;      // [P]
  double* y = sh + P;   // [Mp]
  const long long c = cells[blockIdx.x];
  for (int a = threadIdx.x; a < P; a += blockDim.x) cs[a] = coef[(long long)a * ncell + c];
  __syncthreads();
  for (int m = threadIdx.x; m < Mp; m += blockDim.x) {
    double v = INFINITY;
    if (m < M) {
      const double* row = phi + (long long)m * P;
      v = 0.0;
      for (int a = 0; a < P; ++a) v = fma(cs[a], row[a], v);
    }
    y[m] = v;
  }
  __syncthreads();
  // bitonic sort, ascending
  for (int k = 2; k <= Mp; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < Mp; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const double a = y[i], b = y[l];
          const bool up = (i & k) == 0;
          if (up ? (a > b) : (a < b)) {
            y[i] = b;
            y[l] = a;
          }
        }
      }
      __syncthreads();
    }
  for (int t = threadIdx.x; t < nq; t += blockDim.x) out[(long long)t * n_cells + blockIdx.x] = y[kidx[t] - 1];
}

}  // namespace

int launch_gpc_quantiles(const double* coef, long long ncell, int P, const int32_t* cells, int n_cells,
                         const double* phi, int M, const int32_t* kidx, int nq, double* out, void* stream) {
  if (n_cells <= 0) return (int)cudaSuccess;
  int Mp = 1;
  while (Mp < M) Mp <<= 1;
  const size_t smem = sizeof(double) * (size_t)(P + Mp);
  cudaError_t e = cudaFuncSetAttribute(gpc_quantile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  gpc_quantile_kernel<<<n_cells, kQuantThreads, smem, (cudaStream_t)stream>>>(coef, ncell, P, cells, n_cells, phi,
                                                                              M, Mp, kidx, nq, out);
  return (int)cudaGetLastError();
}

}  // namespace sclbm
