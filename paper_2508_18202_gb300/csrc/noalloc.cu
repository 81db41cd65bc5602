// noalloc.cu -- sc_lbm_quad_moments_noalloc: the quadrature mean / standard
// deviation reduction of sc_lbm_moments for a per-node field the caller
// already holds, run without any device allocation and without a handle or
// workspace.
//
// Who needs it: callers that cannot allocate device memory at the point where
// they want the statistics -- a process whose free HBM is already reserved by
// another allocator (a PyTorch caching allocator or a serving pool that takes
// the device's memory up front, where cudaMalloc fails or forces a cache
// flush), and code on a latency-critical stream, where cudaMalloc / cudaFree
// would synchronise the whole device.  Such a caller cannot size and hand
// over a workspace either.
//
// The quadrature weights travel by value, as an 8 KB __grid_constant__ kernel
// parameter (the launch copies them, so the caller's host array may be reused
// as soon as the call returns, and a captured launch keeps its own copy).  The
// one piece of device scratch left, the counter of non-finite inputs, lives in
// a fixed file-scope device array: a static __device__ symbol that every GPU
// on which the library's module is loaded holds until the process exits.  Its
// device address, and the device's SM count that sizes the grid, are looked
// up once per device by the first call made with that device current; that
// first call must not be inside a stream capture.  Later calls issue only a
// memset, the kernel and (with d_nonfinite) a device-to-device copy, all of
// which a stream capture records.  All calls share the counter (it is cleared
// at the start of each call): calls whose device work overlaps (different
// streams without ordering, several host threads) race on it.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <stdarg.h>

#include <mutex>

#include "sclbm.h"

namespace {

constexpr int kNoallocMaxNodes = SC_NOALLOC_MAX_NODES;
constexpr int kMaxDevices = 64;

// The device scratch of the entry point, a file-scope array at a 256-byte
// boundary: one word, the count of non-finite field values (cleared per
// call).  Its size does not depend on the request; the request's limit
// (kNoallocMaxNodes) comes from the kernel-parameter space of the weights.
constexpr int kNoallocScratchWords = 1;
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoallocScratchWords];

// The weights a_j by value: 8 KB, inside the 32 KB kernel-parameter limit.
struct QuadWeights {
  double a[kNoallocMaxNodes];
};
static_assert(sizeof(QuadWeights) + 64 <= 32764, "kernel parameter space");

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

// printf-style message into the caller's buffer (nothing when err is NULL).
void put_err(char* err, size_t err_len, const char* fmt, ...) {
  if (!err || !err_len) return;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(err, err_len, fmt, ap);
  va_end(ap);
}

// Device address of the counter and the SM count of the current device (looked up once per device, with that device current).
int setup_for_current_device(void** out, int* sms, char* err, size_t err_len) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    put_err(err, err_len, "cudaGetDevice failed: %s", cudaGetErrorString(e));
    return SC_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    put_err(err, err_len, "device ordinal %d beyond the %d devices the scratch table covers", dev, kMaxDevices);
    return SC_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      put_err(err, err_len, "cudaGetSymbolAddress of the no-alloc counter failed on device %d: %s", dev,
              cudaGetErrorString(e));
      return SC_ERR_CUDA;
    }
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || n < 1) {
      put_err(err, err_len, "cudaDeviceGetAttribute(MultiProcessorCount) failed on device %d: %s", dev,
              cudaGetErrorString(e));
      return SC_ERR_CUDA;
    }
    g_sm_count[dev] = n;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  *sms = g_sm_count[dev];
  return SC_OK;
}

// Per cell c: s1 = sum_j a_j Q_j(c), s2 = sum_j a_j Q_j(c)^2 (FP64, nodes in
// order), mean = s1 / sum_j a_j, std = sqrt(max(s2 / sum_j a_j - mean^2, 0))
// -- the same arithmetic as the handle path's moment reduction.  Non-finite
// Q_j(c) are counted in the counter.  Every lane of a warp reads the same
// weight at the same time: a broadcast from the parameter bank.
__global__ void __launch_bounds__(256) quad_moments_noalloc_kernel(
    const double* __restrict__ field, long long n_cells, int n_nodes, const __grid_constant__ QuadWeights w,
    double wsum, double* __restrict__ mean, double* __restrict__ stdev, unsigned long long* nonfinite) {
  unsigned bad = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n_cells; c += stride) {
    double s1 = 0.0, s2 = 0.0;
    for (int j = 0; j < n_nodes; ++j) {
      const double q = field[(long long)j * n_cells + c];
      if (!isfinite(q)) ++bad;
      const double aq = w.a[j] * q;
      s1 += aq;
      s2 += aq * q;
    }
    const double m = s1 / wsum;
    double var = s2 / wsum - m * m;
    if (var < 0.0) var = 0.0;
    mean[c] = m;
    stdev[c] = sqrt(var);
  }
  const unsigned total = __reduce_add_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0 && total) atomicAdd(nonfinite, (unsigned long long)total);
}

}  // namespace

extern "C" int sc_lbm_quad_moments_noalloc(const double* d_field, int n_nodes, long long n_cells,
                                           const double* weights, double* d_mean, double* d_stdev,
                                           unsigned long long* d_nonfinite, void* stream, char* err,
                                           size_t err_len) {
  if (err && err_len) err[0] = '\0';
  if (n_nodes < 1 || n_cells < 0) {
    put_err(err, err_len, "n_nodes = %d and n_cells = %lld must be >= 1 and >= 0", n_nodes, n_cells);
    return SC_ERR_ARG;
  }
  if (n_nodes > kNoallocMaxNodes) {
    put_err(err, err_len, "n_nodes = %d exceeds the no-alloc maximum of %d nodes", n_nodes,
            kNoallocMaxNodes);
    return SC_ERR_SCRATCH;
  }
  if (!weights) {
    put_err(err, err_len, "null weights");
    return SC_ERR_ARG;
  }
  double wsum = 0.0;
  for (int j = 0; j < n_nodes; ++j) wsum += weights[j];
  if (!(wsum > 0.0) || !isfinite(wsum)) {
    put_err(err, err_len, "the weights must have a positive finite sum");
    return SC_ERR_ARG;
  }
  if (n_cells > 0 && (!d_field || !d_mean || !d_stdev)) {
    put_err(err, err_len, "null field or output pointer");
    return SC_ERR_ARG;
  }
  void* base = nullptr;
  int sms = 0;
  int rc = setup_for_current_device(&base, &sms, err, err_len);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* d_count = (unsigned long long*)base;
  QuadWeights w;
  memcpy(w.a, weights, sizeof(double) * (size_t)n_nodes);
  memset(w.a + n_nodes, 0, sizeof(double) * (size_t)(kNoallocMaxNodes - n_nodes));
  cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess && n_cells > 0) {
    // grid-stride loop: at most 8 resident blocks of 256 threads per SM
    long long blocks = (n_cells + 255) / 256;
    if (blocks > 8LL * sms) blocks = 8LL * sms;
    quad_moments_noalloc_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_field, n_cells, n_nodes, w, wsum,
                                                                 d_mean, d_stdev, d_count);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && d_nonfinite)
    e = cudaMemcpyAsync(d_nonfinite, d_count, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) {
    put_err(err, err_len, "CUDA error in the no-alloc moment reduction: %s", cudaGetErrorString(e));
    return SC_ERR_CUDA;
  }
  return SC_OK;
}
