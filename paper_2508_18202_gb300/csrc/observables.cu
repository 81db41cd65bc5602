// observables.cu -- the observables of libsclbm for sm_103a (GB300): the
// initial populations, the ensemble statistics of the quadrature and the gPC
// projection (arXiv:2508.18202 Sec. 2.3, Eqs. quad_moments, coef_discrete),
// the vertical profiles with their 95% band, one node's exported populations
// and velocity, per-node time averages, the Q-criterion and the state check.
// They read the populations the stream-collide kernels of lbm_kernels.cu
// leave behind (layout and AA time levels are described there) and do not
// depend on the collision, so they are compiled once, in this unit.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "lbm_device.cuh"
#include "sclbm_internal.h"

namespace sclbm {
namespace {

// ------------------------------------------------------------ initialisation
// Every slot of every row (padding included): g = 0 (shifted) or f = w.
template <class S, bool SHIFT>
__global__ void init_kernel(S* g, long long pitch, long long total) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int i = (int)((k / pitch) % kQ);
    using T = typename Store<S>::C;
    T v = T(0);
    if constexpr (!SHIFT) {
      v = i == 0 ? T(1.0 / 3.0) : (i <= 6 ? T(1.0 / 18.0) : T(1.0 / 36.0));
    }
    Store<S>::st(g + k, v);
  }
}

// ------------------------------------------------------------ observables
// Populations of time level n at a fluid cell (natural layout at even n,
// pulled at odd n) in the compute type, as stored: the in-place precisions
// give g_i = f_i - w_i (SHIFT), the FP64 plain path f_i.  The moments are
// summed on these values (macro), so the shift's precision carries into the
// observables; f_i itself is rebuilt only where it is exported.
template <class S, bool SHIFT>
__device__ __forceinline__ void gather_pops(const StepParams& P, const DevDomain& D, int node,
                                            unsigned long long n, int x, int y, int z,
                                            long long idx, LinkWord lw,
                                            typename Store<S>::C g[kQ]) {
  using T = typename Store<S>::C;
  if constexpr (!SHIFT) {
    // FP64 plain: two arrays, natural layout in the current one
    const double* cur = reinterpret_cast<const double*>((n & 1ull) ? D.g2 : D.g) +
                        (long long)node * kQ * D.pitch;
#pragma unroll
    for (int i = 0; i < kQ; ++i) g[i] = T(cur[(long long)i * D.pitch + idx]);
  } else {
    const Node<S> N = node_view<S>(D, node);
    if ((n & 1ull) == 0) {
#pragma unroll
      for (int i = 0; i < kQ; ++i) g[i] = Store<S>::ld(N.g + (long long)i * D.pitch + idx);
    } else {
      // P.wp is the inflow factor of level n (the launch's n_host)
      T ux, uy, uz;
      if (lw & kLinkSlow) {
        const ListedRef L = listed_ref(D, listed_index(D, idx));
        inflow_velocity<S>(N, z, wind_pull<T>(P), ux, uy, uz);
        listed_pull<S, false>(L, N.g, N.bout, ux, uy, uz, wind_pull<T>(P).scale, g);
      } else {
        wall_velocity<S>(N, lw, z, wind_pull<T>(P), ux, uy, uz);
        fast_pull<S, false>(N.g + idx, lw, (int)D.pitch, D.nx, D.nx * D.ny, ux, uy, uz, wind_pull<T>(P).scale,
                            g);
      }
    }
  }
}

// Density and velocity from the populations gather_pops gives (Sec. 2.2:
// rho = sum_i f_i, rho u = sum_i c_i f_i).  SHIFT: g_i = f_i - w_i, so
// rho = 1 + sum_i g_i and, as sum_i w_i c_i = 0, rho u = sum_i c_i g_i; both
// sums run over the small deviations from rest, as in the collision.
template <class T, bool SHIFT>
__device__ __forceinline__ void macro(const T g[kQ], T& rho, T& ux, T& uy, T& uz) {
  T m0 = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    m0 += g[i];
    if (CX(i)) jx += CX(i) > 0 ? g[i] : -g[i];
    if (CY(i)) jy += CY(i) > 0 ? g[i] : -g[i];
    if (CZ(i)) jz += CZ(i) > 0 ? g[i] : -g[i];
  }
  rho = SHIFT ? T(1) + m0 : m0;
  ux = jx / rho;
  uy = jy / rho;
  uz = jz / rho;
}

// |u| in the compute type T from the velocity macro() gives: (ux^2 + uy^2) +
// uz^2, each operation rounded once (no contraction) and the correctly
// rounded square root, so a host reproduces it bit for bit from an exported
// velocity.  The in-place precisions take it in FP32 (the velocity carries
// FP32 rounding already; an FP64 square root costs the FP64 pipe a dozen
// operations per node and cell), the FP64 plain path in FP64.
template <class T>
__device__ __forceinline__ T speed(T ux, T uy, T uz) {
  if constexpr (sizeof(T) == 4)
    return __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(ux, ux), __fmul_rn(uy, uy)), __fmul_rn(uz, uz)));
  else
    return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy)), __dmul_rn(uz, uz)));
}

// mean = S1 / W, std = sqrt(max(S2 / W - mean^2, 0)) (Eq. quad_moments; the
// clamp guards negative sparse-grid weights), each operation rounded once so
// that every kernel finishing sums gives the same bits for the same sums.
__device__ __forceinline__ void finish_moments(double s1, double s2, double wsum, double& mean, double& sd) {
  mean = __ddiv_rn(s1, wsum);
  double var = __dsub_rn(__ddiv_rn(s2, wsum), __dmul_rn(mean, mean));
  if (var < 0.0) var = 0.0;
  sd = __dsqrt_rn(var);
}

// Compensated FP32 sum of products (the Dot2 scheme of Ogita, Rump & Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005): the running
// sum is the unevaluated pair hi + lo.  Each term b q, with b = bh + bl a
// double split into two floats and q a float, enters as the exact product
// bh q = p + e (TwoProduct by FMA) plus the small bl q; TwoSum (Knuth) adds p
// to hi exactly and the rounding errors gather in lo; a final Fast2Sum keeps
// |lo| <= ulp(hi) / 2, so hi + lo is the float pair nearest the sum.  The
// result carries about twice FP32's precision (relative error near
// n 2^-48 of the sum of |terms| for n terms).
//
// Two gPC terms go at once on Blackwell's packed FP32x2 operations
// (__fmul2_rn, __ffma2_rn, __fadd2_rn; x - y as fma(y, -1, x), one rounding of
// the exact difference), at half the instructions.  Each packed operation
// rounds lane by lane as its scalar counterpart (checked on 4 M random,
// subnormal and cancelling operands), but the compiled sequence is not always
// the scalar one step for step: its sums can differ from the scalar scheme's
// in the last bits (at most 2^-47 of the sum of |terms| in a 13-term check),
// which is the scheme's own error level; the GPU tests hold the sums to 1e-12
// of the sum of |terms| against the FP64 projection.
struct DF {
  float hi, lo;
};
struct DF2 {
  float2 hi, lo;  // .x: term a, .y: term a + 1
};
__device__ __forceinline__ float2 sub2(float2 x, float2 y) {
  return __ffma2_rn(y, make_float2(-1.0f, -1.0f), x);
}
// s += b q for two terms; b = (bh_a, bh_a+1, bl_a, bl_a+1).
__device__ __forceinline__ void df2_dot_add(DF2& s, float4 b, float2 q) {
  const float2 bh = make_float2(b.x, b.y), bl = make_float2(b.z, b.w);
  const float2 p = __fmul2_rn(bh, q);
  const float2 e = __ffma2_rn(bh, q, make_float2(-p.x, -p.y));
  const float2 t = __fmul2_rn(bl, q);
  const float2 sum = __fadd2_rn(s.hi, p);
  const float2 bb = sub2(sum, s.hi);
  const float2 err = __fadd2_rn(sub2(s.hi, sub2(sum, bb)), sub2(p, bb));
  const float2 lo = __fadd2_rn(s.lo, __fadd2_rn(err, __fadd2_rn(e, t)));
  const float2 hi = __fadd2_rn(sum, lo);
  s.lo = sub2(lo, sub2(hi, sum));
  s.hi = hi;
}
// The pair nearest a double (its value to 48 bits) and back.
__device__ __forceinline__ DF df_from(double v) {
  DF s;
  s.hi = __double2float_rn(v);
  s.lo = __double2float_rn(v - (double)s.hi);
  return s;
}
__device__ __forceinline__ double df_value(DF s) { return (double)s.hi + (double)s.lo; }

// Ensemble statistics of |u| per cell (Eq. quad_moments) and the gPC
// projection (Eq. coef_discrete): one thread per cell runs over the nodes in
// order, S1, S2 and the gPC sums in FP64.  This form serves the FP64 plain
// path and the time-averaged fields (FP64 per-node averages); the in-place
// precisions' current |u| goes through moments_pair_kernel.  PM >= A.P is the
// compile-time size of the coefficient array (a small basis holds few
// registers).  raw: write the sums S1, S2 (and the gPC sums); with accumulate
// the sums start from the values in the output arrays, so node ranges reduced
// one after another (waves, shards) continue one sum per cell and carry the
// bits of one reduction over all nodes.
// AVG: the per-node time averages (A.avg) instead of the current |u|.
template <class S, bool SHIFT, int PM, bool AVG>
__global__ void __launch_bounds__(256) moments_kernel(const __grid_constant__ StepParams P, MomentArgs A) {
  using T = typename Store<S>::C;
  const DevDomain& D = P.dom[A.domain];
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  bool bad = false;
  if (c < D.ncell) {
    const unsigned long long n = P.n_host;
    const int x = (int)(c % D.nx);
    const int y = (int)((c / D.nx) % D.ny);
    const int z = (int)(c / ((long long)D.nx * D.ny));
    const LinkWord lw = __ldg(D.link + c);
    const bool acc = A.raw && A.accumulate;
    double s1 = acc ? A.mean[c] : 0.0, s2 = acc ? A.stdev[c] : 0.0;
    double coef[PM > 0 ? PM : 1];
#pragma unroll
    for (int a = 0; a < PM; ++a) coef[a] = (acc && a < A.P) ? A.coef[(long long)a * D.ncell + c] : 0.0;
    if (!(lw & kLinkSolid)) {
      for (int j = 0; j < A.nq; ++j) {
        double q;
        if constexpr (AVG) {
          q = A.avg[(long long)j * D.ncell + c] * A.avg_scale;
          if (!isfinite(q)) bad = true;
        } else {
          T g[kQ];
          gather_pops<S, SHIFT>(P, D, j, n, x, y, z, c, lw, g);
          T rho, ux, uy, uz;
          macro<T, SHIFT>(g, rho, ux, uy, uz);
          if (!(rho > T(0)) || !isfinite(double(ux + uy + uz)) || !isfinite(double(rho))) bad = true;
          q = double(speed<T>(ux, uy, uz));
        }
        const double* ab = A.ab + (long long)j * A.stride;
        const double aq = ab[0] * q;
        s1 += aq;
        s2 = fma(aq, q, s2);
#pragma unroll
        for (int a = 0; a < PM; ++a)
          if (a < A.P) coef[a] = fma(ab[1 + a], q, coef[a]);
      }
    }
    if (A.raw) {
      A.mean[c] = s1;
      A.stdev[c] = s2;
    } else {
      finish_moments(s1, s2, A.wsum, A.mean[c], A.stdev[c]);
    }
    if (A.coef) {
#pragma unroll
      for (int a = 0; a < PM; ++a)
        if (a < A.P) A.coef[(long long)a * D.ncell + c] = coef[a];
    }
  }
  const unsigned any = __ballot_sync(0xffffffffu, bad);
  if (any && (threadIdx.x & 31) == 0) atomicOr(P.err, kErrDiverged);
}

// The same statistics for the in-place precisions (|u| of the current level
// from the shifted populations, in FP32): one thread per cell over the nodes
// in order, S1 and S2 in FP64, the gPC sums as compensated FP32 pairs two
// terms at a time (df2_dot_add) -- |u| is a float, so each product is exact
// to 48 bits and the FP64 pipe, a small fraction of the FP32 rate, is left to
// S1 and S2.  PM = gpc_pair_pad(A.P) is the padded basis size and the row
// length of A.abf (its pad terms are zero and are not written).  raw and
// accumulate as in moments_kernel: S1 and S2 continue one FP64 sum per cell,
// the pair sums restart from the nearest pair of the stored double, which
// agrees with one reduction over all nodes to the pairs' 48-bit rounding.
// This form serves the small bases (PM <= kMomCellMaxP); a large basis holds
// too many accumulators per thread for it and goes to moments_split_kernel.
constexpr int kMomCellMaxP = 12;

template <class S, int PM>
__global__ void __launch_bounds__(256) moments_pair_kernel(const __grid_constant__ StepParams P, MomentArgs A) {
  using T = typename Store<S>::C;
  constexpr int NP = PM > 0 ? PM / 2 : 1;
  const DevDomain& D = P.dom[A.domain];
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  bool bad = false;
  if (c < D.ncell) {
    const unsigned long long n = P.n_host;
    const int x = (int)(c % D.nx);
    const int y = (int)((c / D.nx) % D.ny);
    const int z = (int)(c / ((long long)D.nx * D.ny));
    const LinkWord lw = __ldg(D.link + c);
    const bool acc = A.raw && A.accumulate;
    double s1 = acc ? A.mean[c] : 0.0, s2 = acc ? A.stdev[c] : 0.0;
    DF2 cf[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int a = 2 * k;
      const DF u = df_from((acc && a < A.P) ? A.coef[(long long)a * D.ncell + c] : 0.0);
      const DF v = df_from((acc && a + 1 < A.P) ? A.coef[(long long)(a + 1) * D.ncell + c] : 0.0);
      cf[k].hi = make_float2(u.hi, v.hi);
      cf[k].lo = make_float2(u.lo, v.lo);
    }
    if (!(lw & kLinkSolid)) {
      const float4* bf = A.abf;
      const double* ab = A.ab;
      for (int j = 0; j < A.nq; ++j, bf += NP, ab += A.stride) {
        T g[kQ];
        gather_pops<S, true>(P, D, j, n, x, y, z, c, lw, g);
        T rho, ux, uy, uz;
        macro<T, true>(g, rho, ux, uy, uz);
        if (!(rho > T(0)) || !isfinite(ux + uy + uz) || !isfinite(rho)) bad = true;
        const float qf = speed<T>(ux, uy, uz);
        const double q = double(qf);
        const double aq = __ldg(ab) * q;
        s1 += aq;
        s2 = fma(aq, q, s2);
        if constexpr (PM > 0) {
          const float2 q2 = make_float2(qf, qf);
#pragma unroll
          for (int k = 0; k < NP; ++k) df2_dot_add(cf[k], __ldg(bf + k), q2);
        }
      }
    }
    if (A.raw) {
      A.mean[c] = s1;
      A.stdev[c] = s2;
    } else {
      finish_moments(s1, s2, A.wsum, A.mean[c], A.stdev[c]);
    }
    if (A.coef) {
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const int a = 2 * k;
        if (a < A.P) A.coef[(long long)a * D.ncell + c] = df_value(DF{cf[k].hi.x, cf[k].lo.x});
        if (a + 1 < A.P) A.coef[(long long)(a + 1) * D.ncell + c] = df_value(DF{cf[k].hi.y, cf[k].lo.y});
      }
    }
  }
  const unsigned any = __ballot_sync(0xffffffffu, bad);
  if (any && (threadIdx.x & 31) == 0) atomicOr(P.err, kErrDiverged);
}

// The large-basis form of moments_pair_kernel, with the node loop split over
// warp pairs: warps 2p and 2p + 1 of a block share 32 consecutive cells and take
// the nodes two at a time, warp 2p evaluating |u| at node j, warp 2p + 1 at
// node j + 1 (each warp reads whole 128-byte rows), and trade the values
// through shared memory.  Each thread of a pair then carries half of its
// cell's sums over both nodes, in node order: the thread of warp 2p the FP64
// S1 (as fma(a_j q_j, 1, S1), which is the rounded sum), that of warp 2p + 1
// the FP64 S2 (fma(a_j q_j, q_j, S2)), and each the compensated FP32 pair
// sums of half the gPC terms, two terms at a time (df2_dot_add) -- |u| is a
// float, so each product is exact to 48 bits and the FP64 pipe, a small
// fraction of the FP32 rate, is left to S1 and S2.  Every sum sees the nodes
// in the order and with the operations of a one-thread loop, while a thread's
// chain of dependent loads and arithmetic is half as long and it holds half
// the accumulators.  PM = gpc_pair_pad(A.P) is the padded basis size (a
// multiple of 4) and the row length of A.abf; its pad terms are zero and are
// not written.  raw and accumulate as in moments_pair_kernel; the two forms
// give the same bits (measured on 6-, 10- and 21-term bases).  Three blocks per SM (80 registers, a few bytes
// spilled at the largest bases) beat two unspilled ones: the wait on
// dependent loads and arithmetic, not the instruction count, bounds this
// reduction.
constexpr int kMomPairs = 4;  // warp pairs per block (256 threads, 128 cells)

template <class S, int PM>
__global__ void __launch_bounds__(64 * kMomPairs, 3) moments_split_kernel(const __grid_constant__ StepParams P,
                                                                         MomentArgs A) {
  using T = typename Store<S>::C;
  static_assert(PM % 4 == 0, "two packed pairs of terms per thread pair");
  constexpr int NH = PM > 0 ? PM / 4 : 1;  // packed pairs per thread
  // the values a warp hands to its partner: [buffer][pair][warp of the pair][lane]
  __shared__ float x_qf[2][kMomPairs][2][32];
  __shared__ double x_q[2][kMomPairs][2][32];
  __shared__ double x_aq[2][kMomPairs][2][32];
  const DevDomain& D = P.dom[A.domain];
  const int lane = threadIdx.x & 31;
  const int k = (threadIdx.x >> 5) & 1;  // 0: node j, S1, terms [0, PM/2); 1: node j + 1, S2, the rest
  const int pr = threadIdx.x >> 6;
  const long long c = (blockIdx.x * (long long)kMomPairs + pr) * 32 + lane;
  const bool inside = c < D.ncell;
  int x = 0, y = 0, z = 0;
  LinkWord lw = kLinkSolid;
  if (inside) {
    x = (int)(c % D.nx);
    y = (int)((c / D.nx) % D.ny);
    z = (int)(c / ((long long)D.nx * D.ny));
    lw = __ldg(D.link + c);
  }
  const bool fluid = inside && !(lw & kLinkSolid);
  const unsigned long long n = P.n_host;
  const bool acc = A.raw && A.accumulate;
  double s = (inside && acc) ? (k == 0 ? A.mean[c] : A.stdev[c]) : 0.0;
  DF2 cf[NH];
#pragma unroll
  for (int t = 0; t < NH; ++t) {
    const int a = 2 * (k * NH + t);
    const DF u = df_from((inside && acc && a < A.P) ? A.coef[(long long)a * D.ncell + c] : 0.0);
    const DF v = df_from((inside && acc && a + 1 < A.P) ? A.coef[(long long)(a + 1) * D.ncell + c] : 0.0);
    cf[t].hi = make_float2(u.hi, v.hi);
    cf[t].lo = make_float2(u.lo, v.lo);
  }
  bool bad = false;
  int buf = 0;
  for (int j = 0; j < A.nq; j += 2, buf ^= 1) {
    const int jn = j + k;  // the node this warp evaluates
    const bool two = j + 1 < A.nq;
    float qf = 0.0f;
    double q = 0.0, aq = 0.0;
    if (fluid && jn < A.nq) {
      T g[kQ];
      gather_pops<S, true>(P, D, jn, n, x, y, z, c, lw, g);
      T rho, ux, uy, uz;
      macro<T, true>(g, rho, ux, uy, uz);
      if (!(rho > T(0)) || !isfinite(ux + uy + uz) || !isfinite(rho)) bad = true;
      qf = speed<T>(ux, uy, uz);
      q = double(qf);
      aq = __ldg(A.ab + (long long)jn * A.stride) * q;
    }
    x_qf[buf][pr][k][lane] = qf;
    x_q[buf][pr][k][lane] = q;
    x_aq[buf][pr][k][lane] = aq;
    // the two warps of the pair meet (named barrier 1 + pr, 64 threads); the
    // alternating buffers keep the next exchange from overwriting this one
    asm volatile("bar.sync %0, 64;" ::"r"(1 + pr) : "memory");
    const float qf_o = x_qf[buf][pr][k ^ 1][lane];
    const double q_o = x_q[buf][pr][k ^ 1][lane];
    const double aq_o = x_aq[buf][pr][k ^ 1][lane];
    const float qf0 = k ? qf_o : qf, qf1 = k ? qf : qf_o;
    const double aq0 = k ? aq_o : aq, aq1 = k ? aq : aq_o;
    if (fluid) {
      s = fma(aq0, k ? q_o : 1.0, s);
      if (two) s = fma(aq1, k ? q : 1.0, s);
      if constexpr (PM > 0) {
        const float4* b = A.abf + (long long)j * (PM / 2) + k * NH;
        const float2 q0 = make_float2(qf0, qf0);
#pragma unroll
        for (int t = 0; t < NH; ++t) df2_dot_add(cf[t], __ldg(b + t), q0);
        if (two) {
          const float2 q1 = make_float2(qf1, qf1);
#pragma unroll
          for (int t = 0; t < NH; ++t) df2_dot_add(cf[t], __ldg(b + PM / 2 + t), q1);
        }
      }
    }
  }
  x_q[buf][pr][k][lane] = s;
  asm volatile("bar.sync %0, 64;" ::"r"(1 + pr) : "memory");
  const double s_o = x_q[buf][pr][k ^ 1][lane];
  if (inside) {
    if (k == 0) {
      if (A.raw) {
        A.mean[c] = s;
        A.stdev[c] = s_o;
      } else {
        finish_moments(s, s_o, A.wsum, A.mean[c], A.stdev[c]);
      }
    }
    if (A.coef) {
#pragma unroll
      for (int t = 0; t < NH; ++t) {
        const int a = 2 * (k * NH + t);
        if (a < A.P) A.coef[(long long)a * D.ncell + c] = df_value(DF{cf[t].hi.x, cf[t].lo.x});
        if (a + 1 < A.P) A.coef[(long long)(a + 1) * D.ncell + c] = df_value(DF{cf[t].hi.y, cf[t].lo.y});
      }
    }
  }
  const unsigned any = __ballot_sync(0xffffffffu, bad);
  if (any && lane == 0) atomicOr(P.err, kErrDiverged);
}

// Vertical profiles: one warp per (column, layer); lanes take nodes and the
// FP64 sums are combined with warp shuffles.
template <class S, bool SHIFT>
__global__ void profiles_kernel(const __grid_constant__ StepParams P, MomentArgs A) {
  using T = typename Store<S>::C;
  const DevDomain& D = P.dom[A.domain];
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= A.n_p * D.nz) return;
  const int p = warp / D.nz;
  const int z = warp % D.nz;
  const int x = A.probes[2 * p], y = A.probes[2 * p + 1];
  const long long c = cidx(D, x, y, z);
  const LinkWord lw = __ldg(D.link + c);
  const unsigned long long n = P.n_host;
  double s1 = 0.0, s2 = 0.0;
  for (int j = lane; j < A.nq; j += 32) {
    double q = 0.0;
    if (!(lw & kLinkSolid)) {
      if (A.avg) {
        q = A.avg[(long long)j * D.ncell + c] * A.avg_scale;
      } else {
        T g[kQ];
        gather_pops<S, SHIFT>(P, D, j, n, x, y, z, c, lw, g);
        T rho, ux, uy, uz;
        macro<T, SHIFT>(g, rho, ux, uy, uz);
        q = double(speed<T>(ux, uy, uz));
      }
    }
    if (A.prof_nodes) A.prof_nodes[((long long)p * A.nq + j) * D.nz + z] = float(q);
    const double a = A.ab[(long long)j * A.stride];
    s1 += a * q;
    s2 += a * q * q;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (lane == 0) {
    double mean, sd;
    finish_moments(s1, s2, A.wsum, mean, sd);
    double* out = A.prof + ((long long)p * D.nz + z) * 4;
    out[0] = mean;
    out[1] = sd;
    out[2] = mean - 1.959963984540054 * sd;
    out[3] = mean + 1.959963984540054 * sd;
  }
}

// One node's populations (FP64, unshifted) and velocity at the current time.
template <class S, bool SHIFT>
__global__ void export_kernel(const __grid_constant__ StepParams P, int domain, int node,
                              double* f, float* u) {
  using T = typename Store<S>::C;
  const DevDomain& D = P.dom[domain];
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= D.ncell) return;
  const int x = (int)(c % D.nx);
  const int y = (int)((c / D.nx) % D.ny);
  const int z = (int)(c / ((long long)D.nx * D.ny));
  const LinkWord lw = __ldg(D.link + c);
  if (lw & kLinkSolid) {
    if (f)
      for (int i = 0; i < kQ; ++i) f[(long long)i * D.ncell + c] = 0.0;
    if (u) u[c] = u[D.ncell + c] = u[2 * D.ncell + c] = 0.0f;
    return;
  }
  T g[kQ];
  gather_pops<S, SHIFT>(P, D, node, P.n_host, x, y, z, c, lw, g);
  if (f)
#pragma unroll
    for (int i = 0; i < kQ; ++i) f[(long long)i * D.ncell + c] = SHIFT ? double(g[i]) + W<double>(i) : double(g[i]);
  if (u) {
    T rho, ux, uy, uz;
    macro<T, SHIFT>(g, rho, ux, uy, uz);
    u[c] = float(ux);
    u[D.ncell + c] = float(uy);
    u[2 * D.ncell + c] = float(uz);
  }
}

// Count cells whose stored populations sum to a non-finite or non-positive
// density (layout-independent: the stored 19 values of a cell always carry
// its density at the current or previous time level).
// Time average of |u| (the paper's time-averaged velocity magnitude fields,
// Sec. 2.4 step 6): adds |u| at the current level, per (node, cell), in FP64.
template <class S, bool SHIFT>
__global__ void average_add_kernel(const __grid_constant__ StepParams P, int domain, double* avg) {
  using T = typename Store<S>::C;
  const DevDomain& D = P.dom[domain];
  const long long total = D.ncell * D.nodes;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(k / D.ncell);
    const long long c = k - (long long)j * D.ncell;
    const LinkWord lw = __ldg(D.link + c);
    if (lw & kLinkSolid) continue;
    const int x = (int)(c % D.nx), y = (int)((c / D.nx) % D.ny), z = (int)(c / ((long long)D.nx * D.ny));
    T g[kQ];
    gather_pops<S, SHIFT>(P, D, j, P.n_host, x, y, z, c, lw, g);
    T rho, ux, uy, uz;
    macro<T, SHIFT>(g, rho, ux, uy, uz);
    avg[k] += double(speed<T>(ux, uy, uz));
  }
}

// Q-criterion (the vortex identification of the paper's figures):
// Q = (|Omega|^2 - |S|^2) / 2 with S and Omega the symmetric and antisymmetric
// parts of grad u, by central differences (dx = 1) where both neighbours
// along an axis are fluid, one-sided where one is, zero where none is;
// periodic axes wrap; solid cells get 0.
__device__ void qcriterion_cell(const DevDomain& D, const float* __restrict__ u, float* __restrict__ q,
                                long long c) {
  if (D.flags[c]) {
    q[c] = 0.0f;
    return;
  }
  const int xyz[3] = {(int)(c % D.nx), (int)((c / D.nx) % D.ny), (int)(c / ((long long)D.nx * D.ny))};
  const int dim[3] = {D.nx, D.ny, D.nz};
  double J[3][3];  // J[i][a] = d u_i / d x_a
  for (int a = 0; a < 3; ++a) {
    long long nb[2];
    bool ok[2];
    for (int sgn = 0; sgn < 2; ++sgn) {
      int p[3] = {xyz[0], xyz[1], xyz[2]};
      p[a] += sgn ? 1 : -1;
      ok[sgn] = true;
      if (p[a] < 0 || p[a] >= dim[a]) {
        if (D.bc[2 * a] == SC_BC_PERIODIC) p[a] = (p[a] + dim[a]) % dim[a];
        else ok[sgn] = false;
      }
      nb[sgn] = ok[sgn] ? cidx(D, p[0], p[1], p[2]) : c;
      if (ok[sgn] && D.flags[nb[sgn]]) ok[sgn] = false;
    }
    for (int i = 0; i < 3; ++i) {
      const float* ui = u + (long long)i * D.ncell;
      double d = 0.0;
      if (ok[0] && ok[1]) d = 0.5 * ((double)ui[nb[1]] - (double)ui[nb[0]]);
      else if (ok[1]) d = (double)ui[nb[1]] - (double)ui[c];
      else if (ok[0]) d = (double)ui[c] - (double)ui[nb[0]];
      J[i][a] = d;
    }
  }
  double s2 = 0.0, w2 = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int a = 0; a < 3; ++a) {
      const double sv = 0.5 * (J[i][a] + J[a][i]), wv = 0.5 * (J[i][a] - J[a][i]);
      s2 += sv * sv;
      w2 += wv * wv;
    }
  q[c] = (float)(0.5 * (w2 - s2));
}

__global__ void qcriterion_kernel(const __grid_constant__ StepParams P, int domain, const float* __restrict__ u,
                                  float* __restrict__ q) {
  const DevDomain& D = P.dom[domain];
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < D.ncell;
       c += (long long)gridDim.x * blockDim.x)
    qcriterion_cell(D, u, q, c);
}

// The quadrature moments from (possibly all-reduced) sums, as the moment
// kernel finishes them.
__global__ void finalize_moments_kernel(const double* __restrict__ s1, const double* __restrict__ s2, double wsum,
                                        double* __restrict__ mean, double* __restrict__ stdev, long long n) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
    finish_moments(s1[c], s2[c], wsum, mean[c], stdev[c]);
}

__global__ void scale_kernel(const double* __restrict__ in, double sc, double* __restrict__ out, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    out[k] = in[k] * sc;
}

template <class S, bool SHIFT>
__global__ void check_kernel(const __grid_constant__ StepParams P, unsigned long long* count) {
  unsigned long long local = 0;
  for (int d = 0; d < P.n_domains; ++d) {
    const DevDomain& D = P.dom[d];
    const long long total = D.ncell * D.nodes;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
      const long long c = k % D.ncell;
      const int node = (int)(k / D.ncell);
      if (__ldg(D.link + c) & kLinkSolid) continue;
      const S* g = reinterpret_cast<const S*>(D.g) + (long long)node * kQ * D.pitch;
      if constexpr (!SHIFT) {
        if (P.n_host & 1ull) g = reinterpret_cast<const S*>(D.g2) + (long long)node * kQ * D.pitch;
      }
      double rho = SHIFT ? 1.0 : 0.0;
      for (int i = 0; i < kQ; ++i) rho += double(Store<S>::ld(g + (long long)i * D.pitch + c));
      if (!(rho > 0.0) || !isfinite(rho)) ++local;
    }
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0 && local) {
    atomicAdd(count, local);
    atomicOr(P.err, kErrDiverged);
  }
}

int grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  if (g > 152LL * 64) g = 152LL * 64;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

int launch_init_equilibrium(const StepParams& P, int precision, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  for (int d = 0; d < P.n_domains; ++d) {
    const DevDomain& D = P.dom[d];
    const long long total = (long long)D.nodes * kQ * D.pitch;
    int rc = dispatch(precision, [&](auto tag) -> int {
      using S = std::remove_pointer_t<decltype(tag)>;
      if constexpr (std::is_same_v<S, double>) {
        init_kernel<double, false><<<grid_for(total, 256), 256, 0, s>>>((double*)D.g, D.pitch, total);
        init_kernel<double, false><<<grid_for(total, 256), 256, 0, s>>>((double*)D.g2, D.pitch, total);
      } else {
        init_kernel<S, true><<<grid_for(total, 256), 256, 0, s>>>((S*)D.g, D.pitch, total);
      }
      return (int)cudaGetLastError();
    });
    if (rc) return rc;
  }
  return 0;
}

int launch_moments(const StepParams& P, int precision, const MomentArgs& A, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const DevDomain& D = P.dom[A.domain];
  return dispatch(precision, [&](auto tag) -> int {
    using S = std::remove_pointer_t<decltype(tag)>;
    constexpr bool SH = !std::is_same_v<S, double>;
    const int blk = 256;
    if (A.mean) {
      const unsigned grid = (unsigned)((D.ncell + blk - 1) / blk);
      if (A.P > kMaxGpcP) return (int)cudaErrorInvalidValue;
      auto pair = [&](auto pm) {
        constexpr int PM = decltype(pm)::value;
        if constexpr (SH && PM <= kMomCellMaxP) {
          moments_pair_kernel<S, PM><<<grid, blk, 0, s>>>(P, A);
        } else if constexpr (SH) {
          const unsigned g2 = (unsigned)((D.ncell + 32 * kMomPairs - 1) / (32 * kMomPairs));  // two threads a cell
          moments_split_kernel<S, PM><<<g2, 64 * kMomPairs, 0, s>>>(P, A);
        }
      };
      auto go = [&](auto avg) {
        constexpr bool AV = decltype(avg)::value;
        if constexpr (SH && !AV) {
          switch (gpc_pair_pad(A.P)) {
            case 0: pair(std::integral_constant<int, 0>{}); break;
            case 4: pair(std::integral_constant<int, 4>{}); break;
            case 6: pair(std::integral_constant<int, 6>{}); break;
            case 8: pair(std::integral_constant<int, 8>{}); break;
            case 10: pair(std::integral_constant<int, 10>{}); break;
            case 12: pair(std::integral_constant<int, 12>{}); break;
            case 16: pair(std::integral_constant<int, 16>{}); break;
            case 20: pair(std::integral_constant<int, 20>{}); break;
            case 24: pair(std::integral_constant<int, 24>{}); break;
            default: pair(std::integral_constant<int, kMaxGpcP>{}); break;
          }
          static_assert(gpc_pair_pad(kMomCellMaxP) == kMomCellMaxP && gpc_pair_pad(kMomCellMaxP + 1) % 4 == 0,
                        "the split form needs term pairs in two halves");
        } else {
          if (A.P == 0) moments_kernel<S, SH, 0, AV><<<grid, blk, 0, s>>>(P, A);
          else if (A.P <= 3) moments_kernel<S, SH, 3, AV><<<grid, blk, 0, s>>>(P, A);
          else if (A.P <= 6) moments_kernel<S, SH, 6, AV><<<grid, blk, 0, s>>>(P, A);
          else if (A.P <= 10) moments_kernel<S, SH, 10, AV><<<grid, blk, 0, s>>>(P, A);
          else if (A.P <= 15) moments_kernel<S, SH, 15, AV><<<grid, blk, 0, s>>>(P, A);
          else if (A.P <= 21) moments_kernel<S, SH, 21, AV><<<grid, blk, 0, s>>>(P, A);
          else moments_kernel<S, SH, kMaxGpcP, AV><<<grid, blk, 0, s>>>(P, A);
        }
      };
      if (A.avg) go(std::true_type{});
      else go(std::false_type{});
      int rc = (int)cudaGetLastError();
      if (rc) return rc;
    }
    if (A.n_p > 0) {
      const long long warps = (long long)A.n_p * D.nz;
      profiles_kernel<S, SH><<<(unsigned)((warps * 32 + blk - 1) / blk), blk, 0, s>>>(P, A);
    }
    return (int)cudaGetLastError();
  });
}

int launch_export(const StepParams& P, int precision, int domain, int node, double* d_f,
                  float* d_u, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const DevDomain& D = P.dom[domain];
  return dispatch(precision, [&](auto tag) -> int {
    using S = std::remove_pointer_t<decltype(tag)>;
    constexpr bool SH = !std::is_same_v<S, double>;
    export_kernel<S, SH><<<(unsigned)((D.ncell + 255) / 256), 256, 0, s>>>(P, domain, node, d_f, d_u);
    return (int)cudaGetLastError();
  });
}

int launch_average_add(const StepParams& P, int precision, int domain, double* avg, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const DevDomain& D = P.dom[domain];
  return dispatch(precision, [&](auto tag) -> int {
    using S = std::remove_pointer_t<decltype(tag)>;
    constexpr bool SH = !std::is_same_v<S, double>;
    average_add_kernel<S, SH><<<grid_for(D.ncell * D.nodes, 256), 256, 0, s>>>(P, domain, avg);
    return (int)cudaGetLastError();
  });
}

int launch_finalize_moments(const double* s1, const double* s2, double wsum, double* mean, double* stdev,
                            long long n, void* stream) {
  finalize_moments_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(s1, s2, wsum, mean, stdev, n);
  return (int)cudaGetLastError();
}

int launch_scale(const double* in, double s, double* out, long long n, void* stream) {
  scale_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(in, s, out, n);
  return (int)cudaGetLastError();
}

int launch_qcriterion(const StepParams& P, int domain, const float* u, float* q, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  qcriterion_kernel<<<grid_for(P.dom[domain].ncell, 256), 256, 0, s>>>(P, domain, u, q);
  return (int)cudaGetLastError();
}

int launch_check(const StepParams& P, int precision, unsigned long long* d_count, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  return dispatch(precision, [&](auto tag) -> int {
    using S = std::remove_pointer_t<decltype(tag)>;
    constexpr bool SH = !std::is_same_v<S, double>;
    check_kernel<S, SH><<<152 * 8, 256, 0, s>>>(P, d_count);
    return (int)cudaGetLastError();
  });
}

}  // namespace sclbm
