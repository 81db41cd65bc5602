// adjoint.cu -- discrete adjoint of the lattice Boltzmann time step for
// inflow-parameter assimilation (arXiv:2508.18202 Sec. 1 and 2.4 motivate the
// assimilation; the paper itself does not differentiate the solver).
//
// Forward model of one time step n -> n + 1 (BGK, Sec. 2.2, Eq.
// deterministicLBE):
//   f*(x) = C(f^n(x))                       local collision
//   f^{n+1} = A f* + b(theta, n + 1)        streaming and link rules, linear in
//                                           f*, plus the moving-wall term
//                                           b_i = 6 w_i (c_i . u_in(z)) r(n+1)
//                                           on inflow links.
// With J = sum_p |u(x_p, T) - u*_p|^2 and lambda^n = dJ/df^n:
//   lambda^T   = dJ/df^T (probe cells only)
//   lambda*^n  = A^T lambda^{n+1}            (gather over the deliveries of
//                                            each post-collision population)
//   lambda^n   = (dC/df(f^n))^T lambda*^n
//   dJ/dtheta  = sum_n sum_inflow links lambda^{n+1}_i(x) db_i/dtheta.
// The forward states f^n of a segment are recomputed from checkpoints taken
// every L steps (about sqrt(T) checkpoints of about sqrt(T) steps each).
//
// All arrays are FP32 populations g = f - w in natural layout [19][pitch];
// the gradient and the loss accumulate in FP64.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_device.cuh"
#include "sclbm_internal.h"

namespace sclbm {
namespace {

// One FP32 time step of one node, two arrays, push form.
__global__ void __launch_bounds__(256) adj_forward_kernel(const __grid_constant__ StepParams P, AdjArgs A,
                                                          const float* src, float* dst, float r1) {
  const DevDomain& D = P.dom[A.domain];
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= D.ncell) return;
  const LinkWord lw = __ldg(D.link + c);
  if (lw & kLinkSolid) return;
  const int z = (int)(c / ((long long)D.nx * D.ny));
  const long long pc = D.pitch;
  float g[kQ];
#pragma unroll
  for (int i = 0; i < kQ; ++i) g[i] = src[(long long)i * pc + c];
  collide_p<float, true>(P, g);
  Node<float> N;
  N.g = dst;
  N.bout = nullptr;
  N.uinf = A.uin;
  N.uind = nullptr;
  const Wind<float> w1{1.f, 0.f, r1};  // steady inflow: the ramp alone
  if (!(lw & kLinkSlow)) {
    float ux, uy, uz;
    wall_velocity<float>(N, lw, z, w1, ux, uy, uz);
    fast_push<float>(dst + c, lw, (int)pc, D.nx, D.nx * D.ny, ux, uy, uz, r1, g);
    return;
  }
  const ListedRef L = listed_ref(D, A.lmap[c]);
  float ux = 0.f, uy = 0.f, uz = 0.f;
  if (L.word(kWordPushMove)) inflow_velocity<float>(N, z, w1, ux, uy, uz);
  listed_push<float>(L, dst, ux, uy, uz, r1, g);
}

// Listed cell c -> its index in the domain's listed-cell array (entries of
// other cells are never read).
__global__ void adj_listed_map_kernel(const __grid_constant__ StepParams P, int domain, int32_t* lmap) {
  const DevDomain& D = P.dom[domain];
  for (long long li = blockIdx.x * (long long)blockDim.x + threadIdx.x; li < D.nb;
       li += (long long)gridDim.x * blockDim.x)
    lmap[__ldg(D.bcell + li)] = (int32_t)li;
}

// Loss at the probes and the adjoint seed lambda^T = dJ/df^T
// (dJ/df_m = sum_a 2 (u_a - u*_a) (c_ma - u_a) / rho).
__global__ void adj_loss_kernel(const __grid_constant__ StepParams P, AdjArgs A, const float* f, float* lam) {
  const DevDomain& D = P.dom[A.domain];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= A.n_probes) return;
  const int* q = A.probes + 3 * p;
  const long long c = q[0] + (long long)D.nx * (q[1] + (long long)D.ny * q[2]);
  double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < kQ; ++i) {
    const double fi = (double)f[(long long)i * D.pitch + c] + c_lat.wd[i];
    rho += fi;
    j[0] += c_lat.cx[i] * fi;
    j[1] += c_lat.cy[i] * fi;
    j[2] += c_lat.cz[i] * fi;
  }
  const double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
  double e[3], loss = 0.0;
  for (int a = 0; a < 3; ++a) {
    e[a] = u[a] - A.target[3 * p + a];
    loss += e[a] * e[a];
    A.u_probe[3 * p + a] = u[a];
  }
  atomicAdd(A.accum, loss);
  for (int m = 0; m < kQ; ++m) {
    const double cm[3] = {(double)c_lat.cx[m], (double)c_lat.cy[m], (double)c_lat.cz[m]};
    double v = 0.0;
    for (int a = 0; a < 3; ++a) v += 2.0 * e[a] * (cm[a] - u[a]) / rho;
    lam[(long long)m * D.pitch + c] = (float)v;
  }
}

// One reverse step: lambda^n from lambda^{n+1} and the forward state f^n;
// accumulates the inflow-parameter gradient of level n + 1 (ramp r1).
__global__ void __launch_bounds__(256) adj_step_kernel(const __grid_constant__ StepParams P, AdjArgs A,
                                                       const float* f, const float* lam_next, float* lam,
                                                       float r1) {
  const DevDomain& D = P.dom[A.domain];
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double gr0 = 0.0, gr1 = 0.0;
  if (c < D.ncell) {
    const LinkWord lw = __ldg(D.link + c);
    if (!(lw & kLinkSolid)) {
      const int z = (int)(c / ((long long)D.nx * D.ny));
      const long long pc = D.pitch;
      float ls[kQ];
      // lambda*_k(x) = the sum of lambda^{n+1} over the slots the forward
      // step delivers f*_k(x) to (the transpose of the push rules), and the
      // moving-wall terms' share of dJ/dtheta: sum over the slots that receive
      // a term 6 w_i (c_i . u_in(z)) r(n + 1) of lambda^{n+1} there times the
      // term's derivative (summed per cell in FP32, over cells in FP64)
      float g0 = 0.0f, g1 = 0.0f;
      const float4 du0 = A.du[z], du1 = A.du[D.nz + z];
      if (!(lw & kLinkSlow)) {
        // each f*_k goes to the one slot the forward push writes (stream,
        // bounce-back, moving wall, specular lid)
        const int sy = D.nx, sz = D.nx * D.ny;
#pragma unroll
        for (int k = 0; k < kQ; ++k) {
          const int kind = link_kind(lw, OPP(k));
          const int stream = k * (int)pc + (CX(k) + CY(k) * sy + CZ(k) * sz);
          const int spec = REFL(k, 2) * (int)pc + (CX(k) + CY(k) * sy);
          ls[k] = lam_next[c + (kind == kStream ? stream : (kind == kSpecZ ? spec : OPP(k) * (int)pc))];
          if (kind == kMoving) {  // lands in the own slot i = opp(k) with the term of link i
            const int i = OPP(k);
            const float pre = 6.0f * W<float>(i) * r1 * ls[k];
            g0 += pre * (CX(i) * du0.x + CY(i) * du0.y + CZ(i) * du0.z);
            g1 += pre * (CX(i) * du1.x + CY(i) * du1.y + CZ(i) * du1.z);
          }
        }
      } else {
        // listed cell: the deliveries of its compiled record; an outlet copy
        // stored to a slot the cell's own primary delivery also wrote
        // replaces it (listed_push writes the copies last)
        const ListedRef L = listed_ref(D, A.lmap[c]);
        constexpr int kCopies = kOutletPops * kOutletCopies;
        int32_t ex[kCopies];
#pragma unroll
        for (int e = 0; e < kCopies; ++e) ex[e] = L.word(kWordExtra + e);
        const uint32_t mm = (uint32_t)L.word(kWordPushMove);
#pragma unroll
        for (int k = 0; k < kQ; ++k) {
          const int d = L.word(kWordDst + k);
          bool replaced = false;
#pragma unroll
          for (int e = 0; e < kCopies; ++e) replaced |= ex[e] == d;
          const float v = (d >= 0 && !replaced) ? lam_next[d] : 0.0f;
          ls[k] = v;
          if ((mm >> k) & 1u) {
            const int i = OPP(k);
            const float pre = 6.0f * W<float>(i) * r1 * v;
            g0 += pre * (CX(i) * du0.x + CY(i) * du0.y + CZ(i) * du0.z);
            g1 += pre * (CX(i) * du1.x + CY(i) * du1.y + CZ(i) * du1.z);
          }
        }
        constexpr int kPops[kOutletPops] = {2, 8, 10, 12, 14};
#pragma unroll
        for (int e = 0; e < kOutletPops; ++e)
#pragma unroll
          for (int m = 0; m < kOutletCopies; ++m) {
            const int d = ex[e * kOutletCopies + m];
            if (d >= 0) ls[kPops[e]] += lam_next[d];
          }
      }
      gr0 = (double)g0;
      gr1 = (double)g1;
      // forward state of this level
      float rho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        const float fi = f[(long long)i * pc + c] + W<float>(i);
        rho += fi;
        jx += CX(i) * fi;
        jy += CY(i) * fi;
        jz += CZ(i) * fi;
      }
      const float inv = recip(rho);
      const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
      const float usq = ux * ux + uy * uy + uz * uz;
      const float om = recip(P.tau0);
      // alpha = sum_i ls_i df^eq_i/drho, beta_a = sum_i ls_i df^eq_i/dj_a
      float al = 0.0f, bx = 0.0f, by = 0.0f, bz = 0.0f;
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        const float cu = CX(i) * ux + CY(i) * uy + CZ(i) * uz;
        const float wl = W<float>(i) * ls[i];
        al += wl * (1.0f - 4.5f * cu * cu + 1.5f * usq);
        const float t = 3.0f + 9.0f * cu;
        bx += wl * (t * CX(i) - 3.0f * ux);
        by += wl * (t * CY(i) - 3.0f * uy);
        bz += wl * (t * CZ(i) - 3.0f * uz);
      }
#pragma unroll
      for (int m = 0; m < kQ; ++m)
        lam[(long long)m * pc + c] = (1.0f - om) * ls[m] + om * (al + CX(m) * bx + CY(m) * by + CZ(m) * bz);
    }
  }
  // warps without a moving-wall contribution skip the FP64 reduction
  if (!__any_sync(0xffffffffu, gr0 != 0.0 || gr1 != 0.0)) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    gr0 += __shfl_xor_sync(0xffffffffu, gr0, o);
    gr1 += __shfl_xor_sync(0xffffffffu, gr1, o);
  }
  if ((threadIdx.x & 31) == 0 && (gr0 != 0.0 || gr1 != 0.0)) {
    atomicAdd(A.accum + 1, gr0);
    atomicAdd(A.accum + 2, gr1);
  }
}

__global__ void fill_zero_kernel(float* p, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    p[k] = 0.0f;
}

unsigned blocks_for(long long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

int launch_adj_forward(const StepParams& P, const AdjArgs& A, const float* src, float* dst, float r1,
                       void* stream) {
  const DevDomain& D = P.dom[A.domain];
  adj_forward_kernel<<<blocks_for(D.ncell), 256, 0, (cudaStream_t)stream>>>(P, A, src, dst, r1);
  return (int)cudaGetLastError();
}

int launch_adj_loss(const StepParams& P, const AdjArgs& A, const float* f, float* lam, void* stream) {
  adj_loss_kernel<<<(A.n_probes + 63) / 64, 64, 0, (cudaStream_t)stream>>>(P, A, f, lam);
  return (int)cudaGetLastError();
}

int launch_adj_step(const StepParams& P, const AdjArgs& A, const float* f, const float* lam_next, float* lam,
                    float r1, void* stream) {
  const DevDomain& D = P.dom[A.domain];
  adj_step_kernel<<<blocks_for(D.ncell), 256, 0, (cudaStream_t)stream>>>(P, A, f, lam_next, lam, r1);
  return (int)cudaGetLastError();
}

int launch_adj_listed_map(const StepParams& P, int domain, int32_t* lmap, void* stream) {
  const long long nb = P.dom[domain].nb;
  adj_listed_map_kernel<<<(unsigned)(nb > 0 ? (nb + 255) / 256 : 1), 256, 0, (cudaStream_t)stream>>>(P, domain, lmap);
  return (int)cudaGetLastError();
}

int launch_fill_zero(float* p, long long n, void* stream) {
  fill_zero_kernel<<<(unsigned)((n + 255) / 256 < 152 * 32 ? (n + 255) / 256 : 152 * 32), 256, 0,
                     (cudaStream_t)stream>>>(p, n);
  return (int)cudaGetLastError();
}

}  // namespace sclbm
