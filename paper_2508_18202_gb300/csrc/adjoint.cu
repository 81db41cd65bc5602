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

// lambda*_k(x): the sum of lambda^{n+1} over every slot that the forward
// step delivers f*_k(x) to (the transpose of the push rules).
__device__ float gather_deliveries(const DevDomain& D, const float* lam, int k, int x, int y, int z,
                                   long long c, LinkWord lw) {
  const long long pc = D.pitch;
  const int cx = c_lat.cx[k], cy = c_lat.cy[k], cz = c_lat.cz[k], ok = c_lat.opp[k];
  float s = 0.0f;
  if (link_kind(lw, ok) == kStream) {
    s = lam[(long long)k * pc + c + link_offset(D, k)];
  } else {
    const Cross q = classify(D, x + cx, y + cy, z + cz);
    const float own = lam[(long long)ok * pc + c];
    if (q.n == 0) {
      const long long t = cidx(D, q.p[0], q.p[1], q.p[2]);
      s = D.flags[t] == 0 ? lam[(long long)k * pc + t] : own;
    } else if (q.n == 1) {
      const int kind = D.bc[q.f[0]];
      if (kind == SC_BC_BOUNCE_BACK || kind == SC_BC_VELOCITY) {
        s = own;
      } else if (kind == SC_BC_FREE_SLIP) {
        const int a = q.f[0] >> 1;
        int t[3] = {x + cx, y + cy, z + cz};
        t[a] = a == 0 ? x : (a == 1 ? y : z);
        const Cross ct = classify(D, t[0], t[1], t[2]);
        const long long tp = cidx(D, ct.p[0], ct.p[1], ct.p[2]);
        s = D.flags[tp] == 0 ? lam[(long long)c_lat.refl[k][a] * pc + tp] : own;
      }
      // OUTFLOW: the population leaves the domain
    } else {
      const int k0 = D.bc[q.f[0]], k1 = D.bc[q.f[1]];
      if (k0 == SC_BC_BOUNCE_BACK || k1 == SC_BC_BOUNCE_BACK || k0 == SC_BC_VELOCITY ||
          k1 == SC_BC_VELOCITY || (k0 == SC_BC_FREE_SLIP && k1 == SC_BC_FREE_SLIP))
        s = own;
    }
  }
  if ((lw & kLinkOutlet) && cx == -1) {
    // (1) transverse neighbour on the outlet plane
    {
      const Cross q = classify(D, x, y + cy, z + cz);
      if (q.n == 0) {
        const long long t = cidx(D, q.p[0], q.p[1], q.p[2]);
        if (D.flags[t] == 0) s += lam[(long long)k * pc + t];
      }
    }
    // (2) own link k whose transverse source is solid
    {
      const Cross q = classify(D, x, y - cy, z - cz);
      if (q.n == 0 && D.flags[cidx(D, q.p[0], q.p[1], q.p[2])] != 0) s += lam[(long long)k * pc + c];
    }
    // (3) outflow + free-slip edge
    for (int a = 1; a < 3; ++a) {
      const int ca = a == 1 ? cy : cz;
      if (ca == 0) continue;
      const int face = 2 * a + (ca > 0 ? 1 : 0);
      const int pos = (a == 1 ? y : z) + ca;
      const int lim = a == 1 ? D.ny : D.nz;
      if (D.bc[face] == SC_BC_FREE_SLIP && (pos < 0 || pos >= lim))
        s += lam[(long long)c_lat.refl[k][a] * pc + c];
    }
  }
  return s;
}

// True when the pull rule of link i at the cell carries the moving-wall term.
__device__ __forceinline__ bool velocity_link(const DevDomain& D, int i, int x, int y, int z) {
  const Cross q = classify(D, x - c_lat.cx[i], y - c_lat.cy[i], z - c_lat.cz[i]);
  if (q.n == 1) return D.bc[q.f[0]] == SC_BC_VELOCITY;
  if (q.n == 2) {
    const int k0 = D.bc[q.f[0]], k1 = D.bc[q.f[1]];
    return k0 != SC_BC_BOUNCE_BACK && k1 != SC_BC_BOUNCE_BACK &&
           (k0 == SC_BC_VELOCITY || k1 == SC_BC_VELOCITY);
  }
  return false;
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
      const int x = (int)(c % D.nx), y = (int)((c / D.nx) % D.ny), z = (int)(c / ((long long)D.nx * D.ny));
      const long long pc = D.pitch;
      float ls[kQ];
      if (!(lw & kLinkSlow)) {
        // each f*_k goes to the one slot the forward push writes (stream,
        // bounce-back, moving wall, specular lid): lambda*_k is lambda^{n+1}
        // there
        const int sy = D.nx, sz = D.nx * D.ny;
#pragma unroll
        for (int k = 0; k < kQ; ++k) {
          const int kind = link_kind(lw, OPP(k));
          const int stream = k * (int)pc + (CX(k) + CY(k) * sy + CZ(k) * sz);
          const int spec = REFL(k, 2) * (int)pc + (CX(k) + CY(k) * sy);
          ls[k] = lam_next[c + (kind == kStream ? stream : (kind == kSpecZ ? spec : OPP(k) * (int)pc))];
        }
      } else {
        float lg[kQ];
#pragma unroll 1
        for (int k = 0; k < kQ; ++k) lg[k] = gather_deliveries(D, lam_next, k, x, y, z, c, lw);
#pragma unroll
        for (int k = 0; k < kQ; ++k) ls[k] = lg[k];
      }
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
      // inflow links of this cell at level n + 1
      if (lw & kLinkVel) {
        const float4 du0 = A.du[z], du1 = A.du[D.nz + z];
#pragma unroll 1
        for (int i = 1; i < kQ; ++i) {
          if (link_kind(lw, i) == kStream) continue;
          if (!(lw & kLinkSlow) ? link_kind(lw, i) != kMoving : !velocity_link(D, i, x, y, z)) continue;
          const double li = (double)lam_next[(long long)i * pc + c];
          const double pre = 6.0 * c_lat.wd[i] * (double)r1;
          const double d0 = c_lat.cx[i] * (double)du0.x + c_lat.cy[i] * (double)du0.y + c_lat.cz[i] * (double)du0.z;
          const double d1 = c_lat.cx[i] * (double)du1.x + c_lat.cy[i] * (double)du1.y + c_lat.cz[i] * (double)du1.z;
          gr0 += li * pre * d0;
          gr1 += li * pre * d1;
        }
      }
    }
  }
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
