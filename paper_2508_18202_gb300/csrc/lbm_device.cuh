// lbm_device.cuh -- device-side building blocks shared by the forward and the
// adjoint kernels of libsclbm: D3Q19 tables, population storage types, the
// BGK(+Smagorinsky) collision, and the per-link boundary rules (in pull form
// for the odd AA level and in push form for the deliveries).  Included by
// the CUDA translation units only.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "sclbm_internal.h"

namespace sclbm {
namespace {

// ------------------------------------------------------------ lattice
__host__ __device__ constexpr int CX(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int CY(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int CZ(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int OPP(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr int C2(int i) { return CX(i) * CX(i) + CY(i) * CY(i) + CZ(i) * CZ(i); }
template <class T>
__host__ __device__ constexpr T W(int i) {
  return C2(i) == 0 ? T(1.0 / 3.0) : (C2(i) == 1 ? T(1.0 / 18.0) : T(1.0 / 36.0));
}
__host__ __device__ constexpr int DIR(int x, int y, int z) {
  for (int i = 0; i < kQ; ++i)
    if (CX(i) == x && CY(i) == y && CZ(i) == z) return i;
  return 0;
}
// direction i with its component along axis a negated (specular reflection)
__host__ __device__ constexpr int REFL(int i, int a) {
  return DIR(a == 0 ? -CX(i) : CX(i), a == 1 ? -CY(i) : CY(i), a == 2 ? -CZ(i) : CZ(i));
}
// slot in the outflow plane of the five directions with c_x = -1
__host__ __device__ constexpr int KOUT(int i) {
  return i == 2 ? 0 : i == 8 ? 1 : i == 10 ? 2 : i == 12 ? 3 : i == 14 ? 4 : -1;
}

// The same tables for run-time directions (compact boundary code).
struct LatticeTables {
  int cx[kQ], cy[kQ], cz[kQ], opp[kQ], kout[kQ], refl[kQ][3];
  float wf[kQ];
  double wd[kQ];
};
__constant__ LatticeTables c_lat = {
    {CX(0), CX(1), CX(2), CX(3), CX(4), CX(5), CX(6), CX(7), CX(8), CX(9), CX(10), CX(11), CX(12),
     CX(13), CX(14), CX(15), CX(16), CX(17), CX(18)},
    {CY(0), CY(1), CY(2), CY(3), CY(4), CY(5), CY(6), CY(7), CY(8), CY(9), CY(10), CY(11), CY(12),
     CY(13), CY(14), CY(15), CY(16), CY(17), CY(18)},
    {CZ(0), CZ(1), CZ(2), CZ(3), CZ(4), CZ(5), CZ(6), CZ(7), CZ(8), CZ(9), CZ(10), CZ(11), CZ(12),
     CZ(13), CZ(14), CZ(15), CZ(16), CZ(17), CZ(18)},
    {OPP(0), OPP(1), OPP(2), OPP(3), OPP(4), OPP(5), OPP(6), OPP(7), OPP(8), OPP(9), OPP(10),
     OPP(11), OPP(12), OPP(13), OPP(14), OPP(15), OPP(16), OPP(17), OPP(18)},
    {KOUT(0), KOUT(1), KOUT(2), KOUT(3), KOUT(4), KOUT(5), KOUT(6), KOUT(7), KOUT(8), KOUT(9),
     KOUT(10), KOUT(11), KOUT(12), KOUT(13), KOUT(14), KOUT(15), KOUT(16), KOUT(17), KOUT(18)},
    {{REFL(0, 0), REFL(0, 1), REFL(0, 2)},    {REFL(1, 0), REFL(1, 1), REFL(1, 2)},
     {REFL(2, 0), REFL(2, 1), REFL(2, 2)},    {REFL(3, 0), REFL(3, 1), REFL(3, 2)},
     {REFL(4, 0), REFL(4, 1), REFL(4, 2)},    {REFL(5, 0), REFL(5, 1), REFL(5, 2)},
     {REFL(6, 0), REFL(6, 1), REFL(6, 2)},    {REFL(7, 0), REFL(7, 1), REFL(7, 2)},
     {REFL(8, 0), REFL(8, 1), REFL(8, 2)},    {REFL(9, 0), REFL(9, 1), REFL(9, 2)},
     {REFL(10, 0), REFL(10, 1), REFL(10, 2)}, {REFL(11, 0), REFL(11, 1), REFL(11, 2)},
     {REFL(12, 0), REFL(12, 1), REFL(12, 2)}, {REFL(13, 0), REFL(13, 1), REFL(13, 2)},
     {REFL(14, 0), REFL(14, 1), REFL(14, 2)}, {REFL(15, 0), REFL(15, 1), REFL(15, 2)},
     {REFL(16, 0), REFL(16, 1), REFL(16, 2)}, {REFL(17, 0), REFL(17, 1), REFL(17, 2)},
     {REFL(18, 0), REFL(18, 1), REFL(18, 2)}},
    {W<float>(0), W<float>(1), W<float>(2), W<float>(3), W<float>(4), W<float>(5), W<float>(6),
     W<float>(7), W<float>(8), W<float>(9), W<float>(10), W<float>(11), W<float>(12), W<float>(13),
     W<float>(14), W<float>(15), W<float>(16), W<float>(17), W<float>(18)},
    {W<double>(0), W<double>(1), W<double>(2), W<double>(3), W<double>(4), W<double>(5),
     W<double>(6), W<double>(7), W<double>(8), W<double>(9), W<double>(10), W<double>(11),
     W<double>(12), W<double>(13), W<double>(14), W<double>(15), W<double>(16), W<double>(17),
     W<double>(18)},
};

// ------------------------------------------------------------ storage
template <class S>
struct Store;
template <>
struct Store<float> {
  using C = float;
  static __device__ __forceinline__ float ld(const float* p) { return *p; }
  static __device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }
  static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
};
template <>
struct Store<__nv_bfloat16> {
  using C = float;
  static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ float ldcg(const __nv_bfloat16* p) {
    return __bfloat162float(__ldcg(p));
  }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};
template <>
struct Store<__half> {
  using C = float;
  static __device__ __forceinline__ float ld(const __half* p) { return __half2float(*p); }
  static __device__ __forceinline__ float ldcg(const __half* p) { return __half2float(__ldcg(p)); }
  static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
};
template <>
struct Store<double> {
  using C = double;
  static __device__ __forceinline__ double ld(const double* p) { return *p; }
  static __device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
  static __device__ __forceinline__ void st(double* p, double v) { *p = v; }
};

template <class S, bool CG>
__device__ __forceinline__ typename Store<S>::C LD(const S* p) {
  if constexpr (CG) return Store<S>::ldcg(p);
  else return Store<S>::ld(p);
}

// Loads of the geometry (link words, class bytes) that every node of a launch
// reads again: an L2 evict-last policy keeps them resident while the
// populations stream through (measured: +1.5% on both AA levels of the
// 13-node LES ensemble, where the 16.8 MB of link words otherwise left L2
// between nodes).
__device__ __forceinline__ uint64_t keep_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ unsigned long long ld_keep(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(keep_policy()));
  return v;
}
__device__ __forceinline__ uint8_t ld_keep(const uint8_t* p) {
  unsigned short v;
  asm volatile("ld.global.nc.L2::cache_hint.u8 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(keep_policy()));
  return (uint8_t)v;
}
__device__ __forceinline__ uint16_t ld_keep(const uint16_t* p) {
  unsigned short v;
  asm volatile("ld.global.nc.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(keep_policy()));
  return (uint16_t)v;
}

// ------------------------------------------------------------ collision
// Correctly rounded reciprocal (the same value as 1 / x in IEEE arithmetic).
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }

// BGK with the Smagorinsky effective relaxation time (Sec. 2.2).  SHIFT:
// populations are g = f - w.  The non-equilibrium stress uses the exact
// second moment of the D3Q19 second-order equilibrium, rho/3 I + rho u u.
template <class T, bool SHIFT>
__device__ __forceinline__ void collide(T g[kQ], T tau0, T smag18c2, bool smag_on) {
  T m0 = T(0), jx = T(0), jy = T(0), jz = T(0);
  T pxx = T(0), pyy = T(0), pzz = T(0), pxy = T(0), pxz = T(0), pyz = T(0);
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    m0 += g[i];
    if (CX(i)) jx += CX(i) > 0 ? g[i] : -g[i];
    if (CY(i)) jy += CY(i) > 0 ? g[i] : -g[i];
    if (CZ(i)) jz += CZ(i) > 0 ? g[i] : -g[i];
    if (CX(i)) pxx += g[i];
    if (CY(i)) pyy += g[i];
    if (CZ(i)) pzz += g[i];
    if (CX(i) * CY(i)) pxy += CX(i) * CY(i) > 0 ? g[i] : -g[i];
    if (CX(i) * CZ(i)) pxz += CX(i) * CZ(i) > 0 ? g[i] : -g[i];
    if (CY(i) * CZ(i)) pyz += CY(i) * CZ(i) > 0 ? g[i] : -g[i];
  }
  const T rho = SHIFT ? T(1) + m0 : m0;
  const T inv = recip(rho);
  const T ux = jx * inv, uy = jy * inv, uz = jz * inv;
  const T usq = ux * ux + uy * uy + uz * uz;
  T tau = tau0;
  if (smag_on) {
    // Pi^neq = sum c c g - (m0/3 I + rho u u); m0 = rho - 1 (shifted) or rho
    const T third = m0 * T(1.0 / 3.0);
    const T nxx = pxx - third - rho * ux * ux;
    const T nyy = pyy - third - rho * uy * uy;
    const T nzz = pzz - third - rho * uz * uz;
    const T nxy = pxy - rho * ux * uy;
    const T nxz = pxz - rho * ux * uz;
    const T nyz = pyz - rho * uy * uz;
    const T pipi = nxx * nxx + nyy * nyy + nzz * nzz + T(2) * (nxy * nxy + nxz * nxz + nyz * nyz);
    const T pin = sqrt(T(2) * pipi + T(1e-30));
    tau = T(0.5) * (tau0 + sqrt(tau0 * tau0 + smag18c2 * pin * inv));
  }
  const T omega = recip(tau);
  const T base = m0;  // shifted: w (rho - 1) part; plain: w rho part
  // Opposite pairs (i, i + 1), i odd, share c_i . u up to the sign: the
  // bracket of the equilibrium splits into an even part
  // base + rho (4.5 cu^2 - 1.5 u^2) and an odd part 3 rho cu; the weight
  // multiplies last (a rounded 3 w would bias the momentum of every
  // collision).
  const T r15 = T(1.5) * usq;
  g[0] = g[0] - omega * (g[0] - W<T>(0) * (base - rho * r15));
#pragma unroll
  for (int i = 1; i < kQ; i += 2) {
    const T cu = T(CX(i)) * ux + T(CY(i)) * uy + T(CZ(i)) * uz;
    const T even = base + rho * (T(4.5) * cu * cu - r15);
    const T odd = T(3) * rho * cu;
    g[i] = g[i] - omega * (g[i] - W<T>(i) * (even + odd));
    g[i + 1] = g[i + 1] - omega * (g[i + 1] - W<T>(i) * (even - odd));
  }
}

// ------------------------------------------------------------ regularized collision
// Component a of c_i, and the Hermite polynomials of c_i (c_s^2 = 1/3):
//   H2_ab = c_a c_b - d_ab / 3,  H3_abg = c_a c_b c_g - (c_a d_bg + c_b d_ag + c_g d_ab) / 3.
__host__ __device__ constexpr int CA(int i, int a) { return a == 0 ? CX(i) : (a == 1 ? CY(i) : CZ(i)); }
__host__ __device__ constexpr double H3(int i, int a, int b, int g) {
  return (double)(CA(i, a) * CA(i, b) * CA(i, g)) -
         ((b == g ? CA(i, a) : 0) + (a == g ? CA(i, b) : 0) + (a == b ? CA(i, g) : 0)) / 3.0;
}
// The third-order combinations D3Q19 carries, k = 0..2 sums and 3..5
// differences of (xxy, yzz), (xzz, xyy), (yyz, xxz), divided by their D3Q19
// norms sum_i w_i h_k(c_i)^2 = 2/27 (sums) and 6/27 (differences).
__host__ __device__ constexpr double H3K(int i, int k) {
  return k == 0 ? (H3(i, 0, 0, 1) + H3(i, 1, 2, 2)) * 13.5
       : k == 1 ? (H3(i, 0, 2, 2) + H3(i, 0, 1, 1)) * 13.5
       : k == 2 ? (H3(i, 1, 1, 2) + H3(i, 0, 0, 2)) * 13.5
       : k == 3 ? (H3(i, 0, 0, 1) - H3(i, 1, 2, 2)) * 4.5
       : k == 4 ? (H3(i, 0, 2, 2) - H3(i, 0, 1, 1)) * 4.5
                : (H3(i, 1, 1, 2) - H3(i, 0, 0, 2)) * 4.5;
}

// Recursive regularized collision with the third-order equilibrium (Sec. 2.2,
// Eq. deterministicLBE, Eq. hermiteCoeff):
//   f* = f^eq + (1 - 1/tau_eff) f^(1),
//   f^eq_i  = w_i [rho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u^2) + sum_k h_k(c_i) E_k / N_k],
//   f^(1)_i = w_i [4.5 H2(c_i) : a2 + sum_k h_k(c_i) A_k / N_k],
// with a2 = Pi^neq (the second-order Hermite coefficient of f - f^eq), E_k the
// combinations of rho u_a u_b u_g and A_k those of the recursion
// a3_abg = u_a a2_bg + u_b a2_ag + u_g a2_ab.  tau_eff as in collide.  SHIFT as
// in collide (the rho part then carries rho - 1).
template <class T, bool SHIFT>
__device__ __forceinline__ void collide_rr(T g[kQ], T tau0, T smag18c2, bool smag_on) {
  T m0 = T(0), jx = T(0), jy = T(0), jz = T(0);
  T pxx = T(0), pyy = T(0), pzz = T(0), pxy = T(0), pxz = T(0), pyz = T(0);
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    m0 += g[i];
    if (CX(i)) jx += CX(i) > 0 ? g[i] : -g[i];
    if (CY(i)) jy += CY(i) > 0 ? g[i] : -g[i];
    if (CZ(i)) jz += CZ(i) > 0 ? g[i] : -g[i];
    if (CX(i)) pxx += g[i];
    if (CY(i)) pyy += g[i];
    if (CZ(i)) pzz += g[i];
    if (CX(i) * CY(i)) pxy += CX(i) * CY(i) > 0 ? g[i] : -g[i];
    if (CX(i) * CZ(i)) pxz += CX(i) * CZ(i) > 0 ? g[i] : -g[i];
    if (CY(i) * CZ(i)) pyz += CY(i) * CZ(i) > 0 ? g[i] : -g[i];
  }
  const T rho = SHIFT ? T(1) + m0 : m0;
  const T inv = recip(rho);
  const T ux = jx * inv, uy = jy * inv, uz = jz * inv;
  const T usq = ux * ux + uy * uy + uz * uz;
  const T third = m0 * T(1.0 / 3.0);
  const T nxx = pxx - third - rho * ux * ux;
  const T nyy = pyy - third - rho * uy * uy;
  const T nzz = pzz - third - rho * uz * uz;
  const T nxy = pxy - rho * ux * uy;
  const T nxz = pxz - rho * ux * uz;
  const T nyz = pyz - rho * uy * uz;
  T tau = tau0;
  if (smag_on) {
    const T pipi = nxx * nxx + nyy * nyy + nzz * nzz + T(2) * (nxy * nxy + nxz * nxz + nyz * nyz);
    const T pin = sqrt(T(2) * pipi + T(1e-30));
    tau = T(0.5) * (tau0 + sqrt(tau0 * tau0 + smag18c2 * pin * inv));
  }
  const T keep = T(1) - recip(tau);
  // third-order content after collision: E + keep * A per component
  const T rx = rho * ux, ry = rho * uy, rz = rho * uz;
  const T t_xxy = rx * ux * uy + keep * (T(2) * ux * nxy + uy * nxx);
  const T t_yzz = ry * uz * uz + keep * (T(2) * uz * nyz + uy * nzz);
  const T t_xzz = rx * uz * uz + keep * (T(2) * uz * nxz + ux * nzz);
  const T t_xyy = rx * uy * uy + keep * (T(2) * uy * nxy + ux * nyy);
  const T t_yyz = ry * uy * uz + keep * (T(2) * uy * nyz + uz * nyy);
  const T t_xxz = rx * ux * uz + keep * (T(2) * ux * nxz + uz * nxx);
  const T k3[6] = {t_xxy + t_yzz, t_xzz + t_xyy, t_yyz + t_xxz, t_xxy - t_yzz, t_xzz - t_xyy, t_yyz - t_xxz};
  // second-order non-equilibrium, scaled by keep and 4.5 = 1 / (2 c_s^4)
  const T kxx = T(4.5) * keep * nxx, kyy = T(4.5) * keep * nyy, kzz = T(4.5) * keep * nzz;
  const T kxy = T(9) * keep * nxy, kxz = T(9) * keep * nxz, kyz = T(9) * keep * nyz;
  const T base = m0;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const T cu = T(CX(i)) * ux + T(CY(i)) * uy + T(CZ(i)) * uz;
    T v = base + rho * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq);
    v += T(CX(i) * CX(i) - 1.0 / 3.0) * kxx + T(CY(i) * CY(i) - 1.0 / 3.0) * kyy +
         T(CZ(i) * CZ(i) - 1.0 / 3.0) * kzz;
    if (CX(i) * CY(i)) v += T(CX(i) * CY(i)) * kxy;
    if (CX(i) * CZ(i)) v += T(CX(i) * CZ(i)) * kxz;
    if (CY(i) * CZ(i)) v += T(CY(i) * CZ(i)) * kyz;
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (H3K(i, k) != 0.0) v += T(H3K(i, k)) * k3[k];
    g[i] = W<T>(i) * v;
  }
}

// ------------------------------------------------------------ two cells at once
// The BGK(+Smagorinsky) collision of collide<float, true> for two cells, one
// in each lane of Blackwell's packed FP32x2 operations (__fadd2_rn,
// __fmul2_rn, __ffma2_rn; each lane rounds as the scalar operation does):
// the even level of the 16-bit storage modes, at half the arithmetic
// instructions per cell.  The
// moments come from the sums s = g_i + g_opp(i) and differences d = g_i -
// g_opp(i) of the nine opposite pairs, and the equilibrium's even part
// base + rho (4.5 (c.u)^2 - 1.5 u^2) from (4.5 rho) (c.u)^2 + (base - rho 1.5
// u^2): the same quantities as collide(), summed and rounded in another
// order.  Reciprocals and square roots are taken lane by lane, correctly
// rounded.
__device__ __forceinline__ float2 p2dup(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 p2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p2sub(float2 a, float2 b) { return __ffma2_rn(b, p2dup(-1.0f), a); }
__device__ __forceinline__ float2 p2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ void collide_pair(float2 g[kQ], float tau0, float smag18c2, bool smag_on) {
  // pairs (2p + 1, 2p + 2): c = (1,0,0) (0,1,0) (0,0,1) (1,1,0) (1,-1,0)
  // (1,0,1) (1,0,-1) (0,1,1) (0,1,-1) and their opposites
  float2 s = p2add(g[1], g[2]), d = p2sub(g[1], g[2]);
  float2 m0 = p2add(g[0], s), jx = d, pxx = s;
  s = p2add(g[3], g[4]), d = p2sub(g[3], g[4]);
  m0 = p2add(m0, s);
  float2 jy = d, pyy = s;
  s = p2add(g[5], g[6]), d = p2sub(g[5], g[6]);
  m0 = p2add(m0, s);
  float2 jz = d, pzz = s;
  s = p2add(g[7], g[8]), d = p2sub(g[7], g[8]);
  m0 = p2add(m0, s), jx = p2add(jx, d), jy = p2add(jy, d), pxx = p2add(pxx, s), pyy = p2add(pyy, s);
  float2 pxy = s;
  s = p2add(g[9], g[10]), d = p2sub(g[9], g[10]);
  m0 = p2add(m0, s), jx = p2add(jx, d), jy = p2sub(jy, d), pxx = p2add(pxx, s), pyy = p2add(pyy, s);
  pxy = p2sub(pxy, s);
  s = p2add(g[11], g[12]), d = p2sub(g[11], g[12]);
  m0 = p2add(m0, s), jx = p2add(jx, d), jz = p2add(jz, d), pxx = p2add(pxx, s), pzz = p2add(pzz, s);
  float2 pxz = s;
  s = p2add(g[13], g[14]), d = p2sub(g[13], g[14]);
  m0 = p2add(m0, s), jx = p2add(jx, d), jz = p2sub(jz, d), pxx = p2add(pxx, s), pzz = p2add(pzz, s);
  pxz = p2sub(pxz, s);
  s = p2add(g[15], g[16]), d = p2sub(g[15], g[16]);
  m0 = p2add(m0, s), jy = p2add(jy, d), jz = p2add(jz, d), pyy = p2add(pyy, s), pzz = p2add(pzz, s);
  float2 pyz = s;
  s = p2add(g[17], g[18]), d = p2sub(g[17], g[18]);
  m0 = p2add(m0, s), jy = p2add(jy, d), jz = p2sub(jz, d), pyy = p2add(pyy, s), pzz = p2add(pzz, s);
  pyz = p2sub(pyz, s);

  const float2 rho = p2add(p2dup(1.0f), m0);
  const float2 inv = make_float2(recip(rho.x), recip(rho.y));
  const float2 ux = p2mul(jx, inv), uy = p2mul(jy, inv), uz = p2mul(jz, inv);
  const float2 usq = p2fma(uz, uz, p2fma(uy, uy, p2mul(ux, ux)));
  float2 omega = p2dup(recip(tau0));
  if (smag_on) {
    // Pi^neq = sum c c g - (m0/3 I + rho u u), as in collide()
    const float2 third = p2mul(m0, p2dup(1.0f / 3.0f));
    const float2 rx = p2mul(rho, ux), ry = p2mul(rho, uy), rz = p2mul(rho, uz);
    const float2 nxx = p2sub(pxx, p2fma(rx, ux, third));
    const float2 nyy = p2sub(pyy, p2fma(ry, uy, third));
    const float2 nzz = p2sub(pzz, p2fma(rz, uz, third));
    const float2 nxy = p2sub(pxy, p2mul(rx, uy));
    const float2 nxz = p2sub(pxz, p2mul(rx, uz));
    const float2 nyz = p2sub(pyz, p2mul(ry, uz));
    const float2 dia = p2fma(nzz, nzz, p2fma(nyy, nyy, p2mul(nxx, nxx)));
    const float2 off = p2fma(nyz, nyz, p2fma(nxz, nxz, p2mul(nxy, nxy)));
    // 2 Pi:Pi + 1e-30 = 2 (diagonal) + 4 (off-diagonal) + 1e-30
    const float2 a = p2fma(p2dup(4.0f), off, p2fma(p2dup(2.0f), dia, p2dup(1e-30f)));
    const float2 pin = make_float2(sqrtf(a.x), sqrtf(a.y));
    const float2 b = p2fma(p2dup(smag18c2), p2mul(pin, inv), p2dup(tau0 * tau0));
    const float2 tau = p2mul(p2dup(0.5f), p2add(p2dup(tau0), make_float2(sqrtf(b.x), sqrtf(b.y))));
    omega = make_float2(recip(tau.x), recip(tau.y));
  }
  const float2 nom = p2mul(omega, p2dup(-1.0f));
  const float2 base = p2sub(m0, p2mul(rho, p2mul(p2dup(1.5f), usq)));  // m0 - 1.5 rho u^2
  const float2 r45 = p2mul(p2dup(4.5f), rho), r3 = p2mul(p2dup(3.0f), rho);
  // g_i - omega (g_i - w_i e_i), the weight multiplying last as in collide()
  g[0] = p2fma(nom, p2fma(p2dup(-W<float>(0)), base, g[0]), g[0]);
  auto relax = [&](int i, float2 cu) {
    const float2 even = p2fma(r45, p2mul(cu, cu), base);
    const float2 odd = p2mul(r3, cu);
    const float2 nw = p2dup(-W<float>(i));
    g[i] = p2fma(nom, p2fma(nw, p2add(even, odd), g[i]), g[i]);
    g[i + 1] = p2fma(nom, p2fma(nw, p2sub(even, odd), g[i + 1]), g[i + 1]);
  };
  relax(1, ux);
  relax(3, uy);
  relax(5, uz);
  relax(7, p2add(ux, uy));
  relax(9, p2sub(ux, uy));
  relax(11, p2add(ux, uz));
  relax(13, p2sub(ux, uz));
  relax(15, p2add(uy, uz));
  relax(17, p2sub(uy, uz));
}

// Two x-adjacent 16-bit populations as one 32-bit word (the lower address,
// the even cell, in the low half) and the FP32 pair they stand for.
template <class S>
struct Pair16;
template <>
struct Pair16<__nv_bfloat16> {
  static __device__ __forceinline__ float2 unpack(uint32_t w) {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
  }
  static __device__ __forceinline__ uint32_t pack(float2 v) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);  // each lane rounded to nearest even
    uint32_t w;
    memcpy(&w, &h, sizeof w);
    return w;
  }
};
template <>
struct Pair16<__half> {
  static __device__ __forceinline__ float2 unpack(uint32_t w) {
    __half2 h;
    memcpy(&h, &w, sizeof w);
    return __half22float2(h);
  }
  static __device__ __forceinline__ uint32_t pack(float2 v) {
    const __half2 h = __floats2half2_rn(v.x, v.y);
    uint32_t w;
    memcpy(&w, &h, sizeof w);
    return w;
  }
};

// The collision of the compiled unit: BGK(+Smagorinsky), or the recursive
// regularized form in the unit built with SCLBM_RR_UNIT.
template <class T, bool SHIFT>
__device__ __forceinline__ void collide_p(const StepParams& P, T g[kQ]) {
#ifdef SCLBM_RR_UNIT
  if constexpr (sizeof(T) == 8)
    collide_rr<T, SHIFT>(g, T(P.tau0_d), T(P.smag18c2_d), P.csmag_on);
  else
    collide_rr<T, SHIFT>(g, T(P.tau0), T(P.smag18c2), P.csmag_on);
#else
  if constexpr (sizeof(T) == 8)
    collide<T, SHIFT>(g, T(P.tau0_d), T(P.smag18c2_d), P.csmag_on);
  else
    collide<T, SHIFT>(g, T(P.tau0), T(P.smag18c2), P.csmag_on);
#endif
}

// ------------------------------------------------------------ boundary helpers
__device__ __forceinline__ long long cidx(const DevDomain& D, int x, int y, int z) {
  return (long long)x + (long long)D.nx * ((long long)y + (long long)D.ny * z);
}

// Per-node pointers.
template <class S>
struct Node {
  S* g;                // [19][pitch]
  float* bout;         // [nz*ny][5]
  const float4* uinf;  // [nz]
  const double* uind;  // [nz][3]
};


// ------------------------------------------------------------ fast link rules
// Links of kind kStream, kBounce, kMoving and kSpecZ resolve to an address
// (and, for kMoving, an added moving-wall term), so cells whose links are all
// of these kinds update without branches.  Offsets are 32-bit element
// offsets from the cell's own slot 0 (a node holds fewer than 2^31
// populations).

// 6 w_i (c_i . u) r, direction i known at compile time; u is the wall
// velocity turned to the arrival level's direction, r its scale.
template <class T>
__device__ __forceinline__ T wall_term(int i, T ux, T uy, T uz, T r) {
  return T(6) * W<T>(i) * (T(CX(i)) * ux + T(CY(i)) * uy + T(CZ(i)) * uz) * r;
}

// Pull of the odd AA level (swapped layout in place).
template <class S, bool CG>
__device__ __forceinline__ void fast_pull(const S* base, LinkWord lw, int pc, int sy, int sz,
                                          typename Store<S>::C ux, typename Store<S>::C uy,
                                          typename Store<S>::C uz, typename Store<S>::C r,
                                          typename Store<S>::C g[kQ]) {
  using T = typename Store<S>::C;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const int kind = link_kind(lw, i);
    const int stream = OPP(i) * pc - (CX(i) + CY(i) * sy + CZ(i) * sz);
    const int spec = OPP(REFL(i, 2)) * pc - (CX(i) + CY(i) * sy);
    const int off = kind == kStream ? stream : (kind == kSpecZ ? spec : i * pc);
    T v = LD<S, CG>(base + off);
    if (kind == kMoving) v += wall_term<T>(i, ux, uy, uz, r);
    g[i] = v;
  }
}

// Delivery of the post-collision populations (odd AA level in place, or the
// two-array push form with base in the destination array).
template <class S>
__device__ __forceinline__ void fast_push(S* base, LinkWord lw, int pc, int sy, int sz,
                                          typename Store<S>::C ux, typename Store<S>::C uy,
                                          typename Store<S>::C uz, typename Store<S>::C r1,
                                          const typename Store<S>::C g[kQ]) {
  using T = typename Store<S>::C;
#pragma unroll
  for (int j = 0; j < kQ; ++j) {
    const int kind = link_kind(lw, OPP(j));
    const int stream = j * pc + (CX(j) + CY(j) * sy + CZ(j) * sz);
    const int spec = REFL(j, 2) * pc + (CX(j) + CY(j) * sy);
    const int off = kind == kStream ? stream : (kind == kSpecZ ? spec : OPP(j) * pc);
    T v = g[j];
    if (kind == kMoving) v += wall_term<T>(OPP(j), ux, uy, uz, r1);
    Store<S>::st(base + off, v);
  }
}

// ------------------------------------------------------------ listed cells
// Word w of the compiled rules of listed cell li (transposed records).
struct ListedRef {
  const int32_t* p;
  long long stride;
  __device__ __forceinline__ int word(int w) const { return __ldg(p + w * stride); }
};
__device__ __forceinline__ ListedRef listed_ref(const DevDomain& D, long long li) {
  ListedRef L;
  L.p = D.ltab + li;
  L.stride = D.lstride;
  return L;
}

// Pull of the odd AA level for a listed cell from its compiled rules: g0 is
// the node's population base, bo its outflow plane (float).
template <class S, bool CG>
__device__ __forceinline__ void listed_pull(const ListedRef& L, const S* g0, const float* bo,
                                            typename Store<S>::C ux, typename Store<S>::C uy,
                                            typename Store<S>::C uz, typename Store<S>::C r,
                                            typename Store<S>::C g[kQ]) {
  using T = typename Store<S>::C;
  const uint32_t bm = (uint32_t)L.word(kWordBoutMask), pm = (uint32_t)L.word(kWordPullMove);
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const int s = L.word(kWordSrc + i);
    T v = ((bm >> i) & 1u) ? T(__ldcg(bo + s)) : LD<S, CG>(g0 + s);
    if ((pm >> i) & 1u) v += wall_term<T>(i, ux, uy, uz, r);
    g[i] = v;
  }
}

// Deliveries of a listed cell's post-collision populations into the node's
// array g0 (AA in place, or the destination array of a two-array step).
template <class S>
__device__ __forceinline__ void listed_push(const ListedRef& L, S* g0, typename Store<S>::C ux,
                                            typename Store<S>::C uy, typename Store<S>::C uz,
                                            typename Store<S>::C r1, const typename Store<S>::C g[kQ]) {
  using T = typename Store<S>::C;
  const uint32_t mm = (uint32_t)L.word(kWordPushMove);
#pragma unroll
  for (int j = 0; j < kQ; ++j) {
    const int d = L.word(kWordDst + j);
    T v = g[j];
    if ((mm >> j) & 1u) v += wall_term<T>(OPP(j), ux, uy, uz, r1);
    if (d >= 0) Store<S>::st(g0 + d, v);
  }
  // outlet copies after the primary deliveries (they may replace one)
  constexpr int kPops[kOutletPops] = {2, 8, 10, 12, 14};
#pragma unroll
  for (int e = 0; e < kOutletPops; ++e)
#pragma unroll
    for (int m = 0; m < kOutletCopies; ++m) {
      const int d = L.word(kWordExtra + e * kOutletCopies + m);
      if (d >= 0) Store<S>::st(g0 + d, g[kPops[e]]);
    }
}

// Index of cell idx in the ascending listed-cell array of the domain.
__device__ __forceinline__ long long listed_index(const DevDomain& D, long long idx) {
  long long lo = 0, hi = D.nb - 1;
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    if (__ldg(D.bcell + mid) < idx) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Inflow factors of a launch in the compute type T: arrival level n (pulls)
// and n + 1 (pushes).
template <class T>
__device__ __forceinline__ Wind<T> wind_pull(const StepParams& P) {
  if constexpr (sizeof(T) == 8) return P.wpd;
  else return P.wp;
}
template <class T>
__device__ __forceinline__ Wind<T> wind_push(const StepParams& P) {
  if constexpr (sizeof(T) == 8) return P.wqd;
  else return P.wq;
}

// Inflow table row of layer z of a node, as stored (the steady direction).
template <class S>
__device__ __forceinline__ void table_velocity(const Node<S>& N, int z, typename Store<S>::C& ux,
                                               typename Store<S>::C& uy, typename Store<S>::C& uz) {
  using T = typename Store<S>::C;
  if constexpr (sizeof(T) == 8) {
    ux = T(N.uind[3 * z]);
    uy = T(N.uind[3 * z + 1]);
    uz = T(N.uind[3 * z + 2]);
  } else {
    const float4 u = N.uinf[z];
    ux = T(u.x);
    uy = T(u.y);
    uz = T(u.z);
  }
}

// Inflow velocity of layer z of a node at the level of factor w: the table
// row turned by the level's direction offset (the scale is applied by the
// moving-wall term).
template <class S>
__device__ __forceinline__ void inflow_velocity(const Node<S>& N, int z, Wind<typename Store<S>::C> w,
                                                typename Store<S>::C& ux, typename Store<S>::C& uy,
                                                typename Store<S>::C& uz) {
  using T = typename Store<S>::C;
  T x, y;
  table_velocity<S>(N, z, x, y, uz);
  ux = w.cos_d * x - w.sin_d * y;
  uy = w.sin_d * x + w.cos_d * y;
}

// The same for the moving-wall term of a bulk cell: zero when the cell has
// no inflow link, so the table is not read.  TURN = false reads the table
// row alone (launches whose factors do not turn the inflow).
template <class S, bool TURN = true>
__device__ __forceinline__ void wall_velocity(const Node<S>& N, LinkWord lw, int z,
                                              Wind<typename Store<S>::C> w, typename Store<S>::C& ux,
                                              typename Store<S>::C& uy, typename Store<S>::C& uz) {
  using T = typename Store<S>::C;
  ux = uy = uz = T(0);
  if (!(lw & kLinkVel)) return;
  if constexpr (TURN) inflow_velocity<S>(N, z, w, ux, uy, uz);
  else table_velocity<S>(N, z, ux, uy, uz);
}

// ------------------------------------------------------------ per-node views
template <class S>
__device__ __forceinline__ Node<S> node_view(const DevDomain& D, int node) {
  Node<S> N;
  N.g = reinterpret_cast<S*>(D.g) + (long long)node * kQ * D.pitch;
  N.bout = D.bout ? D.bout + (long long)node * D.nz * D.ny * 5 : nullptr;
  N.uinf = D.uin_f + (long long)node * D.nz;
  N.uind = D.uin_d + (long long)node * D.nz * 3;
  return N;
}

// Outlet cells save their five post-collision populations with c_x = -1
// into the outflow plane at even levels.
template <class S>
__device__ __forceinline__ void save_outlet(const DevDomain& D, const Node<S>& N, int y, int z,
                                            const typename Store<S>::C g[kQ]) {
  float* b = N.bout + ((long long)z * D.ny + y) * 5;
  b[0] = float(g[2]);
  b[1] = float(g[8]);
  b[2] = float(g[10]);
  b[3] = float(g[12]);
  b[4] = float(g[14]);
}

// ------------------------------------------------------------ host dispatch
// Calls f with a null pointer of the population storage type of a precision.
template <class F>
int dispatch(int precision, F&& f) {
  switch (precision) {
    case SC_P_FP32_SHIFT: return f((float*)nullptr);
    case SC_P_BF16_STORE: return f((__nv_bfloat16*)nullptr);
    case SC_P_FP16_STORE: return f((__half*)nullptr);
    case SC_P_FP64_PLAIN: return f((double*)nullptr);
    default: return (int)cudaErrorInvalidValue;
  }
}

}  // namespace
}  // namespace sclbm
