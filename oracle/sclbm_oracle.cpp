/*
 * sclbm_oracle.cpp -- plain, slow, obviously-correct FP64 CPU oracle for the
 * stochastic-collocation lattice Boltzmann pipeline of arXiv:2508.18202
 * ("Uncertain data assimilation for urban wind flow simulations with
 * OpenLB-UQ").
 *
 * TEST INFRASTRUCTURE ONLY.  Used by tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py.  The CUDA library never includes, links or
 * calls it, and it shares no code, table or helper with the library.
 *
 * What it restates, in the paper's order and notation:
 *   - D3Q19 velocity set and c_s^2 = 1/3 (Sec. 2.2, Fig. 1); the weights are
 *     not printed in the paper and are the standard 1/3, 1/18, 1/36.
 *   - Lattice Boltzmann equation (Sec. 2.2, Eq. deterministicLBE):
 *     f_i(x + c_i, t + 1) = f_i^eq + (1 - 1/tau_eff) f_i^(1), in two forms:
 *     BGK (f^(1) = f - f^eq, second-order Hermite equilibrium) and the
 *     paper's recursive regularized form (third-order equilibrium on the
 *     D3Q19-supported Hermite polynomials; f^(1) rebuilt from its second-order
 *     Hermite coefficient and the third-order one obtained recursively).
 *   - Effective relaxation time and Smagorinsky-Lilly viscosity (Sec. 2.2,
 *     Eqs. tauEff and turbVisc), |S| evaluated from the local non-equilibrium
 *     stress (the paper does not say how S is evaluated).
 *   - Boundary conditions of Sec. 2.2: bounce-back walls, velocity inflow
 *     (link-wise moving-wall form), free-slip sky (specular reflection);
 *     plus a zero-gradient outflow face that the paper's disk domain lacks.
 *   - Equilibrium initialisation and a start-up ramp of the inflow (Sec. 2.2).
 *   - Quadrature rules (Sec. 2.3-2.4): Gauss-Legendre and Clenshaw-Curtis
 *     Smolyak sparse grids on uniform inputs.
 *   - Quadrature moments (Sec. 2.3, Eq. quad_moments), two-pass.
 *   - gPC projection (Sec. 2.3, Eqs. gPC and coef_discrete), Legendre basis.
 *   - 95% confidence bands of vertical profiles (Sec. 4, Fig. probes).
 *   - Tangent-linear model of the discrete solver by dual numbers, for the
 *     inflow-parameter gradient of a probe misfit (the paper is silent here).
 *
 * Pull formulation, two arrays, no shift of the populations, no blocking.
 */
#include "sclbm_oracle.h"

#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- lattice
// D3Q19 (Sec. 2.2, Fig. 1): rest velocity, 6 axis velocities, 12 face
// diagonals, listed as opposite pairs.
const int Q = 19;
const int CX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
const int CY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
const int CZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

enum { VELOCITY = 0, OUTFLOW = 1, BOUNCE_BACK = 2, FREE_SLIP = 3, PERIODIC = 4 };
constexpr uint8_t MANTLE = 2;  // cell flag: beyond the circular domain's mantle

double weight(int i) {
  int c2 = CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i];
  if (c2 == 0) return 1.0 / 3.0;
  if (c2 == 1) return 1.0 / 18.0;
  return 1.0 / 36.0;
}

int find_dir(int cx, int cy, int cz) {
  for (int i = 0; i < Q; ++i)
    if (CX[i] == cx && CY[i] == cy && CZ[i] == cz) return i;
  return -1;
}

int opposite(int i) { return find_dir(-CX[i], -CY[i], -CZ[i]); }

int comp(int i, int a) { return a == 0 ? CX[i] : (a == 1 ? CY[i] : CZ[i]); }

// Direction i with its component along axis a negated (specular reflection
// at a face normal to a).
int reflect(int i, int a) {
  int c[3] = {CX[i], CY[i], CZ[i]};
  c[a] = -c[a];
  return find_dir(c[0], c[1], c[2]);
}

// ---------------------------------------------------------------- dual numbers
// Forward-mode derivative in two directions, for the tangent-linear model.
struct Dual {
  double v;
  double d[2];
  Dual() : v(0.0) { d[0] = d[1] = 0.0; }
  Dual(double x) : v(x) { d[0] = d[1] = 0.0; }
};
inline Dual operator+(const Dual& a, const Dual& b) {
  Dual r(a.v + b.v);
  r.d[0] = a.d[0] + b.d[0];
  r.d[1] = a.d[1] + b.d[1];
  return r;
}
inline Dual operator-(const Dual& a, const Dual& b) {
  Dual r(a.v - b.v);
  r.d[0] = a.d[0] - b.d[0];
  r.d[1] = a.d[1] - b.d[1];
  return r;
}
inline Dual operator-(const Dual& a) {
  Dual r(-a.v);
  r.d[0] = -a.d[0];
  r.d[1] = -a.d[1];
  return r;
}
inline Dual operator*(const Dual& a, const Dual& b) {
  Dual r(a.v * b.v);
  r.d[0] = a.d[0] * b.v + a.v * b.d[0];
  r.d[1] = a.d[1] * b.v + a.v * b.d[1];
  return r;
}
inline Dual operator/(const Dual& a, const Dual& b) {
  Dual r(a.v / b.v);
  r.d[0] = (a.d[0] * b.v - a.v * b.d[0]) / (b.v * b.v);
  r.d[1] = (a.d[1] * b.v - a.v * b.d[1]) / (b.v * b.v);
  return r;
}
inline Dual& operator+=(Dual& a, const Dual& b) { a = a + b; return a; }
inline Dual sqrt(const Dual& a) {
  Dual r(std::sqrt(a.v));
  r.d[0] = a.d[0] / (2.0 * r.v);
  r.d[1] = a.d[1] / (2.0 * r.v);
  return r;
}
inline double value(double x) { return x; }
inline double value(const Dual& x) { return x.v; }
using std::sqrt;

// ---------------------------------------------------------------- collision
struct Lat {
  const oc_params* p;
  long long ncell;
  int nx, ny, nz;
  long long idx(int x, int y, int z) const {
    return (long long)x + (long long)nx * ((long long)y + (long long)ny * z);
  }
};

// Second-order Hermite equilibrium (the first three terms of the paper's
// equilibrium, Sec. 2.2): w_i rho (1 + c.u/cs2 + (c.u)^2/(2 cs4) - u.u/(2 cs2)).
template <class T>
void equilibrium(const T& rho, const T u[3], T feq[Q]) {
  T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < Q; ++i) {
    T cu = u[0] * T((double)CX[i]) + u[1] * T((double)CY[i]) + u[2] * T((double)CZ[i]);
    feq[i] = T(weight(i)) * rho * (T(1.0) + T(3.0) * cu + T(4.5) * cu * cu - T(1.5) * uu);
  }
}

// ---------------------------------------------------------------- Hermite basis
// Hermite polynomials of the discrete velocity c_i (Sec. 2.2, with
// c_s^2 = 1/3):
//   H^(2)_ab  = c_a c_b - cs2 d_ab,
//   H^(3)_abg = c_a c_b c_g - cs2 (c_a d_bg + c_b d_ag + c_g d_ab).
// Of the third-order ones, D3Q19 carries only the six with two equal indices,
// and only the combinations
//   H_xxy + H_yzz, H_xzz + H_xyy, H_yyz + H_xxz,
//   H_xxy - H_yzz, H_xzz - H_xyy, H_yyz - H_xxz
// are mutually orthogonal under its weights (the "correct orthogonality for
// D3Q19 only" of the paper's reference).  A third-order term of the model is
// the lattice projection onto these six: w_i sum_k h_k(c_i) A_k / N_k with
// A_k the matching combination of a^(3) and N_k = sum_i w_i h_k(c_i)^2, so
// that the lattice moments sum_i h_k(c_i) f_i reproduce A_k exactly.
const double CS2 = 1.0 / 3.0;

double hermite2_of(int i, int a, int b) {
  return (double)(comp(i, a) * comp(i, b)) - (a == b ? CS2 : 0.0);
}

double hermite3(int i, int a, int b, int g) {
  double v = (double)(comp(i, a) * comp(i, b) * comp(i, g));
  if (b == g) v -= CS2 * comp(i, a);
  if (a == g) v -= CS2 * comp(i, b);
  if (a == b) v -= CS2 * comp(i, g);
  return v;
}

// The six supported combinations: k = 0..2 sums, 3..5 differences of the
// index triples (x,x,y)/(y,z,z), (x,z,z)/(x,y,y), (y,y,z)/(x,x,z).
const int TRIP[3][2][3] = {{{0, 0, 1}, {1, 2, 2}}, {{0, 2, 2}, {0, 1, 1}}, {{1, 1, 2}, {0, 0, 2}}};

double hermite3_comb_of(int i, int k) {
  const int (*t)[3] = TRIP[k % 3];
  const double s = k < 3 ? 1.0 : -1.0;
  return hermite3(i, t[0][0], t[0][1], t[0][2]) + s * hermite3(i, t[1][0], t[1][1], t[1][2]);
}

// The values above depend only on the lattice: they are evaluated once, by
// the same expressions, and looked up per cell.
struct HermiteTables {
  double h2[Q][3][3];
  double h3[Q][6];
  double n3[6];
  HermiteTables() {
    for (int i = 0; i < Q; ++i) {
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) h2[i][a][b] = hermite2_of(i, a, b);
      for (int k = 0; k < 6; ++k) h3[i][k] = hermite3_comb_of(i, k);
    }
    for (int k = 0; k < 6; ++k) {
      double n = 0.0;
      for (int i = 0; i < Q; ++i) n += weight(i) * h3[i][k] * h3[i][k];
      n3[k] = n;
    }
  }
};
const HermiteTables& hermite_tables() {
  static const HermiteTables t;
  return t;
}

double hermite2(int i, int a, int b) { return hermite_tables().h2[i][a][b]; }
double hermite3_comb(int i, int k) { return hermite_tables().h3[i][k]; }
double hermite3_norm(int k) { return hermite_tables().n3[k]; }

// The combination k of a symmetric third-order tensor a[3][3][3].
template <class T>
T comb3(const T a[3][3][3], int k) {
  const int (*t)[3] = TRIP[k % 3];
  const T s = T(k < 3 ? 1.0 : -1.0);
  return a[t[0][0]][t[0][1]][t[0][2]] + s * a[t[1][0]][t[1][1]][t[1][2]];
}

// Third-order equilibrium (Sec. 2.2, the equilibrium expanded up to order
// three): the second-order one plus the lattice projection of
// a^(3)_eq = rho u_a u_b u_g.
template <class T>
void equilibrium3(const T& rho, const T u[3], T feq[Q]) {
  equilibrium(rho, u, feq);
  T a3[3][3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int g = 0; g < 3; ++g) a3[a][b][g] = rho * u[a] * u[b] * u[g];
  for (int k = 0; k < 6; ++k) {
    const T A = comb3(a3, k) / T(hermite3_norm(k));
    for (int i = 0; i < Q; ++i) feq[i] += T(weight(i) * hermite3_comb(i, k)) * A;
  }
}

// One recursive regularized collision (Sec. 2.2, Eq. deterministicLBE with
// the regularized non-equilibrium):
//   f^eq third order;
//   a_1^(2)_ab = sum_i H^(2)_ab(c_i) (f_i - f^eq_i)      (Eq. hermiteCoeff, n = 2);
//   a_1^(3)_abg = u_a a_1^(2)_bg + u_b a_1^(2)_ag + u_g a_1^(2)_ab  (recursive);
//   f^(1)_i = w_i [H^(2)(c_i) : a_1^(2) / (2 cs4) + lattice projection of a_1^(3)];
//   tau_eff from Pi^neq = a_1^(2) exactly as in the BGK form;
//   f*_i = f^eq_i + (1 - 1/tau_eff) f^(1)_i.
template <class T>
void collide_rr(const oc_params* p, const T f[Q], T fpost[Q], double* tau_out) {
  T rho(0.0), j[3] = {T(0.0), T(0.0), T(0.0)};
  for (int i = 0; i < Q; ++i) {
    rho += f[i];
    j[0] += T((double)CX[i]) * f[i];
    j[1] += T((double)CY[i]) * f[i];
    j[2] += T((double)CZ[i]) * f[i];
  }
  T u[3];
  for (int a = 0; a < 3; ++a) u[a] = j[a] / rho;
  T feq[Q];
  equilibrium3(rho, u, feq);
  T a2[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      a2[a][b] = T(0.0);
      for (int i = 0; i < Q; ++i) a2[a][b] += T(hermite2(i, a, b)) * (f[i] - feq[i]);
    }
  T a3[3][3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int g = 0; g < 3; ++g) a3[a][b][g] = u[a] * a2[b][g] + u[b] * a2[a][g] + u[g] * a2[a][b];
  T f1[Q];
  for (int i = 0; i < Q; ++i) {
    T s2(0.0);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) s2 += T(hermite2(i, a, b)) * a2[a][b];
    f1[i] = T(weight(i)) * s2 / T(2.0 * CS2 * CS2);
  }
  for (int k = 0; k < 6; ++k) {
    const T A = comb3(a3, k) / T(hermite3_norm(k));
    for (int i = 0; i < Q; ++i) f1[i] += T(weight(i) * hermite3_comb(i, k)) * A;
  }
  T tau(p->tau0);
  if (p->csmag != 0.0) {
    T PiPi(0.0);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) PiPi += a2[a][b] * a2[a][b];
    T Pin = sqrt(T(2.0) * PiPi + T(1e-30));
    double c2 = p->csmag * p->csmag;
    tau = T(0.5) * (T(p->tau0) + sqrt(T(p->tau0 * p->tau0) + T(18.0 * c2) * Pin / rho));
  }
  if (tau_out) *tau_out = value(tau);
  const T keep = T(1.0) - T(1.0) / tau;
  for (int i = 0; i < Q; ++i) fpost[i] = feq[i] + keep * f1[i];
}

// One BGK(+Smagorinsky) collision of one cell (Sec. 2.2):
//   rho = sum f, u = sum c f / rho,
//   Pi^neq = sum c c (f - f^eq),
//   S = -Pi^neq / (2 rho cs2 tau_eff), |S| = sqrt(2 S:S),
//   tau_eff = 3 (nu + (C_S dx)^2 |S|) + 1/2  (dx = dt = 1, Eq. tauEff),
// which with tau0 = 3 nu + 1/2 solves to
//   tau_eff = (tau0 + sqrt(tau0^2 + 18 C_S^2 sqrt(2 Pi:Pi) / rho)) / 2,
// then f* = f - (f - f^eq) / tau_eff.  An optional body force F enters by
// Guo's scheme (only the Poiseuille pin uses it).
template <class T>
void collide(const oc_params* p, const T f[Q], T fpost[Q], double* tau_out) {
  if (p->collision == 1) {
    collide_rr(p, f, fpost, tau_out);
    return;
  }
  T rho(0.0), j[3] = {T(0.0), T(0.0), T(0.0)};
  for (int i = 0; i < Q; ++i) {
    rho += f[i];
    j[0] += T((double)CX[i]) * f[i];
    j[1] += T((double)CY[i]) * f[i];
    j[2] += T((double)CZ[i]) * f[i];
  }
  const bool forced = p->force[0] != 0.0 || p->force[1] != 0.0 || p->force[2] != 0.0;
  T u[3];
  for (int a = 0; a < 3; ++a) u[a] = (j[a] + T(0.5 * p->force[a])) / rho;
  T feq[Q];
  equilibrium(rho, u, feq);
  T tau(p->tau0);
  if (p->csmag != 0.0) {
    T Pi[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Pi[a][b] = T(0.0);
    for (int i = 0; i < Q; ++i) {
      T fneq = f[i] - feq[i];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Pi[a][b] += T((double)(comp(i, a) * comp(i, b))) * fneq;
    }
    T PiPi(0.0);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) PiPi += Pi[a][b] * Pi[a][b];
    // The 1e-30 keeps the square root differentiable at Pi = 0.
    T Pin = sqrt(T(2.0) * PiPi + T(1e-30));
    double c2 = p->csmag * p->csmag;
    tau = T(0.5) * (T(p->tau0) + sqrt(T(p->tau0 * p->tau0) + T(18.0 * c2) * Pin / rho));
  }
  if (tau_out) *tau_out = value(tau);
  T omega = T(1.0) / tau;
  for (int i = 0; i < Q; ++i) fpost[i] = f[i] - omega * (f[i] - feq[i]);
  if (forced) {
    T pref = T(1.0) - T(0.5) * omega;
    for (int i = 0; i < Q; ++i) {
      T cu = u[0] * T((double)CX[i]) + u[1] * T((double)CY[i]) + u[2] * T((double)CZ[i]);
      T s(0.0);
      for (int a = 0; a < 3; ++a) {
        T term = T(3.0) * (T((double)comp(i, a)) - u[a]) + T(9.0) * cu * T((double)comp(i, a));
        s += term * T(p->force[a]);
      }
      fpost[i] += pref * T(weight(i)) * s;
    }
  }
}

// ---------------------------------------------------------------- streaming
// Start-up ramp of the inflow (Sec. 2.2: the boundary velocity is increased
// to its target over time; the shape is not printed).  Reading:
// r(m) = (1 - cos(pi min(m, T_r) / T_r)) / 2 at arrival time level m, r = 1
// for T_r = 0.
double ramp(int Tr, long long m) {
  if (Tr <= 0) return 1.0;
  long long mm = m < Tr ? m : Tr;
  return 0.5 * (1.0 - std::cos(M_PI * (double)mm / (double)Tr));
}

bool is_periodic_axis(const oc_params* p, int a) { return p->bc[2 * a] == PERIODIC; }

// Value of f_i at fluid cell (x,y,z) at time level m = n + 1, pulled from the
// post-collision field of time n.  Rules (walls half-way between cells):
//   source p = x - c_i (periodic axes wrapped);
//   p inside and fluid            -> f*_i(p)                   (streaming)
//   p inside and solid            -> f*_opp(i)(x)              (bounce-back)
//   p inside and beyond the mantle (flag 2, the circular domain's local
//     velocity boundary)          -> the VELOCITY rule below
//   p across exactly one face of kind
//     BOUNCE_BACK                 -> f*_opp(i)(x)
//     VELOCITY                    -> f*_opp(i)(x) + 6 w_i rho_w (c_i . u_w(z)) r(m)
//     FREE_SLIP (normal a)        -> f*_refl_a(i)(s), s = x - c_i + c_ia e_a, if s fluid,
//                                    else bounce-back
//     OUTFLOW   (normal a)        -> f*_i(s), same s, if s fluid, else f*_i(x)
//   p across two faces (D3Q19 has no link crossing three; c_i then has
//   exactly the two crossed components, so the cell itself is the only
//   in-domain source)
//                                 -> bounce-back if any face is BOUNCE_BACK,
//                                    else the VELOCITY rule if any face is
//                                    VELOCITY, else f*_i'(x) with i' = i
//                                    reflected across every FREE_SLIP face
//                                    crossed (FREE_SLIP + FREE_SLIP is thus
//                                    bounce-back, OUTFLOW + FREE_SLIP a
//                                    reflection in the cell itself).
// The moving-wall rule of a velocity boundary: f*_opp(i)(x) + 6 w_i
// (c_i . u_w(z)) r(m), rho_w = 1.
template <class T>
T velocity_link(const T* fpost, const Lat& L, const T* uin, double r, long long xi, int z, int i) {
  T cu = T((double)CX[i]) * uin[3 * z + 0] + T((double)CY[i]) * uin[3 * z + 1] +
         T((double)CZ[i]) * uin[3 * z + 2];
  return fpost[(long long)opposite(i) * L.ncell + xi] + T(6.0 * weight(i) * r) * cu;
}

template <class T>
T pull(const Lat& L, const uint8_t* flags, const T* fpost, const T* uin, double r,
       int x, int y, int z, int i) {
  const oc_params* p = L.p;
  const int n[3] = {L.nx, L.ny, L.nz};
  int xc[3] = {x, y, z};
  int s[3] = {x - CX[i], y - CY[i], z - CZ[i]};
  int crossed[3];
  int nc = 0;
  for (int a = 0; a < 3; ++a) {
    if (is_periodic_axis(p, a)) {
      s[a] = ((s[a] % n[a]) + n[a]) % n[a];
      continue;
    }
    if (s[a] < 0) crossed[nc++] = 2 * a;
    else if (s[a] >= n[a]) crossed[nc++] = 2 * a + 1;
  }
  const long long xi = L.idx(x, y, z);
  const int oi = opposite(i);
  if (nc == 0) {
    long long si = L.idx(s[0], s[1], s[2]);
    if (flags[si] == 0) return fpost[(long long)i * L.ncell + si];
    if (flags[si] == MANTLE) return velocity_link(fpost, L, uin, r, xi, z, i);
    return fpost[(long long)oi * L.ncell + xi];
  }
  int kind;
  if (nc == 1) {
    kind = p->bc[crossed[0]];
  } else {
    bool bb = false, vel = false;
    for (int k = 0; k < nc; ++k) {
      if (p->bc[crossed[k]] == BOUNCE_BACK) bb = true;
      if (p->bc[crossed[k]] == VELOCITY) vel = true;
    }
    if (!bb && !vel) {
      int ir = i;
      for (int k = 0; k < nc; ++k)
        if (p->bc[crossed[k]] == FREE_SLIP) ir = reflect(ir, crossed[k] / 2);
      return fpost[(long long)ir * L.ncell + xi];
    }
    kind = bb ? BOUNCE_BACK : VELOCITY;
  }
  if (kind == BOUNCE_BACK) return fpost[(long long)oi * L.ncell + xi];
  if (kind == VELOCITY) return velocity_link(fpost, L, uin, r, xi, z, i);
  // single face: FREE_SLIP or OUTFLOW; s = x - c_i with the normal component removed
  const int a = crossed[0] / 2;
  int src[3] = {xc[0] - CX[i], xc[1] - CY[i], xc[2] - CZ[i]};
  src[a] = xc[a];
  for (int b = 0; b < 3; ++b)
    if (is_periodic_axis(p, b)) src[b] = ((src[b] % n[b]) + n[b]) % n[b];
  long long si = L.idx(src[0], src[1], src[2]);
  if (kind == FREE_SLIP) {
    if (flags[si] == 0) return fpost[(long long)reflect(i, a) * L.ncell + si];
    if (flags[si] == MANTLE) return velocity_link(fpost, L, uin, r, xi, z, i);
    return fpost[(long long)oi * L.ncell + xi];
  }
  // OUTFLOW
  if (flags[si] == 0) return fpost[(long long)i * L.ncell + si];
  return fpost[(long long)i * L.ncell + xi];
}

template <class T>
void run_steps(const oc_params* p, const uint8_t* flags, const T* uin, T* f, long long n0,
               int n_steps) {
  Lat L{p, (long long)p->nx * p->ny * p->nz, p->nx, p->ny, p->nz};
  std::vector<T> fpost((size_t)Q * L.ncell);
  for (int s = 0; s < n_steps; ++s) {
    // collide every fluid cell at time n
#pragma omp parallel for schedule(static)
    for (int z = 0; z < L.nz; ++z)
      for (int y = 0; y < L.ny; ++y)
        for (int x = 0; x < L.nx; ++x) {
          long long c = L.idx(x, y, z);
          if (flags[c] != 0) continue;
          T fl[Q], fp[Q];
          for (int i = 0; i < Q; ++i) fl[i] = f[(long long)i * L.ncell + c];
          collide(p, fl, fp, nullptr);
          for (int i = 0; i < Q; ++i) fpost[(long long)i * L.ncell + c] = fp[i];
        }
    // stream into time n + 1
    const double r = ramp(p->ramp_steps, n0 + s + 1);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < L.nz; ++z)
      for (int y = 0; y < L.ny; ++y)
        for (int x = 0; x < L.nx; ++x) {
          long long c = L.idx(x, y, z);
          if (flags[c] != 0) continue;
          for (int i = 0; i < Q; ++i)
            f[(long long)i * L.ncell + c] = pull(L, flags, fpost.data(), uin, r, x, y, z, i);
        }
  }
}

int check_params(const oc_params* p) {
  if (!p || p->nx < 1 || p->ny < 1 || p->nz < 1) return -1;
  for (int a = 0; a < 3; ++a) {
    bool lo = p->bc[2 * a] == PERIODIC, hi = p->bc[2 * a + 1] == PERIODIC;
    if (lo != hi) return -1;
  }
  for (int k = 0; k < 6; ++k)
    if (p->bc[k] < 0 || p->bc[k] > 4) return -1;
  if (!(p->tau0 > 0.5)) return -1;
  if (p->collision != 0 && p->collision != 1) return -1;
  if (p->collision == 1 && (p->force[0] != 0.0 || p->force[1] != 0.0 || p->force[2] != 0.0)) return -1;
  return 0;
}

// ---------------------------------------------------------------- SplitMix64
// Steele, Lea & Flood (2014), "Fast splittable pseudorandom number generators".
struct SplitMix64 {
  uint64_t s;
  explicit SplitMix64(uint64_t seed) : s(seed) {}
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ULL;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  }
  // integer draw U{a..b}
  int uniform(int a, int b) { return a + (int)(next() % (uint64_t)(b - a + 1)); }
};

// ---------------------------------------------------------------- quadrature
// 1-D Gauss-Legendre on [-1,1] (weights summing to 2), closed forms for
// n <= 5, nodes ascending.
int gauss_legendre(int n, double* x, double* w) {
  if (n == 1) {
    x[0] = 0.0; w[0] = 2.0;
  } else if (n == 2) {
    double r = 1.0 / sqrt(3.0);
    x[0] = -r; x[1] = r; w[0] = 1.0; w[1] = 1.0;
  } else if (n == 3) {
    double r = sqrt(3.0 / 5.0);
    x[0] = -r; x[1] = 0.0; x[2] = r;
    w[0] = 5.0 / 9.0; w[1] = 8.0 / 9.0; w[2] = 5.0 / 9.0;
  } else if (n == 4) {
    double a = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0));
    double b = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
    double wa = (18.0 + sqrt(30.0)) / 36.0, wb = (18.0 - sqrt(30.0)) / 36.0;
    x[0] = -b; x[1] = -a; x[2] = a; x[3] = b;
    w[0] = wb; w[1] = wa; w[2] = wa; w[3] = wb;
  } else if (n == 5) {
    double a = sqrt(5.0 - 2.0 * sqrt(10.0 / 7.0)) / 3.0;
    double b = sqrt(5.0 + 2.0 * sqrt(10.0 / 7.0)) / 3.0;
    double wa = (322.0 + 13.0 * sqrt(70.0)) / 900.0, wb = (322.0 - 13.0 * sqrt(70.0)) / 900.0;
    x[0] = -b; x[1] = -a; x[2] = 0.0; x[3] = a; x[4] = b;
    w[0] = wb; w[1] = wa; w[2] = 128.0 / 225.0; w[3] = wa; w[4] = wb;
  } else {
    return -1;
  }
  return 0;
}

int cc_points(int level) { return level == 1 ? 1 : (1 << (level - 1)) + 1; }

// 1-D Clenshaw-Curtis rule of a level (1-based) on [-1,1], weights summing to 2.
// x_k = -cos(pi k / n), n = m - 1, with the midpoint, end points and mirrored
// pairs forced exact; w_k = (c_k / n) (1 - sum_{j=1}^{n/2} b_j cos(2 j k pi / n)
// / (4 j^2 - 1)), c_0 = c_n = 1, c_k = 2 otherwise, b_{n/2} = 1 for even n,
// b_j = 2 otherwise.
void clenshaw_curtis(int level, std::vector<double>& x, std::vector<double>& w) {
  int m = cc_points(level);
  x.assign(m, 0.0);
  w.assign(m, 0.0);
  if (m == 1) {
    x[0] = 0.0; w[0] = 2.0;
    return;
  }
  int n = m - 1;
  for (int k = 0; k < m; ++k) x[k] = -std::cos((double)k * M_PI / (double)n);
  for (int k = 0; 2 * k < n; ++k) x[n - k] = -x[k];
  x[0] = -1.0; x[n] = 1.0;
  if (n % 2 == 0) x[n / 2] = 0.0;
  for (int k = 0; k <= n; ++k) {
    double s = 0.0;
    for (int j = 1; j <= n / 2; ++j) {
      double b = (2 * j == n) ? 1.0 : 2.0;
      double c = std::cos((double)(2 * j * k) * M_PI / (double)n);
      s += b / (double)(4 * j * j - 1) * c;
    }
    double ck = (k == 0 || k == n) ? 1.0 : 2.0;
    w[k] = ck / (double)n * (1.0 - s);
  }
}

long long binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  long long r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

}  // namespace

// ======================================================================= C API
extern "C" {

int oc_lattice(int* cx, int* cy, int* cz, double* w, int* opp) {
  for (int i = 0; i < Q; ++i) {
    if (cx) cx[i] = CX[i];
    if (cy) cy[i] = CY[i];
    if (cz) cz[i] = CZ[i];
    if (w) w[i] = weight(i);
    if (opp) opp[i] = opposite(i);
  }
  return 0;
}

int oc_equilibrium(double rho, const double* u, double* feq) {
  double uu[3] = {u[0], u[1], u[2]};
  equilibrium<double>(rho, uu, feq);
  return 0;
}

int oc_equilibrium3(double rho, const double* u, double* feq) {
  double uu[3] = {u[0], u[1], u[2]};
  equilibrium3<double>(rho, uu, feq);
  return 0;
}

int oc_collide_cell(const oc_params* p, const double* f, double* fpost, double* tau_eff) {
  if (!p || !f || !fpost || check_params(p)) return -1;
  collide<double>(p, f, fpost, tau_eff);
  return 0;
}

double oc_ramp(int ramp_steps, long long m) { return ramp(ramp_steps, m); }

int oc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

// Equilibrium initialisation (Sec. 2.2): f = f^eq(rho, u) on fluid cells,
// solid cells zero.  rho/u may be NULL for rho = 1, u = 0.
int oc_init_equilibrium(const oc_params* p, const uint8_t* flags, const double* rho,
                        const double* u, double* f) {
  if (check_params(p)) return -1;
  long long n = (long long)p->nx * p->ny * p->nz;
  for (long long c = 0; c < n; ++c) {
    double fe[Q];
    double uc[3] = {0.0, 0.0, 0.0};
    double r = 1.0;
    if (rho) r = rho[c];
    if (u) { uc[0] = u[c]; uc[1] = u[n + c]; uc[2] = u[2 * n + c]; }
    if (p->collision == 1) equilibrium3<double>(r, uc, fe);
    else equilibrium<double>(r, uc, fe);
    for (int i = 0; i < Q; ++i) f[(long long)i * n + c] = flags[c] ? 0.0 : fe[i];
  }
  return 0;
}

// Advance n_steps time steps from time level n0.  uin[nz][3] is the inflow
// velocity per cell layer used by VELOCITY faces.
int oc_run(const oc_params* p, const uint8_t* flags, const double* uin, double* f,
           long long n0, int n_steps) {
  if (check_params(p) || !flags || !uin || !f || n_steps < 0) return -1;
  run_steps<double>(p, flags, uin, f, n0, n_steps);
  return 0;
}

// rho[ncell], u[3][ncell] of the natural-layout state; solid cells: rho = 0, u = 0.
int oc_macros(const oc_params* p, const uint8_t* flags, const double* f, double* rho,
              double* u) {
  if (check_params(p)) return -1;
  long long n = (long long)p->nx * p->ny * p->nz;
  for (long long c = 0; c < n; ++c) {
    if (flags[c]) {
      if (rho) rho[c] = 0.0;
      if (u) u[c] = u[n + c] = u[2 * n + c] = 0.0;
      continue;
    }
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
      double fi = f[(long long)i * n + c];
      r += fi;
      j[0] += CX[i] * fi;
      j[1] += CY[i] * fi;
      j[2] += CZ[i] * fi;
    }
    if (rho) rho[c] = r;
    if (u) {
      u[c] = j[0] / r;
      u[n + c] = j[1] / r;
      u[2 * n + c] = j[2] / r;
    }
  }
  return 0;
}

int oc_splitmix64(uint64_t seed, int n, uint64_t* out) {
  SplitMix64 g(seed);
  for (int k = 0; k < n; ++k) out[k] = g.next();
  return 0;
}

// Seeded synthetic urban geometry (the paper's real buildings are not
// available).  Explicit half-open boxes [x0,x1)x[y0,y1)x[z0,z1) if n_boxes > 0,
// else n_buildings rectangular blocks drawn in this order per block:
// wx, wy ~ U{fp_min..fp_max}; h ~ U{h_min..min(h_max, nz-4)};
// x0 ~ U{nx/8 .. nx - nx/8 - wx}; y0 ~ U{2 .. ny - 2 - wy};
// block = [x0,x0+wx) x [y0,y0+wy) x [0,h).
int oc_geometry(int nx, int ny, int nz, uint64_t seed, int n_buildings, int fp_min,
                int fp_max, int h_min, int h_max, const int32_t* boxes, int n_boxes,
                uint8_t* flags) {
  if (nx < 1 || ny < 1 || nz < 1 || !flags) return -1;
  long long n = (long long)nx * ny * nz;
  std::memset(flags, 0, (size_t)n);
  auto fill = [&](int x0, int y0, int z0, int x1, int y1, int z1) {
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (z0 < 0) z0 = 0;
    if (x1 > nx) x1 = nx;
    if (y1 > ny) y1 = ny;
    if (z1 > nz) z1 = nz;
    for (int z = z0; z < z1; ++z)
      for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) flags[x + (long long)nx * (y + (long long)ny * z)] = 1;
  };
  if (n_boxes > 0) {
    for (int b = 0; b < n_boxes; ++b) {
      const int32_t* B = boxes + 6 * b;
      fill(B[0], B[1], B[2], B[3], B[4], B[5]);
    }
    return 0;
  }
  SplitMix64 g(seed);
  int hm = h_max < nz - 4 ? h_max : nz - 4;
  for (int k = 0; k < n_buildings; ++k) {
    if (fp_max < fp_min || hm < h_min) return -1;
    int wx = g.uniform(fp_min, fp_max);
    int wy = g.uniform(fp_min, fp_max);
    int h = g.uniform(h_min, hm);
    int xa = nx / 8, xb = nx - nx / 8 - wx;
    int ya = 2, yb = ny - 2 - wy;
    if (xb < xa || yb < ya) return -1;
    int x0 = g.uniform(xa, xb);
    int y0 = g.uniform(ya, yb);
    fill(x0, y0, 0, x0 + wx, y0 + wy, h);
  }
  return 0;
}

// Probe columns (x, y) for vertical profiles: SplitMix64 stream seeded with
// seed + 1; draw x ~ U{nx/8..nx-1}, y ~ U{0..ny-1}; accept when the ground
// cell (x, y, 0) is fluid and the column is new.
// Circular domain (Sec. 2.2: a disk of radius R whose mantle carries a local
// velocity boundary): every cell whose centre (x + 1/2, y + 1/2) lies more
// than R from the axis (nx / 2, ny / 2) is beyond the mantle, flag 2, in all
// layers (buildings there included).
int oc_mark_mantle(int nx, int ny, int nz, double radius, uint8_t* flags) {
  if (nx < 1 || ny < 1 || nz < 1 || !flags || !(radius > 0.0)) return -1;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const double dx = x + 0.5 - 0.5 * nx, dy = y + 0.5 - 0.5 * ny;
      if (dx * dx + dy * dy <= radius * radius) continue;
      for (int z = 0; z < nz; ++z) flags[x + (long long)nx * (y + (long long)ny * z)] = MANTLE;
    }
  return 0;
}

int oc_probe_columns(int nx, int ny, int nz, uint64_t seed, const uint8_t* flags, int n,
                     int32_t* xy) {
  (void)nz;
  SplitMix64 g(seed + 1ULL);
  int got = 0;
  for (long long tries = 0; got < n; ++tries) {
    if (tries > 1000000) return -1;
    int x = g.uniform(nx / 8, nx - 1);
    int y = g.uniform(0, ny - 1);
    if (flags[x + (long long)nx * y] != 0) continue;
    bool dup = false;
    for (int k = 0; k < got; ++k)
      if (xy[2 * k] == x && xy[2 * k + 1] == y) dup = true;
    if (dup) continue;
    xy[2 * got] = x;
    xy[2 * got + 1] = y;
    ++got;
  }
  return 0;
}

// Probe points (x, y, z): same stream, x ~ U{nx/8..nx-1}, y ~ U{0..ny-1},
// z ~ U{0..nz-3}; accept fluid, new points.
int oc_probe_points(int nx, int ny, int nz, uint64_t seed, const uint8_t* flags, int n,
                    int32_t* xyz) {
  SplitMix64 g(seed + 1ULL);
  int got = 0;
  for (long long tries = 0; got < n; ++tries) {
    if (tries > 1000000) return -1;
    int x = g.uniform(nx / 8, nx - 1);
    int y = g.uniform(0, ny - 1);
    int z = g.uniform(0, nz - 3);
    if (flags[x + (long long)nx * (y + (long long)ny * z)] != 0) continue;
    bool dup = false;
    for (int k = 0; k < got; ++k)
      if (xyz[3 * k] == x && xyz[3 * k + 1] == y && xyz[3 * k + 2] == z) dup = true;
    if (dup) continue;
    xyz[3 * got] = x;
    xyz[3 * got + 1] = y;
    xyz[3 * got + 2] = z;
    ++got;
  }
  return 0;
}

// Power-law inflow per cell layer (the configuration's profile; the paper's
// own profile is logarithmic, Sec. 3): h = k + 1/2 above the ground face,
// u_in(k) = u_ref (1 + xi) (h / H)^alpha (cos theta, sin theta, 0).
int oc_inflow(int nz, double u_ref, double xi, double alpha, double H, double theta_deg,
              double* uin) {
  if (nz < 1 || !(H > 0.0)) return -1;
  double th = theta_deg * M_PI / 180.0;
  for (int k = 0; k < nz; ++k) {
    double h = (double)k + 0.5;
    double mag = u_ref * (1.0 + xi) * std::pow(h / H, alpha);
    uin[3 * k + 0] = mag * std::cos(th);
    uin[3 * k + 1] = mag * std::sin(th);
    uin[3 * k + 2] = 0.0;
  }
  return 0;
}

// Probabilists' Hermite polynomial He_n(x) by the three-term recurrence
// He_{k+1} = x He_k - k He_{k-1}.
static double hermite_e(int n, double x) {
  double a = 1.0, b = x;
  if (n == 0) return a;
  for (int k = 1; k < n; ++k) {
    double c = x * b - k * a;
    a = b;
    b = c;
  }
  return b;
}

// n-point Gauss-Hermite rule for the standard normal density (Sec. 2.4 step 3,
// the dense tensor-product Gauss-Hermite quadrature): nodes are the roots of
// He_n, found by bisection between the sign changes of He_n on a fine grid;
// probability weights n! / (n He_{n-1}(x_k))^2.
static void gauss_hermite(int n, std::vector<double>& x, std::vector<double>& w) {
  x.clear();
  w.clear();
  const double L = std::sqrt(4.0 * n + 2.0) + 1.0;
  const int grid = 400 * n + 1;
  double xa = -L, fa = hermite_e(n, xa);
  for (int g = 1; g < grid; ++g) {
    double xb = -L + 2.0 * L * g / (grid - 1), fb = hermite_e(n, xb);
    if (fb == 0.0) {
      x.push_back(xb);
    } else if (fa != 0.0 && (fa < 0.0) != (fb < 0.0)) {
      double lo = xa, hi = xb, flo = fa;
      for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi), fm = hermite_e(n, mid);
        if (fm == 0.0 || mid == lo || mid == hi) { lo = hi = mid; break; }
        if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; }
        else hi = mid;
      }
      x.push_back(0.5 * (lo + hi));
    }
    xa = xb;
    fa = fb;
  }
  double fact = 1.0;
  for (int k = 2; k <= n; ++k) fact *= k;
  for (double xk : x) {
    double h = (double)n * hermite_e(n - 1, xk);
    w.push_back(fact / (h * h));
  }
}

// Logarithmic wind profile (Sec. 3): u(h) = u_ref (1 + xi) ln((h + z0)/z0) /
// ln((H + z0)/z0) (cos theta, sin theta, 0), h = k + 1/2 above the ground
// face, z0 the roughness length, both in cells.
int oc_inflow_log(int nz, double u_ref, double xi, double z0, double H, double theta_deg, double* uin) {
  if (nz < 1 || !(H > 0.0) || !(z0 > 0.0)) return -1;
  double th = theta_deg * M_PI / 180.0;
  double den = std::log((H + z0) / z0);
  for (int k = 0; k < nz; ++k) {
    double h = (double)k + 0.5;
    double mag = u_ref * (1.0 + xi) * std::log((h + z0) / z0) / den;
    uin[3 * k + 0] = mag * std::cos(th);
    uin[3 * k + 1] = mag * std::sin(th);
    uin[3 * k + 2] = 0.0;
  }
  return 0;
}

// Quadrature rules with probability weights.
//   rule 0: tensor Gauss-Legendre, `level` points per dimension (1..5)
//   rule 1: Clenshaw-Curtis Smolyak sparse grid of level L (1-based):
//           sum over L <= |i| <= L+d-1 of (-1)^(L+d-1-|i|) C(d-1, L+d-1-|i|)
//           times the tensor rule of 1-D levels i.
//   (rules 0 and 1: uniform inputs on prod [lo_t, hi_t])
//   rule 2: tensor Gauss-Hermite, `level` points per dimension (1..40), for
//           normal inputs with mean lo_t and standard deviation hi_t.
// Nodes are returned in lexicographic order of their integer index on the
// finest 1-D grid (first coordinate most significant).  Z[n][d], w[n].
// With Z == NULL only the count is returned.
int oc_quadrature(int rule, int d, int level, const double* lo, const double* hi, int* n_out,
                  double* Z, double* w, int cap) {
  if (d < 1 || d > 3 || level < 1 || !n_out) return -1;
  std::map<std::vector<int>, double> acc;   // finest index -> weight
  std::vector<double> finest_x;
  if (rule == 0) {
    if (level > 5) return -1;
    double x1[5], w1[5];
    gauss_legendre(level, x1, w1);
    finest_x.assign(x1, x1 + level);
    std::vector<int> k(d, 0);
    while (true) {
      double prod = 1.0;
      for (int t = 0; t < d; ++t) prod *= w1[k[t]] * 0.5;
      acc[k] += prod;
      int t = d - 1;
      while (t >= 0 && ++k[t] == level) { k[t] = 0; --t; }
      if (t < 0) break;
    }
  } else if (rule == 1) {
    if (level > 12) return -1;
    const int mmax = cc_points(level);
    std::vector<double> wtmp;
    clenshaw_curtis(level, finest_x, wtmp);
    std::vector<std::vector<double>> x1(level + 1), w1(level + 1);
    for (int l = 1; l <= level; ++l) {
      clenshaw_curtis(l, x1[l], w1[l]);
      for (double& v : w1[l]) v *= 0.5;
    }
    std::vector<int> i(d, 1);
    while (true) {
      int s = 0;
      for (int t = 0; t < d; ++t) s += i[t];
      if (s >= level && s <= level + d - 1) {
        int e = level + d - 1 - s;
        long long coef = binom(d - 1, e) * ((e % 2) ? -1 : 1);
        std::vector<int> k(d, 0);
        while (true) {
          double prod = (double)coef;
          std::vector<int> K(d);
          for (int t = 0; t < d; ++t) {
            int m = cc_points(i[t]);
            prod *= w1[i[t]][k[t]];
            K[t] = (m == 1) ? (mmax - 1) / 2 : k[t] * ((mmax - 1) / (m - 1));
          }
          acc[K] += prod;
          int t = d - 1;
          while (t >= 0 && ++k[t] == cc_points(i[t])) { k[t] = 0; --t; }
          if (t < 0) break;
        }
      }
      int t = d - 1;
      while (t >= 0 && ++i[t] > level) { i[t] = 1; --t; }
      if (t < 0) break;
    }
  } else if (rule == 2) {
    if (level > 40) return -1;
    std::vector<double> w1;
    gauss_hermite(level, finest_x, w1);
    if ((int)finest_x.size() != level) return -1;
    std::vector<int> k(d, 0);
    while (true) {
      double prod = 1.0;
      for (int t = 0; t < d; ++t) prod *= w1[k[t]];
      acc[k] += prod;
      int t = d - 1;
      while (t >= 0 && ++k[t] == level) { k[t] = 0; --t; }
      if (t < 0) break;
    }
  } else {
    return -1;
  }
  int n = (int)acc.size();
  *n_out = n;
  if (!Z) return 0;
  if (n > cap) return -2;
  int j = 0;
  for (const auto& kv : acc) {
    for (int t = 0; t < d; ++t) {
      double x = finest_x[kv.first[t]];
      Z[(long long)j * d + t] = rule == 2 ? lo[t] + hi[t] * x
                                          : 0.5 * (lo[t] + hi[t]) + 0.5 * (hi[t] - lo[t]) * x;
    }
    w[j] = kv.second;
    ++j;
  }
  return 0;
}

// Quadrature moments (Sec. 2.3, Eq. quad_moments), two-pass:
// W = sum a_j, E = sum a_j Q_j / W, Var = sum a_j (Q_j - E)^2 / W,
// std = sqrt(max(Var, 0)); cells with Var < 0 (possible with negative
// sparse-grid weights) are clamped and counted.  Q[nq][ncell].
int oc_moments_two_pass(int nq, long long ncell, const double* a, const double* Q,
                        double* mean, double* stdev, long long* n_clamped) {
  if (nq < 1) return -1;
  double W = 0.0;
  for (int j = 0; j < nq; ++j) W += a[j];
  long long clamped = 0;
  for (long long c = 0; c < ncell; ++c) {
    double e = 0.0;
    for (int j = 0; j < nq; ++j) e += a[j] * Q[(long long)j * ncell + c];
    e /= W;
    double v = 0.0;
    for (int j = 0; j < nq; ++j) {
      double dq = Q[(long long)j * ncell + c] - e;
      v += a[j] * dq * dq;
    }
    v /= W;
    if (v < 0.0) { v = 0.0; ++clamped; }
    mean[c] = e;
    stdev[c] = std::sqrt(v);
  }
  if (n_clamped) *n_clamped = clamped;
  return 0;
}

// Vertical profiles with 95% confidence bands (Sec. 4, Table probes and the
// profile figure).  For column p and layer z: mean and std over the nodes as
// above, lo/hi = mean -/+ 1.959963984540054 std (Gaussian band; the paper
// does not print its construction).  prof[p][z][4] = (mean, std, lo, hi),
// prof_nodes[p][j][z] = Q_j at the column.
int oc_profiles(int nq, int nx, int ny, int nz, const double* a, const double* Q, int n_p,
                const int32_t* xy, double* prof, double* prof_nodes) {
  long long ncell = (long long)nx * ny * nz;
  std::vector<double> vals(nq);
  double W = 0.0;
  for (int j = 0; j < nq; ++j) W += a[j];
  for (int p = 0; p < n_p; ++p)
    for (int z = 0; z < nz; ++z) {
      long long c = xy[2 * p] + (long long)nx * (xy[2 * p + 1] + (long long)ny * z);
      double e = 0.0;
      for (int j = 0; j < nq; ++j) {
        vals[j] = Q[(long long)j * ncell + c];
        e += a[j] * vals[j];
      }
      e /= W;
      double v = 0.0;
      for (int j = 0; j < nq; ++j) v += a[j] * (vals[j] - e) * (vals[j] - e);
      v /= W;
      if (v < 0.0) v = 0.0;
      double s = std::sqrt(v);
      double* P = prof + ((long long)p * nz + z) * 4;
      P[0] = e;
      P[1] = s;
      P[2] = e - 1.959963984540054 * s;
      P[3] = e + 1.959963984540054 * s;
      if (prof_nodes)
        for (int j = 0; j < nq; ++j) prof_nodes[((long long)p * nq + j) * nz + z] = vals[j];
    }
  return 0;
}

// Total-degree multi-indices in graded order: degree 0, 1, ..., and within a
// degree alpha_1 descending, then alpha_2 descending, ...
static void mi_rec(int pos, int rem, int d, std::vector<int>& cur,
                   std::vector<std::vector<int>>& res) {
  if (pos == d - 1) {
    cur[pos] = rem;
    res.push_back(cur);
    return;
  }
  for (int v = rem; v >= 0; --v) {
    cur[pos] = v;
    mi_rec(pos + 1, rem - v, d, cur, res);
  }
}

static void multi_indices(int d, int degree, std::vector<std::vector<int>>& out) {
  out.clear();
  std::vector<int> cur(d, 0);
  for (int t = 0; t <= degree; ++t) mi_rec(0, t, d, cur, out);
}

int oc_gpc_basis_size(int d, int degree) {
  if (d < 1 || degree < 0) return -1;
  return (int)binom(degree + d, d);
}

// Orthonormal Legendre basis for uniform inputs (Sec. 2.3, Eq. gPC; the paper
// names Hermite for its Gaussian inputs): Phi_n(s) = sqrt(2n+1) P_n(s) on
// s in [-1,1], P_n by the three-term recurrence, products over dimensions.
// s[nq][d] are the nodes mapped to [-1,1]; phi[nq][P].
int oc_gpc_basis(int d, int degree, int nq, const double* s, double* phi) {
  std::vector<std::vector<int>> mi;
  multi_indices(d, degree, mi);
  int P = (int)mi.size();
  for (int j = 0; j < nq; ++j) {
    std::vector<std::vector<double>> leg(d, std::vector<double>(degree + 1));
    for (int t = 0; t < d; ++t) {
      double x = s[(long long)j * d + t];
      leg[t][0] = 1.0;
      if (degree >= 1) leg[t][1] = x;
      for (int n = 1; n < degree; ++n)
        leg[t][n + 1] = ((2.0 * n + 1.0) * x * leg[t][n] - n * leg[t][n - 1]) / (n + 1.0);
    }
    for (int al = 0; al < P; ++al) {
      double v = 1.0;
      for (int t = 0; t < d; ++t) {
        int n = mi[al][t];
        v *= std::sqrt(2.0 * n + 1.0) * leg[t][n];
      }
      phi[(long long)j * P + al] = v;
    }
  }
  return 0;
}

// The same basis with a polynomial family per run: family 0 Legendre as
// above (s in [-1,1]), family 1 orthonormal probabilists' Hermite
// He_n(x) / sqrt(n!) for standard-normal x (the paper's Gaussian inputs,
// Sec. 2.3-2.4); products over dimensions in the same graded order.
int oc_gpc_basis_family(int d, int degree, int family, int nq, const double* s, double* phi) {
  if (family == 0) return oc_gpc_basis(d, degree, nq, s, phi);
  if (family != 1) return -1;
  std::vector<std::vector<int>> mi;
  multi_indices(d, degree, mi);
  int P = (int)mi.size();
  for (int j = 0; j < nq; ++j)
    for (int al = 0; al < P; ++al) {
      double v = 1.0;
      for (int t = 0; t < d; ++t) {
        int n = mi[al][t];
        double fact = 1.0;
        for (int k = 2; k <= n; ++k) fact *= k;
        v *= hermite_e(n, s[(long long)j * d + t]) / std::sqrt(fact);
      }
      phi[(long long)j * P + al] = v;
    }
  return 0;
}

// Discrete projection (Sec. 2.3, Eq. coef_discrete) with gamma_alpha = 1 for
// the orthonormal basis: coef[alpha][c] = sum_j a_j Q_j(c) Phi_alpha(Z_j).
int oc_gpc_project(int nq, int P, long long ncell, const double* a, const double* Q,
                   const double* phi, double* coef) {
  for (int al = 0; al < P; ++al)
    for (long long c = 0; c < ncell; ++c) {
      double s = 0.0;
      for (int j = 0; j < nq; ++j)
        s += a[j] * Q[(long long)j * ncell + c] * phi[(long long)j * P + al];
      coef[(long long)al * ncell + c] = s;
    }
  return 0;
}

// Tangent-linear model: the discrete solver run on dual numbers.  duin[2][nz][3]
// holds d u_in / d theta_k for two parameters.  Returns, at time level n_steps,
// loss = sum_p |u(x_p) - u_target_p|^2, dloss[2] = its derivatives, the probe
// velocities u_probe[n_probe][3], and the final populations (values) in f.
int oc_tangent_run(const oc_params* p, const uint8_t* flags, const double* uin,
                   const double* duin, double* f, int n_steps, int n_probe,
                   const int32_t* probes, const double* u_target, double* loss,
                   double* dloss, double* u_probe) {
  if (check_params(p)) return -1;
  long long n = (long long)p->nx * p->ny * p->nz;
  std::vector<Dual> U(3 * p->nz), F((size_t)Q * n);
  for (int k = 0; k < 3 * p->nz; ++k) {
    U[k].v = uin[k];
    U[k].d[0] = duin[k];
    U[k].d[1] = duin[3 * p->nz + k];
  }
  for (long long k = 0; k < (long long)Q * n; ++k) F[k] = Dual(f[k]);
  run_steps<Dual>(p, flags, U.data(), F.data(), 0, n_steps);
  Dual J(0.0);
  for (int q = 0; q < n_probe; ++q) {
    long long c = probes[3 * q] + (long long)p->nx * (probes[3 * q + 1] + (long long)p->ny * probes[3 * q + 2]);
    Dual r(0.0), j[3];
    for (int i = 0; i < Q; ++i) {
      const Dual& fi = F[(long long)i * n + c];
      r += fi;
      j[0] += Dual((double)CX[i]) * fi;
      j[1] += Dual((double)CY[i]) * fi;
      j[2] += Dual((double)CZ[i]) * fi;
    }
    for (int a = 0; a < 3; ++a) {
      Dual u = j[a] / r;
      if (u_probe) u_probe[3 * q + a] = u.v;
      Dual e = u - Dual(u_target[3 * q + a]);
      J += e * e;
    }
  }
  *loss = J.v;
  dloss[0] = J.d[0];
  dloss[1] = J.d[1];
  for (long long k = 0; k < (long long)Q * n; ++k) f[k] = F[k].v;
  return 0;
}

}  // extern "C"
