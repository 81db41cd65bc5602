// sclbm_internal.h -- structures shared by the host side of libsclbm and its
// CUDA kernels.  Not part of the public ABI (include/sclbm.h is).
#pragma once

#include <stddef.h>
#include <stdint.h>
#include <vector_types.h>

#include <string>
#include <vector>

#include "../../include/sclbm.h"

namespace sclbm {

constexpr int kQ = 19;
constexpr int kMaxDomains = SC_MAX_DOMAINS;
constexpr int kMaxGpcP = 28;     // largest gPC basis the reduction kernel keeps in registers
// The basis sizes the in-place precisions' reduction is compiled for: the gPC
// basis size P padded up to an even size of at least 4 while P <= 12 (one
// thread a cell sums two terms at a time), to a multiple of 4 above (two
// threads a cell, each half the term pairs).  It is also the row length of
// the pair table abf.
constexpr int gpc_pair_pad(int P) {
  return P <= 0 ? 0 : P <= 4 ? 4 : P <= 12 ? (P + 1) / 2 * 2 : (P + 3) / 4 * 4;
}
static_assert(kMaxGpcP % 4 == 0, "the pair table's rows split into two halves of term pairs");
constexpr int kRun = 256;        // cells per run of the TMA-staged kernels; the row pitch is a multiple

// Link word per cell (64 bits).  Bits 2i, 2i+1 give the kind of link i, the
// rule that supplies f_i from the source x - c_i:
//   kStream  in-domain fluid source, no periodic wrap
//   kBounce  bounce-back (solid source, wall face, two walls, two free-slip faces)
//   kMoving  bounce-back plus the moving-wall term of an inflow face
//   kSpecZ   specular reflection at a free-slip z face from a fluid in-plane source
// Links of any other kind (outflow, free slip on an x/y face, periodic wraps
// of fluid sources, outflow + free-slip edges) carry a nonzero placeholder
// kind and mark the cell kLinkComplex: such cells take the general path.
using LinkWord = unsigned long long;
constexpr int kStream = 0, kBounce = 1, kMoving = 2, kSpecZ = 3;
constexpr LinkWord kLinkSolid = 1ull << 40;    // the cell itself is solid
constexpr LinkWord kLinkOutlet = 1ull << 41;   // fluid cell on an OUTFLOW +x face
constexpr LinkWord kLinkComplex = 1ull << 42;  // some link needs the general rules
constexpr LinkWord kLinkVel = 1ull << 43;      // some link carries the moving-wall term
constexpr LinkWord kLinkKinds = (1ull << 38) - 1ull;
// Cells without these bits take the fast path.
constexpr LinkWord kLinkSlow = kLinkSolid | kLinkOutlet | kLinkComplex;

#ifdef __CUDACC__
__host__ __device__
#endif
inline int link_kind(LinkWord w, int i) { return (int)((w >> (2 * i)) & 3ull); }

// Per-cell class byte read by the bulk loops (one byte, so the decision for
// the next cell costs little L2 traffic); the link word is read only where
// kClsWall is set.
constexpr uint8_t kClsSkip = 1;      // solid, or listed for the general boundary path
constexpr uint8_t kClsWall = 2;      // some link does not stream
constexpr uint8_t kClsMoveSpec = 4;  // some link is a moving wall or specular

// Device error word bits.
constexpr unsigned kErrDiverged = 1u;
constexpr unsigned kErrTimeout = 2u;

// Listed cells (outlet plane, free-slip x/y faces, periodic wraps) carry their
// link rules compiled into offsets on the host, so the odd AA level updates
// them with two rounds of independent loads.  Offsets are element offsets
// from the node's population base (slot * pitch + cell) or, for outflow
// pulls, from the node's outflow plane ((z * ny + y) * 5 + k).
constexpr int kOutletPops = 5;                         // f*_j with c_jx = -1
constexpr int kOutletCopies = 4;                       // extra deliveries each
struct alignas(16) ListedLinks {
  int32_t src[kQ];                                     // pull source of link i
  int32_t dst[kQ];                                     // delivery of f*_j, -1: leaves
  int32_t extra[kOutletPops * kOutletCopies];          // outlet copies of f*_{2,8,10,12,14}, -1: none
  uint32_t bout_mask;                                  // bit i: src[i] is in the outflow plane
  uint32_t pull_move;                                  // bit i: pull of link i adds 6 w_i (c_i.u) r
  uint32_t push_move;                                  // bit j: delivery of f*_j adds the term of opp(j)
  int32_t z;                                           // the cell's layer (inflow table row)
  uint32_t pad[2];
};
static_assert(sizeof(ListedLinks) == 256, "ListedLinks is 256 bytes");
// On the device the records are stored transposed, word w of listed cell li at
// ltab[w * lstride + li], so a warp over consecutive listed cells reads each
// word coalesced.
constexpr int kListedWords = (int)(sizeof(ListedLinks) / 4);
constexpr int kWordSrc = 0, kWordDst = kQ, kWordExtra = 2 * kQ;
constexpr int kWordBoutMask = 2 * kQ + kOutletPops * kOutletCopies;
constexpr int kWordPullMove = kWordBoutMask + 1, kWordPushMove = kWordBoutMask + 2;
constexpr int kWordZ = kWordBoutMask + 3;

// Inflow factor of one time level: the node's inflow table u(z) is turned
// about z by the level's direction offset delta and scaled by r s, the
// start-up ramp times the level's speed factor.  The moving-wall term takes
// the turned velocity and multiplies by `scale` last (steady inflow:
// cos_d = 1, sin_d = 0, scale = r).
template <class T>
struct Wind {
  T cos_d, sin_d, scale;
};

// Cell flags of the host geometry: 0 fluid, 1 solid (buildings), kFlagMantle
// beyond the mantle of a circular domain (links into it take the velocity rule).
constexpr uint8_t kFlagMantle = 2;

// Per-domain view handed to the kernels (plain pointers into the workspace).
struct DevDomain {
  int nx, ny, nz, nodes;
  long long ncell;
  int bc[6];
  const uint8_t* flags;     // [ncell]
  const LinkWord* link;     // [ncell]
  const uint8_t* cls;       // [ncell] kCls* bits: what the bulk loops need to know
  const float4* uin_f;      // [nodes][nz] (ux, uy, uz, 0)
  const double* uin_d;      // [nodes][nz][3]
  long long pitch;          // population row stride (elements), multiple of kRun
  void* g;                  // [nodes][19][pitch] storage (AA) or FP64 array A
  void* g2;                 // FP64 plain: array B, else null
  float* bout;              // [nodes][nz*ny][5] outflow plane (AA only)
  const int32_t* bcell;     // [nb] fluid cells with a boundary link or on the outlet (ascending)
  const int32_t* ltab;      // [kListedWords][lstride] their compiled link rules (transposed records)
  long long lstride;
  long long nb;
  long long tiles_x, tiles_y, tiles_z, tiles_per_node;
  long long tile_begin;     // first global tile of this domain
  long long bitem_begin;    // first global boundary item (node-major) of this domain
  long long runs_per_node;  // pitch / kRun
  long long run_begin;      // first global run of this domain
};

struct StepParams {
  int n_domains;
  DevDomain dom[kMaxDomains];
  float tau0;
  float smag18c2;             // 18 C_S^2
  double tau0_d, smag18c2_d;
  int csmag_on;
  unsigned long long n_host;  // time level of the state (observables, persistent start)
  // Inflow factors of the launch: wp at arrival level n (odd-level pulls,
  // observables of level n), wq at level n + 1 (odd-level and FP64 pushes).
  // A persistent launch runs only levels over which both stay fixed.
  Wind<float> wp, wq;
  Wind<double> wpd, wqd;
  unsigned int* err;          // latched error bits
  long long total_tiles;       // bulk tiles of all domains and nodes
  long long total_bitems;      // boundary (node, cell) items of all domains
  long long total_runs;        // runs of kRun cells of all domains and nodes
  int tma;                     // bulk kernels staged through shared memory by TMA
  int odd85, even85;           // per-thread odd / even kernels sized for 3 blocks (85 registers)
  int even_pair;               // 16-bit storage, BGK: even level two x-adjacent cells per thread,
                               // kernel sized for 2 or 3 resident blocks (0: one cell per thread)
  int bx, by, bz, order;
  // persistent mode
  unsigned int* bar_count;
  unsigned int* bar_gen;
  long long spin_limit;
  int never_arrive;
  int n_steps;                // persistent: steps per launch
  int plain_node;             // FP64 plain path: node advanced by this launch
  int plain_domain;
};

// ------------------------------------------------------------ host numerics
// Implemented in host_numerics.cpp (IEEE double, no FP contraction).
int hn_quadrature(int rule, int d, int level, const double* lo, const double* hi,
                  std::vector<double>& Z, std::vector<double>& w);
int hn_geometry(const sc_domain_desc& D, std::vector<uint8_t>& flags);
// Circular domain (disk_radius > 0): every column whose centre (x + 1/2,
// y + 1/2) lies more than disk_radius from (nx / 2, ny / 2) becomes
// kFlagMantle in all layers.
void hn_mark_mantle(const sc_domain_desc& D, std::vector<uint8_t>& flags);
int hn_probe_columns(const sc_domain_desc& D, const uint8_t* flags, int n, int32_t* xy);
int hn_probe_points(const sc_domain_desc& D, const uint8_t* flags, int n, int32_t* xyz);
void hn_link_words(const sc_domain_desc& D, const uint8_t* flags, std::vector<LinkWord>& link);
void hn_boundary_cells(const std::vector<LinkWord>& link, std::vector<int32_t>& cells);
void hn_cell_classes(const std::vector<LinkWord>& link, std::vector<uint8_t>& cls);
void hn_listed_links(const sc_domain_desc& D, const uint8_t* flags, const std::vector<LinkWord>& link,
                     const std::vector<int32_t>& cells, long long pitch, std::vector<ListedLinks>& tab);
void hn_inflow(int nz, double u_ref, double xi, double alpha, double H, double theta_deg, double* uin,
               int profile = 0, double z0 = 0.1);
int hn_gpc_size(int d, int degree);
void hn_gpc_basis(int d, int degree, const double* s /*[d]*/, double* phi /*[P]*/, bool hermite = false);
double hn_ramp(int ramp_steps, long long m);
// Time-varying inflow (Sec. 2.2, Sec. 3): n targets of speed factor s_k and
// direction offset d_k (degrees), target 0 from level 0, target k >= 1
// reached over `interp` levels from level k * per on, the last one held.
// hn_series_unwrap makes the directions continuous (each move along the
// shorter arc, a half turn clockwise); hn_series_at takes those.
void hn_series_unwrap(int n, const double* dir_deg, double* unwrapped);
void hn_series_at(int n, const double* speed, const double* unwrapped, long long per, long long interp,
                  long long m, double* s, double* d);
// The first level after m at which the inflow factor (ramp r(m) over
// ramp_steps levels times the series) may differ from its value at m.
long long hn_wind_next_change(int ramp_steps, int n, long long per, long long interp, long long m);

// ------------------------------------------------------------ kernel launchers
// Implemented in lbm_kernels.cu.  All return cudaError_t as int.
int launch_aa_step(const StepParams& P, int precision, void* stream, int parity);
int launch_aa_persistent(const StepParams& P, int precision, void* stream, int grid);
int launch_plain_step(const StepParams& P, unsigned long long n, void* stream);
int aa_persistent_max_grid(const StepParams& P, int precision, int* grid);
// The same step launchers with the recursive regularized collision
// (lbm_kernels_rr.cu).
namespace rr {
int launch_aa_step(const StepParams& P, int precision, void* stream, int parity);
int launch_aa_persistent(const StepParams& P, int precision, void* stream, int grid);
int launch_plain_step(const StepParams& P, unsigned long long n, void* stream);
int aa_persistent_max_grid(const StepParams& P, int precision, int* grid);
}  // namespace rr
int launch_init_equilibrium(const StepParams& P, int precision, void* stream);
struct MomentArgs {
  int domain;
  const double* ab;        // [nq][stride] : a_j then a_j * Phi_alpha(Z_j)
  const float4* abf;       // [nq][gpc_pair_pad(P) / 2] : a_j * Phi_alpha(Z_j) of terms (a, a + 1) as
                           // (hi_a, hi_a+1, lo_a, lo_a+1) floats, hi + lo to 48 bits; zero pad terms
  int stride;              // row length of ab (basis size of the configuration + 1)
  int nq, P;               // P: coefficients to produce (0 = none)
  double wsum;
  double* mean;
  double* stdev;
  double* coef;            // [P][ncell] or null
  const int32_t* probes;   // device [n_p][2]
  int n_p;
  double* prof;            // device
  float* prof_nodes;       // device or null
  const double* avg;       // [nq][ncell] time-accumulated |u|, or null for the current |u|
  double avg_scale;        // 1 / samples
  int raw;                 // 1: write the sums S1, S2 (and gPC sums) into mean / stdev / coef
  int accumulate;          // with raw: the sums start from the values already in mean / stdev / coef
};
int launch_moments(const StepParams& P, int precision, const MomentArgs& A, void* stream);
int launch_export(const StepParams& P, int precision, int domain, int node, double* d_f,
                  float* d_u, void* stream);
// Adds |u| of every node of a domain at the current time level to avg[nq][ncell].
int launch_average_add(const StepParams& P, int precision, int domain, double* avg, void* stream);
// mean = s1 / wsum, stdev = sqrt(max(s2 / wsum - mean^2, 0)), n cells.
int launch_finalize_moments(const double* s1, const double* s2, double wsum, double* mean, double* stdev,
                            long long n, void* stream);
// out[k] = s * in[k], k < n.
int launch_scale(const double* in, double s, double* out, long long n, void* stream);
// Q-criterion of a velocity field u[3][ncell] of a domain into q[ncell].
int launch_qcriterion(const StepParams& P, int domain, const float* u, float* q, void* stream);
// Confidence bounds from the gPC surrogate (quantiles.cu): per listed cell
// the k-th smallest of sum_a coef[a][cell] phi[m][a] over the M samples.
int launch_gpc_quantiles(const double* coef, long long ncell, int P, const int32_t* cells, int n_cells,
                         const double* phi, int M, const int32_t* kidx, int nq, double* out, void* stream);
int launch_check(const StepParams& P, int precision, unsigned long long* d_count, void* stream);

// Adjoint of one node's time step (adjoint.cu).
struct AdjArgs {
  int domain;
  const float4* uin;      // [nz] inflow of the node
  const float4* du;       // [2][nz] d u_in / d u_ref, d u_in / d alpha
  const int32_t* probes;  // [n_probes][3]
  const double* target;   // [n_probes][3]
  double* u_probe;        // [n_probes][3]
  int n_probes;
  double* accum;          // [0] loss, [1] dJ/du_ref, [2] dJ/dalpha
  const int32_t* lmap;    // [ncell]: listed cell -> index in the listed-cell array
};
int launch_adj_forward(const StepParams& P, const AdjArgs& A, const float* src, float* dst, float r1,
                       void* stream);  // r1: ramp r(n + 1) of the step's pushes
int launch_adj_loss(const StepParams& P, const AdjArgs& A, const float* f, float* lam, void* stream);
int launch_adj_step(const StepParams& P, const AdjArgs& A, const float* f, const float* lam_next, float* lam,
                    float r1, void* stream);
int launch_fill_zero(float* p, long long n, void* stream);
int launch_adj_listed_map(const StepParams& P, int domain, int32_t* lmap, void* stream);

}  // namespace sclbm
