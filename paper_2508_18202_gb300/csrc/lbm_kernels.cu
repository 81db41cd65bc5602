// lbm_kernels.cu -- CUDA kernels of libsclbm for sm_103a (GB300).
//
// Stream-collide of the D3Q19 lattice Boltzmann equation (arXiv:2508.18202
// Sec. 2.2, Eq. deterministicLBE) with BGK collision and the Smagorinsky
// effective relaxation time (Eqs. tauEff, turbVisc), for every collocation
// node of every domain of an ensemble.  The observables read from these
// populations (the quadrature / gPC reductions of Sec. 2.3 among them) are
// in observables.cu.
//
// Layout (structure of arrays, x fastest): population i of node j of a
// domain lives at g[(j*19 + i)*pitch + c], c = x + nx*(y + ny*z), with the
// row pitch a multiple of 256 cells and guard zones before and after the
// array.  The in-place precisions store g_i = f_i - w_i (the shift keeps the
// FP32/BF16/FP16 mantissa for the deviation from rest) and advance with the
// AA access pattern: at an even time level a cell reads its own 19 slots and
// writes the post-collision values back to the opposite slots of the same
// cell; at an odd level it pulls f_i from slot opp(i) of the upstream
// neighbour x - c_i and pushes f*_i into slot i of the downstream neighbour
// x + c_i.  Every slot is then read and written by exactly one thread per
// step, so one array suffices (152 B per fluid cell update in FP32).
//
// Every fluid cell carries a 64-bit link word whose 2-bit kind per direction
// selects the rule of link i in the bulk kernels: stream from the neighbour,
// bounce-back into the own slot (solid source, wall face), the moving-wall
// rule of an inflow face or the circular mantle (own slot plus the wall
// term), or specular reflection at a free-slip z face (the in-plane
// neighbour's slot).  Cells with any other link (outflow, free slip on an x
// or y face, periodic wraps) are listed on the host, their rules compiled
// into per-cell offset records, and updated by the listed blocks of the same
// launch.  Together the kinds and the records realise the per-link rules of
// the pull formulation:
//   source inside and solid            -> bounce-back
//   one face crossed: BOUNCE_BACK      -> bounce-back
//                     VELOCITY         -> bounce-back + 6 w_i (c_i . u_in(z)) r(t)
//                     FREE_SLIP        -> specular reflection from the in-plane
//                                         neighbour (bounce-back if it is solid)
//                     OUTFLOW (+x)     -> copy of f*_i from the transverse
//                                         neighbour on the outlet plane (own
//                                         value if that cell is solid)
//   two faces crossed: any wall        -> bounce-back; else any inflow ->
//                                         moving wall; else the cell's own f*
//                                         reflected across each free-slip face.
// The outflow copy reads a neighbour's post-collision value that the AA
// odd step overwrites in place, so even steps also save the five f*_i with
// c_ix = -1 of every outlet cell into a small per-node plane (bout) that the
// odd step reads.
//
// Two forms of the bulk kernels: per-thread loads (one cell per thread, a
// z-slab per thread), and TMA-staged ones in which a CTA streams runs of 256
// consecutive cells through a 4-stage shared-memory pipeline filled by 1-D
// bulk copies (cp.async.bulk + mbarrier).  The even level stores back with
// bulk copies too; the odd level loads the 19 shifted row windows (widened
// by 16 bytes on each side for alignment) and stores per thread.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "lbm_device.cuh"
#include "sclbm_internal.h"

namespace sclbm {
namespace {

// ------------------------------------------------------------ per-cell updates
// Even time level: a fluid cell reads its own 19 slots and writes the
// post-collision populations to the opposite slots; outlet cells also save
// their five populations with c_x = -1 into the outflow plane.
template <class S, bool CG>
__device__ __forceinline__ void cell_even(const StepParams& P, const DevDomain& D,
                                          const Node<S>& N, LinkWord lw, int y, int z,
                                          long long idx) {
  using T = typename Store<S>::C;
  const int pc = (int)D.pitch;
  S* base = N.g + idx;
  T g[kQ];
#pragma unroll
  for (int i = 0; i < kQ; ++i) g[i] = LD<S, CG>(base + i * pc);
  collide_p<T, true>(P, g);
#pragma unroll
  for (int i = 0; i < kQ; ++i) Store<S>::st(base + OPP(i) * pc, g[i]);
  if (lw & kLinkOutlet) save_outlet<S>(D, N, y, z, g);
}

// ------------------------------------------------------------ step driver
// A tile is a block_x * block_y patch of one x-y plane range, slab_z deep,
// of one node of one domain.  Decoded once per block (32-bit arithmetic; tile
// counts stay below 2^31) and shared with the block's threads.
struct TileRef {
  int d, node, x, y, z0, z1;
  bool valid;
};

struct TileHead {
  int d, node, x0, y0, z0;
};

__device__ __forceinline__ TileHead decode_tile_head(const StepParams& P, unsigned t) {
  TileHead H;
  int d = 0;
  for (int k = 1; k < P.n_domains; ++k)
    if ((long long)t >= P.dom[k].tile_begin) d = k;
  const DevDomain& D = P.dom[d];
  const unsigned local = t - (unsigned)D.tile_begin;
  const unsigned nodes = (unsigned)D.nodes, tpn = (unsigned)D.tiles_per_node;
  unsigned ct;
  if (P.order == 0) {
    H.node = (int)(local % nodes);
    ct = local / nodes;
  } else {
    H.node = (int)(local / tpn);
    ct = local % tpn;
  }
  const unsigned tx = (unsigned)D.tiles_x, txy = tx * (unsigned)D.tiles_y;
  const unsigned tz = ct / txy, rem = ct - tz * txy;
  const unsigned ty = rem / tx;
  H.d = d;
  H.x0 = (int)(rem - ty * tx) * P.bx;
  H.y0 = (int)ty * P.by;
  H.z0 = (int)tz * P.bz;
  return H;
}

// Block-wide decode of tile t: thread (0,0) decodes, the block reads it.
// CPT: x-adjacent cells per thread (the tile is then CPT * blockDim.x cells
// wide, P.bx = CPT * blockDim.x); R.x is the thread's first cell.
template <int CPT = 1>
__device__ __forceinline__ TileRef block_tile(const StepParams& P, unsigned t) {
  __shared__ TileHead s_head;
  if (threadIdx.x == 0 && threadIdx.y == 0) s_head = decode_tile_head(P, t);
  __syncthreads();
  const TileHead H = s_head;
  TileRef R;
  const DevDomain& D = P.dom[H.d];
  R.d = H.d;
  R.node = H.node;
  R.x = H.x0 + CPT * threadIdx.x;
  R.y = H.y0 + threadIdx.y;
  R.z0 = H.z0;
  R.z1 = min(H.z0 + P.bz, D.nz);
  R.valid = R.x < D.nx && R.y < D.ny;
  return R;
}

// Even level over the z-slab of a tile.  The link word of the next cell is
// loaded one cell ahead so the population loads do not wait on it.
// LISTED_APART: listed cells (outlet, general boundary) are left to the
// leading blocks of the launch, so the bulk path carries no outlet save.
// Even level, bulk cells of a z-run: n cells, plane apart, from base (slot 0
// of the first cell) and their class bytes cp.  Only these scalars stay live
// in the loop; the next cell's class byte is loaded one cell ahead.
template <class S, bool CG>
__device__ __forceinline__ void even_run(const StepParams& P, S* base, const uint8_t* cp, int pc, int plane,
                                         int n) {
  using T = typename Store<S>::C;
  uint8_t next = ld_keep(cp);
  for (int k = 0; k < n; ++k, base += plane, cp += plane) {
    const uint8_t cls = next;
    if (k + 1 < n) next = ld_keep(cp + plane);
    if (cls & kClsSkip) continue;
    T g[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) g[i] = LD<S, CG>(base + i * pc);
    collide_p<T, true>(P, g);
#pragma unroll
    for (int i = 0; i < kQ; ++i) Store<S>::st(base + OPP(i) * pc, g[i]);
  }
}

// LISTED_APART: listed cells (outlet, general boundary) are left to the
// leading blocks of the launch, so the bulk path carries no outlet save.
template <class S, bool CG, bool LISTED_APART>
__device__ __forceinline__ void even_tile(const StepParams& P, const TileRef& R) {
  if (!R.valid) return;
  const DevDomain& D = P.dom[R.d];
  const int plane = D.nx * D.ny;
  const int idx0 = R.x + D.nx * (R.y + D.ny * R.z0);
  if (LISTED_APART) {
    even_run<S, CG>(P, reinterpret_cast<S*>(D.g) + (long long)R.node * kQ * D.pitch + idx0, D.cls + idx0,
                    (int)D.pitch, plane, R.z1 - R.z0);
    return;
  }
  const Node<S> N = node_view<S>(D, R.node);
  int idx = idx0;
  for (int z = R.z0; z < R.z1; ++z, idx += plane) {
    const LinkWord lw = __ldg(D.link + idx);
    if (lw & kLinkSolid) continue;
    cell_even<S, CG>(P, D, N, lw, R.y, z, idx);
  }
}

// Odd level over the z-slab of a tile.  A warp whose cells are all interior
// (or skipped) takes the plain streaming form; a warp with any wall, inflow
// or lid link takes the link-kind form for all its cells, so neither
// diverges.  The next cell's link word is loaded one cell ahead.
// ROT: the launch's factors may turn the inflow (a series); without it the
// table velocity is read once and only scaled, which keeps the 64-register
// kernels free of the second velocity (the host sends launches that turn to
// the kernels compiled with ROT).
template <class S, bool CG, bool ROT>
__device__ __forceinline__ void odd_bulk_tile(const StepParams& P, const TileRef& R) {
  using T = typename Store<S>::C;
  if (!R.valid) return;
  const DevDomain& D = P.dom[R.d];
  const int sy = D.nx, sz = D.nx * D.ny;
  const int idx0 = R.x + D.nx * (R.y + D.ny * R.z0);
  const int pc = (int)D.pitch;
  S* base = reinterpret_cast<S*>(D.g) + (long long)R.node * kQ * D.pitch + idx0;
  const LinkWord* lp = D.link + idx0;
  const float4* uinf = D.uin_f + (long long)R.node * D.nz;
  const double* uind = D.uin_d + (long long)R.node * D.nz * 3;
  LinkWord next = ld_keep(lp);
  for (int z = R.z0; z < R.z1; ++z, base += sz, lp += sz) {
    const LinkWord lw = next;
    if (z + 1 < R.z1) next = ld_keep(lp + sz);
    const bool interior = __all_sync(__activemask(), lw == 0 || (lw & kLinkSlow));
    if (lw & kLinkSlow) continue;   // solid, outlet or general-boundary cell
    T g[kQ];
    if (interior) {
      // The 19 neighbour offsets are loop-invariant; hoisted out of the z
      // loop they would hold 19 registers and spill at the 64-register
      // budget.  Hiding the strides from the optimiser per cell makes each
      // offset one multiply-add at its load or store instead.
      int pcv = pc, syv = sy, szv = sz;
      asm volatile("" : "+r"(pcv), "+r"(syv), "+r"(szv));
#pragma unroll
      for (int i = 0; i < kQ; ++i)
        g[i] = LD<S, CG>(base + (OPP(i) * pcv - (CX(i) + CY(i) * syv + CZ(i) * szv)));
      collide_p<T, true>(P, g);
      asm volatile("" : "+r"(pcv), "+r"(syv), "+r"(szv));
#pragma unroll
      for (int j = 0; j < kQ; ++j) Store<S>::st(base + (j * pcv + (CX(j) + CY(j) * syv + CZ(j) * szv)), g[j]);
    } else {
      Node<S> N;
      N.g = nullptr;
      N.bout = nullptr;
      N.uinf = uinf;
      N.uind = uind;
      T ux, uy, uz;
      wall_velocity<S, ROT>(N, lw, z, wind_pull<T>(P), ux, uy, uz);
      fast_pull<S, CG>(base, lw, pc, sy, sz, ux, uy, uz, wind_pull<T>(P).scale, g);
      collide_p<T, true>(P, g);
      if constexpr (ROT) wall_velocity<S>(N, lw, z, wind_push<T>(P), ux, uy, uz);
      fast_push<S>(base, lw, pc, sy, sz, ux, uy, uz, wind_push<T>(P).scale, g);
    }
  }
}

// Listed (node, cell) items: item -> domain, node and cell index.
__device__ __forceinline__ int decode_bitem(const StepParams& P, long long item, int* node, long long* idx) {
  int d = 0;
  for (int k = 1; k < P.n_domains; ++k)
    if (item >= P.dom[k].bitem_begin) d = k;
  const DevDomain& D = P.dom[d];
  const long long k = item - D.bitem_begin;
  *node = (int)(k / D.nb);
  *idx = __ldg(D.bcell + (k % D.nb));
  return d;
}

// Listed cells of the odd level: one thread per (node, listed cell), from
// the compiled link rules (one round of table loads, one of population
// loads).
template <class S, bool CG, bool ROT>
__device__ __forceinline__ void odd_boundary_item(const StepParams& P, long long item) {
  using T = typename Store<S>::C;
  if (item >= P.total_bitems) return;
  int d = 0;
  for (int k = 1; k < P.n_domains; ++k)
    if (item >= P.dom[k].bitem_begin) d = k;
  const DevDomain& D = P.dom[d];
  const long long k = item - D.bitem_begin;
  const int node = (int)(k / D.nb);
  const long long li = k % D.nb;
  // every load below depends only on the record's words, so the cell costs
  // two rounds of memory latency (words, then populations and inflow)
  const ListedRef L = listed_ref(D, li);
  const Node<S> N = node_view<S>(D, node);
  const int z = L.word(kWordZ);
  T ux, uy, uz;
  if constexpr (ROT) inflow_velocity<S>(N, z, wind_pull<T>(P), ux, uy, uz);
  else table_velocity<S>(N, z, ux, uy, uz);
  T g[kQ];
  listed_pull<S, CG>(L, N.g, N.bout, ux, uy, uz, wind_pull<T>(P).scale, g);
  collide_p<T, true>(P, g);
  if constexpr (ROT) inflow_velocity<S>(N, z, wind_push<T>(P), ux, uy, uz);
  listed_push<S>(L, N.g, ux, uy, uz, wind_push<T>(P).scale, g);
}

// Listed cells of the even level (local update; outlet cells save their
// outflow plane values).
template <class S, bool CG>
__device__ __forceinline__ void even_boundary_item(const StepParams& P, long long item) {
  if (item >= P.total_bitems) return;
  int node;
  long long idx;
  const DevDomain& D = P.dom[decode_bitem(P, item, &node, &idx)];
  const int y = (int)((idx / D.nx) % D.ny);
  const int z = (int)(idx / ((long long)D.nx * D.ny));
  const LinkWord lw = __ldg(D.link + idx);
  cell_even<S, CG>(P, D, node_view<S>(D, node), lw, y, z, idx);
}

// Blocks of an even or odd launch that carry the listed (node, cell) items:
// ceil(items / threads) of them, spread evenly over the grid (every q-th
// block) so their long-latency work overlaps the bulk tiles throughout the
// launch.  Returns true for a listed block, with its rank among the listed
// blocks in *index, else the rank among the bulk blocks (the tile index).
__device__ __forceinline__ bool block_role(const StepParams& P, unsigned* index) {
  const long long threads = (long long)blockDim.x * blockDim.y;
  const unsigned listed = (unsigned)((P.total_bitems + threads - 1) / threads);
  const unsigned b = blockIdx.x;
  if (listed == 0) {
    *index = b;
    return false;
  }
  const unsigned q = gridDim.x / listed;  // >= 1: the grid is tiles + listed blocks
  if (b % q == 0 && b / q < listed) {
    *index = b / q;
    return true;
  }
  *index = b - min((b + q - 1) / q, listed);
  return false;
}

// Even time level for every (domain, node, tile).  The even level carries no
// boundary term, so its launches have no time-dependent parameter.
// MINB: resident blocks of 256 threads the register budget is sized for
// (4: at most 64 registers; 3: at most 85), chosen by the autotuner; the
// odd kernel with MINB = 3 is also the one that turns the inflow.
template <class S, int MINB>
__global__ void __launch_bounds__(256, MINB) aa_even_kernel(const __grid_constant__ StepParams P) {
  unsigned k;
  if (block_role(P, &k)) {
    const long long item = k * (long long)(blockDim.x * blockDim.y) + threadIdx.y * blockDim.x + threadIdx.x;
    even_boundary_item<S, false>(P, item);
    return;
  }
  even_tile<S, false, true>(P, block_tile(P, k));
}

#ifndef SCLBM_RR_UNIT
// Even level with 16-bit storage, two x-adjacent cells per thread (the first
// at an even x of a domain with even nx, so each pair of populations is one
// aligned 32-bit word): the run of pairs of a z-slab.  A pair whose cells
// are both bulk cells moves its populations as 32-bit words and collides in
// the two lanes of the packed FP32x2 operations; a pair with one bulk cell
// (the other solid or listed, and updated by the listed blocks) loads and
// stores that cell alone, in both lanes.  The class bytes of the next pair
// are loaded one cell ahead.
template <class S>
__device__ __forceinline__ void even_run_pair(const StepParams& P, S* base, const uint8_t* cp, int pc, int plane,
                                              int n) {
  uint16_t next = ld_keep(reinterpret_cast<const uint16_t*>(cp));
  for (int k = 0; k < n; ++k, base += plane, cp += plane) {
    const unsigned cls = next;
    if (k + 1 < n) next = ld_keep(reinterpret_cast<const uint16_t*>(cp + plane));
    const bool a = !(cls & kClsSkip), b = !((cls >> 8) & kClsSkip);
    if (!(a || b)) continue;
    float2 g[kQ];
    if (a && b) {
#pragma unroll
      for (int i = 0; i < kQ; ++i) g[i] = Pair16<S>::unpack(*reinterpret_cast<const uint32_t*>(base + i * pc));
    } else {
      const S* c = a ? base : base + 1;
#pragma unroll
      for (int i = 0; i < kQ; ++i) g[i] = p2dup(Store<S>::ld(c + i * pc));
    }
    collide_pair(g, P.tau0, P.smag18c2, P.csmag_on);
    if (a && b) {
#pragma unroll
      for (int i = 0; i < kQ; ++i) *reinterpret_cast<uint32_t*>(base + OPP(i) * pc) = Pair16<S>::pack(g[i]);
    } else {
      S* c = a ? base : base + 1;
#pragma unroll
      for (int i = 0; i < kQ; ++i) Store<S>::st(c + OPP(i) * pc, g[i].x);
    }
  }
}

// Even time level with 16-bit storage, two cells per thread (launched with
// the tiling of pair_tiling: tiles 2 * blockDim.x cells wide); the listed
// cells ride in blocks spread over the grid as in aa_even_kernel.  MINB:
// resident blocks of 256 threads (2: no spills at 110 registers; 3: 80
// registers, a few bytes spilled, half as many warps again in flight).
template <class S, int MINB>
__global__ void __launch_bounds__(256, MINB) aa_even_pair_kernel(const __grid_constant__ StepParams P) {
  unsigned k;
  if (block_role(P, &k)) {
    const long long item = k * (long long)(blockDim.x * blockDim.y) + threadIdx.y * blockDim.x + threadIdx.x;
    even_boundary_item<S, false>(P, item);
    return;
  }
  const TileRef R = block_tile<2>(P, k);
  if (!R.valid) return;
  const DevDomain& D = P.dom[R.d];
  const int plane = D.nx * D.ny;
  const int idx0 = R.x + D.nx * (R.y + D.ny * R.z0);
  even_run_pair<S>(P, reinterpret_cast<S*>(D.g) + (long long)R.node * kQ * D.pitch + idx0, D.cls + idx0,
                   (int)D.pitch, plane, R.z1 - R.z0);
}

#endif

// Odd time level in one launch: the listed blocks take the listed boundary
// cells (one thread per (node, cell)), the rest the tiles of bulk cells.  The
// two sets touch disjoint slots, so the long-latency boundary work overlaps
// with the bulk stream.  The inflow factors of the odd level n (pulls) and
// of level n + 1 (pushes) come with the launch.
template <class S, int MINB>
__global__ void __launch_bounds__(256, MINB) aa_odd_bulk_kernel(const __grid_constant__ StepParams P) {
  unsigned k;
  if (block_role(P, &k)) {
    const long long item = k * (long long)(blockDim.x * blockDim.y) + threadIdx.y * blockDim.x + threadIdx.x;
    odd_boundary_item<S, false, MINB != 4>(P, item);
    return;
  }
  odd_bulk_tile<S, false, MINB != 4>(P, block_tile(P, k));
}

// Odd time level, listed boundary cells alone (after the TMA odd kernel of the
// same level; the two touch disjoint slots).
template <class S>
__global__ void __launch_bounds__(256) aa_odd_boundary_kernel(const __grid_constant__ StepParams P) {
  const long long item = blockIdx.x * (long long)(blockDim.x * blockDim.y) + threadIdx.y * blockDim.x + threadIdx.x;
  odd_boundary_item<S, false, true>(P, item);
}

// ------------------------------------------------------------ TMA-staged bulk kernels
// Warp-specialised pipeline: 8 consumer warps (one cell of a 256-cell run per
// thread) compute from shared memory while one producer warp keeps kStages
// runs in flight with 1-D bulk copies.  full[s] completes when the bytes of
// stage s have landed (transaction count); empty[s] when the 8 consumer warps
// are done with it.
constexpr int kStages = 4;
constexpr int kConsumerWarps = kRun / 32;
constexpr int kTmaThreads = kRun + 32;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

constexpr long long kMbarPolls = 1LL << 22;  // bounded mbarrier polls (each may suspend briefly)

// Bounded wait for a phase of an mbarrier; latches kErrTimeout on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, const StepParams& P) {
  const long long limit = P.spin_limit < kMbarPolls ? P.spin_limit : kMbarPolls;
  for (long long k = 0; k < limit; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  atomicOr(P.err, kErrTimeout);
  return false;
}
__device__ __forceinline__ void bulk_load(void* sdst, const void* gsrc, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(sdst)),
      "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
               "r"(smem_u32(ssrc)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_le1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// A run is kRun consecutive cells of one node of one domain.
struct RunRef {
  int d, node;
  long long c0;
};
__device__ __forceinline__ RunRef decode_run(const StepParams& P, long long r) {
  RunRef R;
  int d = 0;
  for (int k = 1; k < P.n_domains; ++k)
    if (r >= P.dom[k].run_begin) d = k;
  const DevDomain& D = P.dom[d];
  const unsigned local = (unsigned)(r - D.run_begin);
  unsigned k;
  if (P.order == 0) {
    R.node = (int)(local % (unsigned)D.nodes);
    k = local / (unsigned)D.nodes;
  } else {
    R.node = (int)(local / (unsigned)D.runs_per_node);
    k = local % (unsigned)D.runs_per_node;
  }
  R.d = d;
  R.c0 = (long long)k * kRun;
  return R;
}

template <class S>
__device__ __forceinline__ S* run_rows(const StepParams& P, const RunRef& R) {
  const DevDomain& D = P.dom[R.d];
  return reinterpret_cast<S*>(D.g) + (long long)R.node * kQ * D.pitch + R.c0;
}

// Producer: after an expired wait, wait (bounded) for the loads still in
// flight before the CTA leaves.
__device__ __forceinline__ void drain_loads(uint64_t* full, long long from, long long to) {
  for (long long j = from; j < to; ++j)
    for (long long k = 0; k < kMbarPolls; ++k)
      if (mbar_try_wait(&full[j % kStages], (unsigned)((j / kStages) & 1))) break;
}

template <class S>
__device__ __forceinline__ void even_issue_load(const StepParams& P, long long r, S* stage, uint64_t* full) {
  const RunRef R = decode_run(P, r);
  const DevDomain& D = P.dom[R.d];
  const S* src = run_rows<S>(P, R);
  mbar_expect_tx(full, kQ * kRun * sizeof(S));
  for (int k = 0; k < kQ; ++k) bulk_load(stage + k * kRun, src + (long long)k * D.pitch, kRun * sizeof(S), full);
}

template <class S>
__device__ __forceinline__ void even_issue_store(const StepParams& P, long long r, const S* stage) {
  const RunRef R = decode_run(P, r);
  const DevDomain& D = P.dom[R.d];
  S* dst = run_rows<S>(P, R);
  for (int k = 0; k < kQ; ++k) bulk_store(dst + (long long)k * D.pitch, stage + k * kRun, kRun * sizeof(S));
  bulk_commit();
}

// Even level, TMA-staged.  The consumers collide in place in the stage
// (opposite rows) and the producer streams the stage back with bulk stores.
template <class S>
__global__ void __launch_bounds__(kTmaThreads, 2) aa_even_tma_kernel(const __grid_constant__ StepParams P) {
  using T = typename Store<S>::C;
  extern __shared__ __align__(128) unsigned char smem[];
  S* buf = reinterpret_cast<S*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)kStages * kQ * kRun * sizeof(S));
  uint64_t* empty = full + kStages;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    fence_mbar_init();
  }
  __syncthreads();
  const long long first = blockIdx.x, stride = gridDim.x;
  const long long iters = P.total_runs > first ? (P.total_runs - first + stride - 1) / stride : 0;
  if (warp == kConsumerWarps) {
    if (lane != 0) return;
    long long loaded = 0;
    for (; loaded < iters && loaded < kStages; ++loaded)
      even_issue_load<S>(P, first + loaded * stride, buf + (loaded % kStages) * kQ * kRun, &full[loaded % kStages]);
    for (long long k = 0; k < iters; ++k) {
      const int s = (int)(k % kStages);
      if (!mbar_wait(&empty[s], (unsigned)((k / kStages) & 1), P)) {
        drain_loads(full, k, loaded);
        break;
      }
      even_issue_store<S>(P, first + k * stride, buf + s * kQ * kRun);
      // refill the stage of iteration k - 1 once its stores have read it
      if (k >= 1 && loaded < iters) {
        bulk_wait_read_le1();
        const int sp = (int)((k - 1) % kStages);
        even_issue_load<S>(P, first + loaded * stride, buf + sp * kQ * kRun, &full[sp]);
        ++loaded;
      }
    }
    bulk_wait_all();
    return;
  }
  for (long long k = 0; k < iters; ++k) {
    const int s = (int)(k % kStages);
    if (!mbar_wait(&full[s], (unsigned)((k / kStages) & 1), P)) break;
    const RunRef R = decode_run(P, first + k * stride);
    const DevDomain& D = P.dom[R.d];
    S* sb = buf + s * kQ * kRun;
    const long long c = R.c0 + tid;
    T g[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) g[i] = Store<S>::ld(sb + i * kRun + tid);
    const LinkWord lw = c < D.ncell ? __ldg(D.link + c) : kLinkSolid;
    if (!(lw & kLinkSolid)) {
      collide_p<T, true>(P, g);
      if (lw & kLinkOutlet) {
        const int y = (int)((c / D.nx) % D.ny), z = (int)(c / ((long long)D.nx * D.ny));
        save_outlet<S>(D, node_view<S>(D, R.node), y, z, g);
      }
    }
    // solid and padding cells only swap their (never read) slots
#pragma unroll
    for (int i = 0; i < kQ; ++i) Store<S>::st(sb + OPP(i) * kRun + tid, g[i]);
    fence_async_smem();
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}

template <class S>
__device__ __forceinline__ void odd_issue_load(const StepParams& P, long long r, S* stage, uint64_t* full) {
  constexpr int PADE = 16 / sizeof(S);
  constexpr int RW = kRun + 2 * PADE;
  const RunRef R = decode_run(P, r);
  const DevDomain& D = P.dom[R.d];
  const S* src = run_rows<S>(P, R);
  const long long sy = D.nx, sz = (long long)D.nx * D.ny;
  mbar_expect_tx(full, kQ * RW * sizeof(S));
#pragma unroll
  for (int k = 0; k < kQ; ++k)
    bulk_load(stage + k * RW, src + (long long)k * D.pitch + CY(k) * sy + CZ(k) * sz - PADE, RW * sizeof(S), full);
}

// Odd level bulk cells, TMA-staged loads: row k of a run is read at the
// window c0 + off(k) - c_kx - PADE .. + kRun + 2 PADE (16-byte aligned), the
// value for cell t sits at t + PADE + c_kx.  Bounce-back links read the own
// slot from global memory; stores go straight to global memory.
template <class S>
__global__ void __launch_bounds__(kTmaThreads, 2) aa_odd_tma_kernel(const __grid_constant__ StepParams P) {
  using T = typename Store<S>::C;
  constexpr int PADE = 16 / sizeof(S);
  constexpr int RW = kRun + 2 * PADE;
  extern __shared__ __align__(128) unsigned char smem[];
  S* buf = reinterpret_cast<S*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)kStages * kQ * RW * sizeof(S));
  uint64_t* empty = full + kStages;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    fence_mbar_init();
  }
  __syncthreads();
  const long long first = blockIdx.x, stride = gridDim.x;
  const long long iters = P.total_runs > first ? (P.total_runs - first + stride - 1) / stride : 0;
  if (warp == kConsumerWarps) {
    if (lane != 0) return;
    long long loaded = 0;
    for (; loaded < iters && loaded < kStages; ++loaded)
      odd_issue_load<S>(P, first + loaded * stride, buf + (loaded % kStages) * kQ * RW, &full[loaded % kStages]);
    for (long long k = 0; loaded < iters; ++k) {
      const int s = (int)(k % kStages);
      if (!mbar_wait(&empty[s], (unsigned)((k / kStages) & 1), P)) {
        drain_loads(full, k, loaded);
        return;
      }
      odd_issue_load<S>(P, first + loaded * stride, buf + s * kQ * RW, &full[s]);
      ++loaded;
    }
    return;
  }
  for (long long k = 0; k < iters; ++k) {
    const int s = (int)(k % kStages);
    if (!mbar_wait(&full[s], (unsigned)((k / kStages) & 1), P)) break;
    const RunRef R = decode_run(P, first + k * stride);
    const DevDomain& D = P.dom[R.d];
    const S* sb = buf + s * kQ * RW;
    const long long c = R.c0 + tid;
    const LinkWord lw = c < D.ncell ? __ldg(D.link + c) : kLinkSlow;
    T g[kQ];
    const bool bulk = !(lw & kLinkSlow);
    if (bulk) {
#pragma unroll
      for (int i = 0; i < kQ; ++i) g[i] = Store<S>::ld(sb + OPP(i) * RW + tid + PADE + CX(OPP(i)));
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);  // stage s is no longer read
    if (bulk) {
      const Node<S> N = node_view<S>(D, R.node);
      S* base = N.g + c;
      const int pc = (int)D.pitch, sy = D.nx, sz = D.nx * D.ny;
      const int z = (int)(c / ((long long)sz));
      T ux, uy, uz;
      wall_velocity<S>(N, lw, z, wind_pull<T>(P), ux, uy, uz);
      // links that do not stream take their value from the own or the
      // in-plane slot in global memory
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        const int kind = link_kind(lw, i);
        if (kind == kStream) continue;
        const int off = kind == kSpecZ ? OPP(REFL(i, 2)) * pc - (CX(i) + CY(i) * sy) : i * pc;
        T v = Store<S>::ld(base + off);
        if (kind == kMoving) v += wall_term<T>(i, ux, uy, uz, wind_pull<T>(P).scale);
        g[i] = v;
      }
      collide_p<T, true>(P, g);
      wall_velocity<S>(N, lw, z, wind_push<T>(P), ux, uy, uz);
      fast_push<S>(base, lw, pc, sy, sz, ux, uy, uz, wind_push<T>(P).scale, g);
    }
  }
}

// ------------------------------------------------------------ persistent form
// Bounded grid barrier (sense by generation).  Gives up after spin_limit
// polls, latches kErrTimeout and returns false; every block then leaves.
__device__ bool grid_barrier(const StepParams& P, unsigned int& gen) {
  __syncthreads();
  bool ok = true;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();
    const unsigned int expected = gridDim.x + (P.never_arrive ? 1u : 0u);
    const unsigned int arrived = atomicAdd(P.bar_count, 1u) + 1u;
    if (arrived == expected) {
      atomicExch(P.bar_count, 0u);
      __threadfence();
      atomicAdd(P.bar_gen, 1u);
    } else {
      long long spins = 0;
      while (*reinterpret_cast<volatile unsigned int*>(P.bar_gen) == gen) {
        if (*reinterpret_cast<volatile unsigned int*>(P.err) & kErrTimeout) { ok = false; break; }
        if (++spins > P.spin_limit) {
          atomicOr(P.err, kErrTimeout);
          ok = false;
          break;
        }
        __nanosleep(32);
      }
    }
    gen += 1u;
    __threadfence();
  }
  __shared__ int s_ok;
  if (threadIdx.x == 0 && threadIdx.y == 0) s_ok = ok ? 1 : 0;
  __syncthreads();
  return s_ok != 0;
}

// One cooperative launch advances n_steps; blocks stride over the work of
// each level and meet at a grid barrier between time steps.
// ROT as for the odd tile: the host picks the form that turns the inflow
// for chunks whose factors do.
template <class S, bool ROT>
__global__ void __launch_bounds__(256, 3) aa_persistent_kernel(const __grid_constant__ StepParams P) {
  __shared__ unsigned long long s_n;
  __shared__ unsigned int s_gen;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    s_n = P.n_host;
    s_gen = *reinterpret_cast<volatile unsigned int*>(P.bar_gen);
  }
  __syncthreads();
  unsigned long long n = s_n;
  unsigned int gen = s_gen;
  const long long threads = (long long)P.bx * P.by;
  const long long bblocks = (P.total_bitems + threads - 1) / threads;
  for (int s = 0; s < P.n_steps; ++s) {
    if ((n & 1ull) == 0) {
      for (long long t = blockIdx.x; t < P.total_tiles; t += gridDim.x) {
        even_tile<S, true, false>(P, block_tile(P, (unsigned)t));
        __syncthreads();  // the shared tile head is rewritten next iteration
      }
    } else {
      for (long long t = blockIdx.x; t < P.total_tiles; t += gridDim.x) {
        odd_bulk_tile<S, true, ROT>(P, block_tile(P, (unsigned)t));
        __syncthreads();
      }
      // bulk and boundary cells touch disjoint slots: no barrier between them
      for (long long b = blockIdx.x; b < bblocks; b += gridDim.x)
        odd_boundary_item<S, true, ROT>(P, b * threads + threadIdx.y * P.bx + threadIdx.x);
    }
    if (!grid_barrier(P, gen)) return;
    ++n;
  }
}

// ------------------------------------------------------------ FP64 plain path
// Two arrays, push form, one node per launch.  Blocks [0, tiles_per_node)
// take the bulk cells, the rest the listed boundary cells.
__global__ void __launch_bounds__(256) plain_step_kernel(const __grid_constant__ StepParams P,
                                                         unsigned long long n) {
  const DevDomain& D = P.dom[P.plain_domain];
  const int node = P.plain_node;
  const long long pc = D.pitch;
  double* A = reinterpret_cast<double*>(D.g) + (long long)node * kQ * pc;
  double* B = reinterpret_cast<double*>(D.g2) + (long long)node * kQ * pc;
  const double* src = (n & 1ull) ? B : A;
  double* dst = (n & 1ull) ? A : B;
  const long long sy = D.nx, sz = (long long)D.nx * D.ny;
  const long long b = blockIdx.x;
  if (b < D.tiles_per_node) {
    const int tx = (int)(b % D.tiles_x);
    const int ty = (int)((b / D.tiles_x) % D.tiles_y);
    const int tz = (int)(b / (D.tiles_x * D.tiles_y));
    const int x = tx * P.bx + threadIdx.x;
    const int y = ty * P.by + threadIdx.y;
    if (x >= D.nx || y >= D.ny) return;
    const int z0 = tz * P.bz, z1 = min(z0 + P.bz, D.nz);
    Node<double> N;
    N.g = dst;
    N.bout = nullptr;
    N.uinf = nullptr;
    N.uind = D.uin_d + (long long)node * D.nz * 3;
    for (int z = z0; z < z1; ++z) {
      const long long idx = cidx(D, x, y, z);
      const LinkWord lw = __ldg(D.link + idx);
      if (lw & kLinkSlow) continue;
      double g[kQ];
#pragma unroll
      for (int i = 0; i < kQ; ++i) g[i] = src[(long long)i * pc + idx];
      collide_p<double, false>(P, g);
      double ux, uy, uz;
      wall_velocity<double>(N, lw, z, P.wqd, ux, uy, uz);
      fast_push<double>(dst + idx, lw, (int)pc, (int)sy, (int)sz, ux, uy, uz, P.wqd.scale, g);
    }
    return;
  }
  const long long item = (b - D.tiles_per_node) * (long long)(P.bx * P.by) + threadIdx.y * P.bx + threadIdx.x;
  if (item >= D.nb) return;
  const long long idx = __ldg(D.bcell + item);
  const int z = (int)(idx / ((long long)D.nx * D.ny));
  const ListedRef L = listed_ref(D, item);
  Node<double> N;
  N.g = dst;
  N.bout = nullptr;
  N.uinf = nullptr;
  N.uind = D.uin_d + (long long)node * D.nz * 3;
  double g[kQ];
#pragma unroll
  for (int i = 0; i < kQ; ++i) g[i] = src[(long long)i * pc + idx];
  collide_p<double, false>(P, g);
  double ux = 0.0, uy = 0.0, uz = 0.0;
  if (L.word(kWordPushMove)) inflow_velocity<double>(N, z, P.wqd, ux, uy, uz);
  listed_push<double>(L, dst, ux, uy, uz, P.wqd.scale, g);
}



template <class S>
size_t even_tma_smem() { return (size_t)kStages * kQ * kRun * sizeof(S) + 2 * kStages * sizeof(uint64_t); }
template <class S>
size_t odd_tma_smem() {
  return (size_t)kStages * kQ * (kRun + 2 * (16 / sizeof(S))) * sizeof(S) + 2 * kStages * sizeof(uint64_t);
}

template <class S>
int tma_grid(int* grid) {
  static int cached = 0;
  if (!cached) {
    int dev = 0, sms = 0, a = 0, b = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaFuncSetAttribute(aa_even_tma_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)even_tma_smem<S>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(aa_odd_tma_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)odd_tma_smem<S>());
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, aa_even_tma_kernel<S>, kTmaThreads, even_tma_smem<S>());
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, aa_odd_tma_kernel<S>, kTmaThreads, odd_tma_smem<S>());
    if (e != cudaSuccess) return (int)e;
    const int per = a < b ? a : b;
    if (per < 1) return (int)cudaErrorInvalidConfiguration;
    cached = sms * per;
  }
  *grid = cached;
  return 0;
}

}  // namespace

// ======================================================================= launchers
// The unit built with SCLBM_RR_UNIT (the recursive regularized collision)
// provides the step launchers in namespace rr; the observables and the
// initialisation do not depend on the collision and live in observables.cu.
#ifdef SCLBM_RR_UNIT
namespace rr {
#endif
// Whether a launch's inflow factors turn the table velocity (a direction
// offset at either level); only the kernels compiled with ROT apply a turn.
inline bool turns_inflow(const StepParams& P) {
  return !(P.wp.cos_d == 1.0f && P.wp.sin_d == 0.0f && P.wq.cos_d == 1.0f && P.wq.sin_d == 0.0f);
}

#ifndef SCLBM_RR_UNIT
// The launch parameters of the two-cells-per-thread even kernel: the same
// launch with tiles 2 * bx cells wide.
StepParams pair_tiling(const StepParams& P) {
  StepParams Q = P;
  Q.bx = 2 * P.bx;
  long long begin = 0;
  for (int d = 0; d < Q.n_domains; ++d) {
    DevDomain& D = Q.dom[d];
    D.tiles_x = (D.nx + Q.bx - 1) / Q.bx;
    D.tiles_per_node = D.tiles_x * D.tiles_y * D.tiles_z;
    D.tile_begin = begin;
    begin += D.tiles_per_node * D.nodes;
  }
  Q.total_tiles = begin;
  return Q;
}
#endif

int launch_aa_step(const StepParams& P, int precision, void* stream, int parity) {
  dim3 block(P.bx, P.by);
  cudaStream_t s = (cudaStream_t)stream;
  return dispatch(precision, [&](auto tag) -> int {
    using S = std::remove_pointer_t<decltype(tag)>;
    if constexpr (std::is_same_v<S, double>) return (int)cudaErrorInvalidValue;
    else {
      int tgrid = 0;
      if (P.tma) {
        int rc = tma_grid<S>(&tgrid);
        if (rc) return rc;
        if ((long long)tgrid > P.total_runs) tgrid = (int)P.total_runs;
      }
      // listed items ride in blocks spread over the per-thread launches
      const long long threads = (long long)P.bx * P.by;
      const unsigned lgrid = (unsigned)(P.total_tiles + (P.total_bitems + threads - 1) / threads);
      if (parity == 0) {
#ifndef SCLBM_RR_UNIT
        if constexpr (sizeof(S) == 2) {
          if (P.even_pair && !P.tma) {
            const StepParams Q = pair_tiling(P);
            const unsigned qgrid = (unsigned)(Q.total_tiles + (Q.total_bitems + threads - 1) / threads);
            if (P.even_pair == 3) aa_even_pair_kernel<S, 3><<<qgrid, block, 0, s>>>(Q);
            else aa_even_pair_kernel<S, 2><<<qgrid, block, 0, s>>>(Q);
            return (int)cudaGetLastError();
          }
        }
#endif
        if (P.tma) aa_even_tma_kernel<S><<<tgrid, kTmaThreads, even_tma_smem<S>(), s>>>(P);
        else if (P.even85) aa_even_kernel<S, 3><<<lgrid, block, 0, s>>>(P);
        else aa_even_kernel<S, 4><<<lgrid, block, 0, s>>>(P);
      } else {
        if (P.tma) {
          aa_odd_tma_kernel<S><<<tgrid, kTmaThreads, odd_tma_smem<S>(), s>>>(P);
          const long long grid = (P.total_bitems + 255) / 256;
          aa_odd_boundary_kernel<S><<<(unsigned)(grid > 0 ? grid : 1), 256, 0, s>>>(P);
        } else if (P.odd85 || turns_inflow(P)) {
          aa_odd_bulk_kernel<S, 3><<<lgrid, block, 0, s>>>(P);
        } else {
          aa_odd_bulk_kernel<S, 4><<<lgrid, block, 0, s>>>(P);
        }
      }
      return (int)cudaGetLastError();
    }
  });
}

int aa_persistent_max_grid(const StepParams& P, int precision, int* grid) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = P.bx * P.by;
  int rc = dispatch(precision, [&](auto tag) -> int {
    using S = std::remove_pointer_t<decltype(tag)>;
    if constexpr (std::is_same_v<S, double>) return (int)cudaErrorInvalidValue;
    else {
      // the grid serves both forms: the smaller of their occupancies
      int a = 0, b = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, aa_persistent_kernel<S, false>, threads, 0);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, aa_persistent_kernel<S, true>, threads, 0);
      per = std::min(a, b);
      return (int)e;
    }
  });
  *grid = sms * per;
  return rc;
}

int launch_aa_persistent(const StepParams& P, int precision, void* stream, int grid) {
  dim3 block(P.bx, P.by);
  cudaStream_t s = (cudaStream_t)stream;
  return dispatch(precision, [&](auto tag) -> int {
    using S = std::remove_pointer_t<decltype(tag)>;
    if constexpr (std::is_same_v<S, double>) return (int)cudaErrorInvalidValue;
    else {
      void* args[] = {(void*)&P};
      const void* fn = turns_inflow(P) ? (const void*)aa_persistent_kernel<S, true>
                                       : (const void*)aa_persistent_kernel<S, false>;
      return (int)cudaLaunchCooperativeKernel(fn, dim3(grid), block, args, 0, s);
    }
  });
}

int launch_plain_step(const StepParams& P, unsigned long long n, void* stream) {
  const DevDomain& D = P.dom[P.plain_domain];
  dim3 block(P.bx, P.by);
  cudaStream_t s = (cudaStream_t)stream;
  const long long threads = (long long)P.bx * P.by;
  const long long grid = D.tiles_per_node + (D.nb + threads - 1) / threads;
  // the time level of the plain path is tracked on the host
  plain_step_kernel<<<(unsigned)grid, block, 0, s>>>(P, n);
  return (int)cudaGetLastError();
}

#ifdef SCLBM_RR_UNIT
}  // namespace rr
#endif

}  // namespace sclbm
