// lbm_kernels.cu -- CUDA kernels of libsclbm for sm_103a (GB300).
//
// Stream-collide of the D3Q19 lattice Boltzmann equation (arXiv:2508.18202
// Sec. 2.2, Eq. deterministicLBE) with BGK collision and the Smagorinsky
// effective relaxation time (Eqs. tauEff, turbVisc), for every collocation
// node of every domain of an ensemble, plus the quadrature / gPC reductions
// of Sec. 2.3 (Eqs. quad_moments, coef_discrete).
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
__device__ __forceinline__ TileRef block_tile(const StepParams& P, unsigned t) {
  __shared__ TileHead s_head;
  if (threadIdx.x == 0 && threadIdx.y == 0) s_head = decode_tile_head(P, t);
  __syncthreads();
  const TileHead H = s_head;
  TileRef R;
  const DevDomain& D = P.dom[H.d];
  R.d = H.d;
  R.node = H.node;
  R.x = H.x0 + threadIdx.x;
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

#ifndef SCLBM_RR_UNIT
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
struct DF {
  float hi, lo;
};
__device__ __forceinline__ void df_dot_add(DF& s, float2 b, float q) {
  const float p = __fmul_rn(b.x, q);
  const float e = __fmaf_rn(b.x, q, -p);
  const float t = __fmul_rn(b.y, q);
  const float sum = __fadd_rn(s.hi, p);
  const float bb = __fsub_rn(sum, s.hi);
  const float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(sum, bb)), __fsub_rn(p, bb));
  const float lo = __fadd_rn(s.lo, __fadd_rn(err, __fadd_rn(e, t)));
  const float hi = __fadd_rn(sum, lo);
  s.lo = __fsub_rn(lo, __fsub_rn(hi, sum));
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
// order.  S1 and S2 accumulate in FP64.  The gPC sums accumulate in FP64 on
// the FP64 plain path and, on the in-place (FP32-arithmetic) paths, as
// compensated FP32 pairs (df_dot_add), which keeps the FP64 pipe for S1 and
// S2: |u| is a float there, so each product is exact to 48 bits.  PM >= A.P is
// the compile-time size of the coefficient array (a small basis holds few
// registers).  raw: write the sums S1, S2 (and the gPC sums); with accumulate
// the sums start from the values in the output arrays, so node ranges reduced
// one after another (waves, shards) continue one sum per cell: S1 and S2 then
// carry the bits of one reduction over all nodes, the gPC pair sums agree
// with it to their 48-bit rounding.
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
    // compensated pair sums where |u| is a float (the time averages are
    // FP64 and take the FP64 sums)
    constexpr bool PAIR = SHIFT && !AVG;
    double coef[PM > 0 ? PM : 1];
    DF cf[PAIR && PM > 0 ? PM : 1];
#pragma unroll
    for (int a = 0; a < PM; ++a) {
      const double v = (acc && a < A.P) ? A.coef[(long long)a * D.ncell + c] : 0.0;
      if constexpr (PAIR) cf[a] = df_from(v);
      else coef[a] = v;
    }
    if (!(lw & kLinkSolid)) {
      for (int j = 0; j < A.nq; ++j) {
        double q;
        float qf = 0.0f;
        if constexpr (AVG) {
          q = A.avg[(long long)j * D.ncell + c] * A.avg_scale;
          if (!isfinite(q)) bad = true;
        } else {
          T g[kQ];
          gather_pops<S, SHIFT>(P, D, j, n, x, y, z, c, lw, g);
          T rho, ux, uy, uz;
          macro<T, SHIFT>(g, rho, ux, uy, uz);
          if (!(rho > T(0)) || !isfinite(double(ux + uy + uz)) || !isfinite(double(rho))) bad = true;
          const T sp = speed<T>(ux, uy, uz);
          q = double(sp);
          qf = float(sp);
        }
        const double* ab = A.ab + (long long)j * A.stride;
        const double aq = ab[0] * q;
        s1 += aq;
        s2 = fma(aq, q, s2);
        if constexpr (PAIR) {
          const float2* bf = A.abf + (long long)j * A.P;
#pragma unroll
          for (int a = 0; a < PM; ++a)
            if (a < A.P) df_dot_add(cf[a], bf[a], qf);
        } else {
#pragma unroll
          for (int a = 0; a < PM; ++a)
            if (a < A.P) coef[a] = fma(ab[1 + a], q, coef[a]);
        }
      }
    }
    if constexpr (PAIR) {
#pragma unroll
      for (int a = 0; a < PM; ++a) coef[a] = df_value(cf[a]);
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

#endif  // SCLBM_RR_UNIT

int grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  if (g > 152LL * 64) g = 152LL * 64;
  return (int)(g < 1 ? 1 : g);
}

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
// initialisation do not depend on the collision and live in the BGK unit only.
#ifdef SCLBM_RR_UNIT
namespace rr {
#endif
// Whether a launch's inflow factors turn the table velocity (a direction
// offset at either level); only the kernels compiled with ROT apply a turn.
inline bool turns_inflow(const StepParams& P) {
  return !(P.wp.cos_d == 1.0f && P.wp.sin_d == 0.0f && P.wq.cos_d == 1.0f && P.wq.sin_d == 0.0f);
}

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
#else
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
      auto go = [&](auto avg) {
        constexpr bool AV = decltype(avg)::value;
        if (A.P == 0) moments_kernel<S, SH, 0, AV><<<grid, blk, 0, s>>>(P, A);
        else if (A.P <= 3) moments_kernel<S, SH, 3, AV><<<grid, blk, 0, s>>>(P, A);
        else if (A.P <= 6) moments_kernel<S, SH, 6, AV><<<grid, blk, 0, s>>>(P, A);
        else if (A.P <= 10) moments_kernel<S, SH, 10, AV><<<grid, blk, 0, s>>>(P, A);
        else if (A.P <= 15) moments_kernel<S, SH, 15, AV><<<grid, blk, 0, s>>>(P, A);
        else if (A.P <= 21) moments_kernel<S, SH, 21, AV><<<grid, blk, 0, s>>>(P, A);
        else moments_kernel<S, SH, kMaxGpcP, AV><<<grid, blk, 0, s>>>(P, A);
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

#endif  // SCLBM_RR_UNIT

}  // namespace sclbm
