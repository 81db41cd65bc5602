/*
 * sclbm.h -- C ABI of libsclbm, the GB300 (sm_103a) implementation of the
 * data-parallel hot path of the non-intrusive stochastic-collocation lattice
 * Boltzmann method of arXiv:2508.18202 (Zhong, Teutscher, Kummerlaender,
 * Krause, Frank, Simonis: "Uncertain data assimilation for urban wind flow
 * simulations with OpenLB-UQ").
 *
 * The problem (Sec. 2.1): incompressible flow whose inflow boundary data are
 * uncertain; the uncertainty is carried by a vector Z of independent random
 * inputs (relative wind-speed error, profile exponent, wind direction).  The
 * method (Sec. 2.4, steps 2-7): pick a quadrature rule {Z^(j), a_j} on the
 * input space (Sec. 2.3), run the deterministic D3Q19 lattice Boltzmann solver
 * (Sec. 2.2) at every node with that node's inflow, then reduce the
 * per-node quantities of interest to quadrature moments (Eq. quad_moments),
 * gPC coefficients (Eqs. gPC, coef_discrete) and vertical-profile confidence
 * bands (Sec. 4).
 *
 * Conventions
 *   - Every function returns an int status: SC_OK (0) or a negative SC_ERR_*.
 *     Nothing aborts the process; no C++ exception crosses the ABI.  After an
 *     error on a handle, sc_lbm_last_error() names the cause.
 *   - Cell index: c = x + nx*(y + ny*z), x fastest.  Faces: 0 -x, 1 +x,
 *     2 -y, 3 +y, 4 -z (ground), 5 +z (sky).
 *   - "device" pointers are CUDA device memory owned by the caller; "host"
 *     pointers are ordinary (optionally pinned) host memory owned by the
 *     caller.  The library never frees caller memory.  The only memory the
 *     library owns is the small host-side state behind an sc_lbm_t and the
 *     fixed scratch array of sc_lbm_quad_moments_noalloc (below).
 *   - All device work of a handle is issued on the CUDA stream given to
 *     sc_lbm_init and is asynchronous unless a function says it synchronises.
 *     Device-side failures (non-finite populations, an expired wait) are
 *     latched in the workspace and reported by the next synchronising call.
 */
#ifndef SCLBM_H
#define SCLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define SC_OK 0
#define SC_ERR_ARG (-1)          /* invalid argument or configuration          */
#define SC_ERR_WORKSPACE (-2)    /* workspace missing, misaligned or too small */
#define SC_ERR_CUDA (-3)         /* a CUDA runtime call failed                 */
#define SC_ERR_DIVERGED (-4)     /* non-finite or non-positive density seen    */
#define SC_ERR_TIMEOUT (-5)      /* a bounded device-side wait expired         */
#define SC_ERR_UNSUPPORTED (-6)  /* valid request this build does not support  */
#define SC_ERR_STATE (-7)        /* call not valid in the handle's state       */
#define SC_ERR_SCRATCH (-8)      /* request exceeds the fixed no-alloc scratch */

/* ------------------------------------------------------------ enumerations */
/* collision model */
#define SC_COLL_BGK 0  /* BGK (+ Smagorinsky), second-order equilibrium       */
#define SC_COLL_RR 1   /* recursive regularized, third-order equilibrium      */
/* boundary kind per face (Sec. 2.2 boundary list; OUTFLOW added for channels) */
#define SC_BC_VELOCITY 0     /* prescribed inflow velocity (moving-wall links) */
#define SC_BC_OUTFLOW 1      /* zero-gradient outflow; only on face 1 (+x)     */
#define SC_BC_BOUNCE_BACK 2  /* no-slip wall, half-way bounce-back             */
#define SC_BC_FREE_SLIP 3    /* specular reflection (the paper's sky)          */
#define SC_BC_PERIODIC 4     /* both faces of an axis must be periodic         */

/* uncertain inputs (Sec. 2.1 Eq. mult_noise, Sec. 3), uniform on [lo, hi]    */
#define SC_IN_SPEED_REL 0    /* xi: inflow speed u_ref (1 + xi)                */
#define SC_IN_ALPHA 1        /* power-law exponent alpha                       */
#define SC_IN_ANGLE_DEG 2    /* wind direction theta in degrees                */

/* quadrature rules (Sec. 2.3-2.4)                                            */
#define SC_Q_GL 0            /* tensor Gauss-Legendre, quad_level points/dim   */
#define SC_Q_CC_SMOLYAK 1    /* Clenshaw-Curtis Smolyak grid, level (1-based)  */
#define SC_Q_GH 2            /* tensor Gauss-Hermite, quad_level points/dim,
                                for normal inputs (Sec. 2.4 step 3)            */

/* inflow profile shape (Sec. 3) */
#define SC_PROFILE_POWER 0   /* u_ref (1 + xi) (h/H)^alpha                     */
#define SC_PROFILE_LOG 1     /* u_ref (1 + xi) ln((h+z0)/z0) / ln((H+z0)/z0)   */

/* population precision                                                       */
#define SC_P_FP64_PLAIN 0    /* FP64, unshifted, two arrays, one node per launch */
#define SC_P_FP32_SHIFT 1    /* FP32 storing g_i = f_i - w_i, in place (AA)     */
#define SC_P_BF16_STORE 2    /* BF16 storage of g_i, FP32 arithmetic            */
#define SC_P_FP16_STORE 3    /* FP16 storage of g_i, FP32 arithmetic            */

/* execution of sc_lbm_step for the in-place precisions                       */
#define SC_EXEC_LAUNCH 0     /* one kernel launch per time step                */
#define SC_EXEC_GRAPH 1      /* replay of a captured CUDA graph of steps       */
#define SC_EXEC_PERSISTENT 2 /* one cooperative launch, grid barrier per step  */

#define SC_MAX_DOMAINS 8
#define SC_MAX_NODES 512

/* ------------------------------------------------------------ configuration */
/* One simulation domain (a box of nx*ny*nz cells, lattice units dx = dt = 1).
 * Geometry: the half-open boxes [x0,x1)x[y0,y1)x[z0,z1) in `boxes` when
 * n_boxes > 0, else n_buildings seeded rectangular blocks standing on the
 * ground (see sc_lbm_geometry).  quad_level: points per dimension (SC_Q_GL,
 * 1..5; SC_Q_GH, 1..40) or the sparse-grid level (SC_Q_CC_SMOLYAK) used for
 * this domain.
 * disk_radius > 0 makes the domain the paper's cylinder (Sec. 2.2: a disk of
 * radius R around the buildings whose mantle carries a local velocity
 * boundary): every column whose centre (x + 1/2, y + 1/2) lies more than R
 * from (nx / 2, ny / 2) is outside (flag 2), and a link from a fluid cell
 * into it takes the velocity rule of a VELOCITY face with the inflow of the
 * cell's layer.  The box faces still apply where the disk reaches them; a
 * circular domain takes no OUTFLOW face (SC_ERR_UNSUPPORTED).  0 (the
 * zero-initialised default): the plain box.  Negative or non-finite:
 * SC_ERR_ARG.                                                              */
typedef struct {
  int nx, ny, nz;
  uint64_t geom_seed;
  int n_buildings, fp_min, fp_max, h_min, h_max;
  const int32_t* boxes; /* host, [n_boxes][6], read during calls only */
  int n_boxes;
  int bc[6];
  int quad_level;
  double disk_radius;
} sc_domain_desc;

/* The ensemble.  tau0 = 3 nu + 1/2 (Eq. tauEff with dx = dt = 1); c_smag is
 * the Smagorinsky constant C_S of Eq. turbVisc (0 = plain BGK).  Nominal
 * inflow u_in(z) = u_ref (1 + xi) (h/H)^alpha (cos theta, sin theta, 0) with
 * h = z + 1/2 and H = H_ref (H_ref <= 0 selects the domain height nz); each
 * uncertain input k replaces xi, alpha or theta by the node coordinate.
 * ramp_steps: length of the start-up ramp of the inflow (0 = impulsive).
 * gpc_degree: total degree of the Legendre gPC projection, -1 for none.
 * collision: SC_COLL_BGK (second-order equilibrium, f* = f - (f - f^eq) /
 * tau_eff) or SC_COLL_RR, the paper's recursive regularized form (Sec. 2.2,
 * Eqs. deterministicLBE and hermiteCoeff): third-order equilibrium on the six
 * third-order Hermite combinations D3Q19 carries, non-equilibrium rebuilt from
 * its second-order Hermite coefficient and the third-order one obtained by
 * the recursion a3_abg = u_a a2_bg + u_b a2_ag + u_g a2_ab; tau_eff as for
 * BGK.  Zero-initialised configs select BGK.
 * Inputs: with SC_Q_GL / SC_Q_CC_SMOLYAK input k is uniform on [lo[k], hi[k]]
 * and the gPC basis is orthonormal Legendre; with SC_Q_GH it is normal with
 * mean lo[k] and standard deviation hi[k] (the paper's Gaussian speed and
 * direction perturbations, Eq. mult_noise: SC_IN_SPEED_REL with mean 0 and
 * std 0.1 is zeta_1 - 1, SC_IN_ANGLE_DEG with std 6 is zeta_2 in degrees)
 * and the basis is orthonormal probabilists' Hermite He_n / sqrt(n!).
 * profile: SC_PROFILE_POWER (default) or SC_PROFILE_LOG, the paper's
 * logarithmic wind profile with roughness length z0 > 0 in cells (alpha
 * unused).
 * time_average: 1 reserves FP64 accumulators (8 B per cell and node) for the
 * time-averaged |u| fields (sc_lbm_average_*), 0 none.
 * node_begin, node_count: the collocation nodes this handle runs, the range
 * [node_begin, node_begin + node_count) of every domain's rule (node_count 0:
 * to the end).  The nodes are independent runs (Sec. 2.4 step 5), so an
 * ensemble shards across processes / GPUs by node ranges; each shard adds
 * its sc_lbm_moment_sums to the others' and finishes with
 * sc_lbm_moments_from_sums.  Default 0, 0: all nodes.                       */
typedef struct {
  int n_domains;
  const sc_domain_desc* domains; /* host, read during calls only */
  double tau0, c_smag;
  double u_ref, alpha, angle_deg, H_ref;
  int n_inputs;
  int inputs[3];
  double lo[3], hi[3];
  int quad_rule;
  int ramp_steps;
  int precision;
  int gpc_degree;
  int collision;
  int profile;
  double z0;
  int time_average;
  int node_begin, node_count;
} sc_lbm_config;

/* Launch shape of the stream-collide kernels (chosen by sc_lbm_autotune or
 * set by the caller).  block_x (multiple of 32) by block_y threads, at most
 * 256, cover a block_x * block_y patch of an x-y plane; each thread walks
 * slab_z cells in z.  tile_order 0 runs the nodes of one patch back to back (shared geometry
 * stays in L2), 1 runs all patches of one node first.  graph_steps: time
 * steps per captured graph (SC_EXEC_GRAPH).  variant 0 loads per thread
 * with a register budget for 4 resident blocks of 256 threads, 2 the same
 * for 3 blocks, 3 uses 4 blocks for the even and 3 for the odd level, 1
 * streams runs of 256 consecutive cells through shared memory with TMA bulk
 * copies (needs nx a multiple of 16 bytes of populations; launch and graph
 * modes only).  With BF16 / FP16 storage, the BGK collision and an even nx
 * in every domain, variants 0 and 3 run the even level with two x-adjacent
 * cells per thread (one 32-bit access per population pair, the collision on
 * packed FP32x2 operations; the block then covers 2 * block_x cells in x),
 * sized for 2 (variant 0) or 3 (variant 3) resident blocks; the results
 * equal the one-cell form's to FP32 rounding, not bit for bit.  Default:
 * 64 x 2, slab 8, tile order 1, variant 0, launch mode.                     */
typedef struct {
  int block_x, block_y, slab_z, tile_order, exec_mode, graph_steps, variant;
} sc_lbm_tuning;

typedef struct sc_lbm_s* sc_lbm_t;

/* ------------------------------------------------------------ host-only calls
 * These need no GPU and touch no device memory.                            */

/* Bytes of device workspace sc_lbm_init needs for cfg.  SC_ERR_ARG when the
 * configuration is invalid.                                                  */
int sc_lbm_workspace_size(const sc_lbm_config* cfg, size_t* bytes_out);

/* Collocation nodes and probability weights of `domain` (Sec. 2.3 Eq.
 * coef_discrete's {Z^(j), a_j}; Sec. 2.4 step 3).  Z: host [n][n_inputs],
 * w: host [n].  With Z == NULL only *n_nodes is written.  Nodes are ordered
 * lexicographically by their integer index on the finest 1-D grid; sparse
 * grid weights may be negative.  SC_ERR_ARG if cap < *n_nodes.  The result
 * is bit-for-bit reproducible (IEEE double, no contraction).               */
int sc_lbm_quadrature(const sc_lbm_config* cfg, int domain, int* n_nodes, double* Z,
                      double* w, int cap);

/* Cell flags (0 fluid, 1 solid, 2 beyond the mantle of a circular domain)
 * of `domain` into host uint8 [nz*ny*nx].
 * Seeded blocks use SplitMix64 (Steele, Lea & Flood 2014) on geom_seed; per
 * block, in this order: wx, wy ~ U{fp_min..fp_max}; h ~ U{h_min..min(h_max,
 * nz-4)}; x0 ~ U{nx/8 .. nx - nx/8 - wx}; y0 ~ U{2 .. ny - 2 - wy}; with
 * U{a..b} = a + (next mod (b - a + 1)).  The paper's geometry is a real
 * scene (Sec. 3) that is not available; this generator stands in for it.   */
int sc_lbm_geometry(const sc_lbm_config* cfg, int domain, uint8_t* flags);

/* n distinct probe columns (host int32 [n][2] = x, y) with a fluid ground
 * cell, drawn from SplitMix64(geom_seed + 1): x ~ U{nx/8..nx-1}, y ~
 * U{0..ny-1} (Sec. 4, Table probes, stands in for the paper's P1-P3).      */
int sc_lbm_probe_columns(const sc_lbm_config* cfg, int domain, int n, int32_t* xy);

/* n distinct fluid probe points (host int32 [n][3]) from the same stream:
 * x ~ U{nx/8..nx-1}, y ~ U{0..ny-1}, z ~ U{0..nz-3}.                       */
int sc_lbm_probe_points(const sc_lbm_config* cfg, int domain, int n, int32_t* xyz);

/* ------------------------------------------------------------ device calls */

/* Create a handle: validates cfg, builds the quadrature, geometry, link
 * classification and inflow tables on the host, uploads them into the
 * caller's device workspace d_ws (>= sc_lbm_workspace_size bytes, 256-byte
 * aligned) on `cuda_stream` (a cudaStream_t, NULL = legacy default stream),
 * and sets every node's populations to the equilibrium at rho = 1, u = 0
 * (Sec. 2.2).  flags_host, if non-NULL, supplies host uint8 solid flags per
 * domain (flags_host[d] of [nz*ny*nx], nonzero = solid) instead of the
 * configured geometry; a circular domain's mantle is applied on top.
 * The workspace must stay allocated until sc_lbm_destroy.                  */
int sc_lbm_init(const sc_lbm_config* cfg, void* d_ws, size_t bytes, void* cuda_stream,
                const uint8_t* const* flags_host, sc_lbm_t* out);

/* Reset every node to the initial equilibrium and the step count to 0.     */
int sc_lbm_reset(sc_lbm_t h);

/* Advance every node of every domain by n_steps time steps of the lattice
 * Boltzmann equation (Sec. 2.2, Eq. deterministicLBE) with BGK collision,
 * Smagorinsky effective relaxation time (Eqs. tauEff, turbVisc) and the
 * boundary conditions of the domain's faces and buildings.  Asynchronous.  */
int sc_lbm_step(sc_lbm_t h, int n_steps);

/* Quadrature reduction of the velocity magnitude |u| at the current time
 * (Sec. 2.4 steps 6-7):
 *   mean  = sum_j a_j Q_j / sum_j a_j, std = sqrt(max(var, 0)) with
 *   var = sum_j a_j Q_j^2 / sum_j a_j - mean^2 (FP64 accumulation)
 *   (Eq. quad_moments); d_mean, d_std: [nz*ny*nx] doubles, solid cells 0;
 *   gpc: d_gpc_coef [P][ncell] doubles, coef_alpha = sum_j a_j Q_j
 *   Phi_alpha(Z^(j)) for the orthonormal Legendre basis (Eq. coef_discrete,
 *   gamma = 1), P = C(gpc_degree + n_inputs, n_inputs) <= 28, graded order;
 *   NULL skips it.  Q_j = |u| is formed in the path's arithmetic (FP32 for
 *   the in-place precisions, FP64 for SC_P_FP64_PLAIN); the gPC sums run in
 *   FP64 on the FP64 path and as compensated FP32 pairs (about 48 bits,
 *   products exact) on the others;
 *   profiles at the n_p columns probe_xy (host int32 [n_p][2]):
 *   d_prof [n_p][nz][4] doubles = (mean, std, mean - 1.96 std,
 *   mean + 1.96 std) (95% band, Sec. 4) and optional d_prof_nodes
 *   [n_p][n_nodes][nz] floats with each node's profile.
 * out_host != 0: all outputs are host pointers; the call then copies from
 * workspace staging and synchronises the stream before returning.
 * Returns SC_ERR_DIVERGED if a non-finite or non-positive density was met.  */
int sc_lbm_moments(sc_lbm_t h, int domain, double* mean, double* stdev,
                   const int32_t* probe_xy, int n_p, double* prof, float* prof_nodes,
                   double* gpc_coef, int out_host);

/* Velocity of one node at the current time: d_u device float [3][ncell],
 * solid cells 0.                                                            */
int sc_lbm_velocity(sc_lbm_t h, int domain, int node, float* d_u);

/* Sharded ensembles and waves (the nodes are independent runs, Sec. 2.4
 * step 5; the quadrature sums of Eq. quad_moments and Eq. coef_discrete add
 * over node ranges): the raw FP64 sums of the handle's nodes,
 * d_s1 = sum_j a_j Q_j, d_s2 = sum_j a_j Q_j^2 (device double [ncell]) and,
 * if d_gpc_sums is not NULL, sum_j a_j Q_j Phi_alpha(Z_j) ([P][ncell]).
 * accumulate = 0 overwrites the three arrays; accumulate = 1 adds this
 * handle's nodes to the sums already in them, continuing each cell's FP64
 * sum node by node, so ranges [0, k) then [k, n) reduced into the same
 * arrays give the bits of one handle over [0, n).  Other values: SC_ERR_ARG.
 * sc_lbm_weight_sum gives the handle's sum_j a_j (host);
 * sc_lbm_rule_weight_sum (host-only, no handle) the sum over every node of
 * the domain's rule, in node order.  After the shards' sums and weight sums
 * are added (an all-reduce), sc_lbm_moments_from_sums writes mean = S1 / W
 * and std = sqrt(max(S2 / W - mean^2, 0)) (Eq. quad_moments) into d_mean,
 * d_stdev (device double [ncell]).  The gPC coefficients are the summed gPC
 * sums themselves.  Asynchronous.                                          */
int sc_lbm_moment_sums(sc_lbm_t h, int domain, double* d_s1, double* d_s2, double* d_gpc_sums,
                       int accumulate);
int sc_lbm_weight_sum(sc_lbm_t h, int domain, double* wsum);
int sc_lbm_rule_weight_sum(const sc_lbm_config* cfg, int domain, double* wsum);
int sc_lbm_moments_from_sums(sc_lbm_t h, int domain, const double* d_s1, const double* d_s2, double wsum,
                             double* d_mean, double* d_stdev);

/* Time-averaged velocity magnitude fields (Sec. 2.4 step 6, the paper's
 * time-averaged QoI), for configurations with time_average = 1 (else
 * SC_ERR_STATE).  sc_lbm_average_reset zeroes the accumulators;
 * sc_lbm_average_add adds |u| of every node of every domain at the current
 * time level as one sample (FP64 sums); sc_lbm_average_moments is
 * sc_lbm_moments (same arguments and outputs) applied to the per-node time
 * averages Q_j = sum over samples / samples; sc_lbm_average_field writes the
 * time average of one node into d_q (device double [ncell]).  Both readers
 * need at least one sample (else SC_ERR_STATE).  Asynchronous on the
 * handle's stream except where out_host = 1.                               */
int sc_lbm_average_reset(sc_lbm_t h);
int sc_lbm_average_add(sc_lbm_t h);
int sc_lbm_average_samples(sc_lbm_t h, long long* samples);
int sc_lbm_average_moments(sc_lbm_t h, int domain, double* mean, double* stdev,
                           const int32_t* probe_xy, int n_p, double* prof, float* prof_nodes,
                           double* gpc_coef, int out_host);
int sc_lbm_average_field(sc_lbm_t h, int domain, int node, double* d_q);

/* Confidence bounds from the gPC surrogate (Sec. 2.4 step 7: confidence
 * intervals from the expansion coefficients; Sec. 4 profile bands).  For
 * each of n_cells cells (host int32 cell indices c = x + nx (y + ny z) of
 * `domain`) the surrogate Q(s) = sum_a c_a(x) Phi_a(s) is evaluated at
 * n_samples input samples and the q-quantile is its k-th smallest value,
 * k = ceil(q n_samples) in double arithmetic, clamped to [1, n_samples].
 * d_coef: device double [P][ncell], the coefficients sc_lbm_moments or
 * sc_lbm_average_moments wrote for this domain.  samples: host double
 * [n_samples][n_inputs] in the basis's standard coordinates: s = (2 Z - lo
 * - hi) / (hi - lo) in [-1, 1] for the Legendre basis (SC_Q_GL,
 * SC_Q_CC_SMOLYAK), s = (Z - lo) / hi, standard normal, for the Hermite
 * basis (SC_Q_GH).  The caller draws them (any design: random, midpoints).
 * q: host double [n_q], each in [0, 1].  d_out: device double
 * [n_q][n_cells].  Asynchronous on the handle's stream (the host arrays may
 * be reused when the call returns).  SC_ERR_ARG for a configuration with
 * gpc_degree < 0, n_cells outside [0, SC_QUANTILE_MAX_CELLS], n_samples
 * outside [1, SC_QUANTILE_MAX_SAMPLES], n_q outside [1, SC_QUANTILE_MAX_Q],
 * a cell outside the domain, q outside [0, 1], a non-finite sample or a
 * null array.                                                              */
#define SC_QUANTILE_MAX_SAMPLES 8192
#define SC_QUANTILE_MAX_CELLS 65536
#define SC_QUANTILE_MAX_Q 16
int sc_lbm_gpc_quantiles(sc_lbm_t h, int domain, const double* d_coef, int n_cells, const int32_t* cells,
                         int n_samples, const double* samples, int n_q, const double* q, double* d_out);

/* Q-criterion of a velocity field (the vortex identification of the paper's
 * Q-criterion figures): d_u device float [3][ncell] (for instance from
 * sc_lbm_velocity), d_q device float [ncell] receives
 * Q = (|Omega|^2 - |S|^2) / 2 of grad u by central differences (dx = 1),
 * one-sided next to solid cells and non-periodic faces; solid cells 0.     */
int sc_lbm_qcriterion(sc_lbm_t h, int domain, const float* d_u, float* d_q);

/* Populations f_i (unshifted, natural layout) of one node at the current
 * time: d_f device double [19][ncell]; solid cells 0.  Velocity order:
 * 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 the face diagonals as opposite
 * pairs (+1,+1,0),(-1,-1,0),(+1,-1,0),(-1,+1,0),(+1,0,+1),(-1,0,-1),
 * (+1,0,-1),(-1,0,+1),(0,+1,+1),(0,-1,-1),(0,+1,-1),(0,-1,+1).             */
int sc_lbm_populations(sc_lbm_t h, int domain, int node, double* d_f);

/* Launch shape: sc_lbm_autotune times candidate shapes on the current
 * configuration, keeps the fastest and resets the populations afterwards
 * (tuning steps advance the state).  cache_path (host string, may be NULL)
 * names a JSON file whose entry for this GPU and configuration is reused or
 * written.  Synchronises.                                                   */
int sc_lbm_autotune(sc_lbm_t h, const char* cache_path);
int sc_lbm_set_tuning(sc_lbm_t h, const sc_lbm_tuning* t);
int sc_lbm_get_tuning(sc_lbm_t h, sc_lbm_tuning* t);

/* Counters: time steps taken, kernels launched by this handle so far.      */
int sc_lbm_counters(sc_lbm_t h, long long* steps, long long* kernel_launches);

/* Wait for the handle's stream and report latched device errors
 * (SC_ERR_DIVERGED, SC_ERR_TIMEOUT) once.                                  */
int sc_lbm_sync(sc_lbm_t h);

/* Scan every node for non-finite or non-positive density now (latches
 * SC_ERR_DIVERGED) and synchronise; *n_bad receives the count.             */
int sc_lbm_check(sc_lbm_t h, long long* n_bad);

/* Test hook for the bounded device-side waits: a nonzero value makes the
 * next persistent launch wait for a grid-barrier arrival that never comes,
 * so the wait expires after `spin_limit` polls and the launch returns
 * SC_ERR_TIMEOUT (through sc_lbm_sync) with the device still usable.        */
int sc_lbm_debug_barrier(sc_lbm_t h, int never_arrive, long long spin_limit);

/* Host snapshot of the full state (populations, outflow plane, step count)
 * for checkpoint / resume.  sc_lbm_state_size gives the bytes; save copies
 * to host_buf and synchronises; load restores from a buffer written by save
 * for the same configuration (checked by a header checksum).               */
int sc_lbm_state_size(sc_lbm_t h, size_t* bytes);
int sc_lbm_save(sc_lbm_t h, void* host_buf, size_t bytes);
int sc_lbm_load(sc_lbm_t h, const void* host_buf, size_t bytes);

/* ------------------------------------------------------------ assimilation
 * The paper assimilates measured inflow by prescribing it at the boundary
 * (Sec. 2.4 step 5) and names data assimilation as the purpose (Sec. 1); it
 * does not differentiate the solver.  These calls add gradient-based
 * estimation of the inflow parameters from velocity probes.              */

/* Replace the nominal inflow parameters (u_ref, alpha, theta in degrees) and
 * rebuild every node's inflow table.  Synchronises the handle's stream.    */
int sc_lbm_set_inflow(sc_lbm_t h, double u_ref, double alpha, double angle_deg);

/* ------------------------------------------------------------ time-varying inflow
 * Hourly targets of wind speed and direction joined by an interpolation
 * interval (Sec. 2.2: after the start-up ramp the boundary velocity moves
 * gradually to the next target magnitude and direction; Sec. 2.4 step 1 and
 * Sec. 3: one measured target per hour, perturbed per node as
 * U_H(t) zeta_1 and Theta(t) + zeta_2).
 *
 * speed[k]: target k's wind speed relative to the configuration's u_ref
 * (factor >= 0); dir_deg[k]: its direction relative to the configuration's
 * (degrees).  Target 0 holds from level 0; target k >= 1 takes over at
 * level k * steps_per_target: over the next interp_steps levels the speed
 * factor s and the direction offset delta move linearly from target k - 1
 * to target k (the direction along the shorter arc, a half turn clockwise),
 * lam = min(o, interp_steps) / interp_steps at offset o (a jump when
 * interp_steps = 0); after the last target it holds.  At time level m every
 * node's inflow table u(z) is used as (a u_x - b u_y, b u_x + a u_y, m_ u_z)
 * with a = r s cos(delta), b = r s sin(delta), m_ = r s and r the start-up
 * ramp: the node's speed factor and direction offset, applied to U_H(m)
 * and Theta(m), give exactly this.
 *
 * Levels count from the handle's level 0 (sc_lbm_reset keeps the series).
 * The call copies the arrays (host memory, n_targets each); it takes effect
 * from the next step.  n_targets = 0 removes the series (steady inflow).
 * Stretches of levels over which the factor stays fixed run in the tuned
 * execution mode; a level inside an interpolation interval or the ramp is
 * launched alone.  The adjoint returns SC_ERR_UNSUPPORTED while a series
 * is set.  Errors: SC_ERR_ARG for n_targets outside
 * [0, SC_SERIES_MAX_TARGETS], a null array with n_targets > 0, a
 * non-finite or negative speed factor, a non-finite direction,
 * steps_per_target outside [1, 2^40] or interp_steps outside
 * [0, steps_per_target].                                                 */
#define SC_SERIES_MAX_TARGETS 100000
int sc_lbm_set_inflow_series(sc_lbm_t h, int n_targets, const double* speed, const double* dir_deg,
                             long long steps_per_target, long long interp_steps);

/* Host-only: the factor (a, b, m_) above at time level `level` >= 0 for a
 * ramp of ramp_steps levels and a series (n_targets = 0: none) into
 * factor[3].  Needs no handle and no GPU.  SC_ERR_ARG as above, or for
 * ramp_steps < 0, level < 0 or a null factor.                            */
int sc_lbm_inflow_factor(int ramp_steps, int n_targets, const double* speed, const double* dir_deg,
                         long long steps_per_target, long long interp_steps, long long level, double* factor);

/* Host-only: the first level after `level` at which the factor above may
 * change (LLONG_MAX if it never does) into *next.  sc_lbm_step runs the
 * levels [level, *next - 1) of a stretch in the tuned execution mode with
 * that one factor; the level before a change is launched alone.  Same
 * arguments and errors as sc_lbm_inflow_factor.                          */
int sc_lbm_inflow_next_change(int ramp_steps, int n_targets, const double* speed, const double* dir_deg,
                              long long steps_per_target, long long interp_steps, long long level,
                              long long* next);

/* Device bytes the adjoint needs for this domain, step count, checkpoint
 * count (0 = ceil(sqrt(n_steps))) and probe count (1..256).                */
int sc_lbm_adjoint_workspace_size(sc_lbm_t h, int domain, int n_steps, int n_snapshots,
                                  int n_probes, size_t* bytes);

/* Loss and gradient of the probe misfit for one collocation node:
 *   J = sum_p |u(x_p, T) - u_target_p|^2 at time level T = n_steps of a run
 *   from the equilibrium at rho = 1, u = 0 with that node's inflow, and
 *   dJ/d(u_ref, alpha) by the discrete adjoint of the FP32 BGK step (the
 *   transpose of the collision Jacobian and of the streaming / link rules),
 *   with the forward states recomputed per segment from n_snapshots
 *   checkpoints (0 = ceil(sqrt(n_steps))) and the gradient accumulated in
 *   FP64.  alpha is the node's power-law exponent.
 * probes: host int32 [n_probes][3] fluid cells; u_target: host double
 * [n_probes][3]; d_ws: device workspace of sc_lbm_adjoint_workspace_size
 * bytes (256-byte aligned), caller-owned, overwritten; loss_out: host double;
 * grad_out: host double[2]; u_probe_out: host double [n_probes][3] or NULL.
 * Leaves the handle's populations untouched; synchronises.
 * SC_ERR_UNSUPPORTED when c_smag > 0, collision is not SC_COLL_BGK (the
 * adjoint covers BGK), profile is not SC_PROFILE_POWER, an inflow series is
 * set or the domain is circular (disk_radius > 0).                         */
int sc_lbm_adjoint(sc_lbm_t h, int domain, int node, const int32_t* probes, int n_probes,
                   const double* u_target, int n_steps, int n_snapshots, void* d_ws, size_t bytes,
                   double* loss_out, double* grad_out, double* u_probe_out);

const char* sc_lbm_last_error(sc_lbm_t h);
int sc_lbm_destroy(sc_lbm_t h);

/* ------------------------------------------------------------ no-alloc form
 * The paper has no counterpart to this call: it is a library facility.
 *
 * The per-cell quadrature mean and standard deviation of sc_lbm_moments
 * (same FP64 arithmetic, nodes in order) for a per-node field the caller
 * already holds, with no handle, no workspace and no device allocation.
 * For callers that cannot allocate device memory where they need the
 * statistics: a process whose free HBM is already reserved by another
 * allocator (a caching allocator or a serving pool that takes the device's
 * memory up front, where cudaMalloc fails or forces a cache flush), or code
 * on a latency-critical stream, where cudaMalloc / cudaFree would
 * synchronise the device.  It calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *
 * The weights travel by value as a kernel parameter (8 KB).  The one piece
 * of scratch, a counter of non-finite inputs, is one 8-byte word of a
 * fixed file-scope device array (256-byte aligned) held by every GPU that
 * loads the library until the process exits; its size does not depend on
 * the request.  The first call on each device (with that device current)
 * looks up its address and the device's SM count and must not be made
 * inside a stream capture; every later call issues only a memset, one
 * kernel and, with d_nonfinite, a device-to-device copy on `stream`, so it
 * may be captured into a CUDA graph (the graph keeps the weights it was
 * captured with).  Every call shares the counter and clears it at its
 * start: calls whose device work overlaps (unordered streams, several host
 * threads) race on it.
 *
 * d_field: device double [n_nodes][n_cells], Q_j(c) of node j at cell c;
 * weights: host double [n_nodes], the quadrature weights a_j (their sum must
 * be positive and finite), read during the call only (the array may be
 * reused as soon as the call returns);
 * d_mean, d_stdev: device double [n_cells] outputs,
 *   mean = sum_j a_j Q_j / sum_j a_j,
 *   std  = sqrt(max(sum_j a_j Q_j^2 / sum_j a_j - mean^2, 0));
 * d_nonfinite: device unsigned long long or NULL, receives the count of
 * non-finite Q_j(c); stream: CUDA stream (NULL = legacy default stream); the
 * call is asynchronous on it.  err: host buffer of err_len bytes or NULL,
 * receives a message on failure.
 * Returns SC_ERR_SCRATCH when n_nodes > SC_NOALLOC_MAX_NODES, SC_ERR_ARG for
 * other invalid arguments, SC_ERR_CUDA when a CUDA call fails.             */
#define SC_NOALLOC_MAX_NODES 1024
int sc_lbm_quad_moments_noalloc(const double* d_field, int n_nodes, long long n_cells,
                                const double* weights, double* d_mean, double* d_stdev,
                                unsigned long long* d_nonfinite, void* stream, char* err,
                                size_t err_len);

#ifdef __cplusplus
}
#endif
#endif /* SCLBM_H */
