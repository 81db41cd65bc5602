// api.cu -- the C ABI of libsclbm (include/sclbm.h): validation, workspace
// layout, the handle, and the host-side driving of the CUDA kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sclbm_internal.h"

using namespace sclbm;

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxProbes = 256;
constexpr long long kSpinLimit = 1LL << 26;  // bounded barrier polls (~seconds)

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

size_t storage_bytes(int precision) {
  switch (precision) {
    case SC_P_FP64_PLAIN: return 8;
    case SC_P_FP32_SHIFT: return 4;
    default: return 2;
  }
}

// Offsets of every buffer inside the caller's workspace.
struct DomLayout {
  int nq = 0, P = 0;
  long long ncell = 0, pitch = 0;
  size_t guard = 0;
  long long nb_max = 0;
  size_t flags = 0, link = 0, cls = 0, bcell = 0, ltab = 0, uin_f = 0, uin_d = 0, g = 0, g2 = 0, bout = 0, ab = 0;
  size_t abf = 0;  // [nq][gpc_pair_pad(P) / 2] float4 (hi_a, hi_a+1, lo_a, lo_a+1) of a_j Phi(Z_j)
  size_t avg = 0;  // time-averaged |u| accumulators [nq][ncell] (FP64), when configured
};
struct Layout {
  size_t hdr = 0, probes = 0;
  size_t st_mean = 0, st_std = 0, st_coef = 0, st_prof = 0, st_pnodes = 0;
  size_t q_phi = 0, q_cells = 0, q_k = 0;  // gPC quantile scratch (gpc_degree >= 0)
  DomLayout dom[kMaxDomains];
  size_t total = 0;
};

struct Header {  // first 256 bytes of the workspace
  unsigned long long check_count;
  unsigned int err;
  unsigned int bar_count;
  unsigned int bar_gen;
};

int validate(const sc_lbm_config* c, std::string& why) {
  if (!c) { why = "null config"; return SC_ERR_ARG; }
  if (c->n_domains < 1 || c->n_domains > kMaxDomains || !c->domains) {
    why = "n_domains must be 1.." + std::to_string(kMaxDomains);
    return SC_ERR_ARG;
  }
  if (!(c->tau0 > 0.5)) { why = "tau0 must exceed 1/2"; return SC_ERR_ARG; }
  if (c->c_smag < 0) { why = "c_smag must be >= 0"; return SC_ERR_ARG; }
  if (c->n_inputs < 1 || c->n_inputs > 3) { why = "n_inputs must be 1..3"; return SC_ERR_ARG; }
  for (int k = 0; k < c->n_inputs; ++k) {
    if (c->inputs[k] < SC_IN_SPEED_REL || c->inputs[k] > SC_IN_ANGLE_DEG) {
      why = "bad input kind";
      return SC_ERR_ARG;
    }
    if (c->quad_rule == SC_Q_GH) {
      if (!(c->hi[k] > 0.0)) { why = "normal inputs need a standard deviation hi > 0"; return SC_ERR_ARG; }
    } else if (!(c->hi[k] > c->lo[k])) {
      why = "input range must have hi > lo";
      return SC_ERR_ARG;
    }
  }
  if (c->quad_rule != SC_Q_GL && c->quad_rule != SC_Q_CC_SMOLYAK && c->quad_rule != SC_Q_GH) {
    why = "bad quad_rule";
    return SC_ERR_ARG;
  }
  if (c->profile != SC_PROFILE_POWER && c->profile != SC_PROFILE_LOG) { why = "bad profile"; return SC_ERR_ARG; }
  if (c->profile == SC_PROFILE_LOG && !(c->z0 > 0.0)) { why = "log profile needs z0 > 0"; return SC_ERR_ARG; }
  if (c->precision < SC_P_FP64_PLAIN || c->precision > SC_P_FP16_STORE) { why = "bad precision"; return SC_ERR_ARG; }
  if (c->ramp_steps < 0 || c->ramp_steps > 10000000) { why = "bad ramp_steps"; return SC_ERR_ARG; }
  if (c->gpc_degree > 8) { why = "gpc_degree too large"; return SC_ERR_UNSUPPORTED; }
  if (c->collision != SC_COLL_BGK && c->collision != SC_COLL_RR) { why = "bad collision"; return SC_ERR_ARG; }
  if (c->time_average != 0 && c->time_average != 1) { why = "time_average must be 0 or 1"; return SC_ERR_ARG; }
  if (c->node_begin < 0 || c->node_count < 0) { why = "node range must be non-negative"; return SC_ERR_ARG; }
  if (c->gpc_degree >= 0 && hn_gpc_size(c->n_inputs, c->gpc_degree) > kMaxGpcP) {
    why = "gPC basis larger than " + std::to_string(kMaxGpcP);
    return SC_ERR_UNSUPPORTED;
  }
  for (int d = 0; d < c->n_domains; ++d) {
    const sc_domain_desc& D = c->domains[d];
    if (D.nx < 1 || D.ny < 1 || D.nz < 1) { why = "domain sizes must be positive"; return SC_ERR_ARG; }
    if (((long long)D.nx * D.ny * D.nz + kRun) * 19 >= (1LL << 31)) {
      why = "domain too large (19 populations per node must stay below 2^31)";
      return SC_ERR_UNSUPPORTED;
    }
    for (int a = 0; a < 3; ++a) {
      const bool lo = D.bc[2 * a] == SC_BC_PERIODIC, hi = D.bc[2 * a + 1] == SC_BC_PERIODIC;
      if (lo != hi) { why = "periodic faces come in pairs"; return SC_ERR_ARG; }
    }
    for (int f = 0; f < 6; ++f) {
      if (D.bc[f] < SC_BC_VELOCITY || D.bc[f] > SC_BC_PERIODIC) { why = "bad face kind"; return SC_ERR_ARG; }
      if (D.bc[f] == SC_BC_OUTFLOW && f != 1) {
        why = "OUTFLOW is supported on face 1 (+x) only";
        return SC_ERR_UNSUPPORTED;
      }
    }
    if (D.quad_level < 1) { why = "quad_level must be >= 1"; return SC_ERR_ARG; }
    if (!(D.disk_radius >= 0.0) || !std::isfinite(D.disk_radius)) {
      why = "disk_radius must be finite and >= 0";
      return SC_ERR_ARG;
    }
    if (D.disk_radius > 0.0 && D.bc[1] == SC_BC_OUTFLOW) {
      why = "a circular domain (disk_radius > 0) takes no OUTFLOW face";
      return SC_ERR_UNSUPPORTED;
    }
  }
  return SC_OK;
}

int node_count(const sc_lbm_config* c, int d, std::vector<double>* Z, std::vector<double>* w) {
  std::vector<double> z, ww;
  int rc = hn_quadrature(c->quad_rule, c->n_inputs, c->domains[d].quad_level, c->lo, c->hi, z, ww);
  if (rc) return -1;
  if (Z) *Z = z;
  if (w) *w = ww;
  return (int)ww.size();
}

// The collocation nodes a handle runs: [node_begin, node_begin + node_count)
// of the full rule (node_count 0: to the end).  Ranks of a sharded ensemble
// each run one such range and add their moment sums.
int shard_nodes(const sc_lbm_config* c, int d, std::vector<double>* Z, std::vector<double>* w) {
  std::vector<double> z, ww;
  const int n = node_count(c, d, &z, &ww);
  if (n < 0) return -1;
  const int b = c->node_begin, cnt = c->node_count > 0 ? c->node_count : n - c->node_begin;
  if (b < 0 || b >= n || cnt < 1 || b + cnt > n) return -1;
  if (Z) Z->assign(z.begin() + (size_t)b * c->n_inputs, z.begin() + (size_t)(b + cnt) * c->n_inputs);
  if (w) w->assign(ww.begin() + b, ww.begin() + b + cnt);
  return cnt;
}

int plan(const sc_lbm_config* c, Layout& L, std::string& why) {
  int rc = validate(c, why);
  if (rc) return rc;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  L.hdr = take(sizeof(Header));
  L.probes = take(sizeof(int32_t) * 2 * kMaxProbes);
  const size_t sb = storage_bytes(c->precision);
  const int P = c->gpc_degree >= 0 ? hn_gpc_size(c->n_inputs, c->gpc_degree) : 0;
  long long max_cell = 0;
  int max_nz = 0, max_nq = 0;
  for (int d = 0; d < c->n_domains; ++d) {
    const sc_domain_desc& D = c->domains[d];
    DomLayout& M = L.dom[d];
    M.nq = shard_nodes(c, d, nullptr, nullptr);
    if (M.nq < 0) { why = "node range outside the quadrature rule"; return SC_ERR_ARG; }
    if (M.nq < 1) { why = "quadrature level not supported"; return SC_ERR_ARG; }
    if (M.nq > SC_MAX_NODES) { why = "too many collocation nodes"; return SC_ERR_UNSUPPORTED; }
    M.P = P;
    M.ncell = (long long)D.nx * D.ny * D.nz;
    M.flags = take((size_t)M.ncell);
    M.link = take(sizeof(LinkWord) * (size_t)M.ncell);
    M.cls = take((size_t)M.ncell);
    // listed cells lie on faces of kind OUTFLOW, PERIODIC or FREE_SLIP
    const long long area[3] = {(long long)D.ny * D.nz, (long long)D.nx * D.nz, (long long)D.nx * D.ny};
    M.nb_max = 0;
    for (int f = 0; f < 6; ++f)
      if (D.bc[f] == SC_BC_OUTFLOW || D.bc[f] == SC_BC_PERIODIC || D.bc[f] == SC_BC_FREE_SLIP)
        M.nb_max += area[f >> 1];
    M.nb_max = std::min(M.nb_max, M.ncell);
    M.bcell = take(sizeof(int32_t) * (size_t)M.nb_max);
    M.ltab = take(sizeof(ListedLinks) * (size_t)M.nb_max);
    M.uin_f = take(16 * (size_t)M.nq * D.nz);
    M.uin_d = take(24 * (size_t)M.nq * D.nz);
    M.pitch = (M.ncell + kRun - 1) / kRun * kRun;
    // guard zones around the population array: the staged odd-level loads
    // read row windows up to nx*ny + nx + 16 bytes outside a row
    M.guard = align_up(sb * ((size_t)D.nx * D.ny + D.nx + kRun + 64));
    off = align_up(off + M.guard);
    M.g = take(sb * kQ * (size_t)M.pitch * M.nq);
    off = align_up(off + M.guard);
    if (c->precision == SC_P_FP64_PLAIN) M.g2 = take(sb * kQ * (size_t)M.pitch * M.nq);
    else M.bout = take(sizeof(float) * 5 * (size_t)D.nz * D.ny * M.nq);
    M.ab = take(sizeof(double) * (size_t)M.nq * (P + 1));
    M.abf = take(2 * sizeof(float) * (size_t)M.nq * (size_t)(P > 0 ? gpc_pair_pad(P) : 2));
    if (c->time_average) M.avg = take(sizeof(double) * (size_t)M.nq * (size_t)M.ncell);
    max_cell = std::max(max_cell, M.ncell);
    max_nz = std::max(max_nz, D.nz);
    max_nq = std::max(max_nq, M.nq);
  }
  L.st_mean = take(sizeof(double) * (size_t)max_cell);
  L.st_std = take(sizeof(double) * (size_t)max_cell);
  L.st_coef = take(sizeof(double) * (size_t)max_cell * P);
  L.st_prof = take(sizeof(double) * 4 * (size_t)kMaxProbes * max_nz);
  L.st_pnodes = take(sizeof(float) * (size_t)kMaxProbes * max_nq * max_nz);
  if (P > 0) {
    L.q_phi = take(sizeof(double) * (size_t)SC_QUANTILE_MAX_SAMPLES * P);
    L.q_cells = take(sizeof(int32_t) * (size_t)SC_QUANTILE_MAX_CELLS);
    L.q_k = take(sizeof(int32_t) * (size_t)SC_QUANTILE_MAX_Q);
  }
  L.total = off;
  return SC_OK;
}

// ------------------------------------------------------------ tiny JSON cache
std::string tune_key(const sc_lbm_config* c, const char* gpu) {
  std::string k = std::string(gpu) + "|p" + std::to_string(c->precision) + "|s" +
                  std::to_string(c->c_smag > 0 ? 1 : 0);
  for (int d = 0; d < c->n_domains; ++d) {
    const sc_domain_desc& D = c->domains[d];
    k += "|" + std::to_string(D.nx) + "x" + std::to_string(D.ny) + "x" + std::to_string(D.nz) +
         "n" + std::to_string(D.quad_level);
  }
  return k;
}

std::map<std::string, std::vector<int>> read_cache(const char* path) {
  std::map<std::string, std::vector<int>> m;
  if (!path) return m;
  FILE* fh = fopen(path, "r");
  if (!fh) return m;
  std::string s;
  char buf[4096];
  size_t got;
  while ((got = fread(buf, 1, sizeof buf, fh)) > 0) s.append(buf, got);
  fclose(fh);
  size_t pos = 0;
  while (true) {
    size_t q0 = s.find('"', pos);
    if (q0 == std::string::npos) break;
    size_t q1 = s.find('"', q0 + 1);
    if (q1 == std::string::npos) break;
    std::string key = s.substr(q0 + 1, q1 - q0 - 1);
    size_t b0 = s.find('[', q1), b1 = s.find(']', q1);
    if (b0 == std::string::npos || b1 == std::string::npos) break;
    std::vector<int> v;
    std::string body = s.substr(b0 + 1, b1 - b0 - 1);
    char* p = &body[0];
    while (*p) {
      char* e;
      long x = strtol(p, &e, 10);
      if (e == p) { ++p; continue; }
      v.push_back((int)x);
      p = e;
    }
    m[key] = v;
    pos = b1 + 1;
  }
  return m;
}

void write_cache(const char* path, const std::map<std::string, std::vector<int>>& m) {
  if (!path) return;
  std::string tmp = std::string(path) + ".tmp";
  FILE* fh = fopen(tmp.c_str(), "w");
  if (!fh) return;
  fprintf(fh, "{\n");
  size_t k = 0;
  for (const auto& kv : m) {
    fprintf(fh, "  \"%s\": [", kv.first.c_str());
    for (size_t t = 0; t < kv.second.size(); ++t) fprintf(fh, "%s%d", t ? ", " : "", kv.second[t]);
    fprintf(fh, "]%s\n", ++k < m.size() ? "," : "");
  }
  fprintf(fh, "}\n");
  fclose(fh);
  rename(tmp.c_str(), path);
}

uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ULL) {
  const unsigned char* p = (const unsigned char*)data;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ULL;
  }
  return h;
}

}  // namespace

// ======================================================================= handle
struct sc_lbm_s {
  sc_lbm_config cfg;
  std::vector<sc_domain_desc> doms;
  std::vector<std::vector<int32_t>> boxes;
  Layout L;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t stream = nullptr;
  StepParams P;
  std::vector<double> wsum;
  std::vector<int> nq;
  std::vector<std::vector<double>> Z;         // collocation nodes per domain
  std::vector<std::vector<uint8_t>> flags;    // solid flags per domain (host copy)
  int gpcP = 0;
  sc_lbm_tuning tune;
  long long steps = 0, launches = 0;
  long long avg_samples = 0;                  // samples in the time-average accumulators
  const double* avg_read = nullptr;           // set while the moments read the time average
  std::string err;
  cudaGraphExec_t graph = nullptr;
  // the adjoint's sweeps captured as one graph, replayed while its
  // arguments (domain, step and checkpoint counts, workspace) stay the same
  cudaGraphExec_t adj_graph = nullptr;
  std::vector<long long> adj_key;
  int graph_len = 0;
  Wind<float> graph_wind{};                   // the inflow factor the graph was captured with
  // time-varying inflow (empty: steady): speed factors, continuous
  // direction offsets (degrees), levels per target, interpolation levels
  std::vector<double> series_speed, series_dir;
  long long series_per = 1, series_interp = 0;
  int persist_grid = 0;
  int never_arrive = 0;
  long long spin_limit = kSpinLimit;
  int tma_ok = 0;  // every domain's rows meet the 16-byte alignment of bulk copies
  Header* hdr() const { return reinterpret_cast<Header*>(ws + L.hdr); }
};

namespace {

// NVTX range for the duration of a scope (named in profiler timelines; a
// no-op when no tool is attached).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

int fail(sc_lbm_t h, int rc, const std::string& why) {
  if (h) h->err = why;
  return rc;
}

int cuda_fail(sc_lbm_t h, cudaError_t e, const char* where) {
  if (h) h->err = std::string(where) + ": " + cudaGetErrorString(e);
  return SC_ERR_CUDA;
}

#define CK(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);         \
  } while (0)

// Whether the two-cells-per-thread kernels can run: 16-bit storage, the BGK
// collision and an even nx in every domain (the first cell of a pair then
// sits at an even index, and each pair of populations is one aligned word).
bool pairs_ok(const sc_lbm_t h) {
  if (h->cfg.collision == SC_COLL_RR) return false;
  if (h->cfg.precision != SC_P_BF16_STORE && h->cfg.precision != SC_P_FP16_STORE) return false;
  for (int d = 0; d < h->P.n_domains; ++d)
    if (h->P.dom[d].nx % 2) return false;
  return true;
}

void apply_tiling(sc_lbm_t h) {
  StepParams& P = h->P;
  P.bx = h->tune.block_x;
  P.by = h->tune.block_y;
  P.bz = h->tune.slab_z;
  P.order = h->tune.tile_order;
  long long begin = 0, bbegin = 0, rbegin = 0;
  for (int d = 0; d < P.n_domains; ++d) {
    DevDomain& D = P.dom[d];
    D.tiles_x = (D.nx + P.bx - 1) / P.bx;
    D.tiles_y = (D.ny + P.by - 1) / P.by;
    D.tiles_z = (D.nz + P.bz - 1) / P.bz;
    D.tiles_per_node = D.tiles_x * D.tiles_y * D.tiles_z;
    D.tile_begin = begin;
    begin += D.tiles_per_node * D.nodes;
    D.bitem_begin = bbegin;
    bbegin += D.nb * D.nodes;
    D.runs_per_node = D.pitch / kRun;
    D.run_begin = rbegin;
    rbegin += D.runs_per_node * D.nodes;
  }
  P.total_tiles = begin;
  P.total_bitems = bbegin;
  P.total_runs = rbegin;
  P.tma = (h->tune.variant == 1 && h->tma_ok && h->tune.exec_mode != SC_EXEC_PERSISTENT) ? 1 : 0;
  P.even85 = h->tune.variant == 2 ? 1 : 0;
  P.odd85 = (h->tune.variant == 2 || h->tune.variant == 3) ? 1 : 0;
  // 16-bit storage with the BGK collision, every domain's rows pairing up
  // (even nx): two x-adjacent cells per thread on the even level in variants
  // 0 (kernel sized for 2 resident blocks) and 3 (3 blocks)
  const bool pairs = pairs_ok(h) && !P.tma;
  P.even_pair = !pairs ? 0 : h->tune.variant == 0 ? 2 : h->tune.variant == 3 ? 3 : 0;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    h->graph_len = 0;
  }
  h->persist_grid = 0;
}

int check_tuning(const sc_lbm_tuning& t) {
  // the step kernels are compiled for at most 256 threads per block
  if (t.block_x < 32 || t.block_x % 32 || t.block_y < 1 || t.block_x * t.block_y > 256) return SC_ERR_ARG;
  if (t.slab_z < 1 || t.slab_z > 4096) return SC_ERR_ARG;
  if (t.tile_order < 0 || t.tile_order > 1) return SC_ERR_ARG;
  if (t.exec_mode < SC_EXEC_LAUNCH || t.exec_mode > SC_EXEC_PERSISTENT) return SC_ERR_ARG;
  if (t.graph_steps < 1 || t.graph_steps > 100000) return SC_ERR_ARG;
  if (t.variant < 0 || t.variant > 3) return SC_ERR_ARG;
  return SC_OK;
}

int reset_state(sc_lbm_t h) {
  int rc = launch_init_equilibrium(h->P, h->cfg.precision, h->stream);
  if (rc) return cuda_fail(h, (cudaError_t)rc, "init kernel");
  ++h->launches;
  CK(cudaMemsetAsync(h->ws + h->L.hdr, 0, sizeof(Header), h->stream));
  h->steps = 0;
  return SC_OK;
}

// Inflow factor of ramp r, speed factor s and direction offset d (degrees).
// No offset gives exactly (1, 0, r s), the steady form.
Wind<double> wind_of(double r, double s, double d) {
  const double rad = d * (M_PI / 180.0);
  return Wind<double>{cos(rad), sin(rad), r * s};
}

// Inflow factor of time level m: start-up ramp times the series' speed
// factor, turned by its direction offset.
Wind<double> wind_at(const sc_lbm_t h, long long m) {
  double s = 1.0, d = 0.0;
  if (!h->series_speed.empty())
    hn_series_at((int)h->series_speed.size(), h->series_speed.data(), h->series_dir.data(), h->series_per,
                 h->series_interp, m, &s, &d);
  return wind_of(hn_ramp(h->cfg.ramp_steps, m), s, d);
}

Wind<float> to_float(const Wind<double>& w) { return Wind<float>{(float)w.cos_d, (float)w.sin_d, (float)w.scale}; }

// Factors of a launch that advances level lvl: pulls at lvl, pushes at lvl + 1.
void set_winds(const sc_lbm_t h, StepParams& P, long long lvl) {
  P.wpd = wind_at(h, lvl);
  P.wqd = wind_at(h, lvl + 1);
  P.wp = to_float(P.wpd);
  P.wq = to_float(P.wqd);
}

// The same factor at both ends (steps inside a stretch of constant inflow).
void set_winds(StepParams& P, const Wind<double>& w) {
  P.wpd = P.wqd = w;
  P.wp = P.wq = to_float(w);
}

// First level after m at which the inflow factor may change.
long long next_change(const sc_lbm_t h, long long m) {
  return hn_wind_next_change(h->cfg.ramp_steps, (int)h->series_speed.size(), h->series_per, h->series_interp, m);
}

// n steps with one launch each, starting at time level `start`
int run_launches(sc_lbm_t h, long long start, int n) {
  for (int s = 0; s < n; ++s) {
    const long long lvl = start + s;
    const int parity = (int)(lvl & 1);
    StepParams P = h->P;
    set_winds(h, P, lvl);
    int rc = h->cfg.collision == SC_COLL_RR ? rr::launch_aa_step(P, h->cfg.precision, h->stream, parity)
                                            : launch_aa_step(P, h->cfg.precision, h->stream, parity);
    if (rc) return cuda_fail(h, (cudaError_t)rc, "aa_step launch");
    h->launches += parity && h->P.tma ? 2 : 1;  // TMA odd levels: bulk + boundary kernels
  }
  return SC_OK;
}

// Replays of a captured graph of G steps (even/odd pairs, G even) starting
// at an even time level, over levels [t, t + n) of constant inflow factor w.
// The graph holds w in its launch parameters; it is captured again when a
// stretch with another factor comes.
int run_graph(sc_lbm_t h, long long t, int n, const Wind<double>& w) {
  const int G = h->tune.graph_steps + (h->tune.graph_steps & 1);
  if (!h->stream) return run_launches(h, t, n);  // capture needs a non-default stream
  if ((t & 1) && n > 0) {
    int rc = run_launches(h, t, 1);
    if (rc) return rc;
    ++t;
    --n;
  }
  const int reps = n / G;
  if (reps == 0) return run_launches(h, t, n);
  const Wind<float> wf = to_float(w);
  const bool same = h->graph_wind.cos_d == wf.cos_d && h->graph_wind.sin_d == wf.sin_d &&
                    h->graph_wind.scale == wf.scale;
  if (!h->graph || h->graph_len != G || !same) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    h->graph_len = 0;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = 0;
    StepParams P = h->P;
    set_winds(P, w);
    for (int s = 0; s < G && !rc; ++s)
      rc = h->cfg.collision == SC_COLL_RR ? rr::launch_aa_step(P, h->cfg.precision, h->stream, s & 1)
                                          : launch_aa_step(P, h->cfg.precision, h->stream, s & 1);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(h, (cudaError_t)rc, "graph capture launch");
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    h->graph_len = G;
    h->graph_wind = wf;
  }
  for (int r = 0; r < reps; ++r) {
    Range rg("graph replay");
    CK(cudaGraphLaunch(h->graph, h->stream));
    h->launches += G + (h->P.tma ? G / 2 : 0);  // TMA odd levels launch two kernels
  }
  return run_launches(h, t + (long long)reps * G, n - reps * G);
}

// Persistent launches over levels [t, t + n) of constant inflow factor w.
int run_persistent(sc_lbm_t h, long long t, int n, const Wind<double>& w) {
  if (!h->persist_grid) {
    int grid = 0;
    int rc = h->cfg.collision == SC_COLL_RR ? rr::aa_persistent_max_grid(h->P, h->cfg.precision, &grid)
                                            : aa_persistent_max_grid(h->P, h->cfg.precision, &grid);
    if (rc || grid < 1) return cuda_fail(h, (cudaError_t)(rc ? rc : cudaErrorInvalidConfiguration), "occupancy");
    h->persist_grid = (int)std::min<long long>(grid, h->P.total_tiles);
  }
  const int chunk = 500;
  for (int done = 0; done < n;) {
    const int k = std::min(chunk, n - done);
    StepParams P = h->P;
    set_winds(P, w);
    P.n_steps = k;
    P.n_host = (unsigned long long)(t + done);
    P.never_arrive = h->never_arrive;
    P.spin_limit = h->spin_limit;
    CK(cudaMemsetAsync(&h->hdr()->bar_count, 0, sizeof(unsigned int), h->stream));
    int rc = h->cfg.collision == SC_COLL_RR
                 ? rr::launch_aa_persistent(P, h->cfg.precision, h->stream, h->persist_grid)
                 : launch_aa_persistent(P, h->cfg.precision, h->stream, h->persist_grid);
    if (rc) return cuda_fail(h, (cudaError_t)rc, "persistent launch");
    ++h->launches;
    done += k;
  }
  return SC_OK;
}

int run_plain(sc_lbm_t h, int n) {
  for (int d = 0; d < h->P.n_domains; ++d)
    for (int j = 0; j < h->P.dom[d].nodes; ++j) {
      StepParams P = h->P;
      P.plain_domain = d;
      P.plain_node = j;
      for (int s = 0; s < n; ++s) {
        set_winds(h, P, h->steps + s);
        int rc = h->cfg.collision == SC_COLL_RR
                     ? rr::launch_plain_step(P, (unsigned long long)(h->steps + s), h->stream)
                     : launch_plain_step(P, (unsigned long long)(h->steps + s), h->stream);
        if (rc) return cuda_fail(h, (cudaError_t)rc, "plain_step launch");
        ++h->launches;
      }
    }
  return SC_OK;
}

// AA steps from level h->steps: stretches over which the inflow factor is
// constant go to the tuned execution mode (graph replays, persistent
// launches or plain launches); a step whose two factors differ (start-up
// ramp, a move between series targets) is launched alone with both.
int run_aa(sc_lbm_t h, int n) {
  long long t = h->steps;
  while (n > 0) {
    const long long e = next_change(h, t);  // W(m) = W(t) for m in [t, e)
    const long long c = std::min<long long>(n, e - 1 - t);  // steps t .. t + c - 1 see W(t) at both ends
    int rc;
    if (c <= 0) {
      rc = run_launches(h, t, 1);
      t += 1;
      n -= 1;
    } else {
      const Wind<double> w = wind_at(h, t);
      if (h->tune.exec_mode == SC_EXEC_GRAPH) rc = run_graph(h, t, (int)c, w);
      else if (h->tune.exec_mode == SC_EXEC_PERSISTENT) rc = run_persistent(h, t, (int)c, w);
      else rc = run_launches(h, t, (int)c);
      t += c;
      n -= (int)c;
    }
    if (rc) return rc;
  }
  return SC_OK;
}

int do_steps(sc_lbm_t h, int n) {
  if (n <= 0) return SC_OK;
  int rc;
  if (h->cfg.precision == SC_P_FP64_PLAIN) rc = run_plain(h, n);
  else rc = run_aa(h, n);
  if (rc == SC_OK) h->steps += n;
  return rc;
}

int read_err(sc_lbm_t h, unsigned* bits) {
  CK(cudaStreamSynchronize(h->stream));
  unsigned v = 0;
  CK(cudaMemcpy(&v, &h->hdr()->err, sizeof v, cudaMemcpyDeviceToHost));
  if (v) CK(cudaMemset(&h->hdr()->err, 0, sizeof(unsigned)));
  *bits = v;
  return SC_OK;
}

// Kernel parameters with the host's time level (observables need its parity
// and, at odd levels, its inflow factor).
StepParams params_now(sc_lbm_t h) {
  StepParams P = h->P;
  P.n_host = (unsigned long long)h->steps;
  set_winds(h, P, h->steps);
  return P;
}

int err_status(sc_lbm_t h, unsigned bits) {
  if (bits & kErrTimeout) return fail(h, SC_ERR_TIMEOUT, "a bounded device-side wait expired");
  if (bits & kErrDiverged) return fail(h, SC_ERR_DIVERGED, "non-finite or non-positive density");
  return SC_OK;
}

}  // namespace

// ======================================================================= C ABI
extern "C" {

int sc_lbm_workspace_size(const sc_lbm_config* cfg, size_t* bytes_out) {
  if (!bytes_out) return SC_ERR_ARG;
  Layout L;
  std::string why;
  int rc = plan(cfg, L, why);
  if (rc) return rc;
  *bytes_out = L.total;
  return SC_OK;
}

int sc_lbm_quadrature(const sc_lbm_config* cfg, int domain, int* n_nodes, double* Z, double* w,
                      int cap) {
  std::string why;
  if (!n_nodes || validate(cfg, why)) return SC_ERR_ARG;
  if (domain < 0 || domain >= cfg->n_domains) return SC_ERR_ARG;
  std::vector<double> z, ww;
  int n = node_count(cfg, domain, &z, &ww);
  if (n < 1) return SC_ERR_ARG;
  *n_nodes = n;
  if (!Z) return SC_OK;
  if (cap < n || !w) return SC_ERR_ARG;
  memcpy(Z, z.data(), sizeof(double) * z.size());
  memcpy(w, ww.data(), sizeof(double) * ww.size());
  return SC_OK;
}

int sc_lbm_geometry(const sc_lbm_config* cfg, int domain, uint8_t* flags) {
  std::string why;
  if (!flags || validate(cfg, why)) return SC_ERR_ARG;
  if (domain < 0 || domain >= cfg->n_domains) return SC_ERR_ARG;
  std::vector<uint8_t> f;
  int rc = hn_geometry(cfg->domains[domain], f);
  if (rc) return rc;
  memcpy(flags, f.data(), f.size());
  return SC_OK;
}

int sc_lbm_probe_columns(const sc_lbm_config* cfg, int domain, int n, int32_t* xy) {
  std::string why;
  if (!xy || n < 0 || validate(cfg, why)) return SC_ERR_ARG;
  if (domain < 0 || domain >= cfg->n_domains) return SC_ERR_ARG;
  std::vector<uint8_t> f;
  int rc = hn_geometry(cfg->domains[domain], f);
  if (rc) return rc;
  return hn_probe_columns(cfg->domains[domain], f.data(), n, xy);
}

int sc_lbm_probe_points(const sc_lbm_config* cfg, int domain, int n, int32_t* xyz) {
  std::string why;
  if (!xyz || n < 0 || validate(cfg, why)) return SC_ERR_ARG;
  if (domain < 0 || domain >= cfg->n_domains) return SC_ERR_ARG;
  std::vector<uint8_t> f;
  int rc = hn_geometry(cfg->domains[domain], f);
  if (rc) return rc;
  return hn_probe_points(cfg->domains[domain], f.data(), n, xyz);
}

int sc_lbm_init(const sc_lbm_config* cfg, void* d_ws, size_t bytes, void* cuda_stream,
                const uint8_t* const* flags_host, sc_lbm_t* out) {
  if (!out) return SC_ERR_ARG;
  *out = nullptr;
  Range range("sc_lbm_init");
  Layout L;
  std::string why;
  int rc = plan(cfg, L, why);
  if (rc) return rc;
  if (!d_ws || ((uintptr_t)d_ws % kAlign) != 0 || bytes < L.total) return SC_ERR_WORKSPACE;
  sc_lbm_t h = new (std::nothrow) sc_lbm_s();
  if (!h) return SC_ERR_ARG;
  h->cfg = *cfg;
  h->doms.assign(cfg->domains, cfg->domains + cfg->n_domains);
  h->boxes.resize(cfg->n_domains);
  for (int d = 0; d < cfg->n_domains; ++d) {
    const sc_domain_desc& D = cfg->domains[d];
    if (D.n_boxes > 0 && D.boxes) h->boxes[d].assign(D.boxes, D.boxes + 6 * D.n_boxes);
    h->doms[d].boxes = h->boxes[d].empty() ? nullptr : h->boxes[d].data();
  }
  h->cfg.domains = h->doms.data();
  h->L = L;
  h->ws = (char*)d_ws;
  h->ws_bytes = bytes;
  h->stream = (cudaStream_t)cuda_stream;
  const sc_lbm_config& c = h->cfg;
  StepParams& P = h->P;
  memset(&P, 0, sizeof P);
  P.n_domains = c.n_domains;
  P.tau0 = (float)c.tau0;
  P.tau0_d = c.tau0;
  P.smag18c2 = (float)(18.0 * c.c_smag * c.c_smag);
  P.smag18c2_d = 18.0 * c.c_smag * c.c_smag;
  P.csmag_on = c.c_smag > 0 ? 1 : 0;
  Header* H = h->hdr();
  P.err = &H->err;
  P.bar_count = &H->bar_count;
  P.bar_gen = &H->bar_gen;
  P.spin_limit = kSpinLimit;
  h->gpcP = c.gpc_degree >= 0 ? hn_gpc_size(c.n_inputs, c.gpc_degree) : 0;

  // host tables (kept alive until the stream is synchronised below)
  std::vector<std::vector<uint8_t>> flags(c.n_domains);
  std::vector<std::vector<LinkWord>> links(c.n_domains);
  std::vector<std::vector<int32_t>> bcells(c.n_domains);
  std::vector<std::vector<uint8_t>> classes(c.n_domains);
  std::vector<std::vector<ListedLinks>> ltabs(c.n_domains);
  std::vector<std::vector<int32_t>> ltab_words(c.n_domains);
  std::vector<std::vector<float>> uinf(c.n_domains);
  std::vector<std::vector<double>> uind(c.n_domains), abt(c.n_domains);
  std::vector<std::vector<float>> abft(c.n_domains);
  h->wsum.assign(c.n_domains, 0.0);
  h->nq.assign(c.n_domains, 0);
  for (int d = 0; d < c.n_domains; ++d) {
    const sc_domain_desc& D = c.domains[d];
    const DomLayout& M = L.dom[d];
    if (flags_host && flags_host[d]) {
      flags[d].assign(flags_host[d], flags_host[d] + M.ncell);
      for (auto& v : flags[d]) v = v ? 1 : 0;
      hn_mark_mantle(D, flags[d]);
    } else {
      rc = hn_geometry(D, flags[d]);
      if (rc) { delete h; return rc; }
    }
    hn_link_words(D, flags[d].data(), links[d]);
    hn_boundary_cells(links[d], bcells[d]);
    hn_cell_classes(links[d], classes[d]);
    if ((long long)bcells[d].size() > L.dom[d].nb_max) {
      delete h;
      return SC_ERR_ARG;  // cannot happen: listed cells lie on the counted faces
    }
    hn_listed_links(D, flags[d].data(), links[d], bcells[d], L.dom[d].pitch, ltabs[d]);
    std::vector<double> Z, w;
    shard_nodes(&c, d, &Z, &w);
    const int nq = (int)w.size();
    h->nq[d] = nq;
    h->Z.push_back(Z);
    double ws = 0.0;
    for (double v : w) ws += v;
    h->wsum[d] = ws;
    const double H = c.H_ref > 0 ? c.H_ref : (double)D.nz;
    uinf[d].assign((size_t)nq * D.nz * 4, 0.0f);
    uind[d].assign((size_t)nq * D.nz * 3, 0.0);
    abt[d].assign((size_t)nq * (h->gpcP + 1), 0.0);
    std::vector<double> phi(h->gpcP > 0 ? h->gpcP : 1);
    for (int j = 0; j < nq; ++j) {
      double xi = 0.0, al = c.alpha, th = c.angle_deg;
      double s[3] = {0, 0, 0};
      for (int t = 0; t < c.n_inputs; ++t) {
        const double zt = Z[(size_t)j * c.n_inputs + t];
        if (c.inputs[t] == SC_IN_SPEED_REL) xi = zt;
        else if (c.inputs[t] == SC_IN_ALPHA) al = zt;
        else th = zt;
        // basis coordinate: [-1, 1] (uniform inputs) or standard normal
        s[t] = c.quad_rule == SC_Q_GH ? (zt - c.lo[t]) / c.hi[t]
                                      : (2.0 * zt - c.lo[t] - c.hi[t]) / (c.hi[t] - c.lo[t]);
      }
      double* ud = &uind[d][(size_t)j * D.nz * 3];
      hn_inflow(D.nz, c.u_ref, xi, al, H, th, ud, c.profile, c.z0);
      for (int k = 0; k < D.nz; ++k)
        for (int a = 0; a < 3; ++a) uinf[d][((size_t)j * D.nz + k) * 4 + a] = (float)ud[3 * k + a];
      abt[d][(size_t)j * (h->gpcP + 1)] = w[j];
      if (h->gpcP > 0) {
        hn_gpc_basis(c.n_inputs, c.gpc_degree, s, phi.data(), c.quad_rule == SC_Q_GH);
        for (int a = 0; a < h->gpcP; ++a) abt[d][(size_t)j * (h->gpcP + 1) + 1 + a] = w[j] * phi[a];
      }
    }
    DevDomain& V = P.dom[d];
    V.nx = D.nx;
    V.ny = D.ny;
    V.nz = D.nz;
    V.nodes = nq;
    V.ncell = M.ncell;
    for (int f = 0; f < 6; ++f) V.bc[f] = D.bc[f];
    V.flags = (const uint8_t*)(h->ws + M.flags);
    V.link = (const LinkWord*)(h->ws + M.link);
    V.cls = (const uint8_t*)(h->ws + M.cls);
    V.bcell = (const int32_t*)(h->ws + M.bcell);
    V.ltab = (const int32_t*)(h->ws + M.ltab);
    V.lstride = M.nb_max;
    V.nb = (long long)bcells[d].size();
    V.uin_f = (const float4*)(h->ws + M.uin_f);
    V.uin_d = (const double*)(h->ws + M.uin_d);
    V.pitch = M.pitch;
    V.g = h->ws + M.g;
    V.g2 = c.precision == SC_P_FP64_PLAIN ? (void*)(h->ws + M.g2) : nullptr;
    V.bout = c.precision == SC_P_FP64_PLAIN ? nullptr : (float*)(h->ws + M.bout);
  }
  h->tma_ok = c.precision != SC_P_FP64_PLAIN;
  for (int d = 0; d < c.n_domains; ++d)
    if (c.domains[d].nx % (int)(16 / storage_bytes(c.precision)) != 0) h->tma_ok = 0;
  // default launch shape
  h->tune.variant = 0;
  h->tune.block_x = 64;
  h->tune.block_y = 2;
  h->tune.slab_z = 8;
  h->tune.tile_order = 1;
  h->tune.exec_mode = SC_EXEC_LAUNCH;
  h->tune.graph_steps = 50;
  apply_tiling(h);

  auto up = [&](size_t off, const void* src, size_t n) {
    return cudaMemcpyAsync(h->ws + off, src, n, cudaMemcpyHostToDevice, h->stream);
  };
  cudaError_t e = cudaSuccess;
  for (int d = 0; d < c.n_domains && e == cudaSuccess; ++d) {
    const DomLayout& M = L.dom[d];
    e = up(M.flags, flags[d].data(), flags[d].size());
    if (e == cudaSuccess) e = up(M.link, links[d].data(), sizeof(LinkWord) * links[d].size());
    if (e == cudaSuccess) e = up(M.cls, classes[d].data(), classes[d].size());
    if (e == cudaSuccess && !bcells[d].empty())
      e = up(M.bcell, bcells[d].data(), sizeof(int32_t) * bcells[d].size());
    if (e == cudaSuccess && !ltabs[d].empty()) {
      // transpose the records: word w of cell k at [w * nb_max + k]
      const size_t nbm = (size_t)M.nb_max, n = ltabs[d].size();
      ltab_words[d].assign(nbm * kListedWords, -1);
      for (size_t k = 0; k < n; ++k) {
        const int32_t* rec = reinterpret_cast<const int32_t*>(&ltabs[d][k]);
        for (int w = 0; w < kListedWords; ++w) ltab_words[d][(size_t)w * nbm + k] = rec[w];
      }
      e = up(M.ltab, ltab_words[d].data(), sizeof(int32_t) * ltab_words[d].size());
    }
    if (e == cudaSuccess) e = up(M.uin_f, uinf[d].data(), sizeof(float) * uinf[d].size());
    if (e == cudaSuccess) e = up(M.uin_d, uind[d].data(), sizeof(double) * uind[d].size());
    if (e == cudaSuccess) e = up(M.ab, abt[d].data(), sizeof(double) * abt[d].size());
    if (e == cudaSuccess && h->gpcP > 0) {
      // each a_j Phi_alpha(Z_j) as hi = fl32(v), lo = fl32(v - hi): 48 bits of
      // it; terms a, a + 1 share a float4 (hi_a, hi_a+1, lo_a, lo_a+1), rows
      // padded with zero terms to gpc_pair_pad(P)
      const int Pp = gpc_pair_pad(h->gpcP);
      std::vector<float>& f = abft[d];
      f.assign((size_t)2 * M.nq * Pp, 0.0f);
      for (int j = 0; j < M.nq; ++j)
        for (int a = 0; a < h->gpcP; ++a) {
          const double v = abt[d][(size_t)j * (h->gpcP + 1) + 1 + a];
          const float hi = (float)v;
          const size_t e = ((size_t)j * (Pp / 2) + a / 2) * 4 + (a & 1);
          f[e] = hi;
          f[e + 2] = (float)(v - (double)hi);
        }
      e = up(M.abf, f.data(), sizeof(float) * f.size());
    }
    if (e == cudaSuccess && M.avg)
      e = cudaMemsetAsync(h->ws + M.avg, 0, sizeof(double) * (size_t)M.nq * (size_t)M.ncell, h->stream);
    if (e == cudaSuccess && M.bout)
      e = cudaMemsetAsync(h->ws + M.bout, 0, sizeof(float) * 5 * (size_t)c.domains[d].nz * c.domains[d].ny * M.nq, h->stream);
  }
  if (e != cudaSuccess) {
    int r = cuda_fail(h, e, "upload");
    delete h;
    return r;
  }
  rc = reset_state(h);
  if (rc == SC_OK) {
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = cuda_fail(h, e, "init sync");
  }
  h->flags = std::move(flags);
  if (rc) {
    delete h;
    return rc;
  }
  *out = h;
  return SC_OK;
}

int sc_lbm_reset(sc_lbm_t h) {
  if (!h) return SC_ERR_ARG;
  return reset_state(h);
}

int sc_lbm_step(sc_lbm_t h, int n_steps) {
  if (!h || n_steps < 0) return SC_ERR_ARG;
  Range r("sc_lbm_step");
  return do_steps(h, n_steps);
}

int sc_lbm_moments(sc_lbm_t h, int domain, double* mean, double* stdev, const int32_t* probe_xy,
                   int n_p, double* prof, float* prof_nodes, double* gpc_coef, int out_host) {
  if (!h || domain < 0 || domain >= h->P.n_domains) return SC_ERR_ARG;
  Range r("sc_lbm_moments");
  if (n_p < 0 || n_p > kMaxProbes || (n_p > 0 && (!probe_xy || !prof))) return SC_ERR_ARG;
  if ((mean == nullptr) != (stdev == nullptr)) return SC_ERR_ARG;
  if (gpc_coef && h->gpcP == 0) return fail(h, SC_ERR_ARG, "gpc_degree < 0 in the configuration");
  const DevDomain& D = h->P.dom[domain];
  for (int p = 0; p < n_p; ++p) {
    const int x = probe_xy[2 * p], y = probe_xy[2 * p + 1];
    if (x < 0 || x >= D.nx || y < 0 || y >= D.ny) return fail(h, SC_ERR_ARG, "probe outside the domain");
  }
  const Layout& L = h->L;
  MomentArgs A;
  A.domain = domain;
  A.ab = (const double*)(h->ws + L.dom[domain].ab);
  A.abf = (const float4*)(h->ws + L.dom[domain].abf);
  A.nq = h->nq[domain];
  A.stride = h->gpcP + 1;
  A.P = gpc_coef ? h->gpcP : 0;
  A.wsum = h->wsum[domain];
  A.mean = out_host ? (mean ? (double*)(h->ws + L.st_mean) : nullptr) : mean;
  A.stdev = out_host ? (stdev ? (double*)(h->ws + L.st_std) : nullptr) : stdev;
  A.coef = out_host ? (gpc_coef ? (double*)(h->ws + L.st_coef) : nullptr) : gpc_coef;
  A.probes = (const int32_t*)(h->ws + L.probes);
  A.n_p = n_p;
  A.prof = out_host ? (double*)(h->ws + L.st_prof) : prof;
  A.prof_nodes = out_host ? (prof_nodes ? (float*)(h->ws + L.st_pnodes) : nullptr) : prof_nodes;
  A.avg = h->avg_read;
  A.avg_scale = h->avg_samples > 0 ? 1.0 / (double)h->avg_samples : 0.0;
  A.raw = 0;
  A.accumulate = 0;
  if (n_p > 0)
    CK(cudaMemcpyAsync(h->ws + L.probes, probe_xy, sizeof(int32_t) * 2 * n_p, cudaMemcpyHostToDevice,
                       h->stream));
  int rc = launch_moments(params_now(h), h->cfg.precision, A, h->stream);
  if (rc) return cuda_fail(h, (cudaError_t)rc, "moments launch");
  h->launches += (A.mean ? 1 : 0) + (n_p > 0 ? 1 : 0);
  if (!out_host) return SC_OK;
  const size_t nc = (size_t)D.ncell;
  if (mean) CK(cudaMemcpyAsync(mean, A.mean, sizeof(double) * nc, cudaMemcpyDeviceToHost, h->stream));
  if (stdev) CK(cudaMemcpyAsync(stdev, A.stdev, sizeof(double) * nc, cudaMemcpyDeviceToHost, h->stream));
  if (gpc_coef)
    CK(cudaMemcpyAsync(gpc_coef, A.coef, sizeof(double) * nc * h->gpcP, cudaMemcpyDeviceToHost, h->stream));
  if (n_p > 0) {
    CK(cudaMemcpyAsync(prof, A.prof, sizeof(double) * 4 * n_p * D.nz, cudaMemcpyDeviceToHost, h->stream));
    if (prof_nodes)
      CK(cudaMemcpyAsync(prof_nodes, A.prof_nodes, sizeof(float) * (size_t)n_p * A.nq * D.nz,
                         cudaMemcpyDeviceToHost, h->stream));
  }
  unsigned bits = 0;
  rc = read_err(h, &bits);
  if (rc) return rc;
  return err_status(h, bits);
}

int sc_lbm_moment_sums(sc_lbm_t h, int domain, double* d_s1, double* d_s2, double* d_gpc_sums,
                       int accumulate) {
  if (!h || !d_s1 || !d_s2 || domain < 0 || domain >= h->P.n_domains) return SC_ERR_ARG;
  if (accumulate != 0 && accumulate != 1) return fail(h, SC_ERR_ARG, "accumulate must be 0 or 1");
  Range r("sc_lbm_moment_sums");
  if (d_gpc_sums && h->gpcP == 0) return fail(h, SC_ERR_ARG, "gpc_degree < 0 in the configuration");
  MomentArgs A;
  A.domain = domain;
  A.ab = (const double*)(h->ws + h->L.dom[domain].ab);
  A.abf = (const float4*)(h->ws + h->L.dom[domain].abf);
  A.nq = h->nq[domain];
  A.stride = h->gpcP + 1;
  A.P = d_gpc_sums ? h->gpcP : 0;
  A.wsum = h->wsum[domain];
  A.mean = d_s1;
  A.stdev = d_s2;
  A.coef = d_gpc_sums;
  A.probes = nullptr;
  A.n_p = 0;
  A.prof = nullptr;
  A.prof_nodes = nullptr;
  A.avg = nullptr;
  A.avg_scale = 0.0;
  A.raw = 1;
  A.accumulate = accumulate;
  int rc = launch_moments(params_now(h), h->cfg.precision, A, h->stream);
  if (rc) return cuda_fail(h, (cudaError_t)rc, "moment sums launch");
  ++h->launches;
  return SC_OK;
}

int sc_lbm_rule_weight_sum(const sc_lbm_config* cfg, int domain, double* wsum) {
  std::string why;
  if (!wsum || validate(cfg, why)) return SC_ERR_ARG;
  if (domain < 0 || domain >= cfg->n_domains) return SC_ERR_ARG;
  std::vector<double> w;
  if (node_count(cfg, domain, nullptr, &w) < 1) return SC_ERR_ARG;
  double ws = 0.0;  // node order, as a handle over the whole rule sums it
  for (double v : w) ws += v;
  *wsum = ws;
  return SC_OK;
}

int sc_lbm_weight_sum(sc_lbm_t h, int domain, double* wsum) {
  if (!h || !wsum || domain < 0 || domain >= h->P.n_domains) return SC_ERR_ARG;
  *wsum = h->wsum[domain];
  return SC_OK;
}

int sc_lbm_moments_from_sums(sc_lbm_t h, int domain, const double* d_s1, const double* d_s2, double wsum,
                             double* d_mean, double* d_stdev) {
  if (!h || !d_s1 || !d_s2 || !d_mean || !d_stdev || domain < 0 || domain >= h->P.n_domains) return SC_ERR_ARG;
  if (!(wsum > 0.0)) return fail(h, SC_ERR_ARG, "weight sum must be positive");
  int rc = launch_finalize_moments(d_s1, d_s2, wsum, d_mean, d_stdev, h->P.dom[domain].ncell, h->stream);
  if (rc) return cuda_fail(h, (cudaError_t)rc, "finalize launch");
  ++h->launches;
  return SC_OK;
}

int sc_lbm_gpc_quantiles(sc_lbm_t h, int domain, const double* d_coef, int n_cells, const int32_t* cells,
                         int n_samples, const double* samples, int n_q, const double* q, double* d_out) {
  if (!h || domain < 0 || domain >= h->P.n_domains) return SC_ERR_ARG;
  if (h->gpcP == 0) return fail(h, SC_ERR_ARG, "gpc_degree < 0 in the configuration");
  if (n_cells < 0 || n_cells > SC_QUANTILE_MAX_CELLS || n_samples < 1 || n_samples > SC_QUANTILE_MAX_SAMPLES ||
      n_q < 1 || n_q > SC_QUANTILE_MAX_Q || !samples || !q || (n_cells > 0 && (!cells || !d_coef || !d_out)))
    return fail(h, SC_ERR_ARG, "quantiles: bad counts or null arrays");
  const DevDomain& D = h->P.dom[domain];
  for (int i = 0; i < n_cells; ++i)
    if (cells[i] < 0 || cells[i] >= D.ncell) return fail(h, SC_ERR_ARG, "quantiles: cell outside the domain");
  std::vector<int32_t> kidx((size_t)n_q);
  for (int i = 0; i < n_q; ++i) {
    if (!(q[i] >= 0.0 && q[i] <= 1.0)) return fail(h, SC_ERR_ARG, "quantiles: probabilities must lie in [0, 1]");
    const double k = std::ceil(q[i] * (double)n_samples);
    kidx[(size_t)i] = (int32_t)std::min<double>(n_samples, std::max<double>(1.0, k));
  }
  const int d = h->cfg.n_inputs, P = h->gpcP;
  std::vector<double> phi((size_t)n_samples * P);
  for (int m = 0; m < n_samples; ++m) {
    for (int t = 0; t < d; ++t)
      if (!std::isfinite(samples[(size_t)m * d + t])) return fail(h, SC_ERR_ARG, "quantiles: non-finite sample");
    hn_gpc_basis(d, h->cfg.gpc_degree, samples + (size_t)m * d, phi.data() + (size_t)m * P,
                 h->cfg.quad_rule == SC_Q_GH);
  }
  if (n_cells == 0) return SC_OK;
  std::vector<int32_t> cl(cells, cells + n_cells);
  const Layout& L = h->L;
  // pageable sources: each copy has taken its data when the call returns
  CK(cudaMemcpyAsync(h->ws + L.q_phi, phi.data(), sizeof(double) * phi.size(), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->ws + L.q_cells, cl.data(), sizeof(int32_t) * cl.size(), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->ws + L.q_k, kidx.data(), sizeof(int32_t) * kidx.size(), cudaMemcpyHostToDevice, h->stream));
  const int rc = launch_gpc_quantiles(d_coef, D.ncell, P, (const int32_t*)(h->ws + L.q_cells), n_cells,
                                      (const double*)(h->ws + L.q_phi), n_samples,
                                      (const int32_t*)(h->ws + L.q_k), n_q, d_out, h->stream);
  if (rc) return cuda_fail(h, (cudaError_t)rc, "quantile launch");
  ++h->launches;
  return SC_OK;
}

int sc_lbm_average_reset(sc_lbm_t h) {
  if (!h) return SC_ERR_ARG;
  if (!h->cfg.time_average) return fail(h, SC_ERR_STATE, "time_average = 0 in the configuration");
  for (int d = 0; d < h->P.n_domains; ++d) {
    const DomLayout& M = h->L.dom[d];
    CK(cudaMemsetAsync(h->ws + M.avg, 0, sizeof(double) * (size_t)M.nq * (size_t)M.ncell, h->stream));
  }
  h->avg_samples = 0;
  return SC_OK;
}

int sc_lbm_average_add(sc_lbm_t h) {
  if (!h) return SC_ERR_ARG;
  if (!h->cfg.time_average) return fail(h, SC_ERR_STATE, "time_average = 0 in the configuration");
  for (int d = 0; d < h->P.n_domains; ++d) {
    int rc = launch_average_add(params_now(h), h->cfg.precision, d, (double*)(h->ws + h->L.dom[d].avg),
                                h->stream);
    if (rc) return cuda_fail(h, (cudaError_t)rc, "average launch");
    ++h->launches;
  }
  ++h->avg_samples;
  return SC_OK;
}

int sc_lbm_average_moments(sc_lbm_t h, int domain, double* mean, double* stdev, const int32_t* probe_xy,
                           int n_p, double* prof, float* prof_nodes, double* gpc_coef, int out_host) {
  if (!h || domain < 0 || domain >= h->P.n_domains) return SC_ERR_ARG;
  if (!h->cfg.time_average) return fail(h, SC_ERR_STATE, "time_average = 0 in the configuration");
  if (h->avg_samples < 1) return fail(h, SC_ERR_STATE, "no samples in the time average");
  h->avg_read = (const double*)(h->ws + h->L.dom[domain].avg);
  const int rc = sc_lbm_moments(h, domain, mean, stdev, probe_xy, n_p, prof, prof_nodes, gpc_coef, out_host);
  h->avg_read = nullptr;
  return rc;
}

int sc_lbm_average_field(sc_lbm_t h, int domain, int node, double* d_q) {
  if (!h || !d_q || domain < 0 || domain >= h->P.n_domains) return SC_ERR_ARG;
  if (node < 0 || node >= h->P.dom[domain].nodes) return SC_ERR_ARG;
  if (!h->cfg.time_average) return fail(h, SC_ERR_STATE, "time_average = 0 in the configuration");
  if (h->avg_samples < 1) return fail(h, SC_ERR_STATE, "no samples in the time average");
  const DomLayout& M = h->L.dom[domain];
  const double* acc = (const double*)(h->ws + M.avg) + (size_t)node * (size_t)M.ncell;
  int rc = launch_scale(acc, 1.0 / (double)h->avg_samples, d_q, M.ncell, h->stream);
  if (rc) return cuda_fail(h, (cudaError_t)rc, "average field launch");
  ++h->launches;
  return SC_OK;
}

int sc_lbm_average_samples(sc_lbm_t h, long long* samples) {
  if (!h || !samples) return SC_ERR_ARG;
  *samples = h->avg_samples;
  return SC_OK;
}

int sc_lbm_qcriterion(sc_lbm_t h, int domain, const float* d_u, float* d_q) {
  if (!h || !d_u || !d_q || domain < 0 || domain >= h->P.n_domains) return SC_ERR_ARG;
  int rc = launch_qcriterion(params_now(h), domain, d_u, d_q, h->stream);
  if (rc) return cuda_fail(h, (cudaError_t)rc, "qcriterion launch");
  ++h->launches;
  return SC_OK;
}

int sc_lbm_velocity(sc_lbm_t h, int domain, int node, float* d_u) {
  if (!h || !d_u || domain < 0 || domain >= h->P.n_domains) return SC_ERR_ARG;
  if (node < 0 || node >= h->P.dom[domain].nodes) return SC_ERR_ARG;
  int rc = launch_export(params_now(h), h->cfg.precision, domain, node, nullptr, d_u, h->stream);
  if (rc) return cuda_fail(h, (cudaError_t)rc, "export launch");
  ++h->launches;
  return SC_OK;
}

int sc_lbm_populations(sc_lbm_t h, int domain, int node, double* d_f) {
  if (!h || !d_f || domain < 0 || domain >= h->P.n_domains) return SC_ERR_ARG;
  if (node < 0 || node >= h->P.dom[domain].nodes) return SC_ERR_ARG;
  int rc = launch_export(params_now(h), h->cfg.precision, domain, node, d_f, nullptr, h->stream);
  if (rc) return cuda_fail(h, (cudaError_t)rc, "export launch");
  ++h->launches;
  return SC_OK;
}

int sc_lbm_set_tuning(sc_lbm_t h, const sc_lbm_tuning* t) {
  if (!h || !t || check_tuning(*t)) return SC_ERR_ARG;
  CK(cudaStreamSynchronize(h->stream));
  h->tune = *t;
  apply_tiling(h);
  return SC_OK;
}

int sc_lbm_get_tuning(sc_lbm_t h, sc_lbm_tuning* t) {
  if (!h || !t) return SC_ERR_ARG;
  *t = h->tune;
  return SC_OK;
}

int sc_lbm_autotune(sc_lbm_t h, const char* cache_path) {
  if (!h) return SC_ERR_ARG;
  Range range("sc_lbm_autotune");
  if (h->cfg.precision == SC_P_FP64_PLAIN) return SC_OK;  // the plain path is not tuned
  int dev = 0;
  cudaDeviceProp prop;
  CK(cudaGetDevice(&dev));
  CK(cudaGetDeviceProperties(&prop, dev));
  const std::string key = tune_key(&h->cfg, prop.name);
  auto cache = read_cache(cache_path);
  auto it = cache.find(key);
  if (it != cache.end() && it->second.size() == 7) {
    sc_lbm_tuning t{it->second[0], it->second[1], it->second[2], it->second[3],
                    it->second[4], it->second[5], it->second[6]};
    if (check_tuning(t) == SC_OK) return sc_lbm_set_tuning(h, &t);
  }
  int maxnx = 0;
  for (int d = 0; d < h->P.n_domains; ++d) maxnx = std::max(maxnx, h->P.dom[d].nx);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  long long lups = 0;
  for (int d = 0; d < h->P.n_domains; ++d) lups += h->P.dom[d].ncell * h->P.dom[d].nodes;
  const int reps = (int)std::max<long long>(4, std::min<long long>(40, 2000000000LL / std::max(1LL, lups)));
  float best = 1e30f;
  sc_lbm_tuning best_t = h->tune;
  auto time_it = [&](const sc_lbm_tuning& t, float* ms) -> int {
    int rc = sc_lbm_set_tuning(h, &t);
    if (rc) return rc;
    rc = do_steps(h, 2);
    if (rc) return rc;
    CK(cudaEventRecord(e0, h->stream));
    rc = do_steps(h, 2 * reps);
    if (rc) return rc;
    CK(cudaEventRecord(e1, h->stream));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(ms, e0, e1));
    return SC_OK;
  };
  struct Timed {
    float ms;
    sc_lbm_tuning t;
  };
  std::vector<Timed> timed;
  auto try_all = [&](const std::vector<sc_lbm_tuning>& cand) -> int {
    for (const auto& t : cand) {
      float ms = 0;
      int rc = time_it(t, &ms);
      if (rc) return rc;
      timed.push_back({ms, t});
      if (ms < best) {
        best = ms;
        best_t = t;
      }
    }
    return SC_OK;
  };
  // stage 1: block shape and z-slab, patch-major order
  std::vector<sc_lbm_tuning> cand;
  const int bxs[] = {32, 64, 128, 256};
  const int bys[] = {1, 2, 4, 8};
  const int bzs[] = {2, 4, 8, 16, 32};
  for (int bx : bxs) {
    for (int by : bys)
      for (int bz : bzs) {
        if (bx * by > 256 || bx * by < 64) continue;
        if (bx > 32 && bx / 2 >= maxnx) continue;
        cand.push_back({bx, by, bz, 1, SC_EXEC_LAUNCH, 50, 0});
      }
  }
  int rc = try_all(cand);
  if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
  // stage 2: register budgets and tile order on the three fastest shapes
  std::sort(timed.begin(), timed.end(), [](const Timed& a, const Timed& b) { return a.ms < b.ms; });
  cand.clear();
  for (size_t k = 0; k < timed.size() && k < 3; ++k) {
    const sc_lbm_tuning t = timed[k].t;
    for (int order = 0; order < 2; ++order)
      for (int v : {0, 2, 3}) {
        if (order == t.tile_order && v == t.variant) continue;
        cand.push_back({t.block_x, t.block_y, t.slab_z, order, SC_EXEC_LAUNCH, 50, v});
      }
  }
  if (h->tma_ok)
    for (int order = 0; order < 2; ++order) cand.push_back({128, 2, 1, order, SC_EXEC_LAUNCH, 50, 1});
  rc = try_all(cand);
  if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
  // execution mode for the best shape
  for (int mode : {SC_EXEC_GRAPH, SC_EXEC_PERSISTENT}) {
    sc_lbm_tuning t = best_t;
    t.exec_mode = mode;
    if (mode == SC_EXEC_PERSISTENT && t.variant == 1) {
      t.variant = 0;  // the persistent form loads one cell per thread
      t.block_x = 64;
      t.block_y = 2;
    }
    float ms = 0;
    int rc = time_it(t, &ms);
    if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
    if (ms < best * 0.98f) { best = ms; best_t = t; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  rc = sc_lbm_set_tuning(h, &best_t);
  if (rc) return rc;
  rc = reset_state(h);
  if (rc) return rc;
  unsigned bits = 0;
  rc = read_err(h, &bits);
  if (rc) return rc;
  if (cache_path) {
    cache[key] = {best_t.block_x, best_t.block_y, best_t.slab_z, best_t.tile_order, best_t.exec_mode,
                  best_t.graph_steps, best_t.variant};
    write_cache(cache_path, cache);
  }
  return err_status(h, bits);
}

int sc_lbm_counters(sc_lbm_t h, long long* steps, long long* kernel_launches) {
  if (!h) return SC_ERR_ARG;
  if (steps) *steps = h->steps;
  if (kernel_launches) *kernel_launches = h->launches;
  return SC_OK;
}

int sc_lbm_sync(sc_lbm_t h) {
  if (!h) return SC_ERR_ARG;
  unsigned bits = 0;
  int rc = read_err(h, &bits);
  if (rc) return rc;
  return err_status(h, bits);
}

int sc_lbm_check(sc_lbm_t h, long long* n_bad) {
  if (!h) return SC_ERR_ARG;
  unsigned long long* cnt = &h->hdr()->check_count;
  CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), h->stream));
  int rc = launch_check(params_now(h), h->cfg.precision, cnt, h->stream);
  if (rc) return cuda_fail(h, (cudaError_t)rc, "check launch");
  ++h->launches;
  unsigned long long v = 0;
  CK(cudaMemcpyAsync(&v, cnt, sizeof v, cudaMemcpyDeviceToHost, h->stream));
  unsigned bits = 0;
  rc = read_err(h, &bits);
  if (rc) return rc;
  if (n_bad) *n_bad = (long long)v;
  return err_status(h, bits);
}

int sc_lbm_debug_barrier(sc_lbm_t h, int never_arrive, long long spin_limit) {
  if (!h || spin_limit < 1) return SC_ERR_ARG;
  h->never_arrive = never_arrive ? 1 : 0;
  h->spin_limit = spin_limit;
  return SC_OK;
}

// Snapshot: header, then per domain the population arrays and outflow plane.
struct SnapHeader {
  uint64_t magic, version, cfg_hash, payload_hash, steps, bytes;
};

static uint64_t cfg_hash(sc_lbm_t h) {
  uint64_t k = fnv1a(&h->cfg.precision, sizeof(int));
  for (int d = 0; d < h->P.n_domains; ++d) {
    const DevDomain& D = h->P.dom[d];
    int v[5] = {D.nx, D.ny, D.nz, D.nodes, 0};
    k = fnv1a(v, sizeof v, k);
  }
  return k;
}

static size_t payload_bytes(sc_lbm_t h) {
  size_t b = 0;
  const size_t sb = storage_bytes(h->cfg.precision);
  for (int d = 0; d < h->P.n_domains; ++d) {
    const DevDomain& D = h->P.dom[d];
    b += sb * kQ * (size_t)D.pitch * D.nodes * (h->cfg.precision == SC_P_FP64_PLAIN ? 2 : 1);
    if (D.bout) b += sizeof(float) * 5 * (size_t)D.nz * D.ny * D.nodes;
  }
  return b;
}

int sc_lbm_state_size(sc_lbm_t h, size_t* bytes) {
  if (!h || !bytes) return SC_ERR_ARG;
  *bytes = sizeof(SnapHeader) + payload_bytes(h);
  return SC_OK;
}

int sc_lbm_save(sc_lbm_t h, void* host_buf, size_t bytes) {
  if (!h || !host_buf) return SC_ERR_ARG;
  const size_t need = sizeof(SnapHeader) + payload_bytes(h);
  if (bytes < need) return SC_ERR_ARG;
  char* out = (char*)host_buf + sizeof(SnapHeader);
  const size_t sb = storage_bytes(h->cfg.precision);
  for (int d = 0; d < h->P.n_domains; ++d) {
    const DevDomain& D = h->P.dom[d];
    size_t n = sb * kQ * (size_t)D.pitch * D.nodes;
    CK(cudaMemcpyAsync(out, D.g, n, cudaMemcpyDeviceToHost, h->stream));
    out += n;
    if (D.g2) {
      CK(cudaMemcpyAsync(out, D.g2, n, cudaMemcpyDeviceToHost, h->stream));
      out += n;
    }
    if (D.bout) {
      size_t nb = sizeof(float) * 5 * (size_t)D.nz * D.ny * D.nodes;
      CK(cudaMemcpyAsync(out, D.bout, nb, cudaMemcpyDeviceToHost, h->stream));
      out += nb;
    }
  }
  CK(cudaStreamSynchronize(h->stream));
  SnapHeader hd;
  hd.magic = 0x53434C424D534E50ULL;
  hd.version = 1;
  hd.cfg_hash = cfg_hash(h);
  hd.payload_hash = fnv1a((const char*)host_buf + sizeof(SnapHeader), need - sizeof(SnapHeader));
  hd.steps = (uint64_t)h->steps;
  hd.bytes = need;
  memcpy(host_buf, &hd, sizeof hd);
  return SC_OK;
}

int sc_lbm_load(sc_lbm_t h, const void* host_buf, size_t bytes) {
  if (!h || !host_buf || bytes < sizeof(SnapHeader)) return SC_ERR_ARG;
  SnapHeader hd;
  memcpy(&hd, host_buf, sizeof hd);
  const size_t need = sizeof(SnapHeader) + payload_bytes(h);
  if (hd.magic != 0x53434C424D534E50ULL || hd.version != 1 || hd.bytes != need || bytes < need)
    return fail(h, SC_ERR_ARG, "not a snapshot of this configuration");
  if (hd.cfg_hash != cfg_hash(h)) return fail(h, SC_ERR_ARG, "snapshot configuration differs");
  if (hd.payload_hash != fnv1a((const char*)host_buf + sizeof(SnapHeader), need - sizeof(SnapHeader)))
    return fail(h, SC_ERR_ARG, "snapshot checksum mismatch");
  const char* in = (const char*)host_buf + sizeof(SnapHeader);
  const size_t sb = storage_bytes(h->cfg.precision);
  for (int d = 0; d < h->P.n_domains; ++d) {
    const DevDomain& D = h->P.dom[d];
    size_t n = sb * kQ * (size_t)D.pitch * D.nodes;
    CK(cudaMemcpyAsync(D.g, in, n, cudaMemcpyHostToDevice, h->stream));
    in += n;
    if (D.g2) {
      CK(cudaMemcpyAsync(D.g2, in, n, cudaMemcpyHostToDevice, h->stream));
      in += n;
    }
    if (D.bout) {
      size_t nb = sizeof(float) * 5 * (size_t)D.nz * D.ny * D.nodes;
      CK(cudaMemcpyAsync(D.bout, in, nb, cudaMemcpyHostToDevice, h->stream));
      in += nb;
    }
  }
  CK(cudaStreamSynchronize(h->stream));
  h->steps = (long long)hd.steps;
  return SC_OK;
}

// ------------------------------------------------------------ inflow update
// Node inflow u_in(z) = u_ref (1 + xi) (h/H)^alpha (cos theta, sin theta, 0)
// with the node's coordinates replacing xi, alpha or theta.
static void node_inflow(const sc_lbm_config& c, const std::vector<double>& Z, int j, int nz, double* ud,
                        double* alpha_out) {
  double xi = 0.0, al = c.alpha, th = c.angle_deg;
  for (int t = 0; t < c.n_inputs; ++t) {
    const double zt = Z[(size_t)j * c.n_inputs + t];
    if (c.inputs[t] == SC_IN_SPEED_REL) xi = zt;
    else if (c.inputs[t] == SC_IN_ALPHA) al = zt;
    else th = zt;
  }
  const double H = c.H_ref > 0 ? c.H_ref : (double)nz;
  hn_inflow(nz, c.u_ref, xi, al, H, th, ud, c.profile, c.z0);
  if (alpha_out) *alpha_out = al;
}

int sc_lbm_set_inflow(sc_lbm_t h, double u_ref, double alpha, double angle_deg) {
  if (!h || !(u_ref == u_ref) || !(alpha == alpha) || !(angle_deg == angle_deg)) return SC_ERR_ARG;
  h->cfg.u_ref = u_ref;
  h->cfg.alpha = alpha;
  h->cfg.angle_deg = angle_deg;
  CK(cudaStreamSynchronize(h->stream));
  for (int d = 0; d < h->P.n_domains; ++d) {
    const int nz = h->doms[d].nz, nq = h->nq[d];
    std::vector<double> ud((size_t)nq * nz * 3);
    std::vector<float> uf((size_t)nq * nz * 4, 0.0f);
    for (int j = 0; j < nq; ++j) {
      node_inflow(h->cfg, h->Z[d], j, nz, &ud[(size_t)j * nz * 3], nullptr);
      for (int k = 0; k < nz; ++k)
        for (int a = 0; a < 3; ++a) uf[((size_t)j * nz + k) * 4 + a] = (float)ud[((size_t)j * nz + k) * 3 + a];
    }
    CK(cudaMemcpy(h->ws + h->L.dom[d].uin_f, uf.data(), sizeof(float) * uf.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->ws + h->L.dom[d].uin_d, ud.data(), sizeof(double) * ud.size(), cudaMemcpyHostToDevice));
  }
  return SC_OK;
}

namespace {
int check_series(int n, const double* speed, const double* dir_deg, long long per, long long interp) {
  if (n < 0 || n > SC_SERIES_MAX_TARGETS) return SC_ERR_ARG;
  if (n == 0) return SC_OK;
  if (!speed || !dir_deg || per < 1 || per > (1LL << 40) || interp < 0 || interp > per) return SC_ERR_ARG;
  for (int k = 0; k < n; ++k)
    if (!std::isfinite(speed[k]) || speed[k] < 0.0 || !std::isfinite(dir_deg[k])) return SC_ERR_ARG;
  return SC_OK;
}
}  // namespace

int sc_lbm_set_inflow_series(sc_lbm_t h, int n_targets, const double* speed, const double* dir_deg,
                             long long steps_per_target, long long interp_steps) {
  if (!h) return SC_ERR_ARG;
  if (check_series(n_targets, speed, dir_deg, steps_per_target, interp_steps))
    return fail(h, SC_ERR_ARG, "inflow series: need 0 <= n_targets <= SC_SERIES_MAX_TARGETS, finite speed "
                               "factors >= 0 and directions, 1 <= steps_per_target <= 2^40, "
                               "0 <= interp_steps <= steps_per_target");
  h->series_speed.assign(speed, speed + n_targets);
  h->series_dir.assign((size_t)n_targets, 0.0);
  hn_series_unwrap(n_targets, dir_deg, h->series_dir.data());
  h->series_per = n_targets ? steps_per_target : 1;
  h->series_interp = n_targets ? interp_steps : 0;
  return SC_OK;
}

int sc_lbm_inflow_factor(int ramp_steps, int n_targets, const double* speed, const double* dir_deg,
                         long long steps_per_target, long long interp_steps, long long level, double* factor) {
  if (ramp_steps < 0 || level < 0 || !factor ||
      check_series(n_targets, speed, dir_deg, steps_per_target, interp_steps))
    return SC_ERR_ARG;
  std::vector<double> un((size_t)n_targets);
  hn_series_unwrap(n_targets, dir_deg, un.data());
  double sp = 1.0, d = 0.0;
  if (n_targets > 0) hn_series_at(n_targets, speed, un.data(), steps_per_target, interp_steps, level, &sp, &d);
  const Wind<double> w = wind_of(hn_ramp(ramp_steps, level), sp, d);
  factor[0] = w.scale * w.cos_d;
  factor[1] = w.scale * w.sin_d;
  factor[2] = w.scale;
  return SC_OK;
}

int sc_lbm_inflow_next_change(int ramp_steps, int n_targets, const double* speed, const double* dir_deg,
                              long long steps_per_target, long long interp_steps, long long level,
                              long long* next) {
  if (ramp_steps < 0 || level < 0 || !next ||
      check_series(n_targets, speed, dir_deg, steps_per_target, interp_steps))
    return SC_ERR_ARG;
  *next = hn_wind_next_change(ramp_steps, n_targets, n_targets ? steps_per_target : 1,
                              n_targets ? interp_steps : 0, level);
  return SC_OK;
}

// ------------------------------------------------------------ adjoint
namespace {
struct AdjLayout {
  size_t accum, probes, target, uprobe, uin, du, lmap, states, state_bytes, total;
  int K, L;
};

int adj_plan(sc_lbm_t h, int domain, int n_steps, int n_snapshots, int n_probes, AdjLayout& A) {
  if (domain < 0 || domain >= h->P.n_domains || n_steps < 1 || n_snapshots < 0 || n_probes < 1 ||
      n_probes > 256)
    return SC_ERR_ARG;
  int K = n_snapshots > 0 ? n_snapshots : (int)ceil(sqrt((double)n_steps));
  if (K > n_steps) K = n_steps;
  const int L = (n_steps + K - 1) / K;
  K = (n_steps + L - 1) / L;
  const DevDomain& D = h->P.dom[domain];
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  A.accum = take(3 * sizeof(double));
  A.probes = take(3 * sizeof(int32_t) * (size_t)n_probes);
  A.target = take(3 * sizeof(double) * (size_t)n_probes);
  A.uprobe = take(3 * sizeof(double) * (size_t)n_probes);
  A.uin = take(16 * (size_t)D.nz);
  A.du = take(32 * (size_t)D.nz);
  A.lmap = take(sizeof(int32_t) * (size_t)D.ncell);
  A.state_bytes = align_up(sizeof(float) * kQ * (size_t)D.pitch);
  A.states = off;
  A.K = K;
  A.L = L;
  A.total = off + A.state_bytes * (size_t)(K + L + 4);
  return SC_OK;
}
}  // namespace

int sc_lbm_adjoint_workspace_size(sc_lbm_t h, int domain, int n_steps, int n_snapshots, int n_probes,
                                  size_t* bytes) {
  if (!h || !bytes) return SC_ERR_ARG;
  AdjLayout A;
  int rc = adj_plan(h, domain, n_steps, n_snapshots, n_probes, A);
  if (rc) return rc;
  *bytes = A.total;
  return SC_OK;
}

int sc_lbm_adjoint(sc_lbm_t h, int domain, int node, const int32_t* probes, int n_probes,
                   const double* u_target, int n_steps, int n_snapshots, void* d_ws, size_t bytes,
                   double* loss_out, double* grad_out, double* u_probe_out) {
  if (!h || !probes || !u_target || !loss_out || !grad_out) return SC_ERR_ARG;
  Range range("sc_lbm_adjoint");
  if (h->cfg.c_smag != 0.0 || h->cfg.collision != SC_COLL_BGK)
    return fail(h, SC_ERR_UNSUPPORTED, "the adjoint covers BGK (c_smag = 0, SC_COLL_BGK)");
  if (h->cfg.profile != SC_PROFILE_POWER)
    return fail(h, SC_ERR_UNSUPPORTED, "the adjoint's parameters are those of the power-law profile");
  if (!h->series_speed.empty())
    return fail(h, SC_ERR_UNSUPPORTED, "the adjoint covers a steady inflow (no inflow series set)");
  if (domain >= 0 && domain < (int)h->doms.size() && h->doms[domain].disk_radius > 0.0)
    return fail(h, SC_ERR_UNSUPPORTED, "the adjoint covers box domains (disk_radius = 0)");
  AdjLayout L;
  int rc = adj_plan(h, domain, n_steps, n_snapshots, n_probes, L);
  if (rc) return fail(h, rc, "bad adjoint arguments");
  if (node < 0 || node >= h->nq[domain]) return fail(h, SC_ERR_ARG, "node out of range");
  if (!d_ws || ((uintptr_t)d_ws % kAlign) != 0 || bytes < L.total) return SC_ERR_WORKSPACE;
  const DevDomain& D = h->P.dom[domain];
  for (int p = 0; p < n_probes; ++p) {
    const int x = probes[3 * p], y = probes[3 * p + 1], z = probes[3 * p + 2];
    if (x < 0 || x >= D.nx || y < 0 || y >= D.ny || z < 0 || z >= D.nz)
      return fail(h, SC_ERR_ARG, "probe outside the domain");
    if (h->flags[domain][(size_t)x + (size_t)D.nx * ((size_t)y + (size_t)D.ny * z)])
      return fail(h, SC_ERR_ARG, "probe in a solid cell");
  }
  char* ws = (char*)d_ws;
  // host tables: the node's inflow and its derivatives
  std::vector<double> ud((size_t)D.nz * 3);
  double al = 0.0;
  node_inflow(h->cfg, h->Z[domain], node, D.nz, ud.data(), &al);
  const double H = h->cfg.H_ref > 0 ? h->cfg.H_ref : (double)D.nz;
  std::vector<float> uin((size_t)D.nz * 4, 0.0f), du((size_t)D.nz * 8, 0.0f);
  for (int k = 0; k < D.nz; ++k) {
    const double lh = log(((double)k + 0.5) / H);
    for (int a = 0; a < 3; ++a) {
      const double u = ud[3 * k + a];
      uin[4 * k + a] = (float)u;
      du[4 * k + a] = (float)(h->cfg.u_ref != 0.0 ? u / h->cfg.u_ref : 0.0);  // d/du_ref
      du[4 * (D.nz + k) + a] = (float)(u * lh);                               // d/dalpha
    }
  }
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemset(ws + L.accum, 0, 3 * sizeof(double)));
  CK(cudaMemcpy(ws + L.probes, probes, 3 * sizeof(int32_t) * (size_t)n_probes, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ws + L.target, u_target, 3 * sizeof(double) * (size_t)n_probes, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ws + L.uin, uin.data(), sizeof(float) * uin.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ws + L.du, du.data(), sizeof(float) * du.size(), cudaMemcpyHostToDevice));
  AdjArgs A;
  A.domain = domain;
  A.uin = (const float4*)(ws + L.uin);
  A.du = (const float4*)(ws + L.du);
  A.probes = (const int32_t*)(ws + L.probes);
  A.target = (const double*)(ws + L.target);
  A.u_probe = (double*)(ws + L.uprobe);
  A.n_probes = n_probes;
  A.accum = (double*)(ws + L.accum);
  A.lmap = (const int32_t*)(ws + L.lmap);
  auto state = [&](int k) { return (float*)(ws + L.states + L.state_bytes * (size_t)k); };
  float* snap0 = state(0);           // K checkpoints
  float* seg0 = state(L.K);          // L segment states
  float* lamA = state(L.K + L.L);
  float* lamB = state(L.K + L.L + 1);
  float* fa = state(L.K + L.L + 2);
  float* fb = state(L.K + L.L + 3);
  const long long nstate = (long long)kQ * D.pitch;
  const StepParams& P = h->P;
  auto ck = [&](int r, const char* what) { return r ? cuda_fail(h, (cudaError_t)r, what) : SC_OK; };
  // The device work of one gradient: forward sweep with checkpoints every L
  // steps from the equilibrium start, loss and seed at level T, then per
  // segment (last first) the recompute of its states and the reverse steps.
  const size_t sf = L.state_bytes / sizeof(float);
  auto issue = [&]() -> int {
    int r;
    if ((r = ck(launch_adj_listed_map(P, domain, (int32_t*)(ws + L.lmap), h->stream), "adjoint map"))) return r;
    if ((r = ck(launch_fill_zero(fa, nstate, h->stream), "adjoint fill"))) return r;
    if ((r = ck(launch_fill_zero(fb, nstate, h->stream), "adjoint fill"))) return r;
    float* cur = fa;
    float* nxt = fb;
    for (int n = 0; n < n_steps; ++n) {
      if (n % L.L == 0)
        CK(cudaMemcpyAsync(snap0 + (size_t)(n / L.L) * sf, cur, sizeof(float) * nstate, cudaMemcpyDeviceToDevice,
                           h->stream));
      if ((r = ck(launch_adj_forward(P, A, cur, nxt, (float)hn_ramp(h->cfg.ramp_steps, n + 1), h->stream),
                  "adjoint forward")))
        return r;
      std::swap(cur, nxt);
    }
    if ((r = ck(launch_fill_zero(lamA, nstate, h->stream), "adjoint fill"))) return r;
    if ((r = ck(launch_fill_zero(lamB, nstate, h->stream), "adjoint fill"))) return r;
    if ((r = ck(launch_adj_loss(P, A, cur, lamA, h->stream), "adjoint loss"))) return r;
    float* lnext = lamA;
    float* lcur = lamB;
    for (int sgm = L.K - 1; sgm >= 0; --sgm) {
      const int n0 = sgm * L.L, n1 = std::min(n0 + L.L, n_steps);
      CK(cudaMemcpyAsync(seg0, snap0 + (size_t)sgm * sf, sizeof(float) * nstate, cudaMemcpyDeviceToDevice,
                         h->stream));
      for (int n = n0; n < n1 - 1; ++n)
        if ((r = ck(launch_adj_forward(P, A, seg0 + (size_t)(n - n0) * sf, seg0 + (size_t)(n - n0 + 1) * sf,
                                       (float)hn_ramp(h->cfg.ramp_steps, n + 1), h->stream),
                    "adjoint recompute")))
          return r;
      for (int n = n1 - 1; n >= n0; --n) {
        if ((r = ck(launch_adj_step(P, A, seg0 + (size_t)(n - n0) * sf, lnext, lcur,
                                    (float)hn_ramp(h->cfg.ramp_steps, n + 1), h->stream),
                    "adjoint step")))
          return r;
        std::swap(lnext, lcur);
      }
    }
    return SC_OK;
  };
  // Replays of one captured graph while the arguments that shape the sweep
  // stay the same (the node's inflow tables, probes and targets are read
  // from the workspace, uploaded above); the legacy default stream cannot
  // be captured and runs the launches directly.
  const std::vector<long long> key = {domain, n_steps, L.K, L.L, n_probes, (long long)(uintptr_t)d_ws,
                                      (long long)bytes, h->cfg.ramp_steps};
  if (h->stream) {
    if (!h->adj_graph || h->adj_key != key) {
      if (h->adj_graph) cudaGraphExecDestroy(h->adj_graph);
      h->adj_graph = nullptr;
      h->adj_key.clear();
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
      rc = issue();
      cudaError_t e = cudaStreamEndCapture(h->stream, &g);
      if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture (adjoint)");
      e = cudaGraphInstantiate(&h->adj_graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate (adjoint)");
      h->adj_key = key;
    }
    CK(cudaGraphLaunch(h->adj_graph, h->stream));
  } else {
    rc = issue();
    if (rc) return rc;
  }
  h->launches += 2LL * n_steps + (n_steps - L.K) + 5;
  double acc[3];
  CK(cudaMemcpyAsync(acc, ws + L.accum, sizeof acc, cudaMemcpyDeviceToHost, h->stream));
  if (u_probe_out)
    CK(cudaMemcpyAsync(u_probe_out, ws + L.uprobe, 3 * sizeof(double) * (size_t)n_probes,
                       cudaMemcpyDeviceToHost, h->stream));
  unsigned bits = 0;
  rc = read_err(h, &bits);
  if (rc) return rc;
  *loss_out = acc[0];
  grad_out[0] = acc[1];
  grad_out[1] = acc[2];
  return err_status(h, bits);
}

const char* sc_lbm_last_error(sc_lbm_t h) {
  if (!h) return "null handle";
  return h->err.c_str();
}

int sc_lbm_destroy(sc_lbm_t h) {
  if (!h) return SC_ERR_ARG;
  cudaStreamSynchronize(h->stream);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->adj_graph) cudaGraphExecDestroy(h->adj_graph);
  delete h;
  return SC_OK;
}

}  // extern "C"
