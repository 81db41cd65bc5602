// host_numerics.cpp -- host-side numerics of libsclbm: quadrature rules,
// seeded geometry and probes, boundary link classification, inflow tables and
// the gPC basis.  Compiled with -ffp-contract=off so that the quadrature
// nodes and weights are the same bits on every host.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <thread>
#include <vector>

#include "sclbm_internal.h"

namespace sclbm {
namespace {

// Runs f(z0, z1) over [0, nz) split into contiguous ranges on up to
// hardware_concurrency threads (one thread below 2^16 cells of work, an item
// weighing `plane` cells).  The ranges write disjoint outputs, so the result
// does not depend on the split.
template <class F>
void parallel_layers(int nz, long long plane, F&& f) {
  unsigned nt = std::thread::hardware_concurrency();
  if (nt == 0) nt = 1;
  nt = std::min<unsigned>(nt, 32u);
  nt = std::min<unsigned>(nt, (unsigned)std::max(1, nz));
  if ((long long)nz * plane < (1LL << 16)) nt = 1;
  if (nt <= 1) {
    f(0, nz);
    return;
  }
  std::vector<std::thread> pool;
  pool.reserve(nt);
  for (unsigned t = 0; t < nt; ++t) {
    const int z0 = (int)((long long)nz * t / nt), z1 = (int)((long long)nz * (t + 1) / nt);
    try {
      pool.emplace_back([&f, z0, z1] { f(z0, z1); });
    } catch (...) {
      f(z0, z1);  // no thread to be had: this range runs on the calling thread
    }
  }
  for (auto& th : pool) th.join();
}

// D3Q19 velocities (rest, axis pairs, face-diagonal pairs), Sec. 2.2 Fig. 1.
const int kCx[kQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
const int kCy[kQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
const int kCz[kQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014).
struct Rng {
  uint64_t state;
  uint64_t next() {
    state += 0x9E3779B97F4A7C15ULL;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  }
  int draw(int lo, int hi) {  // U{lo..hi}
    uint64_t span = (uint64_t)(hi - lo + 1);
    return lo + (int)(next() % span);
  }
};

// 1-D Gauss-Legendre on [-1, 1] (weights sum 2), n <= 5, closed forms.
bool gl_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  x.clear();
  w.clear();
  switch (n) {
    case 1:
      x = {0.0};
      w = {2.0};
      return true;
    case 2: {
      double r = 1.0 / sqrt(3.0);
      x = {-r, r};
      w = {1.0, 1.0};
      return true;
    }
    case 3: {
      double r = sqrt(3.0 / 5.0);
      x = {-r, 0.0, r};
      w = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
      return true;
    }
    case 4: {
      double inner = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0));
      double outer = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
      double w_in = (18.0 + sqrt(30.0)) / 36.0;
      double w_out = (18.0 - sqrt(30.0)) / 36.0;
      x = {-outer, -inner, inner, outer};
      w = {w_out, w_in, w_in, w_out};
      return true;
    }
    case 5: {
      double inner = sqrt(5.0 - 2.0 * sqrt(10.0 / 7.0)) / 3.0;
      double outer = sqrt(5.0 + 2.0 * sqrt(10.0 / 7.0)) / 3.0;
      double w_in = (322.0 + 13.0 * sqrt(70.0)) / 900.0;
      double w_out = (322.0 - 13.0 * sqrt(70.0)) / 900.0;
      x = {-outer, -inner, 0.0, inner, outer};
      w = {w_out, w_in, 128.0 / 225.0, w_in, w_out};
      return true;
    }
    default:
      return false;
  }
}

int cc_size(int level) { return level <= 1 ? 1 : (1 << (level - 1)) + 1; }

// 1-D Clenshaw-Curtis rule of `level` on [-1, 1], weights summing to 2:
// nodes -cos(k pi / n) with exact 0, +-1 and mirror pairs; weights
// (c_k / n) (1 - sum_{j=1}^{n/2} b_j cos(2 j k pi / n) / (4 j^2 - 1)).
void cc_rule(int level, std::vector<double>& x, std::vector<double>& w) {
  const int m = cc_size(level);
  x.assign(m, 0.0);
  w.assign(m, 0.0);
  if (m == 1) {
    w[0] = 2.0;
    return;
  }
  const int n = m - 1;
  for (int k = 0; k <= n; ++k) x[k] = -cos((double)k * M_PI / (double)n);
  for (int k = 0; 2 * k < n; ++k) x[n - k] = -x[k];
  x[0] = -1.0;
  x[n] = 1.0;
  if ((n & 1) == 0) x[n / 2] = 0.0;
  for (int k = 0; k <= n; ++k) {
    double acc = 0.0;
    for (int j = 1; j <= n / 2; ++j) {
      double bj = (2 * j == n) ? 1.0 : 2.0;
      double cj = cos((double)(2 * j * k) * M_PI / (double)n);
      acc += bj / (double)(4 * j * j - 1) * cj;
    }
    double ck = (k == 0 || k == n) ? 1.0 : 2.0;
    w[k] = ck / (double)n * (1.0 - acc);
  }
}

long long choose(int n, int k) {
  if (k < 0 || k > n) return 0;
  long long r = 1;
  for (int t = 1; t <= k; ++t) r = r * (n - k + t) / t;
  return r;
}

// Accumulator keyed by the finest-grid integer index, filled in enumeration
// order (so each node's weight is summed in the order of contributions).
// Orthonormal probabilists' Hermite polynomials p_0..p_{n-1} at x:
// p_0 = 1, p_1 = x, sqrt(k+1) p_{k+1} = x p_k - sqrt(k) p_{k-1}.
double christoffel_sum(int n, double x) {
  double a = 1.0, b = x, s = 1.0;
  if (n > 1) s += b * b;
  for (int k = 1; k + 1 < n; ++k) {
    const double c = (x * b - sqrt((double)k) * a) / sqrt((double)(k + 1));
    a = b;
    b = c;
    s += c * c;
  }
  return s;
}

// n-point Gauss-Hermite rule for the standard normal density by the
// Golub-Welsch construction: the nodes are the eigenvalues of the symmetric
// tridiagonal Jacobi matrix of the orthonormal probabilists' Hermite
// polynomials (zero diagonal, off-diagonal sqrt(k)), found by cyclic Jacobi
// rotations (n <= 40, so cost is no concern) and polished by Newton steps on
// the recurrence.  The probability weights are
// the reciprocal Christoffel sums 1 / sum_{k<n} p_k(x)^2 at the nodes, which
// keeps the tiny tail weights accurate in relative terms.  Nodes are then
// made exactly antisymmetric and the weights symmetric.
bool gh_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  if (n < 1 || n > 40) return false;
  std::vector<double> A((size_t)n * n, 0.0);
  for (int k = 1; k < n; ++k) A[(size_t)k * n + k - 1] = A[(size_t)(k - 1) * n + k] = sqrt((double)k);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
    if (off < 1e-60) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        // rotation angle zeroing A[p][q]: tan(2 phi) = 2 apq / (aqq - app)
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - sn * akq;
          A[(size_t)k * n + q] = sn * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - sn * aqk;
          A[(size_t)q * n + k] = sn * apk + c * aqk;
        }
      }
  }
  x.assign(n, 0.0);
  for (int k = 0; k < n; ++k) x[k] = A[(size_t)k * n + k];
  std::sort(x.begin(), x.end());
  // two Newton steps on p_n (p_n' = sqrt(n) p_{n-1}) polish the eigenvalues
  for (int k = 0; k < n; ++k)
    for (int it = 0; it < 2; ++it) {
      double a = 1.0, b = x[k];
      for (int m = 1; m < n; ++m) {
        const double c = (x[k] * b - sqrt((double)m) * a) / sqrt((double)(m + 1));
        a = b;
        b = c;
      }
      if (n > 1 && a != 0.0) x[k] -= b / (sqrt((double)n) * a);
    }
  for (int k = 0; k < n / 2; ++k) {
    const double xs = 0.5 * (x[n - 1 - k] - x[k]);
    x[k] = -xs;
    x[n - 1 - k] = xs;
  }
  if (n & 1) x[n / 2] = 0.0;
  w.assign(n, 0.0);
  for (int k = 0; k < n; ++k) w[k] = 1.0 / christoffel_sum(n, x[k]);
  for (int k = 0; k < n / 2; ++k) w[k] = w[n - 1 - k] = 0.5 * (w[k] + w[n - 1 - k]);
  return true;
}

struct NodeAcc {
  int d;
  std::vector<int> keys;       // [count][d]
  std::vector<double> weight;  // [count]
  void add(const int* key, double v) {
    const int count = (int)weight.size();
    for (int e = 0; e < count; ++e) {
      if (std::equal(key, key + d, keys.begin() + (size_t)e * d)) {
        weight[e] += v;
        return;
      }
    }
    keys.insert(keys.end(), key, key + d);
    weight.push_back(0.0 + v);
  }
};

}  // namespace

int hn_quadrature(int rule, int d, int level, const double* lo, const double* hi,
                  std::vector<double>& Z, std::vector<double>& w) {
  if (d < 1 || d > 3 || level < 1) return SC_ERR_ARG;
  NodeAcc acc{d, {}, {}};
  std::vector<double> fine_x;
  if (rule == SC_Q_GL) {
    std::vector<double> x1, w1;
    if (!gl_rule(level, x1, w1)) return SC_ERR_ARG;
    fine_x = x1;
    std::vector<double> pw(level);
    for (int k = 0; k < level; ++k) pw[k] = w1[k] * 0.5;
    int total = 1;
    for (int t = 0; t < d; ++t) total *= level;
    for (int flat = 0; flat < total; ++flat) {
      int key[3];
      int rem = flat;
      for (int t = d - 1; t >= 0; --t) {
        key[t] = rem % level;
        rem /= level;
      }
      double prod = 1.0;
      for (int t = 0; t < d; ++t) prod *= pw[key[t]];
      acc.add(key, prod);
    }
  } else if (rule == SC_Q_CC_SMOLYAK) {
    if (level > 12) return SC_ERR_ARG;
    std::vector<double> wf;
    cc_rule(level, fine_x, wf);
    const int mfine = cc_size(level);
    std::vector<std::vector<double>> wl(level + 1);
    for (int l = 1; l <= level; ++l) {
      std::vector<double> xl;
      cc_rule(l, xl, wl[l]);
      for (double& v : wl[l]) v = v * 0.5;
    }
    // multi-indices i in {1..level}^d, i_1 most significant
    int total = 1;
    for (int t = 0; t < d; ++t) total *= level;
    for (int flat = 0; flat < total; ++flat) {
      int lv[3];
      int rem = flat;
      for (int t = d - 1; t >= 0; --t) {
        lv[t] = rem % level + 1;
        rem /= level;
      }
      int sum = 0;
      for (int t = 0; t < d; ++t) sum += lv[t];
      if (sum < level || sum > level + d - 1) continue;
      const int e = level + d - 1 - sum;
      const long long coef = (e & 1 ? -1 : 1) * choose(d - 1, e);
      int cnt = 1;
      for (int t = 0; t < d; ++t) cnt *= cc_size(lv[t]);
      for (int g = 0; g < cnt; ++g) {
        int k[3], key[3];
        int r2 = g;
        for (int t = d - 1; t >= 0; --t) {
          k[t] = r2 % cc_size(lv[t]);
          r2 /= cc_size(lv[t]);
        }
        double prod = (double)coef;
        for (int t = 0; t < d; ++t) {
          const int m = cc_size(lv[t]);
          prod *= wl[lv[t]][k[t]];
          key[t] = (m == 1) ? (mfine - 1) / 2 : k[t] * ((mfine - 1) / (m - 1));
        }
        acc.add(key, prod);
      }
    }
  } else if (rule == SC_Q_GH) {
    std::vector<double> w1;
    if (!gh_rule(level, fine_x, w1)) return SC_ERR_ARG;
    int total = 1;
    for (int t = 0; t < d; ++t) total *= level;
    for (int flat = 0; flat < total; ++flat) {
      int key[3];
      int rem = flat;
      for (int t = d - 1; t >= 0; --t) {
        key[t] = rem % level;
        rem /= level;
      }
      double prod = 1.0;
      for (int t = 0; t < d; ++t) prod *= w1[key[t]];
      acc.add(key, prod);
    }
  } else {
    return SC_ERR_ARG;
  }
  const int count = (int)acc.weight.size();
  std::vector<int> order(count);
  for (int e = 0; e < count; ++e) order[e] = e;
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    return std::lexicographical_compare(acc.keys.begin() + (size_t)a * d,
                                        acc.keys.begin() + (size_t)a * d + d,
                                        acc.keys.begin() + (size_t)b * d,
                                        acc.keys.begin() + (size_t)b * d + d);
  });
  Z.assign((size_t)count * d, 0.0);
  w.assign(count, 0.0);
  for (int r = 0; r < count; ++r) {
    const int e = order[r];
    for (int t = 0; t < d; ++t) {
      double x = fine_x[acc.keys[(size_t)e * d + t]];
      Z[(size_t)r * d + t] = rule == SC_Q_GH ? lo[t] + hi[t] * x  // normal: mean lo, std hi
                                             : 0.5 * (lo[t] + hi[t]) + 0.5 * (hi[t] - lo[t]) * x;
    }
    w[r] = acc.weight[e];
  }
  return SC_OK;
}

void hn_mark_mantle(const sc_domain_desc& D, std::vector<uint8_t>& flags) {
  if (!(D.disk_radius > 0.0)) return;
  const double r2 = D.disk_radius * D.disk_radius, cx = 0.5 * D.nx, cy = 0.5 * D.ny;
  const size_t plane = (size_t)D.nx * D.ny;
  for (int y = 0; y < D.ny; ++y) {
    const double ey = (y + 0.5) - cy;
    for (int x = 0; x < D.nx; ++x) {
      const double ex = (x + 0.5) - cx;
      if (ex * ex + ey * ey > r2)
        for (int z = 0; z < D.nz; ++z) flags[(size_t)x + (size_t)D.nx * y + plane * z] = kFlagMantle;
    }
  }
}

int hn_geometry(const sc_domain_desc& D, std::vector<uint8_t>& flags) {
  const long long n = (long long)D.nx * D.ny * D.nz;
  flags.assign((size_t)n, 0);
  auto box = [&](int x0, int y0, int z0, int x1, int y1, int z1) {
    x0 = std::max(x0, 0);
    y0 = std::max(y0, 0);
    z0 = std::max(z0, 0);
    x1 = std::min(x1, D.nx);
    y1 = std::min(y1, D.ny);
    z1 = std::min(z1, D.nz);
    for (int z = z0; z < z1; ++z)
      for (int y = y0; y < y1; ++y) {
        uint8_t* row = flags.data() + (size_t)D.nx * ((size_t)y + (size_t)D.ny * z);
        for (int x = x0; x < x1; ++x) row[x] = 1;
      }
  };
  if (D.n_boxes > 0) {
    if (!D.boxes) return SC_ERR_ARG;
    for (int b = 0; b < D.n_boxes; ++b) {
      const int32_t* B = D.boxes + 6 * b;
      box(B[0], B[1], B[2], B[3], B[4], B[5]);
    }
    hn_mark_mantle(D, flags);
    return SC_OK;
  }
  Rng rng{D.geom_seed};
  const int hcap = std::min(D.h_max, D.nz - 4);
  for (int b = 0; b < D.n_buildings; ++b) {
    if (D.fp_max < D.fp_min || hcap < D.h_min) return SC_ERR_ARG;
    const int wx = rng.draw(D.fp_min, D.fp_max);
    const int wy = rng.draw(D.fp_min, D.fp_max);
    const int h = rng.draw(D.h_min, hcap);
    const int xlo = D.nx / 8, xhi = D.nx - D.nx / 8 - wx;
    const int ylo = 2, yhi = D.ny - 2 - wy;
    if (xhi < xlo || yhi < ylo) return SC_ERR_ARG;
    const int x0 = rng.draw(xlo, xhi);
    const int y0 = rng.draw(ylo, yhi);
    box(x0, y0, 0, x0 + wx, y0 + wy, h);
  }
  hn_mark_mantle(D, flags);
  return SC_OK;
}

int hn_probe_columns(const sc_domain_desc& D, const uint8_t* flags, int n, int32_t* xy) {
  Rng rng{D.geom_seed + 1ULL};
  int have = 0;
  long long attempts = 0;
  while (have < n) {
    if (++attempts > 1000000) return SC_ERR_ARG;
    const int x = rng.draw(D.nx / 8, D.nx - 1);
    const int y = rng.draw(0, D.ny - 1);
    if (flags[(size_t)x + (size_t)D.nx * y]) continue;
    bool seen = false;
    for (int k = 0; k < have && !seen; ++k) seen = xy[2 * k] == x && xy[2 * k + 1] == y;
    if (seen) continue;
    xy[2 * have] = x;
    xy[2 * have + 1] = y;
    ++have;
  }
  return SC_OK;
}

int hn_probe_points(const sc_domain_desc& D, const uint8_t* flags, int n, int32_t* xyz) {
  Rng rng{D.geom_seed + 1ULL};
  int have = 0;
  long long attempts = 0;
  while (have < n) {
    if (++attempts > 1000000) return SC_ERR_ARG;
    const int x = rng.draw(D.nx / 8, D.nx - 1);
    const int y = rng.draw(0, D.ny - 1);
    const int z = rng.draw(0, D.nz - 3);
    if (flags[(size_t)x + (size_t)D.nx * ((size_t)y + (size_t)D.ny * z)]) continue;
    bool seen = false;
    for (int k = 0; k < have && !seen; ++k)
      seen = xyz[3 * k] == x && xyz[3 * k + 1] == y && xyz[3 * k + 2] == z;
    if (seen) continue;
    xyz[3 * have] = x;
    xyz[3 * have + 1] = y;
    xyz[3 * have + 2] = z;
    ++have;
  }
  return SC_OK;
}

// Per-cell link word (see sclbm_internal.h): the kind of each link from the
// pull rules of the face kinds and the geometry.
void hn_link_words(const sc_domain_desc& D, const uint8_t* flags, std::vector<LinkWord>& link) {
  const long long n = (long long)D.nx * D.ny * D.nz;
  link.assign((size_t)n, 0ull);
  const int dims[3] = {D.nx, D.ny, D.nz};
  auto flag_at = [&](const int* q) {
    return flags[(size_t)q[0] + (size_t)D.nx * ((size_t)q[1] + (size_t)D.ny * q[2])];
  };
  auto fluid_at = [&](const int* q) { return flag_at(q) == 0; };
  // neighbour offsets of the 18 moving directions
  long long noff[kQ];
  for (int i = 0; i < kQ; ++i)
    noff[i] = (long long)kCx[i] + (long long)D.nx * ((long long)kCy[i] + (long long)D.ny * kCz[i]);
  // layers [z0, z1): each cell's word depends on the flags alone
  auto layers = [&](int z0, int z1) {
  for (int z = z0; z < z1; ++z)
    for (int y = 0; y < D.ny; ++y)
      for (int x = 0; x < D.nx; ++x) {
        const size_t c = (size_t)x + (size_t)D.nx * ((size_t)y + (size_t)D.ny * z);
        if (flags[c]) {
          link[c] = kLinkSolid;
          continue;
        }
        // a fluid cell away from every face whose 18 neighbours are fluid
        // streams on every link: word 0 (the common case, decided first)
        if (x > 0 && x < D.nx - 1 && y > 0 && y < D.ny - 1 && z > 0 && z < D.nz - 1) {
          bool all = true;
          for (int i = 1; i < kQ && all; ++i) all = flags[(size_t)((long long)c - noff[i])] == 0;
          if (all) {
            link[c] = 0;
            continue;
          }
        }
        const int xc[3] = {x, y, z};
        LinkWord word = 0;
        bool complex_cell = false, vel = false;
        for (int i = 0; i < kQ; ++i) {
          const int ci[3] = {kCx[i], kCy[i], kCz[i]};
          int p[3] = {x - ci[0], y - ci[1], z - ci[2]};
          int faces[3], nf = 0;
          bool wrapped = false;
          for (int a = 0; a < 3; ++a) {
            if (p[a] >= 0 && p[a] < dims[a]) continue;
            if (D.bc[2 * a] == SC_BC_PERIODIC) {
              p[a] = (p[a] + dims[a]) % dims[a];
              wrapped = true;
            } else {
              faces[nf++] = 2 * a + (p[a] >= dims[a] ? 1 : 0);
            }
          }
          int kind = kStream;
          if (nf == 0) {
            if (flag_at(p) == kFlagMantle) {
              kind = kMoving;  // the circular mantle's velocity boundary
              vel = true;
            } else if (!fluid_at(p)) {
              kind = kBounce;
            } else if (wrapped) {
              kind = kBounce;  // placeholder: streaming across a periodic face
              complex_cell = true;
            }
          } else {
            bool bb = false, vl = false, all_fs = true, out = false;
            for (int k = 0; k < nf; ++k) {
              const int kd = D.bc[faces[k]];
              if (kd == SC_BC_BOUNCE_BACK) bb = true;
              if (kd == SC_BC_VELOCITY) vl = true;
              if (kd == SC_BC_OUTFLOW) out = true;
              if (kd != SC_BC_FREE_SLIP) all_fs = false;
            }
            if (bb) {
              kind = kBounce;
            } else if (vl) {
              kind = kMoving;
              vel = true;
            } else if (nf == 2 && all_fs) {
              kind = kBounce;
            } else if (nf == 1 && !out && faces[0] / 2 == 2 && !wrapped) {
              // free slip at a z face: in-plane source x - (c_x, c_y, 0)
              int s[3] = {xc[0] - ci[0], xc[1] - ci[1], xc[2]};
              kind = fluid_at(s) ? kSpecZ : kBounce;
              if (flag_at(s) == kFlagMantle) {
                kind = kMoving;
                vel = true;
              }
            } else {
              kind = kBounce;  // placeholder: outflow or free slip on an x/y face
              complex_cell = true;
            }
          }
          word |= (LinkWord)kind << (2 * i);
        }
        if (complex_cell) word |= kLinkComplex;
        if (vel) word |= kLinkVel;
        if (x == D.nx - 1 && D.bc[1] == SC_BC_OUTFLOW) word |= kLinkOutlet;
        link[c] = word;
      }
  };
  parallel_layers(D.nz, (long long)D.nx * D.ny, layers);
}

// Fluid cells that need the general boundary path of the odd AA level: a
// link of a kind the fast path does not cover, or a cell on the outlet.
void hn_boundary_cells(const std::vector<LinkWord>& link, std::vector<int32_t>& cells) {
  cells.clear();
  for (size_t c = 0; c < link.size(); ++c)
    if (!(link[c] & kLinkSolid) && (link[c] & (kLinkOutlet | kLinkComplex))) cells.push_back((int32_t)c);
}

void hn_cell_classes(const std::vector<LinkWord>& link, std::vector<uint8_t>& cls) {
  cls.assign(link.size(), 0);
  for (size_t c = 0; c < link.size(); ++c) {
    const LinkWord w = link[c];
    if (w == 0) continue;  // streams on every link: class 0
    uint8_t k = 0;
    if (w & kLinkSlow) k |= kClsSkip;
    for (int i = 0; i < kQ; ++i) {
      const int kind = link_kind(w, i);
      if (kind != kStream) k |= kClsWall;
      if (kind == kMoving || kind == kSpecZ) k |= kClsMoveSpec;
    }
    cls[c] = k;
  }
}

namespace {

int h_opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
int h_dir(int x, int y, int z) {
  for (int i = 0; i < kQ; ++i)
    if (kCx[i] == x && kCy[i] == y && kCz[i] == z) return i;
  return 0;
}
int h_refl(int i, int a) {
  return h_dir(a == 0 ? -kCx[i] : kCx[i], a == 1 ? -kCy[i] : kCy[i], a == 2 ? -kCz[i] : kCz[i]);
}
int h_kout(int i) { return i == 2 ? 0 : i == 8 ? 1 : i == 10 ? 2 : i == 12 ? 3 : i == 14 ? 4 : -1; }

struct HCross {
  int n;     // faces crossed
  int f[2];  // face ids
  int p[3];  // position with periodic axes wrapped
};

HCross h_classify(const sc_domain_desc& D, int px, int py, int pz) {
  HCross c;
  c.n = 0;
  c.f[0] = c.f[1] = -1;
  int p[3] = {px, py, pz};
  const int n[3] = {D.nx, D.ny, D.nz};
  for (int a = 0; a < 3; ++a) {
    if (D.bc[2 * a] == SC_BC_PERIODIC) {
      if (p[a] < 0) p[a] += n[a];
      else if (p[a] >= n[a]) p[a] -= n[a];
    } else if (p[a] < 0) {
      c.f[c.n < 2 ? c.n : 1] = 2 * a;
      ++c.n;
    } else if (p[a] >= n[a]) {
      c.f[c.n < 2 ? c.n : 1] = 2 * a + 1;
      ++c.n;
    }
  }
  for (int a = 0; a < 3; ++a) c.p[a] = p[a];
  return c;
}

}  // namespace

// Compiles the per-link rules of the listed cells (pull form of the odd AA
// level, and the matching deliveries) into offsets:
//   source inside and solid            -> bounce-back (own slot)
//   one face crossed: BOUNCE_BACK      -> bounce-back
//                     VELOCITY         -> bounce-back + 6 w_i (c_i . u_in(z)) r
//                     FREE_SLIP        -> specular reflection from the in-plane
//                                         neighbour (bounce-back if it is solid)
//                     OUTFLOW (+x)     -> f*_i of the transverse neighbour on the
//                                         outlet plane, saved at the even level
//                                         (own saved value if that cell is solid)
//   two faces crossed: any wall        -> bounce-back; else any inflow ->
//                                         moving wall; else (outflow + free
//                                         slip) the cell's own saved f* reflected
//                                         across the free-slip face.
// Deliveries are the transpose: f*_j goes where the pull of the receiving
// link reads it; outlet cells also copy their f*_j with c_jx = -1 to the
// outlet links that read them (after the primary deliveries, which they may
// replace).
void hn_listed_links(const sc_domain_desc& D, const uint8_t* flags, const std::vector<LinkWord>& link,
                     const std::vector<int32_t>& cells, long long pitch, std::vector<ListedLinks>& tab) {
  const long long plane = (long long)D.nx * D.ny;
  auto cidx = [&](const int* p) { return (long long)p[0] + (long long)D.nx * p[1] + plane * p[2]; };
  auto loff = [&](int i) { return (long long)kCx[i] + (long long)kCy[i] * D.nx + (long long)kCz[i] * plane; };
  tab.assign(cells.size(), ListedLinks{});
  // records [k0, k1): each depends on the flags and link words alone
  auto records = [&](int k0, int k1) {
  for (size_t k = (size_t)k0; k < (size_t)k1; ++k) {
    const long long idx = cells[k];
    const int x = (int)(idx % D.nx), y = (int)((idx / D.nx) % D.ny), z = (int)(idx / plane);
    const int xyz[3] = {x, y, z};
    const LinkWord lw = link[(size_t)idx];
    ListedLinks& L = tab[k];
    memset(&L, 0, sizeof(L));
    L.z = z;
    for (int i = 0; i < kQ; ++i) {
      const long long own = (long long)i * pitch + idx;
      long long src = own;
      if (link_kind(lw, i) == kStream) {
        src = (long long)h_opp(i) * pitch + idx - loff(i);
      } else {
        const int cx = kCx[i], cy = kCy[i], cz = kCz[i];
        const HCross c = h_classify(D, x - cx, y - cy, z - cz);
        if (c.n == 0) {
          const long long p = cidx(c.p);
          if (flags[p] == 0) src = (long long)h_opp(i) * pitch + p;
          else if (flags[p] == kFlagMantle) L.pull_move |= 1u << i;
        } else if (c.n == 1) {
          const int kind = D.bc[c.f[0]];
          if (kind == SC_BC_VELOCITY) {
            L.pull_move |= 1u << i;
          } else if (kind != SC_BC_BOUNCE_BACK) {
            const int a = c.f[0] >> 1;
            int sv[3] = {x - cx, y - cy, z - cz};
            sv[a] = xyz[a];
            const HCross cs = h_classify(D, sv[0], sv[1], sv[2]);
            const long long sp = cidx(cs.p);
            if (kind == SC_BC_FREE_SLIP) {
              if (flags[sp] == 0) src = (long long)h_opp(h_refl(i, a)) * pitch + sp;
              else if (flags[sp] == kFlagMantle) L.pull_move |= 1u << i;
            } else {  // OUTFLOW on +x
              L.bout_mask |= 1u << i;
              src = flags[sp] == 0 ? ((long long)cs.p[2] * D.ny + cs.p[1]) * 5 + h_kout(i)
                                   : ((long long)z * D.ny + y) * 5 + h_kout(i);
            }
          }
        } else {
          const int k0 = D.bc[c.f[0]], k1 = D.bc[c.f[1]];
          if (k0 == SC_BC_BOUNCE_BACK || k1 == SC_BC_BOUNCE_BACK) {
          } else if (k0 == SC_BC_VELOCITY || k1 == SC_BC_VELOCITY) {
            L.pull_move |= 1u << i;
          } else if (!(k0 == SC_BC_FREE_SLIP && k1 == SC_BC_FREE_SLIP)) {
            const int fs = (k0 == SC_BC_FREE_SLIP) ? c.f[0] : c.f[1];
            L.bout_mask |= 1u << i;
            src = ((long long)z * D.ny + y) * 5 + h_kout(h_refl(i, fs >> 1));
          }
        }
      }
      L.src[i] = (int32_t)src;
    }
    for (int j = 0; j < kQ; ++j) {
      const int oj = h_opp(j);
      const long long own = (long long)oj * pitch + idx;
      long long dst = own;
      if (link_kind(lw, oj) == kStream) {
        dst = (long long)j * pitch + idx + loff(j);
      } else {
        const int cx = kCx[j], cy = kCy[j], cz = kCz[j];
        const HCross c = h_classify(D, x + cx, y + cy, z + cz);
        if (c.n == 0) {
          const long long q = cidx(c.p);
          if (flags[q] == 0) dst = (long long)j * pitch + q;
          else if (flags[q] == kFlagMantle) L.push_move |= 1u << j;
        } else if (c.n == 1) {
          const int kind = D.bc[c.f[0]];
          if (kind == SC_BC_VELOCITY) {
            L.push_move |= 1u << j;
          } else if (kind == SC_BC_FREE_SLIP) {
            const int a = c.f[0] >> 1;
            int t[3] = {x + cx, y + cy, z + cz};
            t[a] = xyz[a];
            const HCross ct = h_classify(D, t[0], t[1], t[2]);
            const long long tp = cidx(ct.p);
            if (flags[tp] == 0) dst = (long long)h_refl(j, a) * pitch + tp;
            else if (flags[tp] == kFlagMantle) L.push_move |= 1u << j;
          } else if (kind != SC_BC_BOUNCE_BACK) {
            dst = -1;  // OUTFLOW: leaves the domain
          }
        } else {
          const int k0 = D.bc[c.f[0]], k1 = D.bc[c.f[1]];
          if (k0 == SC_BC_BOUNCE_BACK || k1 == SC_BC_BOUNCE_BACK) {
          } else if (k0 == SC_BC_VELOCITY || k1 == SC_BC_VELOCITY) {
            L.push_move |= 1u << j;
          } else if (!(k0 == SC_BC_FREE_SLIP && k1 == SC_BC_FREE_SLIP)) {
            dst = -1;  // outflow + free slip: delivered by the outlet copies
          }
        }
      }
      L.dst[j] = (int32_t)dst;
    }
    for (int m = 0; m < kOutletPops * kOutletCopies; ++m) L.extra[m] = -1;
    if (lw & kLinkOutlet) {
      const int pops[kOutletPops] = {2, 8, 10, 12, 14};
      for (int e = 0; e < kOutletPops; ++e) {
        const int j = pops[e], cy = kCy[j], cz = kCz[j];
        int m = 0;
        // (1) the transverse neighbour on the outlet plane copies it
        {
          const HCross c = h_classify(D, x, y + cy, z + cz);
          if (c.n == 0 && flags[cidx(c.p)] == 0)
            L.extra[e * kOutletCopies + m++] = (int32_t)((long long)j * pitch + cidx(c.p));
        }
        // (2) own link j whose transverse source is solid takes its own value
        {
          const HCross c = h_classify(D, x, y - cy, z - cz);
          if (c.n == 0 && flags[cidx(c.p)] != 0) L.extra[e * kOutletCopies + m++] = (int32_t)((long long)j * pitch + idx);
        }
        // (3) outflow + free-slip edge: reflected copy into the own cell
        for (int a = 1; a < 3; ++a) {
          const int cj = a == 1 ? cy : cz;
          if (cj == 0) continue;
          const int face = 2 * a + (cj > 0 ? 1 : 0);
          const int pos = (a == 1 ? y : z) + cj;
          const int lim = a == 1 ? D.ny : D.nz;
          if (D.bc[face] == SC_BC_FREE_SLIP && (pos < 0 || pos >= lim))
            L.extra[e * kOutletCopies + m++] = (int32_t)((long long)h_refl(j, a) * pitch + idx);
        }
      }
    }
  }
  };
  parallel_layers((int)cells.size(), 64, records);  // a record costs about 64 cells of link words
}

void hn_inflow(int nz, double u_ref, double xi, double alpha, double H, double theta_deg,
               double* uin, int profile, double z0) {
  const double theta = theta_deg * M_PI / 180.0;
  const double c = cos(theta), s = sin(theta);
  const double lden = profile == SC_PROFILE_LOG ? log((H + z0) / z0) : 1.0;
  for (int k = 0; k < nz; ++k) {
    const double h = (double)k + 0.5;
    const double speed = profile == SC_PROFILE_LOG ? u_ref * (1.0 + xi) * log((h + z0) / z0) / lden
                                                   : u_ref * (1.0 + xi) * pow(h / H, alpha);
    uin[3 * k + 0] = speed * c;
    uin[3 * k + 1] = speed * s;
    uin[3 * k + 2] = 0.0;
  }
}

double hn_ramp(int ramp_steps, long long m) {
  if (ramp_steps <= 0) return 1.0;
  const long long mm = m < ramp_steps ? m : ramp_steps;
  return 0.5 * (1.0 - cos(M_PI * (double)mm / (double)ramp_steps));
}

void hn_series_unwrap(int n, const double* dir_deg, double* unwrapped) {
  if (n <= 0) return;
  unwrapped[0] = dir_deg[0];
  for (int k = 1; k < n; ++k) {
    // the change in [-180, 180): fmod keeps the sign of its first argument
    double turn = fmod(dir_deg[k] - dir_deg[k - 1] + 180.0, 360.0);
    if (turn < 0.0) turn += 360.0;
    unwrapped[k] = unwrapped[k - 1] + (turn - 180.0);
  }
}

void hn_series_at(int n, const double* speed, const double* unwrapped, long long per, long long interp,
                  long long m, double* s, double* d) {
  const long long k = m / per;
  if (k <= 0 || k >= n) {
    const int t = k <= 0 ? 0 : n - 1;
    *s = speed[t];
    *d = unwrapped[t];
    return;
  }
  const long long o = m - k * per;
  const double lam = interp == 0 ? 1.0 : (double)std::min(o, interp) / (double)interp;
  *s = speed[k - 1] + lam * (speed[k] - speed[k - 1]);
  *d = unwrapped[k - 1] + lam * (unwrapped[k] - unwrapped[k - 1]);
}

long long hn_wind_next_change(int ramp_steps, int n, long long per, long long interp, long long m) {
  if (m + 1 <= (long long)ramp_steps) return m + 1;  // r(m) rises up to level ramp_steps
  if (n < 2) return LLONG_MAX;
  // target k >= 1 changes the factor at levels k per + 1 .. k per + interp
  // (at k per alone when interp = 0)
  const long long k = m / per;
  if (interp > 0 && k >= 1 && k <= n - 1 && m + 1 <= k * per + interp) return m + 1;
  if (k + 1 <= n - 1) return (k + 1) * per + (interp > 0 ? 1 : 0);
  return LLONG_MAX;
}

int hn_gpc_size(int d, int degree) {
  if (degree < 0) return 0;
  return (int)choose(degree + d, d);
}

// Orthonormal Legendre products on [-1, 1]^d, graded order: total degree
// ascending; within a degree the exponent of the first input descending, then
// of the second, ...
void hn_gpc_basis(int d, int degree, const double* s, double* phi, bool hermite) {
  double leg[3][16];
  for (int t = 0; t < d; ++t) {
    leg[t][0] = 1.0;
    if (degree >= 1) leg[t][1] = s[t];
    if (hermite) {
      // orthonormal probabilists' Hermite: He_{n+1} = x He_n - n He_{n-1}, / sqrt(n!)
      for (int n = 1; n < degree; ++n) leg[t][n + 1] = s[t] * leg[t][n] - n * leg[t][n - 1];
      double fact = 1.0;
      for (int n = 0; n <= degree; ++n) {
        if (n > 1) fact *= n;
        leg[t][n] /= sqrt(fact);
      }
    } else {
      for (int n = 1; n < degree; ++n)
        leg[t][n + 1] = ((2 * n + 1) * s[t] * leg[t][n] - n * leg[t][n - 1]) / (double)(n + 1);
      for (int n = 0; n <= degree; ++n) leg[t][n] *= sqrt(2.0 * n + 1.0);
    }
  }
  int out = 0;
  for (int tot = 0; tot <= degree; ++tot) {
    if (d == 1) {
      phi[out++] = leg[0][tot];
    } else if (d == 2) {
      for (int a0 = tot; a0 >= 0; --a0) phi[out++] = leg[0][a0] * leg[1][tot - a0];
    } else {
      for (int a0 = tot; a0 >= 0; --a0)
        for (int a1 = tot - a0; a1 >= 0; --a1)
          phi[out++] = leg[0][a0] * leg[1][a1] * leg[2][tot - a0 - a1];
    }
  }
}

}  // namespace sclbm
