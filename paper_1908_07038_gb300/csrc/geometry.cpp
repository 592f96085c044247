// Host geometry of the octahedral reduced Gaussian grid (see geometry.h).
//
// Construction route: the mesh is generated edge by edge.  The zipper walk of
// every band yields the band's cross edges in longitude order; triangle k of
// the band lies between cross edges k and k+1, so the two dual-face end
// points of every edge (the centroids of its two triangles, or the pole) are
// known from the walk position without any geometric test.  Volumes are then
// gathered per node over its CSR row.
//
// Per-quantity definitions (FP64, evaluated exactly as written, no FMA
// contraction; the build passes -ffp-contract=off):
//   latitude        : Newton in colatitude on the cosine series of P_2N
//   centroid lat    : ((lat_p + lat_p) + lat_q) / 3, p = row with two vertices
//   midpoint lat    : lat_r on a ring edge, 0.5 * (lat_r + lat_s) across rows
//   end-point offset: longitude of the end point minus the edge midpoint, in
//                     turns, rounded once from the exact rational
//   S_e             : (R * (lat_L - lat_R), -(2 pi R * (off_L - off_R)))
//   segment p -> q  : -((2 pi dturns) * sin(0.5 (lat_p + lat_q))) * sinc(0.5 (lat_q - lat_p))
//   V_i             : R^2 * compensated sum of the signed segment integrals
#include "geometry.h"
#include "compsum.h"
#include "patterns.h"

#include <algorithm>
#include <cmath>
#include <cstring>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace atlasgb {
namespace {

const double kPi = 3.14159265358979323846;
const double kTwoPi = 2.0 * kPi;
const double kHalfPi = 0.5 * kPi;

inline int64_t gcd_i64(int64_t a, int64_t b) {
  a = a < 0 ? -a : a;
  b = b < 0 ? -b : b;
  while (b != 0) {
    int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}
// correctly rounded double of p/q (exact integers below 2^53 after reduction)
inline double ratio(int64_t p, int64_t q) {
  int64_t g = gcd_i64(p, q);
  if (g > 1) {
    p /= g;
    q /= g;
  }
  return static_cast<double>(p) / static_cast<double>(q);
}
inline double sinc(double x) { return x == 0.0 ? 1.0 : std::sin(x) / x; }

int row_points(int N, int r) { return 4 * ((r < N) ? r + 1 : 2 * N - r) + 16; }

// P_n(cos t) and dP/dt from the cosine series; the argument m*t is split
// into its rounded product and exact remainder.
void legendre_cos_series(int n, const std::vector<double>& coef, double t, double& P, double& dP) {
  Comp pv, dv;
  for (int k = 0; 2 * k < n; ++k) {
    const double m = static_cast<double>(n - 2 * k);
    double a, e;
    tprod(m, t, a, e);
    const double ca = std::cos(a), sa = std::sin(a);
    const double cm = ca - e * sa;
    const double sm = sa + e * ca;
    pv.add_prod(2.0 * coef[k], cm);
    dv.add_prod(-2.0 * coef[k] * m, sm);
  }
  if (n % 2 == 0) pv.add(coef[n / 2]);
  P = pv.value();
  dP = dv.value();
}

}  // namespace

// Roots of P_n as colatitudes (ascending from the north pole).  The cosine
// series of the Legendre polynomial, P_n(cos t) = sum_k g_k g_{n-k}
// cos((n-2k) t) with g_k = binom(2k, k) / 4^k, is evaluated directly in the
// colatitude so that the polar roots keep their relative accuracy.
void gauss_colatitudes(int n, double* theta) {
  std::vector<double> g(static_cast<size_t>(n) + 1), coef(static_cast<size_t>(n) / 2 + 1);
  g[0] = 1.0;
  for (int k = 1; k <= n; ++k) g[k] = g[k - 1] * static_cast<double>(2 * k - 1) / static_cast<double>(2 * k);
  for (int k = 0; 2 * k <= n; ++k) coef[k] = g[k] * g[n - k];
  const int half = (n + 1) / 2;
#pragma omp parallel for schedule(dynamic, 8)
  for (int k = 0; k < half; ++k) {
    double t = kPi * (static_cast<double>(k) + 0.75) / (static_cast<double>(n) + 0.5);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre_cos_series(n, coef, t, P, dP);
      const double step = P / dP;
      t -= step;
      if (std::fabs(step) <= 1e-15 * (t > 1.0 ? t : 1.0)) {
        legendre_cos_series(n, coef, t, P, dP);  // one polishing step
        t -= P / dP;
        break;
      }
    }
    theta[k] = t;
  }
  for (int k = 0; k < n / 2; ++k) theta[n - 1 - k] = kPi - theta[k];
  if (n % 2 == 1) theta[n / 2] = kHalfPi;
}

bool build_grid(int N, Grid& g) {
  if (N < 1 || N > 8000) return false;
  g.N = N;
  g.nlat = 2 * N;
  g.pl.resize(g.nlat);
  g.off.resize(g.nlat + 1);
  g.colat.resize(g.nlat);
  g.lat.resize(g.nlat);
  gauss_colatitudes(g.nlat, g.colat.data());
  for (int r = 0; r < g.nlat; ++r) g.lat[r] = kHalfPi - g.colat[r];
  for (int r = 0; r < N; ++r) g.lat[g.nlat - 1 - r] = -g.lat[r];
  g.off[0] = 0;
  for (int r = 0; r < g.nlat; ++r) {
    g.pl[r] = row_points(N, r);
    g.off[r + 1] = g.off[r] + g.pl[r];
  }
  g.nnodes = g.off[g.nlat];
  g.lonlat.resize(static_cast<size_t>(2 * g.nnodes));
#pragma omp parallel for schedule(dynamic, 16)
  for (int r = 0; r < g.nlat; ++r)
    for (int j = 0; j < g.pl[r]; ++j) {
      const int64_t i = g.off[r] + j;
      g.lonlat[2 * i] = kTwoPi * ratio(j, g.pl[r]);
      g.lonlat[2 * i + 1] = g.lat[r];
    }
  return true;
}

namespace {

// One step of the zipper walk of band (r, r+1): true if the northern row
// advances.  Compare the next longitudes (ia+1)/n1 and (ib+1)/n2; on a tie
// the row with fewer points advances, and between equal rows the northern.
inline bool north_advances(int64_t ia, int64_t ib, int64_t n1, int64_t n2) {
  if (ia == n1) return false;
  if (ib == n2) return true;
  const int64_t ln = (ia + 1) * n2, ls = (ib + 1) * n1;
  if (ln != ls) return ln < ls;
  return n1 <= n2;
}

struct ForwardEdges {
  std::vector<int32_t> first;  // [V+1] first edge id with this node as 'a'
  std::vector<int32_t> b;      // [E] second endpoint, sorted within each node
  int64_t find(int32_t a, int32_t bb) const {
    for (int32_t e = first[a]; e < first[a + 1]; ++e)
      if (b[e] == bb) return e;
    return -1;
  }
};

}  // namespace

bool build_mesh(const Grid& g, Mesh& m) {
  if (g.regional()) return build_regional_mesh(g, m);
  m.grid = &g;
  const int nlat = g.nlat;
  const int64_t V = g.nnodes;
  // ---- forward-edge counts: ring (next, wrap), pole, cross edges ----
  std::vector<int32_t> cnt(static_cast<size_t>(V) + 1, 0);
  for (int r = 0; r < nlat; ++r) {
    const int n = g.pl[r];
    const int64_t o = g.off[r];
    for (int j = 0; j < n; ++j) {
      int c = 0;
      if (j < n - 1) ++c;                                    // (j, j+1)
      if (j == 0) ++c;                                       // wrap (0, n-1)
      if ((r == 0 || r == nlat - 1) && j < n / 2) ++c;       // pole edge (j, j+n/2)
      cnt[o + j] += c;
    }
  }
  for (int r = 0; r + 1 < nlat; ++r) {  // cross edges of band r, one per walk position
    const int64_t n1 = g.pl[r], n2 = g.pl[r + 1];
    int64_t ia = 0, ib = 0;
    for (int64_t k = 0; k < n1 + n2; ++k) {
      cnt[g.off[r] + (ia % n1)] += 1;  // cross edge k = (N(ia), S(ib)), before the step
      if (north_advances(ia, ib, n1, n2)) ++ia; else ++ib;
    }
  }
  ForwardEdges fe;
  fe.first.assign(static_cast<size_t>(V) + 1, 0);
  for (int64_t i = 0; i < V; ++i) fe.first[i + 1] = fe.first[i] + cnt[i];
  const int64_t E = fe.first[V];
  // ring edges V, cross edges 2V - n_first - n_last, pole edges (n_first + n_last)/2
  if (E != 3 * V - (g.pl[0] + g.pl[nlat - 1]) / 2) return false;
  m.nedges = E;
  fe.b.assign(static_cast<size_t>(E), -1);
  std::vector<int32_t> fill(fe.first.begin(), fe.first.end() - 1);
  for (int r = 0; r < nlat; ++r) {
    const int n = g.pl[r];
    const int32_t o = static_cast<int32_t>(g.off[r]);
    for (int j = 0; j < n; ++j) {
      const int32_t a = o + j;
      if (j < n - 1) fe.b[fill[a]++] = a + 1;
      if (j == 0) fe.b[fill[a]++] = o + n - 1;
      if ((r == 0 || r == nlat - 1) && j < n / 2) fe.b[fill[a]++] = a + n / 2;
    }
  }
  for (int r = 0; r + 1 < nlat; ++r) {
    const int64_t n1 = g.pl[r], n2 = g.pl[r + 1];
    int64_t ia = 0, ib = 0;
    for (int64_t k = 0; k < n1 + n2; ++k) {
      const int32_t a = static_cast<int32_t>(g.off[r] + (ia % n1));
      fe.b[fill[a]++] = static_cast<int32_t>(g.off[r + 1] + (ib % n2));
      if (north_advances(ia, ib, n1, n2)) ++ia; else ++ib;
    }
  }
  for (int64_t i = 0; i < V; ++i) {
    std::sort(fe.b.begin() + fe.first[i], fe.b.begin() + fe.first[i + 1]);
    for (int32_t e = fe.first[i] + 1; e < fe.first[i + 1]; ++e)
      if (fe.b[e] == fe.b[e - 1]) return false;  // a pole edge may not repeat a side
  }
  m.e2n.resize(static_cast<size_t>(2 * E));
  m.is_pole.assign(static_cast<size_t>(E), 0);
  for (int64_t a = 0; a < V; ++a)
    for (int32_t e = fe.first[a]; e < fe.first[a + 1]; ++e) {
      m.e2n[2 * e] = static_cast<int32_t>(a);
      m.e2n[2 * e + 1] = fe.b[e];
    }
  for (int r = 0; r < nlat; r += nlat - 1) {
    const int n = g.pl[r];
    for (int j = 0; j < n / 2; ++j) {
      const int64_t e = fe.find(static_cast<int32_t>(g.off[r] + j), static_cast<int32_t>(g.off[r] + j + n / 2));
      if (e < 0) return false;
      m.is_pole[e] = 1;
    }
  }
  // ---- CSR node -> edges (ascending edge id) ----
  m.n2e_ptr.assign(static_cast<size_t>(V) + 1, 0);
  for (int64_t e = 0; e < E; ++e) {
    m.n2e_ptr[m.e2n[2 * e] + 1]++;
    m.n2e_ptr[m.e2n[2 * e + 1] + 1]++;
  }
  for (int64_t i = 0; i < V; ++i) m.n2e_ptr[i + 1] += m.n2e_ptr[i];
  m.n2e.resize(static_cast<size_t>(2 * E));
  m.n2e_sign.resize(static_cast<size_t>(2 * E));
  {
    std::vector<int32_t> pos(m.n2e_ptr.begin(), m.n2e_ptr.end() - 1);
    for (int64_t e = 0; e < E; ++e) {
      const int32_t a = m.e2n[2 * e], b = m.e2n[2 * e + 1];
      m.n2e[pos[a]] = static_cast<int32_t>(e);
      m.n2e_sign[pos[a]++] = 1;
      m.n2e[pos[b]] = static_cast<int32_t>(e);
      m.n2e_sign[pos[b]++] = -1;
    }
  }
  // ---- triangles and dual-face end points from the zipper walk ----
  int64_t T = 0;
  for (int r = 0; r + 1 < nlat; ++r) T += g.pl[r] + g.pl[r + 1];
  m.ntri = T;
  m.tri.resize(static_cast<size_t>(3 * T));
  m.side_off.assign(static_cast<size_t>(2 * E), 0.0);
  m.side_lat.assign(static_cast<size_t>(2 * E), 0.0);
  m.mid_lat.assign(static_cast<size_t>(E), 0.0);
  std::vector<int64_t> tri_base(static_cast<size_t>(nlat), 0);
  for (int r = 0; r + 1 < nlat; ++r) tri_base[r + 1] = tri_base[r] + g.pl[r] + g.pl[r + 1];
  bool ok = true;
#pragma omp parallel for schedule(dynamic, 1) reduction(&& : ok)
  for (int r = 0; r < nlat - 1; ++r) {
    const int s = r + 1;
    const int64_t n1 = g.pl[r], n2 = g.pl[s];
    const int64_t o1 = g.off[r], o2 = g.off[s];
    const int64_t D = 6 * n1 * n2;  // every longitude of the band is an integer / D turns
    const double lat_r = g.lat[r], lat_s = g.lat[s];
    const double cent_n = ((lat_r + lat_r) + lat_s) / 3.0;  // two vertices in the northern row
    const double cent_s = ((lat_s + lat_s) + lat_r) / 3.0;  // two vertices in the southern row
    auto node = [&](int64_t o, int64_t n, int64_t j) { return static_cast<int32_t>(o + (j % n)); };
    auto set_side = [&](int64_t e, int side, double off, double lat) {
      m.side_off[2 * e + side] = off;
      m.side_lat[2 * e + side] = lat;
    };
    // cross edge k is bounded by triangle k on its left (east) and k-1 on its right (west)
    int64_t ia = 0, ib = 0;
    const int64_t K = n1 + n2;
    int64_t e_first = -1;
    for (int64_t k = 0; k < K; ++k) {
      const bool north = north_advances(ia, ib, n1, n2);
      const int64_t xa = ia * 6 * n2, xb = ib * 6 * n1;  // west cross edge, both ends
      const int64_t xc = north ? (ia + 1) * 6 * n2 : (ib + 1) * 6 * n1;
      const int64_t cD = (xa + xb + xc) / 3;
      const double clat = north ? cent_n : cent_s;
      int32_t* t = &m.tri[3 * (tri_base[r] + k)];
      t[0] = node(o1, n1, ia);
      if (north) { t[1] = node(o1, n1, ia + 1); t[2] = node(o2, n2, ib); }
      else { t[1] = node(o2, n2, ib); t[2] = node(o2, n2, ib + 1); }
      // west cross edge (N(ia), S(ib)): this triangle is on its left
      const int64_t ew = fe.find(node(o1, n1, ia), node(o2, n2, ib));
      if (ew < 0) { ok = false; break; }
      if (k == 0) e_first = ew;
      set_side(ew, 0, ratio(2 * cD - (xa + xb), 2 * D), clat);
      // east cross edge: this triangle is on its right
      const int64_t na = north ? ia + 1 : ia, nb = north ? ib : ib + 1;
      const int64_t ee = (k + 1 < K) ? fe.find(node(o1, n1, na), node(o2, n2, nb)) : e_first;
      if (ee < 0) { ok = false; break; }
      set_side(ee, 1, ratio(2 * cD - (na * 6 * n2 + nb * 6 * n1), 2 * D), clat);
      // ring edge of the advancing row
      if (north) {
        // row r edge (ia, ia+1); the triangle lies south of it
        const int32_t u = node(o1, n1, ia), v = node(o1, n1, ia + 1);
        const bool wrap = (ia + 1 == n1);
        const int64_t er = wrap ? fe.find(v, u) : fe.find(u, v);
        if (er < 0) { ok = false; break; }
        const int side = wrap ? 0 : 1;  // eastward edge: south is right; the wrap edge runs west
        set_side(er, side, ratio(2 * cD - (xa + (ia + 1) * 6 * n2), 2 * D), clat);
        if (r == 0) set_side(er, 1 - side, 0.0, kHalfPi);  // the face continues to the pole
        ++ia;
      } else {
        // row s edge (ib, ib+1); the triangle lies north of it
        const int32_t u = node(o2, n2, ib), v = node(o2, n2, ib + 1);
        const bool wrap = (ib + 1 == n2);
        const int64_t er = wrap ? fe.find(v, u) : fe.find(u, v);
        if (er < 0) { ok = false; break; }
        const int side = wrap ? 1 : 0;  // eastward edge: north is left
        set_side(er, side, ratio(2 * cD - (xb + (ib + 1) * 6 * n1), 2 * D), clat);
        if (s == nlat - 1) set_side(er, 1 - side, 0.0, -kHalfPi);
        ++ib;
      }
    }
  }
  if (!ok) return false;
  // midpoint latitude of every edge: its row, or the mean of the two rows
  std::vector<int32_t> row_of(static_cast<size_t>(V));
  for (int r = 0; r < nlat; ++r)
    for (int64_t i = g.off[r]; i < g.off[r + 1]; ++i) row_of[i] = r;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < E; ++e) {
    const int ra = row_of[m.e2n[2 * e]], rb = row_of[m.e2n[2 * e + 1]];
    m.mid_lat[e] = (ra == rb) ? g.lat[ra] : 0.5 * (g.lat[ra] + g.lat[rb]);
  }
  return true;
}

bool build_dual(const Mesh& m, double R, Dual& d) {
  if (m.grid->regional()) return build_regional_dual(m, R, d);
  const Grid& g = *m.grid;
  const int64_t V = g.nnodes, E = m.nedges;
  if (!(R > 0)) return false;
  d.R = R;
  d.S.assign(static_cast<size_t>(2 * E), 0.0);
  d.V.assign(static_cast<size_t>(V), 0.0);
  d.coslat.resize(static_cast<size_t>(V));
  d.pole_nphi.assign(static_cast<size_t>(V), 0.0);
  const double C = kTwoPi * R;
  std::vector<double> seg(static_cast<size_t>(2 * E), 0.0);  // integrals of c_R -> m and m -> c_L
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < E; ++e) {
    if (m.is_pole[e]) {
      const int32_t a = m.e2n[2 * e];
      const bool north = a < g.pl[0];
      const double sp = C * ratio(1, north ? g.pl[0] : g.pl[g.nlat - 1]);
      d.S[2 * e] = 0.0;
      d.S[2 * e + 1] = north ? sp : -sp;
      continue;
    }
    const double offL = m.side_off[2 * e], offR = m.side_off[2 * e + 1];
    const double latL = m.side_lat[2 * e], latR = m.side_lat[2 * e + 1], latm = m.mid_lat[e];
    d.S[2 * e] = R * (latL - latR);
    d.S[2 * e + 1] = -(C * (offL - offR));
    const double d1 = -offR, d2 = offL;
    seg[2 * e] = -((kTwoPi * d1) * std::sin(0.5 * (latR + latm))) * sinc(0.5 * (latm - latR));
    seg[2 * e + 1] = -((kTwoPi * d2) * std::sin(0.5 * (latm + latL))) * sinc(0.5 * (latL - latm));
  }
  const double R2 = R * R;
  const int nlat = g.nlat;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < V; ++i) {
    Comp acc;
    for (int32_t q = m.n2e_ptr[i]; q < m.n2e_ptr[i + 1]; ++q) {
      const int32_t e = m.n2e[q];
      if (m.is_pole[e]) continue;
      if (m.n2e_sign[q] > 0) {
        acc.add(seg[2 * e]);
        acc.add(seg[2 * e + 1]);
      } else {
        acc.add(-seg[2 * e]);
        acc.add(-seg[2 * e + 1]);
      }
    }
    const int r = static_cast<int>(std::upper_bound(g.off.begin(), g.off.end(), i) - g.off.begin()) - 1;
    if (r == 0 || r == nlat - 1) {
      acc.add(kTwoPi * ratio(1, g.pl[r]));  // pole segment of the polar cell
      const double sp = C * ratio(1, g.pl[r]);
      d.pole_nphi[i] = (r == 0) ? sp : -sp;
    }
    d.V[i] = R2 * acc.value();
    d.coslat[i] = std::cos(g.lat[r]);
  }
  return true;
}

// ---------------------------------------------------------------------------
// Stencil tables.  n_ie denotes the outward normal of cell i on the face of
// edge e: s_ie S_e for a regular edge, S_e at both ends of a pole edge.
// ---------------------------------------------------------------------------
namespace {

inline int32_t other_end(const Mesh& m, int32_t e, int64_t i) {
  const int32_t a = m.e2n[2 * e], b = m.e2n[2 * e + 1];
  return a == i ? b : a;
}
inline void normal_of(const Mesh& m, const Dual& d, int32_t q, double& nl, double& np) {
  const int32_t e = m.n2e[q];
  const double s = m.is_pole[e] ? 1.0 : static_cast<double>(m.n2e_sign[q]);
  nl = s * d.S[2 * e];
  np = s * d.S[2 * e + 1];
}
// normal of cell j on the face it shares with cell i through edge e
inline void normal_seen_from(const Mesh& m, const Dual& d, int32_t e, int64_t j, double& nl, double& np) {
  const double s = m.is_pole[e] ? 1.0 : (m.e2n[2 * e] == j ? 1.0 : -1.0);
  nl = s * d.S[2 * e];
  np = s * d.S[2 * e + 1];
}

// gradient weights of row i on its edge through CSR slot q
inline void grad_w(const Mesh& m, const Dual& d, int64_t i, int32_t q, double& w0, double& w1) {
  double nl, np;
  normal_of(m, d, q, nl, np);
  w0 = nl / (2.0 * d.V[i]);
  w1 = d.coslat[i] * np / (2.0 * d.V[i]);
}
// divergence weights of row i towards neighbour j (regular edge)
inline void div_w(const Dual& d, int64_t i, int64_t j, double nl, double np, double& w0, double& w1) {
  w0 = nl / (2.0 * d.V[i]);
  w1 = np * d.coslat[j] / (2.0 * d.V[i]);
}
// phi-coefficient of v_i in the divergence of row i:
//   [ sum_regular n_phi (cos_j - cos_i)/2 - cos_i n_pole,phi ] / V_i
double div_vdiag(const Mesh& m, const Dual& d, int64_t i) {
  Comp acc;
  const double ci = d.coslat[i];
  for (int32_t q = m.n2e_ptr[i]; q < m.n2e_ptr[i + 1]; ++q) {
    const int32_t e = m.n2e[q];
    if (m.is_pole[e]) continue;
    double nl, np;
    normal_of(m, d, q, nl, np);
    const int32_t j = other_end(m, e, i);
    acc.add_prod(np, 0.5 * (d.coslat[j] - ci));
  }
  acc.add_prod(-ci, d.pole_nphi[i]);
  return acc.value() / d.V[i];
}

}  // namespace

namespace {
bool build_stencil_by_id(const Mesh& m, const Dual& d, int op, Stencil& s);
}  // namespace

// Entry order within each node's row: first the neighbours on the node's own
// grid row at offsets -2, -1, +1, +2 along the row (a ring on global grids;
// those present, in that order), then the others by ascending id.  Every
// kernel accumulates a node's terms in this order, so all of them give the
// same bits; the node-group kernels take a group's in-group row neighbours
// from registers because their positions are known.
namespace {
void row_neighbours_first(const Grid& g, Stencil& s) {
  const bool ring = !g.regional();
#pragma omp parallel
  {
    std::vector<std::pair<int, int32_t>> row_e;  // (offset, entry)
    std::vector<int32_t> rest, nbr;
    std::vector<double> w;
#pragma omp for schedule(static)
    for (int r = 0; r < g.nlat; ++r) {
      const int64_t a = g.off[r], n = g.off[r + 1] - g.off[r];
      for (int64_t i = a; i < a + n; ++i) {
        const int32_t q0 = s.ptr[i], q1 = s.ptr[i + 1];
        row_e.clear();
        rest.clear();
        for (int32_t q = q0; q < q1; ++q) {
          const int64_t j = s.nbr[q];
          int64_t off = j - i;
          if (j >= a && j < a + n && ring) {
            off = ((j - i) % n + n) % n;  // ring offset in (-n/2, n/2]
            if (2 * off > n) off -= n;
          }
          if (j >= a && j < a + n && off != 0 && off >= -2 && off <= 2)
            row_e.emplace_back(static_cast<int>(off), q);
          else
            rest.push_back(q);
        }
        if (row_e.empty()) continue;
        std::stable_sort(row_e.begin(), row_e.end(),
                         [](const std::pair<int, int32_t>& x, const std::pair<int, int32_t>& y) { return x.first < y.first; });
        nbr.clear();
        w.clear();
        auto take = [&](int32_t q) {
          nbr.push_back(s.nbr[q]);
          w.push_back(s.w[2 * static_cast<int64_t>(q)]);
          w.push_back(s.w[2 * static_cast<int64_t>(q) + 1]);
        };
        for (const auto& x : row_e) take(x.second);
        for (int32_t q : rest) take(q);
        for (int32_t k = 0; k < q1 - q0; ++k) {
          s.nbr[q0 + k] = nbr[k];
          s.w[2 * static_cast<int64_t>(q0 + k)] = w[2 * k];
          s.w[2 * static_cast<int64_t>(q0 + k) + 1] = w[2 * k + 1];
        }
      }
    }
  }
}
}  // namespace

bool build_stencil(const Mesh& m, const Dual& d, int op, Stencil& s) {
  if (!build_stencil_by_id(m, d, op, s)) return false;
  row_neighbours_first(*m.grid, s);
  return true;
}

namespace {
// Rows in ascending neighbour id.
bool build_stencil_by_id(const Mesh& m, const Dual& d, int op, Stencil& s) {
  if (m.grid->regional()) return build_regional_stencil(m, d, op, s);
  if (op == OP_CURL_ADJ) {
    // the exact transpose of the curl's table (its faces are the regular
    // edges, a symmetric pattern)
    Stencil c;
    if (!build_stencil_by_id(m, d, OP_CURL, c)) return false;
    return transpose_stencil(c, s);
  }
  const int64_t V = m.grid->nnodes;
  s.ptr.assign(static_cast<size_t>(V) + 1, 0);
  const bool regular_only = (op == OP_DIV || op == OP_DIV_ADJ || op == OP_CURL);
  if (op == OP_LAP) {
    s.nin = 1; s.nout = 1; s.has_b = false; s.scalar_w = true;
    // L = D G as sparse matrices; the row sums of L vanish (G applied to a
    // constant is zero), so only the off-diagonal entries are stored.
    std::vector<double> vdiag(static_cast<size_t>(V));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < V; ++i) vdiag[i] = div_vdiag(m, d, i);
    struct Acc { int32_t col; Comp v; };
    auto row = [&](int64_t i, std::vector<Acc>& out) {
      out.clear();
      auto add = [&](int32_t col, double a, double b) {
        for (auto& x : out)
          if (x.col == col) { x.v.add_prod(a, b); return; }
        out.push_back(Acc{col, Comp{}});
        out.back().v.add_prod(a, b);
      };
      // D row i: (k, du, dv); diagonal pieces kept separate
      auto g_row = [&](int64_t k, double du, double dv) {
        for (int32_t q = m.n2e_ptr[k]; q < m.n2e_ptr[k + 1]; ++q) {
          double gl, gp;
          grad_w(m, d, k, q, gl, gp);
          const int32_t j = other_end(m, m.n2e[q], k);
          add(j, du, gl); add(j, dv, gp);
          add(static_cast<int32_t>(k), du, -gl); add(static_cast<int32_t>(k), dv, -gp);
        }
      };
      for (int32_t q = m.n2e_ptr[i]; q < m.n2e_ptr[i + 1]; ++q) {
        const int32_t e = m.n2e[q];
        if (m.is_pole[e]) continue;
        double nl, np, du, dv;
        normal_of(m, d, q, nl, np);
        const int32_t k = other_end(m, e, i);
        div_w(d, i, k, nl, np, du, dv);
        g_row(k, du, dv);
        g_row(i, -du, -dv);
      }
      g_row(i, 0.0, vdiag[i]);
      std::sort(out.begin(), out.end(), [](const Acc& x, const Acc& y) { return x.col < y.col; });
    };
    std::vector<int32_t> len(static_cast<size_t>(V));
#pragma omp parallel
    {
      std::vector<Acc> buf;
#pragma omp for schedule(dynamic, 256)
      for (int64_t i = 0; i < V; ++i) {
        row(i, buf);
        len[i] = static_cast<int32_t>(buf.size()) - 1;  // minus the diagonal
      }
    }
    for (int64_t i = 0; i < V; ++i) {
      if (static_cast<int64_t>(s.ptr[i]) + len[i] > INT32_MAX) return false;
      s.ptr[i + 1] = s.ptr[i] + len[i];
    }
    s.nbr.resize(static_cast<size_t>(s.ptr[V]));
    s.w.assign(static_cast<size_t>(2 * s.ptr[V]), 0.0);
#pragma omp parallel
    {
      std::vector<Acc> buf;
#pragma omp for schedule(dynamic, 256)
      for (int64_t i = 0; i < V; ++i) {
        row(i, buf);
        int32_t q = s.ptr[i];
        for (auto& x : buf) {
          if (x.col == i) continue;
          s.nbr[q] = x.col;
          s.w[2 * static_cast<int64_t>(q)] = x.v.value();
          ++q;
        }
      }
    }
    return true;
  }
  // 1-ring stencils
  for (int64_t i = 0; i < V; ++i) {
    int32_t c = 0;
    for (int32_t q = m.n2e_ptr[i]; q < m.n2e_ptr[i + 1]; ++q)
      if (!(regular_only && m.is_pole[m.n2e[q]])) ++c;
    s.ptr[i + 1] = s.ptr[i] + c;
  }
  const int64_t nnz = s.ptr[V];
  s.nbr.resize(static_cast<size_t>(nnz));
  s.w.resize(static_cast<size_t>(2 * nnz));
  s.has_b = (op != OP_GRAD);
  s.scalar_w = false;
  s.nin = (op == OP_GRAD || op == OP_DIV_ADJ || op == OP_VGRAD) ? 1 : 2;
  s.nout = 3 - s.nin;
  if (s.has_b) s.b.assign(static_cast<size_t>(2 * V), 0.0);
  std::vector<double> vdiag;
  if (op == OP_DIV || op == OP_DIV_ADJ || op == OP_CURL) {
    vdiag.resize(static_cast<size_t>(V));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < V; ++i) vdiag[i] = div_vdiag(m, d, i);
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < V; ++i) {
    int32_t o = s.ptr[i];
    Comp b0, b1;
    for (int32_t q = m.n2e_ptr[i]; q < m.n2e_ptr[i + 1]; ++q) {
      const int32_t e = m.n2e[q];
      if (regular_only && m.is_pole[e]) continue;
      const int32_t j = other_end(m, e, i);
      double w0 = 0, w1 = 0;
      if (op == OP_GRAD) {
        grad_w(m, d, i, q, w0, w1);
      } else if (op == OP_DIV) {
        double nl, np;
        normal_of(m, d, q, nl, np);
        div_w(d, i, j, nl, np, w0, w1);
      } else if (op == OP_CURL) {
        // circulation = flux of G = (v, -u cos): the divergence weights with
        // the inputs exchanged and the u weight negated (inputs are (u, v))
        double nl, np, dl, dp;
        normal_of(m, d, q, nl, np);
        div_w(d, i, j, nl, np, dl, dp);
        w0 = -dp;
        w1 = dl;
      } else if (op == OP_VGRAD) {
        // gradient weights; on the pole edge the antipode's component enters
        // reversed: -w (x_j + x_i) = -w (x_j - x_i) - 2 w x_i
        grad_w(m, d, i, q, w0, w1);
        if (m.is_pole[e]) {
          w0 = -w0;
          w1 = -w1;
          b0.add(2.0 * w0);
          b1.add(2.0 * w1);
        }
      } else if (op == OP_GRAD_ADJ) {
        // column i of row j of the gradient: weights of row j towards node i
        double nl, np;
        normal_seen_from(m, d, e, j, nl, np);
        w0 = nl / (2.0 * d.V[j]);
        w1 = d.coslat[j] * np / (2.0 * d.V[j]);
        double r0, r1;
        grad_w(m, d, i, q, r0, r1);
        b0.add(w0); b0.add(-r0);
        b1.add(w1); b1.add(-r1);
      } else {  // OP_DIV_ADJ: column i of row j of the divergence
        double nl, np;
        normal_seen_from(m, d, e, j, nl, np);
        div_w(d, j, i, nl, np, w0, w1);
        double own_l, own_p, r0, r1;
        normal_of(m, d, q, own_l, own_p);
        div_w(d, i, j, own_l, own_p, r0, r1);
        b0.add(w0); b0.add(-r0);
        b1.add(w1); b1.add(-r1);
      }
      s.nbr[o] = j;
      s.w[2 * static_cast<int64_t>(o)] = w0;
      s.w[2 * static_cast<int64_t>(o) + 1] = w1;
      ++o;
    }
    if (op == OP_DIV) {
      s.b[2 * i] = 0.0;
      s.b[2 * i + 1] = vdiag[i];
    } else if (op == OP_CURL) {
      s.b[2 * i] = -vdiag[i];
      s.b[2 * i + 1] = 0.0;
    } else if (op == OP_VGRAD) {
      s.b[2 * i] = b0.value();
      s.b[2 * i + 1] = b1.value();
    } else if (op == OP_GRAD_ADJ) {
      s.b[2 * i] = b0.value();
      s.b[2 * i + 1] = b1.value();
    } else if (op == OP_DIV_ADJ) {
      s.b[2 * i] = b0.value();
      b1.add(vdiag[i]);
      s.b[2 * i + 1] = b1.value();
    }
  }
  return true;
}

}  // namespace

bool build_group_stencil(const Stencil& s, const Grid& g, GroupStencil& gs) {
  const int64_t V = static_cast<int64_t>(s.ptr.size()) - 1;
  if (V != g.nnodes || static_cast<int64_t>(g.off.size()) != g.nlat + 1 || V >= (int64_t(1) << 28)) return false;
  const int nw = s.scalar_w ? 1 : 2;
  gs.nw = nw;
  // groups: every row cut into runs of kGroup nodes (the last one shorter)
  gs.first.clear();
  gs.row_start.clear();
  for (int r = 0; r < g.nlat; ++r)
    for (int64_t i = g.off[r]; i < g.off[r + 1]; i += kGroup) {
      gs.row_start.push_back(i == g.off[r] ? 1 : 0);
      gs.first.push_back(i);
    }
  const int64_t ng = static_cast<int64_t>(gs.first.size());
  gs.first.push_back(V);
  // merged rows: sizes first, then contents
  std::vector<int32_t> len(static_cast<size_t>(ng));
  auto merged = [&](int64_t gi, std::vector<int32_t>& cols) {
    cols.clear();
    for (int64_t i = gs.first[gi]; i < gs.first[gi + 1]; ++i)
      for (int32_t q = s.ptr[i]; q < s.ptr[i + 1]; ++q) cols.push_back(s.nbr[q]);
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
  };
#pragma omp parallel
  {
    std::vector<int32_t> cols;
#pragma omp for schedule(static)
    for (int64_t gi = 0; gi < ng; ++gi) {
      merged(gi, cols);
      len[gi] = static_cast<int32_t>(cols.size());
    }
  }
  gs.head.assign(static_cast<size_t>(4 * ng), 0);
  int64_t nent = 0;
  for (int64_t gi = 0; gi < ng; ++gi) {
    gs.head[4 * gi + 1] = static_cast<int32_t>(nent);
    nent += len[gi];
    if (nent > INT32_MAX) return false;
    gs.head[4 * gi + 2] = static_cast<int32_t>(nent);
  }
  gs.hdr.assign(static_cast<size_t>(nent), 0u);
  gs.w.assign(static_cast<size_t>(nent) * kGroup * nw, 0.0);
#pragma omp parallel
  {
    std::vector<int32_t> cols;
#pragma omp for schedule(static)
    for (int64_t gi = 0; gi < ng; ++gi) {
      merged(gi, cols);
      const int64_t f = gs.first[gi];
      const int count = static_cast<int>(gs.first[gi + 1] - f);
      const int32_t q0 = gs.head[4 * gi + 1];
      int nb = 0, imask = 0;
      for (size_t k = 0; k < cols.size(); ++k) {
        if (cols[k] < f) ++nb;
        else if (cols[k] < f + count) imask |= 1 << (cols[k] - f);
      }
      for (int t = 0; t < count; ++t) {
        const int64_t i = f + t;
        for (int32_t q = s.ptr[i]; q < s.ptr[i + 1]; ++q) {
          const size_t k = static_cast<size_t>(std::lower_bound(cols.begin(), cols.end(), s.nbr[q]) - cols.begin());
          const size_t e = static_cast<size_t>(q0) + k;
          gs.hdr[e] |= 1u << (28 + t);
          for (int c = 0; c < nw; ++c) gs.w[(e * kGroup + t) * nw + c] = s.w[2 * static_cast<int64_t>(q) + c];
        }
      }
      for (size_t k = 0; k < cols.size(); ++k) gs.hdr[static_cast<size_t>(q0) + k] |= static_cast<uint32_t>(cols[k]);
      gs.head[4 * gi] = static_cast<int32_t>(f);
      gs.head[4 * gi + 3] = nb | (count << 16) | (imask << 20);
    }
  }
  return true;
}

namespace {

// The union of the stencil rows of the four nodes first .. first + 3 (one
// grid row, nodes row0 .. row0 + rowlen - 1, periodic) in pattern P's order
// (patterns.h): the run of own-row offsets, then the other neighbours by
// ascending id.  True, with the union in `order`, when it matches P entry
// by entry and every node's row is a subsequence of it.
template <class P>
bool union_of(const Stencil& s, int64_t first, int64_t row0, int64_t rowlen, std::vector<int32_t>& order) {
  order.clear();
  if (rowlen < P::NRUN) return false;
  for (int e = 0; e < P::NRUN; ++e) {
    int64_t o = (first - row0 + P::RUN0 + e) % rowlen;
    if (o < 0) o += rowlen;
    order.push_back(static_cast<int32_t>(row0 + o));
  }
  std::vector<int32_t> rest;
  for (int t = 0; t < kGroup; ++t)
    for (int32_t q = s.ptr[first + t]; q < s.ptr[first + t + 1]; ++q)
      if (std::find(order.begin(), order.end(), s.nbr[q]) == order.end()) rest.push_back(s.nbr[q]);
  std::sort(rest.begin(), rest.end());
  rest.erase(std::unique(rest.begin(), rest.end()), rest.end());
  order.insert(order.end(), rest.begin(), rest.end());
  if (static_cast<int>(order.size()) != P::U) return false;
  for (int e = 0; e < P::U; ++e) {
    int m = 0;
    for (int t = 0; t < kGroup; ++t)
      for (int32_t q = s.ptr[first + t]; q < s.ptr[first + t + 1]; ++q)
        if (s.nbr[q] == order[e]) m |= 1 << t;
    if (m != P::mask(e)) return false;
  }
  for (int t = 0; t < kGroup; ++t) {
    int at = -1;
    for (int32_t q = s.ptr[first + t]; q < s.ptr[first + t + 1]; ++q) {
      const int pos = static_cast<int>(std::find(order.begin(), order.end(), s.nbr[q]) - order.begin());
      if (pos <= at) return false;
      at = pos;
    }
  }
  return true;
}

}  // namespace

bool build_tile_stencil(const GroupStencil& gs, const Stencil& s, int groups_per_tile, TileStencil& ts, bool unions,
                        int rows_per_tile) {
  const int64_t ng = static_cast<int64_t>(gs.first.size()) - 1;
  const int nw = gs.nw;
  ts.nw = nw;
  ts.groups_per_tile = groups_per_tile;
  ts.unions = unions;
  // every group's grid row: its first node and the end of the row
  std::vector<int64_t> grow0(static_cast<size_t>(ng)), grow1(static_cast<size_t>(ng));
  for (int64_t gi = 0, r0 = 0; gi < ng; ++gi) {
    if (gs.row_start[gi]) r0 = gs.first[gi];
    grow0[gi] = r0;
  }
  for (int64_t gi = ng - 1, r1 = gs.first[ng]; gi >= 0; --gi) {
    grow1[gi] = r1;
    if (gs.row_start[gi]) r1 = gs.first[gi];
  }
  // grid rows as runs of groups
  std::vector<int64_t> rg;
  for (int64_t gi = 0; gi < ng; ++gi)
    if (gs.row_start[gi]) rg.push_back(gi);
  rg.push_back(ng);
  const int64_t nrows = static_cast<int64_t>(rg.size()) - 1;
  const int rows = std::max(1, std::min({rows_per_tile, kMaxTileRows, groups_per_tile}));
  const int64_t G = std::max(1, groups_per_tile / rows);  // groups per grid row of a tile
  // Units: runs of `rows` grid rows (the last one shorter).  Tile k of a
  // unit holds groups k G .. k G + G - 1 of each of its rows (rows of a
  // unit differ by a group at most, so these are neighbours).  A unit with
  // a tile that needs more than kTileRanges copy runs is cut into single
  // rows.
  struct Span {
    int64_t ga[kMaxTileRows], gb[kMaxTileRows];
    int n;
    int64_t unit;
  };
  std::vector<uint8_t> single(static_cast<size_t>(nrows), 0);
  std::vector<Span> spans;
  std::vector<int64_t> ufirst, urow0, urows;
  std::vector<int32_t> utile;
  auto cut_units = [&]() {
    spans.clear();
    ufirst.clear();
    urow0.clear();
    urows.clear();
    utile.clear();
    for (int64_t r0 = 0; r0 < nrows;) {
      const int64_t nr = single[r0] ? 1 : std::min<int64_t>(rows, nrows - r0);
      const int64_t u = static_cast<int64_t>(ufirst.size());
      ufirst.push_back(gs.first[rg[r0]]);
      urow0.push_back(r0);
      urows.push_back(nr);
      utile.push_back(static_cast<int32_t>(spans.size()));
      int64_t most = 0;
      for (int64_t r = r0; r < r0 + nr; ++r) most = std::max(most, (rg[r + 1] - rg[r] + G - 1) / G);
      for (int64_t k = 0; k < most; ++k) {
        Span sp{};
        sp.unit = u;
        for (int64_t r = r0; r < r0 + nr; ++r) {
          const int64_t ga = rg[r] + k * G, gb = std::min(ga + G, rg[r + 1]);
          if (ga < gb) {
            sp.ga[sp.n] = ga;
            sp.gb[sp.n] = gb;
            ++sp.n;
          }
        }
        spans.push_back(sp);
      }
      r0 += nr;
    }
    ufirst.push_back(gs.first[ng]);
    utile.push_back(static_cast<int32_t>(spans.size()));
  };
  for (int pass = 0;; ++pass) {
    cut_units();
    const int64_t nt = static_cast<int64_t>(spans.size());
    if (nt >= INT32_MAX) return false;
    ts.head.assign(static_cast<size_t>(nt * kTileHead), 0);
    std::vector<std::vector<uint32_t>> blobs(static_cast<size_t>(nt));
    std::vector<uint8_t> bad(static_cast<size_t>(nt), 0);
    bool fits = true;
    int32_t max_slots = 0, max_blob = 0, max_groups = 0;
    int64_t n_union = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(max : max_slots, max_blob, max_groups) reduction(+ : n_union)
    for (int64_t t = 0; t < nt; ++t) {
      // the tile's groups, row by row
      std::vector<int64_t> gl;
      for (int p = 0; p < spans[t].n; ++p)
        for (int64_t gi = spans[t].ga[p]; gi < spans[t].gb[p]; ++gi) gl.push_back(gi);
      const int ngt = static_cast<int>(gl.size());
      // the node ids the tile reads: own nodes and every neighbour, ascending
      std::vector<int32_t> ids;
      for (const int64_t gi : gl) {
        for (int64_t i = gs.first[gi]; i < gs.first[gi + 1]; ++i) ids.push_back(static_cast<int32_t>(i));
        for (int32_t q = gs.head[4 * gi + 1]; q < gs.head[4 * gi + 2]; ++q)
          ids.push_back(static_cast<int32_t>(gs.hdr[q] & 0x0fffffffu));
      }
      std::sort(ids.begin(), ids.end());
      ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
      int32_t* h = &ts.head[static_cast<size_t>(t * kTileHead)];
      int nr = 0;
      for (size_t k = 0; k < ids.size();) {
        size_t e = k + 1;
        while (e < ids.size() && ids[e] == ids[e - 1] + 1) ++e;
        if (nr == kTileRanges) {
          nr = kTileRanges + 1;
          break;
        }
        h[8 + 4 * nr] = ids[k];
        h[8 + 4 * nr + 1] = static_cast<int32_t>(e - k);
        h[8 + 4 * nr + 2] = static_cast<int32_t>(k);
        ++nr;
        k = e;
      }
      if (nr > kTileRanges) {
        bad[t] = 1;
        continue;
      }
      auto slot = [&](int32_t j) {
        return static_cast<uint32_t>(std::lower_bound(ids.begin(), ids.end(), j) - ids.begin());
      };
      const bool has_b = s.has_b;
      std::vector<uint32_t>& b = blobs[t];
      auto put_f = [&](size_t at, double v) {
        const float x = static_cast<float>(v);
        std::memcpy(&b[at], &x, 4);
      };
      // head part: tile info, group heads, B term
      const size_t o_b = 4 + 4 * static_cast<size_t>(ngt);
      const size_t o_data = o_b + (has_b ? 8 * static_cast<size_t>(ngt) : 0);
      b.assign(o_data, 0u);
      b[0] = static_cast<uint32_t>(ngt);
      b[2] = static_cast<uint32_t>(gs.first[gl[0]]);
      for (int k = 0; k < ngt; ++k) {
        const int64_t gi = gl[k];
        if (has_b)
          for (int64_t i = gs.first[gi]; i < gs.first[gi + 1]; ++i)
            for (int c = 0; c < 2; ++c)
              put_f(o_b + 8 * static_cast<size_t>(k) + 2 * static_cast<size_t>(i - gs.first[gi]) + c, s.b[2 * i + c]);
      }
      // group header k: slot of the group's first node, word offset of its
      // data, its first node, count | regular << 16 | union << 17 | D << 20
      std::vector<int32_t> order;
      for (int k = 0; k < ngt; ++k) {
        const int64_t gi = gl[k];
        const int cnt = static_cast<int>(gs.first[gi + 1] - gs.first[gi]);
        // a union group (patterns.h): slots [U] (padded to a multiple of
        // four; entries of the group's own nodes hold their slots, unused),
        // then the weights of every (entry, node holding it) in union order,
        // nw floats each (padded likewise)
        if (unions && cnt == kGroup &&
            (s.scalar_w ? union_of<pat::Ring2>(s, gs.first[gi], grow0[gi], grow1[gi] - grow0[gi], order)
                        : union_of<pat::Ring1>(s, gs.first[gi], grow0[gi], grow1[gi] - grow0[gi], order))) {
          const int U = static_cast<int>(order.size());
          const size_t off = b.size();
          b[4 + 4 * k] = slot(static_cast<int32_t>(gs.first[gi]));
          b[4 + 4 * k + 1] = static_cast<uint32_t>(off);
          b[4 + 4 * k + 2] = static_cast<uint32_t>(gs.first[gi]);
          b[4 + 4 * k + 3] = static_cast<uint32_t>(cnt) | 1u << 16 | 1u << 17 | static_cast<uint32_t>(U) << 20;
          const size_t o_w = off + ((static_cast<size_t>(U) + 3) & ~size_t(3));
          b.resize(o_w, 0u);
          for (int e = 0; e < U; ++e) b[off + static_cast<size_t>(e)] = slot(order[e]);
          for (int e = 0; e < U; ++e)
            for (int u = 0; u < kGroup; ++u) {
              const int64_t i = gs.first[gi] + u;
              for (int32_t q = s.ptr[i]; q < s.ptr[i + 1]; ++q) {
                if (s.nbr[q] != order[e]) continue;
                for (int c = 0; c < nw; ++c) {
                  b.push_back(0u);
                  put_f(b.size() - 1, s.w[2 * static_cast<int64_t>(q) + c]);
                }
              }
            }
          b.resize((b.size() + 3) & ~size_t(3), 0u);
          ++n_union;
          continue;
        }
        // per-node rows: D = the group's longest stencil row, slots [D][4]
        // then weights as f32x2 pairs [D][4][nw][2]; entry e of node t is
        // its row's e-th term, or (own slot, weight 0) past its row's end
        int D = 0;
        for (int u = 0; u < cnt; ++u) {
          const int64_t i = gs.first[gi] + u;
          D = std::max(D, static_cast<int>(s.ptr[i + 1] - s.ptr[i]));
        }
        if (D > kMaxTileRow) {
          bad[t] = 2;
          break;
        }
        // a regular group: four nodes whose first R entries are their
        // neighbours at row offsets -1, +1 (one-ring tables, R = 2) or -2, -1,
        // +1, +2 (the Laplacian, R = 4), wherever that neighbour is a node
        // of the group; the kernels then read those values from registers
        const int R = s.scalar_w ? 4 : 2;
        static const int kOffLap[4] = {-2, -1, 1, 2}, kOffRing[2] = {-1, 1};
        const int* dr = s.scalar_w ? kOffLap : kOffRing;
        bool reg = cnt == kGroup && D >= R;
        for (int u = 0; u < cnt && reg; ++u) {
          const int64_t i = gs.first[gi] + u;
          const int32_t deg = s.ptr[i + 1] - s.ptr[i];
          for (int r = 0; r < R && reg; ++r) {
            const int tt = u + dr[r];
            if (tt >= 0 && tt < kGroup) reg = deg > r && s.nbr[s.ptr[i] + r] == gs.first[gi] + tt;
          }
        }
        const size_t off = b.size();
        b[4 + 4 * k] = slot(static_cast<int32_t>(gs.first[gi]));
        b[4 + 4 * k + 1] = static_cast<uint32_t>(off);
        b[4 + 4 * k + 2] = static_cast<uint32_t>(gs.first[gi]);
        b[4 + 4 * k + 3] = static_cast<uint32_t>(cnt) | (reg ? 1u << 16 : 0u) | static_cast<uint32_t>(D) << 20;
        b.resize(off + static_cast<size_t>(D) * 4 * (1 + 2 * nw), 0u);
        const size_t o_w = off + static_cast<size_t>(D) * 4;
        for (int u = 0; u < 4; ++u) {
          const int64_t i = gs.first[gi] + std::min(u, cnt - 1);
          const uint32_t own = slot(static_cast<int32_t>(i));
          const int32_t deg = u < cnt ? s.ptr[i + 1] - s.ptr[i] : 0;
          for (int e = 0; e < D; ++e) {
            b[off + 4 * static_cast<size_t>(e) + u] = e < deg ? slot(s.nbr[s.ptr[i] + e]) : own;
            for (int c = 0; c < nw; ++c) {
              const double v = e < deg ? s.w[2 * static_cast<int64_t>(s.ptr[i] + e) + c] : 0.0;
              const size_t at = o_w + ((static_cast<size_t>(e) * 4 + u) * nw + c) * 2;
              put_f(at, v);
              put_f(at + 1, v);
            }
          }
        }
      }
      if (bad[t]) continue;
      b.resize((b.size() + 3) & ~size_t(3), 0u);
      const size_t words = b.size();
      h[0] = static_cast<int32_t>(gs.first[gl[0]]);
      h[1] = ngt;
      h[2] = nr;
      h[3] = static_cast<int32_t>(ids.size());
      h[5] = static_cast<int32_t>(4 * words);
      max_slots = std::max(max_slots, static_cast<int32_t>(ids.size()));
      max_blob = std::max(max_blob, static_cast<int32_t>(4 * words));
      max_groups = std::max(max_groups, static_cast<int32_t>(ngt));
    }
    // a tile with too many copy runs: cut its unit into single rows and
    // start again (once); other failures keep the per-node kernels
    bool again = false;
    for (int64_t t = 0; t < nt; ++t) {
      if (!bad[t]) continue;
      const int64_t u = spans[t].unit;
      if (bad[t] == 2 || urows[u] == 1 || pass > 0) {
        fits = false;
        break;
      }
      for (int64_t r = urow0[u]; r < urow0[u] + urows[u]; ++r) single[r] = 1;
      again = true;
    }
    if (!fits) return false;
    if (again) continue;
    size_t total = 0;
    for (int64_t t = 0; t < nt; ++t) {
      ts.head[static_cast<size_t>(t * kTileHead) + 4] = static_cast<int32_t>(total / 4);
      total += blobs[t].size();
      if (total / 4 > static_cast<size_t>(INT32_MAX)) return false;
    }
    ts.blob.resize(total);
    size_t pos = 0;
    for (int64_t t = 0; t < nt; ++t) {
      std::copy(blobs[t].begin(), blobs[t].end(), ts.blob.begin() + static_cast<std::ptrdiff_t>(pos));
      pos += blobs[t].size();
    }
    ts.first = ufirst;
    ts.unit_tile = utile;
    ts.ntiles = nt;
    ts.rows_per_tile = rows;
    ts.max_slots = max_slots;
    ts.max_blob = max_blob;
    ts.max_groups = max_groups;
    ts.union_groups = n_union;
    return true;
  }
}

bool build_edge_gather(const Mesh& m, const Dual& d, int op, EdgeGather& eg, bool averaged) {
  if (m.grid->regional()) return false;  // the two-pass variant covers global grids only
  const int64_t V = m.grid->nnodes, E = m.nedges;
  const bool div = (op == OP_DIV);
  eg.ptr.assign(static_cast<size_t>(V) + 1, 0);
  for (int64_t i = 0; i < V; ++i) {
    int32_t c = 0;
    for (int32_t q = m.n2e_ptr[i]; q < m.n2e_ptr[i + 1]; ++q)
      if (!(div && m.is_pole[m.n2e[q]])) ++c;
    eg.ptr[i + 1] = eg.ptr[i] + c;
  }
  eg.ent.resize(static_cast<size_t>(eg.ptr[V]));
  eg.inv_v.resize(static_cast<size_t>(V));
  eg.cos_v.resize(static_cast<size_t>(V));
  eg.pole_coef.assign(static_cast<size_t>(V), 0.0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < V; ++i) {
    int32_t o = eg.ptr[i];
    for (int32_t q = m.n2e_ptr[i]; q < m.n2e_ptr[i + 1]; ++q) {
      const int32_t e = m.n2e[q];
      if (div && m.is_pole[e]) continue;
      // difference-form edge flux S_e (x_b - x_a)/2 enters both ends with +1;
      // a pole edge enters its second end with -1 (its normal is the same at
      // both ends).  The averaged flux S_e (x_a + x_b)/2 enters the ends of a
      // regular edge with the sign of the outward normal, +1 at a and -1 at
      // b, and both ends of a pole edge with +1.
      const bool second = m.n2e_sign[q] < 0;
      const bool neg = averaged ? (second && !m.is_pole[e]) : (m.is_pole[e] && second);
      eg.ent[o++] = (e << 1) | (neg ? 1 : 0);
    }
    eg.inv_v[i] = 1.0 / d.V[i];
    eg.cos_v[i] = d.coslat[i] / d.V[i];
    eg.pole_coef[i] = -(d.coslat[i] * d.pole_nphi[i]) / d.V[i];
  }
  eg.dcos.resize(static_cast<size_t>(E));
  for (int64_t e = 0; e < E; ++e) eg.dcos[e] = d.coslat[m.e2n[2 * e + 1]] - d.coslat[m.e2n[2 * e]];
  return true;
}

bool check_geometry(const Mesh& m, const Dual& d, double tol, double& worst, int64_t& bad_node, const char** why) {
  const Grid& g = *m.grid;
  const int64_t V = g.nnodes, E = m.nedges;
  const bool regional = g.regional();
  worst = 0.0;
  bad_node = -1;
  auto bad = [&](int64_t i, const char* w) {
    bad_node = i;
    if (why) *why = w;
    return false;
  };
  if (static_cast<int64_t>(m.n2e_ptr.size()) != V + 1 || m.n2e_ptr[0] != 0 || m.n2e_ptr[V] != 2 * E)
    return bad(-1, "node->edge offsets do not cover 2E entries");
  if (static_cast<int64_t>(d.S.size()) != 2 * E || static_cast<int64_t>(d.V.size()) != V ||
      (regional && static_cast<int64_t>(d.Sb.size()) != 2 * E))
    return bad(-1, "dual arrays have the wrong sizes");
  for (int64_t e = 0; e < E; ++e) {
    const int32_t a = m.e2n[2 * e], b = m.e2n[2 * e + 1];
    if (a < 0 || b >= V || !(a < b)) return bad(-1, "edge ends out of range or not ordered");
  }
  for (int64_t i = 0; i < V; ++i)
    if (m.n2e_ptr[i + 1] < m.n2e_ptr[i]) return bad(i, "node->edge offsets decrease");
  // every node's row, in parallel: incidence, signs, closure, volume; the
  // first failing node (lowest id) is reported
  std::vector<uint8_t> code(static_cast<size_t>(V), 0);
  std::vector<double> res(static_cast<size_t>(V), 0.0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < V; ++i) {
    Comp c0, c1;
    double absum = 0.0;
    uint8_t c = 0;
    for (int32_t q = m.n2e_ptr[i]; q < m.n2e_ptr[i + 1] && c == 0; ++q) {
      const int32_t e = m.n2e[q];
      if (e < 0 || e >= E) {
        c = 1;
        break;
      }
      const int32_t a = m.e2n[2 * e], b = m.e2n[2 * e + 1];
      const int s = m.n2e_sign[q];
      if (!((a == i && s == 1) || (b == i && s == -1))) {
        c = 2;
        break;
      }
      const double sg = m.is_pole[e] ? 1.0 : static_cast<double>(s);
      double nx = sg * d.S[2 * e], ny = sg * d.S[2 * e + 1];
      if (regional) {
        nx += 0.5 * d.Sb[2 * e];
        ny += 0.5 * d.Sb[2 * e + 1];
      }
      c0.add(nx);
      c1.add(ny);
      absum += std::fabs(nx) + std::fabs(ny);
    }
    if (c == 0) {
      const double r = (std::fabs(c0.value()) + std::fabs(c1.value())) / (absum > 0 ? absum : 1.0);
      res[i] = r;
      if (!(r <= tol)) c = 3;
      else if (!(d.V[i] > 0)) c = 4;
    }
    code[i] = c;
  }
  static const char* const kWhy[5] = {"", "edge id out of range", "edge not incident to its node, or wrong sign",
                                      "dual cell does not close", "dual volume is not positive"};
  for (int64_t i = 0; i < V; ++i) {
    if (!(res[i] <= worst)) worst = std::isnan(res[i]) ? res[i] : std::max(worst, res[i]);
    if (code[i]) return bad(i, kWhy[code[i]]);
  }
  std::vector<uint8_t> seen(static_cast<size_t>(E), 0);
  for (int64_t q = 0; q < 2 * E; ++q) {
    const int32_t e = m.n2e[q];
    seen[e] = static_cast<uint8_t>(seen[e] < 3 ? seen[e] + 1 : 3);
  }
  for (int64_t e = 0; e < E; ++e)
    if (seen[e] != 2) return bad(-1, "an edge does not appear exactly twice in the node->edge rows");
  return true;
}

}  // namespace atlasgb
