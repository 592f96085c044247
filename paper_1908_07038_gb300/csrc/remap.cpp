// Host side of grid-to-grid remapping: locate every target point in the
// source mesh and compute its three interpolation weights.
//
// The paper remaps a field from an O32 grid to an F8 grid with a linear
// element-based interpolation in three dimensions over the sphere (Sec. 4.3,
// Fig. 6).  Here a target with unit vector p is located in the source
// triangle whose plane the ray from the centre along p crosses inside the
// triangle, and its weights are the barycentric coordinates of that
// crossing point:
// t p = a + u (b - a) + v (c - a) solved by Cramer's rule, weights
// (1 - u - v, u, v).  Of several containing triangles (a crossing on a shared
// edge or vertex, up to 1e-12) the one whose smallest weight is largest is
// taken, the lowest triangle id on equality.
//
// Search: the target's latitude selects the row band (rows r, r+1) it lies
// between; in that band and the two next to it, the triangles sorted by the
// longitude of their centroid are searched by bisection and the few nearest
// are tested (all of the band if those miss).  Targets north of the first
// row or south of the last (the polar caps carry no triangle) are not
// located.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <functional>
#include <utility>
#include <vector>

#include "geometry.h"

namespace atlasgb {

namespace {

constexpr double kPi = 3.14159265358979323846;

struct Vec3 {
  double x, y, z;
};
inline Vec3 unit_vec(double lon, double lat) {
  return Vec3{std::cos(lat) * std::cos(lon), std::cos(lat) * std::sin(lon), std::sin(lat)};
}
inline Vec3 sub(const Vec3& a, const Vec3& b) { return Vec3{a.x - b.x, a.y - b.y, a.z - b.z}; }
inline Vec3 cross(const Vec3& a, const Vec3& b) {
  return Vec3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double dot(const Vec3& a, const Vec3& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Barycentric weights of the ray crossing; false if the ray misses the
// triangle's plane on the near side.
inline bool crossing(const Vec3& p, const Vec3& a, const Vec3& b, const Vec3& c, double w[3]) {
  const Vec3 e1 = sub(b, a), e2 = sub(c, a);
  const Vec3 T{-a.x, -a.y, -a.z};
  const Vec3 P = cross(p, e2);
  const double det = dot(e1, P);
  if (std::fabs(det) < 1e-300) return false;
  const double inv = 1.0 / det;
  const double u = dot(T, P) * inv;
  const Vec3 Q = cross(T, e1);
  const double v = dot(p, Q) * inv;
  const double t = dot(e2, Q) * inv;
  if (t <= 0) return false;
  w[0] = 1.0 - u - v;
  w[1] = u;
  w[2] = v;
  return true;
}

}  // namespace

bool build_remap(const Mesh& m, const double* tgt_lonlat, int64_t ntgt, std::vector<int32_t>& nodes,
                 std::vector<double>& weights, int64_t& not_located) {
  const Grid& g = *m.grid;
  const int nbands = g.nlat - 1;
  std::vector<Vec3> vx(static_cast<size_t>(g.nnodes));
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < g.nnodes; ++i) vx[i] = unit_vec(g.lonlat[2 * i], g.lonlat[2 * i + 1]);
  // triangles of each band (contiguous, n_r + n_{r+1} per band), sorted by
  // the longitude of their centroid
  std::vector<int64_t> band0(static_cast<size_t>(nbands) + 1, 0);
  for (int b = 0; b < nbands; ++b) band0[b + 1] = band0[b] + g.pl[b] + g.pl[b + 1];
  if (band0[nbands] != m.ntri) return false;
  std::vector<std::pair<double, int64_t>> order(static_cast<size_t>(m.ntri));
#pragma omp parallel for schedule(dynamic, 4)
  for (int b = 0; b < nbands; ++b) {
    for (int64_t q = band0[b]; q < band0[b + 1]; ++q) {
      const Vec3 &a = vx[m.tri[3 * q]], &bb = vx[m.tri[3 * q + 1]], &c = vx[m.tri[3 * q + 2]];
      double lon = std::atan2(a.y + bb.y + c.y, a.x + bb.x + c.x);
      if (lon < 0) lon += 2.0 * kPi;
      order[q] = {lon, q};
    }
    std::sort(order.begin() + band0[b], order.begin() + band0[b + 1]);
  }
  nodes.assign(static_cast<size_t>(3 * ntgt), -1);
  weights.assign(static_cast<size_t>(3 * ntgt), 0.0);
  int64_t missed = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : missed)
  for (int64_t t = 0; t < ntgt; ++t) {
    const double lon_t = tgt_lonlat[2 * t], lat_t = tgt_lonlat[2 * t + 1];
    const Vec3 p = unit_vec(lon_t, lat_t);
    double lon = std::fmod(lon_t, 2.0 * kPi);
    if (lon < 0) lon += 2.0 * kPi;
    // band: rows r, r+1 with lat[r] >= lat_t >= lat[r+1] (latitudes descend)
    int r = static_cast<int>(std::upper_bound(g.lat.begin(), g.lat.end(), lat_t, std::greater<double>()) -
                             g.lat.begin()) - 1;
    double best = -1e300;
    int64_t bq = -1;
    double bw[3] = {0, 0, 0};
    auto test = [&](int64_t q) {
      double w[3];
      if (!crossing(p, vx[m.tri[3 * q]], vx[m.tri[3 * q + 1]], vx[m.tri[3 * q + 2]], w)) return;
      const double mn = std::min(w[0], std::min(w[1], w[2]));
      if (mn < -1e-12) return;
      if (mn > best || (mn == best && q < bq)) {
        best = mn;
        bq = q;
        bw[0] = w[0]; bw[1] = w[1]; bw[2] = w[2];
      }
    };
    for (int pass = 0; pass < 2 && bq < 0; ++pass) {
      for (int b = std::max(0, r - 1); b <= std::min(nbands - 1, r + 1); ++b) {
        const int64_t n = band0[b + 1] - band0[b];
        if (pass == 1) {  // the near candidates missed: the whole band
          for (int64_t q = band0[b]; q < band0[b + 1]; ++q) test(q);
          continue;
        }
        const auto first = order.begin() + band0[b], last = order.begin() + band0[b + 1];
        const int64_t pos = std::lower_bound(first, last, std::make_pair(lon, int64_t(-1))) - first;
        for (int64_t d = -4; d <= 4; ++d) {
          const int64_t k = ((pos + d) % n + n) % n;
          test(order[band0[b] + k].second);
        }
      }
    }
    if (bq < 0) {
      ++missed;
      continue;
    }
    for (int k = 0; k < 3; ++k) {
      nodes[3 * t + k] = m.tri[3 * bq + k];
      weights[3 * t + k] = bw[k];
    }
  }
  not_located = missed;
  return true;
}

bool build_regular_gaussian_grid(int N, Grid& g) {
  if (N < 1 || N > 8000) return false;
  g.N = N;
  g.nlat = 2 * N;
  g.octahedral = false;
  g.pl.assign(g.nlat, 4 * N);
  g.off.resize(g.nlat + 1);
  g.colat.resize(g.nlat);
  g.lat.resize(g.nlat);
  gauss_colatitudes(g.nlat, g.colat.data());
  for (int r = 0; r < g.nlat; ++r) g.lat[r] = kPi / 2 - g.colat[r];
  for (int r = 0; r < N; ++r) g.lat[g.nlat - 1 - r] = -g.lat[r];
  g.off[0] = 0;
  for (int r = 0; r < g.nlat; ++r) g.off[r + 1] = g.off[r] + g.pl[r];
  g.nnodes = g.off[g.nlat];
  g.lonlat.resize(static_cast<size_t>(2 * g.nnodes));
  for (int r = 0; r < g.nlat; ++r)
    for (int j = 0; j < g.pl[r]; ++j) {
      const int64_t i = g.off[r] + j;
      g.lonlat[2 * i] = 2.0 * kPi * (static_cast<double>(j) / static_cast<double>(g.pl[r]));
      g.lonlat[2 * i + 1] = g.lat[r];
    }
  return true;
}

}  // namespace atlasgb
