// Regional (limited-area) grids with map projections (see geometry.h).
//
// The paper notes that Atlas generates meshes for the regional grids of
// limited-area models, and that operators taking the grid's projection into
// account were still being worked on (Sec. 2.2.3, Sec. 5).  This file builds
// such a grid, its mesh and median dual, and the operator tables:
//
//   grid   : a rectangle [xmin, xmax] x [ymin, ymax] of the projection plane,
//            x_j = xmin + j (xmax - xmin)/(nx - 1), y_r = ymax - r (ymax - ymin)/(ny - 1),
//            node id r nx + j (rows north to south of the plane, x ascending);
//            plane coordinates are kept on the unit sphere (radians, or
//            metres divided by the projection's radius)
//   mesh   : quad (r, j) split along its diagonal (r, j)-(r+1, j+1) into the
//            counter-clockwise triangles {a, a+nx+1, a+1} and {a, a+nx, a+nx+1},
//            a = r nx + j; edges a < b sorted by (a, b); node->edge CSR
//   dual   : median dual in the plane: the face of edge a->b is the polyline
//            centroid - midpoint - centroid (midpoint - centroid on the
//            boundary) with its integrated normal n_e oriented from a to b;
//            A_i = sum of one third of the adjacent triangle areas; a
//            boundary edge carries its outward normal n_b, split in halves
//            between its end nodes
//   metric : orthogonal plane coordinates with scale factors h_x, h_y (true
//            length = R h dx on a sphere of radius R), taken at the nodes;
//            V_i = h_x,i h_y,i A_i
//
// Face values: (f_i + f_j)/2 on an interior face and (5 f_i + f_j)/6 on a
// boundary half edge (the choice that makes the edge-based Green-Gauss
// gradient equal to the area-weighted average of the linear-element
// gradients, hence exact for fields linear in the plane at every node).  With
// the closure sum_e s_ie n_e + sum_b n_b/2 = 0 of each dual cell this gives
// the difference form with c_ie = s_ie n_e/2 + n_b/12:
//   grad_x(i) = sum_j c^x_ij (f_j - f_i) / (A_i h_x,i)        (same for y)
//   div(i)    = sum_j c_ij . (F_j - F_i) / V_i, F = (h_y u, h_x v)
//   curl(i)   = sum_j c_ij . (F_j - F_i) / V_i, F = (h_y v, -h_x u)
// and the Laplacian, adjoints and vector gradient from these tables.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "compsum.h"
#include "geometry.h"

namespace atlasgb {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kDeg = kPi / 180.0;

struct Proj {
  int kind = 0;
  // rotated lon-lat: frame vectors of the rotated sphere
  double e1[3] = {1, 0, 0}, e2[3] = {0, 1, 0}, e3[3] = {0, 0, 1};
  // Mercator and Lambert
  double lon0 = 0;
  double n = 1, F = 1, rho0 = 0;
};

inline void unit(double lon, double lat, double v[3]) {
  v[0] = std::cos(lat) * std::cos(lon);
  v[1] = std::cos(lat) * std::sin(lon);
  v[2] = std::sin(lat);
}

// (lon, lat, h_x, h_y) of the plane point (x, y) on the unit sphere;
// returns false where the point is outside the projection's valid range
bool inverse(const Proj& p, double x, double y, double& lon, double& lat, double& hx, double& hy) {
  if (p.kind == PROJ_ROTATED_LONLAT) {
    const double cy = std::cos(y), sy = std::sin(y), cx = std::cos(x), sx = std::sin(x);
    double v[3];
    for (int k = 0; k < 3; ++k) v[k] = cy * cx * p.e1[k] + cy * sx * p.e2[k] + sy * p.e3[k];
    lon = std::atan2(v[1], v[0]);
    lat = std::atan2(v[2], std::hypot(v[0], v[1]));
    hx = cy;
    hy = 1.0;
    return cy > 1e-3;
  }
  if (p.kind == PROJ_MERCATOR) {
    lon = p.lon0 + x;
    lat = std::atan(std::sinh(y));
    hx = hy = 1.0 / std::cosh(y);
    return std::fabs(y) <= 7.0;
  }
  if (p.kind == PROJ_POLAR_STEREOGRAPHIC) {
    // tangent plane at the pole (p.n = +1 north, -1 south), projected from
    // the opposite pole: rho = 2 tan(pi/4 - |lat|/2), the central meridian
    // lon0 pointing to -y from the north pole (+y from the south pole)
    const double rho = std::hypot(x, y);
    const double c = 2.0 * std::atan(0.5 * rho);  // angular distance from the pole
    lat = p.n * (0.5 * kPi - c);
    lon = p.lon0 + std::atan2(x, -p.n * y);
    hx = hy = std::cos(0.5 * c) * std::cos(0.5 * c);  // 1/k, k = 2/(1 + sin|lat|)
    return std::cos(c) > -1.0 + 1e-6;
  }
  // Lambert conformal conic, tangent at lat0: rho = F / tan(pi/4 + lat/2)^n,
  // x = rho sin(theta), y = rho0 - rho cos(theta), theta = n (lon - lon0)
  const double s = p.n > 0 ? 1.0 : -1.0;
  const double rho = s * std::hypot(x, p.rho0 - y);
  const double theta = std::atan2(s * x, s * (p.rho0 - y));
  if (!(std::fabs(theta) < kPi * std::fabs(p.n)) || rho == 0.0) return false;
  lon = p.lon0 + theta / p.n;
  lat = 2.0 * std::atan(std::pow(p.F / rho, 1.0 / p.n)) - 0.5 * kPi;
  hx = hy = std::cos(lat) / (p.n * rho);
  return std::cos(lat) > 1e-3;
}

}  // namespace

bool build_regional_grid(int projection, int nx, int ny, const double* prm, Grid& g, const char** why) {
  auto bad = [&](const char* w) {
    if (why) *why = w;
    return false;
  };
  if (!prm) return bad("params is NULL");
  if (nx < 2 || ny < 2) return bad("a regional grid needs nx >= 2 and ny >= 2");
  if (static_cast<int64_t>(nx) * ny > (int64_t(1) << 28)) return bad("too many points (nx * ny > 2^28)");
  const double xmin = prm[0], xmax = prm[1], ymin = prm[2], ymax = prm[3];
  if (!(std::isfinite(xmin) && std::isfinite(xmax) && std::isfinite(ymin) && std::isfinite(ymax)) ||
      !(xmin < xmax) || !(ymin < ymax))
    return bad("the domain needs finite xmin < xmax and ymin < ymax");
  Proj p;
  p.kind = projection;
  double scale = 1.0;  // plane units per unit-sphere unit
  if (projection == PROJ_ROTATED_LONLAT) {
    if (xmax - xmin >= 360.0) return bad("a rotated lon-lat domain spans less than 360 degrees");
    if (std::fabs(ymin) >= 90.0 || std::fabs(ymax) >= 90.0) return bad("rotated latitudes must lie in (-90, 90)");
    const double spl = prm[4] * kDeg, spp = prm[5] * kDeg;  // rotated south pole (GRIB convention)
    if (!(std::fabs(prm[5]) <= 90.0)) return bad("south pole latitude out of range");
    unit(spl, spp + 0.5 * kPi, p.e1);
    unit(spl + kPi, -spp, p.e3);
    p.e2[0] = p.e3[1] * p.e1[2] - p.e3[2] * p.e1[1];
    p.e2[1] = p.e3[2] * p.e1[0] - p.e3[0] * p.e1[2];
    p.e2[2] = p.e3[0] * p.e1[1] - p.e3[1] * p.e1[0];
    scale = 1.0 / kDeg;
  } else if (projection == PROJ_POLAR_STEREOGRAPHIC) {
    const double radius = prm[4];
    if (!(radius > 0) || !std::isfinite(radius)) return bad("the projection radius must be positive");
    if (prm[6] != 90.0 && prm[6] != -90.0) return bad("the polar stereographic pole latitude must be 90 or -90");
    scale = radius;
    p.lon0 = prm[5] * kDeg;
    p.n = prm[6] > 0 ? 1.0 : -1.0;
  } else if (projection == PROJ_MERCATOR || projection == PROJ_LAMBERT_CONFORMAL) {
    const double radius = prm[4];
    if (!(radius > 0) || !std::isfinite(radius)) return bad("the projection radius must be positive");
    scale = radius;
    p.lon0 = prm[5] * kDeg;
    if (projection == PROJ_MERCATOR) {
      if ((xmax - xmin) / radius >= 2 * kPi) return bad("a Mercator domain spans less than 2 pi radius");
    } else {
      const double lat0 = prm[6] * kDeg;
      if (!(std::fabs(prm[6]) > 1e-6 && std::fabs(prm[6]) < 90.0 - 1e-6))
        return bad("the Lambert tangent latitude must lie in (-90, 0) or (0, 90) degrees");
      p.n = std::sin(lat0);
      const double t0 = std::tan(0.25 * kPi + 0.5 * lat0);
      p.F = std::cos(lat0) * std::pow(t0, p.n) / p.n;
      p.rho0 = p.F / std::pow(t0, p.n);
      const double apex = p.rho0 * radius;  // the cone's apex (the pole) is at (0, apex)
      if (xmin <= 0.0 && xmax >= 0.0 && (p.n > 0 ? ymax >= apex : ymin <= apex))
        return bad("the Lambert domain contains the pole or crosses the cut opposite lon0");
    }
  } else {
    return bad("unknown projection");
  }
  const int64_t V = static_cast<int64_t>(nx) * ny;
  g.N = 0;
  g.octahedral = false;
  g.projection = projection;
  g.nx = nx;
  g.nlat = ny;
  g.nnodes = V;
  for (int k = 0; k < 8; ++k) g.proj_params[k] = prm[k];
  g.pl.assign(static_cast<size_t>(ny), nx);
  g.off.resize(static_cast<size_t>(ny) + 1);
  for (int r = 0; r <= ny; ++r) g.off[r] = static_cast<int64_t>(r) * nx;
  g.lonlat.resize(static_cast<size_t>(2 * V));
  g.xy.resize(static_cast<size_t>(2 * V));
  g.h.resize(static_cast<size_t>(2 * V));
  const double dx = (xmax - xmin) / (nx - 1), dy = (ymax - ymin) / (ny - 1);
  int bad_points = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad_points)
  for (int r = 0; r < ny; ++r) {
    const double y = (ymax - r * dy) / scale;
    for (int j = 0; j < nx; ++j) {
      const double x = (xmin + j * dx) / scale;
      const int64_t i = static_cast<int64_t>(r) * nx + j;
      double lon = 0, lat = 0, hx = 1, hy = 1;
      if (!inverse(p, x, y, lon, lat, hx, hy)) ++bad_points;
      g.xy[2 * i] = x;
      g.xy[2 * i + 1] = y;
      g.lonlat[2 * i] = lon;
      g.lonlat[2 * i + 1] = lat;
      g.h[2 * i] = hx;
      g.h[2 * i + 1] = hy;
    }
  }
  if (bad_points) return bad("the domain reaches a pole or leaves the projection's valid range");
  g.lat.resize(static_cast<size_t>(ny));
  g.colat.resize(static_cast<size_t>(ny));
  for (int r = 0; r < ny; ++r) {  // latitude of each row's first node
    g.lat[r] = g.lonlat[2 * g.off[r] + 1];
    g.colat[r] = 0.5 * kPi - g.lat[r];
  }
  return true;
}

namespace {

// id of edge (a, b), a < b, of the structured triangulation: node a's forward
// edges are, in order, a+1 (if j < nx-1), a+nx (if r < ny-1), a+nx+1 (both)
inline int64_t edge_id(const std::vector<int64_t>& first, int nx, int64_t a, int64_t b) {
  if (b == a + 1) return first[a];
  const bool has_right = (a % nx) != nx - 1;
  if (b == a + nx) return first[a] + (has_right ? 1 : 0);
  return first[a] + 2;  // b == a + nx + 1
}

}  // namespace

bool build_regional_mesh(const Grid& g, Mesh& m) {
  if (!g.regional()) return false;
  const int nx = g.nx, ny = g.nlat;
  const int64_t V = g.nnodes;
  m.grid = &g;
  m.ntri = 2 * static_cast<int64_t>(nx - 1) * (ny - 1);
  m.nedges = static_cast<int64_t>(nx - 1) * ny + static_cast<int64_t>(nx) * (ny - 1) +
             static_cast<int64_t>(nx - 1) * (ny - 1);
  if (2 * m.nedges >= (int64_t(1) << 31)) return false;
  m.e2n.resize(static_cast<size_t>(2 * m.nedges));
  m.is_pole.assign(static_cast<size_t>(m.nedges), 0);
  int64_t e = 0;
  for (int64_t a = 0; a < V; ++a) {
    const int r = static_cast<int>(a / nx), j = static_cast<int>(a % nx);
    const bool right = j < nx - 1, down = r < ny - 1;
    if (right) { m.e2n[2 * e] = static_cast<int32_t>(a); m.e2n[2 * e + 1] = static_cast<int32_t>(a + 1); ++e; }
    if (down) { m.e2n[2 * e] = static_cast<int32_t>(a); m.e2n[2 * e + 1] = static_cast<int32_t>(a + nx); ++e; }
    if (right && down) {
      m.e2n[2 * e] = static_cast<int32_t>(a);
      m.e2n[2 * e + 1] = static_cast<int32_t>(a + nx + 1);
      ++e;
    }
  }
  if (e != m.nedges) return false;
  m.tri.resize(static_cast<size_t>(3 * m.ntri));
  int64_t t = 0;
  for (int r = 0; r + 1 < ny; ++r)
    for (int j = 0; j + 1 < nx; ++j) {
      const int32_t a = static_cast<int32_t>(static_cast<int64_t>(r) * nx + j);
      const int32_t tri0[3] = {a, a + nx + 1, a + 1}, tri1[3] = {a, a + nx, a + nx + 1};
      for (int k = 0; k < 3; ++k) m.tri[3 * t + k] = tri0[k];
      ++t;
      for (int k = 0; k < 3; ++k) m.tri[3 * t + k] = tri1[k];
      ++t;
    }
  // node -> edge CSR, ascending edge id per node
  m.n2e_ptr.assign(static_cast<size_t>(V) + 1, 0);
  for (int64_t q = 0; q < 2 * m.nedges; ++q) ++m.n2e_ptr[m.e2n[q] + 1];
  for (int64_t i = 0; i < V; ++i) m.n2e_ptr[i + 1] += m.n2e_ptr[i];
  m.n2e.resize(static_cast<size_t>(2 * m.nedges));
  m.n2e_sign.resize(static_cast<size_t>(2 * m.nedges));
  std::vector<int32_t> fill(m.n2e_ptr.begin(), m.n2e_ptr.end() - 1);
  for (int64_t k = 0; k < m.nedges; ++k)
    for (int s = 0; s < 2; ++s) {
      const int32_t i = m.e2n[2 * k + s];
      m.n2e[fill[i]] = static_cast<int32_t>(k);
      m.n2e_sign[fill[i]] = s == 0 ? 1 : -1;
      ++fill[i];
    }
  m.side_off.clear();
  m.side_lat.clear();
  m.mid_lat.clear();
  return true;
}

bool build_regional_dual(const Mesh& m, double R, Dual& d) {
  const Grid& g = *m.grid;
  if (!g.regional() || !(R > 0)) return false;
  const int nx = g.nx;
  const int64_t V = g.nnodes, E = m.nedges, T = m.ntri;
  std::vector<int64_t> first(static_cast<size_t>(V) + 1, 0);
  for (int64_t k = 0; k < E; ++k) ++first[m.e2n[2 * k] + 1];
  for (int64_t i = 0; i < V; ++i) first[i + 1] += first[i];
  std::vector<double> n(static_cast<size_t>(2 * E), 0.0), nb(static_cast<size_t>(2 * E), 0.0);
  std::vector<double> tc(static_cast<size_t>(2 * E), 0.0);  // centroid of an edge's (last) triangle
  std::vector<uint8_t> cnt(static_cast<size_t>(E), 0);
  std::vector<Comp> area(static_cast<size_t>(V));
  const double* xy = g.xy.data();
  for (int64_t t = 0; t < T; ++t) {
    const int32_t* v = &m.tri[3 * t];
    const double x0 = xy[2 * v[0]], y0 = xy[2 * v[0] + 1];
    const double x1 = xy[2 * v[1]], y1 = xy[2 * v[1] + 1];
    const double x2 = xy[2 * v[2]], y2 = xy[2 * v[2] + 1];
    const double cx = (x0 + x1 + x2) / 3.0, cy = (y0 + y1 + y2) / 3.0;
    const double at = 0.5 * ((x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0));
    if (!(at > 0)) return false;
    for (int k = 0; k < 3; ++k) area[v[k]].add(at / 3.0);
    for (int k = 0; k < 3; ++k) {
      const int64_t p = v[k], q = v[(k + 1) % 3];
      const int64_t a = std::min(p, q), b = std::max(p, q);
      const int64_t e = edge_id(first, nx, a, b);
      if (e < 0 || e >= E || m.e2n[2 * e] != a || m.e2n[2 * e + 1] != b) return false;
      const double mx = 0.5 * (xy[2 * a] + xy[2 * b]), my = 0.5 * (xy[2 * a + 1] + xy[2 * b + 1]);
      // integrated normal of the segment midpoint -> centroid, oriented a -> b
      double sx = cy - my, sy = -(cx - mx);
      if (sx * (xy[2 * b] - xy[2 * a]) + sy * (xy[2 * b + 1] - xy[2 * a + 1]) < 0) {
        sx = -sx;
        sy = -sy;
      }
      n[2 * e] += sx;
      n[2 * e + 1] += sy;
      tc[2 * e] = cx;
      tc[2 * e + 1] = cy;
      ++cnt[e];
    }
  }
  for (int64_t e = 0; e < E; ++e) {
    if (cnt[e] == 2) continue;
    if (cnt[e] != 1) return false;
    const int32_t a = m.e2n[2 * e], b = m.e2n[2 * e + 1];
    const double ex = xy[2 * b] - xy[2 * a], ey = xy[2 * b + 1] - xy[2 * a + 1];
    const double mx = 0.5 * (xy[2 * a] + xy[2 * b]), my = 0.5 * (xy[2 * a + 1] + xy[2 * b + 1]);
    double ox = ey, oy = -ex;  // away from the triangle's centroid
    if (ox * (tc[2 * e] - mx) + oy * (tc[2 * e + 1] - my) > 0) {
      ox = -ox;
      oy = -oy;
    }
    nb[2 * e] = ox;
    nb[2 * e + 1] = oy;
  }
  d.R = R;
  d.S.resize(static_cast<size_t>(2 * E));
  d.Sb.resize(static_cast<size_t>(2 * E));
  for (int64_t q = 0; q < 2 * E; ++q) {
    d.S[q] = R * n[q];
    d.Sb[q] = R * nb[q];
  }
  d.A.resize(static_cast<size_t>(V));
  d.V.resize(static_cast<size_t>(V));
  d.coslat.resize(static_cast<size_t>(V));
  d.pole_nphi.assign(static_cast<size_t>(V), 0.0);
  for (int64_t i = 0; i < V; ++i) {
    d.A[i] = R * R * area[i].value();
    d.V[i] = g.h[2 * i] * g.h[2 * i + 1] * d.A[i];
    d.coslat[i] = std::cos(g.lonlat[2 * i + 1]);
  }
  return true;
}

// ---------------------------------------------------------------- tables
namespace {

// difference-form coefficient vector of row i on its CSR slot q
inline void coef(const Mesh& m, const Dual& d, int32_t q, double& cx, double& cy) {
  const int32_t e = m.n2e[q];
  const double s = static_cast<double>(m.n2e_sign[q]);
  cx = 0.5 * s * d.S[2 * e] + d.Sb[2 * e] / 12.0;
  cy = 0.5 * s * d.S[2 * e + 1] + d.Sb[2 * e + 1] / 12.0;
}
inline int32_t far_node(const Mesh& m, int32_t e, int64_t i) {
  const int32_t a = m.e2n[2 * e], b = m.e2n[2 * e + 1];
  return a == i ? b : a;
}

// one-ring tables of the gradient (op OP_GRAD), divergence (OP_DIV) and curl
void one_ring(const Mesh& m, const Dual& d, int op, Stencil& s) {
  const Grid& g = *m.grid;
  const int64_t V = g.nnodes;
  s.ptr.assign(m.n2e_ptr.begin(), m.n2e_ptr.end());
  const int64_t nnz = s.ptr[V];
  s.nbr.resize(static_cast<size_t>(nnz));
  s.w.resize(static_cast<size_t>(2 * nnz));
  s.scalar_w = false;
  s.nin = op == OP_GRAD ? 1 : 2;
  s.nout = 3 - s.nin;
  s.has_b = op != OP_GRAD;
  if (s.has_b) s.b.assign(static_cast<size_t>(2 * V), 0.0);
  const double* h = g.h.data();
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < V; ++i) {
    const double hxi = h[2 * i], hyi = h[2 * i + 1];
    Comp b0, b1;
    for (int32_t q = m.n2e_ptr[i]; q < m.n2e_ptr[i + 1]; ++q) {
      const int32_t j = far_node(m, m.n2e[q], i);
      double cx, cy;
      coef(m, d, q, cx, cy);
      double w0, w1;
      if (op == OP_GRAD) {
        w0 = cx / (d.A[i] * hxi);
        w1 = cy / (d.A[i] * hyi);
      } else if (op == OP_DIV) {  // F = (h_y u, h_x v)
        w0 = cx * h[2 * j + 1] / d.V[i];
        w1 = cy * h[2 * j] / d.V[i];
        b0.add_prod(cx, (h[2 * j + 1] - hyi) / d.V[i]);
        b1.add_prod(cy, (h[2 * j] - hxi) / d.V[i]);
      } else {  // OP_CURL: F = (h_y v, -h_x u); inputs (u, v)
        w0 = -cy * h[2 * j] / d.V[i];
        w1 = cx * h[2 * j + 1] / d.V[i];
        b0.add_prod(-cy, (h[2 * j] - hxi) / d.V[i]);
        b1.add_prod(cx, (h[2 * j + 1] - hyi) / d.V[i]);
      }
      s.nbr[q] = j;
      s.w[2 * static_cast<int64_t>(q)] = w0;
      s.w[2 * static_cast<int64_t>(q) + 1] = w1;
    }
    if (s.has_b) {
      s.b[2 * i] = b0.value();
      s.b[2 * i + 1] = b1.value();
    }
  }
}

}  // namespace

bool transpose_stencil(const Stencil& a, Stencil& t) {
  if (a.scalar_w) return false;
  const int64_t V = static_cast<int64_t>(a.ptr.size()) - 1;
  t.nin = a.nout;
  t.nout = a.nin;
  t.has_b = true;
  t.scalar_w = false;
  t.ptr = a.ptr;
  t.nbr = a.nbr;
  t.w.assign(a.w.size(), 0.0);
  t.b.assign(static_cast<size_t>(2 * V), 0.0);
  bool ok = true;
#pragma omp parallel for schedule(static) reduction(&& : ok)
  for (int64_t i = 0; i < V; ++i) {
    Comp b[2];
    if (a.has_b) {
      b[0].add(a.b[2 * i]);
      b[1].add(a.b[2 * i + 1]);
    }
    for (int32_t q = a.ptr[i]; q < a.ptr[i + 1]; ++q) {
      const int32_t j = a.nbr[q];
      int32_t r = a.ptr[j];
      while (r < a.ptr[j + 1] && a.nbr[r] != i) ++r;
      if (r == a.ptr[j + 1]) {
        ok = false;  // not a symmetric sparsity pattern
        continue;
      }
      for (int p = 0; p < 2; ++p) {
        const double wji = a.w[2 * static_cast<int64_t>(r) + p];
        t.w[2 * static_cast<int64_t>(q) + p] = wji;
        b[p].add(wji);
        b[p].add(-a.w[2 * static_cast<int64_t>(q) + p]);
      }
    }
    t.b[2 * i] = b[0].value();
    t.b[2 * i + 1] = b[1].value();
  }
  return ok;
}

bool compose_stencil(const Stencil& dd, const Stencil& gg, Stencil& l) {
  if (dd.nin != 2 || dd.nout != 1 || gg.nin != 1 || gg.nout != 2 || gg.has_b || dd.scalar_w || gg.scalar_w)
    return false;
  const int64_t V = static_cast<int64_t>(dd.ptr.size()) - 1;
  struct Ent { int32_t col; double c[2]; };
  struct Acc { int32_t col; Comp v; };
  // full matrix rows with the diagonal split into one piece per slot, so that
  // no product is formed from a pre-summed entry
  auto matrix_row = [](const Stencil& s, int64_t i, std::vector<Ent>& out) {
    out.clear();
    for (int32_t q = s.ptr[i]; q < s.ptr[i + 1]; ++q) {
      const double w0 = s.w[2 * static_cast<int64_t>(q)], w1 = s.w[2 * static_cast<int64_t>(q) + 1];
      out.push_back(Ent{s.nbr[q], {w0, w1}});
      out.push_back(Ent{static_cast<int32_t>(i), {-w0, -w1}});
    }
    if (s.has_b) out.push_back(Ent{static_cast<int32_t>(i), {s.b[2 * i], s.b[2 * i + 1]}});
  };
  auto row = [&](int64_t i, std::vector<Ent>& dr, std::vector<Ent>& gr, std::vector<Acc>& acc) {
    acc.clear();
    matrix_row(dd, i, dr);
    for (const Ent& x : dr) {
      matrix_row(gg, x.col, gr);
      for (const Ent& y : gr) {
        Acc* hit = nullptr;
        for (auto& a : acc)
          if (a.col == y.col) { hit = &a; break; }
        if (!hit) {
          acc.push_back(Acc{y.col, Comp{}});
          hit = &acc.back();
        }
        hit->v.add_prod(x.c[0], y.c[0]);
        hit->v.add_prod(x.c[1], y.c[1]);
      }
    }
    std::sort(acc.begin(), acc.end(), [](const Acc& p, const Acc& q) { return p.col < q.col; });
  };
  std::vector<int32_t> len(static_cast<size_t>(V));
#pragma omp parallel
  {
    std::vector<Ent> dr, gr;
    std::vector<Acc> acc;
#pragma omp for schedule(dynamic, 256)
    for (int64_t i = 0; i < V; ++i) {
      row(i, dr, gr, acc);
      len[i] = static_cast<int32_t>(acc.size()) - 1;  // minus the diagonal
    }
  }
  l.nin = l.nout = 1;
  l.has_b = false;
  l.scalar_w = true;
  l.ptr.assign(static_cast<size_t>(V) + 1, 0);
  for (int64_t i = 0; i < V; ++i) {
    if (static_cast<int64_t>(l.ptr[i]) + len[i] > INT32_MAX) return false;
    l.ptr[i + 1] = l.ptr[i] + len[i];
  }
  l.nbr.resize(static_cast<size_t>(l.ptr[V]));
  l.w.assign(static_cast<size_t>(2 * l.ptr[V]), 0.0);
  l.b.clear();
#pragma omp parallel
  {
    std::vector<Ent> dr, gr;
    std::vector<Acc> acc;
#pragma omp for schedule(dynamic, 256)
    for (int64_t i = 0; i < V; ++i) {
      row(i, dr, gr, acc);
      int32_t q = l.ptr[i];
      for (auto& a : acc) {
        if (a.col == i) continue;
        l.nbr[q] = a.col;
        l.w[2 * static_cast<int64_t>(q)] = a.v.value();
        ++q;
      }
    }
  }
  return true;
}

bool build_regional_stencil(const Mesh& m, const Dual& d, int op, Stencil& s) {
  if (!m.grid->regional() || d.A.empty()) return false;
  switch (op) {
    case OP_GRAD:
    case OP_VGRAD:  // no pole faces: each component's gradient
      one_ring(m, d, OP_GRAD, s);
      return true;
    case OP_DIV:
    case OP_CURL:
      one_ring(m, d, op, s);
      return true;
    case OP_GRAD_ADJ:
    case OP_DIV_ADJ:
    case OP_CURL_ADJ: {
      Stencil a;
      one_ring(m, d, op == OP_GRAD_ADJ ? OP_GRAD : (op == OP_DIV_ADJ ? OP_DIV : OP_CURL), a);
      return transpose_stencil(a, s);
    }
    case OP_LAP: {
      Stencil gs, ds;
      one_ring(m, d, OP_GRAD, gs);
      one_ring(m, d, OP_DIV, ds);
      return compose_stencil(ds, gs, s);
    }
    default:
      return false;
  }
}

}  // namespace atlasgb
