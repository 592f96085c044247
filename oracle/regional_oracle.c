/*
 * TEST INFRASTRUCTURE: FP64 CPU oracle of the nabla operators on regional
 * (limited-area) grids with map projections.  Only tests/ and the smoke
 * check use it; it shares no code with the product library.
 *
 * The paper says Atlas meshes the regional grids of limited-area models and
 * names operators that account for the projection as follow-up work (Sec.
 * 2.2.3, Sec. 5).  The definitions written out here:
 *
 *  Grid.  A rectangle of the projection plane, x_j = xmin + j (xmax-xmin)/(nx-1),
 *   y_r = ymax - r (ymax-ymin)/(ny-1), node r nx + j.  Plane coordinates are
 *   taken on the unit sphere (radians for rotated lon-lat, metres over the
 *   projection radius otherwise).  Inverse projections on the unit sphere:
 *    - rotated lon-lat with rotated south pole (lp, pp): the geographic unit
 *      vector is Rz(lp) Ry(-(pi/2 + pp)) applied to the rotated one (so the
 *      rotated origin lies at (lp, pp + 90 deg) and the rotated north pole at
 *      the antipode of the south pole); scale factors (cos y, 1);
 *    - Mercator: lat = 2 atan(exp y) - pi/2, lon = lon0 + x; scale cos(lat);
 *    - Lambert conformal conic tangent at lat1 (Snyder 1987, Map Projections
 *      - A Working Manual, ch. 15, spherical form with origin latitude lat1):
 *      n = sin lat1, F = cos lat1 tan^n(pi/4 + lat1/2) / n,
 *      rho(lat) = F / tan^n(pi/4 + lat/2), rho0 = rho(lat1); inverse
 *      rho = sgn(n) sqrt(x^2 + (rho0 - y)^2), theta = atan2(sgn(n) x, sgn(n)(rho0 - y)),
 *      lat = 2 atan((F/rho)^(1/n)) - pi/2, lon = lon0 + theta/n; the scale
 *      factor k = cos lat1 tan^n(pi/4+lat1/2) / (cos lat tan^n(pi/4+lat/2)),
 *      h = 1/k;
 *    - polar stereographic (Snyder 1987, ch. 21, spherical form, tangent at
 *      the pole): see reg_inverse.
 *  Mesh.  Each quad (r, j) is cut along its diagonal (r, j)-(r+1, j+1).  An
 *   edge lies on the domain boundary when both its ends lie on the same side
 *   of the rectangle.
 *  Dual.  Median dual in the plane: in every triangle (i, j, k) (counter-
 *   clockwise) cell i owns the quadrilateral i, m_ij, c, m_ik (m: edge
 *   midpoints, c: centroid), of area one third of the triangle's.  Its
 *   boundary, traversed counter-clockwise, consists of m_ij -> c -> m_ik and,
 *   where the edge lies on the domain boundary, i -> m_ij or m_ik -> i.  A
 *   segment P -> Q has the outward normal R (Q_y - P_y, -(Q_x - P_x)).
 *  Face values.  (f_i + f_j)/2 on the segments of edge ij's face, (5 f_i + f_j)/6
 *   on a boundary half edge.
 *  Closure.  The outward normals of a closed cell sum to zero, so with
 *   face value f_i + w (f_j - f_i) (w = 1/2 or 1/6) the segment sum
 *   sum n fv equals sum n w (f_j - f_i) exactly in exact arithmetic; the
 *   oracle evaluates this closure-exact form, free of the cancellation
 *   between terms of size |f| sum|n| of the averaged form, which is kept as
 *   orc_reg_gradient_averaged for the check that both agree within the
 *   closure residual.
 *  Operators (h_x, h_y scale factors at node i, A_i = R^2 times the cell's
 *   plane area, sums over the segments of cell i, Dot2 summation):
 *    gradient    g_x = sum n_x fv / (A_i h_x,i),  g_y = sum n_y fv / (A_i h_y,i)
 *    divergence  sum (n_x F1v + n_y F2v) / (A_i h_x,i h_y,i), (F1, F2) = (h_y u, h_x v)
 *    curl        the same with (F1, F2) = (h_y v, -h_x u)
 *    Laplacian   divergence of the FP64 gradient
 *    adjoints    transposed application of the rows of the gradient and
 *                divergence, rows written entry by entry from the sums above
 *    vector gradient: the gradient of each component.
 * Pins: tests/test_oracle_regional.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define RPI 3.14159265358979323846

typedef struct { double s, c; } racc;
static void r_two_sum(double a, double b, double *s, double *e) {
  *s = a + b;
  double z = *s - a;
  *e = (a - (*s - z)) + (b - z);
}
static void r_add(racc *a, double x) {
  double s, e;
  r_two_sum(a->s, x, &s, &e);
  a->s = s;
  a->c += e;
}
static void r_add_prod(racc *a, double x, double y) {
  double p = x * y, e = fma(x, y, -p), s, t;
  r_two_sum(a->s, p, &s, &t);
  a->s = s;
  a->c += t + e;
}
static double r_val(const racc *a) { return a->s + a->c; }

typedef struct {
  int proj, nx, ny;
  double R;
  int64_t V, T;
  double *x, *y, *lon, *lat, *hx, *hy, *A;
  int32_t *tri;              /* [T][3], counter-clockwise */
  int32_t *n2t_ptr, *n2t;    /* triangles of each node */
} orc_reg;

void orc_reg_free(orc_reg *g) {
  if (!g) return;
  free(g->x); free(g->y); free(g->lon); free(g->lat); free(g->hx); free(g->hy); free(g->A);
  free(g->tri); free(g->n2t_ptr); free(g->n2t);
  free(g);
}

/* inverse projection of the unit-sphere plane point (x, y); returns 0 on success */
static int reg_inverse(int proj, const double *p, double x, double y, double *lon, double *lat, double *hx,
                       double *hy) {
  if (proj == 0) {
    double lp = p[4] * RPI / 180.0, pp = p[5] * RPI / 180.0;
    double v0 = cos(y) * cos(x), v1 = cos(y) * sin(x), v2 = sin(y);
    double b = -(0.5 * RPI + pp);
    double w0 = v0 * cos(b) + v2 * sin(b), w1 = v1, w2 = -v0 * sin(b) + v2 * cos(b); /* Ry(b) */
    double u0 = w0 * cos(lp) - w1 * sin(lp), u1 = w0 * sin(lp) + w1 * cos(lp);      /* Rz(lp) */
    *lon = atan2(u1, u0);
    *lat = asin(w2 > 1.0 ? 1.0 : (w2 < -1.0 ? -1.0 : w2));
    *hx = cos(y);
    *hy = 1.0;
    return 0;
  }
  if (proj == 1) {
    *lon = p[5] * RPI / 180.0 + x;
    *lat = 2.0 * atan(exp(y)) - 0.5 * RPI;
    *hx = *hy = cos(*lat);
    return 0;
  }
  if (proj == 3) {
    /* polar stereographic from the opposite pole onto the plane tangent at
     * the pole p[6] = +-90: rho = sqrt(x^2 + y^2), sin|lat| =
     * (4 - rho^2)/(4 + rho^2), cos lat = 4 rho/(4 + rho^2), the meridian lon0
     * along -y from the north pole (+y from the south pole), scale factor
     * h = 4/(4 + rho^2) */
    double north = p[6] > 0 ? 1.0 : -1.0;
    double r2 = x * x + y * y;
    *lat = north * atan2(4.0 - r2, 4.0 * sqrt(r2));
    *lon = p[5] * RPI / 180.0 + atan2(x, -north * y);
    *hx = *hy = 4.0 / (4.0 + r2);
    return 0;
  }
  if (proj == 2) {
    double lat1 = p[6] * RPI / 180.0, n = sin(lat1);
    double t1 = tan(0.25 * RPI + 0.5 * lat1);
    double F = cos(lat1) * pow(t1, n) / n, rho0 = F / pow(t1, n);
    double sg = n > 0 ? 1.0 : -1.0;
    double rho = sg * sqrt(x * x + (rho0 - y) * (rho0 - y));
    double th = atan2(sg * x, sg * (rho0 - y));
    if (rho == 0.0) return -1;
    *lat = 2.0 * atan(pow(F / rho, 1.0 / n)) - 0.5 * RPI;
    *lon = p[5] * RPI / 180.0 + th / n;
    double k = cos(lat1) * pow(t1, n) / (cos(*lat) * pow(tan(0.25 * RPI + 0.5 * *lat), n));
    *hx = *hy = 1.0 / k;
    return 0;
  }
  return -1;
}

static int on_boundary_edge(const orc_reg *g, int32_t a, int32_t b) {
  int ra = a / g->nx, ca = a % g->nx, rb = b / g->nx, cb = b % g->nx;
  if (ra == rb && (ra == 0 || ra == g->ny - 1)) return 1;
  if (ca == cb && (ca == 0 || ca == g->nx - 1)) return 1;
  return 0;
}

orc_reg *orc_reg_build(int proj, int nx, int ny, const double *prm, double R) {
  if (nx < 2 || ny < 2 || proj < 0 || proj > 3 || !(R > 0)) return NULL;
  orc_reg *g = (orc_reg *)calloc(1, sizeof(orc_reg));
  if (!g) return NULL;
  g->proj = proj; g->nx = nx; g->ny = ny; g->R = R;
  g->V = (int64_t)nx * ny;
  g->T = 2 * (int64_t)(nx - 1) * (ny - 1);
  size_t V = (size_t)g->V;
  g->x = malloc(V * sizeof(double)); g->y = malloc(V * sizeof(double));
  g->lon = malloc(V * sizeof(double)); g->lat = malloc(V * sizeof(double));
  g->hx = malloc(V * sizeof(double)); g->hy = malloc(V * sizeof(double));
  g->A = calloc(V, sizeof(double));
  g->tri = malloc((size_t)g->T * 3 * sizeof(int32_t));
  g->n2t_ptr = calloc(V + 1, sizeof(int32_t));
  g->n2t = malloc((size_t)g->T * 3 * sizeof(int32_t));
  if (!g->x || !g->y || !g->lon || !g->lat || !g->hx || !g->hy || !g->A || !g->tri || !g->n2t_ptr || !g->n2t) {
    orc_reg_free(g);
    return NULL;
  }
  double scale = proj == 0 ? 180.0 / RPI : prm[4];
  double dx = (prm[1] - prm[0]) / (nx - 1), dy = (prm[3] - prm[2]) / (ny - 1);
  for (int r = 0; r < ny; ++r)
    for (int j = 0; j < nx; ++j) {
      int64_t i = (int64_t)r * nx + j;
      g->x[i] = (prm[0] + j * dx) / scale;
      g->y[i] = (prm[3] - r * dy) / scale;
      if (reg_inverse(proj, prm, g->x[i], g->y[i], &g->lon[i], &g->lat[i], &g->hx[i], &g->hy[i])) {
        orc_reg_free(g);
        return NULL;
      }
    }
  int64_t t = 0;
  for (int r = 0; r + 1 < ny; ++r)
    for (int j = 0; j + 1 < nx; ++j) {
      int32_t a = r * nx + j;
      int32_t q[2][3] = {{a, a + 1, a + nx + 1}, {a, a + nx + 1, a + nx}};
      for (int s = 0; s < 2; ++s, ++t) {
        int32_t *v = &g->tri[3 * t];
        v[0] = q[s][0]; v[1] = q[s][1]; v[2] = q[s][2];
        double ar = (g->x[v[1]] - g->x[v[0]]) * (g->y[v[2]] - g->y[v[0]]) -
                    (g->x[v[2]] - g->x[v[0]]) * (g->y[v[1]] - g->y[v[0]]);
        if (ar < 0) { int32_t z = v[1]; v[1] = v[2]; v[2] = z; ar = -ar; }
        for (int k = 0; k < 3; ++k) g->A[v[k]] += R * R * (0.5 * ar) / 3.0;
        for (int k = 0; k < 3; ++k) g->n2t_ptr[v[k] + 1]++;
      }
    }
  for (size_t i = 0; i < V; ++i) g->n2t_ptr[i + 1] += g->n2t_ptr[i];
  int32_t *fill = malloc(V * sizeof(int32_t));
  if (!fill) { orc_reg_free(g); return NULL; }
  memcpy(fill, g->n2t_ptr, V * sizeof(int32_t));
  for (int64_t s = 0; s < g->T; ++s)
    for (int k = 0; k < 3; ++k) g->n2t[fill[g->tri[3 * s + k]]++] = (int32_t)s;
  free(fill);
  return g;
}

void orc_reg_counts(const orc_reg *g, int64_t *out) { out[0] = g->V; out[1] = g->T; }

void orc_reg_get(const orc_reg *g, double *lonlat, double *xy, double *h, double *A, int32_t *tri) {
  for (int64_t i = 0; i < g->V; ++i) {
    if (lonlat) { lonlat[2 * i] = g->lon[i]; lonlat[2 * i + 1] = g->lat[i]; }
    if (xy) { xy[2 * i] = g->x[i]; xy[2 * i + 1] = g->y[i]; }
    if (h) { h[2 * i] = g->hx[i]; h[2 * i + 1] = g->hy[i]; }
    if (A) A[i] = g->A[i];
  }
  if (tri) memcpy(tri, g->tri, (size_t)g->T * 3 * sizeof(int32_t));
}

/* ------------------------------------------------------------------------ */
/* Boundary segments of cell i: outward normal (times R) and the face value */
/* wa f_a + wb f_b.                                                          */
/* ------------------------------------------------------------------------ */
typedef struct { double nx, ny; int32_t a, b; double wa, wb; } rseg;

static int cell_segments(const orc_reg *g, int64_t i, rseg *out) {
  int ns = 0;
  double R = g->R;
  for (int32_t p = g->n2t_ptr[i]; p < g->n2t_ptr[i + 1]; ++p) {
    const int32_t *v = &g->tri[3 * g->n2t[p]];
    int s = v[0] == i ? 0 : (v[1] == i ? 1 : 2);
    int32_t j = v[(s + 1) % 3], k = v[(s + 2) % 3];
    double xi = g->x[i], yi = g->y[i];
    double cx = (g->x[v[0]] + g->x[v[1]] + g->x[v[2]]) / 3.0, cy = (g->y[v[0]] + g->y[v[1]] + g->y[v[2]]) / 3.0;
    double mjx = 0.5 * (xi + g->x[j]), mjy = 0.5 * (yi + g->y[j]);
    double mkx = 0.5 * (xi + g->x[k]), mky = 0.5 * (yi + g->y[k]);
    rseg s1 = {R * (cy - mjy), -R * (cx - mjx), (int32_t)i, j, 0.5, 0.5};
    rseg s2 = {R * (mky - cy), -R * (mkx - cx), (int32_t)i, k, 0.5, 0.5};
    out[ns++] = s1;
    out[ns++] = s2;
    if (on_boundary_edge(g, (int32_t)i, j)) {
      rseg sb = {R * (mjy - yi), -R * (mjx - xi), (int32_t)i, j, 5.0 / 6.0, 1.0 / 6.0};
      out[ns++] = sb;
    }
    if (on_boundary_edge(g, (int32_t)i, k)) {
      rseg sb = {R * (yi - mky), -R * (xi - mkx), (int32_t)i, k, 5.0 / 6.0, 1.0 / 6.0};
      out[ns++] = sb;
    }
  }
  return ns;
}

static double rfld(const void *x, int f32, int64_t ld, int64_t i, int l) {
  return f32 ? (double)((const float *)x)[i * ld + l] : ((const double *)x)[i * ld + l];
}

static int rcheck(const orc_reg *g, const int64_t *nodes, int64_t count) {
  if (!nodes) return 0;
  for (int64_t q = 0; q < count; ++q)
    if (nodes[q] < 0 || nodes[q] >= g->V) return -1;
  return 0;
}

/* gradient of node i, all levels, into gx[nlev], gy[nlev] */
static void reg_grad_node(const orc_reg *g, const void *f, int f32, int64_t ld, int nlev, int64_t i, double *gx,
                          double *gy) {
  rseg seg[32];
  int ns = cell_segments(g, i, seg);
  for (int l = 0; l < nlev; ++l) {
    racc ax = {0, 0}, ay = {0, 0};
    double fi = rfld(f, f32, ld, i, l);
    for (int s = 0; s < ns; ++s) {
      double d = seg[s].wb * (rfld(f, f32, ld, seg[s].b, l) - fi);
      r_add_prod(&ax, seg[s].nx, d);
      r_add_prod(&ay, seg[s].ny, d);
    }
    gx[l] = r_val(&ax) / (g->A[i] * g->hx[i]);
    gy[l] = r_val(&ay) / (g->A[i] * g->hy[i]);
  }
}

/* the averaged form sum n (wa f_i + wb f_j), for the closure check */
int orc_reg_gradient_averaged(const orc_reg *g, const void *f, int f32, int64_t ld, int nlev, double *gx,
                              double *gy) {
  if (!g || !f || nlev < 0 || ld < nlev) return -1;
  rseg seg[32];
  for (int64_t i = 0; i < g->V; ++i) {
    int ns = cell_segments(g, i, seg);
    for (int l = 0; l < nlev; ++l) {
      racc ax = {0, 0}, ay = {0, 0};
      for (int s = 0; s < ns; ++s) {
        double fa = seg[s].wa * rfld(f, f32, ld, seg[s].a, l), fb = seg[s].wb * rfld(f, f32, ld, seg[s].b, l);
        r_add_prod(&ax, seg[s].nx, fa); r_add_prod(&ax, seg[s].nx, fb);
        r_add_prod(&ay, seg[s].ny, fa); r_add_prod(&ay, seg[s].ny, fb);
      }
      gx[i * nlev + l] = r_val(&ax) / (g->A[i] * g->hx[i]);
      gy[i * nlev + l] = r_val(&ay) / (g->A[i] * g->hy[i]);
    }
  }
  return 0;
}

/* h_j x_j - h_i x_i to within a few ulps */
static double rdiff(double hj, double xj, double hi, double xi) {
  double pj = hj * xj, ej = fma(hj, xj, -pj), pi = hi * xi, ei = fma(hi, xi, -pi), s, t;
  r_two_sum(pj, -pi, &s, &t);
  return s + (t + (ej - ei));
}

/* flux form, closure-exact: sum n w . (F_j - F_i) / (A h_x h_y) with
 * F1 = s1 h_y p, F2 = s2 h_x q */
static double reg_flux_node(const orc_reg *g, const rseg *seg, int ns, int64_t i, const void *p, const void *q,
                            int f32, int64_t ld, int l, double s1, double s2) {
  racc a = {0, 0};
  double pi = rfld(p, f32, ld, i, l), qi = rfld(q, f32, ld, i, l);
  for (int s = 0; s < ns; ++s) {
    int32_t cb = seg[s].b;
    double d1 = s1 * rdiff(g->hy[cb], rfld(p, f32, ld, cb, l), g->hy[i], pi);
    double d2 = s2 * rdiff(g->hx[cb], rfld(q, f32, ld, cb, l), g->hx[i], qi);
    r_add_prod(&a, seg[s].nx, seg[s].wb * d1);
    r_add_prod(&a, seg[s].ny, seg[s].wb * d2);
  }
  return r_val(&a) / (g->A[i] * g->hx[i] * g->hy[i]);
}

int orc_reg_gradient(const orc_reg *g, const void *f, int f32, int64_t ld, int nlev, const int64_t *nodes,
                     int64_t count, double *gx, double *gy) {
  if (!g || !f || nlev < 0 || ld < nlev || rcheck(g, nodes, count)) return -1;
  int64_t n = nodes ? count : g->V;
  for (int64_t q = 0; q < n; ++q) reg_grad_node(g, f, f32, ld, nlev, nodes ? nodes[q] : q, gx + q * nlev, gy + q * nlev);
  return 0;
}

int orc_reg_divergence(const orc_reg *g, const void *u, const void *v, int f32, int64_t ld, int nlev,
                       const int64_t *nodes, int64_t count, double *out) {
  if (!g || !u || !v || nlev < 0 || ld < nlev || rcheck(g, nodes, count)) return -1;
  int64_t n = nodes ? count : g->V;
  rseg seg[32];
  for (int64_t q = 0; q < n; ++q) {
    int64_t i = nodes ? nodes[q] : q;
    int ns = cell_segments(g, i, seg);
    for (int l = 0; l < nlev; ++l) out[q * nlev + l] = reg_flux_node(g, seg, ns, i, u, v, f32, ld, l, 1.0, 1.0);
  }
  return 0;
}

int orc_reg_curl(const orc_reg *g, const void *u, const void *v, int f32, int64_t ld, int nlev,
                 const int64_t *nodes, int64_t count, double *out) {
  if (!g || !u || !v || nlev < 0 || ld < nlev || rcheck(g, nodes, count)) return -1;
  int64_t n = nodes ? count : g->V;
  rseg seg[32];
  for (int64_t q = 0; q < n; ++q) {
    int64_t i = nodes ? nodes[q] : q;
    int ns = cell_segments(g, i, seg);
    /* (F1, F2) = (h_y v, -h_x u) */
    for (int l = 0; l < nlev; ++l) out[q * nlev + l] = reg_flux_node(g, seg, ns, i, v, u, f32, ld, l, 1.0, -1.0);
  }
  return 0;
}

/* Laplacian = divergence of the FP64 gradient, which is evaluated at every
 * node the cell's segments reference */
int orc_reg_laplacian(const orc_reg *g, const void *f, int f32, int64_t ld, int nlev, const int64_t *nodes,
                      int64_t count, double *out) {
  if (!g || !f || nlev < 0 || ld < nlev || rcheck(g, nodes, count)) return -1;
  int64_t n = nodes ? count : g->V;
  int nl = nlev > 0 ? nlev : 1;
  double *gx = malloc(sizeof(double) * 32 * nl), *gy = malloc(sizeof(double) * 32 * nl);
  if (!gx || !gy) { free(gx); free(gy); return -2; }
  rseg seg[32];
  int32_t cols[32];
  for (int64_t q = 0; q < n; ++q) {
    int64_t i = nodes ? nodes[q] : q;
    int ns = cell_segments(g, i, seg), nc = 0;
    for (int s = 0; s < ns; ++s)
      for (int e = 0; e < 2; ++e) {
        int32_t c = e ? seg[s].b : seg[s].a;
        int seen = 0;
        for (int t = 0; t < nc; ++t) seen |= cols[t] == c;
        if (!seen) { reg_grad_node(g, f, f32, ld, nlev, c, gx + nc * nl, gy + nc * nl); cols[nc++] = c; }
      }
    for (int l = 0; l < nlev; ++l) {
      racc a = {0, 0};
      for (int s = 0; s < ns; ++s) {
        int ta = 0, tb = 0;
        while (cols[ta] != seg[s].a) ++ta;
        while (cols[tb] != seg[s].b) ++tb;
        double d1 = rdiff(g->hy[seg[s].b], gx[tb * nl + l], g->hy[i], gx[ta * nl + l]);
        double d2 = rdiff(g->hx[seg[s].b], gy[tb * nl + l], g->hx[i], gy[ta * nl + l]);
        r_add_prod(&a, seg[s].nx, seg[s].wb * d1);
        r_add_prod(&a, seg[s].ny, seg[s].wb * d2);
      }
      out[q * nlev + l] = r_val(&a) / (g->A[i] * g->hx[i] * g->hy[i]);
    }
  }
  free(gx); free(gy);
  return 0;
}

/* nodes of the cells whose rows can reference column k: k and its mesh neighbours */
static int ring_of(const orc_reg *g, int64_t k, int32_t *ring) {
  int nr = 0;
  ring[nr++] = (int32_t)k;
  for (int32_t p = g->n2t_ptr[k]; p < g->n2t_ptr[k + 1]; ++p)
    for (int e = 0; e < 3; ++e) {
      int32_t c = g->tri[3 * g->n2t[p] + e], seen = 0;
      for (int t = 0; t < nr; ++t) seen |= ring[t] == c;
      if (!seen) ring[nr++] = c;
    }
  return nr;
}

/* x = G^T (y0, y1): x_k = sum_i G_x(i, k) y0_i + G_y(i, k) y1_i, the row
 * entries being those of the closure-exact form: n w_b / (A_i h_i) on the
 * segment's far node and its negative on node i */
int orc_reg_gradient_adjoint(const orc_reg *g, const void *y0, const void *y1, int f32, int64_t ld, int nlev,
                             const int64_t *nodes, int64_t count, double *x) {
  if (!g || !y0 || !y1 || nlev < 0 || ld < nlev || rcheck(g, nodes, count)) return -1;
  int64_t n = nodes ? count : g->V;
  rseg seg[32];
  int32_t ring[32];
  for (int64_t q = 0; q < n; ++q) {
    int64_t k = nodes ? nodes[q] : q;
    int nr = ring_of(g, k, ring);
    for (int l = 0; l < nlev; ++l) {
      racc a = {0, 0};
      for (int t = 0; t < nr; ++t) {
        int64_t i = ring[t];
        int ns = cell_segments(g, i, seg);
        double cx = rfld(y0, f32, ld, i, l) / (g->A[i] * g->hx[i]), cy = rfld(y1, f32, ld, i, l) / (g->A[i] * g->hy[i]);
        for (int s = 0; s < ns; ++s) {
          double w = (seg[s].b == k ? seg[s].wb : 0.0) - (i == k ? seg[s].wb : 0.0);
          if (w == 0.0) continue;
          r_add_prod(&a, seg[s].nx * w, cx);
          r_add_prod(&a, seg[s].ny * w, cy);
        }
      }
      x[q * nlev + l] = r_val(&a);
    }
  }
  return 0;
}

/* (xu, xv) = D^T d: row i of D (closure-exact form) has u-entries
 * n_x w_b h_y,col / (A_i h_x,i h_y,i) on the segment's far node and minus
 * that with h_y,i on node i, and v-entries likewise with n_y and h_x */
int orc_reg_divergence_adjoint(const orc_reg *g, const void *d, int f32, int64_t ld, int nlev,
                               const int64_t *nodes, int64_t count, double *xu, double *xv) {
  if (!g || !d || nlev < 0 || ld < nlev || rcheck(g, nodes, count)) return -1;
  int64_t n = nodes ? count : g->V;
  rseg seg[32];
  int32_t ring[32];
  for (int64_t q = 0; q < n; ++q) {
    int64_t k = nodes ? nodes[q] : q;
    int nr = ring_of(g, k, ring);
    for (int l = 0; l < nlev; ++l) {
      racc au = {0, 0}, av = {0, 0};
      for (int t = 0; t < nr; ++t) {
        int64_t i = ring[t];
        int ns = cell_segments(g, i, seg);
        double c = rfld(d, f32, ld, i, l) / (g->A[i] * g->hx[i] * g->hy[i]);
        for (int s = 0; s < ns; ++s) {
          double w = (seg[s].b == k ? seg[s].wb : 0.0) - (i == k ? seg[s].wb : 0.0);
          if (w == 0.0) continue;
          r_add_prod(&au, seg[s].nx * w * g->hy[k], c);
          r_add_prod(&av, seg[s].ny * w * g->hx[k], c);
        }
      }
      xu[q * nlev + l] = r_val(&au);
      xv[q * nlev + l] = r_val(&av);
    }
  }
  return 0;
}

/* closure residual of every cell: the sum of its outward segment normals
 * (two components) and the sum of their absolute values */
void orc_reg_closure(const orc_reg *g, double *res, double *absum) {
  rseg seg[32];
  for (int64_t i = 0; i < g->V; ++i) {
    int ns = cell_segments(g, i, seg);
    racc a0 = {0, 0}, a1 = {0, 0};
    double s = 0;
    for (int k = 0; k < ns; ++k) {
      r_add(&a0, seg[k].nx);
      r_add(&a1, seg[k].ny);
      s += fabs(seg[k].nx) + fabs(seg[k].ny);
    }
    res[2 * i] = r_val(&a0);
    res[2 * i + 1] = r_val(&a1);
    absum[i] = s;
  }
}
