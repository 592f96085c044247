/*
 * atlas_oracle.c -- plain, slow FP64 CPU oracle for the median-dual
 * finite-volume nabla operators on the octahedral reduced Gaussian grid.
 *
 * TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the CPU
 * legs of the benchmark (its CPU baseline and its oracle arm) load this
 * library. The product library
 * (paper_1908_07038_gb300) never links, loads or calls it, and this file
 * includes nothing from the product.
 *
 * What the paper fixes: Atlas supplies gradient, divergence, curl and
 * Laplacian operators on a Mesh built from a Grid, applied to Fields through
 * a FunctionSpace (paper Sec. 2.3, Fig. 1 and Fig. 2).  The paper prints no
 * formula for them, so every function below states the reading it implements
 * (Green's theorem on the median dual in the (lon, lat) plane with the
 * spherical metric).  All pins live in tests/test_oracle_*.py.
 *
 * Conventions
 *   rows r = 0..2N-1 north->south; row r holds n_r = 4i+16 points, i = r+1
 *   (r < N) or 2N-r (r >= N); longitude of point j is j/n_r turns; node id =
 *   off[r] + j.  Fields are field[node][level] with a leading dimension ld.
 *   Radius R in metres; gradients in 1/m.
 *
 * Canonical evaluation (the host geometry of the product follows the same
 * per-quantity definitions, written separately; both are pinned here):
 *   lat_r          : Newton on the colatitude form of P_2N (see gauss_colat)
 *   centroid lat   : ((phi_p + phi_p) + phi_q) / 3, p = row holding two vertices
 *   midpoint lat   : phi_r (ring edge) or 0.5*(phi_r + phi_s) (cross edge)
 *   side offset    : RN(rational longitude of the face end point minus the
 *                    edge midpoint, in turns); 0 for the pole point
 *   S_e            : ( R*(phi_L - phi_R), -(C*(off_L - off_R)) ), C = 2*pi*R
 *   segment p->q   : I = -((2*pi*dturns) * sin(0.5*(phi_p+phi_q))) * sinc(0.5*(phi_q-phi_p))
 *   V_i            : (R*R) * (compensated sum of the signed segment integrals)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
static const double TWO_PI = 2.0 * M_PI;
static const double HALF_PI = 0.5 * M_PI;

/* ------------------------------------------------------------------------ */
/* Error-free transformations and compensated accumulation                   */
/* (Ogita, Rump, Oishi 2005: TwoSum, TwoProduct via fma, Dot2).              */
/* ------------------------------------------------------------------------ */
static void two_sum(double a, double b, double *s, double *e) {
  double x = a + b;
  double z = x - a;
  *e = (a - (x - z)) + (b - z);
  *s = x;
}
static void two_prod(double a, double b, double *p, double *e) {
  double x = a * b;
  *e = fma(a, b, -x);
  *p = x;
}
typedef struct { double s, c; } acc_t;
static void acc_add(acc_t *a, double x) {
  double s, e;
  two_sum(a->s, x, &s, &e);
  a->s = s;
  a->c += e;
}
static void acc_add_prod(acc_t *a, double x, double y) {
  double p, e;
  two_prod(x, y, &p, &e);
  acc_add(a, p);
  a->c += e;
}
static double acc_val(const acc_t *a) { return a->s + a->c; }

static double sinc(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

static int64_t gcd64(int64_t a, int64_t b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b) { int64_t t = a % b; a = b; b = t; }
  return a;
}
/* Round-to-nearest double of the rational p/q (q > 0, |p|,q < 2^53 after
 * reduction; IEEE division of two exact doubles is correctly rounded). */
static double rat(int64_t p, int64_t q) {
  int64_t g = gcd64(p, q);
  if (g > 1) { p /= g; q /= g; }
  return (double)p / (double)q;
}

/* ------------------------------------------------------------------------ */
/* a1. Gaussian latitudes.                                                   */
/* The 2N Gaussian latitudes are the roots of the Legendre polynomial P_2N.  */
/* With x = cos(theta) (theta = colatitude), P_n has the finite cosine       */
/* series P_n(cos t) = sum_{k=0..n} g_k g_{n-k} cos((n-2k) t), where          */
/* g_k = binom(2k,k)/4^k.  Newton in theta on this series keeps full          */
/* relative accuracy near the poles, where x-based iteration loses it.       */
/* ------------------------------------------------------------------------ */
static void legendre_theta(int n, const double *c, double t, double *P, double *dP) {
  /* c[k] = g_k g_{n-k} for k = 0..n/2; terms k and n-k are paired. */
  acc_t p = {0, 0}, d = {0, 0};
  for (int k = 0; 2 * k < n; ++k) {
    double m = (double)(n - 2 * k);
    double a, e;
    two_prod(m, t, &a, &e); /* m*t = a + e exactly */
    double ca = cos(a), sa = sin(a);
    double cm = ca - e * sa; /* cos(a+e) to first order in e (|e| <= ulp(a)/2) */
    double sm = sa + e * ca;
    acc_add_prod(&p, 2.0 * c[k], cm);
    acc_add_prod(&d, -2.0 * c[k] * m, sm);
  }
  if (n % 2 == 0) acc_add(&p, c[n / 2]);
  *P = acc_val(&p);
  *dP = acc_val(&d);
}

/* Colatitudes theta_k (k = 0..n-1, ascending from the north pole) of the roots
 * of P_n.  The northern half is iterated; the southern half is its mirror
 * image pi - theta, which is exact for the roots of an even/odd polynomial. */
int orc_gauss_colatitudes(int n, double *theta) {
  if (n < 1) return -1;
  double *g = (double *)malloc(sizeof(double) * (size_t)(n + 1));
  double *c = (double *)malloc(sizeof(double) * (size_t)(n / 2 + 1));
  if (!g || !c) { free(g); free(c); return -2; }
  g[0] = 1.0;
  for (int k = 1; k <= n; ++k) g[k] = g[k - 1] * (double)(2 * k - 1) / (double)(2 * k);
  for (int k = 0; 2 * k <= n; ++k) c[k] = g[k] * g[n - k];
  int half = (n + 1) / 2;
  for (int k = 0; k < half; ++k) {
    /* classical initial guess: x_k ~ cos(pi (k + 3/4) / (n + 1/2)) */
    double t = M_PI * ((double)k + 0.75) / ((double)n + 0.5);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre_theta(n, c, t, &P, &dP);
      double dt = P / dP;
      t -= dt;
      if (fabs(dt) <= 1e-15 * (t > 1.0 ? t : 1.0)) {
        legendre_theta(n, c, t, &P, &dP); /* one more step after convergence */
        t -= P / dP;
        break;
      }
    }
    theta[k] = t;
  }
  for (int k = 0; k < n / 2; ++k) theta[n - 1 - k] = M_PI - theta[k];
  if (n % 2 == 1) theta[n / 2] = HALF_PI;
  free(g);
  free(c);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Mesh data structure of the oracle.                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
  int N, nlat;
  int64_t nnodes, ntri, nedges;
  double R;
  int32_t *pl;      /* [nlat] */
  int64_t *off;     /* [nlat+1] */
  double *lat;      /* [nlat] radians */
  double *colat;    /* [nlat] */
  int32_t *node_row, *node_j; /* [nnodes] */
  /* triangles */
  int32_t *tri;     /* [ntri][3] node ids */
  int32_t *tri_r;   /* [ntri][3] row of each vertex */
  int32_t *tri_j;   /* [ntri][3] unwrapped longitude index */
  /* edges, sorted by (a,b), a<b */
  int32_t *e2n;     /* [E][2] */
  uint8_t *is_pole; /* [E] */
  int32_t *n2e_ptr; /* [V+1] */
  int32_t *n2e;     /* [2E] ascending edge id */
  int8_t *n2e_sign; /* [2E] +1 at a, -1 at b */
  /* dual */
  double *S;        /* [E][2] (S_lambda, S_phi), oriented from a to b */
  double *V;        /* [V] */
  double *coslat;   /* [V] */
  double *pole_nphi;/* [V] phi-component of the pole face normal (0 if none) */
  /* per-edge side data used while building the dual */
  double *side_off; /* [E][2] (L,R) offset in turns from the edge midpoint */
  double *side_phi; /* [E][2] latitude of the side end point */
  double *mid_phi;  /* [E] */
  int8_t *side_set; /* [E][2] */
} orc_mesh;

static int row_size(int N, int r) {
  int i = (r < N) ? r + 1 : 2 * N - r;
  return 4 * i + 16;
}

static int64_t node_id(const orc_mesh *m, int r, int j) {
  int n = m->pl[r];
  int jj = j % n;
  if (jj < 0) jj += n;
  return m->off[r] + jj;
}

static int64_t find_edge(const orc_mesh *m, int32_t a, int32_t b) {
  int64_t lo = 0, hi = m->nedges - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) / 2;
    int32_t ea = m->e2n[2 * mid], eb = m->e2n[2 * mid + 1];
    if (ea == a && eb == b) return mid;
    if (ea < a || (ea == a && eb < b)) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

static int cmp_u64(const void *x, const void *y) {
  uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
  return (a > b) - (a < b);
}

void orc_free(orc_mesh *m);

/* a2 + a3 + a4: grid, zipper triangulation with pole edges, CSR, median dual.
 * regular = 0: the octahedral grid O<N> (rows of 4i+16 points); regular = 1:
 * the regular Gaussian grid F<N> (4N points on every row, paper Sec. 4.3,
 * Fig. 4), meshed by the same zipper (every band is then an equal-row band).
 * Returns NULL on invalid N or allocation failure. */
orc_mesh *orc_build_grid(int N, double R, int regular) {
  if (N < 1 || N > 8000 || !(R > 0)) return NULL;
  orc_mesh *m = (orc_mesh *)calloc(1, sizeof(orc_mesh));
  if (!m) return NULL;
  m->N = N;
  m->nlat = 2 * N;
  m->R = R;
  int nlat = m->nlat;
  m->pl = (int32_t *)malloc(sizeof(int32_t) * nlat);
  m->off = (int64_t *)malloc(sizeof(int64_t) * (nlat + 1));
  m->lat = (double *)malloc(sizeof(double) * nlat);
  m->colat = (double *)malloc(sizeof(double) * nlat);
  if (!m->pl || !m->off || !m->lat || !m->colat) { orc_free(m); return NULL; }

  /* a1: latitudes, north to south */
  if (orc_gauss_colatitudes(nlat, m->colat)) { orc_free(m); return NULL; }
  for (int r = 0; r < nlat; ++r) m->lat[r] = HALF_PI - m->colat[r];
  for (int r = 0; r < N; ++r) m->lat[nlat - 1 - r] = -m->lat[r];

  /* a2: octahedral (or regular) rows */
  m->off[0] = 0;
  for (int r = 0; r < nlat; ++r) {
    m->pl[r] = regular ? 4 * N : row_size(N, r);
    m->off[r + 1] = m->off[r] + m->pl[r];
  }
  int64_t V = m->off[nlat];
  m->nnodes = V;
  m->node_row = (int32_t *)malloc(sizeof(int32_t) * V);
  m->node_j = (int32_t *)malloc(sizeof(int32_t) * V);
  m->coslat = (double *)malloc(sizeof(double) * V);
  if (!m->node_row || !m->node_j || !m->coslat) { orc_free(m); return NULL; }
  for (int r = 0; r < nlat; ++r) {
    double c = cos(m->lat[r]);
    for (int j = 0; j < m->pl[r]; ++j) {
      m->node_row[m->off[r] + j] = r;
      m->node_j[m->off[r] + j] = j;
      m->coslat[m->off[r] + j] = c;
    }
  }

  /* a3: zipper triangulation of every band (r, r+1).  Advance on the row
   * whose next longitude is smaller; on a tie advance the row with fewer
   * points, and if both rows are equal (equator band) the northern row. */
  int64_t T = 0;
  for (int r = 0; r + 1 < nlat; ++r) T += m->pl[r] + m->pl[r + 1];
  m->ntri = T;
  m->tri = (int32_t *)malloc(sizeof(int32_t) * 3 * T);
  m->tri_r = (int32_t *)malloc(sizeof(int32_t) * 3 * T);
  m->tri_j = (int32_t *)malloc(sizeof(int32_t) * 3 * T);
  if (!m->tri || !m->tri_r || !m->tri_j) { orc_free(m); return NULL; }
  int64_t t = 0;
  for (int r = 0; r + 1 < nlat; ++r) {
    int s = r + 1;
    int64_t n1 = m->pl[r], n2 = m->pl[s];
    int64_t ia = 0, ib = 0;
    while (ia < n1 || ib < n2) {
      int north;
      if (ia == n1) north = 0;
      else if (ib == n2) north = 1;
      else {
        int64_t ln = (ia + 1) * n2, ls = (ib + 1) * n1; /* compare (ia+1)/n1 with (ib+1)/n2 */
        if (ln < ls) north = 1;
        else if (ln > ls) north = 0;
        else north = (n1 <= n2);
      }
      int32_t *tv = m->tri + 3 * t, *tr = m->tri_r + 3 * t, *tj = m->tri_j + 3 * t;
      if (north) {
        tr[0] = r; tj[0] = (int32_t)ia;
        tr[1] = r; tj[1] = (int32_t)(ia + 1);
        tr[2] = s; tj[2] = (int32_t)ib;
        ++ia;
      } else {
        tr[0] = r; tj[0] = (int32_t)ia;
        tr[1] = s; tj[1] = (int32_t)ib;
        tr[2] = s; tj[2] = (int32_t)(ib + 1);
        ++ib;
      }
      for (int k = 0; k < 3; ++k) tv[k] = (int32_t)node_id(m, tr[k], tj[k]);
      ++t;
    }
  }

  /* Edges: the three sides of every triangle, deduplicated, plus the pole
   * edges (j, j + n/2) of the first and last row. */
  int npole_n = m->pl[0] / 2, npole_s = m->pl[nlat - 1] / 2;
  uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (3 * T + npole_n + npole_s));
  if (!keys) { orc_free(m); return NULL; }
  int64_t nk = 0;
  for (int64_t q = 0; q < T; ++q)
    for (int k = 0; k < 3; ++k) {
      uint32_t a = (uint32_t)m->tri[3 * q + k], b = (uint32_t)m->tri[3 * q + (k + 1) % 3];
      if (a > b) { uint32_t x = a; a = b; b = x; }
      keys[nk++] = ((uint64_t)a << 32) | b;
    }
  qsort(keys, (size_t)nk, sizeof(uint64_t), cmp_u64);
  int64_t nu = 0;
  for (int64_t q = 0; q < nk; ++q)
    if (q == 0 || keys[q] != keys[q - 1]) keys[nu++] = keys[q];
  int64_t nreg = nu;
  for (int j = 0; j < npole_n; ++j)
    keys[nu++] = ((uint64_t)(m->off[0] + j) << 32) | (uint64_t)(m->off[0] + j + npole_n);
  for (int j = 0; j < npole_s; ++j)
    keys[nu++] = ((uint64_t)(m->off[nlat - 1] + j) << 32) | (uint64_t)(m->off[nlat - 1] + j + npole_s);
  qsort(keys, (size_t)nu, sizeof(uint64_t), cmp_u64);
  for (int64_t q = 1; q < nu; ++q)
    if (keys[q] == keys[q - 1]) { free(keys); orc_free(m); return NULL; } /* a pole edge may not repeat a side */
  (void)nreg;
  int64_t E = nu;
  m->nedges = E;
  m->e2n = (int32_t *)malloc(sizeof(int32_t) * 2 * E);
  m->is_pole = (uint8_t *)calloc((size_t)E, 1);
  if (!m->e2n || !m->is_pole) { free(keys); orc_free(m); return NULL; }
  for (int64_t e = 0; e < E; ++e) {
    m->e2n[2 * e] = (int32_t)(keys[e] >> 32);
    m->e2n[2 * e + 1] = (int32_t)(keys[e] & 0xffffffffu);
  }
  free(keys);
  for (int j = 0; j < npole_n; ++j) {
    int64_t e = find_edge(m, (int32_t)(m->off[0] + j), (int32_t)(m->off[0] + j + npole_n));
    m->is_pole[e] = 1;
  }
  for (int j = 0; j < npole_s; ++j) {
    int64_t e = find_edge(m, (int32_t)(m->off[nlat - 1] + j), (int32_t)(m->off[nlat - 1] + j + npole_s));
    m->is_pole[e] = 1;
  }

  /* CSR node -> edges in ascending edge id (edges are visited in order). */
  m->n2e_ptr = (int32_t *)calloc((size_t)(V + 1), sizeof(int32_t));
  m->n2e = (int32_t *)malloc(sizeof(int32_t) * 2 * E);
  m->n2e_sign = (int8_t *)malloc((size_t)(2 * E));
  if (!m->n2e_ptr || !m->n2e || !m->n2e_sign) { orc_free(m); return NULL; }
  for (int64_t e = 0; e < E; ++e) {
    m->n2e_ptr[m->e2n[2 * e] + 1]++;
    m->n2e_ptr[m->e2n[2 * e + 1] + 1]++;
  }
  for (int64_t i = 0; i < V; ++i) m->n2e_ptr[i + 1] += m->n2e_ptr[i];
  int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * V);
  if (!fill) { orc_free(m); return NULL; }
  for (int64_t i = 0; i < V; ++i) fill[i] = m->n2e_ptr[i];
  for (int64_t e = 0; e < E; ++e) {
    int32_t a = m->e2n[2 * e], b = m->e2n[2 * e + 1];
    m->n2e[fill[a]] = (int32_t)e; m->n2e_sign[fill[a]] = 1; fill[a]++;
    m->n2e[fill[b]] = (int32_t)e; m->n2e_sign[fill[b]] = -1; fill[b]++;
  }
  free(fill);

  /* a4: median dual.  For every triangle and each of its sides, the dual face
   * piece inside the triangle runs from the side midpoint to the triangle
   * centroid.  The centroid is stored on the left (L) or right (R) of the
   * side's orientation a->b, as an offset from the midpoint in the
   * triangle's own unwrapped longitude frame, so that the stored data do not
   * depend on where the frame wraps. */
  m->side_off = (double *)calloc((size_t)(2 * E), sizeof(double));
  m->side_phi = (double *)calloc((size_t)(2 * E), sizeof(double));
  m->mid_phi = (double *)calloc((size_t)E, sizeof(double));
  m->side_set = (int8_t *)calloc((size_t)(2 * E), 1);
  m->S = (double *)calloc((size_t)(2 * E), sizeof(double));
  m->V = (double *)calloc((size_t)V, sizeof(double));
  m->pole_nphi = (double *)calloc((size_t)V, sizeof(double));
  if (!m->side_off || !m->side_phi || !m->mid_phi || !m->side_set || !m->S || !m->V || !m->pole_nphi) {
    orc_free(m); return NULL;
  }
  for (int64_t q = 0; q < T; ++q) {
    const int32_t *tv = m->tri + 3 * q, *tr = m->tri_r + 3 * q, *tj = m->tri_j + 3 * q;
    int r = tr[0] < tr[2] ? tr[0] : tr[2];
    int s = r + 1;
    int64_t nr = m->pl[r], ns = m->pl[s];
    int64_t D = 6 * nr * ns; /* common denominator of every longitude in the band */
    int64_t xD[3];           /* longitude * D of each vertex (turns) */
    for (int k = 0; k < 3; ++k) xD[k] = (tr[k] == r) ? (int64_t)tj[k] * 6 * ns : (int64_t)tj[k] * 6 * nr;
    int64_t cD = (xD[0] + xD[1] + xD[2]) / 3; /* exact: every xD is a multiple of 6 */
    /* centroid latitude: the row holding two vertices counts twice */
    int nr_cnt = (tr[0] == r) + (tr[1] == r) + (tr[2] == r);
    int p = (nr_cnt == 2) ? r : s, qq = (nr_cnt == 2) ? s : r;
    double cphi = ((m->lat[p] + m->lat[p]) + m->lat[qq]) / 3.0;
    for (int k = 0; k < 3; ++k) {
      int k2 = (k + 1) % 3;
      int ia = k, ib = k2;
      if (tv[ia] > tv[ib]) { ia = k2; ib = k; }
      int64_t e = find_edge(m, tv[ia], tv[ib]);
      if (e < 0) { orc_free(m); return NULL; }
      int64_t mD2 = xD[ia] + xD[ib]; /* 2 * midpoint * D */
      double phia = m->lat[tr[ia]], phib = m->lat[tr[ib]];
      double mphi = (tr[ia] == tr[ib]) ? phia : 0.5 * (m->lat[r] + m->lat[s]);
      /* left/right of a->b in the (lon, lat) plane */
      double la = (double)xD[ia] / (double)D, lb = (double)xD[ib] / (double)D, lc = (double)cD / (double)D;
      double cross = (lb - la) * (cphi - phia) - (phib - phia) * (lc - la);
      int side = (cross > 0) ? 0 : 1; /* 0 = L, 1 = R */
      if (m->side_set[2 * e + side]) { orc_free(m); return NULL; }
      m->side_set[2 * e + side] = 1;
      m->side_off[2 * e + side] = rat(2 * cD - mD2, 2 * D);
      m->side_phi[2 * e + side] = cphi;
      m->mid_phi[e] = mphi;
      /* A side with both ends on the first or last row has no triangle on its
       * pole side: the face continues from the midpoint straight to the pole
       * at the midpoint's longitude. */
      if (tr[ia] == tr[ib] && (tr[ia] == 0 || tr[ia] == nlat - 1)) {
        double pphi = (tr[ia] == 0) ? HALF_PI : -HALF_PI;
        double pcross = (lb - la) * (pphi - phia);
        int pside = (pcross > 0) ? 0 : 1;
        if (pside == side || m->side_set[2 * e + pside]) { orc_free(m); return NULL; }
        m->side_set[2 * e + pside] = 1;
        m->side_off[2 * e + pside] = 0.0;
        m->side_phi[2 * e + pside] = pphi;
      }
    }
  }
  const double C = TWO_PI * R;
  acc_t *vacc = (acc_t *)calloc((size_t)V, sizeof(acc_t));
  if (!vacc) { orc_free(m); return NULL; }
  for (int64_t e = 0; e < E; ++e) {
    int32_t a = m->e2n[2 * e], b = m->e2n[2 * e + 1];
    if (m->is_pole[e]) {
      int north = (m->node_row[a] == 0);
      double sphi = C * rat(1, m->pl[m->node_row[a]]);
      m->S[2 * e] = 0.0;
      m->S[2 * e + 1] = north ? sphi : -sphi;
      continue;
    }
    if (!m->side_set[2 * e] || !m->side_set[2 * e + 1]) { free(vacc); orc_free(m); return NULL; }
    double offL = m->side_off[2 * e], offR = m->side_off[2 * e + 1];
    double phiL = m->side_phi[2 * e], phiR = m->side_phi[2 * e + 1], phim = m->mid_phi[e];
    m->S[2 * e] = R * (phiL - phiR);
    m->S[2 * e + 1] = -(C * (offL - offR));
    /* segments c_R -> m and m -> c_L; cell a on their left, cell b on their right */
    double d1 = -offR, d2 = offL;
    double I1 = -((TWO_PI * d1) * sin(0.5 * (phiR + phim))) * sinc(0.5 * (phim - phiR));
    double I2 = -((TWO_PI * d2) * sin(0.5 * (phim + phiL))) * sinc(0.5 * (phiL - phim));
    acc_add(&vacc[a], I1); acc_add(&vacc[a], I2);
    acc_add(&vacc[b], -I1); acc_add(&vacc[b], -I2);
  }
  /* the pole segment closes every cell of the first and last row */
  for (int rr = 0; rr < nlat; rr += nlat - 1) {
    double ipole = TWO_PI * rat(1, m->pl[rr]);
    double sphi = C * rat(1, m->pl[rr]);
    for (int j = 0; j < m->pl[rr]; ++j) {
      acc_add(&vacc[m->off[rr] + j], ipole);
      m->pole_nphi[m->off[rr] + j] = (rr == 0) ? sphi : -sphi;
    }
  }
  const double R2 = R * R;
  for (int64_t i = 0; i < V; ++i) m->V[i] = R2 * acc_val(&vacc[i]);
  free(vacc);
  return m;
}

orc_mesh *orc_build(int N, double R) { return orc_build_grid(N, R, 0); }

void orc_free(orc_mesh *m) {
  if (!m) return;
  free(m->pl); free(m->off); free(m->lat); free(m->colat);
  free(m->node_row); free(m->node_j); free(m->coslat);
  free(m->tri); free(m->tri_r); free(m->tri_j);
  free(m->e2n); free(m->is_pole); free(m->n2e_ptr); free(m->n2e); free(m->n2e_sign);
  free(m->S); free(m->V); free(m->pole_nphi);
  free(m->side_off); free(m->side_phi); free(m->mid_phi); free(m->side_set);
  free(m);
}

/* ------------------------------------------------------------------------ */
/* Accessors (copy out into caller buffers).                                 */
/* ------------------------------------------------------------------------ */
void orc_counts(const orc_mesh *m, int64_t *out) {
  out[0] = m->N; out[1] = m->nlat; out[2] = m->nnodes; out[3] = m->ntri; out[4] = m->nedges;
  out[5] = 2 * m->nedges;
}
void orc_get_grid(const orc_mesh *m, int32_t *pl, double *lat, double *colat, double *lonlat) {
  if (pl) memcpy(pl, m->pl, sizeof(int32_t) * m->nlat);
  if (lat) memcpy(lat, m->lat, sizeof(double) * m->nlat);
  if (colat) memcpy(colat, m->colat, sizeof(double) * m->nlat);
  if (lonlat)
    for (int64_t i = 0; i < m->nnodes; ++i) {
      int r = m->node_row[i];
      lonlat[2 * i] = TWO_PI * rat(m->node_j[i], m->pl[r]);
      lonlat[2 * i + 1] = m->lat[r];
    }
}
void orc_get_mesh(const orc_mesh *m, int32_t *tri, int32_t *tri_r, int32_t *tri_j, int32_t *e2n,
                  uint8_t *is_pole, int32_t *n2e_ptr, int32_t *n2e, int8_t *n2e_sign) {
  if (tri) memcpy(tri, m->tri, sizeof(int32_t) * 3 * m->ntri);
  if (tri_r) memcpy(tri_r, m->tri_r, sizeof(int32_t) * 3 * m->ntri);
  if (tri_j) memcpy(tri_j, m->tri_j, sizeof(int32_t) * 3 * m->ntri);
  if (e2n) memcpy(e2n, m->e2n, sizeof(int32_t) * 2 * m->nedges);
  if (is_pole) memcpy(is_pole, m->is_pole, (size_t)m->nedges);
  if (n2e_ptr) memcpy(n2e_ptr, m->n2e_ptr, sizeof(int32_t) * (m->nnodes + 1));
  if (n2e) memcpy(n2e, m->n2e, sizeof(int32_t) * 2 * m->nedges);
  if (n2e_sign) memcpy(n2e_sign, m->n2e_sign, (size_t)(2 * m->nedges));
}
void orc_get_dual(const orc_mesh *m, double *S, double *V, double *coslat, double *pole_nphi) {
  if (S) memcpy(S, m->S, sizeof(double) * 2 * m->nedges);
  if (V) memcpy(V, m->V, sizeof(double) * m->nnodes);
  if (coslat) memcpy(coslat, m->coslat, sizeof(double) * m->nnodes);
  if (pole_nphi) memcpy(pole_nphi, m->pole_nphi, sizeof(double) * m->nnodes);
}

/* ------------------------------------------------------------------------ */
/* Operators.                                                                */
/* Every node i owns the closed dual cell Omega_i with outward face normals  */
/* n_ie: for a regular edge n_ie = s_ie * S_e (s = +1 at a, -1 at b); for a  */
/* pole edge n_ie = S_e at both ends (the pole segment of the cell).  Green's */
/* theorem on the closed cell gives the median-dual gradient                 */
/*   V_i grad f = sum_e n_ie * (f_a + f_b)/2                                  */
/* and, because the faces of a closed cell satisfy sum_e n_ie = 0, the same  */
/* operator is sum_e n_ie (f_j - f_i)/2 with j the far end of e.  The oracle */
/* evaluates that closure-exact form (no cancellation between terms of size  */
/* |f|/h) with Dot2 accumulation; orc_gradient_averaged evaluates the first  */
/* form for the test that the two agree within the closure residual.         */
/* ------------------------------------------------------------------------ */
static double fld(const void *x, int f32, int64_t ld, int64_t i, int k) {
  return f32 ? (double)((const float *)x)[i * ld + k] : ((const double *)x)[i * ld + k];
}
static int32_t far_end(const orc_mesh *m, int64_t e, int64_t i) {
  int32_t a = m->e2n[2 * e], b = m->e2n[2 * e + 1];
  return (a == i) ? b : a;
}
/* outward normal of cell i on the face of edge e (CSR position p) */
static void face_normal(const orc_mesh *m, int64_t p, double *nl, double *np) {
  int64_t e = m->n2e[p];
  double s = m->is_pole[e] ? 1.0 : (double)m->n2e_sign[p];
  *nl = s * m->S[2 * e];
  *np = s * m->S[2 * e + 1];
}

/* gradient at node i, levels 0..nlev-1:
 *   g_lambda = (1/V_i) sum_e n_ie,lambda (f_j - f_i)/2
 *   g_phi    = (cos(phi_i)/V_i) sum_e n_ie,phi (f_j - f_i)/2
 * The lambda component of the metric-weighted flux integral needs no factor;
 * the phi component carries cos(phi_i) because V_i is a cos-weighted area. */
static void grad_node(const orc_mesh *m, const void *f, int f32, int64_t ld, int nlev, int64_t i,
                      double *gx, double *gy) {
  for (int k = 0; k < nlev; ++k) {
    acc_t al = {0, 0}, ap = {0, 0};
    double fi = fld(f, f32, ld, i, k);
    for (int32_t p = m->n2e_ptr[i]; p < m->n2e_ptr[i + 1]; ++p) {
      double nl, np;
      face_normal(m, p, &nl, &np);
      int32_t j = far_end(m, m->n2e[p], i);
      double d = 0.5 * (fld(f, f32, ld, j, k) - fi);
      acc_add_prod(&al, nl, d);
      acc_add_prod(&ap, np, d);
    }
    gx[k] = acc_val(&al) / m->V[i];
    gy[k] = m->coslat[i] * acc_val(&ap) / m->V[i];
  }
}

/* a*c_j - b*c_i evaluated to within a few ulps of the exact value */
static double diff_of_products(double vj, double cj, double vi, double ci) {
  double pj, ej, pi, ei, s, t;
  two_prod(vj, cj, &pj, &ej);
  two_prod(vi, ci, &pi, &ei);
  two_sum(pj, -pi, &s, &t);
  return s + (t + (ej - ei));
}

/* divergence at node i of the vector (u, v) in physical components:
 *   div = (1/(R cos)) [d_lambda u + d_phi (v cos)]
 * discretised as the flux of F = (u, v cos(phi)) through the cell faces,
 *   V_i div_i = sum_{regular e} n_ie . (F_a + F_b)/2,
 * with zero flux through the pole segment (cos = 0 at the pole).  Using
 * closure of the full cell, sum_{regular e} n_ie = -n_pole,i, this is
 *   V_i div_i = sum_{regular e} n_ie . (F_j - F_i)/2 - F_i . n_pole,i.    */
static void div_node(const orc_mesh *m, const void *u, const void *v, int f32, int64_t ld, int nlev,
                     int64_t i, double *out) {
  double ci = m->coslat[i];
  for (int k = 0; k < nlev; ++k) {
    acc_t a = {0, 0};
    double ui = fld(u, f32, ld, i, k), vi = fld(v, f32, ld, i, k);
    for (int32_t p = m->n2e_ptr[i]; p < m->n2e_ptr[i + 1]; ++p) {
      int64_t e = m->n2e[p];
      if (m->is_pole[e]) continue;
      double nl, np;
      face_normal(m, p, &nl, &np);
      int32_t j = far_end(m, e, i);
      double du = 0.5 * (fld(u, f32, ld, j, k) - ui);
      double dv = 0.5 * diff_of_products(fld(v, f32, ld, j, k), m->coslat[j], vi, ci);
      acc_add_prod(&a, nl, du);
      acc_add_prod(&a, np, dv);
    }
    if (m->pole_nphi[i] != 0.0) {
      double pv, ev;
      two_prod(vi, ci, &pv, &ev);
      acc_add_prod(&a, -m->pole_nphi[i], pv);
      acc_add_prod(&a, -m->pole_nphi[i], ev);
    }
    out[k] = acc_val(&a) / m->V[i];
  }
}

static int64_t nsel(const orc_mesh *m, const int64_t *nodes, int64_t count) {
  return nodes ? count : m->nnodes;
}
static int check_nodes(const orc_mesh *m, const int64_t *nodes, int64_t count) {
  if (!nodes) return 0;
  for (int64_t q = 0; q < count; ++q)
    if (nodes[q] < 0 || nodes[q] >= m->nnodes) return -1;
  return 0;
}

/* Outputs are packed [count][nlev]; nodes == NULL selects every node. */
int orc_gradient(const orc_mesh *m, const void *f, int f32, int64_t ld, int nlev,
                 const int64_t *nodes, int64_t count, double *gx, double *gy) {
  if (!m || !f || nlev < 0 || ld < nlev || check_nodes(m, nodes, count)) return -1;
  int64_t n = nsel(m, nodes, count);
  for (int64_t q = 0; q < n; ++q) {
    int64_t i = nodes ? nodes[q] : q;
    grad_node(m, f, f32, ld, nlev, i, gx + q * nlev, gy + q * nlev);
  }
  return 0;
}

int orc_divergence(const orc_mesh *m, const void *u, const void *v, int f32, int64_t ld, int nlev,
                   const int64_t *nodes, int64_t count, double *out) {
  if (!m || !u || !v || nlev < 0 || ld < nlev || check_nodes(m, nodes, count)) return -1;
  int64_t n = nsel(m, nodes, count);
  for (int64_t q = 0; q < n; ++q) {
    int64_t i = nodes ? nodes[q] : q;
    div_node(m, u, v, f32, ld, nlev, i, out + q * nlev);
  }
  return 0;
}

/* Laplacian = divergence of the gradient.  The gradient is evaluated in FP64
 * at the node and its edge neighbours, then the divergence formula is
 * applied to it.  For the selected node i the neighbour gradients are stored
 * in a small local field indexed 0 (= i) .. deg. */
int orc_laplacian(const orc_mesh *m, const void *f, int f32, int64_t ld, int nlev,
                  const int64_t *nodes, int64_t count, double *out) {
  if (!m || !f || nlev < 0 || ld < nlev || check_nodes(m, nodes, count)) return -1;
  int64_t n = nsel(m, nodes, count);
  if (nlev == 0) return 0;
  /* full field: gradient everywhere, then divergence */
  if (!nodes) {
    double *gx = (double *)malloc(sizeof(double) * m->nnodes * nlev);
    double *gy = (double *)malloc(sizeof(double) * m->nnodes * nlev);
    if (!gx || !gy) { free(gx); free(gy); return -2; }
    for (int64_t i = 0; i < m->nnodes; ++i) grad_node(m, f, f32, ld, nlev, i, gx + i * nlev, gy + i * nlev);
    for (int64_t i = 0; i < m->nnodes; ++i) div_node(m, gx, gy, 0, nlev, nlev, i, out + i * nlev);
    free(gx); free(gy);
    return 0;
  }
  /* selected nodes: gradient on the closed 1-ring only */
  double *gx = (double *)malloc(sizeof(double) * 64 * nlev);
  double *gy = (double *)malloc(sizeof(double) * 64 * nlev);
  if (!gx || !gy) { free(gx); free(gy); return -2; }
  for (int64_t q = 0; q < n; ++q) {
    int64_t i = nodes[q];
    int32_t p0 = m->n2e_ptr[i], p1 = m->n2e_ptr[i + 1];
    if (p1 - p0 + 1 > 64) { free(gx); free(gy); return -3; }
    grad_node(m, f, f32, ld, nlev, i, gx, gy);
    for (int32_t p = p0; p < p1; ++p) {
      int32_t j = far_end(m, m->n2e[p], i);
      grad_node(m, f, f32, ld, nlev, j, gx + (1 + p - p0) * nlev, gy + (1 + p - p0) * nlev);
    }
    double ci = m->coslat[i];
    for (int k = 0; k < nlev; ++k) {
      acc_t a = {0, 0};
      double ui = gx[k], vi = gy[k];
      for (int32_t p = p0; p < p1; ++p) {
        int64_t e = m->n2e[p];
        if (m->is_pole[e]) continue;
        double nl, np;
        face_normal(m, p, &nl, &np);
        int32_t j = far_end(m, e, i);
        double uj = gx[(1 + p - p0) * nlev + k], vj = gy[(1 + p - p0) * nlev + k];
        acc_add_prod(&a, nl, 0.5 * (uj - ui));
        acc_add_prod(&a, np, 0.5 * diff_of_products(vj, m->coslat[j], vi, ci));
      }
      if (m->pole_nphi[i] != 0.0) {
        double pv, ev;
        two_prod(vi, ci, &pv, &ev);
        acc_add_prod(&a, -m->pole_nphi[i], pv);
        acc_add_prod(&a, -m->pole_nphi[i], ev);
      }
      out[q * nlev + k] = acc_val(&a) / m->V[i];
    }
  }
  free(gx); free(gy);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Curl and vector gradient (the paper lists nabla operators on fields as   */
/* provided by the library, Sec. 2.3; these two extend the scalar ones to    */
/* tangent vector fields in physical components).                            */
/* ------------------------------------------------------------------------ */

/* vertical vorticity of the tangent vector (u, v) at node i:
 *   zeta = (1/(R cos)) [d_lambda v - d_phi (u cos)].
 * Stokes' theorem on the dual cell: V_i zeta_i is the circulation of (u, v)
 * around the cell boundary, the integral of u R cos dlambda + v R dphi.  On
 * a face whose outward normal is n = R (dphi, -dlambda), that line element
 * is v n_lambda - (u cos) n_phi, so the circulation is the flux of
 * G = (v, -u cos) through the faces, with the face mean of G; the pole
 * segments carry none (dphi = 0 and cos = 0 there).  Closure-exact form, as
 * for the divergence: sum_{regular e} n . (G_j - G_i)/2 - G_i . n_pole,i. */
static void curl_node(const orc_mesh *m, const void *u, const void *v, int f32, int64_t ld, int nlev,
                      int64_t i, double *out) {
  double ci = m->coslat[i];
  for (int k = 0; k < nlev; ++k) {
    acc_t a = {0, 0};
    double ui = fld(u, f32, ld, i, k), vi = fld(v, f32, ld, i, k);
    for (int32_t p = m->n2e_ptr[i]; p < m->n2e_ptr[i + 1]; ++p) {
      int64_t e = m->n2e[p];
      if (m->is_pole[e]) continue;
      double nl, np;
      face_normal(m, p, &nl, &np);
      int32_t j = far_end(m, e, i);
      double dv = 0.5 * (fld(v, f32, ld, j, k) - vi);
      double duc = 0.5 * diff_of_products(fld(u, f32, ld, j, k), m->coslat[j], ui, ci);
      acc_add_prod(&a, nl, dv);
      acc_add_prod(&a, -np, duc);
    }
    if (m->pole_nphi[i] != 0.0) {
      /* - G_i . n_pole = + (u cos)_i n_pole,phi */
      double pu, eu;
      two_prod(ui, ci, &pu, &eu);
      acc_add_prod(&a, m->pole_nphi[i], pu);
      acc_add_prod(&a, m->pole_nphi[i], eu);
    }
    out[k] = acc_val(&a) / m->V[i];
  }
}

/* gradient of one physical component f of a tangent vector field at node i.
 * As the scalar gradient, except on the pole segment: a polar node and its
 * pole-edge neighbour (the node half a turn away on the same row) have
 * opposite local east and north directions, so the neighbour's component
 * enters the pole-face mean with its sign reversed, face value (f_i - f_j)/2.
 * In closure-exact form that face contributes n_pole ((f_i - f_j)/2 - f_i)
 * = -n_pole (f_i + f_j)/2. */
static void vgrad_comp_node(const orc_mesh *m, const void *f, int f32, int64_t ld, int nlev, int64_t i,
                            double *gx, double *gy) {
  for (int k = 0; k < nlev; ++k) {
    acc_t al = {0, 0}, ap = {0, 0};
    double fi = fld(f, f32, ld, i, k);
    for (int32_t p = m->n2e_ptr[i]; p < m->n2e_ptr[i + 1]; ++p) {
      double nl, np;
      face_normal(m, p, &nl, &np);
      int64_t e = m->n2e[p];
      int32_t j = far_end(m, e, i);
      double fj = fld(f, f32, ld, j, k);
      double d = m->is_pole[e] ? -0.5 * (fj + fi) : 0.5 * (fj - fi);
      acc_add_prod(&al, nl, d);
      acc_add_prod(&ap, np, d);
    }
    gx[k] = acc_val(&al) / m->V[i];
    gy[k] = m->coslat[i] * acc_val(&ap) / m->V[i];
  }
}

int orc_curl(const orc_mesh *m, const void *u, const void *v, int f32, int64_t ld, int nlev,
             const int64_t *nodes, int64_t count, double *out) {
  if (!m || !u || !v || nlev < 0 || ld < nlev || check_nodes(m, nodes, count)) return -1;
  int64_t n = nsel(m, nodes, count);
  for (int64_t q = 0; q < n; ++q) {
    int64_t i = nodes ? nodes[q] : q;
    curl_node(m, u, v, f32, ld, nlev, i, out + q * nlev);
  }
  return 0;
}

/* (ux, uy) = gradient of u, (vx, vy) = gradient of v, components of one
 * tangent vector field; outputs packed [count][nlev]. */
int orc_vector_gradient(const orc_mesh *m, const void *u, const void *v, int f32, int64_t ld, int nlev,
                        const int64_t *nodes, int64_t count, double *ux, double *uy, double *vx, double *vy) {
  if (!m || !u || !v || nlev < 0 || ld < nlev || check_nodes(m, nodes, count)) return -1;
  int64_t n = nsel(m, nodes, count);
  for (int64_t q = 0; q < n; ++q) {
    int64_t i = nodes ? nodes[q] : q;
    vgrad_comp_node(m, u, f32, ld, nlev, i, ux + q * nlev, uy + q * nlev);
    vgrad_comp_node(m, v, f32, ld, nlev, i, vx + q * nlev, vy + q * nlev);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoints: the exact transposes of the linear maps above, written as the  */
/* explicit matrix rows of the forward operator and applied transposed.     */
/* Row i of the gradient (component c) has the off-diagonal entries          */
/* w_c(i,j) on every edge neighbour j and the diagonal -sum_j w_c(i,j);      */
/* row i of the divergence has, for u, n_lambda/(2V) on regular neighbours   */
/* and minus their sum on the diagonal, and for v, n_phi cos_j/(2V) on       */
/* regular neighbours and -(sum n_phi cos_i/2 + cos_i n_pole)/V on the       */
/* diagonal.                                                                 */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t col; double c0, c1; } row_entry;

/* Entries of row i; the diagonal is split into one entry per face so that no
 * term is pre-summed (every product is accumulated exactly in Dot2 form).
 * Returns the number of entries written (<= 2*deg + 2). */
static int grad_row(const orc_mesh *m, int64_t i, row_entry *ent) {
  int nent = 0;
  for (int32_t p = m->n2e_ptr[i]; p < m->n2e_ptr[i + 1]; ++p) {
    double nl, np;
    face_normal(m, p, &nl, &np);
    int32_t j = far_end(m, m->n2e[p], i);
    double wl = nl / (2.0 * m->V[i]);
    double wp = m->coslat[i] * np / (2.0 * m->V[i]);
    ent[nent].col = j; ent[nent].c0 = wl; ent[nent].c1 = wp; ++nent;
    ent[nent].col = (int32_t)i; ent[nent].c0 = -wl; ent[nent].c1 = -wp; ++nent;
  }
  return nent;
}
static int div_row(const orc_mesh *m, int64_t i, row_entry *ent) {
  int nent = 0;
  double ci = m->coslat[i];
  for (int32_t p = m->n2e_ptr[i]; p < m->n2e_ptr[i + 1]; ++p) {
    int64_t e = m->n2e[p];
    if (m->is_pole[e]) continue;
    double nl, np;
    face_normal(m, p, &nl, &np);
    int32_t j = far_end(m, e, i);
    double wu = nl / (2.0 * m->V[i]);
    ent[nent].col = j; ent[nent].c0 = wu; ent[nent].c1 = np * m->coslat[j] / (2.0 * m->V[i]); ++nent;
    ent[nent].col = (int32_t)i; ent[nent].c0 = -wu; ent[nent].c1 = -(np * ci / (2.0 * m->V[i])); ++nent;
  }
  if (m->pole_nphi[i] != 0.0) {
    ent[nent].col = (int32_t)i; ent[nent].c0 = 0.0; ent[nent].c1 = -(m->pole_nphi[i] * ci / m->V[i]); ++nent;
  }
  return nent;
}

/* Row i of the curl, written out from the circulation form of curl_node:
 * V_i zeta_i = sum_regular [ n_lambda (v_j - v_i)/2 - n_phi (u_j cos_j - u_i cos_i)/2 ]
 *              + n_pole,phi u_i cos_i,
 * c0 the u coefficient, c1 the v coefficient; the diagonal is split into
 * one entry per face and one for the pole segment. */
static int curl_row(const orc_mesh *m, int64_t i, row_entry *ent) {
  int nent = 0;
  double ci = m->coslat[i];
  for (int32_t p = m->n2e_ptr[i]; p < m->n2e_ptr[i + 1]; ++p) {
    int64_t e = m->n2e[p];
    if (m->is_pole[e]) continue;
    double nl, np;
    face_normal(m, p, &nl, &np);
    int32_t j = far_end(m, e, i);
    ent[nent].col = j; ent[nent].c0 = -(np * m->coslat[j]) / (2.0 * m->V[i]); ent[nent].c1 = nl / (2.0 * m->V[i]);
    ++nent;
    ent[nent].col = (int32_t)i; ent[nent].c0 = (np * ci) / (2.0 * m->V[i]); ent[nent].c1 = -nl / (2.0 * m->V[i]);
    ++nent;
  }
  if (m->pole_nphi[i] != 0.0) {
    ent[nent].col = (int32_t)i; ent[nent].c0 = m->pole_nphi[i] * ci / m->V[i]; ent[nent].c1 = 0.0; ++nent;
  }
  return nent;
}

/* Gradient adjoint x = G^T y with y = (y_lambda, y_phi):
 *   x_k = sum_i [ G_lambda(i,k) y_lambda_i + G_phi(i,k) y_phi_i ].
 * Column k of G is non-zero only on rows i in {k} U neighbours(k). */
int orc_gradient_adjoint(const orc_mesh *m, const void *y0, const void *y1, int f32, int64_t ld, int nlev,
                         const int64_t *nodes, int64_t count, double *x) {
  if (!m || !y0 || !y1 || nlev < 0 || ld < nlev || check_nodes(m, nodes, count)) return -1;
  int64_t n = nsel(m, nodes, count);
  row_entry ent[160];
  acc_t *acc = (acc_t *)malloc(sizeof(acc_t) * (size_t)(nlev > 0 ? nlev : 1));
  if (!acc) return -2;
  for (int64_t q = 0; q < n; ++q) {
    int64_t k = nodes ? nodes[q] : q;
    for (int l = 0; l < nlev; ++l) acc[l].s = acc[l].c = 0.0;
    /* rows i = k, then i = each edge neighbour of k */
    for (int32_t p = m->n2e_ptr[k] - 1; p < m->n2e_ptr[k + 1]; ++p) {
      int64_t i = (p < m->n2e_ptr[k]) ? k : far_end(m, m->n2e[p], k);
      int ne = grad_row(m, i, ent);
      for (int t = 0; t < ne; ++t) {
        if (ent[t].col != k) continue;
        for (int l = 0; l < nlev; ++l) {
          acc_add_prod(&acc[l], ent[t].c0, fld(y0, f32, ld, i, l));
          acc_add_prod(&acc[l], ent[t].c1, fld(y1, f32, ld, i, l));
        }
      }
    }
    for (int l = 0; l < nlev; ++l) x[q * nlev + l] = acc_val(&acc[l]);
  }
  free(acc);
  return 0;
}

/* Divergence adjoint (x_u, x_v) = D^T d. */
int orc_divergence_adjoint(const orc_mesh *m, const void *d, int f32, int64_t ld, int nlev,
                           const int64_t *nodes, int64_t count, double *xu, double *xv) {
  if (!m || !d || nlev < 0 || ld < nlev || check_nodes(m, nodes, count)) return -1;
  int64_t n = nsel(m, nodes, count);
  row_entry ent[160];
  acc_t *au = (acc_t *)malloc(sizeof(acc_t) * (size_t)(nlev > 0 ? nlev : 1));
  acc_t *av = (acc_t *)malloc(sizeof(acc_t) * (size_t)(nlev > 0 ? nlev : 1));
  if (!au || !av) { free(au); free(av); return -2; }
  for (int64_t q = 0; q < n; ++q) {
    int64_t k = nodes ? nodes[q] : q;
    for (int l = 0; l < nlev; ++l) au[l].s = au[l].c = av[l].s = av[l].c = 0.0;
    for (int32_t p = m->n2e_ptr[k] - 1; p < m->n2e_ptr[k + 1]; ++p) {
      int64_t i = (p < m->n2e_ptr[k]) ? k : far_end(m, m->n2e[p], k);
      int ne = div_row(m, i, ent);
      for (int t = 0; t < ne; ++t) {
        if (ent[t].col != k) continue;
        for (int l = 0; l < nlev; ++l) {
          double di = fld(d, f32, ld, i, l);
          acc_add_prod(&au[l], ent[t].c0, di);
          acc_add_prod(&av[l], ent[t].c1, di);
        }
      }
    }
    for (int l = 0; l < nlev; ++l) { xu[q * nlev + l] = acc_val(&au[l]); xv[q * nlev + l] = acc_val(&av[l]); }
  }
  free(au); free(av);
  return 0;
}

/* Curl adjoint (x_u, x_v) = C^T z: column k of C is non-zero only on rows
 * i in {k} U neighbours(k). */
int orc_curl_adjoint(const orc_mesh *m, const void *z, int f32, int64_t ld, int nlev, const int64_t *nodes,
                     int64_t count, double *xu, double *xv) {
  if (!m || !z || nlev < 0 || ld < nlev || check_nodes(m, nodes, count)) return -1;
  int64_t n = nsel(m, nodes, count);
  row_entry ent[160];
  acc_t *au = (acc_t *)malloc(sizeof(acc_t) * (size_t)(nlev > 0 ? nlev : 1));
  acc_t *av = (acc_t *)malloc(sizeof(acc_t) * (size_t)(nlev > 0 ? nlev : 1));
  if (!au || !av) { free(au); free(av); return -2; }
  for (int64_t q = 0; q < n; ++q) {
    int64_t k = nodes ? nodes[q] : q;
    for (int l = 0; l < nlev; ++l) au[l].s = au[l].c = av[l].s = av[l].c = 0.0;
    for (int32_t p = m->n2e_ptr[k] - 1; p < m->n2e_ptr[k + 1]; ++p) {
      int64_t i = (p < m->n2e_ptr[k]) ? k : far_end(m, m->n2e[p], k);
      int ne = curl_row(m, i, ent);
      for (int t = 0; t < ne; ++t) {
        if (ent[t].col != k) continue;
        for (int l = 0; l < nlev; ++l) {
          double zi = fld(z, f32, ld, i, l);
          acc_add_prod(&au[l], ent[t].c0, zi);
          acc_add_prod(&av[l], ent[t].c1, zi);
        }
      }
    }
    for (int l = 0; l < nlev; ++l) { xu[q * nlev + l] = acc_val(&au[l]); xv[q * nlev + l] = acc_val(&av[l]); }
  }
  free(au); free(av);
  return 0;
}

/* Explicit COO triplets of the forward matrices (rows of G: 2V x V, stacked
 * lambda rows then phi rows; rows of D: V x 2V, u columns then v columns).
 * Diagonal pieces are emitted separately (duplicates are summed by the
 * caller).  Returns the number of triplets, or the capacity needed when the
 * buffers are NULL. */
int64_t orc_gradient_triplets(const orc_mesh *m, int64_t *rows, int64_t *cols, double *vals) {
  row_entry ent[160];
  int64_t n = 0;
  for (int64_t i = 0; i < m->nnodes; ++i) {
    int ne = grad_row(m, i, ent);
    for (int t = 0; t < ne; ++t) {
      if (rows) {
        rows[n] = i; cols[n] = ent[t].col; vals[n] = ent[t].c0;
        rows[n + 1] = m->nnodes + i; cols[n + 1] = ent[t].col; vals[n + 1] = ent[t].c1;
      }
      n += 2;
    }
  }
  return n;
}
int64_t orc_divergence_triplets(const orc_mesh *m, int64_t *rows, int64_t *cols, double *vals) {
  row_entry ent[160];
  int64_t n = 0;
  for (int64_t i = 0; i < m->nnodes; ++i) {
    int ne = div_row(m, i, ent);
    for (int t = 0; t < ne; ++t) {
      if (rows) {
        rows[n] = i; cols[n] = ent[t].col; vals[n] = ent[t].c0;
        rows[n + 1] = i; cols[n + 1] = m->nnodes + ent[t].col; vals[n + 1] = ent[t].c1;
      }
      n += 2;
    }
  }
  return n;
}

/* The averaged (textbook Green's theorem) form of the gradient,
 *   V_i g_i = sum_e n_ie (f_a + f_b)/2,
 * evaluated with Dot2.  Used only to check that it agrees with the
 * closure-exact form within the closure residual |f_i| |sum_e n_ie| / V_i. */
int orc_gradient_averaged(const orc_mesh *m, const void *f, int f32, int64_t ld, int nlev,
                          double *gx, double *gy) {
  if (!m || !f || nlev < 0 || ld < nlev) return -1;
  for (int64_t i = 0; i < m->nnodes; ++i)
    for (int k = 0; k < nlev; ++k) {
      acc_t al = {0, 0}, ap = {0, 0};
      for (int32_t p = m->n2e_ptr[i]; p < m->n2e_ptr[i + 1]; ++p) {
        int64_t e = m->n2e[p];
        double nl, np;
        face_normal(m, p, &nl, &np);
        double fa = fld(f, f32, ld, m->e2n[2 * e], k), fb = fld(f, f32, ld, m->e2n[2 * e + 1], k);
        acc_add_prod(&al, nl, 0.5 * fa);
        acc_add_prod(&al, nl, 0.5 * fb);
        acc_add_prod(&ap, np, 0.5 * fa);
        acc_add_prod(&ap, np, 0.5 * fb);
      }
      gx[i * nlev + k] = acc_val(&al) / m->V[i];
      gy[i * nlev + k] = m->coslat[i] * acc_val(&ap) / m->V[i];
    }
  return 0;
}

/* Closure residual of every cell: sum_e n_ie (two components) and sum |n_ie|. */
void orc_closure(const orc_mesh *m, double *res /* [V][2] */, double *absum /* [V] */) {
  for (int64_t i = 0; i < m->nnodes; ++i) {
    acc_t a0 = {0, 0}, a1 = {0, 0};
    double s = 0;
    for (int32_t p = m->n2e_ptr[i]; p < m->n2e_ptr[i + 1]; ++p) {
      double nl, np;
      face_normal(m, p, &nl, &np);
      acc_add(&a0, nl);
      acc_add(&a1, np);
      s += fabs(nl) + fabs(np);
    }
    res[2 * i] = acc_val(&a0);
    res[2 * i + 1] = acc_val(&a1);
    absum[i] = s;
  }
}

/* ------------------------------------------------------------------------ */
/* Remapping (paper Sec. 4.3, Fig. 6: a field on an O32 grid is remapped to */
/* an F8 grid with a linear element-based interpolation in 3D on the       */
/* sphere).  Reading: a target point with unit vector p lies in the source  */
/* triangle whose plane the ray from the centre along p crosses inside the  */
/* triangle; its value is the linear (barycentric) interpolation of the     */
/* three vertex values at that crossing point.  The crossing is solved with */
/* Cramer's rule for t p = a + u (b - a) + v (c - a) (the Moller-Trumbore   */
/* form); weights (1 - u - v, u, v).  Brute force over every triangle; when */
/* several contain the crossing (on a shared edge or vertex, up to 1e-12)   */
/* the one whose smallest weight is largest is taken, the lowest triangle   */
/* id on equality.  A target in a polar cap (north of the first row or      */
/* south of the last, where the mesh has no triangle) is not located.      */
/* ------------------------------------------------------------------------ */
static void unit_vector(double lon, double lat, double v[3]) {
  v[0] = cos(lat) * cos(lon);
  v[1] = cos(lat) * sin(lon);
  v[2] = sin(lat);
}
static void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void node_vector(const orc_mesh *m, int64_t i, double v[3]) {
  int r = m->node_row[i];
  double lon = TWO_PI * ((double)m->node_j[i] / (double)m->pl[r]);
  unit_vector(lon, m->lat[r], v);
}

/* nodes[t][3], w[t][3] for every target (lon, lat) in radians.  Returns 0,
 * or -4 when a target lies in no triangle (its nodes are set to -1). */
int orc_remap(const orc_mesh *m, const double *lonlat, int64_t ntgt, int32_t *nodes, double *w) {
  if (!m || !lonlat || !nodes || !w || ntgt < 0) return -1;
  double *vx = (double *)malloc(sizeof(double) * 3 * m->nnodes);
  if (!vx) return -2;
  for (int64_t i = 0; i < m->nnodes; ++i) node_vector(m, i, vx + 3 * i);
  int rc = 0;
  for (int64_t t = 0; t < ntgt; ++t) {
    double p[3];
    unit_vector(lonlat[2 * t], lonlat[2 * t + 1], p);
    double best = -1e300;
    int64_t bq = -1;
    double bw[3] = {0, 0, 0};
    for (int64_t q = 0; q < m->ntri; ++q) {
      const double *a = vx + 3 * m->tri[3 * q], *b = vx + 3 * m->tri[3 * q + 1], *c = vx + 3 * m->tri[3 * q + 2];
      double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
      double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
      double P[3], Q[3], T[3] = {-a[0], -a[1], -a[2]};
      cross3(p, e2, P);
      double det = dot3(e1, P);
      if (fabs(det) < 1e-300) continue;
      double inv = 1.0 / det;
      double u = dot3(T, P) * inv;
      cross3(T, e1, Q);
      double v = dot3(p, Q) * inv;
      double tt = dot3(e2, Q) * inv;
      if (tt <= 0) continue; /* the far side of the sphere */
      double w0 = 1.0 - u - v;
      double mn = fmin(w0, fmin(u, v));
      if (mn < -1e-12) continue;
      if (mn > best) {
        best = mn;
        bq = q;
        bw[0] = w0; bw[1] = u; bw[2] = v;
      }
    }
    if (bq < 0) {
      nodes[3 * t] = nodes[3 * t + 1] = nodes[3 * t + 2] = -1;
      w[3 * t] = w[3 * t + 1] = w[3 * t + 2] = 0;
      rc = -4;
      continue;
    }
    for (int k = 0; k < 3; ++k) {
      nodes[3 * t + k] = m->tri[3 * bq + k];
      w[3 * t + k] = bw[k];
    }
  }
  free(vx);
  return rc;
}

/* out[t][k] = sum_q w[t][q] f[nodes[t][q]][k], accumulated with Dot2. */
int orc_remap_apply(const int32_t *nodes, const double *w, int64_t ntgt, const void *f, int f32, int64_t ld, int nlev,
                    double *out) {
  if (!nodes || !w || !f || ntgt < 0 || nlev < 0 || ld < nlev) return -1;
  for (int64_t t = 0; t < ntgt; ++t)
    for (int k = 0; k < nlev; ++k) {
      acc_t a = {0, 0};
      for (int q = 0; q < 3; ++q) acc_add_prod(&a, w[3 * t + q], fld(f, f32, ld, nodes[3 * t + q], k));
      out[t * nlev + k] = acc_val(&a);
    }
  return 0;
}
