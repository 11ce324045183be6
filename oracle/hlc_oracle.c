/*
 * hlc_oracle.c -- TEST INFRASTRUCTURE ONLY (see hlc_oracle.h).
 *
 * The slow, obviously-correct CPU statement of HLC2's positional cross-match
 * (arXiv 2301.07331).  Each function names the passage it follows:
 *   - Eq. 1 (Sec. 2.1): the match predicate d(O1, O2) <= r on the sphere,
 *     evaluated through the equivalent squared-chord form
 *     |u1 - u2|^2 <= 4 sin^2(r/2), which is Eq. 1 rewritten without the
 *     catastrophic cancellation of arccos near 0;
 *   - Sec. 4.2 ("hp_nestid"): HEALPix nested ang2pix (Gorski et al. 2005);
 *   - Sec. 3.2 and Algorithm 1: the quad-direction boundary strategy, read
 *     literally (R_A = R_B = r) and in a variant whose RA shift is the RA
 *     extent r / cos(dec) of the radius at the source's declination;
 *   - complete mode: the exact set of Eq. 1 reached through the cell of each
 *     A source and its 8 HEALPix neighbours;
 *   - Eq. 4: per-source error radii, each pair's radius 3 sqrt(e1^2 + e2^2).
 *
 * Compiled with -O2 -ffp-contract=off: every floating-point expression below
 * is evaluated exactly as written, one correctly rounded IEEE binary64
 * operation at a time, with fma() only where spelled out.
 */
#include "hlc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Constants from their definitions (binary128 arithmetic, then rounded).   */
/* ------------------------------------------------------------------------ */

static double g_sin_c[10];
static double g_cos_c[11];
static int g_init = 0;

/* atan(1/x) by its alternating series, in binary128. */
static __float128 atan_inv_q(int x) {
  __float128 xx = (__float128)x * (__float128)x;
  __float128 pw = 1.0Q / (__float128)x; /* x^-(2k+1) */
  __float128 sum = 0.0Q;
  for (int k = 0; k < 80; ++k) {
    __float128 term = pw / (__float128)(2 * k + 1);
    sum += (k & 1) ? -term : term;
    pw /= xx;
  }
  return sum;
}

static void init_constants(void) {
  if (g_init) return;
  /* Machin: pi = 16 atan(1/5) - 4 atan(1/239). */
  __float128 pi = 16.0Q * atan_inv_q(5) - 4.0Q * atan_inv_q(239);
  __float128 p = pi / 180.0Q; /* radians per degree */
  for (int k = 0; k < 10; ++k) {
    int n = 2 * k + 1;
    __float128 pw = 1.0Q, fact = 1.0Q;
    for (int i = 1; i <= n; ++i) {
      pw *= p;
      fact *= (__float128)i;
    }
    __float128 v = pw / fact;
    g_sin_c[k] = (double)((k & 1) ? -v : v);
  }
  for (int k = 0; k < 11; ++k) {
    int n = 2 * k;
    __float128 pw = 1.0Q, fact = 1.0Q;
    for (int i = 1; i <= n; ++i) {
      pw *= p;
      fact *= (__float128)i;
    }
    __float128 v = pw / fact;
    g_cos_c[k] = (double)((k & 1) ? -v : v);
  }
  g_init = 1;
}

void orc_coefficients(double sin_c[10], double cos_c[11]) {
  init_constants();
  memcpy(sin_c, g_sin_c, sizeof(g_sin_c));
  memcpy(cos_c, g_cos_c, sizeof(g_cos_c));
}

/* ------------------------------------------------------------------------ */
/* Canonical trigonometry in degrees.                                         */
/* ------------------------------------------------------------------------ */

void orc_sincos_deg(double x, double* s, double* c) {
  init_constants();
  double q = rint(x / 90.0);       /* nearest quadrant, ties to even */
  double t = x - 90.0 * q;         /* exact: |t| <= 45 */
  double u = t * t;
  double ps = g_sin_c[9];
  for (int k = 8; k >= 0; --k) ps = fma(ps, u, g_sin_c[k]);
  double sn = t * ps;
  double pc = g_cos_c[10];
  for (int k = 9; k >= 0; --k) pc = fma(pc, u, g_cos_c[k]);
  double cs = pc;
  long long n = ((long long)q) & 3;
  switch (n) {
    case 0: *s = sn; *c = cs; break;
    case 1: *s = cs; *c = -sn; break;
    case 2: *s = -sn; *c = -cs; break;
    default: *s = -cs; *c = sn; break;
  }
}

double orc_norm_ra(double ra) {
  double a = fmod(ra, 360.0);
  if (a < 0.0) a += 360.0;
  if (a >= 360.0) a -= 360.0;
  return a;
}

void orc_unitvec(double ra, double dec, double v[3]) {
  double sd, cd, sa, ca;
  orc_sincos_deg(dec, &sd, &cd);
  orc_sincos_deg(ra, &sa, &ca);
  v[0] = cd * ca;
  v[1] = cd * sa;
  v[2] = sd;
}

double orc_chord2(const double a[3], const double b[3]) {
  double dx = a[0] - b[0];
  double dy = a[1] - b[1];
  double dz = a[2] - b[2];
  double s = dx * dx;
  s = fma(dy, dy, s);
  s = fma(dz, dz, s);
  return s;
}

double orc_threshold(double r_arcsec) {
  double h = r_arcsec / 7200.0; /* half radius in degrees */
  double sh, ch;
  orc_sincos_deg(h, &sh, &ch);
  return 4.0 * (sh * sh);
}

double orc_sep_arcsec(double chord2) {
  double half = sqrt(chord2) * 0.5;
  if (half > 1.0) half = 1.0;
  return 2.0 * asin(half) * (648000.0 / M_PI);
}

double orc_complete_max_radius(int order) {
  double side_rad = sqrt(M_PI / 3.0) / ldexp(1.0, order);
  return side_rad * (648000.0 / M_PI) / 8.0;
}

/* Eq. 4 (Sec. 2.1): two sources with error radii e1, e2 match when their
 * distance is at most 3 sqrt(e1^2 + e2^2).  The pair radius in arcsec, in a
 * fixed operation order that is symmetric in the two errors (so swapping the
 * catalogues cannot change a decision): a = e1 e1, b = e2 e2, t = a + b,
 * r = 3 sqrt(t), each step correctly rounded. */
double orc_pair_radius(double e1, double e2) {
  double a = e1 * e1;
  double b = e2 * e2;
  double t = a + b;
  return 3.0 * sqrt(t);
}

/* ------------------------------------------------------------------------ */
/* HEALPix nested scheme (Gorski et al. 2005), "hp_nestid" of Sec. 4.2.     */
/* ------------------------------------------------------------------------ */

static uint64_t interleave(uint64_t ix, uint64_t iy, int order) {
  uint64_t r = 0;
  for (int b = 0; b < order; ++b) {
    r |= ((ix >> b) & 1ull) << (2 * b);
    r |= ((iy >> b) & 1ull) << (2 * b + 1);
  }
  return r;
}

uint64_t orc_fxy2nest(int face, int64_t ix, int64_t iy, int order) {
  uint64_t npface = 1ull << (2 * order);
  return (uint64_t)face * npface + interleave((uint64_t)ix, (uint64_t)iy, order);
}

void orc_nest2fxy(uint64_t pix, int order, int* face, int64_t* ix, int64_t* iy) {
  uint64_t npface = 1ull << (2 * order);
  *face = (int)(pix / npface);
  uint64_t p = pix % npface;
  uint64_t x = 0, y = 0;
  for (int b = 0; b < order; ++b) {
    x |= ((p >> (2 * b)) & 1ull) << b;
    y |= ((p >> (2 * b + 1)) & 1ull) << b;
  }
  *ix = (int64_t)x;
  *iy = (int64_t)y;
}

uint64_t orc_ang2pix(double ra, double dec, int order) {
  double ns = ldexp(1.0, order);
  int64_t nsi = (int64_t)1 << order;
  double sd, cd;
  orc_sincos_deg(dec, &sd, &cd);
  double z = sd;
  double za = fabs(z);
  double tt = ra / 90.0; /* in [0, 4) */
  int face;
  int64_t ix, iy;
  if (za <= 2.0 / 3.0) {
    /* equatorial belt */
    double t1 = ns * (0.5 + tt);
    double t2 = ns * (z * 0.75);
    int64_t jp = (int64_t)floor(t1 - t2); /* ascending edge line index */
    int64_t jm = (int64_t)floor(t1 + t2); /* descending edge line index */
    int64_t ifp = jp >> order;
    int64_t ifm = jm >> order;
    if (ifp == ifm)
      face = (int)(ifp | 4);
    else if (ifp < ifm)
      face = (int)ifp;
    else
      face = (int)(ifm + 8);
    ix = jm & (nsi - 1);
    iy = nsi - (jp & (nsi - 1)) - 1;
  } else {
    /* polar caps */
    int64_t ntt = (int64_t)floor(tt);
    if (ntt >= 4) ntt = 3;
    double tp = tt - (double)ntt;
    double w = 90.0 - fabs(dec);
    double sw, cw;
    orc_sincos_deg(0.5 * w, &sw, &cw);
    /* sqrt(3 (1 - |z|)) = sqrt(6) sin((90 - |dec|) / 2) */
    double tmp = ns * (sqrt(6.0) * sw);
    int64_t jp = (int64_t)floor(tp * tmp);
    int64_t jm = (int64_t)floor((1.0 - tp) * tmp);
    if (jp >= nsi) jp = nsi - 1;
    if (jm >= nsi) jm = nsi - 1;
    if (z > 0.0) {
      face = (int)ntt;
      ix = nsi - jm - 1;
      iy = nsi - jp - 1;
    } else {
      face = (int)(ntt + 8);
      ix = jp;
      iy = jm;
    }
  }
  return orc_fxy2nest(face, ix, iy, order);
}

void orc_pix2ang(uint64_t pix, int order, double* ra, double* dec) {
  int face;
  int64_t ix, iy;
  orc_nest2fxy(pix, order, &face, &ix, &iy);
  double n = ldexp(1.0, order);
  int k = face & 3;
  double z, tt;
  /* polar inverse (only valid where the result has |z| > 2/3) */
  double tmp = 2.0 * n - (double)ix - (double)iy - 1.0;
  int polar = 0;
  if (face < 4 && tmp < n) {
    double jp = n - 1.0 - (double)iy, jm = n - 1.0 - (double)ix;
    (void)jm;
    double tp = (jp + 0.5) / tmp;
    z = 1.0 - (tmp / n) * (tmp / n) / 3.0;
    tt = k + tp;
    polar = 1;
  } else if (face >= 8 && (double)ix + (double)iy + 1.0 < n) {
    double jp = (double)ix, jm = (double)iy;
    double t2 = jp + jm + 1.0;
    double tp = (jp + 0.5) / t2;
    z = -(1.0 - (t2 / n) * (t2 / n) / 3.0);
    tt = k + tp;
    polar = 1;
  }
  if (!polar) {
    double jm, jp;
    if (face < 4) {
      jm = (k + 1) * n + (double)ix;
      jp = k * n + n - 1.0 - (double)iy;
    } else if (face < 8) {
      jm = k * n + (double)ix;
      jp = k * n + n - 1.0 - (double)iy;
    } else {
      jm = k * n + (double)ix;
      jp = (k + 1) * n + n - 1.0 - (double)iy;
    }
    double um = jm + 0.5, up = jp + 0.5;
    tt = (up + um) / (2.0 * n) - 0.5;
    z = (um - up) / (1.5 * n);
  }
  double phi_deg = tt * 90.0;
  phi_deg = fmod(phi_deg, 360.0);
  if (phi_deg < 0) phi_deg += 360.0;
  *ra = phi_deg;
  *dec = asin(z) * (180.0 / M_PI);
}

/* Neighbours from the face layout: faces 0-3 north polar (centred at
 * phi = 45 + 90k deg), 4-7 equatorial (phi = 90k), 8-11 south polar.  Within
 * a face ix grows to the north-east and iy to the north-west, so the south
 * vertex is (0,0), east (n,0), north (n,n), west (0,n).  Crossing an edge
 * between a polar and an equatorial face is a translation of (ix, iy); crossing
 * between two polar faces is a quarter turn about the pole.  Corners where
 * four faces meet (poles, equatorial vertices) have a diagonal neighbour; the
 * eight vertices where three faces meet (z = +-2/3, phi = 90k) do not. */
static int face_step(int face, int64_t x, int64_t y, int64_t n, int* f_out,
                     int64_t* x_out, int64_t* y_out) {
  int k = face & 3;
  int xin = (x >= 0 && x < n), yin = (y >= 0 && y < n);
  if (xin && yin) {
    *f_out = face; *x_out = x; *y_out = y;
    return 1;
  }
  if (!xin && !yin) {
    int xhi = x >= n, yhi = y >= n;
    if (face < 4) {
      if (xhi && yhi) { *f_out = (k + 2) & 3; *x_out = n - 1; *y_out = n - 1; return 1; }
      if (!xhi && !yhi) { *f_out = 8 + k; *x_out = n - 1; *y_out = n - 1; return 1; }
      return 0;
    } else if (face < 8) {
      if (xhi && !yhi) { *f_out = 4 + ((k + 1) & 3); *x_out = 0; *y_out = n - 1; return 1; }
      if (!xhi && yhi) { *f_out = 4 + ((k + 3) & 3); *x_out = n - 1; *y_out = 0; return 1; }
      return 0;
    } else {
      if (!xhi && !yhi) { *f_out = 8 + ((k + 2) & 3); *x_out = 0; *y_out = 0; return 1; }
      if (xhi && yhi) { *f_out = k; *x_out = 0; *y_out = 0; return 1; }
      return 0;
    }
  }
  if (face < 4) {
    if (x >= n) { *f_out = (k + 1) & 3; *x_out = y; *y_out = 2 * n - 1 - x; return 1; }
    if (y >= n) { *f_out = (k + 3) & 3; *x_out = 2 * n - 1 - y; *y_out = x; return 1; }
    if (x < 0) { *f_out = 4 + k; *x_out = x + n; *y_out = y; return 1; }
    *f_out = 4 + ((k + 1) & 3); *x_out = x; *y_out = y + n; return 1;
  } else if (face < 8) {
    if (x >= n) { *f_out = k; *x_out = x - n; *y_out = y; return 1; }
    if (y >= n) { *f_out = (k + 3) & 3; *x_out = x; *y_out = y - n; return 1; }
    if (x < 0) { *f_out = 8 + ((k + 3) & 3); *x_out = x + n; *y_out = y; return 1; }
    *f_out = 8 + k; *x_out = x; *y_out = y + n; return 1;
  } else {
    if (x >= n) { *f_out = 4 + ((k + 1) & 3); *x_out = x - n; *y_out = y; return 1; }
    if (y >= n) { *f_out = 4 + k; *x_out = x; *y_out = y - n; return 1; }
    if (x < 0) { *f_out = 8 + ((k + 3) & 3); *x_out = y; *y_out = -1 - x; return 1; }
    *f_out = 8 + ((k + 1) & 3); *x_out = -1 - y; *y_out = x; return 1;
  }
}

int orc_neighbours(uint64_t pix, int order, int64_t out[8]) {
  static const int dxs[8] = {-1, -1, -1, 0, 1, 1, 1, 0};
  static const int dys[8] = {-1, 0, 1, 1, 1, 0, -1, -1};
  int face;
  int64_t ix, iy;
  orc_nest2fxy(pix, order, &face, &ix, &iy);
  int64_t n = (int64_t)1 << order;
  int cnt = 0;
  for (int d = 0; d < 8; ++d) {
    int f2;
    int64_t x2, y2;
    if (face_step(face, ix + dxs[d], iy + dys[d], n, &f2, &x2, &y2)) {
      out[d] = (int64_t)orc_fxy2nest(f2, x2, y2, order);
      ++cnt;
    } else {
      out[d] = -1;
    }
  }
  return cnt;
}

/* ------------------------------------------------------------------------ */
/* Quad-direction cells (Sec. 3.2, Algorithm 1).                             */
/* ------------------------------------------------------------------------ */

static double wrap_ra(double x) {
  double y = x;
  if (y < 0.0)
    y += 360.0;
  else if (y >= 360.0)
    y -= 360.0;
  if (y >= 360.0) y = 0.0;
  return y;
}

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return (x > y) - (x < y);
}

/* The RA shift of the cos(Dec) variant: the RA extent R / cos(dec) of an
 * angle R at declination dec (canonical cosine), 180 deg at most (and where
 * cos(dec) is 0). */
static double ra_shift_cos(double R, double dec) {
  double sd, cd;
  orc_sincos_deg(dec, &sd, &cd);
  double c = fabs(cd);
  double RA = c > 0.0 ? R / c : 180.0;
  if (RA > 180.0) RA = 180.0;
  return RA;
}

/* cosdec = 0: Algorithm 1 read literally (R_A = R_B = r in degrees);
 * cosdec = 1: the variant with R_A = R / cos(dec), R_B = R. */
static int quad_cells_impl(double ra, double dec, double r_arcsec, int order, int cosdec,
                           uint64_t out[5]) {
  double R = r_arcsec / 3600.0; /* R_B = r in degrees */
  double RA = cosdec ? ra_shift_cos(R, dec) : R;
  double dec_plus = dec + R;
  if (dec_plus > 90.0) dec_plus = 90.0;
  double dec_minus = dec - R;
  if (dec_minus < -90.0) dec_minus = -90.0;
  uint64_t p[5];
  p[0] = orc_ang2pix(ra, dec, order);
  p[1] = orc_ang2pix(wrap_ra(ra + RA), dec, order);
  p[2] = orc_ang2pix(wrap_ra(ra - RA), dec, order);
  p[3] = orc_ang2pix(ra, dec_minus, order);
  p[4] = orc_ang2pix(ra, dec_plus, order);
  qsort(p, 5, sizeof(uint64_t), cmp_u64);
  int m = 0;
  for (int i = 0; i < 5; ++i)
    if (m == 0 || p[i] != out[m - 1]) out[m++] = p[i];
  return m;
}

int orc_quad_cells(double ra, double dec, double r_arcsec, int order, uint64_t out[5]) {
  return quad_cells_impl(ra, dec, r_arcsec, order, 0, out);
}

int orc_quad_cells_cos(double ra, double dec, double r_arcsec, int order, uint64_t out[5]) {
  return quad_cells_impl(ra, dec, r_arcsec, order, 1, out);
}

/* ------------------------------------------------------------------------ */
/* Matching.                                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint64_t key;
  uint32_t idx;
} kv_t;

static int cmp_kv(const void* a, const void* b) {
  const kv_t* x = (const kv_t*)a;
  const kv_t* y = (const kv_t*)b;
  if (x->key != y->key) return (x->key > y->key) - (x->key < y->key);
  return (x->idx > y->idx) - (x->idx < y->idx);
}

typedef struct {
  uint64_t ida, idb;
  uint32_t ia, ib;
  double c2;
} pair_t;

static int cmp_pair(const void* a, const void* b) {
  const pair_t* x = (const pair_t*)a;
  const pair_t* y = (const pair_t*)b;
  if (x->ida != y->ida) return (x->ida > y->ida) - (x->ida < y->ida);
  if (x->idb != y->idb) return (x->idb > y->idb) - (x->idb < y->idb);
  if (x->ia != y->ia) return (x->ia > y->ia) - (x->ia < y->ia);
  return (x->ib > y->ib) - (x->ib < y->ib);
}

typedef struct {
  pair_t* v;
  uint64_t n, cap;
} pairvec;

static int push_pair(pairvec* pv, pair_t p) {
  if (pv->n == pv->cap) {
    uint64_t nc = pv->cap ? pv->cap * 2 : 1024;
    pair_t* nv = (pair_t*)realloc(pv->v, nc * sizeof(pair_t));
    if (!nv) return ORC_ENOMEM;
    pv->v = nv;
    pv->cap = nc;
  }
  pv->v[pv->n++] = p;
  return ORC_OK;
}

static int finish(pairvec* pv, uint64_t tests, orc_result* out) {
  qsort(pv->v, pv->n, sizeof(pair_t), cmp_pair);
  uint64_t n = pv->n;
  out->n = n;
  out->pair_tests = tests;
  size_t m = n ? n : 1;
  out->id_a = (uint64_t*)malloc(m * sizeof(uint64_t));
  out->id_b = (uint64_t*)malloc(m * sizeof(uint64_t));
  out->ia = (uint32_t*)malloc(m * sizeof(uint32_t));
  out->ib = (uint32_t*)malloc(m * sizeof(uint32_t));
  out->sep = (double*)malloc(m * sizeof(double));
  out->chord2 = (double*)malloc(m * sizeof(double));
  if (!out->id_a || !out->id_b || !out->ia || !out->ib || !out->sep ||
      !out->chord2) {
    orc_result_free(out);
    free(pv->v);
    return ORC_ENOMEM;
  }
  for (uint64_t i = 0; i < n; ++i) {
    out->id_a[i] = pv->v[i].ida;
    out->id_b[i] = pv->v[i].idb;
    out->ia[i] = pv->v[i].ia;
    out->ib[i] = pv->v[i].ib;
    out->chord2[i] = pv->v[i].c2;
    out->sep[i] = orc_sep_arcsec(pv->v[i].c2);
  }
  free(pv->v);
  return ORC_OK;
}

void orc_result_free(orc_result* r) {
  free(r->id_a); free(r->id_b); free(r->ia); free(r->ib);
  free(r->sep); free(r->chord2);
  memset(r, 0, sizeof(*r));
}

static int valid_inputs(const double* ra, const double* dec, uint64_t n) {
  for (uint64_t i = 0; i < n; ++i) {
    if (!isfinite(ra[i]) || !isfinite(dec[i])) return 0;
    if (dec[i] < -90.0 || dec[i] > 90.0) return 0;
  }
  return 1;
}

/* Unit vectors of a catalogue (normalised RA). */
static double* unit_vectors(const double* ra, const double* dec, uint64_t n) {
  double* v = (double*)malloc((n ? n : 1) * 3 * sizeof(double));
  if (!v) return NULL;
  for (uint64_t i = 0; i < n; ++i)
    orc_unitvec(orc_norm_ra(ra[i]), dec[i], v + 3 * i);
  return v;
}

/* First index in sorted keys[0..n) whose key >= q. */
static uint64_t lower_bound_kv(const kv_t* a, uint64_t n, uint64_t q) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (a[mid].key < q)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

/* err_a/err_b: NULL for one radius (threshold C for every pair); else the
 * per-source error radii of Eq. 4 and each pair's own threshold
 * 4 sin^2(r_ij / 2), r_ij = orc_pair_radius(err_a[i], err_b[j]). */
static int match_complete(const double* ra_a, const double* dec_a,
                          const uint64_t* id_a, const double* err_a, uint64_t na,
                          const double* ra_b, const double* dec_b,
                          const uint64_t* id_b, const double* err_b, uint64_t nb,
                          double C, int order, orc_result* out) {
  double* va = unit_vectors(ra_a, dec_a, na);
  double* vb = unit_vectors(ra_b, dec_b, nb);
  kv_t* kb = (kv_t*)malloc((nb ? nb : 1) * sizeof(kv_t));
  if (!va || !vb || !kb) {
    free(va); free(vb); free(kb);
    return ORC_ENOMEM;
  }
  for (uint64_t j = 0; j < nb; ++j) {
    kb[j].key = orc_ang2pix(orc_norm_ra(ra_b[j]), dec_b[j], order);
    kb[j].idx = (uint32_t)j;
  }
  qsort(kb, nb, sizeof(kv_t), cmp_kv);
  pairvec pv = {0};
  uint64_t tests = 0;
  int rc = ORC_OK;
  for (uint64_t i = 0; i < na && rc == ORC_OK; ++i) {
    uint64_t p = orc_ang2pix(orc_norm_ra(ra_a[i]), dec_a[i], order);
    int64_t nb8[8];
    orc_neighbours(p, order, nb8);
    /* the cell itself plus its distinct present neighbours */
    uint64_t cells[9];
    int nc = 0;
    cells[nc++] = p;
    for (int d = 0; d < 8; ++d) {
      if (nb8[d] < 0) continue;
      int dup = 0;
      for (int e = 0; e < nc; ++e) dup |= (cells[e] == (uint64_t)nb8[d]);
      if (!dup) cells[nc++] = (uint64_t)nb8[d];
    }
    for (int e = 0; e < nc; ++e) {
      uint64_t lo = lower_bound_kv(kb, nb, cells[e]);
      for (uint64_t t = lo; t < nb && kb[t].key == cells[e]; ++t) {
        uint32_t j = kb[t].idx;
        double c2 = orc_chord2(va + 3 * i, vb + 3 * (uint64_t)j);
        ++tests;
        double Cij = err_a ? orc_threshold(orc_pair_radius(err_a[i], err_b[j])) : C;
        if (c2 <= Cij) {
          pair_t pr = {id_a[i], id_b[j], (uint32_t)i, j, c2};
          rc = push_pair(&pv, pr);
          if (rc) break;
        }
      }
    }
  }
  free(va); free(vb); free(kb);
  if (rc) {
    free(pv.v);
    return rc;
  }
  return finish(&pv, tests, out);
}

static int match_quad(const double* ra_a, const double* dec_a,
                      const uint64_t* id_a, uint64_t na, const double* ra_b,
                      const double* dec_b, const uint64_t* id_b, uint64_t nb,
                      double r_arcsec, double C, int order, int cosdec,
                      orc_result* out) {
  double* va = unit_vectors(ra_a, dec_a, na);
  double* vb = unit_vectors(ra_b, dec_b, nb);
  uint64_t* ca = (uint64_t*)malloc((na ? na : 1) * 5 * sizeof(uint64_t));
  uint64_t* cb = (uint64_t*)malloc((nb ? nb : 1) * 5 * sizeof(uint64_t));
  int* nca = (int*)malloc((na ? na : 1) * sizeof(int));
  int* ncb = (int*)malloc((nb ? nb : 1) * sizeof(int));
  kv_t* ea = (kv_t*)malloc((na ? na : 1) * 5 * sizeof(kv_t));
  kv_t* eb = (kv_t*)malloc((nb ? nb : 1) * 5 * sizeof(kv_t));
  int rc = ORC_OK;
  if (!va || !vb || !ca || !cb || !nca || !ncb || !ea || !eb) rc = ORC_ENOMEM;
  uint64_t nea = 0, neb = 0;
  if (rc == ORC_OK) {
    for (uint64_t i = 0; i < na; ++i) {
      nca[i] = quad_cells_impl(orc_norm_ra(ra_a[i]), dec_a[i], r_arcsec, order, cosdec,
                               ca + 5 * i);
      for (int e = 0; e < nca[i]; ++e) {
        ea[nea].key = ca[5 * i + e];
        ea[nea].idx = (uint32_t)i;
        ++nea;
      }
    }
    for (uint64_t j = 0; j < nb; ++j) {
      ncb[j] = quad_cells_impl(orc_norm_ra(ra_b[j]), dec_b[j], r_arcsec, order, cosdec,
                               cb + 5 * j);
      for (int e = 0; e < ncb[j]; ++e) {
        eb[neb].key = cb[5 * j + e];
        eb[neb].idx = (uint32_t)j;
        ++neb;
      }
    }
    qsort(ea, nea, sizeof(kv_t), cmp_kv);
    qsort(eb, neb, sizeof(kv_t), cmp_kv);
  }
  pairvec pv = {0};
  uint64_t tests = 0;
  uint64_t s = 0;
  while (rc == ORC_OK && s < nea) {
    uint64_t cell = ea[s].key;
    uint64_t s_end = s;
    while (s_end < nea && ea[s_end].key == cell) ++s_end;
    uint64_t lo = lower_bound_kv(eb, neb, cell);
    uint64_t hi = lo;
    while (hi < neb && eb[hi].key == cell) ++hi;
    for (uint64_t x = s; x < s_end && rc == ORC_OK; ++x) {
      uint32_t i = ea[x].idx;
      for (uint64_t y = lo; y < hi; ++y) {
        uint32_t j = eb[y].idx;
        double c2 = orc_chord2(va + 3 * (uint64_t)i, vb + 3 * (uint64_t)j);
        ++tests;
        if (!(c2 <= C)) continue;
        /* report the pair once: in the smallest cell the two sets share */
        uint64_t owner = UINT64_MAX;
        for (int e = 0; e < nca[i]; ++e)
          for (int f = 0; f < ncb[j]; ++f)
            if (ca[5 * (uint64_t)i + e] == cb[5 * (uint64_t)j + f] &&
                ca[5 * (uint64_t)i + e] < owner)
              owner = ca[5 * (uint64_t)i + e];
        if (owner != cell) continue;
        pair_t pr = {id_a[i], id_b[j], i, j, c2};
        rc = push_pair(&pv, pr);
        if (rc) break;
      }
    }
    s = s_end;
  }
  free(va); free(vb); free(ca); free(cb); free(nca); free(ncb);
  free(ea); free(eb);
  if (rc) {
    free(pv.v);
    return rc;
  }
  return finish(&pv, tests, out);
}

int orc_match(const double* ra_a, const double* dec_a, const uint64_t* id_a,
              uint64_t na, const double* ra_b, const double* dec_b,
              const uint64_t* id_b, uint64_t nb, double r_arcsec, int order,
              int mode, orc_result* out) {
  memset(out, 0, sizeof(*out));
  if (!(r_arcsec > 0.0) || !(r_arcsec <= 648000.0)) return ORC_EINVAL;
  if (order < 0 || order > 29) return ORC_EINVAL;
  if (mode != 0 && mode != 1 && mode != 2) return ORC_EINVAL;
  if (mode == 0 && r_arcsec > orc_complete_max_radius(order)) return ORC_EINVAL;
  if (na > 0xFFFFFFFFull || nb > 0xFFFFFFFFull) return ORC_EINVAL;
  if (!valid_inputs(ra_a, dec_a, na) || !valid_inputs(ra_b, dec_b, nb))
    return ORC_EINVAL;
  double C = orc_threshold(r_arcsec);
  if (mode == 0)
    return match_complete(ra_a, dec_a, id_a, NULL, na, ra_b, dec_b, id_b, NULL, nb,
                          C, order, out);
  return match_quad(ra_a, dec_a, id_a, na, ra_b, dec_b, id_b, nb, r_arcsec, C,
                    order, mode == 2, out);
}

int orc_match_brute(const double* ra_a, const double* dec_a,
                    const uint64_t* id_a, uint64_t na, const double* ra_b,
                    const double* dec_b, const uint64_t* id_b, uint64_t nb,
                    double r_arcsec, orc_result* out) {
  memset(out, 0, sizeof(*out));
  if (!(r_arcsec > 0.0) || !(r_arcsec <= 648000.0)) return ORC_EINVAL;
  if (!valid_inputs(ra_a, dec_a, na) || !valid_inputs(ra_b, dec_b, nb))
    return ORC_EINVAL;
  double C = orc_threshold(r_arcsec);
  double* va = unit_vectors(ra_a, dec_a, na);
  double* vb = unit_vectors(ra_b, dec_b, nb);
  if (!va || !vb) {
    free(va); free(vb);
    return ORC_ENOMEM;
  }
  pairvec pv = {0};
  int rc = ORC_OK;
  for (uint64_t i = 0; i < na && rc == ORC_OK; ++i)
    for (uint64_t j = 0; j < nb; ++j) {
      double c2 = orc_chord2(va + 3 * i, vb + 3 * j);
      if (c2 <= C) {
        pair_t pr = {id_a[i], id_b[j], (uint32_t)i, (uint32_t)j, c2};
        rc = push_pair(&pv, pr);
        if (rc) break;
      }
    }
  free(va); free(vb);
  if (rc) {
    free(pv.v);
    return rc;
  }
  return finish(&pv, na * nb, out);
}

/* ------------------------------------------------------------------------ */
/* Per-source error radii (Eq. 4).                                           */
/* ------------------------------------------------------------------------ */

static int valid_errors(const double* e, uint64_t n, double* emax) {
  *emax = 0.0;
  for (uint64_t i = 0; i < n; ++i) {
    if (!isfinite(e[i]) || e[i] < 0.0) return 0;
    if (e[i] > *emax) *emax = e[i];
  }
  return 1;
}

int orc_match_eq4(const double* ra_a, const double* dec_a, const uint64_t* id_a,
                  const double* err_a, uint64_t na, const double* ra_b,
                  const double* dec_b, const uint64_t* id_b, const double* err_b,
                  uint64_t nb, int order, orc_result* out) {
  memset(out, 0, sizeof(*out));
  if (order < 0 || order > 29) return ORC_EINVAL;
  if (na > 0xFFFFFFFFull || nb > 0xFFFFFFFFull) return ORC_EINVAL;
  if (!valid_inputs(ra_a, dec_a, na) || !valid_inputs(ra_b, dec_b, nb))
    return ORC_EINVAL;
  double ma, mb;
  if (!valid_errors(err_a, na, &ma) || !valid_errors(err_b, nb, &mb))
    return ORC_EINVAL;
  /* complete mode is exact only while every pair radius is <= theta_L/8 */
  if (orc_pair_radius(ma, mb) > orc_complete_max_radius(order)) return ORC_EINVAL;
  return match_complete(ra_a, dec_a, id_a, err_a, na, ra_b, dec_b, id_b, err_b,
                        nb, 0.0, order, out);
}

int orc_match_brute_eq4(const double* ra_a, const double* dec_a,
                        const uint64_t* id_a, const double* err_a, uint64_t na,
                        const double* ra_b, const double* dec_b,
                        const uint64_t* id_b, const double* err_b, uint64_t nb,
                        orc_result* out) {
  memset(out, 0, sizeof(*out));
  double ma, mb;
  if (!valid_inputs(ra_a, dec_a, na) || !valid_inputs(ra_b, dec_b, nb) ||
      !valid_errors(err_a, na, &ma) || !valid_errors(err_b, nb, &mb))
    return ORC_EINVAL;
  double* va = unit_vectors(ra_a, dec_a, na);
  double* vb = unit_vectors(ra_b, dec_b, nb);
  if (!va || !vb) {
    free(va); free(vb);
    return ORC_ENOMEM;
  }
  pairvec pv = {0};
  int rc = ORC_OK;
  for (uint64_t i = 0; i < na && rc == ORC_OK; ++i)
    for (uint64_t j = 0; j < nb; ++j) {
      double c2 = orc_chord2(va + 3 * i, vb + 3 * j);
      if (c2 <= orc_threshold(orc_pair_radius(err_a[i], err_b[j]))) {
        pair_t pr = {id_a[i], id_b[j], (uint32_t)i, (uint32_t)j, c2};
        rc = push_pair(&pv, pr);
        if (rc) break;
      }
    }
  free(va); free(vb);
  if (rc) {
    free(pv.v);
    return rc;
  }
  return finish(&pv, na * nb, out);
}

/* ------------------------------------------------------------------------ */
/* Array forms of the scalar functions above (plain loops, for the tests).   */
/* ------------------------------------------------------------------------ */

void orc_sincos_deg_n(const double* x, uint64_t n, double* s, double* c) {
  for (uint64_t i = 0; i < n; ++i) orc_sincos_deg(x[i], s + i, c + i);
}

void orc_norm_ra_n(const double* ra, uint64_t n, double* out) {
  for (uint64_t i = 0; i < n; ++i) out[i] = orc_norm_ra(ra[i]);
}

void orc_unitvec_n(const double* ra, const double* dec, uint64_t n,
                   double* v) {
  for (uint64_t i = 0; i < n; ++i)
    orc_unitvec(orc_norm_ra(ra[i]), dec[i], v + 3 * i);
}

void orc_ang2pix_n(const double* ra, const double* dec, uint64_t n, int order,
                   uint64_t* out) {
  for (uint64_t i = 0; i < n; ++i)
    out[i] = orc_ang2pix(orc_norm_ra(ra[i]), dec[i], order);
}

void orc_neighbours_n(const uint64_t* pix, uint64_t n, int order,
                      int64_t* out) {
  for (uint64_t i = 0; i < n; ++i) orc_neighbours(pix[i], order, out + 8 * i);
}

void orc_pix2ang_n(const uint64_t* pix, uint64_t n, int order, double* ra,
                   double* dec) {
  for (uint64_t i = 0; i < n; ++i) orc_pix2ang(pix[i], order, ra + i, dec + i);
}

void orc_quad_cells_n(const double* ra, const double* dec, uint64_t n,
                      double r_arcsec, int order, uint64_t* out, int* cnt) {
  orc_quad_cells_mode_n(ra, dec, n, r_arcsec, order, 0, out, cnt);
}

void orc_quad_cells_mode_n(const double* ra, const double* dec, uint64_t n,
                           double r_arcsec, int order, int cosdec, uint64_t* out, int* cnt) {
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t c[5];
    int m = quad_cells_impl(orc_norm_ra(ra[i]), dec[i], r_arcsec, order, cosdec, c);
    for (int e = 0; e < 5; ++e) out[5 * i + e] = e < m ? c[e] : UINT64_MAX;
    cnt[i] = m;
  }
}

void orc_pair_radius_n(const double* e1, const double* e2, uint64_t n, double* out) {
  for (uint64_t i = 0; i < n; ++i) out[i] = orc_pair_radius(e1[i], e2[i]);
}

void orc_chord2_n(const double* va, const double* vb, uint64_t n, double* out) {
  for (uint64_t i = 0; i < n; ++i) out[i] = orc_chord2(va + 3 * i, vb + 3 * i);
}
