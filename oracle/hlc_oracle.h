/*
 * hlc_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 CPU statement of the positional
 * cross-match that HLC2 (Zhang et al., arXiv 2301.07331) computes: every
 * catalogue-B source within angular radius r of each catalogue-A source
 * (Sec. 2.1, Eq. 1), found through a HEALPix nested index (Sec. 4.2,
 * "hp_nestid") with either the complete 8-neighbour boundary rule or the
 * paper's quad-direction boundary strategy (Sec. 3.2, Algorithm 1).
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the bench
 * may load this library.  It shares no code, header, constant or table with
 * the CUDA library: every constant below is derived here from its
 * mathematical definition.
 *
 * Canonical arithmetic: all floating point is IEEE binary64 with explicit
 * fma() calls and no contraction (compiled with -ffp-contract=off), so each
 * result is a fixed sequence of correctly rounded operations.
 */
#ifndef HLC_ORACLE_H
#define HLC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Polynomial coefficients of sin/cos in degrees: the doubles nearest to
 * (-1)^k (pi/180)^(2k+1)/(2k+1)!  (k = 0..9) and (-1)^k (pi/180)^(2k)/(2k)!
 * (k = 0..10), computed once in binary128. */
void orc_coefficients(double sin_c[10], double cos_c[11]);

/* sin and cos of x degrees, |x| <= 720, by exact reduction to [-45, 45]. */
void orc_sincos_deg(double x, double* s, double* c);

/* RA folded into [0, 360). */
double orc_norm_ra(double ra);

/* Unit vector of (ra, dec) in degrees; ra already normalised. */
void orc_unitvec(double ra, double dec, double v[3]);

/* Squared chord between two unit vectors, fixed operation order. */
double orc_chord2(const double a[3], const double b[3]);

/* Squared-chord threshold 4 sin^2(r/2) for r in arcsec. */
double orc_threshold(double r_arcsec);

/* Separation in arcsec from a squared chord. */
double orc_sep_arcsec(double chord2);

/* HEALPix nested pixel of (ra, dec) degrees at the given order (0..29);
 * ra normalised to [0, 360). */
uint64_t orc_ang2pix(double ra, double dec, int order);

/* (face, ix, iy) <-> nested index. */
void orc_nest2fxy(uint64_t pix, int order, int* face, int64_t* ix, int64_t* iy);
uint64_t orc_fxy2nest(int face, int64_t ix, int64_t iy, int order);

/* The 8 neighbours of a nested pixel, in the direction order
 * (-1,-1) (-1,0) (-1,1) (0,1) (1,1) (1,0) (1,-1) (0,-1) of (dx, dy);
 * a missing neighbour (three-face vertices) is written as -1.
 * Returns the number of present neighbours. */
int orc_neighbours(uint64_t pix, int order, int64_t out[8]);

/* Pixel-centre direction (ra, dec degrees) of a nested pixel (plain libm). */
void orc_pix2ang(uint64_t pix, int order, double* ra, double* dec);

/* Quad-direction cell set of one source (Algorithm 1): the distinct pixels of
 * the source and of its four shifted copies, in ascending order.  Returns the
 * count (1..5). */
int orc_quad_cells(double ra, double dec, double r_arcsec, int order,
                   uint64_t out[5]);

/* The same with the RA copies shifted by R / cos(dec) (at most 180 deg)
 * instead of R: the RA extent of the radius at the source's declination. */
int orc_quad_cells_cos(double ra, double dec, double r_arcsec, int order,
                       uint64_t out[5]);

/* Match result: pairs sorted by (id_a, id_b) unsigned, ties by (ia, ib). */
typedef struct {
  uint64_t n;
  uint64_t* id_a;
  uint64_t* id_b;
  uint32_t* ia;   /* index into catalogue A */
  uint32_t* ib;   /* index into catalogue B */
  double* sep;    /* arcsec */
  double* chord2; /* squared chord, canonical */
  uint64_t pair_tests; /* predicate evaluations */
} orc_result;

/* Error codes. */
#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

/* mode: 0 = complete 8-neighbour, 1 = quad-direction, 2 = quad-direction
 * with the RA shift R / cos(dec). */
int orc_match(const double* ra_a, const double* dec_a, const uint64_t* id_a,
              uint64_t na, const double* ra_b, const double* dec_b,
              const uint64_t* id_b, uint64_t nb, double r_arcsec, int order,
              int mode, orc_result* out);

/* All-pairs reference of the same predicate (tiny inputs only). */
int orc_match_brute(const double* ra_a, const double* dec_a,
                    const uint64_t* id_a, uint64_t na, const double* ra_b,
                    const double* dec_b, const uint64_t* id_b, uint64_t nb,
                    double r_arcsec, orc_result* out);

void orc_result_free(orc_result* r);

/* Eq. 4 pair radius 3 sqrt(e1^2 + e2^2) arcsec (fixed operation order). */
double orc_pair_radius(double e1, double e2);

/* Complete mode with per-source error radii err_a, err_b (arcsec, finite,
 * >= 0): every (A_i, B_j) with separation <= orc_pair_radius(err_a[i],
 * err_b[j]).  ORC_EINVAL when the largest pair radius exceeds
 * orc_complete_max_radius(order). */
int orc_match_eq4(const double* ra_a, const double* dec_a, const uint64_t* id_a,
                  const double* err_a, uint64_t na, const double* ra_b,
                  const double* dec_b, const uint64_t* id_b, const double* err_b,
                  uint64_t nb, int order, orc_result* out);

/* All-pairs form of the same (tiny inputs only). */
int orc_match_brute_eq4(const double* ra_a, const double* dec_a,
                        const uint64_t* id_a, const double* err_a, uint64_t na,
                        const double* ra_b, const double* dec_b,
                        const uint64_t* id_b, const double* err_b, uint64_t nb,
                        orc_result* out);

/* Largest radius (arcsec) for which complete mode is exact at this order:
 * one eighth of the mean pixel side sqrt(pi/3)/2^order. */
double orc_complete_max_radius(int order);


/* Array forms (plain loops over the scalar functions; RA is normalised
 * inside where a function expects it). */
void orc_sincos_deg_n(const double* x, uint64_t n, double* s, double* c);
void orc_norm_ra_n(const double* ra, uint64_t n, double* out);
void orc_unitvec_n(const double* ra, const double* dec, uint64_t n, double* v);
void orc_ang2pix_n(const double* ra, const double* dec, uint64_t n, int order,
                   uint64_t* out);
void orc_neighbours_n(const uint64_t* pix, uint64_t n, int order, int64_t* out);
void orc_pix2ang_n(const uint64_t* pix, uint64_t n, int order, double* ra,
                   double* dec);
void orc_quad_cells_n(const double* ra, const double* dec, uint64_t n,
                      double r_arcsec, int order, uint64_t* out, int* cnt);
void orc_quad_cells_mode_n(const double* ra, const double* dec, uint64_t n,
                           double r_arcsec, int order, int cosdec, uint64_t* out, int* cnt);
void orc_chord2_n(const double* va, const double* vb, uint64_t n, double* out);
void orc_pair_radius_n(const double* e1, const double* e2, uint64_t n, double* out);

#ifdef __cplusplus
}
#endif
#endif
