// Canonical binary64 arithmetic on the device: sin/cos in degrees, unit
// vectors, the squared-chord predicate of Eq. 1 and HEALPix nested ang2pix
// ("hp_nestid", Sec. 4.2; Gorski et al. 2005), plus nested neighbours and the
// quad-direction cell set of Algorithm 1.
//
// Every floating-point step is an explicit round-to-nearest intrinsic
// (__dadd_rn, __dmul_rn, __fma_rn, __ddiv_rn), so the compiler cannot fuse or
// reorder anything: the results are a fixed sequence of IEEE operations.
#pragma once

#include "common.cuh"

namespace hlc {

struct CanonDev {
  double s[10];
  double c[11];
  double sqrt6;
};
__constant__ CanonDev d_canon;

// Neighbour transition table: for base face f and the 3x3 region
// (x below / inside / above the face) x (y below / inside / above), the face
// reached and the coordinate map (see NbrMap).  255 = no neighbour there.
// (Global memory, read through the read-only cache: lanes of a warp index it
// with different faces, which constant memory would serialise.)
__device__ uint8_t d_nbr_face[12][9];
__device__ uint8_t d_nbr_map[12][9];

enum NbrMap : uint8_t {
  NM_SAME = 0,    // inside the face
  NM_SHIFT = 1,   // polar <-> equatorial crossing: (x, y) taken modulo n
  NM_ROT_N1 = 2,  // around the north pole, x overflow: (y, 2n-1-x)
  NM_ROT_N3 = 3,  // around the north pole, y overflow: (2n-1-y, x)
  NM_ROT_S3 = 4,  // around the south pole, x underflow: (y, -1-x)
  NM_ROT_S1 = 5,  // around the south pole, y underflow: (-1-y, x)
  NM_AT_00 = 6,   // diagonal across a four-face vertex, lands on (0, 0)
  NM_AT_NN = 7,   // ... lands on (n-1, n-1)
  NM_AT_0N = 8,   // ... lands on (0, n-1)
  NM_AT_N0 = 9,   // ... lands on (n-1, 0)
};

// ---- sin / cos in degrees --------------------------------------------------
__device__ __forceinline__ void c_sincos_deg(double x, double* s, double* c) {
  double q = rint(__ddiv_rn(x, 90.0));
  double t = __dsub_rn(x, __dmul_rn(90.0, q));  // exact, |t| <= 45
  double u = __dmul_rn(t, t);
  double ps = d_canon.s[9];
#pragma unroll
  for (int k = 8; k >= 0; --k) ps = __fma_rn(ps, u, d_canon.s[k]);
  double sn = __dmul_rn(t, ps);
  double pc = d_canon.c[10];
#pragma unroll
  for (int k = 9; k >= 0; --k) pc = __fma_rn(pc, u, d_canon.c[k]);
  int quad = (int)(((long long)q) & 3);
  double rs, rc;
  if (quad == 0) {
    rs = sn; rc = pc;
  } else if (quad == 1) {
    rs = pc; rc = -sn;
  } else if (quad == 2) {
    rs = -sn; rc = -pc;
  } else {
    rs = -pc; rc = sn;
  }
  *s = rs;
  *c = rc;
}

// Eq. 4 (Sec. 2.1): the radius of a pair with error radii e1, e2 (arcsec),
// 3 sqrt(e1^2 + e2^2), in the fixed order a = e1 e1, b = e2 e2, t = a + b,
// r = 3 sqrt(t), symmetric in the two errors.
__device__ __forceinline__ double c_pair_radius(double e1, double e2) {
  const double a = __dmul_rn(e1, e1), b = __dmul_rn(e2, e2);
  return __dmul_rn(3.0, __dsqrt_rn(__dadd_rn(a, b)));
}

// Squared-chord threshold 4 sin^2(r/2) of a radius r in arcsec.
__device__ __forceinline__ double c_threshold(double r_arcsec) {
  double s, c;
  c_sincos_deg(__ddiv_rn(r_arcsec, 7200.0), &s, &c);
  return __dmul_rn(4.0, __dmul_rn(s, s));
}

__device__ __forceinline__ double c_norm_ra(double ra) {
  if (ra >= 0.0 && ra < 360.0) return ra;  // fmod would return it unchanged
  double a = fmod(ra, 360.0);
  if (a < 0.0) a = __dadd_rn(a, 360.0);
  if (a >= 360.0) a = __dsub_rn(a, 360.0);
  return a;
}

__device__ __forceinline__ void c_unitvec(double ra, double dec, double* x, double* y, double* z) {
  double sd, cd, sa, ca;
  c_sincos_deg(dec, &sd, &cd);
  c_sincos_deg(ra, &sa, &ca);
  *x = __dmul_rn(cd, ca);
  *y = __dmul_rn(cd, sa);
  *z = sd;
}

__device__ __forceinline__ double c_chord2(double ax, double ay, double az, double bx,
                                           double by, double bz) {
  double dx = __dsub_rn(ax, bx);
  double dy = __dsub_rn(ay, by);
  double dz = __dsub_rn(az, bz);
  double s = __dmul_rn(dx, dx);
  s = __fma_rn(dy, dy, s);
  s = __fma_rn(dz, dz, s);
  return s;
}

__device__ __forceinline__ bool c_valid(double ra, double dec) {
  return isfinite(ra) && isfinite(dec) && dec >= -90.0 && dec <= 90.0;
}

// ---- nested index bit interleave --------------------------------------------
__device__ __forceinline__ uint32_t spread_bits(uint32_t v) {
  v &= 0xFFFFu;
  v = (v | (v << 8)) & 0x00FF00FFu;
  v = (v | (v << 4)) & 0x0F0F0F0Fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}
__device__ __forceinline__ uint32_t gather_bits(uint32_t v) {
  v &= 0x55555555u;
  v = (v | (v >> 1)) & 0x33333333u;
  v = (v | (v >> 2)) & 0x0F0F0F0Fu;
  v = (v | (v >> 4)) & 0x00FF00FFu;
  v = (v | (v >> 8)) & 0x0000FFFFu;
  return v;
}
__device__ __forceinline__ uint32_t fxy_to_nest(int face, int ix, int iy, int order) {
  return ((uint32_t)face << (2 * order)) | spread_bits((uint32_t)ix) |
         (spread_bits((uint32_t)iy) << 1);
}

// Per-declination part of ang2pix: z = sin(dec) and, in the polar caps, the
// cap coordinate sqrt(3(1-|z|)) = sqrt(6) sin((90-|dec|)/2).
struct DecPart {
  double z;
  double cap;  // only meaningful when polar
  bool polar;
};

__device__ __forceinline__ DecPart c_dec_part(double dec) {
  DecPart d;
  double sd, cd;
  c_sincos_deg(dec, &sd, &cd);
  d.z = sd;
  d.polar = !(fabs(sd) <= 2.0 / 3.0);
  d.cap = 0.0;
  if (d.polar) {
    double w = __dsub_rn(90.0, fabs(dec));
    double sw, cw;
    c_sincos_deg(__dmul_rn(0.5, w), &sw, &cw);
    d.cap = __dmul_rn(d_canon.sqrt6, sw);
  }
  return d;
}

// Nested pixel of (ra, dec) given the declination part; ra in [0, 360).
__device__ __forceinline__ uint32_t c_pix(double ra, const DecPart& dp, int order) {
  const double ns = (double)(1u << order);
  const int nsi = 1 << order;
  double tt = __ddiv_rn(ra, 90.0);
  int face, ix, iy;
  if (!dp.polar) {
    double t1 = __dmul_rn(ns, __dadd_rn(0.5, tt));
    double t2 = __dmul_rn(ns, __dmul_rn(dp.z, 0.75));
    int jp = (int)floor(__dsub_rn(t1, t2));
    int jm = (int)floor(__dadd_rn(t1, t2));
    int ifp = jp >> order, ifm = jm >> order;
    face = (ifp == ifm) ? (ifp | 4) : (ifp < ifm ? ifp : ifm + 8);
    ix = jm & (nsi - 1);
    iy = nsi - (jp & (nsi - 1)) - 1;
  } else {
    int ntt = (int)floor(tt);
    if (ntt >= 4) ntt = 3;
    double tp = __dsub_rn(tt, (double)ntt);
    double tmp = __dmul_rn(ns, dp.cap);
    int jp = (int)floor(__dmul_rn(tp, tmp));
    int jm = (int)floor(__dmul_rn(__dsub_rn(1.0, tp), tmp));
    jp = min(jp, nsi - 1);
    jm = min(jm, nsi - 1);
    if (dp.z > 0.0) {
      face = ntt;
      ix = nsi - jm - 1;
      iy = nsi - jp - 1;
    } else {
      face = ntt + 8;
      ix = jp;
      iy = jm;
    }
  }
  return fxy_to_nest(face, ix, iy, order);
}

__device__ __forceinline__ uint32_t c_ang2pix(double ra, double dec, int order) {
  DecPart dp = c_dec_part(dec);
  return c_pix(ra, dp, order);
}

// ---- neighbours -------------------------------------------------------------
// Neighbour of (face, ix, iy) one step in direction (dx, dy); -1 if absent.
__device__ __forceinline__ long long nbr_step(int face, int ix, int iy, int dx, int dy,
                                              int order) {
  const int n = 1 << order;
  int x = ix + dx, y = iy + dy;
  int rx = x < 0 ? 0 : (x >= n ? 2 : 1);
  int ry = y < 0 ? 0 : (y >= n ? 2 : 1);
  int r = ry * 3 + rx;
  int f2 = __ldg(&d_nbr_face[face][r]);
  if (f2 == 255) return -1;
  int x2, y2;
  switch (__ldg(&d_nbr_map[face][r])) {
    case NM_SAME: x2 = x; y2 = y; break;
    case NM_SHIFT:
      x2 = x < 0 ? x + n : (x >= n ? x - n : x);
      y2 = y < 0 ? y + n : (y >= n ? y - n : y);
      break;
    case NM_ROT_N1: x2 = y; y2 = 2 * n - 1 - x; break;
    case NM_ROT_N3: x2 = 2 * n - 1 - y; y2 = x; break;
    case NM_ROT_S3: x2 = y; y2 = -1 - x; break;
    case NM_ROT_S1: x2 = -1 - y; y2 = x; break;
    case NM_AT_00: x2 = 0; y2 = 0; break;
    case NM_AT_NN: x2 = n - 1; y2 = n - 1; break;
    case NM_AT_0N: x2 = 0; y2 = n - 1; break;
    default: x2 = n - 1; y2 = 0; break;
  }
  return (long long)fxy_to_nest(f2, x2, y2, order);
}

__constant__ int8_t d_dirs[8][2] = {{-1, -1}, {-1, 0}, {-1, 1}, {0, 1},
                                    {1, 1},   {1, 0},  {1, -1}, {0, -1}};

__device__ __forceinline__ void nest_to_fxy(uint32_t pix, int order, int* face, int* ix, int* iy) {
  *face = (int)(pix >> (2 * order));
  uint32_t p = order ? (pix & ((1u << (2 * order)) - 1u)) : 0u;
  *ix = (int)gather_bits(p);
  *iy = (int)gather_bits(p >> 1);
}

constexpr uint32_t kNoCell = 0xFFFFFFFFu;

// The cell itself in slot 0 and its neighbours in slots 1..8, kNoCell where a
// neighbour is missing (the 7-neighbour corners) or repeats an earlier slot.
// Slot positions are fixed, so callers index the array with constants and it
// stays in registers.  Cells away from their base face's edges take a fast
// path: +-1 on the interleaved x (even) and y (odd) bit fields of the nested
// index directly, with the carry or borrow run through the other field's
// bits.
__device__ __forceinline__ void cell_neighbourhood9(uint32_t pix, int order, uint32_t out[9]) {
  out[0] = pix;
  if (order > 0) {
    const uint32_t lmask = (1u << (2 * order)) - 1u;
    const uint32_t XM = 0x55555555u & lmask, YM = 0xAAAAAAAAu & lmask;
    const uint32_t fb = pix & ~lmask;
    const uint32_t xm = pix & XM, ym = pix & YM;
    if (xm != 0 && xm != XM && ym != 0 && ym != YM) {
      const uint32_t xs[3] = {(xm - 1u) & XM, xm, ((xm | YM) + 1u) & XM};
      const uint32_t ys[3] = {(ym - 2u) & YM, ym, ((ym | XM) + 2u) & YM};
      int m = 1;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
          if (a != 1 || b != 1) out[m++] = fb | xs[a] | ys[b];
      return;
    }
  }
  int face, ix, iy;
  nest_to_fxy(pix, order, &face, &ix, &iy);
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    long long q = nbr_step(face, ix, iy, d_dirs[d][0], d_dirs[d][1], order);
    uint32_t c = q < 0 ? kNoCell : (uint32_t)q;
#pragma unroll
    for (int e = 0; e <= d; ++e)
      if (out[e] == c) c = kNoCell;
    out[d + 1] = c;
  }
}

// The cell itself followed by its distinct present neighbours; returns count.
__device__ __forceinline__ int cell_neighbourhood(uint32_t pix, int order, uint32_t out[9]) {
  uint32_t nb[9];
  cell_neighbourhood9(pix, order, nb);
  int m = 0;
#pragma unroll
  for (int e = 0; e < 9; ++e)
    if (nb[e] != kNoCell) out[m++] = nb[e];
  return m;
}

// The cells of order (order - d), d >= 1, that cover the neighbourhood (the
// cell and its 8 neighbours) of a cell away from its base face's edges: the
// 3x3 block spans at most two parent columns and two parent rows, so slots
// 0..3 hold (x0,y0), (x1,y0), (x0,y1), (x1,y1), kNoCell where a column or
// row repeats.  Returns false (slots untouched) for a cell on a face edge.
__device__ __forceinline__ bool parent_cover4(uint32_t pix, int order, int d, uint32_t out[4]) {
  if (order <= 0 || d < 1 || d > order) return false;
  const uint32_t lmask = (1u << (2 * order)) - 1u;
  const uint32_t XM = 0x55555555u & lmask, YM = 0xAAAAAAAAu & lmask;
  const uint32_t xm = pix & XM, ym = pix & YM;
  if (xm == 0 || xm == XM || ym == 0 || ym == YM) return false;
  const int sh = 2 * d;
  const uint32_t fb = (pix & ~lmask) >> sh;
  const uint32_t x0 = ((xm - 1u) & XM) >> sh, x1 = (((xm | YM) + 1u) & XM) >> sh;
  const uint32_t y0 = ((ym - 2u) & YM) >> sh, y1 = (((ym | XM) + 2u) & YM) >> sh;
  const bool two_x = x1 != x0, two_y = y1 != y0;
  out[0] = fb | x0 | y0;
  out[1] = two_x ? (fb | x1 | y0) : kNoCell;
  out[2] = two_y ? (fb | x0 | y1) : kNoCell;
  out[3] = two_x && two_y ? (fb | x1 | y1) : kNoCell;
  return true;
}

// ---- quad-direction cells (Algorithm 1) --------------------------------------
__device__ __forceinline__ double wrap_ra(double x) {
  double y = x;
  if (y < 0.0)
    y = __dadd_rn(y, 360.0);
  else if (y >= 360.0)
    y = __dsub_rn(y, 360.0);
  if (y >= 360.0) y = 0.0;
  return y;
}

// Distinct pixels of the source and its four shifted copies, ascending.
// RA shift of the cos(Dec) quad variant: R / cos(dec) with the canonical
// cosine, at most 180 deg (and 180 where the cosine is 0).
__device__ __forceinline__ double c_ra_shift_cos(double R, double dec) {
  double s, c;
  c_sincos_deg(dec, &s, &c);
  c = fabs(c);
  double RA = c > 0.0 ? __ddiv_rn(R, c) : 180.0;
  if (RA > 180.0) RA = 180.0;
  return RA;
}

// cosdec: the RA copies are shifted by c_ra_shift_cos(R, dec) instead of R.
__device__ __forceinline__ int c_quad_cells(double ra, double dec, double R, int order,
                                            uint32_t out[5], bool cosdec = false) {
  const double RA = cosdec ? c_ra_shift_cos(R, dec) : R;
  double dp_ = __dadd_rn(dec, R);
  if (dp_ > 90.0) dp_ = 90.0;
  double dm_ = __dsub_rn(dec, R);
  if (dm_ < -90.0) dm_ = -90.0;
  DecPart d0 = c_dec_part(dec);
  uint32_t p[5];
  p[0] = c_pix(ra, d0, order);
  p[1] = c_pix(wrap_ra(__dadd_rn(ra, RA)), d0, order);
  p[2] = c_pix(wrap_ra(__dsub_rn(ra, RA)), d0, order);
  p[3] = c_ang2pix(ra, dm_, order);
  p[4] = c_ang2pix(ra, dp_, order);
  // sort five values (insertion), then drop repeats
#pragma unroll
  for (int i = 1; i < 5; ++i) {
    uint32_t v = p[i];
    int j = i - 1;
    while (j >= 0 && p[j] > v) {
      p[j + 1] = p[j];
      --j;
    }
    p[j + 1] = v;
  }
  int m = 0;
#pragma unroll
  for (int i = 0; i < 5; ++i)
    if (m == 0 || p[i] != out[m - 1]) out[m++] = p[i];
  return m;
}

}  // namespace hlc
