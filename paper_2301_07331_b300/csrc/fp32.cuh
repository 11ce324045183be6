// FP32 unit vectors with a stated error bound, for the guard-band form.
//
// Each angle (float64 degrees) is split exactly into a float hi/lo pair,
// reduced to [-45, 45] deg in float arithmetic (exact: the subtraction of a
// multiple of 90 is exact by Sterbenz' lemma), converted to radians as a
// float-float pair, and its sine and cosine are Taylor polynomials (degree 9
// and 10, truncation below 2e-9 on |x| <= pi/4) corrected to first order for
// the low part.  Each factor is then within ~1.5 ulp of its true value and
// each product component within kUnitVecErr of the true unit vector.
#pragma once

#include "common.cuh"

namespace hlc {

// Bound on |component error| of fp32_unitvec against the exact unit vector.
// Each sine/cosine factor is within ~5e-8 of the truth (polynomial roundings
// below one ulp of 2^-24, truncation below 2e-9, the float-float argument
// within 1e-15); a product adds half an ulp (3e-8): about 1.3e-7 per
// component; stated with margin.
constexpr double kUnitVecErr = 1.6e-7;
// Bound on |sin(dec) - fp32 sine| used by the guarded ang2pix.
constexpr float kSinErr = 1.2e-7f;

// ---- float-float helpers (error-free transformations on the FP32 pipe) ----
struct f2 {
  float hi, lo;
};

__device__ __forceinline__ f2 two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  f2 s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ f2 f2_mulf(f2 a, float b) {
  float p = a.hi * b;
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  return fast_two_sum(p, e);
}

// x = hi + lo exactly up to 2^-53 |x| (lo rounded), with integer operations
// only: hi keeps the top 24 significand bits, lo the next 29 (rounded to 24).
// |x| < 2^-70 (and 0) gives (0, 0); x must be finite.
__device__ __forceinline__ f2 split_f64(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  int e = (int)((b >> 52) & 0x7FFu) - 1023;
  if (e < -70) return {0.f, 0.f};
  unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;  // 53 bits
  unsigned mh = (unsigned)(m >> 29);                                      // 24 bits
  unsigned ml = (unsigned)(m & 0x1FFFFFFFu);                              // 29 bits
  float hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (mh & 0x7FFFFFu));
  float lo = 0.f;
  if (ml) {
    int lz = __clz(ml);        // >= 3
    int top = 31 - lz;         // position of the leading one
    unsigned mant = top > 23 ? (ml >> (top - 23)) : (ml << (23 - top));
    int ex = e - 52 + top;     // exponent of the leading one
    lo = __uint_as_float(sign | ((unsigned)(ex + 127) << 23) | (mant & 0x7FFFFFu));
  }
  return {hi, lo};
}

// Integer-valued rounding on the FP32 pipe (conversion instructions share
// the slow FP64 unit on B300, so they are avoided on the fast paths).
// floor of 0 <= v < 2^23, as float and as int:
__device__ __forceinline__ float floor_pos(float v) {
  return __fadd_rd(v, 8388608.0f) - 8388608.0f;
}
__device__ __forceinline__ int ifloor_pos(float v) {
  return __float_as_int(__fadd_rd(v, 8388608.0f)) - 0x4B000000;
}
// nearest integer of |v| < 2^22, as float and int (ties to even)
__device__ __forceinline__ float round_near(float v, int* iv) {
  float r = __fadd_rn(v, 12582912.0f);  // 1.5 * 2^23
  *iv = __float_as_int(r) - 0x4B400000;
  return r - 12582912.0f;
}
__device__ __forceinline__ float pow2f(int e) {  // 2^e, -126 <= e <= 127
  return __int_as_float((e + 127) << 23);
}

// Bit-level checks on binary64 values (no FP64 instructions).
__device__ __forceinline__ bool bits_finite(double x) {
  return ((unsigned long long)__double_as_longlong(x) & 0x7FF0000000000000ull) !=
         0x7FF0000000000000ull;
}
__device__ __forceinline__ bool bits_abs_le(double x, double lim) {  // |x| <= lim (finite)
  return ((unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull) <=
         (unsigned long long)__double_as_longlong(lim);
}
__device__ __forceinline__ bool bits_in_ra_range(double x) {  // 0 <= x < 360 (or -0)
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return b < 0x4076800000000000ull || b == 0x8000000000000000ull;  // 360.0 = 0x4076800000000000
}

__device__ __forceinline__ void fp32_sincos_reduced(float p, float e, float* s, float* c) {
  // p + e radians, |p| <= pi/4 + tiny, |e| <= 2^-24 |p|
  float p2 = p * p;
  float ps = fmaf(p2, 2.75573192e-6f, -1.98412698e-4f);  // 1/9!, -1/7!
  ps = fmaf(p2, ps, 8.33333333e-3f);                      // 1/5!
  ps = fmaf(p2, ps, -1.66666667e-1f);                     // -1/3!
  float sn = fmaf(p * p2, ps, p);
  float pc = fmaf(p2, -2.75573192e-7f, 2.48015873e-5f);   // -1/10!, 1/8!
  pc = fmaf(p2, pc, -1.38888889e-3f);                     // -1/6!
  pc = fmaf(p2, pc, 4.16666667e-2f);                      // 1/4!
  pc = fmaf(p2, pc, -0.5f);
  float cs = fmaf(p2, pc, 1.0f);
  *s = fmaf(cs, e, sn);
  *c = fmaf(-sn, e, cs);
}

// sin and cos of (xh + xl) degrees, |x| < 1e4, fp32 results.
__device__ __forceinline__ void fp32_sincos_deg2(float xh, float xl, float* s, float* c) {
  int qi;
  float q = round_near(xh * (1.0f / 90.0f), &qi);
  float th = fmaf(-90.0f, q, xh);              // exact (Sterbenz)
  // radians as a float-float pair: (th + xl) * (R_hi + R_lo)
  const float R_hi = 1.745329238e-2f;          // float nearest pi/180
  const float R_lo = 1.351996015e-10f;         // pi/180 - R_hi
  float p = th * R_hi;
  float e = fmaf(th, R_hi, -p);
  e = fmaf(th, R_lo, e);
  e = fmaf(xl, R_hi, e);
  float ps = p + e;
  float pe = e - (ps - p);
  float sn, cs;
  fp32_sincos_reduced(ps, pe, &sn, &cs);
  qi &= 3;
  if (qi == 0) {
    *s = sn; *c = cs;
  } else if (qi == 1) {
    *s = cs; *c = -sn;
  } else if (qi == 2) {
    *s = -sn; *c = -cs;
  } else {
    *s = -cs; *c = sn;
  }
}

__device__ __forceinline__ void fp32_sincos_deg(double x, float* s, float* c) {
  f2 v = split_f64(x);
  fp32_sincos_deg2(v.hi, v.lo, s, c);
}

__device__ __forceinline__ float fp32_sin_deg(double x) {
  float s, c;
  fp32_sincos_deg(x, &s, &c);
  return s;
}

__device__ __forceinline__ float4 fp32_unitvec(double ra, double dec) {
  float sd, cd, sa, ca;
  fp32_sincos_deg(dec, &sd, &cd);
  fp32_sincos_deg(ra, &sa, &ca);
  return make_float4(cd * ca, cd * sa, sd, 0.0f);
}

// sin and cos of a reduced float-float angle p (radians, |p| <= pi/4 + tiny)
// to about 2e-8 relative: the leading Taylor terms are summed in float-float,
// only the small tail is evaluated in float.
__device__ __forceinline__ void f2_sincos_reduced(f2 p, f2* s, f2* c) {
  float x = p.hi;
  float x2 = x * x;
  float ts = fmaf(x2, 2.75573192e-6f, -1.98412698e-4f);
  ts = fmaf(x2, ts, 8.33333333e-3f);
  ts = fmaf(x2, ts, -1.66666667e-1f);
  float tail_s = x * x2 * ts;                       // sin - x
  *s = f2_add(p, f2{tail_s, 0.f});
  f2 h = f2_mul(p, p);                              // p^2 in float-float
  float tc = fmaf(x2, -2.75573192e-7f, 2.48015873e-5f);
  tc = fmaf(x2, tc, -1.38888889e-3f);
  tc = fmaf(x2, tc, 4.16666667e-2f);
  float tail_c = x2 * x2 * tc;                      // cos - 1 + p^2/2
  f2 c0 = f2_add(f2{1.0f, 0.f}, f2{-0.5f * h.hi, -0.5f * h.lo});
  *c = f2_add(c0, f2{tail_c, 0.f});
}

// ---- full float-float sine and cosine (about 1e-14 absolute) ----
// The float pair nearest a double constant (evaluated at compile time).
__host__ __device__ constexpr f2 f2_of(double v) {
  return f2{(float)v, (float)(v - (double)(float)v)};
}
constexpr double kFact[18] = {1.0, 1.0, 2.0, 6.0, 24.0, 120.0, 720.0, 5040.0, 40320.0,
                              362880.0, 3628800.0, 39916800.0, 479001600.0, 6227020800.0,
                              87178291200.0, 1307674368000.0, 20922789888000.0,
                              355687428096000.0};
constexpr f2 kPiOver180 = f2_of(0.017453292519943295769);  // pi / 180

// sin p and cos p of a float-float angle |p| <= pi/4 (+ a little): Taylor
// series, the terms to p^9 (p^8) summed in float-float (Horner in u = p^2),
// the rest (below 2e-9 relative) in float.
__device__ __forceinline__ f2 f2_sin_small(f2 p) {
  const f2 u = f2_mul(p, p);
  const float uh = u.hi;
  constexpr float c17 = (float)(1.0 / kFact[17]), c15 = (float)(-1.0 / kFact[15]),
                  c13 = (float)(1.0 / kFact[13]), c11 = (float)(-1.0 / kFact[11]);
  float tail = fmaf(uh, c17, c15);
  tail = fmaf(uh, tail, c13);
  tail = fmaf(uh, tail, c11);
  f2 acc = f2_add(f2_of(1.0 / kFact[9]), f2_mulf(u, tail));
  acc = f2_add(f2_of(-1.0 / kFact[7]), f2_mul(u, acc));
  acc = f2_add(f2_of(1.0 / kFact[5]), f2_mul(u, acc));
  acc = f2_add(f2_of(-1.0 / kFact[3]), f2_mul(u, acc));
  return f2_add(p, f2_mul(p, f2_mul(u, acc)));
}
__device__ __forceinline__ f2 f2_cos_small(f2 p) {
  const f2 u = f2_mul(p, p);
  const float uh = u.hi;
  constexpr float c16 = (float)(1.0 / kFact[16]), c14 = (float)(-1.0 / kFact[14]),
                  c12 = (float)(1.0 / kFact[12]), c10 = (float)(-1.0 / kFact[10]);
  float tail = fmaf(uh, c16, c14);
  tail = fmaf(uh, tail, c12);
  tail = fmaf(uh, tail, c10);
  f2 acc = f2_add(f2_of(1.0 / kFact[8]), f2_mulf(u, tail));
  acc = f2_add(f2_of(-1.0 / kFact[6]), f2_mul(u, acc));
  acc = f2_add(f2_of(1.0 / kFact[4]), f2_mul(u, acc));
  acc = f2_add(f2_of(-1.0 / kFact[2]), f2_mul(u, acc));
  return f2_add(f2{1.0f, 0.f}, f2_mul(u, acc));
}

// sin of a float-float number of degrees, |x| <= 90 (+ a little): reduced
// by the nearest multiple of 90 (exact), converted to radians in
// float-float, then the sine or cosine series.
__device__ __forceinline__ f2 f2_sin_deg(f2 x) {
  int qi;
  const float q = round_near(x.hi * (1.0f / 90.0f), &qi);
  const f2 t = two_sum(fmaf(-90.0f, q, x.hi), x.lo);  // (the first term exact)
  const f2 p = f2_mul(t, kPiOver180);
  if (qi == 0) return f2_sin_small(p);
  const f2 c = f2_cos_small(p);
  return qi > 0 ? c : f2{-c.hi, -c.lo};
}

// cos of an angle given as a float-float number of degrees, |x| <= 90,
// to about 3e-8 relative (evaluated as sin(90 - |x|)).
__device__ __forceinline__ f2 f2_cos_deg(f2 x) {
  float ah = fabsf(x.hi), al = x.hi < 0.f ? -x.lo : x.lo;
  f2 w = two_sum(90.0f, -ah);  // 90 - |x| in degrees
  w = fast_two_sum(w.hi, w.lo - al);
  bool big = w.hi > 45.0f;
  if (big) w = fast_two_sum(w.hi - 90.0f, w.lo);  // exact (Sterbenz)
  const f2 R = {1.745329238e-2f, 1.351996015e-10f};
  f2 p = f2_mul(w, R);
  f2 sn, cs;
  f2_sincos_reduced(p, &sn, &cs);
  return big ? cs : sn;
}

// Separation of two nearby sources (ra in [0, 360)) in float-float arithmetic
// on the FP32 pipe: haversine form with the angle differences formed exactly
// from the split binary64 inputs and cos(Dec) to ~3e-8 relative, so the
// relative error of the result is below 1e-7 (5e-7 arcsec at 5 arcsec).
// Returns a negative value when the pair is not "nearby" (differences above
// 20 arcsec), in which case the caller uses the binary64 unit vectors.
__device__ __forceinline__ double sep_arcsec_f2(double ra1, double dec1, double ra2,
                                                double dec2) {
  f2 a1 = split_f64(ra1), d1 = split_f64(dec1), a2 = split_f64(ra2), d2 = split_f64(dec2);
  f2 dd = f2_add(d2, f2{-d1.hi, -d1.lo});
  f2 da = f2_add(a2, f2{-a1.hi, -a1.lo});
  if (da.hi > 180.f) da = f2_add(da, f2{-360.f, 0.f});
  if (da.hi < -180.f) da = f2_add(da, f2{360.f, 0.f});
  const float lim = 20.0f / 3600.0f;
  if (fabsf(dd.hi) > lim || fabsf(da.hi) > lim) return -1.0;
  f2 c1 = f2_cos_deg(d1), c2 = f2_cos_deg(d2);
  f2 K = f2_mul(c1, c2);
  const f2 HR = {8.726646192e-3f, 6.759980075e-11f};  // pi/360 as a float pair
  f2 x = f2_mul(dd, HR), y = f2_mul(da, HR);         // half differences, radians
  // sin of the half differences: x - x^3/6 (x <= 5e-5 rad: next term < 1e-19)
  f2 sx = f2_add(x, f2{-x.hi * x.hi * x.hi * (1.0f / 6.0f), 0.f});
  f2 sy = f2_add(y, f2{-y.hi * y.hi * y.hi * (1.0f / 6.0f), 0.f});
  f2 hav = f2_add(f2_mul(sx, sx), f2_mul(K, f2_mul(sy, sy)));
  // v = sqrt(hav) with one float-float Newton correction
  float v0 = sqrtf(hav.hi);
  f2 v = {v0, 0.f};
  if (v0 > 0.f) {
    f2 sq = f2_mul(v, v);
    f2 rem = f2_add(hav, f2{-sq.hi, -sq.lo});
    v = fast_two_sum(v0, rem.hi / (2.0f * v0));
  }
  // asin(v) = v + v^3/6 (+ 3v^5/40 < 1e-22 relative here)
  f2 as = f2_add(v, f2{v.hi * v.hi * v.hi * (1.0f / 6.0f), 0.f});
  const f2 SC = {412529.625f, -1.2505806983e-2f};  // 2 * 648000 / pi as a float pair
  f2 r = f2_mul(as, SC);
  return (double)r.hi + (double)r.lo;
}

// The guard-band decision sep(a, b) <= r taken from sep_arcsec_f2 where it is
// certain: +1 inside, -1 outside, 0 when the binary64 test must decide.
// Undecided: a pair that is not "nearby", a source within 0.1 deg of a pole
// (where cos(Dec) from the split inputs loses relative accuracy), or an
// estimate within m of r, m = kSepRel r + kSepAbs.  For |Dec| <= 89.9 deg
// the estimate is within about 1e-7 relative plus 2e-8 arcsec of the exact
// separation (input splits: 2^-47 relative per coordinate; float-float
// operations near 2^-44; cos(Dec) 3e-8 relative), and the binary64 squared
// chord is within 1e-10 relative of the exact one, so outside m both tests
// give the same answer.
constexpr double kSepRel = 1e-6;
constexpr double kSepAbs = 1e-7;  // arcsec

__device__ __forceinline__ int f2_sep_decide(double ra1, double dec1, double ra2, double dec2,
                                             double r_lo, double r_hi) {
  if (!bits_abs_le(dec1, 89.9) || !bits_abs_le(dec2, 89.9)) return 0;
  const double sv = sep_arcsec_f2(ra1, dec1, ra2, dec2);
  if (sv < 0.0) return 0;
  return sv < r_lo ? 1 : (sv > r_hi ? -1 : 0);
}

// [r_lo, r_hi]: the separations (arcsec) left to the binary64 test.
inline void f2_sep_window(double r_arcsec, double* r_lo, double* r_hi) {
  const double m = kSepRel * r_arcsec + kSepAbs;
  *r_lo = r_arcsec - m;
  *r_hi = r_arcsec + m;
}

// Guard band for an FP32 squared chord computed from such vectors as
// d = a - b (3 float subtractions), s = d.x^2 (+) fma chain.  Returns the
// half-width G such that |s_fp32 - s_exact| <= G whenever s_exact <= C (1+).
inline double fp32_guard_band(double C, double comp_err) {
  const double u = 1.0 / 16777216.0;  // 2^-24
  double D = sqrt(C) * 1.01;           // chord length of interest
  double delta = 2.0 * comp_err * (1.0 + u) + D * u;  // per-component error
  double err = 2.0 * sqrt(3.0) * delta * D + 3.0 * delta * delta;
  err += 4.0 * u * (C + err);  // roundings of the sum of squares
  return 1.5 * err;            // margin factor 1.5
}

}  // namespace hlc
