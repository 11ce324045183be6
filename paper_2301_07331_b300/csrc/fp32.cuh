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

// sin and cos of x degrees (|x| < 1e4), fp32 results.
__device__ __forceinline__ void fp32_sincos_deg(double x, float* s, float* c) {
  float xh = (float)x;
  float xl = (float)(x - (double)xh);          // exact split: x = xh + xl (+ <1e-22)
  float q = rintf(xh * (1.0f / 90.0f));
  float th = fmaf(-90.0f, q, xh);              // exact
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
  int qi = ((int)q) & 3;
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
