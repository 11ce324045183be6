// Host-side derivation of the binary64 constants of the canonical arithmetic
// (compiled by the host C++ compiler, which provides binary128 arithmetic).
//
// sin(x deg) and cos(x deg) are evaluated on |x| <= 45 deg as Horner
// polynomials in x^2 whose coefficients are the Taylor terms of sin/cos in
// degrees, (-1)^k (pi/180)^(2k+1)/(2k+1)! and (-1)^k (pi/180)^(2k)/(2k)!, each
// rounded to the nearest double.  pi comes from Stormer's arctangent formula
// and the terms from their recurrence, both in binary128, whose 113-bit
// significand leaves the final rounding to double unaffected.
#include <cstdint>

namespace hlc {

static __float128 atan_recip(int64_t x) {
  // atan(1/x) = sum_k (-1)^k / ((2k+1) x^(2k+1))
  __float128 inv = (__float128)1 / (__float128)x;
  __float128 inv2 = inv * inv;
  __float128 p = inv, acc = 0;
  for (int k = 0; k < 60; ++k) {
    __float128 t = p / (__float128)(2 * k + 1);
    acc = (k % 2 == 0) ? acc + t : acc - t;
    p *= inv2;
  }
  return acc;
}

void derive_trig_coefficients(double sin_c[10], double cos_c[11]) {
  // pi/4 = 44 atan(1/57) + 7 atan(1/239) - 12 atan(1/682) + 24 atan(1/12943)
  __float128 quarter_pi = 44 * atan_recip(57) + 7 * atan_recip(239) -
                          12 * atan_recip(682) + 24 * atan_recip(12943);
  __float128 rad = quarter_pi * 4 / 180;  // radians per degree
  __float128 rad2 = rad * rad;
  __float128 term = rad;  // rad^(2k+1)/(2k+1)! with alternating sign
  for (int k = 0; k < 10; ++k) {
    sin_c[k] = (double)term;
    term = -term * rad2 / (__float128)((2 * k + 2) * (2 * k + 3));
  }
  term = 1;  // rad^(2k)/(2k)! with alternating sign
  for (int k = 0; k < 11; ++k) {
    cos_c[k] = (double)term;
    term = -term * rad2 / (__float128)((2 * k + 1) * (2 * k + 2));
  }
}

}  // namespace hlc
