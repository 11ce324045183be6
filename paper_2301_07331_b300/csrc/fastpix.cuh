// Guarded FP32 evaluation of the canonical nested ang2pix.
//
// Every discrete decision of the binary64 ang2pix (zone |z| <= 2/3, the two
// floor()s that give the edge-line indices, floor(tt) in the caps) is taken
// from an FP32 / float-float estimate whose distance to the canonical operand
// is bounded; when the estimate lies farther than that bound from the
// decision threshold the decision equals the canonical one, otherwise the
// source falls back to the binary64 path.  The pixel is therefore always the
// canonical pixel.  The fast path issues no FP64 instruction (the double
// inputs are split into float pairs with integer operations): on B300 the
// FP64 pipe runs at a small fraction of the FP32 rate.  About 8e-7 * 2^order
// of the sources take the slow path.
#pragma once

#include "canon.cuh"
#include "fp32.cuh"

namespace hlc {

struct FastDec {
  float z;    // sin(dec), |error| <= kSinErr
  float cap;  // sqrt(6) sin((90-|dec|)/2), relative error <= 2e-7 (caps only)
  bool polar;
  bool ok;    // zone decided with certainty
};

__device__ __forceinline__ FastDec f_dec_part(f2 dec) {
  FastDec d;
  float c_unused;
  fp32_sincos_deg2(dec.hi, dec.lo, &d.z, &c_unused);
  float za = fabsf(d.z);
  d.ok = fabsf(za - 0.666666667f) > kSinErr + 1e-7f;
  d.polar = za > 0.666666667f;
  d.cap = 0.f;
  if (d.polar) {
    // (90 - |dec|) / 2 as a float pair; 90 - |hi| is exact or within 2^-24
    float ah = fabsf(dec.hi), al = dec.hi < 0.f ? -dec.lo : dec.lo;
    f2 w = two_sum(90.0f, -ah);
    w.lo -= al;
    float sw, cw;
    fp32_sincos_deg2(0.5f * w.hi, 0.5f * w.lo, &sw, &cw);
    d.cap = 2.44948974f * sw;
  }
  return d;
}

// floor(v) as an int when v lies farther than e from an integer.
// (0 <= v < 2^23.)
__device__ __forceinline__ bool sure_floorf(float v, float e, int* out) {
  float f = floor_pos(v);
  float r = v - f;
  *out = ifloor_pos(v);
  return r > e && r < 1.0f - e;
}

struct PixConst {
  float kh, kl;  // 2^order / 90 as a float pair
  float inv90h, inv90l;
};

__host__ __device__ inline PixConst pix_const(int order) {
  PixConst c;
  double k = (double)(1u << order) / 90.0;
  c.kh = (float)k;
  c.kl = (float)(k - (double)c.kh);
  c.inv90h = (float)(1.0 / 90.0);
  c.inv90l = (float)(1.0 / 90.0 - (double)c.inv90h);
  return c;
}

// Canonical pixel of (ra, dec), ra in [0, 360) given as a float pair, if the
// estimate decides it with certainty; false when the caller must use the
// binary64 path.
__device__ __forceinline__ bool f_pix(f2 ra, const FastDec& d, int order, const PixConst& K,
                                      uint32_t* out) {
  if (!d.ok) return false;
  const float ns = pow2f(order);
  const int nsi = 1 << order;
  int face, ix, iy;
  if (!d.polar) {
    // ns (0.5 + ra/90) -/+ ns 0.75 z, split into integer and fraction
    f2 t = f2_mul(ra, f2{K.kh, K.kl});
    float ih = floor_pos(t.hi);
    int iih = ifloor_pos(t.hi);
    float a = (t.hi - ih) + t.lo;  // fraction of ns ra / 90
    float t2 = ns * 0.75f * d.z;
    const float e = ns * 4e-7f + 4e-7f;
    int f1, f2i;
    if (!sure_floorf(a + (0.5f * ns - t2), e, &f1)) return false;
    if (!sure_floorf(a + (0.5f * ns + t2), e, &f2i)) return false;
    int jp = iih + f1, jm = iih + f2i;
    int ifp = jp >> order, ifm = jm >> order;
    face = (ifp == ifm) ? (ifp | 4) : (ifp < ifm ? ifp : ifm + 8);
    ix = jm & (nsi - 1);
    iy = nsi - (jp & (nsi - 1)) - 1;
  } else {
    f2 tt = f2_mul(ra, f2{K.inv90h, K.inv90l});
    float fh = floor_pos(tt.hi);
    float fr = (tt.hi - fh) + tt.lo;
    if (!(fr > 1e-6f && fr < 1.0f - 1e-6f)) return false;
    int ntt = ifloor_pos(tt.hi);
    float tp = fr;
    if (ntt >= 4) {
      ntt = 3;
      tp = fr + (fh - 3.0f);
    }
    float tmp = ns * d.cap;
    const float e = ns * 6e-7f + 4e-7f;
    int jp, jm;
    if (!sure_floorf(tp * tmp, e, &jp)) return false;
    if (!sure_floorf((1.0f - tp) * tmp, e, &jm)) return false;
    jp = min(jp, nsi - 1);
    jm = min(jm, nsi - 1);
    if (d.z > 0.f) {
      face = ntt;
      ix = nsi - jm - 1;
      iy = nsi - jp - 1;
    } else {
      face = ntt + 8;
      ix = jp;
      iy = jm;
    }
  }
  *out = fxy_to_nest(face, ix, iy, order);
  return true;
}

// ---- float-float tier for the positions the FP32 estimate left undecided ----
// The same decisions as c_pix, taken from float-float operands: the angles
// split exactly, sin from f2_sin_deg (about 1e-14), the products and sums
// in float-float, so each operand lies within about 1e-13 (ns + 1) of its
// exact value, and the binary64 path's own operands within a few 1e-15
// (ns + 1) of theirs.  A decision is taken only when the operand lies
// farther than kFfMargin (ns + 1) from the threshold (the integer of a
// floor, 2/3 for the zone), several hundred times both errors together, so a
// decided pixel is the canonical one; false leaves the binary64 path to it.
constexpr float kFfMargin = 1e-10f;

// floor(v) when v is farther than e from an integer (v >= -1; the remainder
// r is exact but for its own rounding, ulp(r)/2 <= 6e-8, which e covers).
__device__ __forceinline__ bool ff_floor(f2 v, float e, int* out) {
  const float fl = floorf(v.hi);
  const float r = (v.hi - fl) + v.lo;
  *out = (int)fl;
  return r > e && r < 1.0f - e;
}

__device__ __forceinline__ bool ff_pix(double ra, double dec, int order, uint32_t* out) {
  const PixConst K = pix_const(order);
  const f2 a = split_f64(ra), d = split_f64(dec);
  const f2 z = f2_sin_deg(d);
  const f2 az = z.hi < 0.f ? f2{-z.hi, -z.lo} : z;
  constexpr f2 two3 = f2_of(2.0 / 3.0);
  const f2 dz = f2_add(az, f2{-two3.hi, -two3.lo});
  if (fabsf(dz.hi) <= 1e-12f) return false;  // on the zone boundary
  const bool polar = dz.hi > 0.f;
  const float ns = pow2f(order);
  const int nsi = 1 << order;
  const float e = kFfMargin * (ns + 1.0f) + 2.4e-7f;
  int face, ix, iy;
  if (!polar) {
    // ns (0.5 + ra/90) -/+ 0.75 ns z as floor(ns ra/90) + (fraction + 0.5 ns -/+ 0.75 ns z)
    const f2 t = f2_mul(a, f2{K.kh, K.kl});
    const float ih = floor_pos(t.hi);
    const int iih = ifloor_pos(t.hi);
    const f2 fa = two_sum(t.hi - ih, t.lo);  // (t.hi - ih exact)
    const f2 t2 = f2_mulf(z, 0.75f * ns);
    const f2 base = f2_add(fa, f2{0.5f * ns, 0.f});
    int f1, f2i;
    if (!ff_floor(f2_add(base, f2{-t2.hi, -t2.lo}), e, &f1)) return false;
    if (!ff_floor(f2_add(base, t2), e, &f2i)) return false;
    const int jp = iih + f1, jm = iih + f2i;
    const int ifp = jp >> order, ifm = jm >> order;
    face = (ifp == ifm) ? (ifp | 4) : (ifp < ifm ? ifp : ifm + 8);
    ix = jm & (nsi - 1);
    iy = nsi - (jp & (nsi - 1)) - 1;
  } else {
    const f2 tt = f2_mul(a, f2{K.inv90h, K.inv90l});
    int ntt;
    if (!ff_floor(tt, e, &ntt)) return false;  // RA near a multiple of 90
    const float fh = (float)ntt;
    const f2 fr = two_sum(tt.hi - fh, tt.lo);
    f2 tp = fr;
    if (ntt >= 4) {
      ntt = 3;
      tp = f2_add(fr, f2{fh - 3.0f, 0.f});
    }
    // cap = sqrt(6) sin((90 - |dec|) / 2), in float-float
    const float ah = fabsf(d.hi), al = d.hi < 0.f ? -d.lo : d.lo;
    f2 w = two_sum(90.0f, -ah);
    w = fast_two_sum(w.hi, w.lo - al);
    w = f2{0.5f * w.hi, 0.5f * w.lo};
    constexpr f2 sq6 = f2_of(2.4494897427831780982);  // sqrt(6)
    const f2 cap = f2_mul(f2_sin_small(f2_mul(w, kPiOver180)), sq6);
    const f2 tmp = {cap.hi * ns, cap.lo * ns};  // (exact: ns is a power of two)
    int jp, jm;
    if (!ff_floor(f2_mul(tp, tmp), e, &jp)) return false;
    if (!ff_floor(f2_mul(f2_add(f2{1.0f, 0.f}, f2{-tp.hi, -tp.lo}), tmp), e, &jm)) return false;
    jp = min(jp, nsi - 1);
    jm = min(jm, nsi - 1);
    if (z.hi > 0.f) {
      face = ntt;
      ix = nsi - jm - 1;
      iy = nsi - jp - 1;
    } else {
      face = ntt + 8;
      ix = jp;
      iy = jm;
    }
  }
  *out = fxy_to_nest(face, ix, iy, order);
  return true;
}

// The canonical pixel of (ra, dec) (ra in [0, 360)) for a position the FP32
// estimate left undecided: the float-float tier, else binary64.
__device__ __forceinline__ uint32_t ff_or_c_ang2pix(double ra, double dec, int order) {
  uint32_t p;
  if (ff_pix(ra, dec, order, &p)) return p;
  return c_ang2pix(ra, dec, order);
}

// ra already normalised to [0, 360).
__device__ __forceinline__ uint32_t g_ang2pix(double ra, double dec, int order,
                                              const PixConst& K) {
  uint32_t p;
  FastDec fd = f_dec_part(split_f64(dec));
  if (f_pix(split_f64(ra), fd, order, K, &p)) return p;
  return c_ang2pix(ra, dec, order);
}

// Quad-direction positions (Algorithm 1) through the guarded pixel function:
// the source and its copies at ra + R, ra - R (wrapped), dec - R, dec + R
// (clamped to the poles), in that order.  The shifted coordinates are formed
// in float-float: within about 2e-11 deg of the binary64 statement's values,
// far inside the guard margins, so a decided pixel is the canonical one;
// a shifted RA whose leading float is not in [0, 360) (a wrap at the RA = 0
// face boundary) is left undecided.  Writes the pixel of every decided
// position to p[0..4] and returns the mask of the undecided ones.
// (Ra: the RA shift, Rd itself or the cos(Dec) variant's binary64 shift
// split into float-float.)
__device__ __forceinline__ unsigned g_quad_pos(double ra, double dec, f2 Rd, f2 Ra, int order,
                                               const PixConst& K, uint32_t p[5]) {
  const f2 r0 = split_f64(ra), d0 = split_f64(dec);
  const f2 Rn = {-Rd.hi, -Rd.lo};
  const f2 Ran = {-Ra.hi, -Ra.lo};
  f2 dp = f2_add(d0, Rd);
  if (dp.hi > 90.f || (dp.hi == 90.f && dp.lo > 0.f)) dp = f2{90.f, 0.f};
  f2 dm = f2_add(d0, Rn);
  if (dm.hi < -90.f || (dm.hi == -90.f && dm.lo < 0.f)) dm = f2{-90.f, 0.f};
  f2 rp = f2_add(r0, Ra);
  if (rp.hi > 360.f || (rp.hi == 360.f && rp.lo >= 0.f)) rp = f2_add(rp, f2{-360.f, 0.f});
  f2 rm = f2_add(r0, Ran);
  if (rm.hi < 0.f || (rm.hi == 0.f && rm.lo < 0.f)) rm = f2_add(rm, f2{360.f, 0.f});
  const FastDec f0 = f_dec_part(d0), fm = f_dec_part(dm), fp = f_dec_part(dp);
  unsigned und = 0;
  if (!f_pix(r0, f0, order, K, &p[0])) und |= 1u;
  if (!(rp.hi >= 0.f && rp.hi < 360.f) || !f_pix(rp, f0, order, K, &p[1])) und |= 2u;
  if (!(rm.hi >= 0.f && rm.hi < 360.f) || !f_pix(rm, f0, order, K, &p[2])) und |= 4u;
  if (!f_pix(r0, fm, order, K, &p[3])) und |= 8u;
  if (!f_pix(r0, fp, order, K, &p[4])) und |= 16u;
  return und;
}

// Distinct values of p[0..4], ascending, into out; returns their number.
__device__ __forceinline__ int quad_sort_unique(uint32_t p[5], uint32_t out[5]) {
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
