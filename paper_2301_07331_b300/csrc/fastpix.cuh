// Guarded FP32 evaluation of the canonical nested ang2pix.
//
// Every discrete decision of the binary64 ang2pix (zone |z| <= 2/3, the two
// floor()s that give the edge-line indices, floor(tt) in the caps) is taken
// from an FP32/FP64-mixed estimate whose distance to the canonical operand is
// bounded; when the estimate lies farther than that bound from the decision
// threshold the decision equals the canonical one, otherwise the source falls
// back to the binary64 path.  The pixel is therefore always the canonical
// pixel; only about 2e-7 * 2^order of the sources take the slow path.
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

__device__ __forceinline__ FastDec f_dec_part(double dec) {
  FastDec d;
  d.z = fp32_sin_deg(dec);
  float za = fabsf(d.z);
  d.ok = fabsf(za - 0.666666667f) > kSinErr + 1e-7f;
  d.polar = za > 0.666666667f;
  d.cap = 0.f;
  if (d.polar) {
    double w = 90.0 - fabs(dec);
    d.cap = 2.44948974f * fp32_sin_deg(0.5 * w);
  }
  return d;
}

// Floor of v when v is farther than e from an integer; false otherwise.
__device__ __forceinline__ bool sure_floor(double v, float e, int* out) {
  double f = floor(v);
  float r = (float)(v - f);
  *out = (int)f;
  return r > e && r < 1.0f - e;
}

// Canonical pixel of (ra, dec), ra in [0, 360), if the FP32 estimate decides
// it with certainty; false when the caller must use the binary64 path.
__device__ __forceinline__ bool f_pix(double ra, const FastDec& d, int order, uint32_t* out) {
  if (!d.ok) return false;
  const double ns = (double)(1u << order);
  const int nsi = 1 << order;
  int face, ix, iy;
  if (!d.polar) {
    double t1 = fma(ra, ns * (1.0 / 90.0), 0.5 * ns);
    double t2 = (double)((float)ns * 0.75f * d.z);
    const float e = (float)(ns * 2e-7) + 1e-9f;
    int jp, jm;
    if (!sure_floor(t1 - t2, e, &jp)) return false;
    if (!sure_floor(t1 + t2, e, &jm)) return false;
    int ifp = jp >> order, ifm = jm >> order;
    face = (ifp == ifm) ? (ifp | 4) : (ifp < ifm ? ifp : ifm + 8);
    ix = jm & (nsi - 1);
    iy = nsi - (jp & (nsi - 1)) - 1;
  } else {
    double tt = ra * (1.0 / 90.0);
    int ntt;
    if (!sure_floor(tt, 1e-9f, &ntt)) return false;
    if (ntt >= 4) ntt = 3;
    double tp = tt - (double)ntt;
    double tmp = (double)((float)ns * d.cap);
    const float e = (float)(ns * 2.5e-7) + 1e-9f;
    int jp, jm;
    if (!sure_floor(tp * tmp, e, &jp)) return false;
    if (!sure_floor((1.0 - tp) * tmp, e, &jm)) return false;
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

__device__ __forceinline__ uint32_t g_ang2pix(double ra, double dec, int order) {
  uint32_t p;
  FastDec fd = f_dec_part(dec);
  if (f_pix(ra, fd, order, &p)) return p;
  return c_ang2pix(ra, dec, order);
}

// Quad-direction cells (Algorithm 1) through the guarded pixel function.
__device__ __forceinline__ int g_quad_cells(double ra, double dec, double R, int order,
                                            uint32_t out[5]) {
  double dp_ = dec + R;
  if (dp_ > 90.0) dp_ = 90.0;
  double dm_ = dec - R;
  if (dm_ < -90.0) dm_ = -90.0;
  FastDec f0 = f_dec_part(dec);
  uint32_t p[5];
  double ras[3] = {ra, wrap_ra(__dadd_rn(ra, R)), wrap_ra(__dsub_rn(ra, R))};
  bool have_c0 = false;
  DecPart c0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (!f_pix(ras[i], f0, order, &p[i])) {
      if (!have_c0) {
        c0 = c_dec_part(dec);
        have_c0 = true;
      }
      p[i] = c_pix(ras[i], c0, order);
    }
  }
  p[3] = g_ang2pix(ra, dm_, order);
  p[4] = g_ang2pix(ra, dp_, order);
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
