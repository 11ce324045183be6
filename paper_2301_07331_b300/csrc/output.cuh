// Output rows of the match: ids and separations of each matched pair, then
// the rows in ascending (id_a, id_b) order.
//
// Ordering: the rows are distributed into 2^b buckets by the b bits of id_a
// just below its highest varying bit (a counting scatter, four to eight rows
// per bucket on average), then every bucket is sorted on (id_a, id_b,
// separation bits): by rank counting (a thread per row) when small, by a
// CTA's bitonic network in shared memory when larger.  When a bucket would not fit in shared memory (one id
// matched thousands of times, or all ids equal) the caller falls back to two
// stable LSD radix sorts (by id_b, then by id_a).
#pragma once

#include "canon.cuh"
#include "common.cuh"
#include "fp32.cuh"
#include "match.cuh"

namespace hlc {

constexpr int kBucketCap = 2048;
constexpr int kBucketMid = 256;  // buckets up to this many rows: the small-array sort
constexpr int kBucketThreads = 128;

__device__ __forceinline__ double sep_arcsec_from_chord2(double s) {
  double h = sqrt(s) * 0.5;
  if (h > 1.0) h = 1.0;
  return 2.0 * asin(h) * (648000.0 / 3.141592653589793238462643);
}

// Separation from the original coordinates by the haversine form
// hav(d) = sin^2(dDec/2) + cos(Dec_a) cos(Dec_b) sin^2(dRA/2), with
// cos(Dec_a) cos(Dec_b) = cos^2(mean Dec) - sin^2(dDec/2): one binary64
// cosine per row; short series for the small angles.  Rows whose RA or Dec
// difference exceeds 1 degree (near the poles) use the unit vectors.
__device__ __forceinline__ double sep_arcsec_haversine(double ra1, double dec1, double ra2,
                                                       double dec2) {
  double dd = dec2 - dec1;
  double da = ra2 - ra1;
  if (da > 180.0) da -= 360.0;
  if (da < -180.0) da += 360.0;
  if (fabs(da) > 1.0 || fabs(dd) > 1.0) {
    double ax, ay, az, bx, by, bz;
    c_unitvec(ra1, dec1, &ax, &ay, &az);
    c_unitvec(ra2, dec2, &bx, &by, &bz);
    return sep_arcsec_from_chord2(c_chord2(ax, ay, az, bx, by, bz));
  }
  double sm, cm;
  c_sincos_deg(0.5 * (dec1 + dec2), &sm, &cm);
  const double half_rad = 3.141592653589793238462643 / 360.0;
  double x = dd * half_rad, y = da * half_rad;
  double x2 = x * x, y2 = y * y;
  double sx = x * (1.0 - x2 * (1.0 / 6.0 - x2 * (1.0 / 120.0)));
  double sy = y * (1.0 - y2 * (1.0 / 6.0 - y2 * (1.0 / 120.0)));
  double K = cm * cm - sx * sx;
  double hav = fma(K, sy * sy, sx * sx);
  double v = sqrt(hav);
  double v2 = v * v;
  double as = v * (1.0 + v2 * (1.0 / 6.0 + v2 * (3.0 / 40.0)));
  return 2.0 * as * (648000.0 / 3.141592653589793238462643);
}


// One output row in 32 bytes (one sector), used while the rows are ordered.
struct __align__(32) OutRow {
  uint64_t a, b;
  double s;
  uint32_t job, pad;
};

// The row count of the output kernels: M, or (Mdev given) the device's count
// clamped to M, the bound the caller sized the buffers by (the recheck may
// still have been adding rows when the launches were issued).
__device__ __forceinline__ uint64_t row_count(uint64_t M, const unsigned long long* Mdev) {
  return Mdev ? min((uint64_t)*Mdev, M) : M;
}

// ids + separation of each row, and the bucket histogram of id_a.
template <bool FP32>
__global__ void k_rows(const uint2* __restrict__ rows, uint64_t Mb,
                       const uint32_t* __restrict__ idxA, const uint32_t* __restrict__ idxB,
                       const SrcRec* __restrict__ recA, const SrcRec* __restrict__ recB,
                       const double* __restrict__ axv, const double* __restrict__ ayv,
                       const double* __restrict__ azv, const double* __restrict__ bxv,
                       const double* __restrict__ byv, const double* __restrict__ bzv,
                       int want_sep, OutRow* __restrict__ out, int bshift, uint32_t bmask,
                       uint32_t* __restrict__ bhist,
                       const unsigned long long* __restrict__ Mdev = nullptr) {
  const uint64_t M = row_count(Mb, Mdev);
  for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M;
       m += (uint64_t)gridDim.x * blockDim.x) {
    uint2 p = rows[m];  // entry indices, or source indices when idxA/idxB are null
    SrcRec u = recA[idxA ? idxA[p.x] : p.x], w = recB[idxB ? idxB[p.y] : p.y];
    OutRow o;
    o.a = u.id;
    o.b = w.id;
    o.s = 0.0;
    o.job = 0;
    o.pad = 0;
    if (bhist) o.pad = atomicAdd(&bhist[(uint32_t)(u.id >> bshift) & bmask], 1u);  // rank
    if (want_sep) {
      double sv;
      if (FP32) {
        sv = sep_arcsec_f2(u.ra, u.dec, w.ra, w.dec);
        if (sv < 0.0) sv = sep_arcsec_haversine(u.ra, u.dec, w.ra, w.dec);
      } else {
        sv = sep_arcsec_from_chord2(
            c_chord2(axv[p.x], ayv[p.x], azv[p.x], bxv[p.y], byv[p.y], bzv[p.y]));
      }
      o.s = sv;
    }
    out[m] = o;
  }
}

// Unpack rows into the result columns (used by the radix-sort fallback).
__global__ void k_rows_split(const OutRow* __restrict__ in, uint64_t M, uint64_t* __restrict__ a,
                             uint64_t* __restrict__ b, double* __restrict__ s,
                             uint32_t* __restrict__ job) {
  for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M;
       m += (uint64_t)gridDim.x * blockDim.x) {
    OutRow o = in[m];
    a[m] = o.a;
    b[m] = o.b;
    if (s) s[m] = o.s;
    if (job) job[m] = o.job;
  }
}

__global__ void k_max_u32(const uint32_t* __restrict__ v, uint64_t n, uint32_t* __restrict__ out) {
  uint32_t m = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    m = max(m, v[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Rows to their buckets: offset of the bucket plus the rank the row drew
// there (in OutRow.pad) when the histogram was built.  A single plan's
// bucket is the bmask bits of id_a above bshift; a batched plan's is
// jb[job].x (the job's first bucket) plus the bits jb[job].z of id_a above
// jb[job].y, each job with as many bits as its own row count needs.
__device__ __forceinline__ uint64_t row_bucket(const OutRow& o, int bshift, uint32_t bmask,
                                               const uint4* __restrict__ jb) {
  if (jb) {
    const uint4 J = __ldg(jb + o.job);
    return (uint64_t)J.x + ((uint32_t)(o.a >> J.y) & J.z);
  }
  return (uint32_t)(o.a >> bshift) & bmask;
}

__global__ void k_bucket_scatter(const OutRow* __restrict__ in, uint64_t Mb, int bshift,
                                 uint32_t bmask, const uint4* __restrict__ jb,
                                 const uint32_t* __restrict__ boff,
                                 OutRow* __restrict__ out,
                                 const unsigned long long* __restrict__ Mdev = nullptr) {
  const uint64_t M = row_count(Mb, Mdev);
  for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M;
       m += (uint64_t)gridDim.x * blockDim.x) {
    OutRow o = in[m];
    out[__ldg(boff + row_bucket(o, bshift, bmask, jb)) + o.pad] = o;
  }
}

__device__ __forceinline__ bool row_less(uint64_t a1, uint64_t b1, uint64_t s1, uint64_t a2,
                                         uint64_t b2, uint64_t s2) {
  if (a1 != a2) return a1 < a2;
  if (b1 != b2) return b1 < b2;
  return s1 < s2;
}

// Small buckets (<= kSmallBucket rows): one thread per row counts the rows
// of its bucket that order before it on (id_a, id_b, separation bits), ties
// by position, and writes the row at that rank.  (The bucket's rows are
// adjacent, so the comparisons read from L1.)
constexpr uint32_t kSmallBucket = 32;

// (The first row of each larger bucket appends it to `mid` (up to
// kBucketMid rows) or `big` for k_bucket_sort; one above kBucketCap sets
// DERR_BUCKET and the host orders the rows another way.  nbig[0] counts the
// big ones, nbig[1] the mid ones.)
__global__ void k_bucket_small(const OutRow* __restrict__ t, uint64_t Mb, int bshift,
                               uint32_t bmask, const uint4* __restrict__ jb,
                               const uint32_t* __restrict__ boff,
                               uint64_t* __restrict__ oa, uint64_t* __restrict__ ob,
                               double* __restrict__ os, uint32_t* __restrict__ oj,
                               uint32_t* __restrict__ big, uint32_t* __restrict__ nbig,
                               uint32_t* __restrict__ mid, int* __restrict__ err,
                               const unsigned long long* __restrict__ Mdev = nullptr) {
  const uint64_t M = row_count(Mb, Mdev);
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < M;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const OutRow r = t[p];
    const uint64_t bk = row_bucket(r, bshift, bmask, jb);
    const uint32_t lo = __ldg(boff + bk), hi = __ldg(boff + bk + 1);
    const uint32_t n = hi - lo;
    if (n > kSmallBucket) {
      if (p == lo) {
        if (n > kBucketCap)
          atomicOr(err, DERR_BUCKET);
        else if (n <= kBucketMid)
          mid[atomicAdd(nbig + 1, 1u)] = (uint32_t)bk;
        else
          big[atomicAdd(nbig, 1u)] = (uint32_t)bk;
      }
      continue;
    }
    const uint64_t rs = os ? (uint64_t)__double_as_longlong(r.s) : 0ull;
    uint32_t rank = 0;
    for (uint32_t j = lo; j < hi; ++j) {
      if (j == p) continue;
      const OutRow q = t[j];
      const uint64_t qs = os ? (uint64_t)__double_as_longlong(q.s) : 0ull;
      if (row_less(q.a, q.b, qs, r.a, r.b, rs) ||
          (j < p && q.a == r.a && q.b == r.b && qs == rs))
        ++rank;
    }
    const uint32_t dst = lo + rank;
    oa[dst] = r.a;
    ob[dst] = r.b;
    if (os) os[dst] = r.s;
    if (oj) oj[dst] = r.job;  // every row of a bucket has the same job
  }
}

// One CTA per larger bucket (kSmallBucket < rows <= CAP): bitonic sort in
// shared memory, each thread on one comparator of a stage at a time.  CAP =
// kBucketMid keeps the arrays small (6 KB), so that many CTAs share an SM.
template <int CAP>
__global__ void __launch_bounds__(kBucketThreads) k_bucket_sort(
    const OutRow* __restrict__ t, const uint32_t* __restrict__ boff,
    const uint32_t* __restrict__ big, const uint32_t* __restrict__ nbig, int use_sep,
    uint64_t* __restrict__ oa, uint64_t* __restrict__ ob, double* __restrict__ os,
    uint32_t* __restrict__ oj) {
  __shared__ uint64_t A[CAP], B[CAP], S[CAP];
  const uint32_t nb = *nbig;
  for (uint32_t q = blockIdx.x; q < nb; q += gridDim.x) {
    const uint32_t bk = big[q];
    uint32_t lo = boff[bk], hi = boff[bk + 1];
    uint32_t n = hi - lo;
    if (n <= kSmallBucket || n > (uint32_t)CAP) continue;  // (listed ones are in range)
    uint32_t np = 1;
    while (np < n) np <<= 1;
    for (uint32_t i = threadIdx.x; i < np; i += kBucketThreads) {
      if (i < n) {
        OutRow r = t[lo + i];
        A[i] = r.a;
        B[i] = r.b;
        S[i] = use_sep ? (uint64_t)__double_as_longlong(r.s) : 0ull;
        if (oj) oj[lo + i] = r.job;
      } else {
        A[i] = ~0ull;
        B[i] = ~0ull;
        S[i] = ~0ull;
      }
    }
    __syncthreads();
    for (uint32_t k = 2; k <= np; k <<= 1) {
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        for (uint32_t c = threadIdx.x; c < np / 2; c += kBucketThreads) {
          // comparator c: the pair (i, i + j) with bit j of i clear
          const uint32_t i = ((c & ~(j - 1)) << 1) | (c & (j - 1));
          const uint32_t l = i | j;
          bool up = (i & k) == 0;
          bool gt = row_less(A[l], B[l], S[l], A[i], B[i], S[i]);
          if (gt == up) {
            uint64_t t;
            t = A[i]; A[i] = A[l]; A[l] = t;
            t = B[i]; B[i] = B[l]; B[l] = t;
            t = S[i]; S[i] = S[l]; S[l] = t;
          }
        }
        __syncthreads();
      }
    }
    for (uint32_t i = threadIdx.x; i < n; i += kBucketThreads) {
      oa[lo + i] = A[i];
      ob[lo + i] = B[i];
      if (os) os[lo + i] = __longlong_as_double((long long)S[i]);
    }
    __syncthreads();
  }
}

}  // namespace hlc
