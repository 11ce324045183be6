// Kernels of the cross-match path: source preparation (validation, cell keys,
// quad-direction expansion), sorted payload, neighbour-cell candidates, the
// pair test, the binary64 recheck of guard-band candidates and the output
// rows (ids, separations).
#pragma once

#include "canon.cuh"
#include "common.cuh"
#include "fastpix.cuh"
#include "fp32.cuh"
#include "index.cuh"
#include "learned.cuh"

namespace hlc {

constexpr int kThreads = 256;

// One source in 32 bytes (one DRAM sector): normalised RA, Dec, id.  Written
// in input order by the preparation kernels so that later gathers by source
// index touch a single sector.
struct __align__(32) SrcRec {
  double ra, dec;
  uint64_t id, pad;  // pad: the bits of the source's Eq. 4 error radius (or 0)
};

__device__ __forceinline__ double rec_err(const SrcRec& r) {
  return __longlong_as_double((long long)r.pad);
}

// Largest per-source error radius of a column (Eq. 4), as the bits of a
// non-negative double (whose integer order is the numeric order); a value
// that is not finite or is negative flags invalid input.
__global__ void k_err_max(const double* __restrict__ e, uint64_t n,
                          unsigned long long* __restrict__ out, int* __restrict__ err) {
  unsigned long long m = 0;
  bool bad = false;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    double v = e[i];
    if (!(v >= 0.0) || !(v <= 1.7976931348623157e308)) {
      bad = true;
      continue;
    }
    if (v == 0.0) v = 0.0;  // -0 has the sign bit set
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    m = b > m ? b : m;
  }
  if (bad) atomicOr(err, DERR_INPUT);
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_down_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}
// Number of B entries in a table cell up to which the FP32 join uses the
// table order (sparse regions).
constexpr int kPairUnroll = 4;  // candidates per lane per pair-test iteration
#ifndef HLC_SPARSE_CELL
#define HLC_SPARSE_CELL 32
#endif
constexpr uint32_t kSparseCell = HLC_SPARSE_CELL;

// ---------------------------------------------------------------------------
// Preparation.
// ---------------------------------------------------------------------------

// The bits in which the ids differ (OR of id ^ id[0] over the sources, for
// the output's bucketing), a warp's share added once; every thread calls it.
__device__ __forceinline__ void id_span_flush(unsigned long long* iddiff,
                                              unsigned long long acc) {
  if (!iddiff) return;
  for (int o = 16; o > 0; o >>= 1) acc |= __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicOr(iddiff, acc);
}

// Cell key and identity index of each source (complete mode), with input
// validation (non-finite or |dec| > 90 sets DERR_INPUT).  FAST: guarded FP32
// evaluation with binary64 fallback (same pixels).
// (FAST: sources the guarded estimate cannot decide are queued and finished
// by k_prep_fallback, so that warps do not diverge into the binary64 path.)
// hist (FAST only; null: none): the radix sort's digit histograms of the
// keys, hist_np passes of 8 bits from bit hist_lo, counted here for every key
// this kernel writes for good (the queued ones are counted by the fallback),
// so the sort needs no pass of its own over the keys.
constexpr int kPrepHistPasses = 4;
template <bool FAST>
__global__ void k_prep_keys(const double* __restrict__ ra, const double* __restrict__ dec,
                            const uint64_t* __restrict__ id, uint64_t n, int order, PixConst K,
                            uint32_t* __restrict__ key, uint32_t* __restrict__ idx,
                            SrcRec* __restrict__ rec, uint32_t* __restrict__ slow,
                            unsigned long long* __restrict__ nslow, int* __restrict__ err,
                            const double* __restrict__ perr = nullptr,
                            uint32_t* __restrict__ hist = nullptr, int hist_lo = 0,
                            int hist_np = 0, unsigned long long* __restrict__ iddiff = nullptr) {
  __shared__ uint32_t sh[kPrepHistPasses][256];
  const uint64_t id0 = (iddiff && n) ? id[0] : 0ull;
  unsigned long long idacc = 0;
  if (FAST && hist) {
    for (int t = threadIdx.x; t < kPrepHistPasses * 256; t += blockDim.x) (&sh[0][0])[t] = 0u;
    __syncthreads();
  }
  // (a thread's next source's coordinates and id are loaded while the
  // current one is processed)
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const bool want_id = rec || iddiff;
  double pa = 0.0, pd = 0.0;
  uint64_t pid = 0;
  {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
      pa = ra[i];
      pd = dec[i];
      if (want_id) pid = id[i];
    }
  }
  for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
    uint64_t i = i0 + threadIdx.x;
    bool live = i < n;
    bool defer = false;
    uint32_t kfin = 0;  // the key written
    double a = pa, d = pd;
    const uint64_t idi = pid;
    if (i + stride < n) {
      pa = ra[i + stride];
      pd = dec[i + stride];
      if (want_id) pid = id[i + stride];
    }
    if (live) {
      uint32_t k = 0;
      if (FAST) {
        if (!(bits_finite(a) && bits_abs_le(d, 90.0))) {
          atomicOr(err, DERR_INPUT);
        } else if (!bits_in_ra_range(a)) {
          defer = true;  // RA outside [0, 360): the binary64 path normalises key and record
        } else {
          FastDec fd = f_dec_part(split_f64(d));
          defer = !f_pix(split_f64(a), fd, order, K, &k);
        }
      } else {
        if (!c_valid(a, d)) {
          atomicOr(err, DERR_INPUT);
        } else {
          a = c_norm_ra(a);
          k = c_ang2pix(a, d, order);
        }
      }
      key[i] = k;
      kfin = k;
      if (idx) idx[i] = (uint32_t)i;
      if (iddiff) idacc |= idi ^ id0;
      if (rec) {
        SrcRec r;
        r.ra = a;
        r.dec = d;
        r.id = idi;
        r.pad = perr ? (uint64_t)__double_as_longlong(perr[i]) : 0ull;  // Eq. 4 error radius
        rec[i] = r;
      }
    }
    if (FAST) {
      unsigned b = __ballot_sync(0xffffffffu, defer);
      if (b) {
        int lane = threadIdx.x & 31;
        unsigned long long base = 0;
        if (lane == __ffs(b) - 1) base = atomicAdd(nslow, (unsigned long long)__popc(b));
        base = __shfl_sync(0xffffffffu, base, __ffs(b) - 1);
        if (defer) slow[base + __popc(b & lanemask_lt())] = (uint32_t)i;
      }
      if (hist && live && !defer)  // (an invalid source keeps key 0 and counts as such)
        for (int p = 0; p < hist_np; ++p)
          atomicAdd(&sh[p][(kfin >> (hist_lo + 8 * p)) & 255u], 1u);
    }
  }
  if (FAST && hist) {
    __syncthreads();
    for (int t = threadIdx.x; t < hist_np * 256; t += blockDim.x) {
      const uint32_t c = (&sh[0][0])[t];
      if (c) atomicAdd(hist + t, c);
    }
  }
  id_span_flush(iddiff, idacc);
}

// Binary64 ang2pix of the queued sources (and, with rec, the record's RA
// normalised to [0, 360); with hist, their keys' digits counted).
__global__ void k_prep_fallback(const double* __restrict__ ra, const double* __restrict__ dec,
                                int order, const uint32_t* __restrict__ slow,
                                const unsigned long long* __restrict__ nslow,
                                uint32_t* __restrict__ key, SrcRec* __restrict__ rec = nullptr,
                                uint32_t* __restrict__ hist = nullptr, int hist_lo = 0,
                                int hist_np = 0) {
  __shared__ uint32_t sh[kPrepHistPasses][256];
  const uint64_t ns = *nslow;
  // (blocks beyond the queue's need return at once; the rest count in
  // shared memory and flush once)
  if ((uint64_t)blockIdx.x * blockDim.x >= ns) return;
  if (hist) {
    for (int t = threadIdx.x; t < kPrepHistPasses * 256; t += blockDim.x) (&sh[0][0])[t] = 0u;
    __syncthreads();
  }
  for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ns;
       q += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t i = slow[q];
    const double a = c_norm_ra(ra[i]);
    const uint32_t k = ff_or_c_ang2pix(a, dec[i], order);
    key[i] = k;
    if (rec) rec[i].ra = a;
    for (int p = 0; hist && p < hist_np; ++p)
      atomicAdd(&sh[p][(k >> (hist_lo + 8 * p)) & 255u], 1u);
  }
  if (hist) {
    __syncthreads();
    for (int t = threadIdx.x; t < hist_np * 256; t += blockDim.x) {
      const uint32_t c = (&sh[0][0])[t];
      if (c) atomicAdd(hist + t, c);
    }
  }
}

// Quad-direction cells of each source (Algorithm 1): 5 slots + count.
// (FAST: no FP64 instruction on the way, except the cosine of the cos(Dec)
// variant; a source with an undecided position keeps its decided pixels in
// its cells row, the mask of the undecided ones in count, and is queued for
// k_quad_fallback.)  cosdec: the RA copies are shifted by R / cos(dec)
// (c_ra_shift_cos), the variant beside Algorithm 1's literal R.
template <bool FAST>
__global__ void k_quad_cells(const double* __restrict__ ra, const double* __restrict__ dec,
                             const uint64_t* __restrict__ id, uint64_t n, double R, int order,
                             PixConst K, uint32_t* __restrict__ cells,
                             uint32_t* __restrict__ count, SrcRec* __restrict__ rec,
                             uint32_t* __restrict__ slow, unsigned long long* __restrict__ nslow,
                             int* __restrict__ err, bool cosdec = false,
                             unsigned long long* __restrict__ iddiff = nullptr) {
  const f2 Rd = split_f64(R);
  const uint64_t id0 = (iddiff && id && n) ? id[0] : 0ull;
  unsigned long long idacc = 0;
  // (a thread's next source's coordinates are loaded while the current one
  // is processed)
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  double pa = 0.0, pd = 0.0;
  {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
      pa = ra[i];
      pd = dec[i];
    }
  }
  for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
    uint64_t i = i0 + threadIdx.x;
    bool defer = false;
    double a = pa, d = pd;
    if (i + stride < n) {
      pa = ra[i + stride];
      pd = dec[i + stride];
    }
    if (i < n) {
      uint32_t c[5] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
      int m = 1;
      const bool valid = FAST ? (bits_finite(a) && bits_abs_le(d, 90.0)) : c_valid(a, d);
      if (!valid) {
        atomicOr(err, DERR_INPUT);
        c[0] = 0;
      } else if (FAST) {
        if (!bits_in_ra_range(a)) a = c_norm_ra(a);
        uint32_t p[5] = {0u, 0u, 0u, 0u, 0u};
        const f2 Ra = cosdec ? split_f64(c_ra_shift_cos(R, d)) : Rd;
        const unsigned und = g_quad_pos(a, d, Rd, Ra, order, K, p);
        if (und) {
          defer = true;
#pragma unroll
          for (int e = 0; e < 5; ++e) c[e] = p[e];
          m = (int)und;  // (the mask, until k_quad_fallback)
        } else {
          m = quad_sort_unique(p, c);
        }
      } else {
        a = c_norm_ra(a);
        m = c_quad_cells(a, d, R, order, c, cosdec);
      }
#pragma unroll
      for (int e = 0; e < 5; ++e) cells[5 * i + e] = (defer || e < m) ? c[e] : 0xFFFFFFFFu;
      count[i] = (uint32_t)m;
      if (rec) {
        SrcRec r;
        r.ra = a;  // normalised when valid
        r.dec = d;
        r.id = id[i];
        r.pad = 0;
        rec[i] = r;
      }
      if (iddiff && id) idacc |= id[i] ^ id0;
    }
    if (FAST) {
      unsigned b = __ballot_sync(0xffffffffu, defer);
      if (b) {
        int lane = threadIdx.x & 31;
        unsigned long long base = 0;
        if (lane == __ffs(b) - 1) base = atomicAdd(nslow, (unsigned long long)__popc(b));
        base = __shfl_sync(0xffffffffu, base, __ffs(b) - 1);
        if (defer) slow[base + __popc(b & lanemask_lt())] = (uint32_t)i;
      }
    }
  }
  id_span_flush(iddiff, idacc);
}

// The queued sources of k_quad_cells<true>.  Each warp takes 32 of them,
// lists their undecided (source, position) pairs in shared memory and
// computes the pairs 32 at a time, every lane running the same binary64 pixel
// function on the position's coordinates (formed exactly as c_quad_cells
// states them); each lane then sorts its source's five pixels and drops the
// repeats.
__global__ void __launch_bounds__(kThreads) k_quad_fallback(
    const double* __restrict__ ra, const double* __restrict__ dec, double R, int order,
    const uint32_t* __restrict__ slow, const unsigned long long* __restrict__ nslow,
    uint32_t* __restrict__ cells, uint32_t* __restrict__ count, bool cosdec = false) {
  __shared__ uint8_t s_pair[kThreads / 32][160];   // (lane << 3) | position
  __shared__ uint32_t s_pix[kThreads / 32][160];   // [lane * 5 + position]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = lanemask_lt();
  const uint64_t ns = *nslow;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t q0 = (uint64_t)blockIdx.x * blockDim.x + (uint64_t)(w * 32); q0 < ns;
       q0 += stride) {
    const uint64_t q = q0 + lane;
    const bool live = q < ns;
    const uint32_t i = live ? slow[q] : 0u;
    const unsigned und = live ? count[i] : 0u;
    const double a = live ? c_norm_ra(ra[i]) : 0.0, d = live ? dec[i] : 0.0;
    int npairs = 0;
#pragma unroll
    for (int e = 0; e < 5; ++e) {
      const bool mine = (und >> e) & 1u;
      const unsigned bal = __ballot_sync(0xffffffffu, mine);
      if (mine) s_pair[w][npairs + __popc(bal & lt)] = (uint8_t)((lane << 3) | e);
      npairs += __popc(bal);
    }
    __syncwarp();
    for (int k0 = 0; k0 < npairs; k0 += 32) {
      const int k = k0 + lane;
      const bool act = k < npairs;
      const unsigned v = act ? s_pair[w][k] : (unsigned)(lane << 3);
      const int src = (int)(v >> 3), e = (int)(v & 7u);
      const double sa = __shfl_sync(0xffffffffu, a, src);
      const double sd = __shfl_sync(0xffffffffu, d, src);
      if (act) {
        double pa = sa, pd = sd;
        if (e == 1 || e == 2) {
          const double RA = cosdec ? c_ra_shift_cos(R, sd) : R;
          pa = wrap_ra(e == 1 ? __dadd_rn(sa, RA) : __dsub_rn(sa, RA));
        } else if (e == 3) {
          pd = __dsub_rn(sd, R);
          if (pd < -90.0) pd = -90.0;
        } else if (e == 4) {
          pd = __dadd_rn(sd, R);
          if (pd > 90.0) pd = 90.0;
        }
        s_pix[w][src * 5 + e] = ff_or_c_ang2pix(pa, pd, order);
      }
    }
    __syncwarp();
    if (live) {
      uint32_t p[5], c[5] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
#pragma unroll
      for (int e = 0; e < 5; ++e)
        p[e] = ((und >> e) & 1u) ? s_pix[w][lane * 5 + e] : cells[5ull * i + e];
      const int m = quad_sort_unique(p, c);
#pragma unroll
      for (int e = 0; e < 5; ++e) cells[5ull * i + e] = e < m ? c[e] : 0xFFFFFFFFu;
      count[i] = (uint32_t)m;
    }
    __syncwarp();  // s_pair and s_pix are reused by the next round
  }
}

// One (cell, source) entry per distinct quad cell, at the scanned offsets.
template <typename OffT>
// (hist: the radix sort's digit histograms of the keys written, hist_np
// passes of 8 bits from bit 0, counted in shared memory and added once per
// block)
__global__ void k_quad_emit(const uint32_t* __restrict__ cells, const uint32_t* __restrict__ count,
                            const OffT* __restrict__ off, uint64_t n,
                            uint32_t* __restrict__ key, uint32_t* __restrict__ idx,
                            uint32_t* __restrict__ hist = nullptr, int hist_np = 0) {
  __shared__ uint32_t sh[kPrepHistPasses][256];
  if (hist) {
    for (int t = threadIdx.x; t < kPrepHistPasses * 256; t += blockDim.x) (&sh[0][0])[t] = 0u;
    __syncthreads();
  }
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t o = off[i];
    uint32_t m = count[i];
    for (uint32_t e = 0; e < m; ++e) {
      const uint32_t k = cells[5 * i + e];
      key[o + e] = k;
      idx[o + e] = (uint32_t)i;
      for (int p = 0; hist && p < hist_np; ++p) atomicAdd(&sh[p][(k >> (8 * p)) & 255u], 1u);
    }
  }
  if (hist) {
    __syncthreads();
    for (int t = threadIdx.x; t < hist_np * 256; t += blockDim.x) {
      const uint32_t c = (&sh[0][0])[t];
      if (c) atomicAdd(hist + t, c);
    }
  }
}

// Sorted payload: binary64 canonical unit vectors (plain form).
// (ve, when given: the entries' Eq. 4 error radii.)
__global__ void k_payload64(const SrcRec* __restrict__ rec, const uint32_t* __restrict__ idx,
                            uint64_t m, double* __restrict__ vx, double* __restrict__ vy,
                            double* __restrict__ vz, double* __restrict__ ve = nullptr) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (uint64_t)gridDim.x * blockDim.x) {
    SrcRec r = rec[idx[e]];
    double x = 0, y = 0, z = 0;
    if (c_valid(r.ra, r.dec)) c_unitvec(r.ra, r.dec, &x, &y, &z);
    vx[e] = x;
    vy[e] = y;
    vz[e] = z;
    if (ve) ve[e] = rec_err(r);
  }
}

// Sorted payload of the guard form: FP32 unit vectors with a known error
// bound, in entry order.
// (iddiff, when given, receives the OR of id ^ id of source 0 over all
// entries: the bits in which the ids differ, for the output bucketing.)
// Eq. 4: w = wsign * rho with rho = k9 e^2, k9 = 9 (pi/648000)^2, the
// source's share of the pair's squared radius in radians (+rho for A, -rho
// for B, so that b.w - a.w = -(rho_a + rho_b)); otherwise w = 0.
template <bool EQ4>
__global__ void k_payload32(const SrcRec* __restrict__ rec, const uint32_t* __restrict__ idx,
                            uint64_t m, float4* __restrict__ v,
                            unsigned long long* __restrict__ iddiff, float wsign = 0.f,
                            double k9 = 0.0) {
  const uint64_t id0 = (iddiff && m) ? rec[0].id : 0;
  unsigned long long acc = 0;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (uint64_t)gridDim.x * blockDim.x) {
    SrcRec r = rec[idx[e]];
    float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
    if (bits_finite(r.ra) && bits_abs_le(r.dec, 90.0)) u = fp32_unitvec(r.ra, r.dec);
    if (EQ4) {  // (a compile-time branch: the single-radius form runs no FP64 instruction)
      const double er = rec_err(r);
      u.w = wsign * (float)(er * er * k9);
    }
    v[e] = u;
    acc |= r.id ^ id0;
  }
  if (iddiff) {
    for (int o = 16; o > 0; o >>= 1) acc |= __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicOr(iddiff, acc);
  }
}

__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t* __restrict__ a, uint32_t n,
                                                    uint32_t q) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (a[mid] < q)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Candidates and pair test (one thread per A entry): the neighbourhood of the
// entry's cell (complete mode) or the cell itself (quad mode) is looked up in
// B's cell index and every B entry of those cells is tested.  Loops are
// warp-uniform so that match rows are reserved with one atomic per warp from
// a ballot.
// ---------------------------------------------------------------------------

struct PairSink {
  uint2* rows;                  // (A entry, B entry)
  unsigned long long* count;
  uint64_t cap;
  uint2* band;                  // FP32 form: candidates inside the band
  unsigned long long* band_count;
  uint64_t band_cap;
  unsigned long long* tests;    // algorithmic pair tests
  unsigned long long* dups;     // quad pairs owned by a smaller shared cell
  unsigned long long* heads;    // distinct A cells
  int* err;
};

__device__ __forceinline__ void warp_emit(bool emit, uint32_t ka, uint32_t kb, uint2* rows,
                                          unsigned long long* count, uint64_t cap, int* err) {
  unsigned b = __ballot_sync(0xffffffffu, emit);
  if (b == 0) return;
  int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == __ffs(b) - 1) base = atomicAdd(count, (unsigned long long)__popc(b));
  base = __shfl_sync(0xffffffffu, base, __ffs(b) - 1);
  if (emit) {
    unsigned long long pos = base + __popc(b & lanemask_lt());
    if (pos < cap)
      rows[pos] = make_uint2(ka, kb);
    else
      atomicOr(err, DERR_OVERFLOW);
  }
}

// Rows staged per warp in shared memory and appended to the global list in
// batches: one atomic reservation per flush instead of one per ballot.
template <int CAP>
struct WarpRows {
  uint2* buf;     // this warp's CAP slots in shared memory
  int fill = 0;   // warp-uniform
  __device__ __forceinline__ void add(bool emit, uint32_t ka, uint32_t kb) {
    unsigned b = __ballot_sync(0xffffffffu, emit);
    if (emit) buf[fill + __popc(b & lanemask_lt())] = make_uint2(ka, kb);
    fill += __popc(b);
  }
  __device__ __forceinline__ void flush(uint2* rows, unsigned long long* count, uint64_t cap,
                                        int* err) {
    if (fill == 0) return;
    __syncwarp();
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(count, (unsigned long long)fill);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int i = lane; i < fill; i += 32) {
      if (base + i < cap)
        rows[base + i] = buf[i];
      else
        atomicOr(err, DERR_OVERFLOW);
    }
    __syncwarp();
    fill = 0;
  }
};

// Smallest cell shared by the quad cell lists of two sources.
__device__ __forceinline__ uint32_t quad_owner(const uint32_t* __restrict__ ca,
                                               const uint32_t* __restrict__ cb) {
  uint32_t own = 0xFFFFFFFFu;
#pragma unroll
  for (int e = 0; e < 5; ++e) {
    uint32_t x = ca[e];
    if (x == 0xFFFFFFFFu) break;
#pragma unroll
    for (int f = 0; f < 5; ++f)
      if (cb[f] == x && x < own) own = x;
  }
  return own;
}

struct PairArgs {
  uint64_t mA;
  const uint32_t* keyA;
  CellIndex bix;          // offset table of B (table index)
  LearnedIndex lix;       // learned index over B's unique cells
  const uint32_t* uniqB;  // (learned index) unique cells of B
  const uint32_t* startB; // (learned index) their first entries
  uint64_t uB;
  int order;
  const double *axv, *ayv, *azv, *bxv, *byv, *bzv;
  const float4 *a32, *b32;
  double C;
  float lo32, hi32;
  const uint32_t *idxA, *idxB, *cellsA, *cellsB;
  uint32_t sparse_cell;
  unsigned long long *lhits, *llook;
  const uint8_t* tiled;   // (BUCKET) A entries taken by the tile kernel, or null
  // Eq. 4 (EQ4): binary64 form: the entries' error radii and 9 (pi/648000)^2
  const double *aev, *bev;
  double k9;
};

// BUCKET: B is bucketed by table cell (ordered by fine key only inside dense
// table cells); a sparse table cell is read whole, once per A entry.
// EQ4: each pair has its own radius (Eq. 4).  FP32: the vectors' w carry
// +rho_a / -rho_b, the tested value is s - (rho_a + rho_b) and lo32 / hi32
// are -G / +G around 0.  Binary64: a pair whose s exceeds the bound
// x^2 = 9 (pi/648000)^2 (e_a^2 + e_b^2) >= 4 sin^2(r_ij/2) (with a 1e-12
// margin for rounding) is rejected, the rest are decided against the
// canonical 4 sin^2(r_ij/2).
// (The FP32 table form, the default path, keeps two candidates per lane in
// flight and six CTAs per SM: more warps hide its dependent loads better
// than more candidates per warp; measured 0.443 against 0.469 ms for four
// candidates at four CTAs, 10M x 10M full sky.)
template <bool FP32, bool QUAD, bool LEARNED, bool BUCKET, bool EQ4 = false>
__global__ void __launch_bounds__(kThreads, (FP32 && BUCKET) ? 6 : 1)
    k_pair(const PairArgs pa, PairSink sink) {
  const uint64_t mA = pa.mA;
  const uint32_t* __restrict__ keyA = pa.keyA;
  const CellIndex bix = pa.bix;
  const int order = pa.order;
  const double* __restrict__ axv = pa.axv;
  const double* __restrict__ ayv = pa.ayv;
  const double* __restrict__ azv = pa.azv;
  const double* __restrict__ bxv = pa.bxv;
  const double* __restrict__ byv = pa.byv;
  const double* __restrict__ bzv = pa.bzv;
  const float4* __restrict__ a32 = pa.a32;
  const float4* __restrict__ b32 = pa.b32;
  const double C = pa.C;
  const float lo32 = pa.lo32, hi32 = pa.hi32;
  const uint32_t* __restrict__ idxA = pa.idxA;
  const uint32_t* __restrict__ idxB = pa.idxB;
  const uint32_t* __restrict__ cellsA = pa.cellsA;
  const uint32_t* __restrict__ cellsB = pa.cellsB;
  const uint32_t sparse_cell = pa.sparse_cell;
  unsigned long long nlhit = 0, nllook = 0;
  const uint64_t stride = (uint64_t)gridDim.x * kThreads;
  unsigned long long ntest = 0, ndup = 0, nhead = 0;
  constexpr int kRowCap = 256, kBandCap = FP32 ? 128 : 32;
  __shared__ uint2 s_rows[kThreads / 32][kRowCap];
  __shared__ uint2 s_band[kThreads / 32][kBandCap];
  WarpRows<kRowCap> wrows{s_rows[threadIdx.x >> 5]};
  WarpRows<kBandCap> wband{s_band[threadIdx.x >> 5]};
  // Software pipeline over a thread's A entries: each iteration issues the
  // next entry's loads (key, vector, tile flag; for the FP32 table form also
  // the two offset-table words of its table cell, once its key has arrived)
  // while the current entry's candidates are tested, so that the dependent
  // chain key -> table -> ranges -> B vectors of one entry overlaps the
  // previous entry's tests.
  constexpr bool TABLE = FP32 && !LEARNED && !QUAD;
  struct ALoad {
    bool live;
    uint32_t cell;
    float4 a4;
    double ax, ay, az, ae;
  };
  auto load_a = [&](uint64_t kk, ALoad& L) {
    L.live = kk < mA;
    if (BUCKET && pa.tiled && L.live && pa.tiled[kk]) L.live = false;  // the tile kernel's
    L.cell = L.live ? keyA[kk] : 0u;
    L.a4 = make_float4(0.f, 0.f, 0.f, 0.f);
    L.ax = L.ay = L.az = L.ae = 0.0;
    if (L.live) {
      if (FP32) {
        L.a4 = a32[kk];
      } else {
        L.ax = axv[kk]; L.ay = ayv[kk]; L.az = azv[kk];
        if (EQ4) L.ae = pa.aev[kk];
      }
    }
  };
  auto load_t = [&](const ALoad& L, uint32_t& t0, uint32_t& t1) {
    t0 = t1 = 0u;
    if (TABLE && bix.shift > 0 && L.live) {
      const uint32_t P = L.cell >> bix.shift;
      t0 = __ldg(bix.table + P);
      t1 = __ldg(bix.table + P + 1);
    }
  };
  ALoad acur;
  load_a((uint64_t)blockIdx.x * kThreads + threadIdx.x, acur);
  uint32_t ct0, ct1;
  load_t(acur, ct0, ct1);
  // every thread of the warp runs the same number of outer iterations
  for (uint64_t kb0 = (uint64_t)blockIdx.x * kThreads; kb0 < mA; kb0 += stride) {
    uint64_t k = kb0 + (threadIdx.x);
    ALoad anxt;
    load_a(k + stride, anxt);
    const bool live = acur.live;
    const uint32_t cell = acur.cell;
    const double ax = acur.ax, ay = acur.ay, az = acur.az, ae = acur.ae;
    const float4 a4 = acur.a4;
    // neighbourhood of the A cell (complete) or the cell itself (quad).  In
    // complete mode a sparse region is joined at the order of B's offset
    // table instead: the (at most 4) table cells that cover the fine 3x3
    // block hold a superset of the candidates, so the exact set is the same,
    // and each of their ranges is read straight from the table.
    bool coarse_lane = false;
    uint32_t nb[9];
#pragma unroll
    for (int s = 0; s < 9; ++s) nb[s] = kNoCell;
    if (live) {
      if (QUAD) {
        nb[0] = cell;
      } else {
        bool coarse = false;
        if (FP32 && !LEARNED && bix.shift > 0) {
          if (ct1 - ct0 <= sparse_cell) coarse = parent_cover4(cell, order, bix.shift / 2, nb);
        }
        if (coarse) {
          coarse_lane = true;
        } else {
          cell_neighbourhood9(cell, order, nb);
        }
      }
    }
    // all ranges first (independent loads in flight together), then one
    // warp-uniform loop over the lane's concatenated candidate list
    constexpr int NS = QUAD ? 1 : 9;
    uint32_t rb[NS], re[NS];
    uint32_t total = 0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      uint2 r = make_uint2(0u, 0u);
      if (nb[s] != kNoCell) {
        if (LEARNED) {
          bool hit;
          uint32_t pos = learned_lower_bound(pa.lix, nb[s], &hit);
          nlhit += hit;
          ++nllook;
          if (pos < pa.uB && __ldg(pa.uniqB + pos) == nb[s])
            r = make_uint2(__ldg(pa.startB + pos), __ldg(pa.startB + pos + 1));
        } else if (coarse_lane) {
          r = make_uint2(__ldg(bix.table + nb[s]), __ldg(bix.table + nb[s] + 1));
        } else if (BUCKET) {
          // sparse table cell: read whole (once); dense: ordered, search it
          const uint32_t Q = nb[s] >> bix.shift;
          const uint32_t c0 = __ldg(bix.table + Q), c1 = __ldg(bix.table + Q + 1);
          if (c1 - c0 <= sparse_cell) {
            bool seen = false;
#pragma unroll
            for (int e = 0; e < s; ++e)
              seen |= nb[e] != kNoCell && (nb[e] >> bix.shift) == Q;
            if (!seen) r = make_uint2(c0, c1);
          } else {
            r = cell_range_in(bix.keys, c0, c1, nb[s]);
          }
        } else {
          r = cell_range(bix, nb[s]);
        }
      }
      rb[s] = r.x;
      re[s] = r.y;
      total += r.y - r.x;
    }
    ntest += total;
    uint32_t nt0, nt1;  // the next entry's table words (its key has arrived by now)
    load_t(anxt, nt0, nt1);
    {  // distinct A cells (statistics)
      uint32_t prev = __shfl_up_sync(0xffffffffu, cell, 1);
      if ((threadIdx.x & 31) == 0 && live && k > 0) prev = keyA[k - 1];
      nhead += live && (k == 0 || prev != cell);
    }
    const uint32_t maxT = __reduce_max_sync(0xffffffffu, total);
    const uint32_t srcA = (BUCKET && live && total) ? __ldg(pa.idxA + k) : 0u;
    uint32_t cur = rb[0], end = re[0];
    // U candidates per lane per iteration: their loads are issued together
    constexpr int U = QUAD ? 1 : ((FP32 && BUCKET) ? 2 : kPairUnroll);
    for (uint32_t t = 0; t < maxT; t += U) {
      uint32_t jj[U];
      bool act[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        act[u] = t + u < total;
        jj[u] = 0;
        if (act[u]) {
          while (cur >= end) {  // next non-empty range (constant-index shift)
#pragma unroll
            for (int i = 0; i + 1 < NS; ++i) {
              rb[i] = rb[i + 1];
              re[i] = re[i + 1];
            }
            cur = rb[0];
            end = re[0];
          }
          jj[u] = cur++;
        }
      }
      bool hit[U], band[U];
      bool anyv = false;
      if (FP32) {
        float4 bb[U];
#pragma unroll
        for (int u = 0; u < U; ++u) bb[u] = act[u] ? __ldg(b32 + jj[u]) : a4;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          float dx = a4.x - bb[u].x, dy = a4.y - bb[u].y, dz = a4.z - bb[u].z;
          float s2 = EQ4 ? fmaf(dx, dx, bb[u].w - a4.w) : dx * dx;
          s2 = fmaf(dy, dy, s2);
          s2 = fmaf(dz, dz, s2);
          hit[u] = act[u] && s2 <= lo32;
          band[u] = act[u] && !hit[u] && s2 <= hi32;
          anyv |= hit[u] || band[u];
        }
      } else {
        double bx[U], by[U], bz[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          bx[u] = act[u] ? bxv[jj[u]] : ax;
          by[u] = act[u] ? byv[jj[u]] : ay;
          bz[u] = act[u] ? bzv[jj[u]] : az;
        }
        double be[U];
#pragma unroll
        for (int u = 0; u < U; ++u) be[u] = (EQ4 && act[u]) ? pa.bev[jj[u]] : 0.0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          double s2 = c_chord2(ax, ay, az, bx[u], by[u], bz[u]);
          if (EQ4) {
            const double x2 = (ae * ae + be[u] * be[u]) * pa.k9;
            hit[u] = act[u] && s2 <= x2 * (1.0 + 1e-12) &&
                     s2 <= c_threshold(c_pair_radius(ae, be[u]));
          } else {
            hit[u] = act[u] && s2 <= C;
          }
          band[u] = false;
          anyv |= hit[u];
        }
      }
      if (QUAD && anyv) {
        uint32_t own = quad_owner(cellsA + 5ull * idxA[k], cellsB + 5ull * idxB[jj[0]]);
        if (own != cell) {
          if (hit[0]) ++ndup;
          hit[0] = false;
          band[0] = false;
          anyv = false;
        }
      }
      if (__any_sync(0xffffffffu, anyv)) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          // BUCKET: rows carry source indices (the output reads records)
          const uint32_t ea = BUCKET ? srcA : (uint32_t)k;
          const uint32_t eb =
              BUCKET ? ((hit[u] || band[u]) ? __ldg(pa.idxB + jj[u]) : 0u) : jj[u];
          wrows.add(hit[u], ea, eb);
          if (FP32) wband.add(band[u], ea, eb);
        }
        if (wrows.fill > kRowCap - 32 * U)
          wrows.flush(sink.rows, sink.count, sink.cap, sink.err);
        if (FP32 && wband.fill > kBandCap - 32 * U)
          wband.flush(sink.band, sink.band_count, sink.band_cap, sink.err);
      }
    }
    acur = anxt;
    ct0 = nt0;
    ct1 = nt1;
  }
  wrows.flush(sink.rows, sink.count, sink.cap, sink.err);
  if (FP32) wband.flush(sink.band, sink.band_count, sink.band_cap, sink.err);
  // one atomic per warp for the counters
  for (int o = 16; o > 0; o >>= 1) {
    ntest += __shfl_down_sync(0xffffffffu, ntest, o);
    ndup += __shfl_down_sync(0xffffffffu, ndup, o);
    nhead += __shfl_down_sync(0xffffffffu, nhead, o);
    if (LEARNED) {
      nlhit += __shfl_down_sync(0xffffffffu, nlhit, o);
      nllook += __shfl_down_sync(0xffffffffu, nllook, o);
    }
  }
  if ((threadIdx.x & 31) == 0) {
    if (ntest) atomicAdd(sink.tests, ntest);
    if (ndup) atomicAdd(sink.dups, ndup);
    if (nhead && sink.heads) atomicAdd(sink.heads, nhead);
    if (LEARNED && nllook) {
      atomicAdd(pa.lhits, nlhit);
      atomicAdd(pa.llook, nllook);
    }
  }
}

// Decision for guard-band candidates: the float-float separation decides
// where it is certain (f2_sep_decide); the rest take the binary64 test with
// both vectors recomputed in the canonical arithmetic from the original
// coordinates (counted in n64).
// EQ4: each pair's radius r_ij from the two records' error radii (Eq. 4),
// its own window [r_ij - m, r_ij + m] and threshold 4 sin^2(r_ij/2).
template <bool EQ4>
__global__ void __launch_bounds__(kThreads) k_recheck(
    const uint2* __restrict__ band, const unsigned long long* __restrict__ nband_dev,
    uint64_t band_cap, const uint32_t* __restrict__ idxA, const uint32_t* __restrict__ idxB,
    const SrcRec* __restrict__ recA, const SrcRec* __restrict__ recB, double C, double r_lo,
    double r_hi, uint2* rows, unsigned long long* count, uint64_t cap,
    unsigned long long* __restrict__ n64, int* err) {
  uint64_t nb = *nband_dev;
  if (nb > band_cap) nb = band_cap;
  unsigned long long slow = 0;
  for (uint64_t b0 = (uint64_t)blockIdx.x * kThreads; b0 < nb; b0 += (uint64_t)gridDim.x * kThreads) {
    uint64_t q = b0 + threadIdx.x;
    bool hit = false;
    uint2 p = make_uint2(0u, 0u);
    if (q < nb) {
      p = band[q];  // entry indices, or source indices when idxA/idxB are null
      SrcRec a = recA[idxA ? idxA[p.x] : p.x], b = recB[idxB ? idxB[p.y] : p.y];
      double lo = r_lo, hi = r_hi, Cp = C;
      if (EQ4) {
        const double r = c_pair_radius(rec_err(a), rec_err(b));
        const double m = kSepRel * r + kSepAbs;
        lo = r - m;
        hi = r + m;
        Cp = c_threshold(r);
      }
      const int d = f2_sep_decide(a.ra, a.dec, b.ra, b.dec, lo, hi);
      if (d != 0) {
        hit = d > 0;
      } else {
        ++slow;
        double ax, ay, az, bx, by, bz;
        c_unitvec(a.ra, a.dec, &ax, &ay, &az);
        c_unitvec(b.ra, b.dec, &bx, &by, &bz);
        hit = c_chord2(ax, ay, az, bx, by, bz) <= Cp;
      }
    }
    warp_emit(hit, p.x, p.y, rows, count, cap, err);
  }
  for (int o = 16; o > 0; o >>= 1) slow += __shfl_down_sync(0xffffffffu, slow, o);
  if ((threadIdx.x & 31) == 0 && slow && n64) atomicAdd(n64, slow);
}

template <typename T>
__global__ void k_gather(const T* __restrict__ src, const uint32_t* __restrict__ perm, uint64_t n,
                         T* __restrict__ dst) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    dst[i] = src[perm[i]];
}

__global__ void k_iota(uint32_t* __restrict__ v, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    v[i] = (uint32_t)i;
}

}  // namespace hlc
