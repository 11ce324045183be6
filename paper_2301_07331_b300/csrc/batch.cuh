// Batched cross-match: many independent (A, B, r, order) jobs of uneven size
// matched by one fixed launch sequence.
//
// Every entry carries a composite key (job << cell_bits) | cell, so one radix
// sort groups all jobs' entries by job and, inside a job, by cell.  Catalogue
// B of job j gets its own offset table over the cell range it actually
// occupies, at order L_j - k_j with k_j chosen so the table has about as many
// slots as the job has sources; all tables live in one array whose global
// exclusive scan gives absolute entry offsets directly.  The pair test is one
// persistent launch in which warps pull chunks of A entries from an atomic
// work counter, so heavy and light jobs share the GPU without per-job
// launches.  Complete 8-neighbour mode.
#pragma once

#include "canon.cuh"
#include "common.cuh"
#include "fastpix.cuh"
#include "fp32.cuh"
#include "match.cuh"
#include "output.cuh"

namespace hlc {

struct JobDev {
  const double* ra[2];   // [0] = A, [1] = B
  const double* dec[2];
  const uint64_t* id[2];
  uint64_t n[2];         // sources of A and B
  uint64_t off[2];       // first global entry of A and B
  int L;                 // fine order of the job
  PixConst K;
  double C;              // canonical chord^2 threshold
  double r_lo, r_hi;     // separations (arcsec) left to the binary64 recheck
  float lo32, hi32;      // guard band
  uint64_t toff;         // first slot of the job's B table
  uint32_t tbase;        // first coarse cell covered (order L - tk)
  uint32_t tsize;        // coarse cells covered + 1
  int tk;                // table order = L - tk
};

// Job of global entry i on side s (offsets ascending, njobs + 1 of them).
__device__ __forceinline__ uint32_t job_of(const uint64_t* __restrict__ off, uint32_t njobs,
                                           uint64_t i) {
  uint32_t lo = 0, hi = njobs;  // find last j with off[j] <= i
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= i)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// The composite keys' digit histograms (hist_np passes of 8 bits from bit 0,
// in shared memory, flushed once per block) for the radix sort, which then
// makes no pass of its own over the keys.  The upper digits hold the job,
// the same for most lanes of a warp: a digit common to every counted lane is
// added once by the first of them.
constexpr int kBHistPasses = 8;
__device__ __forceinline__ void bhist_count(uint32_t (*sh)[256], int np, bool counted,
                                            uint64_t k) {
  const unsigned m = __ballot_sync(0xffffffffu, counted);
  if (!m) return;
  const int first = __ffs(m) - 1;
  for (int p = 0; p < np; ++p) {
    const uint32_t dig = (uint32_t)(k >> (8 * p)) & 255u;
    const uint32_t d0 = __shfl_sync(0xffffffffu, dig, first);
    if (__ballot_sync(0xffffffffu, counted && dig == d0) == m) {
      if ((int)(threadIdx.x & 31) == first) atomicAdd(&sh[p][d0], (uint32_t)__popc(m));
    } else if (counted) {
      atomicAdd(&sh[p][dig], 1u);
    }
  }
}

__device__ __forceinline__ void bhist_flush(uint32_t (*sh)[256], int np,
                                            uint32_t* __restrict__ hist) {
  __syncthreads();
  for (int t = threadIdx.x; t < np * 256; t += blockDim.x) {
    const uint32_t c = (&sh[0][0])[t];
    if (c) atomicAdd(hist + t, c);
  }
}

// (hist, when given: the digit histograms of the keys written for good; the
// queued ones are counted by k_bprep_fallback)
template <bool FAST>
__global__ void k_bprep_keys(const JobDev* __restrict__ jobs, const uint64_t* __restrict__ off,
                             uint32_t njobs, int side, uint64_t total, int cell_bits,
                             uint64_t* __restrict__ key, uint32_t* __restrict__ idx,
                             SrcRec* __restrict__ rec, uint32_t* __restrict__ slow,
                             unsigned long long* __restrict__ nslow, int* __restrict__ err,
                             uint32_t* __restrict__ hist = nullptr, int hist_np = 0) {
  __shared__ uint32_t sh[kBHistPasses][256];
  if (hist) {
    for (int t = threadIdx.x; t < kBHistPasses * 256; t += blockDim.x) (&sh[0][0])[t] = 0u;
    __syncthreads();
  }
  // (a thread's next source -- its job, coordinates and id -- is looked up
  // and loaded while the current one is processed)
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint32_t pj = 0;
  double pa = 0.0, pd = 0.0;
  uint64_t pid = 0;
  auto fetch = [&](uint64_t ii) {
    if (ii < total) {
      pj = job_of(off, njobs, ii);
      const JobDev& Jn = jobs[pj];
      const uint64_t ln = ii - Jn.off[side];
      pa = Jn.ra[side][ln];
      pd = Jn.dec[side][ln];
      pid = Jn.id[side][ln];
    }
  };
  fetch((uint64_t)blockIdx.x * blockDim.x + threadIdx.x);
  for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x; i0 < total; i0 += stride) {
    uint64_t i = i0 + threadIdx.x;
    bool defer = false;
    const uint32_t j = pj;
    double a = pa, d = pd;
    const uint64_t idv = pid;
    uint64_t kw = 0;  // the key written
    fetch(i + stride);
    if (i < total) {
      const JobDev& J = jobs[j];
      uint32_t k = 0;
      if (!(bits_finite(a) && bits_abs_le(d, 90.0))) {
        atomicOr(err, DERR_INPUT);
      } else {
        if (!bits_in_ra_range(a)) a = c_norm_ra(a);
        if (FAST) {
          FastDec fd = f_dec_part(split_f64(d));
          defer = !f_pix(split_f64(a), fd, J.L, J.K, &k);
        } else {
          k = c_ang2pix(a, d, J.L);
        }
      }
      kw = ((uint64_t)j << cell_bits) | k;
      key[i] = kw;
      idx[i] = (uint32_t)i;
      SrcRec r;  // (the payload gathers one 32-byte record, not three arrays)
      r.ra = a;
      r.dec = d;
      r.id = idv;
      r.pad = 0;
      rec[i] = r;
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
    // (an invalid source keeps cell 0 and counts as such)
    if (hist) bhist_count(sh, hist_np, i < total && !defer, kw);
  }
  if (hist) bhist_flush(sh, hist_np, hist);
}

__global__ void k_bprep_fallback(const JobDev* __restrict__ jobs, const uint64_t* __restrict__ off,
                                 uint32_t njobs, int side, int cell_bits,
                                 const uint32_t* __restrict__ slow,
                                 const unsigned long long* __restrict__ nslow,
                                 uint64_t* __restrict__ key, uint32_t* __restrict__ hist = nullptr,
                                 int hist_np = 0) {
  __shared__ uint32_t sh[kBHistPasses][256];
  if (hist) {
    for (int t = threadIdx.x; t < kBHistPasses * 256; t += blockDim.x) (&sh[0][0])[t] = 0u;
    __syncthreads();
  }
  const uint64_t ns = *nslow;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  // (every lane runs the same number of rounds, for the warp-wide counting)
  for (uint64_t q0 = (uint64_t)blockIdx.x * blockDim.x; q0 < ns; q0 += stride) {
    const uint64_t q = q0 + threadIdx.x;
    uint64_t kw = 0;
    if (q < ns) {
      uint32_t i = slow[q];
      uint32_t j = job_of(off, njobs, i);
      const JobDev& J = jobs[j];
      uint64_t l = i - J.off[side];
      kw = ((uint64_t)j << cell_bits) |
           ff_or_c_ang2pix(c_norm_ra(J.ra[side][l]), J.dec[side][l], J.L);
      key[i] = kw;
    }
    if (hist) bhist_count(sh, hist_np, q < ns, kw);
  }
  if (hist) bhist_flush(sh, hist_np, hist);
}

// Sorted payload from the records the prep wrote in input order (RA
// normalised): one 32-byte gather per entry.
template <bool FP32>
// (iddiff, when given: the OR of id ^ (an id of the catalogue) over its
// entries, the bits in which its ids differ, for the output bucketing)
__global__ void k_bpayload(const SrcRec* __restrict__ rec, const uint32_t* __restrict__ idx,
                           uint64_t m, float4* __restrict__ v32, double2* __restrict__ rd,
                           double* __restrict__ vx, double* __restrict__ vy,
                           double* __restrict__ vz, uint64_t* __restrict__ id_s,
                           unsigned long long* __restrict__ iddiff = nullptr) {
  const uint64_t id0 = (iddiff && m) ? rec[idx[0]].id : 0ull;
  unsigned long long idacc = 0;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const SrcRec r = rec[idx[e]];
    idacc |= r.id ^ id0;
    if (FP32) {
      v32[e] = fp32_unitvec(r.ra, r.dec);
      rd[e] = make_double2(r.ra, r.dec);
    } else {
      double x, y, z;
      c_unitvec(r.ra, r.dec, &x, &y, &z);
      vx[e] = x;
      vy[e] = y;
      vz[e] = z;
    }
    id_s[e] = r.id;
  }
  id_span_flush(iddiff, idacc);
}

// Autotuner inputs, per job: the sum of the B unit vectors (FP32) and, in a
// second pass, the smallest cosine between a B source and the job's mean
// direction -- the spherical cap the job's B catalogue occupies.  One warp
// per job reads an evenly spaced sample of at most about kCapSamples of its
// B sources (the estimate only picks the job's order).
constexpr uint64_t kCapSamples = 1024;

__device__ __forceinline__ float4 job_b_vec(const JobDev& J, uint64_t l) {
  double a = J.ra[1][l], d = J.dec[1][l];
  if (!(bits_finite(a) && bits_abs_le(d, 90.0))) return make_float4(0.f, 0.f, 0.f, 0.f);
  if (!bits_in_ra_range(a)) a = c_norm_ra(a);
  return fp32_unitvec(a, d);
}

__global__ void k_bjob_mean(const JobDev* __restrict__ jobs, uint32_t njobs,
                            float* __restrict__ acc) {
  const int lane = threadIdx.x & 31;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t j = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < njobs; j += nw) {
    const JobDev& J = jobs[j];
    const uint64_t n = J.n[1];
    const uint64_t step = n > kCapSamples ? n / kCapSamples : 1;
    float sx = 0.f, sy = 0.f, sz = 0.f;
    for (uint64_t l = lane * step; l < n; l += 32 * step) {
      const float4 u = job_b_vec(J, l);
      sx += u.x;
      sy += u.y;
      sz += u.z;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
      sz += __shfl_xor_sync(0xffffffffu, sz, o);
    }
    if (lane == 0) {
      acc[3 * j] = sx;
      acc[3 * j + 1] = sy;
      acc[3 * j + 2] = sz;
    }
  }
}

// (1 - cos, the largest over the sample, as float bits)
__global__ void k_bjob_cap(const JobDev* __restrict__ jobs, uint32_t njobs,
                           const float* __restrict__ dir, unsigned int* __restrict__ cap) {
  const int lane = threadIdx.x & 31;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t j = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < njobs; j += nw) {
    const JobDev& J = jobs[j];
    const uint64_t n = J.n[1];
    const uint64_t step = n > kCapSamples ? n / kCapSamples : 1;
    const float dx = dir[3 * j], dy = dir[3 * j + 1], dz = dir[3 * j + 2];
    float om = 0.f;
    for (uint64_t l = lane * step; l < n; l += 32 * step) {
      const float4 u = job_b_vec(J, l);
      if (u.x == 0.f && u.y == 0.f && u.z == 0.f) continue;  // invalid input
      om = fmaxf(om, fmaxf(1.0f - (u.x * dx + u.y * dy + u.z * dz), 0.0f));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) om = fmaxf(om, __shfl_xor_sync(0xffffffffu, om, o));
    if (lane == 0) cap[j] = __float_as_uint(om);
  }
}

// First and last composite key of every job's sorted B entries.
__global__ void k_job_first_last(const uint64_t* __restrict__ key,
                                 const uint64_t* __restrict__ off, uint32_t njobs,
                                 uint64_t* __restrict__ fl) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < njobs;
       j += gridDim.x * blockDim.x) {
    const uint64_t a = off[j], b = off[j + 1];
    fl[2 * j] = a < b ? key[a] : 0ull;
    fl[2 * j + 1] = a < b ? key[b - 1] : 0ull;
  }
}

// ---- per-job B offset tables -------------------------------------------------
__global__ void k_btable_hist(const uint64_t* __restrict__ key, uint64_t m, int cell_bits,
                              const JobDev* __restrict__ jobs, uint32_t* __restrict__ counts) {
  // keys are sorted: equal slots are contiguous, one atomic per run of lanes
  const uint64_t cmask = (1ull << cell_bits) - 1;
  const int lane = threadIdx.x & 31;
  for (uint64_t e0 = (uint64_t)blockIdx.x * blockDim.x; e0 < m;
       e0 += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t e = e0 + threadIdx.x;
    uint32_t slot = 0xFFFFFFFFu;
    if (e < m) {
      uint64_t k = key[e];
      uint32_t j = (uint32_t)(k >> cell_bits);
      const JobDev& J = jobs[j];
      slot = (uint32_t)(J.toff + (uint32_t)((k & cmask) >> (2 * J.tk)) - J.tbase);
    }
    const uint32_t sp = __shfl_up_sync(0xffffffffu, slot, 1);
    const bool head = slot != 0xFFFFFFFFu && (lane == 0 || sp != slot);
    const unsigned hm = __ballot_sync(0xffffffffu, head);
    const unsigned lm = __ballot_sync(0xffffffffu, slot != 0xFFFFFFFFu);
    if (head) {
      const unsigned later = hm & ~((2u << lane) - 1u);
      const int end = later ? __ffs(later) - 1 : 32 - __clz(lm);
      atomicAdd(counts + slot, (uint32_t)(end - lane));
    }
  }
}

// The fields of a job the pair test needs, held in registers.
struct JobTab {
  int L, tk;
  uint32_t tbase, tsize;
  uint64_t toff;
  double C;
  float lo32, hi32;
};

__device__ __forceinline__ JobTab load_job(const JobDev* __restrict__ jobs, uint32_t j) {
  const JobDev* J = jobs + j;
  JobTab t;
  t.L = J->L;
  t.tk = J->tk;
  t.tbase = J->tbase;
  t.tsize = J->tsize;
  t.toff = J->toff;
  t.C = J->C;
  t.lo32 = J->lo32;
  t.hi32 = J->hi32;
  return t;
}

// [begin, end) of the B entries of job j in fine cell q (composite keys).
__device__ __forceinline__ uint2 bcell_range(const uint64_t* __restrict__ keyB,
                                             const uint32_t* __restrict__ table,
                                             const JobTab& J, uint32_t j, int cell_bits,
                                             uint32_t q) {
  uint32_t Q = q >> (2 * J.tk);
  if (Q < J.tbase || Q - J.tbase + 1 >= J.tsize) return make_uint2(0u, 0u);
  uint64_t slot = J.toff + (Q - J.tbase);
  uint32_t a = __ldg(table + slot), hi = __ldg(table + slot + 1), b = hi;
  uint64_t kq = ((uint64_t)j << cell_bits) | q;
  while (a < b) {
    uint32_t mid = (a + b) >> 1;
    if (__ldg(keyB + mid) < kq)
      a = mid + 1;
    else
      b = mid;
  }
  uint32_t first = a;
  b = hi;
  while (a < b) {
    uint32_t mid = (a + b) >> 1;
    if (__ldg(keyB + mid) <= kq)
      a = mid + 1;
    else
      b = mid;
  }
  return make_uint2(first, a);
}

struct BPairArgs {
  uint64_t mA;
  const uint64_t* keyA;
  const uint64_t* keyB;
  const uint32_t* table;
  const JobDev* jobs;
  int cell_bits;
  const double *axv, *ayv, *azv, *bxv, *byv, *bzv;
  const float4 *a32, *b32;
  uint32_t sparse_cell;
  unsigned long long* work;  // chunk counter
  const uint8_t* tiled;      // A entries taken by the dense-cell kernel, or null
};

// Persistent pair test: each warp takes chunks of 32 A entries from an atomic
// work counter until all entries of all jobs are done.  As in k_pair, a lane
// in a sparse region reads the (at most 4) table cells covering its fine 3x3
// block whole, rows are staged per warp in shared memory, and lanes whose A
// entry the dense-cell kernel takes (tiled) stay idle.  In a dense table cell
// the 9 fine ranges (two binary searches each) are the same for every A
// entry of a cell: they are looked up once per run of equal keys in the
// chunk, the runs' lookups spread over the warp's lanes, and read back from
// shared memory by each lane of the run.
__device__ __forceinline__ int nth_set_bit(unsigned m, int r) {  // r < popc(m), 0-based
  int pos = 0;
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const int c = __popc(m & ((1u << w) - 1u));
    if (r >= c) {
      r -= c;
      m >>= w;
      pos += w;
    }
  }
  return pos;
}

template <bool FP32>
__global__ void __launch_bounds__(kThreads) k_bpair(const BPairArgs pa, PairSink sink) {
  const uint64_t nchunks = (pa.mA + 31) / 32;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const uint64_t cmask = (1ull << pa.cell_bits) - 1;
  unsigned long long ntest = 0;
  constexpr int kRowCap = 256, kBandCap = FP32 ? 128 : 32;
  __shared__ uint2 s_rows[kThreads / 32][kRowCap];
  __shared__ uint2 s_band[kThreads / 32][kBandCap];
  __shared__ uint32_t s_nbc[kThreads / 32][32 * 9];  // 9 cells of each run head
  __shared__ uint2 s_rng[kThreads / 32][32 * 9];     // and their B ranges
  __shared__ uint32_t s_job[kThreads / 32][32];
  WarpRows<kRowCap> wrows{s_rows[warp]};
  WarpRows<kBandCap> wband{s_band[warp]};
  for (;;) {
    unsigned long long chunk = 0;
    if (lane == 0) chunk = atomicAdd(pa.work, 1ull);
    chunk = __shfl_sync(0xffffffffu, chunk, 0);
    if (chunk >= nchunks) break;
    uint64_t k = chunk * 32 + lane;
    bool live = k < pa.mA;
    if (live && pa.tiled && pa.tiled[k]) live = false;
    uint32_t j = 0, cell = 0;
    JobTab J = {0, 0, 0u, 0u, 0ull, 0.0, 0.f, 0.f};
    const uint64_t key = live ? pa.keyA[k] : ~0ull;
    if (live) {
      j = (uint32_t)(key >> pa.cell_bits);
      cell = (uint32_t)(key & cmask);
      J = load_job(pa.jobs, j);
    }
    double ax = 0, ay = 0, az = 0;
    float4 a4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (live) {
      if (FP32)
        a4 = pa.a32[k];
      else {
        ax = pa.axv[k]; ay = pa.ayv[k]; az = pa.azv[k];
      }
    }
    uint32_t nb[9];
#pragma unroll
    for (int s = 0; s < 9; ++s) nb[s] = kNoCell;
    bool coarse = false;
    if (live) {
      uint32_t Q = cell >> (2 * J.tk);
      if (FP32 && J.tk > 0 && Q >= J.tbase && Q - J.tbase + 1 < J.tsize) {
        uint64_t slot = J.toff + (Q - J.tbase);
        if (__ldg(pa.table + slot + 1) - __ldg(pa.table + slot) <= pa.sparse_cell)
          coarse = parent_cover4(cell, J.L, J.tk, nb);
      }
      if (!coarse) cell_neighbourhood9(cell, J.L, nb);
    }
    // the fine ranges of the runs that need them: one lookup per (run, cell)
    const uint64_t kprev = __shfl_up_sync(0xffffffffu, key, 1);
    const bool head = live && (lane == 0 || kprev != key);
    const bool fine = live && !coarse;  // (the same for every lane of a run)
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    const unsigned fine_heads = __ballot_sync(0xffffffffu, head && fine);
    if (fine_heads) {
      if (head && fine) {
#pragma unroll
        for (int s = 0; s < 9; ++s) s_nbc[warp][lane * 9 + s] = nb[s];
        s_job[warp][lane] = j;
      }
      __syncwarp();
      const int ntask = 9 * __popc(fine_heads);
      for (int t = lane; t < ntask; t += 32) {
        const int r = t / 9, s = t - 9 * r;
        const int h = nth_set_bit(fine_heads, r);
        const uint32_t c = s_nbc[warp][h * 9 + s];
        uint2 rg = make_uint2(0u, 0u);
        if (c != kNoCell) {
          const uint32_t jh = s_job[warp][h];
          rg = bcell_range(pa.keyB, pa.table, load_job(pa.jobs, jh), jh, pa.cell_bits, c);
        }
        s_rng[warp][h * 9 + s] = rg;
      }
      __syncwarp();
    }
    // (a live lane's run head: the highest head at or below it)
    const int myhead = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
    uint32_t rb[9], re[9];
    uint32_t total = 0;
#pragma unroll
    for (int s = 0; s < 9; ++s) {
      uint2 r = make_uint2(0u, 0u);
      if (nb[s] != kNoCell) {
        if (coarse) {
          uint32_t c = nb[s];
          if (c >= J.tbase && c - J.tbase + 1 < J.tsize) {
            uint64_t slot = J.toff + (c - J.tbase);
            r = make_uint2(__ldg(pa.table + slot), __ldg(pa.table + slot + 1));
          }
        } else {
          r = s_rng[warp][myhead * 9 + s];
        }
      }
      rb[s] = r.x;
      re[s] = r.y;
      total += r.y - r.x;
    }
    ntest += total;
    const uint32_t maxT = __reduce_max_sync(0xffffffffu, total);
    uint32_t cur = rb[0], end = re[0];
    constexpr int U = 4;
    for (uint32_t t = 0; t < maxT; t += U) {
      uint32_t jj[U];
      bool act[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        act[u] = t + u < total;
        jj[u] = 0;
        if (act[u]) {
          while (cur >= end) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
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
        for (int u = 0; u < U; ++u) bb[u] = act[u] ? __ldg(pa.b32 + jj[u]) : a4;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          float dx = a4.x - bb[u].x, dy = a4.y - bb[u].y, dz = a4.z - bb[u].z;
          float s2 = dx * dx;
          s2 = fmaf(dy, dy, s2);
          s2 = fmaf(dz, dz, s2);
          hit[u] = act[u] && s2 <= J.lo32;
          band[u] = act[u] && !hit[u] && s2 <= J.hi32;
          anyv |= hit[u] || band[u];
        }
      } else {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          hit[u] = act[u] &&
                   c_chord2(ax, ay, az, pa.bxv[jj[u]], pa.byv[jj[u]], pa.bzv[jj[u]]) <= J.C;
          band[u] = false;
          anyv |= hit[u];
        }
      }
      if (__any_sync(0xffffffffu, anyv)) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          wrows.add(hit[u], (uint32_t)k, jj[u]);
          if (FP32) wband.add(band[u], (uint32_t)k, jj[u]);
        }
        if (wrows.fill > kRowCap - 32 * U) wrows.flush(sink.rows, sink.count, sink.cap, sink.err);
        if (FP32 && wband.fill > kBandCap - 32 * U)
          wband.flush(sink.band, sink.band_count, sink.band_cap, sink.err);
      }
    }
  }
  wrows.flush(sink.rows, sink.count, sink.cap, sink.err);
  if (FP32) wband.flush(sink.band, sink.band_count, sink.band_cap, sink.err);
  for (int o = 16; o > 0; o >>= 1) ntest += __shfl_down_sync(0xffffffffu, ntest, o);
  if (lane == 0 && ntest) atomicAdd(sink.tests, ntest);
}

__global__ void __launch_bounds__(kThreads) k_brecheck(
    const uint2* __restrict__ band, const unsigned long long* __restrict__ nband_dev,
    uint64_t band_cap, const uint64_t* __restrict__ keyA, int cell_bits,
    const JobDev* __restrict__ jobs, const double2* __restrict__ rdA,
    const double2* __restrict__ rdB, uint2* rows, unsigned long long* count, uint64_t cap,
    unsigned long long* __restrict__ n64, int* err) {
  uint64_t nb = *nband_dev;
  if (nb > band_cap) nb = band_cap;
  unsigned long long slow = 0;
  for (uint64_t b0 = (uint64_t)blockIdx.x * kThreads; b0 < nb; b0 += (uint64_t)gridDim.x * kThreads) {
    uint64_t q = b0 + threadIdx.x;
    bool hit = false;
    uint2 p = make_uint2(0u, 0u);
    if (q < nb) {
      p = band[q];
      const JobDev* J = jobs + (keyA[p.x] >> cell_bits);
      double2 a = rdA[p.x], b = rdB[p.y];
      const int d = f2_sep_decide(a.x, a.y, b.x, b.y, J->r_lo, J->r_hi);
      if (d != 0) {
        hit = d > 0;
      } else {
        ++slow;
        double ax, ay, az, bx, by, bz;
        c_unitvec(a.x, a.y, &ax, &ay, &az);
        c_unitvec(b.x, b.y, &bx, &by, &bz);
        hit = c_chord2(ax, ay, az, bx, by, bz) <= J->C;
      }
    }
    warp_emit(hit, p.x, p.y, rows, count, cap, err);
  }
  for (int o = 16; o > 0; o >>= 1) slow += __shfl_down_sync(0xffffffffu, slow, o);
  if ((threadIdx.x & 31) == 0 && slow && n64) atomicAdd(n64, slow);
}

// Rows per job (lanes of a warp that share a job add once).
__global__ void k_job_rows(const uint2* __restrict__ rows, uint64_t M,
                           const uint64_t* __restrict__ keyA, int cell_bits,
                           uint32_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  for (uint64_t m0 = (uint64_t)blockIdx.x * blockDim.x; m0 < M;
       m0 += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t m = m0 + threadIdx.x;
    const bool live = m < M;
    const uint32_t j = live ? (uint32_t)(keyA[rows[m].x] >> cell_bits) : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(0xffffffffu, j);
    if (live && lane == __ffs(peers) - 1) atomicAdd(&cnt[j], (uint32_t)__popc(peers));
  }
}

// Rows of a batched match: ids, separation, job; bucket from the job table.
template <bool FP32>
__global__ void k_brows(const uint2* __restrict__ rows, uint64_t M,
                        const uint64_t* __restrict__ keyA, int cell_bits,
                        const uint64_t* __restrict__ idA, const uint64_t* __restrict__ idB,
                        const double* __restrict__ axv, const double* __restrict__ ayv,
                        const double* __restrict__ azv, const double* __restrict__ bxv,
                        const double* __restrict__ byv, const double* __restrict__ bzv,
                        const double2* __restrict__ rdA, const double2* __restrict__ rdB,
                        int want_sep, OutRow* __restrict__ out, const uint4* __restrict__ jb,
                        uint32_t* __restrict__ bhist) {
  for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M;
       m += (uint64_t)gridDim.x * blockDim.x) {
    uint2 p = rows[m];
    OutRow o;
    o.a = idA[p.x];
    o.b = idB[p.y];
    o.job = (uint32_t)(keyA[p.x] >> cell_bits);
    o.pad = 0;
    o.s = 0.0;
    if (bhist)  // the row's rank in its bucket, for the scatter
      o.pad = atomicAdd(&bhist[row_bucket(o, 0, 0u, jb)], 1u);
    if (want_sep) {
      double sv;
      if (FP32) {
        double2 u = rdA[p.x], w = rdB[p.y];
        sv = sep_arcsec_f2(u.x, u.y, w.x, w.y);
        if (sv < 0.0) sv = sep_arcsec_haversine(u.x, u.y, w.x, w.y);
      } else {
        sv = sep_arcsec_from_chord2(
            c_chord2(axv[p.x], ayv[p.x], azv[p.x], bxv[p.y], byv[p.y], bzv[p.y]));
      }
      o.s = sv;
    }
    out[m] = o;
  }
}

}  // namespace hlc
