// Cell offset index of a sorted key array (the calculation-block index of
// Sec. 4.2 / Fig. 7, in B300 form).
//
// The entries of a catalogue are sorted by fine cell key, so every cell is a
// contiguous range.  A dense table T at a coarser order Lt holds, for every
// coarse cell Q, the first entry whose key lies in Q or after it:
// T[Q] = #{entries with key >> s < Q}, s = 2 (L - Lt).  The range of a fine
// cell q is then found by a short binary search of the keys inside
// [T[q >> s], T[(q >> s) + 1]).  Lt is chosen so that the table has about as
// many slots as entries (one to a few keys per window).
#pragma once

#include "common.cuh"

namespace hlc {

struct CellIndex {
  const uint32_t* keys = nullptr;  // sorted fine keys
  const uint32_t* table = nullptr; // 12 * 4^Lt + 1 offsets
  int shift = 0;                   // 2 (L - Lt)
};

// Counts per coarse cell and the number of distinct fine keys (heads).  The
// keys are sorted, so equal coarse cells are contiguous: each warp adds one
// count per run of lanes that share a cell.
__global__ void k_coarse_hist(const uint32_t* __restrict__ keys, uint64_t n, int shift,
                              uint32_t* __restrict__ hist, unsigned long long* __restrict__ heads) {
  unsigned long long h = 0;
  const int lane = threadIdx.x & 31;
  for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x; i0 < n;
       i0 += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t i = i0 + threadIdx.x;
    bool live = i < n;
    uint32_t k = live ? keys[i] : 0xFFFFFFFFu;
    uint32_t prev = __shfl_up_sync(0xffffffffu, k, 1);
    if (live) h += (i == 0 || (lane > 0 ? prev : keys[i - 1]) != k);
    if (hist) {
      uint32_t q = k >> shift;
      uint32_t qp = __shfl_up_sync(0xffffffffu, q, 1);
      bool head = live && (lane == 0 || qp != q);
      unsigned hm = __ballot_sync(0xffffffffu, head);
      unsigned lm = __ballot_sync(0xffffffffu, live);
      if (head) {
        unsigned later = hm & ~((2u << lane) - 1u);  // next run head after this lane
        int end = later ? __ffs(later) - 1 : 32 - __clz(lm);
        atomicAdd(&hist[q], (uint32_t)(end - lane));
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) h += __shfl_down_sync(0xffffffffu, h, o);
  if ((threadIdx.x & 31) == 0 && h) atomicAdd(heads, h);
}

// Offset table of keys sorted by (key >> shift), without atomics or a scan:
// T[q] = first entry whose key >> shift is >= q, for q in [0, S].  Each
// thread fills 8 consecutive slots: one binary search for the first, then a
// gallop forward for each of the others.  It also counts the non-empty slots
// (heads) and, when ndense is given, the entries of slots holding more than
// dense_above entries.
__device__ __forceinline__ uint64_t gallop_lb(const uint32_t* __restrict__ keys, uint64_t m,
                                              int shift, uint64_t from, uint64_t q) {
  uint64_t step = 1, base = from;
  while (base + step <= m && (uint64_t)(__ldg(keys + base + step - 1) >> shift) < q) {
    base += step;
    step <<= 1;
  }
  uint64_t a = base, b = base + step <= m ? base + step : m;
  while (a < b) {
    uint64_t mid = (a + b) >> 1;
    if ((uint64_t)(__ldg(keys + mid) >> shift) < q)
      a = mid + 1;
    else
      b = mid;
  }
  return a;
}

__global__ void k_coarse_table(const uint32_t* __restrict__ keys, uint64_t m, int shift,
                               uint64_t S, uint32_t* __restrict__ T,
                               unsigned long long* __restrict__ heads, uint32_t dense_above,
                               unsigned long long* __restrict__ ndense) {
  unsigned long long h = 0, nd = 0;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t * 8 <= S;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t q0 = t * 8;
    uint64_t lo = 0, hi = m;
    while (lo < hi) {
      uint64_t mid = (lo + hi) >> 1;
      if ((uint64_t)(__ldg(keys + mid) >> shift) < q0)
        lo = mid + 1;
      else
        hi = mid;
    }
    T[q0] = (uint32_t)lo;
    // slots q0 .. q0 + 7 (the last one's end is the next thread's first)
    for (uint64_t q = q0 + 1; q <= q0 + 8; ++q) {
      const uint64_t nxt = q <= S ? gallop_lb(keys, m, shift, lo, q) : m;
      if (q < q0 + 8 && q <= S) T[q] = (uint32_t)nxt;
      if (q - 1 < S) {  // slot q - 1 holds [lo, nxt)
        const uint64_t c = nxt - lo;
        h += c > 0;
        nd += c > dense_above ? c : 0;
      }
      lo = nxt;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    h += __shfl_down_sync(0xffffffffu, h, o);
    nd += __shfl_down_sync(0xffffffffu, nd, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (h && heads) atomicAdd(heads, h);
    if (nd && ndense) atomicAdd(ndense, nd);
  }
}

// [begin, end) of the entries with key q inside the sorted window [lo, hi).
__device__ __forceinline__ uint2 cell_range_in(const uint32_t* __restrict__ keys, uint32_t lo,
                                               uint32_t hi, uint32_t q) {
  uint32_t a = lo, b = hi;
  while (a < b) {  // lower bound of q
    uint32_t mid = (a + b) >> 1;
    if (__ldg(keys + mid) < q)
      a = mid + 1;
    else
      b = mid;
  }
  uint32_t first = a;
  b = hi;
  while (a < b) {  // upper bound of q
    uint32_t mid = (a + b) >> 1;
    if (__ldg(keys + mid) <= q)
      a = mid + 1;
    else
      b = mid;
  }
  return make_uint2(first, a);
}

// [begin, end) of the entries with key q.
__device__ __forceinline__ uint2 cell_range(const CellIndex& ix, uint32_t q) {
  uint32_t Q = q >> ix.shift;
  return cell_range_in(ix.keys, __ldg(ix.table + Q), __ldg(ix.table + Q + 1), q);
}

// Order of the coarse table for m entries at fine order L.
inline int coarse_table_order(uint64_t m, int L) {
  int lt = 0;
  while (lt < L && 12ull * (1ull << (2 * lt)) < m) ++lt;
  return lt;
}

// Highest bit in which the ids differ (OR of id ^ id[0]).
__global__ void k_id_diff(const uint64_t* __restrict__ id, uint64_t n,
                          unsigned long long* __restrict__ out) {
  unsigned long long acc = 0;
  if (n == 0) return;
  uint64_t first = id[0];
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    acc |= id[i] ^ first;
  for (int o = 16; o > 0; o >>= 1) acc |= __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicOr(out, acc);
}

}  // namespace hlc
