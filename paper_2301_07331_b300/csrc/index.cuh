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

// Offset table of keys sorted by (key >> shift), without atomics:
// T[q] = first entry whose key >> shift is >= q, for q in [0, S].  The slots
// are cut into tiles of kTabTile.  k_table_bounds finds the first entry of
// every tile boundary (one binary search each); k_table_tiles then builds a
// tile in shared memory: the first entry of each non-empty slot is marked
// while the tile's entries are read in order, and every slot takes the
// smallest mark at or after it (a suffix minimum whose carry is the next
// tile's first entry).  A tile holding more than kTabScan entries per slot
// searches each slot inside its window instead.  The tiles also count the
// non-empty slots (heads) and, when ndense is given, the entries of slots
// holding more than dense_above entries.
constexpr int kTabTile = 2048;    // slots per tile
constexpr int kTabThreads = 256;  // kTabTile / kTabThreads slots per thread
constexpr int kTabPer = kTabTile / kTabThreads;
constexpr uint64_t kTabScan = 8;

__device__ __forceinline__ uint64_t table_lb(const uint32_t* __restrict__ keys, int shift,
                                             uint64_t lo, uint64_t hi, uint64_t q) {
  while (lo < hi) {
    uint64_t mid = (lo + hi) >> 1;
    if ((uint64_t)(__ldg(keys + mid) >> shift) < q)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// bnd[j] = first entry whose key >> shift is >= j * kTabTile, j in [0, nt]:
// one warp per boundary, a 33-way search (each round the 32 lanes probe 32
// evenly spaced keys of the window and a ballot keeps the part holding the
// bound), so a bound costs about log33(m) dependent loads.
__global__ void k_table_bounds(const uint32_t* __restrict__ keys, uint64_t m, int shift,
                               uint64_t S, uint64_t nt, uint32_t* __restrict__ bnd) {
  const int lane = threadIdx.x & 31;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t j = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j <= nt;
       j += nwarps) {
    const uint64_t q = j * kTabTile;
    uint64_t lo = 0, hi = m;  // the bound lies in [lo, hi]
    if (q >= S) lo = m;
    while (hi - lo > 32) {
      const uint64_t p = lo + ((hi - lo) * (uint64_t)(lane + 1)) / 33;  // lo <= p < hi
      const unsigned below = __ballot_sync(0xffffffffu, (uint64_t)(__ldg(keys + p) >> shift) < q);
      const int c = __popc(below);  // the predicate holds on a prefix of the lanes
      const uint64_t nlo = c ? __shfl_sync(0xffffffffu, p, c - 1) + 1 : lo;
      const uint64_t nhi = c < 32 ? __shfl_sync(0xffffffffu, p, c < 32 ? c : 31) : hi;
      lo = nlo;
      hi = nhi;
    }
    const uint64_t p = lo + lane;
    const unsigned below =
        __ballot_sync(0xffffffffu, p < hi && (uint64_t)(__ldg(keys + p) >> shift) < q);
    if (lane == 0) bnd[j] = (uint32_t)(lo + __popc(below));
  }
}

__global__ void __launch_bounds__(kTabThreads) k_table_tiles(
    const uint32_t* __restrict__ keys, uint64_t m, int shift, uint64_t S, uint64_t nt,
    const uint32_t* __restrict__ bnd, uint32_t* __restrict__ T,
    unsigned long long* __restrict__ heads, uint32_t dense_above,
    unsigned long long* __restrict__ ndense) {
  __shared__ __align__(16) uint32_t sT[kTabTile];
  __shared__ uint32_t s_w[kTabThreads / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  unsigned long long h = 0, nd = 0;
  for (uint64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    const uint64_t q0 = tile * kTabTile;
    const uint64_t nq = (S + 1 - q0) < (uint64_t)kTabTile ? S + 1 - q0 : (uint64_t)kTabTile;
    const uint64_t lo = bnd[tile], hi = bnd[tile + 1];
    for (int i = t; i < kTabTile; i += kTabThreads) sT[i] = 0xFFFFFFFFu;
    __syncthreads();
    if (hi - lo <= kTabScan * kTabTile) {
      // entries [lo, hi) have slots in [q0, q0 + kTabTile): mark run heads
      for (uint64_t e = lo + t; e < hi; e += kTabThreads) {
        const uint32_t c = __ldg(keys + e) >> shift;
        if (e == 0 || (__ldg(keys + e - 1) >> shift) != c) sT[c - q0] = (uint32_t)e;
      }
    } else {
      for (uint64_t i = t; i < nq; i += kTabThreads) {
        const uint64_t q = q0 + i;
        sT[i] = (uint32_t)(q >= S ? m : table_lb(keys, shift, lo, hi, q));
      }
    }
    __syncthreads();
    // suffix minimum: thread t owns slots [kTabPer t, kTabPer (t + 1))
    static_assert(kTabPer == 8, "two 16-byte shared loads per thread");
    uint32_t v[kTabPer];
    {
      const uint4 x0 = reinterpret_cast<const uint4*>(sT)[2 * t];
      const uint4 x1 = reinterpret_cast<const uint4*>(sT)[2 * t + 1];
      v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
      v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
    }
    uint32_t cm = 0xFFFFFFFFu;
#pragma unroll
    for (int j = 0; j < kTabPer; ++j) cm = min(cm, v[j]);
    uint32_t incl = cm;  // min over this lane and the later lanes of the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_down_sync(0xffffffffu, incl, o);
      if (lane + o < 32) incl = min(incl, y);
    }
    if (lane == 0) s_w[warp] = incl;
    __syncthreads();
    uint32_t after = (uint32_t)hi;  // the next tile's first entry
    for (int w = warp + 1; w < kTabThreads / 32; ++w) after = min(after, s_w[w]);
    const uint32_t later = __shfl_down_sync(0xffffffffu, incl, 1);
    if (lane < 31) after = min(after, later);
    const uint32_t next_first = after;  // T of the slot after this thread's chunk
#pragma unroll
    for (int j = kTabPer - 1; j >= 0; --j) {
      after = min(after, v[j]);
      v[j] = after;
    }
#pragma unroll
    for (int j = 0; j < kTabPer; ++j) {
      const uint64_t i = (uint64_t)kTabPer * t + j;
      if (q0 + i < S) {  // slot q0 + i holds [T[q], T[q + 1])
        const uint32_t c = (j + 1 < kTabPer ? v[j + 1] : next_first) - v[j];
        h += c > 0;
        nd += c > dense_above ? c : 0;
      }
    }
    reinterpret_cast<uint4*>(sT)[2 * t] = make_uint4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<uint4*>(sT)[2 * t + 1] = make_uint4(v[4], v[5], v[6], v[7]);
    __syncthreads();
    for (uint64_t i = t; i < nq; i += kTabThreads) T[q0 + i] = sT[i];  // coalesced
    __syncthreads();  // sT and s_w are reused by the next tile
  }
  for (int o = 16; o > 0; o >>= 1) {
    h += __shfl_down_sync(0xffffffffu, h, o);
    nd += __shfl_down_sync(0xffffffffu, nd, o);
  }
  if (lane == 0) {
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

}  // namespace hlc
