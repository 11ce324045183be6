// Single-pass scans with decoupled look-back: an exclusive prefix sum and the
// run-length cell table (unique cells and their start offsets) of sorted keys.
// The cell table is the "HEALPix data block" index of Sec. 4.2 / Fig. 7: each
// non-empty cell becomes a range [start[c], start[c+1]) of the sorted arrays.
#pragma once

#include "common.cuh"
#include "sort.cuh"

namespace hlc {
namespace sc {

constexpr int kBlock = 256;
constexpr int kIpt = 8;
constexpr int kTile = kBlock * kIpt;
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr long long kSpinLimit = 1ll << 26;

// Called by the 32 lanes of the tile's first warp: publish the tile
// aggregate, walk back to the nearest inclusive prefix 32 predecessors at a
// time (one load per lane, a ballot finds the nearest inclusive one, a warp
// sum adds the aggregates up to it), publish this tile's inclusive prefix
// and return its exclusive prefix (to every lane).
__device__ __forceinline__ unsigned long long lookback_prefix(uint32_t tile,
                                                              unsigned long long agg,
                                                              unsigned long long* lb, int* err) {
  const int lane = threadIdx.x & 31;
  if (tile == 0) {
    if (lane == 0) st_release_u64(lb, kFlagInc | agg);
    return 0;
  }
  if (lane == 0) st_release_u64(lb + tile, kFlagAgg | agg);
  unsigned long long excl = 0;
  long long spins = 0;
  int64_t j = (int64_t)tile - 1;  // predecessor read by lane 0
  while (true) {
    const int64_t idx = j - lane;
    // (before tile 0: an inclusive prefix of 0)
    const unsigned long long w = idx >= 0 ? ld_acquire_u64(lb + idx) : kFlagInc;
    const unsigned long long f = w & ~kValMask;
    const unsigned inc = __ballot_sync(0xffffffffu, f == kFlagInc);
    const unsigned wait = __ballot_sync(0xffffffffu, f == 0);
    const int last = inc ? __ffs(inc) - 1 : 31;  // lanes 0..last are needed
    const unsigned need = last == 31 ? 0xffffffffu : (2u << last) - 1u;
    if (wait & need) {
      if (++spins > spin_limit(kSpinLimit)) {
        if (lane == 0) atomicOr(err, DERR_TIMEOUT);
        break;
      }
      continue;
    }
    unsigned long long v = lane <= last ? (w & kValMask) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    excl += v;
    if (inc) break;
    j -= 32;
  }
  if (lane == 0) st_release_u64(lb + tile, kFlagInc | (excl + agg));
  return excl;
}

struct ScanSmem {
  unsigned long long ws[kBlock / 32];
  unsigned long long base;
  uint32_t tile;
};

// out[i] = sum_{k<i} in[i]; *total = sum of all.
template <typename OutT>
__global__ void __launch_bounds__(kBlock) k_scan_excl(const uint32_t* __restrict__ in,
                                                      OutT* __restrict__ out, uint64_t n,
                                                      unsigned long long* lb, uint32_t* ctr,
                                                      unsigned long long* total, int* err) {
  __shared__ ScanSmem S;
  const int t = threadIdx.x;
  if (t == 0) S.tile = atomicAdd(ctr, 1u);
  __syncthreads();
  const uint32_t tile = S.tile;
  const uint64_t e0 = (uint64_t)tile * kTile + (uint64_t)t * kIpt;
  uint32_t v[kIpt];
  unsigned long long sum = 0;
  if (e0 + kIpt <= n) {  // two 16-byte loads (the array is 256-byte aligned)
    uint4 x = *reinterpret_cast<const uint4*>(in + e0);
    uint4 y = *reinterpret_cast<const uint4*>(in + e0 + 4);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
  } else {
#pragma unroll
    for (int i = 0; i < kIpt; ++i) v[i] = (e0 + i < n) ? in[e0 + i] : 0u;
  }
#pragma unroll
  for (int i = 0; i < kIpt; ++i) sum += v[i];
  unsigned long long tot;
  unsigned long long pre = rs::block_excl_scan(sum, S.ws, &tot);
  if (t < 32) {
    const unsigned long long b = lookback_prefix(tile, tot, lb, err);
    if (t == 0) S.base = b;
  }
  __syncthreads();
  unsigned long long run = S.base + pre;
  OutT o[kIpt];
#pragma unroll
  for (int i = 0; i < kIpt; ++i) {
    o[i] = (OutT)run;
    run += v[i];
  }
  if (sizeof(OutT) == 4 && e0 + kIpt <= n) {
    uint4* dst = reinterpret_cast<uint4*>(out + e0);
    dst[0] = make_uint4((uint32_t)o[0], (uint32_t)o[1], (uint32_t)o[2], (uint32_t)o[3]);
    dst[1] = make_uint4((uint32_t)o[4], (uint32_t)o[5], (uint32_t)o[6], (uint32_t)o[7]);
  } else {
#pragma unroll
    for (int i = 0; i < kIpt; ++i)
      if (e0 + i < n) out[e0 + i] = o[i];
  }
  if (e0 < n && e0 + kIpt >= n) *total = run;  // the thread holding element n-1
}

// Cell table of sorted keys at a coarser level (key >> shift): cell_of[e] =
// index of e's cell, uniq[c] = cell id, start[c] = first element of cell c,
// start[m] = n and *m_out = m.
__global__ void __launch_bounds__(kBlock) k_cell_rle(const uint32_t* __restrict__ keys,
                                                     uint64_t n, int shift,
                                                     uint32_t* __restrict__ cell_of,
                                                     uint32_t* __restrict__ uniq,
                                                     uint32_t* __restrict__ start,
                                                     unsigned long long* lb, uint32_t* ctr,
                                                     unsigned long long* m_out, int* err) {
  __shared__ ScanSmem S;
  const int t = threadIdx.x;
  if (t == 0) S.tile = atomicAdd(ctr, 1u);
  __syncthreads();
  const uint32_t tile = S.tile;
  const uint64_t e0 = (uint64_t)tile * kTile + (uint64_t)t * kIpt;
  uint32_t c[kIpt];
  bool head[kIpt];
  unsigned long long sum = 0;
  uint32_t prev = (e0 > 0 && e0 - 1 < n) ? (keys[e0 - 1] >> shift) : 0xFFFFFFFFu;
#pragma unroll
  for (int i = 0; i < kIpt; ++i) {
    if (e0 + i < n) {
      c[i] = keys[e0 + i] >> shift;
      head[i] = (e0 + i == 0) || (c[i] != prev);
      prev = c[i];
    } else {
      head[i] = false;
    }
    sum += head[i];
  }
  unsigned long long tot;
  unsigned long long pre = rs::block_excl_scan(sum, S.ws, &tot);
  if (t < 32) {
    const unsigned long long b = lookback_prefix(tile, tot, lb, err);
    if (t == 0) S.base = b;
  }
  __syncthreads();
  unsigned long long run = S.base + pre;  // heads before element e0
#pragma unroll
  for (int i = 0; i < kIpt; ++i) {
    uint64_t e = e0 + i;
    if (e < n) {
      if (head[i]) {
        uniq[run] = c[i];
        start[run] = (uint32_t)e;
        ++run;
      }
      cell_of[e] = (uint32_t)(run - 1);
      if (e == n - 1) {
        start[run] = (uint32_t)n;
        *m_out = run;
      }
    }
  }
}

}  // namespace sc

inline size_t scan_scratch_bytes(uint64_t n) {
  uint64_t tiles = (n + sc::kTile - 1) / sc::kTile;
  return 256 + (tiles + 1) * 8;
}

// Exclusive scan of n uint32 values into uint64 (or uint32) offsets;
// *total_dev receives the sum (device).  scratch: scan_scratch_bytes(n) bytes.
template <typename OutT>
inline int scan_exclusive(const uint32_t* in, OutT* out, uint64_t n,
                          unsigned long long* total_dev, void* scratch, int* dev_err,
                          cudaStream_t st) {
  if (n == 0) {
    HLC_CUDA(cudaMemsetAsync(total_dev, 0, 8, st));
    return HLC_OK;
  }
  uint64_t tiles = (n + sc::kTile - 1) / sc::kTile;
  uint32_t* ctr = (uint32_t*)scratch;
  unsigned long long* lb = (unsigned long long*)((char*)scratch + 256);
  HLC_CUDA(cudaMemsetAsync(scratch, 0, scan_scratch_bytes(n), st));
  sc::k_scan_excl<OutT><<<(unsigned)tiles, sc::kBlock, 0, st>>>(in, out, n, lb, ctr, total_dev,
                                                                dev_err);
  HLC_LAUNCH_CHECK();
  return HLC_OK;
}

// Cell table of sorted keys (see k_cell_rle); *m_dev receives m (device).
inline int cell_table(const uint32_t* keys, uint64_t n, int shift, uint32_t* cell_of,
                      uint32_t* uniq, uint32_t* start, unsigned long long* m_dev, void* scratch,
                      int* dev_err, cudaStream_t st) {
  if (n == 0) {
    HLC_CUDA(cudaMemsetAsync(m_dev, 0, 8, st));
    HLC_CUDA(cudaMemsetAsync(start, 0, 4, st));
    return HLC_OK;
  }
  uint64_t tiles = (n + sc::kTile - 1) / sc::kTile;
  uint32_t* ctr = (uint32_t*)scratch;
  unsigned long long* lb = (unsigned long long*)((char*)scratch + 256);
  HLC_CUDA(cudaMemsetAsync(scratch, 0, scan_scratch_bytes(n), st));
  sc::k_cell_rle<<<(unsigned)tiles, sc::kBlock, 0, st>>>(keys, n, shift, cell_of, uniq, start, lb,
                                                         ctr, m_dev, dev_err);
  HLC_LAUNCH_CHECK();
  return HLC_OK;
}

}  // namespace hlc
