// Fine order inside the dense table cells of a catalogue sorted by table
// cell only (the FP32 complete-mode layout; Sec. 4.2 / Fig. 7 in B300 form).
//
// The pair test reads a sparse table cell (at most kSparseCell entries)
// whole, so the entries of such a cell may stay in any order; a dense table
// cell is searched by fine key and must be ordered.  The entries of dense
// table cells are listed in table-cell order (each dense cell's entries are a
// contiguous range of either catalogue), radix sorted by full key and written
// back: the list is in table-cell order, so its p-th sorted entry belongs at
// its p-th position.
#pragma once

#include "common.cuh"
#include "canon.cuh"
#include "fp32.cuh"

namespace hlc {

// ---- dense table cells from the table itself ---------------------------
// The dense table cells are few and their entries contiguous in both sorted
// catalogues, so the dense entries are listed from the table (a pass over
// its slots and a scan over blocks of slots, then one range per dense cell)
// instead of from a flag and a scan per entry.
constexpr int kDenseBlkSlots = 1024;  // table slots per block (256 threads x 4)

__device__ __forceinline__ bool dense_slot(const uint32_t* __restrict__ T, uint64_t c, uint64_t S,
                                           uint32_t dense_above) {
  return c < S && (__ldg(T + c + 1) - __ldg(T + c)) > dense_above;
}

// Dense cells per block of kDenseBlkSlots slots (blockDim 256).
__global__ void __launch_bounds__(256) k_dense_cell_blocks(const uint32_t* __restrict__ T,
                                                           uint64_t S, uint32_t dense_above,
                                                           uint32_t* __restrict__ blkcnt) {
  __shared__ uint32_t ws[8];
  const uint64_t c0 = (uint64_t)blockIdx.x * kDenseBlkSlots + 4u * threadIdx.x;
  uint32_t n = 0;
#pragma unroll
  for (int u = 0; u < 4; ++u) n += dense_slot(T, c0 + u, S, dense_above);
  for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < 8; ++w) t += ws[w];
    blkcnt[blockIdx.x] = t;
  }
}

// The dense cells in ascending order: block b writes its cells from blkoff[b].
__global__ void __launch_bounds__(256) k_dense_cell_list(const uint32_t* __restrict__ T,
                                                         uint64_t S, uint32_t dense_above,
                                                         const uint32_t* __restrict__ blkoff,
                                                         uint32_t* __restrict__ cells) {
  __shared__ uint32_t ws[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t c0 = (uint64_t)blockIdx.x * kDenseBlkSlots + 4u * threadIdx.x;
  bool d[4];
  uint32_t n = 0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    d[u] = dense_slot(T, c0 + u, S, dense_above);
    n += d[u];
  }
  uint32_t incl = n;  // inclusive scan of n over the block
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) ws[warp] = incl;
  __syncthreads();
  uint32_t base = blkoff[blockIdx.x];
  for (int w = 0; w < warp; ++w) base += ws[w];
  uint32_t pos = base + incl - n;
#pragma unroll
  for (int u = 0; u < 4; ++u)
    if (d[u]) cells[pos++] = (uint32_t)(c0 + u);
}

// Entry range of each dense cell: from the table (keys null: the catalogue
// the table was built on) or by binary search in another catalogue's keys
// sorted by the same table cell (A against B's table); len for the scan.
__global__ void k_dense_cell_ranges(const uint32_t* __restrict__ cells,
                                    const unsigned long long* __restrict__ ncells,
                                    const uint32_t* __restrict__ T,
                                    const uint32_t* __restrict__ keys, uint64_t m, int shift,
                                    uint2* __restrict__ rng, uint32_t* __restrict__ len) {
  const uint64_t nc = *ncells;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t c = cells[i];
    uint2 r;
    if (!keys) {
      r = make_uint2(__ldg(T + c), __ldg(T + c + 1));
    } else {
      const uint64_t q0 = (uint64_t)c << shift, q1 = (uint64_t)(c + 1) << shift;
      uint64_t lo = 0, hi = m;  // first key >= q0
      while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if ((uint64_t)keys[mid] < q0) lo = mid + 1; else hi = mid;
      }
      const uint64_t a = lo;
      hi = m;  // first key >= q1
      while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if ((uint64_t)keys[mid] < q1) lo = mid + 1; else hi = mid;
      }
      r = make_uint2((uint32_t)a, (uint32_t)lo);
    }
    rng[i] = r;
    len[i] = r.y - r.x;
  }
}

// The dense entries in table-cell order, a thread per entry (a cell may hold
// most of a catalogue, so the work is split by entry, not by cell): entry p
// finds its cell as the last offset <= p, then writes its position, key and
// identity value (p itself).
__global__ void k_dense_fill(const uint2* __restrict__ rng, const uint32_t* __restrict__ off,
                             const unsigned long long* __restrict__ ncells, uint64_t nd,
                             const uint32_t* __restrict__ key, uint32_t* __restrict__ dpos,
                             uint32_t* __restrict__ dkey, uint32_t* __restrict__ dval) {
  const uint64_t nc = *ncells;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nd;
       p += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t lo = 0, hi = nc;  // first cell whose offset exceeds p
    while (lo < hi) {
      const uint64_t mid = (lo + hi) >> 1;
      if (__ldg(off + mid) <= p) lo = mid + 1; else hi = mid;
    }
    const uint64_t i = lo - 1;  // off[0] = 0 <= p, so lo >= 1
    const uint32_t pos = rng[i].x + (uint32_t)(p - __ldg(off + i));
    dpos[p] = pos;
    dkey[p] = key[pos];
    dval[p] = (uint32_t)p;
  }
}

// Sorted dense entries gathered into temporaries (perm[p] = compacted index
// of the p-th smallest key) ...
__global__ void k_dense_gather(const uint32_t* __restrict__ dpos, const uint32_t* __restrict__ perm,
                               uint64_t nd, const uint32_t* __restrict__ idx,
                               const float4* __restrict__ v32, uint32_t* __restrict__ tidx,
                               float4* __restrict__ tv) {
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nd;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t src = dpos[perm[p]];
    tidx[p] = idx[src];
    tv[p] = v32[src];
  }
}

// ... and written back to the dense positions in order.
__global__ void k_dense_scatter(const uint32_t* __restrict__ dpos, uint64_t nd,
                                const uint32_t* __restrict__ skey,
                                const uint32_t* __restrict__ tidx, const float4* __restrict__ tv,
                                uint32_t* __restrict__ key, uint32_t* __restrict__ idx,
                                float4* __restrict__ v32) {
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nd;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t dst = dpos[p];
    key[dst] = skey[p];
    idx[dst] = tidx[p];
    v32[dst] = tv[p];
  }
}

}  // namespace hlc
