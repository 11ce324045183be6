// Fine order inside the dense table cells of a catalogue sorted by table
// cell only (the FP32 complete-mode layout; Sec. 4.2 / Fig. 7 in B300 form).
//
// The pair test reads a sparse table cell (at most kSparseCell entries)
// whole, so the entries of such a cell may stay in any order; a dense table
// cell is searched by fine key and must be ordered.  The entries of dense
// table cells are compacted (order kept), radix sorted by full key and written
// back: the compacted list is in table-cell order, so its p-th sorted entry
// belongs at its p-th position.
#pragma once

#include "common.cuh"
#include "canon.cuh"
#include "fp32.cuh"

namespace hlc {

// 1 where the entry's table cell is dense.
__global__ void k_dense_flags(const uint32_t* __restrict__ key, uint64_t m, int shift,
                              const uint32_t* __restrict__ T, uint32_t dense_above,
                              uint32_t* __restrict__ flag) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t q = key[e] >> shift;
    flag[e] = (__ldg(T + q + 1) - __ldg(T + q)) > dense_above;
  }
}

// Compaction of the dense entries (order kept): positions, keys, identity.
__global__ void k_dense_compact(const uint32_t* __restrict__ key, uint64_t m,
                                const uint32_t* __restrict__ flag, const uint32_t* __restrict__ off,
                                uint32_t* __restrict__ dpos, uint32_t* __restrict__ dkey,
                                uint32_t* __restrict__ dval) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (uint64_t)gridDim.x * blockDim.x) {
    if (flag[e]) {
      const uint32_t p = off[e];
      dpos[p] = (uint32_t)e;
      dkey[p] = key[e];
      dval[p] = p;
    }
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
