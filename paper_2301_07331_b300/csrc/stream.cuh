// Out-of-core matching by coarse partition (the second-level partitioning of
// Sec. 4.2, Eq. 8-9, in B300 form).
//
// When the catalogues live in host memory and do not fit a device-memory
// budget, the sky is cut into HEALPix cells of the coarse order Lc.  A first
// streamed pass counts, per coarse cell, the A sources it owns and the B
// sources it needs: every B source is needed by the coarse cells of its fine
// cell and of that cell's 8 neighbours (the halo), so a pair (A_i, B_j) with
// B_j in the neighbourhood of A_i's fine cell is always available where A_i
// is.  Consecutive coarse cells are grouped so that each group fits the
// budget; for every group the inputs are streamed again through pinned
// buffers on two side streams, the group's A sources and needed B sources are
// selected on the device, and the in-core path matches them.  Each A source
// belongs to one group, so each pair is found exactly once; the groups'
// sorted rows are merged.
#pragma once

#include "canon.cuh"
#include "common.cuh"
#include "fastpix.cuh"

namespace hlc {

// Coarse cells an entry is needed in: its own (A) or the distinct coarse
// cells of its fine cell's neighbourhood (B).  Returns the count (<= 9).
__device__ __forceinline__ int needed_parts(double ra, double dec, int Lf, int Lc, bool halo,
                                            const PixConst& K, uint32_t out[9]) {
  uint32_t p = g_ang2pix(ra, dec, Lf, K);
  int shift = 2 * (Lf - Lc);
  if (!halo) {
    out[0] = p >> shift;
    return 1;
  }
  uint32_t nb[9];
  int m = cell_neighbourhood(p, Lf, nb);
  int k = 0;
  for (int e = 0; e < m; ++e) {
    uint32_t c = nb[e] >> shift;
    bool dup = false;
    for (int f = 0; f < k; ++f) dup |= out[f] == c;
    if (!dup) out[k++] = c;
  }
  return k;
}

// Pass 1: per coarse cell, the number of entries it needs.
__global__ void k_part_count(const double* __restrict__ ra, const double* __restrict__ dec,
                             uint64_t n, int Lf, int Lc, int halo, PixConst K,
                             unsigned long long* __restrict__ counts, int* __restrict__ err) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    double a = ra[i], d = dec[i];
    if (!(bits_finite(a) && bits_abs_le(d, 90.0))) {
      atomicOr(err, DERR_INPUT);
      continue;
    }
    if (!bits_in_ra_range(a)) a = c_norm_ra(a);
    uint32_t pc[9];
    int k = needed_parts(a, d, Lf, Lc, halo != 0, K, pc);
    for (int e = 0; e < k; ++e) atomicAdd(counts + pc[e], 1ull);
  }
}

// Pass 2: append the chunk's entries needed by coarse cells [p0, p1) to the
// group buffers (warp-aggregated cursor).
__global__ void k_part_select(const double* __restrict__ ra, const double* __restrict__ dec,
                              const uint64_t* __restrict__ id, uint64_t n, int Lf, int Lc,
                              int halo, PixConst K, uint32_t p0, uint32_t p1,
                              double* __restrict__ ora, double* __restrict__ odec,
                              uint64_t* __restrict__ oid, unsigned long long* __restrict__ cursor,
                              uint64_t cap, int* __restrict__ err) {
  for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x; i0 < n;
       i0 += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t i = i0 + threadIdx.x;
    bool take = false;
    double a = 0, d = 0;
    if (i < n) {
      a = ra[i];
      d = dec[i];
      if (bits_finite(a) && bits_abs_le(d, 90.0)) {
        double an = bits_in_ra_range(a) ? a : c_norm_ra(a);
        uint32_t pc[9];
        int k = needed_parts(an, d, Lf, Lc, halo != 0, K, pc);
        for (int e = 0; e < k; ++e) take |= (pc[e] >= p0 && pc[e] < p1);
      }
    }
    unsigned b = __ballot_sync(0xffffffffu, take);
    if (b) {
      int lane = threadIdx.x & 31;
      unsigned long long base = 0;
      if (lane == __ffs(b) - 1) base = atomicAdd(cursor, (unsigned long long)__popc(b));
      base = __shfl_sync(0xffffffffu, base, __ffs(b) - 1);
      if (take) {
        unsigned long long pos = base + __popc(b & lanemask_lt());
        if (pos < cap) {
          ora[pos] = a;
          odec[pos] = d;
          oid[pos] = id[i];
        } else {
          atomicOr(err, DERR_OVERFLOW);
        }
      }
    }
  }
}

}  // namespace hlc
