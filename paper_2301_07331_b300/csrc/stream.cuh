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

// Distinct partition groups a source is needed in (A: the group of its
// coarse cell; B: the groups of its halo cells), at most 9.
__device__ __forceinline__ int needed_groups(double ra, double dec, int Lf, int Lc, bool halo,
                                             const PixConst& K,
                                             const uint32_t* __restrict__ cell2group,
                                             uint32_t out[9]) {
  uint32_t pc[9];
  const int k = needed_parts(ra, dec, Lf, Lc, halo, K, pc);
  int m = 0;
  for (int e = 0; e < k; ++e) {
    const uint32_t g = __ldg(cell2group + pc[e]);
    bool dup = false;
    for (int f = 0; f < m; ++f) dup |= out[f] == g;
    if (!dup) out[m++] = g;
  }
  return m;
}

// Pass 1 of the bucketed stream, per chunk: sources per group ...
__global__ void k_group_hist(const double* __restrict__ ra, const double* __restrict__ dec,
                             uint64_t n, int Lf, int Lc, int halo, PixConst K,
                             const uint32_t* __restrict__ cell2group, uint32_t ngroups,
                             uint32_t* __restrict__ gcnt) {
  extern __shared__ uint32_t sh_cnt[];
  for (uint32_t g = threadIdx.x; g < ngroups; g += blockDim.x) sh_cnt[g] = 0;
  __syncthreads();
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    double a = ra[i], d = dec[i];
    if (!(bits_finite(a) && bits_abs_le(d, 90.0))) continue;
    if (!bits_in_ra_range(a)) a = c_norm_ra(a);
    uint32_t gs[9];
    const int m = needed_groups(a, d, Lf, Lc, halo != 0, K, cell2group, gs);
    for (int e = 0; e < m; ++e) atomicAdd(sh_cnt + gs[e], 1u);
  }
  __syncthreads();
  for (uint32_t g = threadIdx.x; g < ngroups; g += blockDim.x)
    if (sh_cnt[g]) atomicAdd(gcnt + g, sh_cnt[g]);
}

// ... their exclusive scan (one block) ...
__global__ void k_small_excl_scan(const uint32_t* __restrict__ cnt, uint32_t n,
                                  uint32_t* __restrict__ off) {
  __shared__ uint32_t ws[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t b0 = 0; b0 < n; b0 += blockDim.x) {
    const uint32_t i = b0 + threadIdx.x;
    const uint32_t v = i < n ? cnt[i] : 0u;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) >= (unsigned)o) x += y;
    }
    if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = x;
    __syncthreads();
    uint32_t wpre = 0;
    for (unsigned w = 0; w < (threadIdx.x >> 5); ++w) wpre += ws[w];
    const uint32_t c = carry;
    if (i < n) off[i] = c + wpre + x - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = c + wpre + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) off[n] = carry;
}

// ... and the scatter of the chunk into group order: each block counts its
// sources per group in shared memory, reserves one range per group with one
// global atomic, then places its sources inside those ranges.
__global__ void k_group_scatter(const double* __restrict__ ra, const double* __restrict__ dec,
                                const uint64_t* __restrict__ id, uint64_t n, int Lf, int Lc,
                                int halo, PixConst K, const uint32_t* __restrict__ cell2group,
                                uint32_t ngroups, const uint32_t* __restrict__ goff,
                                uint32_t* __restrict__ gcur, double* __restrict__ ora,
                                double* __restrict__ odec, uint64_t* __restrict__ oid,
                                int* __restrict__ err) {
  extern __shared__ uint32_t sh[];
  uint32_t* s_cnt = sh;            // ngroups
  uint32_t* s_base = sh + ngroups; // ngroups
  const uint64_t per = ((n + gridDim.x - 1) / gridDim.x + blockDim.x - 1) / blockDim.x * blockDim.x;
  const uint64_t i0 = (uint64_t)blockIdx.x * per, i1 = i0 + per < n ? i0 + per : n;
  for (uint32_t g = threadIdx.x; g < ngroups; g += blockDim.x) s_cnt[g] = 0;
  __syncthreads();
  for (uint64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    double a = ra[i], d = dec[i];
    if (!(bits_finite(a) && bits_abs_le(d, 90.0))) continue;
    if (!bits_in_ra_range(a)) a = c_norm_ra(a);
    uint32_t gs[9];
    const int m = needed_groups(a, d, Lf, Lc, halo != 0, K, cell2group, gs);
    for (int e = 0; e < m; ++e) atomicAdd(s_cnt + gs[e], 1u);
  }
  __syncthreads();
  for (uint32_t g = threadIdx.x; g < ngroups; g += blockDim.x) {
    s_base[g] = s_cnt[g] ? goff[g] + atomicAdd(gcur + g, s_cnt[g]) : 0u;
    s_cnt[g] = 0;
  }
  __syncthreads();
  for (uint64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const double a0 = ra[i], d = dec[i];
    if (!(bits_finite(a0) && bits_abs_le(d, 90.0))) continue;
    const double a = bits_in_ra_range(a0) ? a0 : c_norm_ra(a0);
    uint32_t gs[9];
    const int m = needed_groups(a, d, Lf, Lc, halo != 0, K, cell2group, gs);
    const uint64_t sid = id[i];
    for (int e = 0; e < m; ++e) {
      const uint32_t pos = s_base[gs[e]] + atomicAdd(s_cnt + gs[e], 1u);
      if (pos >= goff[gs[e] + 1]) {
        atomicOr(err, DERR_BOUNDS);
        continue;
      }
      ora[pos] = a0;
      odec[pos] = d;
      oid[pos] = sid;
    }
  }
}

}  // namespace hlc
