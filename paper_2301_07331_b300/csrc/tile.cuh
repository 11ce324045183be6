// Pair test for dense cells: one CTA per A cell, B tiles staged in shared
// memory by the TMA engine (the calculation-block kernel of Sec. 4.3 / Fig. 7
// in B300 form: the A sources of a block against all B sources of its block
// and the neighbouring blocks).
//
// Work items are fine cells of A holding at least kTileMinA entries (in the
// single form: cells that lie in a dense table cell of B, where the A entries
// were put in fine order; in the batched form: every such cell of every job,
// A being sorted by (job, cell)).  For an item the CTA gathers the B ranges of
// the cell and its 8 neighbours (single form: a sparse neighbour table cell
// contributes its whole range, once), copies them round by round into shared
// memory with cp.async.bulk on one mbarrier, and each warp takes a share of
// the staged B vectors while its lanes hold KA A sources each: one broadcast
// shared load per B vector and KA FP32 squared-chord tests.  Rounds are
// padded to whole groups with vectors far from everything and dead A lanes
// hold such a vector too, so the inner loop has no bounds tests.  A lane
// records its candidates of a group in a bit mask; the warp walks them (a
// ballot per step) only when one lane has any.
//
// Tile shape per cell (the density rule): KA, the A sources per lane, is the
// smallest of 1, 2, 4 that covers the cell's A sources in one pass of the 32
// lanes (4 beyond 64 sources), which keeps lanes busy on small cells and
// amortises each shared load over more tests on large ones; the staged round
// is min(kTileCap, the neighbourhood's B count).
//
// Each wait on the mbarrier is bounded: on time-out the kernel flags
// DERR_TIMEOUT, waits (bounded) once more for its own copies and returns.
#pragma once

#include "batch.cuh"
#include "canon.cuh"
#include "common.cuh"
#include "index.cuh"
#include "match.cuh"

namespace hlc {

constexpr int kTileThreads = 256;
constexpr int kTileWarps = kTileThreads / 32;
constexpr int kTileCap = 2048;                      // B vectors per round (32 KB)
constexpr uint32_t kTileMinA = 32;                  // smaller cells stay with the lane kernels
constexpr int kTileGroup = 8;                       // B vectors per any-vote
constexpr int kTileRowCap = 128, kTileBandCap = 64; // staged rows per warp
constexpr long long kTileSpin = 1ll << 24;
constexpr float kFarA = 1e30f, kFarB = -1e30f;      // padding: never within any radius

struct TileArgs {
  const uint32_t* cell;      // (single) item cells (fine ids)
  const uint32_t* start;     // item starts (single: in the dense-subset order), u + 1
  const uint32_t* dpos;      // (single) dense-subset index -> A entry
  const unsigned long long* nitems;
  unsigned* work;            // atomic item counter (zeroed)
  const float4* a32;
  const float4* b32;
  float lo32, hi32;          // (single) guard band
  uint32_t sparse_cell;
  // single form: B's offset table over table cells
  CellIndex bix;
  int order;
  // batched form: composite (job, cell) keys and per-job tables
  const uint64_t* keyA64;
  const uint64_t* keyB64;
  const uint32_t* btable;
  const JobDev* jobs;
  int cell_bits;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < kTileSpin; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Marks the A entries of the items the tile kernel takes; nitems[0] = runs,
// nitems[1] += items taken, nitems[2] += their A entries.  dpos null: the
// starts are A entries already.
__global__ void k_mark_tiled(const uint32_t* __restrict__ start, const uint32_t* __restrict__ dpos,
                             unsigned long long* __restrict__ nitems,
                             uint8_t* __restrict__ tiled) {
  const uint64_t u = nitems[0];
  unsigned long long ni = 0, ne = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < u;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t s0 = start[i], s1 = start[i + 1];
    if (s1 - s0 < kTileMinA) continue;
    ++ni;
    ne += s1 - s0;
    for (uint32_t s = s0; s < s1; ++s) tiled[dpos ? dpos[s] : s] = 1;
  }
  if (ni) {
    atomicAdd(nitems + 1, ni);
    atomicAdd(nitems + 2, ne);
  }
}

// Run starts of sorted 64-bit keys: flag[i] = 1 where a run begins ...
__global__ void k_run_flags64(const uint64_t* __restrict__ key, uint64_t n,
                              uint32_t* __restrict__ flag) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || key[i] != key[i - 1]) ? 1u : 0u;
}

// ... and start[r] = first entry of run r, start[runs] = n (off = exclusive
// scan of flag, *runs its total).
__global__ void k_run_starts(const uint32_t* __restrict__ flag, const uint32_t* __restrict__ off,
                             uint64_t n, const unsigned long long* __restrict__ runs,
                             uint32_t* __restrict__ start) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    if (flag[i]) start[off[i]] = (uint32_t)i;
  if (blockIdx.x == 0 && threadIdx.x == 0) start[*runs] = (uint32_t)n;
}

// One staged round against every A pass of the item, KA A sources per lane.
template <int KA>
__device__ __forceinline__ void tile_round(const float4* __restrict__ sB, uint32_t nr,
                                           uint32_t nrp, uint32_t R0, const uint32_t* s_rb,
                                           const uint32_t* s_off, const float4* __restrict__ a32,
                                           uint32_t a0, uint32_t na, float lo32, float hi32,
                                           int lane, int warp, WarpRows<kTileRowCap>& wrows,
                                           WarpRows<kTileBandCap>& wband, const PairSink& sink,
                                           unsigned long long& ntest) {
  const uint32_t ngroups = nrp / kTileGroup;
  const uint32_t gper = (ngroups + kTileWarps - 1) / kTileWarps;
  const uint32_t jbeg = min(ngroups, warp * gper) * kTileGroup;
  const uint32_t jend = min(ngroups, (warp + 1) * gper) * kTileGroup;
  const uint32_t jreal = jend <= nr ? jend - jbeg : (nr > jbeg ? nr - jbeg : 0u);
  for (uint32_t p0 = 0; p0 < na && jbeg < jend; p0 += 32 * KA) {
    float4 a[KA];
#pragma unroll
    for (int u = 0; u < KA; ++u) {
      const uint32_t q = p0 + (uint32_t)u * 32 + lane;
      a[u] = q < na ? a32[a0 + q] : make_float4(kFarA, kFarA, kFarA, 0.f);
      ntest += q < na ? jreal : 0u;
    }
    for (uint32_t j0 = jbeg; j0 < jend; j0 += kTileGroup) {
      uint32_t mask = 0;
#pragma unroll
      for (int g = 0; g < kTileGroup; ++g) {
        const float4 b = sB[j0 + g];
#pragma unroll
        for (int u = 0; u < KA; ++u) {
          const float dx = a[u].x - b.x, dy = a[u].y - b.y, dz = a[u].z - b.z;
          float s2 = dx * dx;
          s2 = fmaf(dy, dy, s2);
          s2 = fmaf(dz, dz, s2);
          mask |= (s2 <= hi32 ? 1u : 0u) << (g * KA + u);
        }
      }
      if (__any_sync(0xffffffffu, mask != 0u)) {
        // slow path: each lane walks its own candidates
        const int nmax = __reduce_max_sync(0xffffffffu, (unsigned)__popc(mask));
        for (int it = 0; it < nmax; ++it) {
          const bool act = mask != 0u;
          const int bit = act ? __ffs(mask) - 1 : 0;
          mask &= mask - 1u;
          const int g = bit / KA, u = bit % KA;
          const uint32_t j = j0 + g;
          const float4 b = sB[j];
          float4 av = a[0];
#pragma unroll
          for (int v = 1; v < KA; ++v)
            if (u == v) av = a[v];
          const float dx = av.x - b.x, dy = av.y - b.y, dz = av.z - b.z;
          float s2 = dx * dx;
          s2 = fmaf(dy, dy, s2);
          s2 = fmaf(dz, dz, s2);
          const bool hit = act && s2 <= lo32;
          const bool band = act && !hit && s2 <= hi32;
          uint32_t jb = 0;
          if (act) {  // B entry of staged slot R0 + j
            const uint32_t o = R0 + j;
            int sgi = 0;
#pragma unroll 1
            while (sgi < 8 && s_off[sgi + 1] <= o) ++sgi;
            jb = s_rb[sgi] + (o - s_off[sgi]);
          }
          const uint32_t ka = a0 + p0 + (uint32_t)u * 32 + lane;
          wrows.add(hit, ka, jb);
          wband.add(band, ka, jb);
          if (wrows.fill > kTileRowCap - 32) wrows.flush(sink.rows, sink.count, sink.cap, sink.err);
          if (wband.fill > kTileBandCap - 32)
            wband.flush(sink.band, sink.band_count, sink.band_cap, sink.err);
        }
      }
    }
  }
}

template <bool BATCH>
__global__ void __launch_bounds__(kTileThreads) k_pair_tile(const TileArgs ta, PairSink sink) {
  extern __shared__ __align__(128) unsigned char tile_smem[];
  float4* sB = reinterpret_cast<float4*>(tile_smem);
  __shared__ uint2 s_rows[kTileWarps][kTileRowCap];
  __shared__ uint2 s_band[kTileWarps][kTileBandCap];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_rb[9], s_off[10];
  __shared__ unsigned s_item;
  __shared__ int s_abort;
  WarpRows<kTileRowCap> wrows{s_rows[threadIdx.x >> 5]};
  WarpRows<kTileBandCap> wband{s_band[threadIdx.x >> 5]};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = threadIdx.x;
  unsigned long long ntest = 0;
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  __syncthreads();
  uint32_t phase = 0;
  const uint64_t nitems = *ta.nitems;
  const uint64_t cmask = BATCH ? (1ull << ta.cell_bits) - 1 : 0;
  for (;;) {
    if (t == 0) s_item = atomicAdd(ta.work, 1u);
    __syncthreads();
    const unsigned item = s_item;
    if (item >= nitems || s_abort) break;
    const uint32_t st0 = ta.start[item], st1 = ta.start[item + 1];
    const uint32_t na = st1 - st0;
    if (na >= kTileMinA) {
      const uint32_t a0 = BATCH ? st0 : ta.dpos[st0];
      uint32_t cell, order, job = 0;
      float lo32 = ta.lo32, hi32 = ta.hi32;
      JobTab J = {0, 0, 0u, 0u, 0ull, 0.0, 0.f, 0.f};
      if (BATCH) {
        const uint64_t key = ta.keyA64[a0];
        job = (uint32_t)(key >> ta.cell_bits);
        cell = (uint32_t)(key & cmask);
        J = load_job(ta.jobs, job);
        order = (uint32_t)J.L;
        lo32 = J.lo32;
        hi32 = J.hi32;
      } else {
        cell = ta.cell[item];
        order = (uint32_t)ta.order;
      }
      // B ranges of the cell and its neighbours (threads 0..8)
      if (t < 32) {
        uint32_t nb[9];
        cell_neighbourhood9(cell, (int)order, nb);
        uint32_t rb = 0, len = 0;
        if (t < 9) {
          uint32_t c = nb[0];
#pragma unroll
          for (int s = 1; s < 9; ++s)
            if (t == s) c = nb[s];
          if (c != kNoCell) {
            if (BATCH) {
              const uint2 r = bcell_range(ta.keyB64, ta.btable, J, job, ta.cell_bits, c);
              rb = r.x;
              len = r.y - r.x;
            } else {
              const uint32_t Q = c >> ta.bix.shift;
              const uint32_t c0 = __ldg(ta.bix.table + Q), c1 = __ldg(ta.bix.table + Q + 1);
              if (c1 - c0 <= ta.sparse_cell) {
                bool seen = false;
#pragma unroll
                for (int e = 0; e < 9; ++e)
                  seen |= e < t && nb[e] != kNoCell && (nb[e] >> ta.bix.shift) == Q;
                if (!seen) {
                  rb = c0;
                  len = c1 - c0;
                }
              } else {
                const uint2 r = cell_range_in(ta.bix.keys, c0, c1, c);
                rb = r.x;
                len = r.y - r.x;
              }
            }
          }
        }
        uint32_t incl = len;
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
          if (t >= o) incl += y;
        }
        if (t < 9) {
          s_rb[t] = rb;
          s_off[t] = incl - len;
        }
        if (t == 8) s_off[9] = incl;
      }
      __syncthreads();
      const uint32_t total = s_off[9];
      const int ka = na <= 32 ? 1 : (na <= 64 ? 2 : 4);  // the density rule
      for (uint32_t R0 = 0; R0 < total; R0 += kTileCap) {
        const uint32_t nr = min((uint32_t)kTileCap, total - R0);
        if (t == 0) {
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                           smem_u32(&bar)),
                       "r"(nr * 16u)
                       : "memory");
#pragma unroll 1
          for (int s = 0; s < 9; ++s) {
            // part of range s inside [R0, R0 + nr)
            const uint32_t o0 = max(s_off[s], R0), o1 = min(s_off[s + 1], R0 + nr);
            if (o1 > o0) {
              const float4* src = ta.b32 + s_rb[s] + (o0 - s_off[s]);
              asm volatile(
                  "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                  "[%0], [%1], %2, [%3];" ::"r"(smem_u32(sB + (o0 - R0))),
                  "l"(src), "r"((o1 - o0) * 16u), "r"(smem_u32(&bar))
                  : "memory");
            }
          }
        }
        // pad the round to whole groups with vectors far from everything
        const uint32_t nrp = (nr + kTileGroup - 1) / kTileGroup * kTileGroup;
        if ((uint32_t)t < nrp - nr) sB[nr + t] = make_float4(kFarB, kFarB, kFarB, 0.f);
        const bool landed = mbar_wait(&bar, phase);
        if (__syncthreads_or(!landed)) {  // the same decision in every thread
          if (t == 0) {
            atomicOr(sink.err, DERR_TIMEOUT);
            s_abort = 1;
          }
          if (landed == false) mbar_wait(&bar, phase);  // let the copies land before leaving
          __syncthreads();
          break;
        }
        phase ^= 1u;
        if (ka == 1)
          tile_round<1>(sB, nr, nrp, R0, s_rb, s_off, ta.a32, a0, na, lo32, hi32, lane, warp,
                        wrows, wband, sink, ntest);
        else if (ka == 2)
          tile_round<2>(sB, nr, nrp, R0, s_rb, s_off, ta.a32, a0, na, lo32, hi32, lane, warp,
                        wrows, wband, sink, ntest);
        else
          tile_round<4>(sB, nr, nrp, R0, s_rb, s_off, ta.a32, a0, na, lo32, hi32, lane, warp,
                        wrows, wband, sink, ntest);
        __syncthreads();  // the round's buffer is free again
      }
    }
    __syncthreads();  // s_item, s_rb and s_off are rewritten for the next item
  }
  wrows.flush(sink.rows, sink.count, sink.cap, sink.err);
  wband.flush(sink.band, sink.band_count, sink.band_cap, sink.err);
  for (int o = 16; o > 0; o >>= 1) ntest += __shfl_down_sync(0xffffffffu, ntest, o);
  if ((t & 31) == 0 && ntest) atomicAdd(sink.tests, ntest);
}

}  // namespace hlc
