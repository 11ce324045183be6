// Pair test for dense cells: one CTA per A cell, B tiles staged in shared
// memory by the TMA engine (the calculation-block kernel of Sec. 4.3 / Fig. 7
// in B300 form: the A sources of a block against all B sources of its block
// and the neighbouring blocks).
//
// Work items are fine cells of A holding at least kTileMinA entries (in the
// single form: cells that lie in a dense table cell of B, where the A entries
// were put in fine order; in the batched form: every such cell of every job,
// A being sorted by (job, cell)).  A first pass (k_tile_items, a warp per
// cell) finds the B ranges of each cell and its 8 neighbours (single form: a
// sparse neighbour table cell contributes its whole range, once) and cuts the
// cell's A sources into items of at most kTileChunkA, which balances the
// CTAs when a few cells hold far more sources than the rest.  The pair
// kernel is warp-specialised.  Its producer warp takes prepared items from an
// atomic counter, writes a round descriptor and copies the round's B vectors
// into one of two stage buffers with cp.async.bulk (the TMA engine's bulk
// mode: contiguous 16-byte vectors need no tensor map) on the buffer's "full"
// mbarrier.  Eight consumer warps each take a share of a staged round
// while their lanes hold KA A sources each: one broadcast shared load per B
// vector and KA FP32 squared-chord tests; then they arrive on the buffer's
// "empty" mbarrier.  The producer's copies for the next round thus overlap
// the consumers' tests of the current one.  Rounds are padded to whole
// groups with vectors far from everything and dead A lanes hold such a vector
// too, so the inner loop has no bounds tests.  A lane records its candidates
// of a group in a bit mask; the warp walks them (a ballot per step) only when
// one lane has any.
//
// Tile shape per cell: KA, the A sources per lane, is 1 for a cell of 32 A
// sources and otherwise taken by density class (33-64, 65-256, more than 256
// A sources) from TileArgs::ka; a staged round is min(TileArgs::stage, the
// neighbourhood's B count).  The library's rule is KA = 2, 4, 4 (the smallest
// that covers the cell in one pass of the 32 lanes, 4 beyond 64 sources) and
// stage = kTileCap; hlc_autotune times other choices on the caller's jobs.
//
// Every mbarrier wait is bounded: on time-out the kernel flags DERR_TIMEOUT,
// the producer waits (bounded) once more for its last copies, and all warps
// return.
#pragma once

#include "batch.cuh"
#include "canon.cuh"
#include "common.cuh"
#include "index.cuh"
#include "match.cuh"

namespace hlc {

constexpr int kTileThreads = 256;                   // consumer threads (+1 producer warp)
constexpr int kTileWarps = kTileThreads / 32;
constexpr int kTileCap = 1536;                      // B vectors per stage buffer (24 KB)
constexpr uint32_t kTileMinA = 32;                  // smaller cells stay with the lane kernels
constexpr uint32_t kTileChunkA = 128;               // A sources per work item (a larger cell is split)
constexpr int kTileGroup = 8;                       // B vectors per any-vote
constexpr int kTileRowCap = 128, kTileBandCap = 64; // staged rows per warp
constexpr long long kTileSpin = 1ll << 24;
constexpr float kFarA = 1e30f, kFarB = -1e30f;      // padding: never within any radius

struct TileItem;

// The rule's KA per density class and its staged round.
constexpr uint32_t kTileRuleKA[3] = {2u, 4u, 4u};

struct TileArgs {
  uint32_t ka[3];            // A sources per lane by class (33-64, 65-256, >256): 1, 2 or 4
  uint32_t stage;            // B vectors per staged round, 8 .. kTileCap (a multiple of 8)
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
  // the pair kernel: items prepared by k_tile_items
  const TileItem* items;
  const uint32_t *idxA, *idxB;  // non-null: emit source indices (entry -> source)
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
  const long long lim = spin_limit(kTileSpin);
  for (long long it = 0; it < lim; ++it) {
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
// EQ4: the tested value is s - (rho_a + rho_b) from the vectors' w (Eq. 4),
// against lo32 / hi32 = -G / +G.
template <int KA, bool EQ4>
__device__ __forceinline__ void tile_round(const float4* __restrict__ sB, uint32_t nr,
                                           uint32_t nrp, uint32_t R0, const uint32_t* s_rb,
                                           const uint32_t* s_off, const float4* __restrict__ a32,
                                           uint32_t a0, uint32_t na, float lo32, float hi32,
                                           int lane, int warp, WarpRows<kTileRowCap>& wrows,
                                           WarpRows<kTileBandCap>& wband, const PairSink& sink,
                                           const uint32_t* __restrict__ idxA,
                                           const uint32_t* __restrict__ idxB,
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
    // KA >= 2: the lane's A sources in pairs (u, u + 1) on the packed FP32
    // instructions (FFMA2 / FMUL2: one instruction, two tests); each packed
    // operation rounds as its scalar twin (a - b as fma(b, -1, a)), so every
    // s2 is bit for bit the scalar one and the guard band is unchanged
    constexpr int KP = KA >= 2 ? KA / 2 : 1;
    float2 ax[KP], ay[KP], az[KP], aw[KP];
#pragma unroll
    for (int v = 0; v < KP; ++v) {
      const int u0 = KA >= 2 ? 2 * v : 0, u1 = KA >= 2 ? 2 * v + 1 : 0;
      ax[v] = make_float2(a[u0].x, a[u1].x);
      ay[v] = make_float2(a[u0].y, a[u1].y);
      az[v] = make_float2(a[u0].z, a[u1].z);
      aw[v] = make_float2(a[u0].w, a[u1].w);
    }
    const float2 m1 = make_float2(-1.f, -1.f);
    for (uint32_t j0 = jbeg; j0 < jend; j0 += kTileGroup) {
      uint32_t mask = 0;
#pragma unroll
      for (int g = 0; g < kTileGroup; ++g) {
        const float4 b = sB[j0 + g];
        if constexpr (KA >= 2) {
          const float2 bx = make_float2(b.x, b.x), by = make_float2(b.y, b.y),
                       bz = make_float2(b.z, b.z);
#pragma unroll
          for (int v = 0; v < KP; ++v) {
            const float2 dx = __ffma2_rn(bx, m1, ax[v]);
            const float2 dy = __ffma2_rn(by, m1, ay[v]);
            const float2 dz = __ffma2_rn(bz, m1, az[v]);
            float2 s2;
            if constexpr (EQ4)
              s2 = __ffma2_rn(dx, dx, __ffma2_rn(aw[v], m1, make_float2(b.w, b.w)));
            else
              s2 = __fmul2_rn(dx, dx);
            s2 = __ffma2_rn(dy, dy, s2);
            s2 = __ffma2_rn(dz, dz, s2);
            mask |= (s2.x <= hi32 ? 1u : 0u) << (g * KA + 2 * v);
            mask |= (s2.y <= hi32 ? 1u : 0u) << (g * KA + 2 * v + 1);
          }
        } else {
#pragma unroll
          for (int u = 0; u < KA; ++u) {
            const float dx = a[u].x - b.x, dy = a[u].y - b.y, dz = a[u].z - b.z;
            float s2 = EQ4 ? fmaf(dx, dx, b.w - a[u].w) : dx * dx;
            s2 = fmaf(dy, dy, s2);
            s2 = fmaf(dz, dz, s2);
            mask |= (s2 <= hi32 ? 1u : 0u) << (g * KA + u);
          }
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
          float s2 = EQ4 ? fmaf(dx, dx, b.w - av.w) : dx * dx;
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
          uint32_t ka = a0 + p0 + (uint32_t)u * 32 + lane;
          if (idxA && act) {  // rows of source indices
            ka = __ldg(idxA + ka);
            jb = __ldg(idxB + jb);
          }
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

// One dense A cell with the B ranges of its neighbourhood, found ahead of
// the pair test by a warp per cell (the lookups are dependent loads; run apart
// from the test, they overlap across the whole GPU).
struct TileItem {
  uint32_t a0, na;          // this item's A entries (a chunk of its cell's)
  float lo32, hi32;
  uint32_t rb[9], off[10];  // B range start per slot; exclusive prefix of lengths
  uint32_t ncell;           // A sources of the whole cell (its density class)
  uint32_t pad;
};

template <bool BATCH>
__global__ void k_tile_items(const TileArgs ta, TileItem* __restrict__ out,
                             unsigned long long* __restrict__ nout, uint64_t cap) {
  const int lane = threadIdx.x & 31;
  const uint64_t nitems = *ta.nitems;
  const uint64_t cmask = BATCH ? (1ull << ta.cell_bits) - 1 : 0;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t item = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
       item < nitems; item += warps) {
    const uint32_t st0 = ta.start[item], st1 = ta.start[item + 1];
    const uint32_t na = st1 - st0;
    if (na < kTileMinA) continue;
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
    uint32_t nb[9];
    cell_neighbourhood9(cell, (int)order, nb);
    uint32_t rb = 0, len = 0;
    if (lane < 9) {
      uint32_t c = nb[0];
#pragma unroll
      for (int q = 1; q < 9; ++q)
        if (lane == q) c = nb[q];
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
              seen |= e < lane && nb[e] != kNoCell && (nb[e] >> ta.bix.shift) == Q;
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
      if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 8);
    if (total == 0) continue;
    // a cell with many A sources becomes several items of kTileChunkA A
    // sources each, against the same B ranges, so that the densest cells do
    // not keep one CTA busy while the others have run out of work
    const uint32_t nch = (na + kTileChunkA - 1) / kTileChunkA;
    unsigned long long slot = 0;
    if (lane == 0) slot = atomicAdd(nout, (unsigned long long)nch);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    for (uint32_t c = 0; c < nch; ++c) {
      if (slot + c >= cap) break;  // sized for the worst case (na >= 32 per cell); never taken
      TileItem& T = out[slot + c];
      if (lane < 9) {
        T.rb[lane] = rb;
        T.off[lane] = incl - len;
      }
      if (lane == 8) T.off[9] = incl;
      if (lane == 0) {
        T.a0 = a0 + c * kTileChunkA;
        T.na = min(kTileChunkA, na - c * kTileChunkA);
        T.ncell = na;
        T.lo32 = lo32;
        T.hi32 = hi32;
      }
    }
  }
}

struct TileDesc {  // one staged round, written by the producer warp
  uint32_t a0, na, ncell, R0, nr, nrp;
  float lo32, hi32;
  uint32_t rb[9], off[10];
  int done;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Warp-specialised: warp 0 produces (takes prepared items from the work
// counter, writes a round descriptor and issues the bulk copies into one of
// two stage buffers), warps 1..8 consume (test their share of the staged B
// vectors against the item's A sources).  Full/empty mbarrier pairs hand the
// buffers over, so the copies for the next round overlap the tests of the
// current one.
template <bool EQ4>
__global__ void __launch_bounds__(kTileThreads + 32) k_pair_tile(const TileArgs ta,
                                                                 PairSink sink) {
  extern __shared__ __align__(128) unsigned char tile_smem[];
  float4* sB0 = reinterpret_cast<float4*>(tile_smem);
  __shared__ uint2 s_rows[kTileWarps][kTileRowCap];
  __shared__ uint2 s_band[kTileWarps][kTileBandCap];
  __shared__ __align__(8) uint64_t full[2], empty[2];
  __shared__ TileDesc desc[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[b])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[b])),
                   "r"(kTileWarps)
                   : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == 0) {
    // ---------------- producer ----------------
    const uint64_t nitems = *ta.nitems;  // prepared items (k_tile_items)
    uint32_t s = 0;  // rounds issued
    bool ok = true;
    for (;;) {
      unsigned item = 0;
      if (lane == 0) item = atomicAdd(ta.work, 1u);
      item = __shfl_sync(0xffffffffu, item, 0);
      if (item >= nitems) break;
      const TileItem& T = ta.items[item];
      const uint32_t a0 = T.a0, na = T.na, ncell = T.ncell;
      const float lo32 = T.lo32, hi32 = T.hi32;
      const uint32_t rb = lane < 9 ? T.rb[lane] : 0u;
      const uint32_t excl = lane < 10 ? T.off[lane] : 0u;
      const uint32_t incl = lane < 9 ? T.off[lane + 1] : 0u;
      const uint32_t total = T.off[9];
      const uint32_t stage = ta.stage;
      for (uint32_t R0 = 0; R0 < total && ok; R0 += stage) {
        const uint32_t b = s & 1u, use = s >> 1;
        if (!mbar_wait(&empty[b], (use & 1u) ^ 1u)) {  // the consumers freed it
          ok = false;
          break;
        }
        const uint32_t nr = min(stage, total - R0);
        const uint32_t nrp = (nr + kTileGroup - 1) / kTileGroup * kTileGroup;
        float4* sB = sB0 + (size_t)b * kTileCap;
        TileDesc& D = desc[b];
        if (lane < 9) {
          D.rb[lane] = rb;
          D.off[lane] = excl;
        }
        if (lane == 8) D.off[9] = incl;
        if (lane == 0) {
          D.a0 = a0;
          D.na = na;
          D.ncell = ncell;
          D.R0 = R0;
          D.nr = nr;
          D.nrp = nrp;
          D.lo32 = lo32;
          D.hi32 = hi32;
          D.done = 0;
        }
        // pad the round to whole groups with vectors far from everything
        if ((uint32_t)lane < nrp - nr) sB[nr + lane] = make_float4(kFarB, kFarB, kFarB, 0.f);
        __syncwarp();
        if (lane == 0) {
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                           smem_u32(&full[b])),
                       "r"(nr * 16u)
                       : "memory");
        }
        // lanes 0..8 copy their range's part of the round
        if (lane < 9) {
          const uint32_t o0 = max(excl, R0), o1 = min(incl, R0 + nr);
          if (o1 > o0) {
            const float4* src = ta.b32 + rb + (o0 - excl);
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                "[%0], [%1], %2, [%3];" ::"r"(smem_u32(sB + (o0 - R0))),
                "l"(src), "r"((o1 - o0) * 16u), "r"(smem_u32(&full[b]))
                : "memory");
          }
        }
        ++s;
      }
      if (!ok) break;
    }
    // tell the consumers there is nothing more (or, after a time-out, let the
    // last round's copies land first)
    const uint32_t b = s & 1u, use = s >> 1;
    if (ok && mbar_wait(&empty[b], (use & 1u) ^ 1u)) {
      if (lane == 0) {
        desc[b].done = 1;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], 0;" ::"r"(
                         smem_u32(&full[b]))
                     : "memory");
      }
    } else {
      if (lane == 0) atomicOr(sink.err, DERR_TIMEOUT);
      if (s > 0) mbar_wait(&full[(s - 1) & 1u], ((s - 1) >> 1) & 1u);
    }
    return;
  }
  // ---------------- consumers ----------------
  const int cw = warp - 1;
  WarpRows<kTileRowCap> wrows{s_rows[cw]};
  WarpRows<kTileBandCap> wband{s_band[cw]};
  unsigned long long ntest = 0;
  for (uint32_t s = 0;; ++s) {
    const uint32_t b = s & 1u, use = s >> 1;
    if (!mbar_wait(&full[b], use & 1u)) {
      if (lane == 0) atomicOr(sink.err, DERR_TIMEOUT);
      break;
    }
    const TileDesc& D = desc[b];
    if (D.done) break;
    const uint32_t na = D.na;
    const float4* sB = sB0 + (size_t)b * kTileCap;
    const uint32_t nc = D.ncell;  // the class is the whole cell's; KA never above the chunk's need
    int ka = nc <= 32 ? 1 : (int)ta.ka[nc <= 64 ? 0 : (nc <= 256 ? 1 : 2)];
    if (na <= 32) ka = 1;
    else if (na <= 64 && ka > 2) ka = 2;
    if (ka == 1)
      tile_round<1, EQ4>(sB, D.nr, D.nrp, D.R0, D.rb, D.off, ta.a32, D.a0, na, D.lo32, D.hi32, lane,
                    cw, wrows, wband, sink, ta.idxA, ta.idxB, ntest);
    else if (ka == 2)
      tile_round<2, EQ4>(sB, D.nr, D.nrp, D.R0, D.rb, D.off, ta.a32, D.a0, na, D.lo32, D.hi32, lane,
                    cw, wrows, wband, sink, ta.idxA, ta.idxB, ntest);
    else
      tile_round<4, EQ4>(sB, D.nr, D.nrp, D.R0, D.rb, D.off, ta.a32, D.a0, na, D.lo32, D.hi32, lane,
                    cw, wrows, wband, sink, ta.idxA, ta.idxB, ntest);
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[b]);
  }
  wrows.flush(sink.rows, sink.count, sink.cap, sink.err);
  wband.flush(sink.band, sink.band_count, sink.band_cap, sink.err);
  for (int o = 16; o > 0; o >>= 1) ntest += __shfl_down_sync(0xffffffffu, ntest, o);
  if (lane == 0 && ntest) atomicAdd(sink.tests, ntest);
}

}  // namespace hlc
