// Pair test for dense cells: one CTA per work item at a time, B tiles staged
// in shared memory by the TMA engine (the calculation-block kernel of Sec.
// 4.3 / Fig. 7 in B300 form: the A sources of a block against all B sources
// of its block and the neighbouring blocks).
//
// Work items come from fine cells of A holding at least kTileMinA entries (in
// the single form: cells that lie in a dense table cell of B, where the A
// entries were put in fine order; in the batched form: every such cell of
// every job, A being sorted by (job, cell)).  A first pass (k_tile_items, a
// warp per cell) finds the B ranges of each cell and its 8 neighbours (single
// form: a sparse neighbour table cell contributes its whole range, once) and
// cuts the cell into items: its A sources in chunks of at most kTileChunkA,
// its neighbourhood's B sources in windows of at most kTileChunkB, so that no
// item holds a CTA much longer than the others; items of many tests are
// handed out first.  The pair kernel is warp-specialised.  Its producer warp
// takes items from an atomic counter, writes a round descriptor and copies
// the round's B vectors and the item's A vectors into one of two stage
// buffers with cp.async.bulk (the TMA engine's bulk mode: contiguous 16-byte
// vectors need no tensor map) on the buffer's "full" mbarrier.  Eight
// consumer warps each take a share of a staged round while their lanes hold
// KA A sources each, then arrive on the buffer's "empty" mbarrier; the
// producer's copies for the next round overlap the tests of the current one.
//
// The test runs in a local frame: with c the item's first A vector, a' = a -
// c and b' = b - c are of the size of the neighbourhood, and
//   |a - b|^2 = |a'|^2 + |b'|^2 - 2 a'.b'
// keeps FP32's relative precision.  Each consumer warp writes its share of
// the staged B vectors as (b', |b'|^2 + w_b) into slots of its own,
// kTileConv at a time, and each lane keeps -2a' and |a'|^2 - w_a - thr for
// its A sources, so a test is one add and three fused multiply-adds,
// r = (|b'|^2 + w_b) + (|a'|^2 - w_a - thr) - 2a'.b', and a pair is a
// candidate when r < 0 (its sign bit, OR-ed over a group of tests).  thr is
// the guard band's upper edge widened by a bound on the rounding of the
// local form (derived at tile_threshold), so every pair the global-frame
// FP32 test would keep is a candidate.  Candidates are then decided exactly
// as the lane kernels decide them: the squared chord of the global FP32
// vectors (both from the staged copies) against the guard band, so the tile
// kernel's rows equal the lane kernels' bit for bit.
//
// Tile shape per cell: KA, the A sources per lane, is 1 for a cell of 32 A
// sources and otherwise taken by density class (33-64, 65-256, more than 256
// A sources) from TileArgs::ka; a staged round is min(TileArgs::stage, the
// item's B window).  The library's rule is KA = 2, 4, 4 (the smallest that
// covers the cell in one pass of the 32 lanes, 4 beyond 64 sources) and stage
// = kTileCap; hlc_autotune times other choices on the caller's jobs.
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
#ifndef HLC_TILE_MIN_A
#define HLC_TILE_MIN_A 32
#endif
constexpr uint32_t kTileMinA = HLC_TILE_MIN_A;      // smaller cells stay with the lane kernels
constexpr uint32_t kTileChunkA = 128;               // A sources per work item (a larger cell is split)
constexpr uint32_t kTileChunkB = 1024;              // B vectors per work item's window
constexpr uint32_t kTileItemDiv = 8;                // items per cell <= its A sources / 8
constexpr uint64_t kTileHeavy = 32768;              // tests of an item handed out first
constexpr int kTileGroup = 8;                       // B vectors per any-vote
constexpr int kTileRowCap = 128, kTileBandCap = 64; // staged rows per warp
constexpr long long kTileSpin = 1ll << 24;
constexpr float kFarW = 1e30f;                      // padding: r never below zero
constexpr uint32_t kTileConv = 64;                  // B vectors per warp in the local frame
constexpr uint32_t kTileQueue = 64;                 // candidates queued per warp
// dynamic shared memory of k_pair_tile: two stage buffers of B, two of A,
// each consumer warp's local-frame slots and its candidate queue
constexpr int kTileSmemDyn =
    (2 * (kTileCap + (int)kTileChunkA) + kTileWarps * (int)kTileConv) * 16 +
    kTileWarps * (int)kTileQueue * 4;

struct TileItem;

// The rule's KA per density class and its staged round.
constexpr uint32_t kTileRuleKA[3] = {2u, 4u, 4u};

struct TileArgs {
  uint32_t ka[3];            // A sources per lane by class (33-64, 65-256, >256): 1, 2 or 4
  uint32_t stage;            // B vectors per staged round, 8 .. kTileCap (a multiple of 8)
  float rho_max;             // Eq. 4: bound on rho_a + rho_b (0 for the single radius)
  const uint32_t* cell;      // (single) item cells (fine ids)
  const uint32_t* start;     // item starts (single: in the dense-subset order), u + 1
  const uint32_t* end = nullptr;  // (batched) each run's end, the runs listed in any order
  const uint32_t* dpos;      // (single) dense-subset index -> A entry
  const unsigned long long* nitems;  // k_tile_items: cells; k_pair_tile: items (front, back)
  uint64_t icap;             // k_pair_tile: capacity of items (the back ones count down from it)
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

// Runs of at least kTileMinA equal keys among sorted composite keys (the
// batched form's dense cells): a thread per entry finds the run heads (the
// key differs from the previous one and equals the one kTileMinA - 1 further
// on) and the run's end by an exponential, then a binary search.  The runs
// are listed as (start, end) in no particular order; nruns[1] and nruns[2]
// receive their number and their entries, as k_mark_tiled counts them.
__global__ void k_long_runs(const uint64_t* __restrict__ key, uint64_t n,
                            uint32_t* __restrict__ rs, uint32_t* __restrict__ re,
                            unsigned long long* __restrict__ nruns, uint64_t cap) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  unsigned long long nent = 0;
  for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x; i0 < n;
       i0 += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = i0 + threadIdx.x;
    bool head = false;
    uint64_t e = 0;
    if (i < n) {
      const uint64_t k = key[i];
      if ((i == 0 || key[i - 1] != k) && i + kTileMinA - 1 < n && key[i + kTileMinA - 1] == k) {
        head = true;
        uint64_t lo = i + kTileMinA - 1, step = kTileMinA;  // key[lo] == k
        while (lo + step < n && key[lo + step] == k) {
          lo += step;
          step <<= 1;
        }
        uint64_t a = lo + 1, b = lo + step < n ? lo + step : n;  // first != k in [a, b]
        while (a < b) {
          const uint64_t mid = (a + b) >> 1;
          if (key[mid] == k) a = mid + 1; else b = mid;
        }
        e = a;
        nent += e - i;
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, head);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(nruns, (unsigned long long)__popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (head) {
        const uint64_t p = base + __popc(m & lt);
        if (p < cap) {
          rs[p] = (uint32_t)i;
          re[p] = (uint32_t)e;
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) nent += __shfl_down_sync(0xffffffffu, nent, o);
  if (lane == 0 && nent) atomicAdd(nruns + 2, nent);
}

// The A entries of listed runs marked for the tile kernel, a warp per run
// (coalesced byte stores).
__global__ void k_mark_runs(const uint32_t* __restrict__ rs, const uint32_t* __restrict__ re,
                            unsigned long long* __restrict__ nruns, uint8_t* __restrict__ tiled) {
  const uint64_t nr = nruns[0];
  const int lane = threadIdx.x & 31;
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  if (w0 == 0 && lane == 0) nruns[1] = nr;
  for (uint64_t r = w0; r < nr; r += nw)
    for (uint32_t j = rs[r] + lane; j < re[r]; j += 32) tiled[j] = 1;
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


// Upper edge of the local-form filter for one item.  hi is the guard band's
// upper edge of the global-frame test (C + G for a single radius, G under
// Eq. 4; hi > 0), rho the bound on rho_a + rho_b (0 for a single radius), mA
// a bound on |a'|^2 over the item's A sources, u = 2^-24.  Only pairs the
// global-frame test keeps (s2 <= hi) must come out with r < 0, and such a
// pair is near its A source: each of the test's five roundings is relative,
// so D^2 = |a - b|^2 <= (hi + rho) (1 + 6u), and |b'| <= |a'| + D + (tiny).
// The local vectors carry the roundings of a - c and b - c, which move
// |a' - b'|^2 by at most u (2 mA + 4 D^2); the ten roundings of r (three for
// |a'|^2, three for |b'|^2, one for |a'|^2 - w_a - thr, one add, three fused
// multiply-adds) stay below 8u (|a'|^2 + |b'|^2 + 2|a'||b'| + thr + rho) <=
// 8u (8 mA + 2 D^2 + thr + rho).  Summed, r <= hi + 38u (hi + rho) + 66u mA +
// 8u thr - thr, and the value below makes that negative with room for the
// three roundings of its own evaluation.  (Pairs far from every A source may
// have larger errors; they can only become false candidates, which the
// global-frame test then rejects.)
__device__ __forceinline__ float tile_threshold(float hi, float rho, float mA) {
  constexpr float u = 5.9604644775390625e-8f;  // 2^-24
  return (hi + 64.0f * u * (hi + rho) + 128.0f * u * mA) * (1.0f + 16.0f * u);
}

__device__ __forceinline__ float warp_max_nonneg(float v) {
  // non-negative floats order as their bit patterns
  return __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(v)));
}

// A warp's staged rows out to the sink, the entry -> source translation
// (idxA non-null) done here with a row per lane, so that the dependent index
// loads of a whole buffer overlap instead of stalling each candidate.
template <int CAP>
__device__ __forceinline__ void tile_flush(WarpRows<CAP>& w, uint2* rows,
                                           unsigned long long* count, uint64_t cap, int* err,
                                           const uint32_t* __restrict__ idxA,
                                           const uint32_t* __restrict__ idxB) {
  if (w.fill == 0) return;
  __syncwarp();
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(count, (unsigned long long)w.fill);
  base = __shfl_sync(0xffffffffu, base, 0);
  for (int i = lane; i < w.fill; i += 32) {
    uint2 r = w.buf[i];
    if (idxA) r = make_uint2(__ldg(idxA + r.x), __ldg(idxB + r.y));
    if (base + i < cap)
      rows[base + i] = r;
    else
      atomicOr(err, DERR_OVERFLOW);
  }
  __syncwarp();
  w.fill = 0;
}

// A warp's candidates of the current round, decided 32 at a time: the
// global-frame FP32 test of each (A slot qa, B slot j) against the guard band.
template <bool EQ4>
__device__ __forceinline__ void tile_drain(uint32_t* __restrict__ q, uint32_t& qfill,
                                           const float4* __restrict__ sB,
                                           const float4* __restrict__ sA, uint32_t R0,
                                           const uint32_t* s_rb, const uint32_t* s_off,
                                           uint32_t a0, float lo32, float hi32, int lane,
                                           WarpRows<kTileRowCap>& wrows,
                                           WarpRows<kTileBandCap>& wband, const PairSink& sink,
                                           const uint32_t* __restrict__ idxA,
                                           const uint32_t* __restrict__ idxB) {
  __syncwarp();
  for (uint32_t base = 0; base < qfill; base += 32) {
    const uint32_t i = base + (uint32_t)lane;
    const bool act = i < qfill;
    const uint32_t e = act ? q[i] : 0u;
    const uint32_t j = e >> 8, qa = e & 255u;
    const float4 av = sA[qa];
    const float4 b = sB[j];
    const float dx = av.x - b.x, dy = av.y - b.y, dz = av.z - b.z;
    float s2 = EQ4 ? fmaf(dx, dx, b.w - av.w) : dx * dx;
    s2 = fmaf(dy, dy, s2);
    s2 = fmaf(dz, dz, s2);
    const bool hit = act && s2 <= lo32;
    const bool band = act && !hit && s2 <= hi32;
    uint32_t jb = 0;
    if (hit || band) {  // B entry of staged slot R0 + j
      const uint32_t o = R0 + j;
      int sgi = 0;
#pragma unroll 1
      while (sgi < 8 && s_off[sgi + 1] <= o) ++sgi;
      jb = s_rb[sgi] + (o - s_off[sgi]);
    }
    wrows.add(hit, a0 + qa, jb);  // entries; tile_flush translates them
    wband.add(band, a0 + qa, jb);
    if (wrows.fill > kTileRowCap - 32)
      tile_flush(wrows, sink.rows, sink.count, sink.cap, sink.err, idxA, idxB);
    if (wband.fill > kTileBandCap - 32)
      tile_flush(wband, sink.band, sink.band_count, sink.band_cap, sink.err, idxA, idxB);
  }
  __syncwarp();
  qfill = 0;
}

// One staged round against every A pass of the item, KA A sources per lane.
// sB: the round's B vectors and sA: the item's A vectors, both as copied
// (global frame, read only); sC: this warp's kTileConv slots, which receive
// its share of sB in the local frame, kTileConv vectors at a time; q: its
// candidate queue (kTileQueue slots), drained before the round ends.
// EQ4: w holds +rho_a (A) and -rho_b (B) and the tested value is
// s - (rho_a + rho_b) against lo32 / hi32 = -G / +G (Eq. 4).
template <int KA, bool EQ4>
__device__ __forceinline__ void tile_round(const float4* __restrict__ sB,
                                           const float4* __restrict__ sA, float4* __restrict__ sC,
                                           uint32_t* __restrict__ q, uint32_t nr, uint32_t nrp,
                                           uint32_t R0, const uint32_t* s_rb,
                                           const uint32_t* s_off, uint32_t a0, uint32_t na,
                                           float lo32, float hi32, float rho_max, int lane,
                                           int warp, WarpRows<kTileRowCap>& wrows,
                                           WarpRows<kTileBandCap>& wband, const PairSink& sink,
                                           const uint32_t* __restrict__ idxA,
                                           const uint32_t* __restrict__ idxB,
                                           unsigned long long& ntest) {
  // this warp's groups: warp, warp + kTileWarps, ... (dealt out in turn, so
  // that every warp's share spans all the neighbour ranges of the round and
  // the candidates spread evenly over the warps)
  const uint32_t ngroups = nrp / kTileGroup;
  if ((uint32_t)warp >= ngroups) return;
  const uint32_t nmine = (ngroups - (uint32_t)warp + kTileWarps - 1) / kTileWarps;
  uint32_t jreal = 0;  // real B vectors among them
  {
    const uint32_t full_groups = nr / kTileGroup, part = nr % kTileGroup;
    jreal = (full_groups > (uint32_t)warp
                 ? (full_groups - (uint32_t)warp + kTileWarps - 1) / kTileWarps : 0u) *
            kTileGroup;
    if (part && full_groups % kTileWarps == (uint32_t)warp) jreal += part;
  }
  const float4 c = sA[0];
  float mA = 0.f;
  for (uint32_t k = lane; k < na; k += 32) {
    const float4 a = sA[k];
    const float x = a.x - c.x, y = a.y - c.y, z = a.z - c.z;
    mA = fmaxf(mA, fmaf(z, z, fmaf(y, y, x * x)));
  }
  const float thr = tile_threshold(hi32, rho_max, warp_max_nonneg(mA));
  uint32_t qfill = 0;
  constexpr int KP = KA >= 2 ? KA / 2 : 1;
  for (uint32_t p0 = 0; p0 < na; p0 += 32 * KA) {
    // -2a' and |a'|^2 - w_a - thr of the lane's A sources, A sources u and
    // u + 1 side by side (KA >= 2: for the packed FP32 instructions FADD2 /
    // FFMA2, each half rounded as its scalar twin); dead lanes never become
    // candidates
    float2 px[KP], py[KP], pz[KP], pc[KP];
#pragma unroll
    for (int u = 0; u < KA; ++u) {
      const uint32_t k = p0 + (uint32_t)u * 32 + lane;
      float x2 = 0.f, y2 = 0.f, z2 = 0.f, w2 = kFarW;
      if (k < na) {
        const float4 a = sA[k];
        const float x = a.x - c.x, y = a.y - c.y, z = a.z - c.z;
        const float n2 = fmaf(z, z, fmaf(y, y, x * x));
        x2 = -2.f * x;
        y2 = -2.f * y;
        z2 = -2.f * z;
        w2 = (EQ4 ? n2 - a.w : n2) - thr;
      }
      if (u % 2 == 0) {
        px[u / 2] = make_float2(x2, x2);
        py[u / 2] = make_float2(y2, y2);
        pz[u / 2] = make_float2(z2, z2);
        pc[u / 2] = make_float2(w2, w2);
      } else {
        px[u / 2].y = x2;
        py[u / 2].y = y2;
        pz[u / 2].y = z2;
        pc[u / 2].y = w2;
      }
      ntest += k < na ? jreal : 0u;
    }
    constexpr uint32_t kConvGroups = kTileConv / kTileGroup;
    for (uint32_t t0 = 0; t0 < nmine; t0 += kConvGroups) {
      const uint32_t tn = min(nmine - t0, kConvGroups);
      // the B vectors of groups t0 .. t0 + tn to (b', |b'|^2 + w_b) in sC;
      // padding slots to a vector no A source comes near
      __syncwarp();  // (the previous groups' tests are done with sC)
      for (uint32_t i = lane; i < tn * kTileGroup; i += 32) {
        const uint32_t j =
            ((uint32_t)warp + (t0 + i / kTileGroup) * kTileWarps) * kTileGroup + i % kTileGroup;
        float4 v = make_float4(0.f, 0.f, 0.f, kFarW);
        if (j < nr) {
          const float4 b = sB[j];
          const float x = b.x - c.x, y = b.y - c.y, z = b.z - c.z;
          const float n2 = fmaf(z, z, fmaf(y, y, x * x));
          v = make_float4(x, y, z, EQ4 ? n2 + b.w : n2);
        }
        sC[i] = v;
      }
      __syncwarp();
      for (uint32_t t = 0; t < tn; ++t) {
        const uint32_t j0 = ((uint32_t)warp + (t0 + t) * kTileWarps) * kTileGroup;
        const float4* cg = sC + t * kTileGroup;
        uint32_t gm = 0;  // bit g: some test of B vector j0 + g has r < 0
#pragma unroll
        for (int g = 0; g < kTileGroup; ++g) {
          const float4 b = cg[g];
          uint32_t sg = 0;
          if constexpr (KA >= 2) {
            const float2 bx = make_float2(b.x, b.x), by = make_float2(b.y, b.y),
                         bz = make_float2(b.z, b.z), bw = make_float2(b.w, b.w);
#pragma unroll
            for (int v = 0; v < KP; ++v) {
              float2 r = __fadd2_rn(bw, pc[v]);
              r = __ffma2_rn(px[v], bx, r);
              r = __ffma2_rn(py[v], by, r);
              r = __ffma2_rn(pz[v], bz, r);
              sg |= __float_as_uint(r.x) | __float_as_uint(r.y);
            }
          } else {
            float r = b.w + pc[0].x;
            r = fmaf(px[0].x, b.x, r);
            r = fmaf(py[0].x, b.y, r);
            r = fmaf(pz[0].x, b.z, r);
            sg = __float_as_uint(r);
          }
          gm |= (sg >> 31) << g;
        }
        if (__any_sync(0xffffffffu, gm != 0u)) {
          // the flagged vectors' tests again, one bit per candidate test ...
          uint32_t mask = 0;
          for (uint32_t m = gm; m != 0u; m &= m - 1u) {
            const int g = __ffs(m) - 1;
            const float4 b = cg[g];
#pragma unroll
            for (int u = 0; u < KA; ++u) {
              const bool hi_half = u % 2 != 0;
              const int v = u / 2;
              float r = b.w + (hi_half ? pc[v].y : pc[v].x);
              r = fmaf(hi_half ? px[v].y : px[v].x, b.x, r);
              r = fmaf(hi_half ? py[v].y : py[v].x, b.y, r);
              r = fmaf(hi_half ? pz[v].y : pz[v].x, b.z, r);
              mask |= (__float_as_uint(r) >> 31) << (g * KA + u);
            }
          }
          // ... appended to the warp's queue as (B slot, A slot)
          for (;;) {
            const bool act = mask != 0u;
            const unsigned bal = __ballot_sync(0xffffffffu, act);
            if (bal == 0u) break;
            if (qfill + 32 > kTileQueue)
              tile_drain<EQ4>(q, qfill, sB, sA, R0, s_rb, s_off, a0, lo32, hi32, lane, wrows,
                              wband, sink, idxA, idxB);
            if (act) {
              const int bit = __ffs(mask) - 1;
              mask &= mask - 1u;
              const uint32_t j = j0 + (uint32_t)(bit / KA);
              const uint32_t k = p0 + (uint32_t)(bit % KA) * 32 + lane;
              q[qfill + __popc(bal & lanemask_lt())] = (j << 8) | k;
            }
            qfill += __popc(bal);
          }
        }
      }
    }
  }
  tile_drain<EQ4>(q, qfill, sB, sA, R0, s_rb, s_off, a0, lo32, hi32, lane, wrows, wband, sink,
                  idxA, idxB);
}

// A chunk of a dense A cell against a window of the B ranges of its
// neighbourhood, found ahead of the pair test by a warp per cell (the lookups
// are dependent loads; run apart from the test, they overlap across the whole
// GPU).
struct TileItem {
  uint32_t a0, na;          // this item's A entries (a chunk of its cell's)
  float lo32, hi32;
  uint32_t rb[9], off[10];  // B range start per slot; exclusive prefix of lengths
  uint32_t ncell;           // A sources of the whole cell (its density class)
  uint32_t rlo, rhi;        // this item's window [rlo, rhi) of the concatenated ranges
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
    const uint32_t st0 = ta.start[item], st1 = ta.end ? ta.end[item] : ta.start[item + 1];
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
    // the cell becomes items of at most kTileChunkA A sources against B
    // windows of at most kTileChunkB vectors (a multiple of kTileGroup), and
    // at most na / kTileItemDiv items in all, so that the items of every
    // cell fit the array (its capacity is the A entries / kTileItemDiv + 1);
    // items of at least kTileHeavy tests are placed from the front, the rest
    // from the back, and the pair kernel takes the front ones first
    const uint32_t nch_a = (na + kTileChunkA - 1) / kTileChunkA;
    uint32_t nch_b = (total + kTileChunkB - 1) / kTileChunkB;
    nch_b = min(nch_b, max(1u, (na / kTileItemDiv) / nch_a));
    uint32_t wb = (total + nch_b - 1) / nch_b;
    wb = (wb + kTileGroup - 1) / kTileGroup * kTileGroup;
    nch_b = (total + wb - 1) / wb;
    const uint32_t nch = nch_a * nch_b;
    const bool heavy = (uint64_t)min(na, kTileChunkA) * wb >= kTileHeavy;
    unsigned long long slot = 0;
    if (lane == 0) slot = atomicAdd(nout + (heavy ? 0 : 1), (unsigned long long)nch);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    for (uint32_t c = 0; c < nch; ++c) {
      if (slot + c >= cap) break;  // the capacity bounds every cell's items; never taken
      TileItem& T = out[heavy ? slot + c : cap - 1 - (slot + c)];
      const uint32_t ca = c / nch_b, cb = c % nch_b;
      if (lane < 9) {
        T.rb[lane] = rb;
        T.off[lane] = incl - len;
      }
      if (lane == 8) T.off[9] = incl;
      if (lane == 0) {
        T.a0 = a0 + ca * kTileChunkA;
        T.na = min(kTileChunkA, na - ca * kTileChunkA);
        T.ncell = na;
        T.lo32 = lo32;
        T.hi32 = hi32;
        T.rlo = cb * wb;
        T.rhi = min(total, (cb + 1) * wb);
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
// counter, writes a round descriptor and issues the bulk copies of the
// round's B vectors and the item's A vectors into one of two stage buffers),
// warps 1..8 consume (move their share of the staged B vectors to the local
// frame and test it against the item's A sources).  Full/empty mbarrier
// pairs hand the buffers over, so the copies for the next round overlap the
// tests of the current one; the consumers only read the stage buffers.
template <bool EQ4>
__global__ void __launch_bounds__(kTileThreads + 32, 3) k_pair_tile(const TileArgs ta,
                                                                 PairSink sink) {
  extern __shared__ __align__(128) unsigned char tile_smem[];
  float4* sB0 = reinterpret_cast<float4*>(tile_smem);        // 2 x kTileCap
  float4* sA0 = sB0 + 2 * kTileCap;                           // 2 x kTileChunkA
  float4* sC0 = sA0 + 2 * kTileChunkA;                        // kTileWarps x kTileConv
  uint32_t* sQ0 = reinterpret_cast<uint32_t*>(sC0 + kTileWarps * kTileConv);  // x kTileQueue
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
    const uint64_t nfront = ta.nitems[0];                 // prepared items (k_tile_items):
    const uint64_t nitems = nfront + ta.nitems[1];        // the front ones, then the back ones
    uint32_t s = 0;  // rounds issued
    bool ok = true;
    unsigned nxt = 0;  // the next item's index, taken one item ahead
    if (lane == 0) nxt = atomicAdd(ta.work, 1u);
    for (;;) {
      const unsigned item = __shfl_sync(0xffffffffu, nxt, 0);
      if (item >= nitems) break;
      // (taken now, used after this item's rounds: its latency overlaps them)
      if (lane == 0) nxt = atomicAdd(ta.work, 1u);
      const TileItem& T = ta.items[item < nfront ? item : ta.icap - 1 - (item - nfront)];
      const uint32_t a0 = T.a0, na = T.na, ncell = T.ncell;
      const float lo32 = T.lo32, hi32 = T.hi32;
      const uint32_t rb = lane < 9 ? T.rb[lane] : 0u;
      const uint32_t excl = lane < 10 ? T.off[lane] : 0u;
      const uint32_t incl = lane < 9 ? T.off[lane + 1] : 0u;
      const uint32_t rlo = T.rlo, rhi = T.rhi;
      const uint32_t stage = ta.stage;
      for (uint32_t R0 = rlo; R0 < rhi && ok; R0 += stage) {
        const uint32_t b = s & 1u, use = s >> 1;
        if (!mbar_wait(&empty[b], (use & 1u) ^ 1u)) {  // the consumers freed it
          ok = false;
          break;
        }
        const uint32_t nr = min(stage, rhi - R0);
        const uint32_t nrp = (nr + kTileGroup - 1) / kTileGroup * kTileGroup;
        float4* sB = sB0 + (size_t)b * kTileCap;
        float4* sA = sA0 + (size_t)b * kTileChunkA;
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
        __syncwarp();
        if (lane == 0) {
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                           smem_u32(&full[b])),
                       "r"((nr + na) * 16u)
                       : "memory");
        }
        // lanes 0..8 copy their range's part of the round, lane 9 the A chunk
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
        } else if (lane == 9) {
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
              "[%0], [%1], %2, [%3];" ::"r"(smem_u32(sA)),
              "l"(ta.a32 + a0), "r"(na * 16u), "r"(smem_u32(&full[b]))
              : "memory");
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
    const float4* sA = sA0 + (size_t)b * kTileChunkA;
    float4* sC = sC0 + (size_t)cw * kTileConv;
    uint32_t* sQ = sQ0 + (size_t)cw * kTileQueue;
    const uint32_t nc = D.ncell;  // the class is the whole cell's; KA never above the chunk's need
    int ka = nc <= 32 ? 1 : (int)ta.ka[nc <= 64 ? 0 : (nc <= 256 ? 1 : 2)];
    if (na <= 32) ka = 1;
    else if (na <= 64 && ka > 2) ka = 2;
    if (ka == 1)
      tile_round<1, EQ4>(sB, sA, sC, sQ, D.nr, D.nrp, D.R0, D.rb, D.off, D.a0, na, D.lo32,
                         D.hi32, ta.rho_max, lane, cw, wrows, wband, sink, ta.idxA, ta.idxB,
                         ntest);
    else if (ka == 2)
      tile_round<2, EQ4>(sB, sA, sC, sQ, D.nr, D.nrp, D.R0, D.rb, D.off, D.a0, na, D.lo32,
                         D.hi32, ta.rho_max, lane, cw, wrows, wband, sink, ta.idxA, ta.idxB,
                         ntest);
    else
      tile_round<4, EQ4>(sB, sA, sC, sQ, D.nr, D.nrp, D.R0, D.rb, D.off, D.a0, na, D.lo32,
                         D.hi32, ta.rho_max, lane, cw, wrows, wband, sink, ta.idxA, ta.idxB,
                         ntest);
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[b]);
  }
  tile_flush(wrows, sink.rows, sink.count, sink.cap, sink.err, ta.idxA, ta.idxB);
  tile_flush(wband, sink.band, sink.band_count, sink.band_cap, sink.err, ta.idxA, ta.idxB);
  for (int o = 16; o > 0; o >>= 1) ntest += __shfl_down_sync(0xffffffffu, ntest, o);
  if (lane == 0 && ntest) atomicAdd(sink.tests, ntest);
}

}  // namespace hlc
