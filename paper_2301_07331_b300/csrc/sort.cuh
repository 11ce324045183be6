// Device-wide primitives: a stable LSD radix sort of (key, uint32 value)
// pairs in one sweep per 8-bit digit with decoupled look-back, and a
// single-pass exclusive scan built on the same look-back.
//
// The sort of the cell keys is the B300 form of the paper's map from HEALPix
// index to records (Sec. 4.2, Fig. 7): the records of a cell end up
// contiguous, so a cell is a range [start, end) of the sorted arrays.
#pragma once

#include <utility>

#include "common.cuh"

namespace hlc {
namespace rs {

constexpr int kBlock = 256;  // threads per CTA; one thread per digit value
constexpr int kWarps = kBlock / 32;
constexpr int kIpt = 18;     // items per thread (18 measured 4% faster per pass than 15)
constexpr int kTile = kBlock * kIpt;
constexpr int kRadix = 256;
static_assert(kBlock == kRadix, "one thread per digit value");
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr long long kSpinLimit = 1ll << 26;

// Histogram of every digit pass at once.
template <typename K>
__global__ void __launch_bounds__(kBlock) k_digit_hist(const K* __restrict__ keys, uint64_t n,
                                                       int npass, int bit_lo,
                                                       uint32_t* __restrict__ hist) {
  __shared__ uint32_t sh[8][kRadix];
  for (int i = threadIdx.x; i < 8 * kRadix; i += kBlock) sh[i / kRadix][i % kRadix] = 0;
  __syncthreads();
  for (uint64_t e = (uint64_t)blockIdx.x * kBlock + threadIdx.x; e < n;
       e += (uint64_t)gridDim.x * kBlock) {
    K k = keys[e];
    for (int p = 0; p < npass; ++p)
      atomicAdd(&sh[p][(uint32_t)(k >> (bit_lo + 8 * p)) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < npass * kRadix; i += kBlock) {
    uint32_t v = sh[i / kRadix][i % kRadix];
    if (v) atomicAdd(&hist[i], v);
  }
}

// Exclusive scan of one 256-bin histogram per pass (one CTA per pass).
__global__ void __launch_bounds__(kBlock) k_hist_scan(const uint32_t* __restrict__ hist,
                                                      uint32_t* __restrict__ offs) {
  __shared__ uint32_t ws[kWarps];
  int p = blockIdx.x, t = threadIdx.x;
  uint32_t v = hist[p * kRadix + t];
  uint32_t incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if ((t & 31) >= o) incl += y;
  }
  if ((t & 31) == 31) ws[t >> 5] = incl;
  __syncthreads();
  uint32_t wpre = 0;
  for (int w = 0; w < (t >> 5); ++w) wpre += ws[w];
  offs[p * kRadix + t] = wpre + incl - v;
}

// Block-wide exclusive scan of one value per thread (kBlock threads).
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v,
                                                              unsigned long long* ws,
                                                              unsigned long long* total) {
  int t = threadIdx.x;
  unsigned long long incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if ((t & 31) >= o) incl += y;
  }
  if ((t & 31) == 31) ws[t >> 5] = incl;
  __syncthreads();
  unsigned long long wpre = 0, tot = 0;
  for (int w = 0; w < kWarps; ++w) {
    if (w < (t >> 5)) wpre += ws[w];
    tot += ws[w];
  }
  __syncthreads();
  if (total) *total = tot;
  return wpre + incl - v;
}

template <typename K>
struct SweepSmem {
  K keys[kTile];
  uint32_t vals[kTile];
  uint32_t whist[kWarps][kRadix];
  uint32_t dstart[kRadix];
  unsigned long long gbase[kRadix];
  unsigned long long ws[kWarps];
  uint32_t tile;
};

// One digit pass: rank each tile's keys by digit (stable), obtain the tile's
// global offset per digit by decoupled look-back over earlier tiles, and write
// the tile out grouped by digit (coalesced within each digit run).
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// (The look-back words carry their value and flag in one 64-bit word, so
// relaxed accesses suffice: no other data is published through them.)

// Exclusive prefix of digit t over the tiles before `tile`: walk back from
// the predecessor adding published counts until an inclusive prefix is met.
// A predecessor that has published nothing yet is waited for, at most
// spin_limit(kSpinLimit) polls; then DERR_TIMEOUT is flagged and the partial
// prefix returned (every later position stays below the true one, so the
// scatter stays in bounds).
__device__ __forceinline__ unsigned long long lookback_excl(
    const unsigned long long* lookback, uint32_t tile, int t, int* err) {
  unsigned long long excl = 0;
  long long spins = 0;
  const long long lim = spin_limit(kSpinLimit);
  int64_t j = (int64_t)tile - 1;
  while (j >= 0) {
    unsigned long long w = ld_relaxed_u64(lookback + (uint64_t)j * kRadix + t);
    unsigned long long flag = w & ~kValMask;
    if (flag == 0) {
      if (++spins > lim) {
        atomicOr(err, DERR_TIMEOUT);
        break;
      }
      continue;
    }
    excl += w & kValMask;
    if (flag == kFlagInc) break;
    --j;
  }
  return excl;
}

// One array of a digit pass.  A launch may sort two arrays at once (the same
// digit of each): its tiles are numbered across both, the first ntiles
// belonging to d0, and each array keeps its own histogram offsets and
// look-back chain.
template <typename K>
struct SweepDesc {
  const K* kin;
  const uint32_t* vin;
  K* kout;
  uint32_t* vout;
  uint64_t n;
  const uint32_t* goff;          // this pass's global digit offsets
  unsigned long long* lookback;  // this pass's look-back words
  uint32_t ntiles;
};

// The pass over one tile.  FULL: the tile holds kTile entries (every tile
// but an array's last), so no entry needs a bound check and every lane of
// the ranking ballots is live.
template <typename K, bool FULL>
__device__ __forceinline__ void sweep_tile(SweepSmem<K>& S, const int t, const int lane,
                                           const int warp, const uint32_t tile,
                                           const K* __restrict__ kt,
                                           const uint32_t* __restrict__ vt, K* __restrict__ kout,
                                           uint32_t* __restrict__ vout,
                                           const uint32_t* __restrict__ goff,
                                           unsigned long long* __restrict__ lookback,
                                           const uint32_t rem, const uint32_t wo, int shift,
                                           int* __restrict__ err, const uint32_t vbase) {
#define HLC_IN_TILE(o) (FULL || (o) < rem)
  K k[kIpt];
#pragma unroll
  for (int i = 0; i < kIpt; ++i) {
    const uint32_t o = wo + (uint32_t)i * 32;
    k[i] = HLC_IN_TILE(o) ? kt[o] : K(0);
  }
  // publish this tile's digit counts before ranking, so that later tiles'
  // look-backs do not wait for it; the look-back of its own prefix follows
  // the ranking and finds earlier tiles published the same way
#pragma unroll
  for (int i = 0; i < kIpt; ++i)
    if (HLC_IN_TILE(wo + (uint32_t)i * 32))
      atomicAdd(&S.dstart[(uint32_t)(k[i] >> shift) & 255u], 1u);
  __syncthreads();
  const uint32_t cnt = S.dstart[t];
  unsigned long long* slot = lookback + (uint64_t)tile * kRadix + t;
  st_relaxed_u64(slot, (tile == 0 ? kFlagInc : kFlagAgg) | cnt);
  uint32_t r[kIpt];
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int i = 0; i < kIpt; ++i) {
    // lanes holding the same digit: intersect the 8 bit-plane ballots
    const bool valid = HLC_IN_TILE(wo + (uint32_t)i * 32);
    uint32_t d = (uint32_t)(k[i] >> shift) & 255u;
    unsigned peers = FULL ? 0xffffffffu : __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      bool bit = (d >> b) & 1;
      unsigned bb = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? bb : ~bb;
    }
    uint32_t before = valid ? S.whist[warp][d] : 0u;
    r[i] = before + __popc(peers & lt);
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) S.whist[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();

  // thread t owns digit t: warp offsets within the tile
  uint32_t wsum = 0;
  for (int w = 0; w < kWarps; ++w) {
    uint32_t c = S.whist[w][t];
    S.whist[w][t] = wsum;
    wsum += c;
  }
  unsigned long long excl = 0;
  if (tile != 0) {
    excl = lookback_excl(lookback, tile, t, err);
    st_relaxed_u64(slot, kFlagInc | (excl + cnt));
  }
  S.gbase[t] = (unsigned long long)goff[t] + excl;
  unsigned long long dst = block_excl_scan(cnt, S.ws, nullptr);
  S.dstart[t] = (uint32_t)dst;
  __syncthreads();

#pragma unroll
  for (int i = 0; i < kIpt; ++i) {
    const uint32_t o = wo + (uint32_t)i * 32;
    if (HLC_IN_TILE(o)) {
      uint32_t d = (uint32_t)(k[i] >> shift) & 255u;
      uint32_t pos = S.dstart[d] + S.whist[warp][d] + r[i];
      S.keys[pos] = k[i];
      S.vals[pos] = vt ? vt[o] : vbase + o;  // (null: the values are the positions)
    }
  }
  __syncthreads();
  for (uint32_t p = t; p < (FULL ? (uint32_t)kTile : rem); p += kBlock) {
    K kk = S.keys[p];
    int dd = (int)((uint32_t)(kk >> shift) & 255u);
    unsigned long long g = S.gbase[dd] + (p - S.dstart[dd]);
    kout[g] = kk;
    vout[g] = S.vals[p];
  }
#undef HLC_IN_TILE
}

template <typename K>
__global__ void __launch_bounds__(kBlock, sizeof(K) == 8 ? 3 : 4) k_onesweep(
    const SweepDesc<K> d0, const SweepDesc<K> d1, int shift, uint32_t* __restrict__ tile_ctr,
    int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SweepSmem<K>& S = *reinterpret_cast<SweepSmem<K>*>(smem_raw);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) S.tile = atomicAdd(tile_ctr, 1u);
  for (int i = t; i < kWarps * kRadix; i += kBlock) (&S.whist[0][0])[i] = 0;
  S.dstart[t] = 0;  // (kBlock == kRadix) the tile's digit counts first
  __syncthreads();
  // (tiles are taken in order, so every earlier tile of either array has
  // started: the look-back below never waits on a tile not yet running)
  const bool second = S.tile >= d0.ntiles;
  const uint32_t tile = second ? S.tile - d0.ntiles : S.tile;
  const K* __restrict__ kin = second ? d1.kin : d0.kin;
  const uint32_t* __restrict__ vin = second ? d1.vin : d0.vin;
  K* __restrict__ kout = second ? d1.kout : d0.kout;
  uint32_t* __restrict__ vout = second ? d1.vout : d0.vout;
  const uint64_t n = second ? d1.n : d0.n;
  const uint32_t* __restrict__ goff = second ? d1.goff : d0.goff;
  unsigned long long* __restrict__ lookback = second ? d1.lookback : d0.lookback;
  const uint64_t base = (uint64_t)tile * kTile;
  // tile-local 32-bit offsets: entry base + o is valid when o < rem
  const uint32_t rem = (uint32_t)(n - base < (uint64_t)kTile ? n - base : (uint64_t)kTile);
  const uint32_t wo = (uint32_t)warp * (kIpt * 32) + (uint32_t)lane;
  const K* __restrict__ kt = kin + base;
  const uint32_t* __restrict__ vt = vin ? vin + base : nullptr;

  if (rem == (uint32_t)kTile)
    sweep_tile<K, true>(S, t, lane, warp, tile, kt, vt, kout, vout, goff, lookback, rem, wo, shift,
                        err, (uint32_t)base);
  else
    sweep_tile<K, false>(S, t, lane, warp, tile, kt, vt, kout, vout, goff, lookback, rem, wo,
                         shift, err, (uint32_t)base);
}

}  // namespace rs

// Host driver.  keys/vals are sorted in place (the result is copied back if
// the last pass wrote the alternate buffers).  tmp_keys/tmp_vals: n elements;
// scratch: from sort_scratch_bytes().  Returns HLC_OK or an error code; a
// timed-out look-back is reported through dev_err (checked by the caller).
constexpr size_t kSortLookbackOffset = 16640;  // hist | offs | counters | look-back

inline size_t sort_scratch_bytes(uint64_t n, int npass) {
  uint64_t tiles = (n + rs::kTile - 1) / rs::kTile;
  if (tiles == 0) tiles = 1;
  return kSortLookbackOffset + (size_t)npass * tiles * rs::kRadix * 8;
}

// Sorts by the key bits [bit_lo, key_bits).  With in_tmp set, an odd number
// of passes leaves the result in (tmp_keys, tmp_vals) and *in_tmp says so;
// otherwise it is copied back.
// pass_ev, when given, receives events recorded around the digit passes.
// hist_ready: the scratch's digit histograms (npass x 256 counts at its
// start) were counted by the producer of the keys; the histogram pass is
// skipped.
template <typename K>
int radix_sort_pairs(K* keys, uint32_t* vals, K* tmp_keys, uint32_t* tmp_vals, uint64_t n,
                     int key_bits, void* scratch, int* dev_err, cudaStream_t st,
                     int bit_lo = 0, bool* in_tmp = nullptr, cudaEvent_t* pass_ev = nullptr,
                     int* npass_out = nullptr, bool hist_ready = false) {
  if (in_tmp) *in_tmp = false;
  if (n <= 1) return HLC_OK;
  if (bit_lo < 0 || bit_lo >= key_bits) bit_lo = 0;
  int npass = (key_bits - bit_lo + 7) / 8;
  if (npass < 1) npass = 1;
  if (npass > (int)sizeof(K)) npass = (int)sizeof(K);
  uint64_t tiles = (n + rs::kTile - 1) / rs::kTile;
  if (tiles > 0xFFFFFFFFull) {
    set_error("radix sort: too many elements");
    return HLC_EINVAL;
  }
  char* sp = (char*)scratch;
  uint32_t* hist = (uint32_t*)sp;
  uint32_t* offs = (uint32_t*)(sp + 8192);
  uint32_t* ctr = (uint32_t*)(sp + 16384);
  unsigned long long* lb = (unsigned long long*)(sp + kSortLookbackOffset);
  size_t lb_bytes = (size_t)npass * tiles * rs::kRadix * 8;
  HLC_CUDA(cudaMemsetAsync(ctr, 0, 64, st));
  HLC_CUDA(cudaMemsetAsync(lb, 0, lb_bytes, st));
  if (!hist_ready) {
    HLC_CUDA(cudaMemsetAsync(hist, 0, (size_t)npass * rs::kRadix * 4, st));
    rs::k_digit_hist<K><<<grid_for(n, rs::kBlock, num_sms() * 8u), rs::kBlock, 0, st>>>(
        keys, n, npass, bit_lo, hist);
    HLC_LAUNCH_CHECK();
  }
  rs::k_hist_scan<<<npass, rs::kBlock, 0, st>>>(hist, offs);
  HLC_LAUNCH_CHECK();
  size_t smem = sizeof(rs::SweepSmem<K>);
  HLC_CUDA(cudaFuncSetAttribute(rs::k_onesweep<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  K* ka = keys;
  uint32_t* va = vals;
  K* kb = tmp_keys;
  uint32_t* vb = tmp_vals;
  if (npass_out) *npass_out = npass;
  if (pass_ev) cudaEventRecord(pass_ev[0], st);
  for (int p = 0; p < npass; ++p) {
    rs::SweepDesc<K> d{ka, va, kb, vb, n, offs + p * rs::kRadix,
                       lb + (size_t)p * tiles * rs::kRadix, (uint32_t)tiles};
    rs::k_onesweep<K><<<(unsigned)tiles, rs::kBlock, smem, st>>>(d, d, bit_lo + 8 * p, ctr + p,
                                                                 dev_err);
    HLC_LAUNCH_CHECK();
    K* tk = ka; ka = kb; kb = tk;
    uint32_t* tv = va; va = vb; vb = tv;
  }
  if (pass_ev) cudaEventRecord(pass_ev[1], st);
  if (ka != keys && in_tmp) {
    *in_tmp = true;
  } else if (ka != keys) {
    HLC_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(K), cudaMemcpyDeviceToDevice, st));
    HLC_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
  }
  return HLC_OK;
}

// Two arrays sorted by the same key bits [bit_lo, key_bits) at once: one
// launch per digit pass covers the tiles of both (more tiles in flight than
// either alone).  Each array has its own temporaries and scratch (from
// sort_scratch_bytes for its own n); the pass counters live in scr0.  With
// in_tmp set, an odd number of passes leaves both results in the temporary
// buffers and *in_tmp says so (never when only one array needs sorting).
// Either array may be empty.
// hist_ready: each scratch's digit histograms (npass x 256 counts at its
// start) were already counted by the producer of the keys (the prep kernels
// count while they write the keys), so the histogram pass is skipped.
// vals_identity: the values are the positions 0, 1, ... (vals0/vals1 are not
// read, only used as buffers), so the first pass makes them instead of
// loading them.
template <typename K>
int radix_sort_pairs2(K* keys0, uint32_t* vals0, K* tk0, uint32_t* tv0, uint64_t n0, void* scr0,
                      K* keys1, uint32_t* vals1, K* tk1, uint32_t* tv1, uint64_t n1, void* scr1,
                      int key_bits, int* dev_err, cudaStream_t st, int bit_lo, bool* in_tmp,
                      cudaEvent_t* pass_ev = nullptr, int* npass_out = nullptr,
                      bool hist_ready = false, bool vals_identity = false) {
  if (in_tmp) *in_tmp = false;
  if (n0 <= 1 || n1 <= 1) {  // one array (or none) needs sorting: the single form,
    if (npass_out) *npass_out = 0;  // its result copied back in place
    if (n0 > 1)
      return radix_sort_pairs<K>(keys0, vals0, tk0, tv0, n0, key_bits, scr0, dev_err, st, bit_lo,
                                 nullptr, pass_ev, npass_out);
    if (n1 > 1)
      return radix_sort_pairs<K>(keys1, vals1, tk1, tv1, n1, key_bits, scr1, dev_err, st, bit_lo,
                                 nullptr, pass_ev, npass_out);
    return HLC_OK;
  }
  if (bit_lo < 0 || bit_lo >= key_bits) bit_lo = 0;
  int npass = (key_bits - bit_lo + 7) / 8;
  if (npass < 1) npass = 1;
  if (npass > (int)sizeof(K)) npass = (int)sizeof(K);
  const uint64_t t0 = (n0 + rs::kTile - 1) / rs::kTile, t1 = (n1 + rs::kTile - 1) / rs::kTile;
  if (t0 + t1 > 0xFFFFFFFFull) {
    set_error("radix sort: too many elements");
    return HLC_EINVAL;
  }
  char* s0 = (char*)scr0;
  char* s1 = (char*)scr1;
  uint32_t* ctr = (uint32_t*)(s0 + 16384);
  HLC_CUDA(cudaMemsetAsync(ctr, 0, 64, st));
  struct Side {
    K* keys;
    uint32_t* vals;
    K* tk;
    uint32_t* tv;
    uint64_t n, tiles;
    char* sp;
  } sd[2] = {{keys0, vals0, tk0, tv0, n0, t0, s0}, {keys1, vals1, tk1, tv1, n1, t1, s1}};
  for (const Side& q : sd) {
    uint32_t* hist = (uint32_t*)q.sp;
    uint32_t* offs = (uint32_t*)(q.sp + 8192);
    unsigned long long* lb = (unsigned long long*)(q.sp + kSortLookbackOffset);
    HLC_CUDA(cudaMemsetAsync(lb, 0, (size_t)npass * q.tiles * rs::kRadix * 8, st));
    if (!hist_ready) {
      HLC_CUDA(cudaMemsetAsync(hist, 0, (size_t)npass * rs::kRadix * 4, st));
      rs::k_digit_hist<K><<<grid_for(q.n, rs::kBlock, num_sms() * 8u), rs::kBlock, 0, st>>>(
          q.keys, q.n, npass, bit_lo, hist);
      HLC_LAUNCH_CHECK();
    }
    rs::k_hist_scan<<<npass, rs::kBlock, 0, st>>>(hist, offs);
    HLC_LAUNCH_CHECK();
  }
  size_t smem = sizeof(rs::SweepSmem<K>);
  HLC_CUDA(cudaFuncSetAttribute(rs::k_onesweep<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  K* ka[2] = {keys0, keys1};
  uint32_t* va[2] = {vals0, vals1};
  K* kb[2] = {tk0, tk1};
  uint32_t* vb[2] = {tv0, tv1};
  if (npass_out) *npass_out = npass;
  if (pass_ev) cudaEventRecord(pass_ev[0], st);
  for (int p = 0; p < npass; ++p) {
    rs::SweepDesc<K> d[2];
    for (int i = 0; i < 2; ++i)
      d[i] = rs::SweepDesc<K>{ka[i], (vals_identity && p == 0) ? nullptr : va[i], kb[i], vb[i],
                              sd[i].n,
                              (uint32_t*)(sd[i].sp + 8192) + p * rs::kRadix,
                              (unsigned long long*)(sd[i].sp + kSortLookbackOffset) +
                                  (size_t)p * sd[i].tiles * rs::kRadix,
                              (uint32_t)sd[i].tiles};
    rs::k_onesweep<K><<<(unsigned)(t0 + t1), rs::kBlock, smem, st>>>(d[0], d[1], bit_lo + 8 * p,
                                                                     ctr + p, dev_err);
    HLC_LAUNCH_CHECK();
    for (int i = 0; i < 2; ++i) {
      std::swap(ka[i], kb[i]);
      std::swap(va[i], vb[i]);
    }
  }
  if (pass_ev) cudaEventRecord(pass_ev[1], st);
  if (ka[0] != keys0 && in_tmp) {
    *in_tmp = true;
  } else if (ka[0] != keys0) {
    for (int i = 0; i < 2; ++i) {
      HLC_CUDA(cudaMemcpyAsync(sd[i].keys, ka[i], sd[i].n * sizeof(K), cudaMemcpyDeviceToDevice,
                               st));
      HLC_CUDA(cudaMemcpyAsync(sd[i].vals, va[i], sd[i].n * sizeof(uint32_t),
                               cudaMemcpyDeviceToDevice, st));
    }
  }
  return HLC_OK;
}

}  // namespace hlc
