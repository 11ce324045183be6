// Learned cell-offset index (the "learned index" form).
//
// The sorted unique cell keys U[0..m) of a catalogue are split into coarse
// partitions p = key >> shift (HEALPix order Lc).  Inside a partition a key is
// the relative value x = key - (p << shift) in [0, 2^shift), exact in FP32
// for shift <= 24.  Per partition a small model f_p predicts the local
// position of x in U, and the largest error e_p = max_i |f_p(x_i) - i| over the
// partition's own keys is stored.  A lookup evaluates f_p(q) and binary
// searches only [f - e_p - 1, f + e_p + 1]:
//   - PLA: 256 equal-width segments joined at the partition's cumulative key
//     counts (a monotone piecewise-linear fit of the partition's CDF); since
//     f_p is monotone, the lower bound of any query, present or absent, lies
//     in the window, so the search is exact;
//   - MLP: one input, two hidden layers of 32 ReLU units with fixed hashed
//     weights (random features shared by all partitions) and an output layer
//     fitted by least squares per partition; it is not monotone, so every
//     answer is checked against its bracket U[lb-1] < q <= U[lb] and falls
//     back to binary search over the partition when the check fails.
// The plain binary search over the partition is both the fallback and the
// reference every lookup is tested against.
#pragma once

#include "common.cuh"

namespace hlc {

constexpr int kPlaSeg = 256;
constexpr int kMlpH = 32;

struct LearnedIndex {
  const uint32_t* uniq = nullptr;  // sorted unique keys
  const uint32_t* part = nullptr;  // partition offsets into uniq, P + 1
  const float* knots = nullptr;    // PLA: P x (kPlaSeg + 1) local cumulative counts
  const float* w3 = nullptr;       // MLP: P x (kMlpH + 1) output weights (+ bias)
  const uint32_t* err = nullptr;   // P stored error bounds (ceil)
  int shift = 0;                   // key bits below the partition
  int model = 0;                   // HLC_MODEL_PLA or HLC_MODEL_MLP
  uint64_t nparts = 0;             // partitions covered; larger keys sort last
};

// Fixed random features of the MLP (a hash of the unit indices), shared by
// every partition: layer 1 is a hinge basis relu(x - j/32), layer 2 a hashed
// dense 32x32 layer with bias.
inline float mlp_hash_unit(uint32_t a) {
  a ^= a >> 16;
  a *= 0x7feb352dU;
  a ^= a >> 15;
  a *= 0x846ca68bU;
  a ^= a >> 16;
  return (float)(a >> 8) * (1.0f / 16777216.0f);  // [0, 1)
}

struct MlpFixed {
  float w2[kMlpH][kMlpH];
  float b2[kMlpH];
};
__constant__ MlpFixed d_mlp;

inline void mlp_fixed_weights(MlpFixed* m) {
  for (int i = 0; i < kMlpH; ++i) {
    for (int j = 0; j < kMlpH; ++j)
      m->w2[i][j] = mlp_hash_unit(1000u + (uint32_t)(i * kMlpH + j)) * 2.0f - 1.0f;
    m->b2[i] = (mlp_hash_unit(50000u + (uint32_t)i) - 0.5f) * 0.25f;
  }
}

// Hidden activations h2(x) for x in [0, 1).
__device__ __forceinline__ void mlp_hidden(float x, float h2[kMlpH]) {
  float h1[kMlpH];
#pragma unroll
  for (int j = 0; j < kMlpH; ++j) h1[j] = fmaxf(x - (float)j * (1.0f / kMlpH), 0.0f);
#pragma unroll
  for (int i = 0; i < kMlpH; ++i) {
    float acc = d_mlp.b2[i];
#pragma unroll
    for (int j = 0; j < kMlpH; ++j) acc = fmaf(d_mlp.w2[i][j], h1[j], acc);
    h2[i] = fmaxf(acc, 0.0f);
  }
}

__device__ __forceinline__ float learned_predict(const LearnedIndex& L, uint32_t p, uint32_t x,
                                                 uint32_t n_p) {
  if (L.model == HLC_MODEL_PLA) {
    // equal-width segments of the relative key range
    int sb = L.shift >= 8 ? L.shift - 8 : 0;  // log2 segment width
    uint32_t seg = x >> sb;
    if (seg >= (uint32_t)kPlaSeg) seg = kPlaSeg - 1;
    const float* k = L.knots + (size_t)p * (kPlaSeg + 1);
    float k0 = __ldg(k + seg), k1 = __ldg(k + seg + 1);
    float t = (float)(x - (seg << sb)) * (1.0f / (float)(1u << sb));
    return fmaf(t, k1 - k0, k0);
  }
  float h2[kMlpH];
  float xs = (float)x * (1.0f / (float)(1ull << L.shift));
  mlp_hidden(xs, h2);
  const float* w = L.w3 + (size_t)p * (kMlpH + 1);
  float y = __ldg(w + kMlpH);
#pragma unroll
  for (int i = 0; i < kMlpH; ++i) y = fmaf(__ldg(w + i), h2[i], y);
  (void)n_p;
  return y;
}

// Per partition: counts per PLA segment (to be turned into knots).
__global__ void k_pla_hist(const uint32_t* __restrict__ uniq, uint64_t m, int shift,
                           float* __restrict__ knots) {
  int sb = shift >= 8 ? shift - 8 : 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t q = uniq[i];
    uint32_t p = shift >= 32 ? 0u : (q >> shift);
    uint32_t x = q - (shift >= 32 ? 0u : (p << shift));
    uint32_t seg = x >> sb;
    if (seg >= (uint32_t)kPlaSeg) seg = kPlaSeg - 1;
    atomicAdd(knots + (size_t)p * (kPlaSeg + 1) + seg + 1, 1.0f);
  }
}

// Knots = exclusive running counts (one thread per partition; exact in
// float up to 2^24 keys per partition).
__global__ void k_pla_knots(float* __restrict__ knots, uint64_t P) {
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P;
       p += (uint64_t)gridDim.x * blockDim.x) {
    float* k = knots + p * (kPlaSeg + 1);
    float run = 0.f;
    k[0] = 0.f;
    for (int s = 1; s <= kPlaSeg; ++s) {
      run += k[s];
      k[s] = run;
    }
  }
}

// MLP output layer by least squares, one CTA per partition: normal equations
// over at most kMlpSample evenly spaced keys (accumulated per batch of 256 in
// FP32, across batches in FP64), ridge 1e-9 tr/D, Cholesky in FP64.
constexpr int kMlpSample = 2048;

__global__ void __launch_bounds__(256) k_mlp_fit(const uint32_t* __restrict__ uniq,
                                                  const uint32_t* __restrict__ part, uint64_t P,
                                                  int shift, float* __restrict__ w3) {
  constexpr int D = kMlpH + 1;
  constexpr int NPAIR = D * (D + 1) / 2;
  __shared__ float H[256][D + 1];
  __shared__ float Y[256];
  __shared__ double G[D][D];
  __shared__ double rhs[D];
  for (uint64_t p = blockIdx.x; p < P; p += gridDim.x) {
    uint32_t lo = part[p], hi = part[p + 1];
    uint32_t n = hi - lo;
    float* w = w3 + p * D;
    if (n == 0) {
      if (threadIdx.x < D) w[threadIdx.x] = 0.f;
      continue;
    }
    for (int i = threadIdx.x; i < D * D; i += blockDim.x) G[i / D][i % D] = 0.0;
    if (threadIdx.x < D) rhs[threadIdx.x] = 0.0;
    uint32_t S = n < (uint32_t)kMlpSample ? n : (uint32_t)kMlpSample;
    for (uint32_t s0 = 0; s0 < S; s0 += 256) {
      __syncthreads();
      uint32_t s = s0 + threadIdx.x;
      if (s < S) {
        uint32_t i = (uint32_t)(((uint64_t)s * n) / S);
        uint32_t x = uniq[lo + i] - (uint32_t)(p << shift);
        float h[kMlpH];
        mlp_hidden((float)x * (1.0f / (float)(1ull << shift)), h);
        for (int a = 0; a < kMlpH; ++a) H[threadIdx.x][a] = h[a];
        H[threadIdx.x][kMlpH] = 1.0f;
        Y[threadIdx.x] = (float)i;
      } else {
        for (int a = 0; a < D; ++a) H[threadIdx.x][a] = 0.f;
        Y[threadIdx.x] = 0.f;
      }
      __syncthreads();
      uint32_t cnt = min(256u, S - s0);
      for (int pr = threadIdx.x; pr < NPAIR + D; pr += blockDim.x) {
        if (pr < NPAIR) {
          int a = 0, r = pr;
          while (r >= D - a) {
            r -= D - a;
            ++a;
          }
          int b = a + r;
          float acc = 0.f;
          for (uint32_t t = 0; t < cnt; ++t) acc = fmaf(H[t][a], H[t][b], acc);
          G[a][b] += (double)acc;
        } else {
          int a = pr - NPAIR;
          float acc = 0.f;
          for (uint32_t t = 0; t < cnt; ++t) acc = fmaf(H[t][a], Y[t], acc);
          rhs[a] += (double)acc;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double tr = 0;
      for (int a = 0; a < D; ++a) tr += G[a][a];
      double ridge = 1e-9 * (tr / D) + 1e-12;
      for (int a = 0; a < D; ++a) {
        G[a][a] += ridge;
        for (int b = 0; b < a; ++b) G[a][b] = G[b][a];
      }
      for (int j = 0; j < D; ++j) {
        double d = G[j][j];
        for (int k = 0; k < j; ++k) d -= G[j][k] * G[j][k];
        d = d > 1e-300 ? sqrt(d) : 1e-150;
        G[j][j] = d;
        for (int i = j + 1; i < D; ++i) {
          double v = G[i][j];
          for (int k = 0; k < j; ++k) v -= G[i][k] * G[j][k];
          G[i][j] = v / d;
        }
      }
      double y[D];
      for (int i = 0; i < D; ++i) {
        double v = rhs[i];
        for (int k = 0; k < i; ++k) v -= G[i][k] * y[k];
        y[i] = v / G[i][i];
      }
      for (int i = D - 1; i >= 0; --i) {
        double v = y[i];
        for (int k = i + 1; k < D; ++k) v -= G[k][i] * y[k];
        y[i] = v / G[i][i];
      }
      for (int i = 0; i < D; ++i) w[i] = (float)y[i];
    }
    __syncthreads();
  }
}

// Stored error bound of each partition: ceil(max_i |f(x_i) - i|).
__global__ void k_learned_err(LearnedIndex L, uint64_t m, uint32_t* __restrict__ err) {
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < m;
       g += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t q = L.uniq[g];
    uint32_t p = q >> L.shift;
    uint32_t lo = L.part[p];
    uint32_t x = q - (p << L.shift);
    float f = learned_predict(L, p, x, L.part[p + 1] - lo);
    float e = fabsf(f - (float)(g - lo));
    uint32_t ce = (uint32_t)fminf(ceilf(e), 4.0e9f);
    atomicMax(err + p, ce);
  }
}

// Lower bound of q in uniq (exact).  *hit = answered inside the window.
__device__ __forceinline__ uint32_t learned_lower_bound(const LearnedIndex& L, uint32_t q,
                                                        bool* hit) {
  uint32_t p = q >> L.shift;
  *hit = true;
  if (p >= L.nparts) return __ldg(L.part + L.nparts);
  uint32_t lo = __ldg(L.part + p), hi = __ldg(L.part + p + 1);
  if (lo == hi) return lo;
  uint32_t x = q - (p << L.shift);
  float f = learned_predict(L, p, x, hi - lo);
  float e = (float)__ldg(L.err + p) + 1.0f;
  float flo = floorf(f - e), fhi = ceilf(f + e) + 1.0f;
  uint32_t a = flo <= 0.f ? lo : lo + (uint32_t)fminf(flo, (float)(hi - lo));
  uint32_t b = fhi <= 0.f ? lo : lo + (uint32_t)fminf(fhi, (float)(hi - lo));
  if (a > hi) a = hi;
  if (b > hi) b = hi;
  uint32_t s = a, t = b;
  while (s < t) {
    uint32_t mid = (s + t) >> 1;
    if (__ldg(L.uniq + mid) < q)
      s = mid + 1;
    else
      t = mid;
  }
  // bracket check: uniq[s-1] < q <= uniq[s] within the partition
  bool ok = (s == lo || __ldg(L.uniq + s - 1) < q) && (s == hi || __ldg(L.uniq + s) >= q);
  if (ok) return s;
  *hit = false;
  s = lo;
  t = hi;
  while (s < t) {
    uint32_t mid = (s + t) >> 1;
    if (__ldg(L.uniq + mid) < q)
      s = mid + 1;
    else
      t = mid;
  }
  return s;
}

__global__ void k_learned_lookup(LearnedIndex L, const uint32_t* __restrict__ queries,
                                 uint64_t nq, uint32_t* __restrict__ out,
                                 unsigned long long* __restrict__ hits) {
  unsigned long long h = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq;
       i += (uint64_t)gridDim.x * blockDim.x) {
    bool hit;
    out[i] = learned_lower_bound(L, queries[i], &hit);
    h += hit;
  }
  for (int o = 16; o > 0; o >>= 1) h += __shfl_down_sync(0xffffffffu, h, o);
  if ((threadIdx.x & 31) == 0 && h) atomicAdd(hits, h);
}

// The plain offset table the model replaces: binary search inside the
// query's partition.
__global__ void k_part_bsearch_lookup(LearnedIndex L, const uint32_t* __restrict__ queries,
                                      uint64_t nq, uint32_t* __restrict__ out) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t q = queries[i];
    const uint32_t p = q >> L.shift;
    if (p >= L.nparts) {
      out[i] = __ldg(L.part + L.nparts);
      continue;
    }
    uint32_t s = __ldg(L.part + p), t = __ldg(L.part + p + 1);
    while (s < t) {
      const uint32_t mid = (s + t) >> 1;
      if (__ldg(L.uniq + mid) < q)
        s = mid + 1;
      else
        t = mid;
    }
    out[i] = s;
  }
}

}  // namespace hlc
