// The C ABI (include/hlc.h): plan / match / free, the kernel-level entry
// points, device tables and error state.  All kernels live in the headers
// included here (one translation unit, so constant tables are shared).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <queue>
#include <thread>
#include <unistd.h>
#include <atomic>
#include <memory>
#include <chrono>
#include <vector>

#include "canon.cuh"
#include "common.cuh"
#include "fp32.cuh"
#include "index.cuh"
#include "learned.cuh"
#include "match.cuh"
#include "output.cuh"
#include "batch.cuh"
#include "bucket.cuh"
#include "tile.cuh"
#include "stream.cuh"
#include "scan.cuh"
#include "sort.cuh"

namespace hlc {

// ---------------------------------------------------------------------------
// Error state.
// ---------------------------------------------------------------------------
static thread_local char g_msg[1024] = "";
std::atomic<unsigned long long> g_launches{0};

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
}
void clear_error() { g_msg[0] = 0; }

// ---------------------------------------------------------------------------
// Constants and device tables.
// ---------------------------------------------------------------------------
static Canon g_canon;
static std::once_flag g_canon_once;

const Canon& canon() {
  std::call_once(g_canon_once, [] { derive_trig_coefficients(g_canon.s, g_canon.c); });
  return g_canon;
}

// Neighbour transitions from the layout of the 12 base faces: 0-3 around the
// north pole (centres at phi = 45 + 90k deg), 4-7 on the equator (phi = 90k),
// 8-11 around the south pole.  Inside a face x runs to the north-east and y
// to the north-west (south vertex (0,0), north vertex (n,n)).  Polar faces
// meet the equatorial ones edge to edge without rotation; two polar faces
// meet along a meridian, a quarter turn about the pole apart.  Four faces
// meet at the poles and at the equatorial vertices, three at z = +-2/3.
static void build_neighbour_tables(uint8_t face[12][9], uint8_t map[12][9]) {
  for (int f = 0; f < 12; ++f)
    for (int r = 0; r < 9; ++r) {
      face[f][r] = 255;
      map[f][r] = NM_SAME;
    }
  auto set = [&](int f, int rx, int ry, int g, int m) {
    face[f][ry * 3 + rx] = (uint8_t)g;
    map[f][ry * 3 + rx] = (uint8_t)m;
  };
  for (int k = 0; k < 4; ++k) {
    int north = k, eq = 4 + k, south = 8 + k;
    int k1 = (k + 1) & 3, k2 = (k + 2) & 3, k3 = (k + 3) & 3;
    set(north, 1, 1, north, NM_SAME);
    set(north, 2, 1, k1, NM_ROT_N1);
    set(north, 1, 2, k3, NM_ROT_N3);
    set(north, 0, 1, 4 + k, NM_SHIFT);
    set(north, 1, 0, 4 + k1, NM_SHIFT);
    set(north, 2, 2, k2, NM_AT_NN);      // across the north pole
    set(north, 0, 0, 8 + k, NM_AT_NN);   // across the equatorial vertex
    set(eq, 1, 1, eq, NM_SAME);
    set(eq, 2, 1, k, NM_SHIFT);
    set(eq, 1, 2, k3, NM_SHIFT);
    set(eq, 0, 1, 8 + k3, NM_SHIFT);
    set(eq, 1, 0, 8 + k, NM_SHIFT);
    set(eq, 2, 0, 4 + k1, NM_AT_0N);     // east equatorial vertex
    set(eq, 0, 2, 4 + k3, NM_AT_N0);     // west equatorial vertex
    set(south, 1, 1, south, NM_SAME);
    set(south, 2, 1, 4 + k1, NM_SHIFT);
    set(south, 1, 2, 4 + k, NM_SHIFT);
    set(south, 0, 1, 8 + k3, NM_ROT_S3);
    set(south, 1, 0, 8 + k1, NM_ROT_S1);
    set(south, 0, 0, 8 + k2, NM_AT_00);  // across the south pole
    set(south, 2, 2, k, NM_AT_00);       // across the equatorial vertex
  }
}

static std::mutex g_dev_mu;
static bool g_dev_ready[64] = {false};

int ensure_device_tables() {
  int dev = 0;
  HLC_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (dev >= 0 && dev < 64 && g_dev_ready[dev]) return HLC_OK;
  const Canon& K = canon();
  CanonDev cd;
  memcpy(cd.s, K.s, sizeof(cd.s));
  memcpy(cd.c, K.c, sizeof(cd.c));
  cd.sqrt6 = std::sqrt(6.0);
  HLC_CUDA(cudaMemcpyToSymbol(d_canon, &cd, sizeof(cd)));
  uint8_t face[12][9], map[12][9];
  build_neighbour_tables(face, map);
  HLC_CUDA(cudaMemcpyToSymbol(d_nbr_face, face, sizeof(face)));
  HLC_CUDA(cudaMemcpyToSymbol(d_nbr_map, map, sizeof(map)));
  MlpFixed mf;
  mlp_fixed_weights(&mf);
  HLC_CUDA(cudaMemcpyToSymbol(d_mlp, &mf, sizeof(mf)));
  // keep freed stream-ordered allocations cached in the device's default pool
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  if (dev >= 0 && dev < 64) g_dev_ready[dev] = true;
  return HLC_OK;
}

static int dev_err_status(int h, const char* what) {
  if (h & DERR_INPUT) {
    set_error("%s: invalid input (non-finite RA/Dec or |Dec| > 90)", what);
    return HLC_EINVAL;
  }
  if (h & DERR_TIMEOUT) {
    set_error("%s: a bounded device wait gave up", what);
    return HLC_ETIMEOUT;
  }
  if (h & DERR_BOUNDS) {
    set_error("%s: a device bounds check failed", what);
    return HLC_ECUDA;
  }
  return HLC_OK;
}

static int check_dev_err(const int* dev_err, cudaStream_t st, const char* what) {
  int h = 0;
  HLC_CUDA(cudaMemcpyAsync(&h, dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  HLC_CUDA(cudaStreamSynchronize(st));
  return dev_err_status(h, what);
}

// Events and side streams of plans come from a per-device pool and go back
// to it (creating and destroying about twenty per plan cost host time at the
// points where the GPU waits for the next launch).  An object handed back
// may still have work pending; reusing it only orders new work after that.
namespace {
std::mutex g_pool_mu;
struct DevPool {
  std::vector<cudaEvent_t> timed, plain;
  std::vector<cudaStream_t> streams;
};
DevPool g_pool[64];
DevPool& cur_pool() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) d = 0;
  return g_pool[d];
}
}  // namespace

static cudaError_t pool_event(cudaEvent_t* e, bool timed) {
  {
    std::lock_guard<std::mutex> g(g_pool_mu);
    std::vector<cudaEvent_t>& v = timed ? cur_pool().timed : cur_pool().plain;
    if (!v.empty()) {
      *e = v.back();
      v.pop_back();
      return cudaSuccess;
    }
  }
  return timed ? cudaEventCreate(e) : cudaEventCreateWithFlags(e, cudaEventDisableTiming);
}
static void pool_event_back(cudaEvent_t e, bool timed) {
  if (!e) return;
  std::lock_guard<std::mutex> g(g_pool_mu);
  (timed ? cur_pool().timed : cur_pool().plain).push_back(e);
}
static cudaError_t pool_stream(cudaStream_t* s) {
  {
    std::lock_guard<std::mutex> g(g_pool_mu);
    std::vector<cudaStream_t>& v = cur_pool().streams;
    if (!v.empty()) {
      *s = v.back();
      v.pop_back();
      return cudaSuccess;
    }
  }
  return cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
}
static void pool_stream_back(cudaStream_t s) {
  if (!s) return;
  std::lock_guard<std::mutex> g(g_pool_mu);
  cur_pool().streams.push_back(s);
}

// Theta_L / 8 in arcsec: the largest radius for which the complete rule is exact.
static double complete_max_radius(int order) {
  const double pi = 3.14159265358979323846;
  return std::sqrt(pi / 3.0) / std::ldexp(1.0, order) * (648000.0 / pi) / 8.0;
}

// Squared-chord threshold 4 sin^2(r/2) in the canonical arithmetic (host).
static double host_sincos_deg_sin(double x) {
  const Canon& K = canon();
  volatile double q = std::rint(x / 90.0);
  volatile double t = x - 90.0 * q;
  volatile double u = t * t;
  double ps = K.s[9];
  for (int k = 8; k >= 0; --k) ps = std::fma(ps, u, K.s[k]);
  volatile double sn = t * ps;
  double pc = K.c[10];
  for (int k = 9; k >= 0; --k) pc = std::fma(pc, u, K.c[k]);
  switch (((long long)q) & 3) {
    case 0: return sn;
    case 1: return pc;
    case 2: return -sn;
    default: return -pc;
  }
}
static double chord2_threshold(double r_arcsec) {
  volatile double h = r_arcsec / 7200.0;
  volatile double sh = host_sincos_deg_sin(h);
  volatile double sq = sh * sh;
  return 4.0 * sq;
}

// ---------------------------------------------------------------------------
// Plan.
// ---------------------------------------------------------------------------
struct CatDev {
  uint64_t n = 0, m = 0;
  uint32_t* key = nullptr;   // sorted cell keys of the entries
  uint32_t* idx = nullptr;   // source of each sorted entry
  double *vx = nullptr, *vy = nullptr, *vz = nullptr;
  double* ve = nullptr;        // Eq. 4, binary64 form: entry-ordered error radii
  float4* v32 = nullptr;
  double2* rd = nullptr;       // entry-ordered (ra, dec) (batched plans)
  uint64_t* id_s = nullptr;    // entry-ordered ids (batched plans)
  SrcRec* rec = nullptr;       // (ra, dec, id) of each source, input order
  uint32_t* cells5 = nullptr;  // quad: cell set of each source
  uint32_t* table = nullptr;   // coarse offset table (catalogue B)
  int table_shift = 0;
  int table_order = 0;
  uint64_t cells = 0;
  // learned index (catalogue B, HLC_INDEX_LEARNED)
  uint32_t* uniq = nullptr;
  uint32_t* start = nullptr;
  uint64_t u = 0;
  LearnedIndex learned;
  uint64_t parts = 0;
  // FP32 complete form: entries in dense table cells of B (fine-ordered)
  uint64_t ndense = 0;
  // catalogue A: dense fine cells for the tile kernel
  uint32_t* tile_cell = nullptr;
  uint32_t* tile_start = nullptr;
  uint32_t* tile_dpos = nullptr;
  unsigned long long* tile_n = nullptr;  // device: runs, items taken, their entries
  uint8_t* tiled = nullptr;              // 1 for A entries the tile kernel takes
  TileItem* tile_items = nullptr;        // prepared items (B ranges found)
  unsigned long long* tile_nprep = nullptr;  // items placed from the front, from the back
  uint64_t tile_icap = 0;                     // capacity of tile_items
};

// Pinned host memory of streamed plans (the pass-1 runs, the groups' result
// rows, the merged output), pooled between plans: pinning tens of GB takes
// seconds, so released blocks are kept (up to half of the host's physical
// memory) and handed to later requests of the same or a slightly smaller
// size.
static std::mutex g_pin_mu;
static std::vector<std::pair<char*, size_t>> g_pin_pool;
static size_t g_pin_total = 0;

static size_t pinned_pool_limit() {
  const long pages = sysconf(_SC_PHYS_PAGES), psz = sysconf(_SC_PAGE_SIZE);
  return pages > 0 && psz > 0 ? (size_t)pages * (size_t)psz / 2 : (size_t)16 << 30;
}

static char* pinned_acquire(size_t* bytes) {
  {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    size_t best = SIZE_MAX;
    for (size_t i = 0; i < g_pin_pool.size(); ++i) {
      const size_t sz = g_pin_pool[i].second;
      if (sz >= *bytes && sz <= 2 * *bytes + (64u << 20) &&
          (best == SIZE_MAX || sz < g_pin_pool[best].second))
        best = i;
    }
    if (best != SIZE_MAX) {
      char* p = g_pin_pool[best].first;
      *bytes = g_pin_pool[best].second;
      g_pin_total -= *bytes;
      g_pin_pool.erase(g_pin_pool.begin() + best);
      return p;
    }
  }
  void* p = nullptr;
  if (cudaHostAlloc(&p, *bytes, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (char*)p;
}

static void pinned_release(char* p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_pool.push_back({p, bytes});
  g_pin_total += bytes;
  const size_t limit = pinned_pool_limit();
  while (g_pin_total > limit && !g_pin_pool.empty()) {  // drop the oldest blocks
    cudaFreeHost(g_pin_pool.front().first);
    g_pin_total -= g_pin_pool.front().second;
    g_pin_pool.erase(g_pin_pool.begin());
  }
}

// A pooled pinned block owned by one user.
struct PinnedBuf {
  char* p = nullptr;
  size_t bytes = 0;
  PinnedBuf() = default;
  PinnedBuf(const PinnedBuf&) = delete;
  PinnedBuf& operator=(const PinnedBuf&) = delete;
  PinnedBuf(PinnedBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
  ~PinnedBuf() { reset(); }
  bool get(size_t b) {
    reset();
    bytes = b;
    p = pinned_acquire(&bytes);
    return p != nullptr;
  }
  void reset() {
    pinned_release(p, bytes);
    p = nullptr;
    bytes = 0;
  }
};

enum Ctr { C_ROWS = 0, C_BAND, C_TESTS, C_DUPS, C_M, C_TOTAL, C_HEADS_A, C_HEADS_B, C_DENSE,
           C_WORK, C_IDDIFF, C_MAXB, C_SLOW, C_LHITS, C_LLOOK, C_LMAXERR, C_SCRATCH, C_BAND64,
           C_SLOW_A, C_EMAXA, C_EMAXB, C_TILE_TESTS, C_DCELLS, C_N };

}  // namespace hlc

struct hlc_plan_s {
  hlc_params p{};
  hlc::Allocator al;
  hlc::Arena* arena = nullptr;   // plan lifetime
  hlc::Arena* out = nullptr;     // last result
  hlc::CatDev A, B;
  double C = 0;
  double r_lo = 0, r_hi = 0;  // separations left to the binary64 recheck
  bool eq4 = false;           // per-source radii (Eq. 4)
  // tile kernel shape (the rule, or a batched plan's hlc_tune)
  uint32_t tile_ka[3] = {hlc::kTileRuleKA[0], hlc::kTileRuleKA[1], hlc::kTileRuleKA[2]};
  uint32_t tile_stage = hlc::kTileCap;
  double target_per_cell = 0;  // batched order rule (0: kTargetPerCell)
  double k9 = 0;              // 9 (pi/648000)^2: squared pair radius per squared error
  double eq4_rmax = 0;        // largest pair radius (arcsec)
  double eq4_rho_max = 0;     // bound on rho_a + rho_b (squared chord)
  float lo32 = 0, hi32 = 0;
  int join_level = 0;
  int nslot = 9;
  int* dev_err = nullptr;
  unsigned long long* ctr = nullptr;
  hlc_stats stats{};
  unsigned long long launches0 = 0;
  int id_high_bit = -1;
  uint64_t row_cap = 0;
  // batched plans
  uint32_t njobs = 1;
  int cell_bits = 0;
  std::vector<hlc::JobDev> jobs_h;
  hlc::JobDev* jobs_d = nullptr;
  uint64_t* offA_d = nullptr;
  uint64_t* offB_d = nullptr;
  uint64_t* keyA64 = nullptr;
  uint64_t* keyB64 = nullptr;
  uint32_t* btable = nullptr;
  cudaGraphExec_t pair_graph = nullptr;
  uint64_t graph_cap = 0, graph_bcap = 0;
  void* graph_rows = nullptr;
  void* graph_band = nullptr;
  // streamed plans: merged rows on the host
  bool streamed = false;
  hlc::PinnedBuf host_buf;  // streamed plans: the merged rows (pinned, pooled)
  uint64_t host_n = 0;
  uint64_t *host_a = nullptr, *host_b = nullptr;
  double* host_s = nullptr;
  uint32_t sparse_cell = hlc::kSparseCell;
  uint32_t* dcells = nullptr;  // dense cells of B's table, ascending (count at ctr[C_DCELLS])
  bool table_buckets = false;  // FP32 complete mode: entries bucketed by table cell
  uint32_t sort_passes = 0;    // radix passes of the table-cell sorts (ev 7-8: B, 9-10: A)
  uint64_t sort_entries = 0;   // entries those passes moved, summed over the launches
  uint64_t sort_bytes = 0;     // and their algorithmic bytes
  bool sort_timed[2] = {false, false};
  unsigned long long plan_launches = 0;
  cudaEvent_t ev[12] = {};
  bool events = false;
};

namespace hlc {

static cudaStream_t plan_stream(const hlc_plan_t* P) { return (cudaStream_t)P->p.stream; }

static int validate_params(const hlc_params* p) {
  if (!p) {
    set_error("params is NULL");
    return HLC_EINVAL;
  }
  if (p->radius_rule != HLC_RADIUS_FIXED && p->radius_rule != HLC_RADIUS_EQ4) {
    set_error("radius_rule must be HLC_RADIUS_FIXED or HLC_RADIUS_EQ4");
    return HLC_EINVAL;
  }
  const bool eq4 = p->radius_rule == HLC_RADIUS_EQ4;
  if (!eq4 && (!(p->radius_arcsec > 0.0) || !(p->radius_arcsec <= 648000.0))) {
    set_error("radius_arcsec must be in (0, 648000], got %g", p->radius_arcsec);
    return HLC_EINVAL;
  }
  if (p->fine_level < 0 || p->fine_level > 14) {
    set_error("fine_level must be in [0, 14], got %d", p->fine_level);
    return HLC_EINVAL;
  }
  if (p->coarse_level < 0 || p->coarse_level > p->fine_level) {
    set_error("coarse_level must be in [0, fine_level], got %d", p->coarse_level);
    return HLC_EINVAL;
  }
  if (p->boundary != HLC_COMPLETE8 && p->boundary != HLC_QUAD &&
      p->boundary != HLC_QUAD_COSDEC) {
    set_error("boundary must be HLC_COMPLETE8, HLC_QUAD or HLC_QUAD_COSDEC");
    return HLC_EINVAL;
  }
  if (p->precision != HLC_FP64 && p->precision != HLC_FP32_GUARD) {
    set_error("precision must be HLC_FP64 or HLC_FP32_GUARD");
    return HLC_EINVAL;
  }
  if (p->index != HLC_INDEX_BSEARCH && p->index != HLC_INDEX_LEARNED) {
    set_error("index must be HLC_INDEX_BSEARCH or HLC_INDEX_LEARNED");
    return HLC_EINVAL;
  }
  if (p->model != HLC_MODEL_PLA && p->model != HLC_MODEL_MLP) {
    set_error("model must be HLC_MODEL_PLA or HLC_MODEL_MLP");
    return HLC_EINVAL;
  }
  if (!eq4 && p->boundary == HLC_COMPLETE8 &&
      p->radius_arcsec > complete_max_radius(p->fine_level)) {
    set_error("radius %g arcsec exceeds theta_L/8 = %g arcsec at fine_level %d (complete mode)",
              p->radius_arcsec, complete_max_radius(p->fine_level), p->fine_level);
    return HLC_EINVAL;
  }
  if (eq4 && (p->boundary != HLC_COMPLETE8 || p->index != HLC_INDEX_BSEARCH)) {
    set_error("HLC_RADIUS_EQ4 is implemented for complete mode with the binary-searched index");
    return HLC_EUNSUPPORTED;
  }
  if (p->tune) {
    const hlc_tune& t = *p->tune;
    bool ok = t.target_per_cell > 0.0 && t.target_per_cell <= 1e6 && t.stage >= 8 &&
              t.stage <= (uint32_t)kTileCap && t.stage % 8 == 0;
    for (int c = 0; c < 3; ++c) ok = ok && (t.ka[c] == 1 || t.ka[c] == 2 || t.ka[c] == 4);
    if (!ok) {
      set_error("tune: target_per_cell must be > 0, ka in {1, 2, 4}, stage a multiple of 8 in "
                "[8, %d]", kTileCap);
      return HLC_EINVAL;
    }
  }
  if ((p->alloc == nullptr) != (p->dealloc == nullptr)) {
    set_error("alloc and dealloc must both be set or both be NULL");
    return HLC_EINVAL;
  }
  return HLC_OK;
}

static int validate_catalog(const hlc_catalog* c, const char* name) {
  if (!c) {
    set_error("catalogue %s is NULL", name);
    return HLC_EINVAL;
  }
  if (c->n >= (1ull << 31)) {
    set_error("catalogue %s has %llu sources; the limit is 2^31 - 1", name,
              (unsigned long long)c->n);
    return HLC_EINVAL;
  }
  if (c->n && (!c->ra_deg || !c->dec_deg || !c->id)) {
    set_error("catalogue %s has NULL arrays", name);
    return HLC_EINVAL;
  }
  return HLC_OK;
}

static void ev_record(hlc_plan_t* P, int i) {
  if (P->events) cudaEventRecord(P->ev[i], plan_stream(P));
}
static float ev_ms(hlc_plan_t* P, int a, int b) {
  float ms = 0;
  if (P->events) cudaEventElapsedTime(&ms, P->ev[a], P->ev[b]);
  return ms;
}

// Learned index over sorted unique keys uniq[0..m): partition offsets, the
// per-partition model and its stored error bound.  P = number of partitions.
static int build_learned(Arena& ar, const uint32_t* uniq, uint64_t m, int shift, int model,
                         uint64_t P, unsigned long long* total_dev,
                         unsigned long long* scratch_ctr, int* dev_err, cudaStream_t st,
                         LearnedIndex* out) {
  uint32_t* hist = ar.get_n<uint32_t>(P + 1);
  uint32_t* part = ar.get_n<uint32_t>(P + 1);
  uint32_t* err = ar.get_n<uint32_t>(P + 1);
  void* scr = ar.get(scan_scratch_bytes(P + 1));
  if (!hist || !part || !err || !scr) return HLC_ENOMEM;
  HLC_CUDA(cudaMemsetAsync(hist, 0, (P + 1) * 4, st));
  HLC_CUDA(cudaMemsetAsync(err, 0, (P + 1) * 4, st));
  if (m) {
    k_coarse_hist<<<grid_for(m, kThreads), kThreads, 0, st>>>(uniq, m, shift, hist, scratch_ctr);
    HLC_LAUNCH_CHECK();
  }
  HLC_TRY(scan_exclusive<uint32_t>(hist, part, P + 1, total_dev, scr, dev_err, st));
  ar.drop(hist);
  ar.drop(scr);
  LearnedIndex L;
  L.uniq = uniq;
  L.part = part;
  L.err = err;
  L.shift = shift;
  L.model = model;
  L.nparts = P;
  if (model == HLC_MODEL_NONE) {  // partition offsets only
    *out = L;
    return HLC_OK;
  }
  if (model == HLC_MODEL_PLA) {
    float* knots = ar.get_n<float>(P * (kPlaSeg + 1) + 1);
    if (!knots) return HLC_ENOMEM;
    HLC_CUDA(cudaMemsetAsync(knots, 0, (P * (kPlaSeg + 1) + 1) * 4, st));
    if (m) {
      k_pla_hist<<<grid_for(m, kThreads), kThreads, 0, st>>>(uniq, m, shift, knots);
      HLC_LAUNCH_CHECK();
    }
    k_pla_knots<<<grid_for(P, kThreads), kThreads, 0, st>>>(knots, P);
    HLC_LAUNCH_CHECK();
    L.knots = knots;
  } else {
    float* w3 = ar.get_n<float>(P * (kMlpH + 1) + 1);
    if (!w3) return HLC_ENOMEM;
    k_mlp_fit<<<(unsigned)std::min<uint64_t>(P, num_sms() * 8u), 256, 0, st>>>(uniq, part, P, shift,
                                                                          w3);
    HLC_LAUNCH_CHECK();
    L.w3 = w3;
  }
  if (m) {
    k_learned_err<<<grid_for(m, kThreads), kThreads, 0, st>>>(L, m, err);
    HLC_LAUNCH_CHECK();
  }
  *out = L;
  return HLC_OK;
}

// Offset table T[0..S] of m keys sorted by (key >> shift): tile bounds,
// then one CTA per tile of slots.
static int offset_table(hlc_plan_t* P, const uint32_t* keys, uint64_t m, int shift, uint64_t S,
                        uint32_t* T, unsigned long long* heads, uint32_t dense_above,
                        unsigned long long* ndense) {
  Arena& ar = *P->arena;
  cudaStream_t st = plan_stream(P);
  const uint64_t nt = (S + kTabTile) / kTabTile;  // tiles over the S + 1 slots
  uint32_t* bnd = ar.get_n<uint32_t>(nt + 1);
  if (!bnd) return HLC_ENOMEM;
  k_table_bounds<<<grid_for(32 * (nt + 1), kThreads), kThreads, 0, st>>>(keys, m, shift, S, nt,
                                                                         bnd);
  HLC_LAUNCH_CHECK();
  k_table_tiles<<<(unsigned)std::min<uint64_t>(nt, num_sms() * 64u), kTabThreads, 0, st>>>(
      keys, m, shift, S, nt, bnd, T, heads, dense_above, ndense);
  HLC_LAUNCH_CHECK();
  ar.drop(bnd);
  return HLC_OK;
}

// Fine order inside dense table cells (those of B's table T holding more than
// sparse_cell B entries): the dense cells are listed from T, their entries in
// X gathered in cell order, radix sorted by fine key and written back.  With
// items set, the sorted dense keys are also run-length encoded into the tile
// kernel's work items.
static int dense_fixup(hlc_plan_t* P, CatDev& X, const uint32_t* T, int shift, bool items) {
  Arena& ar = *P->arena;
  cudaStream_t st = plan_stream(P);
  const uint64_t n = X.n;
  const int bits = 2 * P->p.fine_level + 4;
  // the dense cells of B's table T (listed by B's pass, reused by A's):
  // each holds more than sparse_cell of B's entries, which bounds their number
  const uint64_t S = 12ull << (2 * P->B.table_order);
  const uint64_t cap = P->B.n / ((uint64_t)P->sparse_cell + 1) + 1;
  if (T == X.table || !P->dcells) {
    const uint64_t nblk = (S + kDenseBlkSlots - 1) / kDenseBlkSlots;
    uint32_t* blkcnt = ar.get_n<uint32_t>(nblk + 1);
    uint32_t* blkoff = ar.get_n<uint32_t>(nblk + 1);
    void* bscr = ar.get(scan_scratch_bytes(nblk));
    P->dcells = ar.get_n<uint32_t>(cap);
    if (!blkcnt || !blkoff || !bscr || !P->dcells) return HLC_ENOMEM;
    k_dense_cell_blocks<<<(unsigned)nblk, 256, 0, st>>>(T, S, P->sparse_cell, blkcnt);
    HLC_LAUNCH_CHECK();
    HLC_TRY(scan_exclusive<uint32_t>(blkcnt, blkoff, nblk, P->ctr + C_DCELLS, bscr, P->dev_err,
                                     st));
    k_dense_cell_list<<<(unsigned)nblk, 256, 0, st>>>(T, S, P->sparse_cell, blkoff, P->dcells);
    HLC_LAUNCH_CHECK();
    for (void* q : {(void*)blkcnt, (void*)blkoff, bscr}) ar.drop(q);
  }
  // their entry ranges in X (from the table for B, by search in A's keys),
  // offsets by a scan over the (bounded) list, the total read back
  uint2* rng = ar.get_n<uint2>(cap);
  uint32_t* len = ar.get_n<uint32_t>(cap + 1);
  uint32_t* off = ar.get_n<uint32_t>(cap + 1);
  void* scr = ar.get(scan_scratch_bytes(cap + 1));
  if (!rng || !len || !off || !scr) return HLC_ENOMEM;
  HLC_CUDA(cudaMemsetAsync(len, 0, (cap + 1) * 4, st));
  k_dense_cell_ranges<<<grid_for(cap, kThreads), kThreads, 0, st>>>(
      P->dcells, P->ctr + C_DCELLS, T, T == X.table ? nullptr : X.key, n, shift, rng, len);
  HLC_LAUNCH_CHECK();
  HLC_TRY(scan_exclusive<uint32_t>(len, off, cap + 1, P->ctr + C_TOTAL, scr, P->dev_err, st));
  unsigned long long nd = 0;
  HLC_CUDA(cudaMemcpyAsync(&nd, P->ctr + C_TOTAL, 8, cudaMemcpyDeviceToHost, st));
  HLC_CUDA(cudaStreamSynchronize(st));
  X.ndense = nd;
  if (nd == 0) {
    for (void* q : {(void*)rng, (void*)len, (void*)off, scr}) ar.drop(q);
    return HLC_OK;
  }
  uint32_t* dpos = ar.get_n<uint32_t>(nd);
  uint32_t* dkey = ar.get_n<uint32_t>(nd);
  uint32_t* dval = ar.get_n<uint32_t>(nd);
  uint32_t* tk = ar.get_n<uint32_t>(nd);
  uint32_t* tv = ar.get_n<uint32_t>(nd);
  float4* tvec = ar.get_n<float4>(nd);
  void* sscr = ar.get(sort_scratch_bytes(nd, (bits + 7) / 8));
  if (!dpos || !dkey || !dval || !tk || !tv || !tvec || !sscr) return HLC_ENOMEM;
  k_dense_fill<<<grid_for(nd, kThreads), kThreads, 0, st>>>(rng, off, P->ctr + C_DCELLS, nd,
                                                             X.key, dpos, dkey, dval);
  HLC_LAUNCH_CHECK();
  if (nd > 1)
    HLC_TRY(radix_sort_pairs<uint32_t>(dkey, dval, tk, tv, nd, bits, sscr, P->dev_err, st));
  k_dense_gather<<<grid_for(nd, kThreads), kThreads, 0, st>>>(dpos, dval, nd, X.idx, X.v32, tv,
                                                              tvec);
  HLC_LAUNCH_CHECK();
  k_dense_scatter<<<grid_for(nd, kThreads), kThreads, 0, st>>>(dpos, nd, dkey, tv, tvec, X.key,
                                                               X.idx, X.v32);
  HLC_LAUNCH_CHECK();
  for (void* q : {(void*)rng, (void*)len, (void*)off, scr, (void*)dval, (void*)tk, (void*)tv,
                  (void*)tvec, sscr})
    ar.drop(q);
  if (!items) {
    ar.drop(dpos);
    ar.drop(dkey);
    return HLC_OK;
  }
  // items: runs of equal key among the sorted dense entries
  uint32_t* cell_of = ar.get_n<uint32_t>(nd + 1);
  void* rscr = ar.get(scan_scratch_bytes(nd));
  HLC_ALLOC(ar, X.tile_cell, uint32_t, nd + 1);
  HLC_ALLOC(ar, X.tile_start, uint32_t, nd + 2);
  HLC_ALLOC(ar, X.tile_n, unsigned long long, 4);
  HLC_ALLOC(ar, X.tiled, uint8_t, n + 1);
  if (!cell_of || !rscr) return HLC_ENOMEM;
  HLC_CUDA(cudaMemsetAsync(X.tile_n, 0, 32, st));
  HLC_TRY(cell_table(dkey, nd, 0, cell_of, X.tile_cell, X.tile_start, X.tile_n, rscr, P->dev_err,
                     st));
  HLC_CUDA(cudaMemsetAsync(X.tiled, 0, n + 1, st));
  k_mark_tiled<<<grid_for(nd, kThreads, num_sms() * 8u), kThreads, 0, st>>>(X.tile_start, dpos,
                                                                       X.tile_n, X.tiled);
  HLC_LAUNCH_CHECK();
  X.tile_dpos = dpos;
  {  // the B ranges of every item, ahead of the pair test
    const uint64_t cap = nd / kTileItemDiv + 1;
    X.tile_icap = cap;
    HLC_ALLOC(ar, X.tile_items, TileItem, cap);
    HLC_ALLOC(ar, X.tile_nprep, unsigned long long, 2);
    HLC_CUDA(cudaMemsetAsync(X.tile_nprep, 0, 16, st));
    TileArgs ta{};
    ta.cell = X.tile_cell;
    ta.start = X.tile_start;
    ta.dpos = dpos;
    ta.nitems = X.tile_n;
    ta.lo32 = P->lo32;
    ta.hi32 = P->hi32;
    ta.sparse_cell = P->sparse_cell;
    ta.bix.keys = P->B.key;
    ta.bix.table = P->B.table;
    ta.bix.shift = P->B.table_shift;
    ta.order = P->join_level;
    k_tile_items<false><<<num_sms() * 16u, 256, 0, st>>>(ta, X.tile_items, X.tile_nprep, cap);
    HLC_LAUNCH_CHECK();
  }
  ar.drop(cell_of);
  ar.drop(rscr);
  ar.drop(dkey);
  return HLC_OK;
}

// Blocks of the batched prep the GPU holds at once (its grid, so that each
// block flushes its digit counts once).
static unsigned bprep_resident_blocks(bool fast) {
  static unsigned blocks[2] = {0, 0};
  unsigned& r = blocks[fast ? 1 : 0];
  if (!r) {
    int b = 0;
    const cudaError_t e =
        fast ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_bprep_keys<true>, kThreads, 0)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_bprep_keys<false>, kThreads, 0);
    if (e != cudaSuccess || b < 1) {
      cudaGetLastError();
      b = 1;
    }
    r = (unsigned)b * num_sms();
  }
  return r;
}

// Blocks of the guarded prep the GPU holds at once (a grid of at most this
// many runs in one wave, each block flushing its digit counts once).
static unsigned prep_resident_blocks() {
  static const unsigned blocks = [] {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_prep_keys<true>, kThreads, 0) !=
            cudaSuccess || b < 1) {
      cudaGetLastError();
      b = 1;
    }
    return (unsigned)b * num_sms();
  }();
  return blocks;
}

// FP32 complete-mode build: entries sorted by table cell only (the radix sort
// runs over the key bits above the fine bits of a table cell, one pass fewer
// at the usual orders) and the FP32 payload gathered in that order.  B gets
// its offset table and fine order inside its dense table cells (the only ones
// the pair test searches; sparse table cells are read whole).  A, built after
// B, is grouped by B's table cells and gets fine order (and tile-kernel work
// items) where B's table cells are dense.
static int bucket_catalog(hlc_plan_t* P, CatDev& X, bool is_b, const double* ra,
                          const double* dec, const uint64_t* id, const double* perr,
                          cudaEvent_t ev[4]) {
  Arena& ar = *P->arena;
  cudaStream_t st = plan_stream(P);
  const int L = P->p.fine_level;
  const uint64_t n = X.n;
  X.m = n;
  X.table_order = is_b ? coarse_table_order(n, L) : P->B.table_order;
  X.table_shift = 2 * (L - X.table_order);
  const uint64_t tsize = 12ull << (2 * X.table_order);
  const int shift = X.table_shift;
  const int bits = 2 * L + 4;
  HLC_ALLOC(ar, X.key, uint32_t, n + 1);
  HLC_ALLOC(ar, X.idx, uint32_t, n + 1);
  if (n) {
    uint32_t* slow = ar.get_n<uint32_t>(n + 1);
    if (!slow) return HLC_ENOMEM;
    HLC_CUDA(cudaMemsetAsync(P->ctr + C_SLOW, 0, 8, st));
    k_prep_keys<true><<<grid_for(n, kThreads), kThreads, 0, st>>>(
        ra, dec, id, n, L, pix_const(L), X.key, X.idx, X.rec, slow, P->ctr + C_SLOW, P->dev_err,
        P->eq4 ? perr : nullptr);
    HLC_LAUNCH_CHECK();
    k_prep_fallback<<<num_sms() * 4u, kThreads, 0, st>>>(ra, dec, L, slow, P->ctr + C_SLOW, X.key,
                                                          X.rec);
    HLC_LAUNCH_CHECK();
    ar.drop(slow);
  }
  cudaEventRecord(ev[1], st);
  if (n > 1) {
    uint32_t* tk = ar.get_n<uint32_t>(n);
    uint32_t* tv = ar.get_n<uint32_t>(n);
    void* scr = ar.get(sort_scratch_bytes(n, (bits - shift + 7) / 8));
    if (!tk || !tv || !scr) return HLC_ENOMEM;
    bool in_tmp = false;
    int np = 0;
    cudaEvent_t* pev = P->events ? P->ev + (is_b ? 7 : 9) : nullptr;
    HLC_TRY(radix_sort_pairs<uint32_t>(X.key, X.idx, tk, tv, n, bits, scr, P->dev_err, st, shift,
                                       &in_tmp, pev, &np));
    P->sort_passes += np;
    if (pev) P->sort_timed[is_b ? 0 : 1] = true;
    P->sort_entries += (uint64_t)np * n;
    P->sort_bytes += 16ull * np * n;
    ar.drop(scr);
    if (in_tmp) {
      std::swap(X.key, tk);
      std::swap(X.idx, tv);
    }
    ar.drop(tk);
    ar.drop(tv);
  }
  HLC_ALLOC(ar, X.v32, float4, n + 1);
  if (n) {
    if (P->eq4)
      k_payload32<true><<<grid_for(n, kThreads), kThreads, 0, st>>>(
          X.rec, X.idx, n, X.v32, is_b ? nullptr : P->ctr + C_IDDIFF, is_b ? -1.f : 1.f, P->k9);
    else
      k_payload32<false><<<grid_for(n, kThreads), kThreads, 0, st>>>(
          X.rec, X.idx, n, X.v32, is_b ? nullptr : P->ctr + C_IDDIFF);
    HLC_LAUNCH_CHECK();
  }
  cudaEventRecord(ev[2], st);
  if (!is_b) {
    if (n > 1 && P->B.ndense > 0) HLC_TRY(dense_fixup(P, X, P->B.table, shift, true));
    return HLC_OK;
  }
  HLC_ALLOC(ar, X.table, uint32_t, tsize + 1);
  HLC_TRY(offset_table(P, X.key, n, shift, tsize, X.table, P->ctr + C_HEADS_B, P->sparse_cell,
                       P->ctr + C_DENSE));
  if (n > 1) {
    unsigned long long nd = 0;
    HLC_CUDA(cudaMemcpyAsync(&nd, P->ctr + C_DENSE, 8, cudaMemcpyDeviceToHost, st));
    HLC_CUDA(cudaStreamSynchronize(st));
    X.ndense = nd;
    if (nd > 0) HLC_TRY(dense_fixup(P, X, X.table, shift, false));
  }
  return HLC_OK;
}

// The FP32 complete form with device inputs builds both catalogues at once
// (A needs only B's table order, a function of B's size): the two preps run
// side by side, A's on the side stream ks; the two radix sorts then run as
// one sort of both arrays on the plan stream (a launch per digit pass covers
// the tiles of both); the two payloads and B's offset table overlap again.
// Every buffer A uses on ks is allocated first, on the plan stream, and
// handed over through ea[0] and e_sorted; the caller joins by making the
// plan stream wait for ea[2] (A's payload done) before A's dense cells are
// ordered against B's table.
static int bucket_pair(hlc_plan_t* P, const hlc_catalog* inB, const hlc_catalog* inA,
                       cudaStream_t ks, cudaEvent_t eb[4], cudaEvent_t ea[4],
                       cudaEvent_t e_sorted) {
  Arena& ar = *P->arena;
  cudaStream_t st = plan_stream(P);
  const int L = P->p.fine_level;
  const int bits = 2 * L + 4;
  CatDev& XB = P->B;
  CatDev& XA = P->A;
  const uint64_t nb = inB->n, na = inA->n;
  XB.n = XB.m = nb;
  XA.n = XA.m = na;
  XB.table_order = XA.table_order = coarse_table_order(nb, L);
  XB.table_shift = XA.table_shift = 2 * (L - XB.table_order);
  const int shift = XB.table_shift;
  const int npass = (bits - shift + 7) / 8;
  const uint64_t tsize = 12ull << (2 * XB.table_order);
  // the preps' buffers of both, and A's payload
  HLC_ALLOC(ar, XB.rec, SrcRec, nb + 1);
  HLC_ALLOC(ar, XB.key, uint32_t, nb + 1);
  HLC_ALLOC(ar, XB.idx, uint32_t, nb + 1);
  HLC_ALLOC(ar, XA.rec, SrcRec, na + 1);
  HLC_ALLOC(ar, XA.key, uint32_t, na + 1);
  HLC_ALLOC(ar, XA.idx, uint32_t, na + 1);
  HLC_ALLOC(ar, XA.v32, float4, na + 1);
  uint32_t *slow_b = nullptr, *slow_a = nullptr;
  HLC_ALLOC(ar, slow_b, uint32_t, nb + 1);
  HLC_ALLOC(ar, slow_a, uint32_t, na + 1);
  HLC_CUDA(cudaMemsetAsync(P->ctr + C_SLOW, 0, 8, st));
  HLC_CUDA(cudaMemsetAsync(P->ctr + C_SLOW_A, 0, 8, st));
  // the sort's scratch, whose digit histograms the preps count as they
  // write the keys (when both catalogues need sorting: the one-sort form,
  // whose first pass also makes the identity values the preps then skip)
  void *scrb = nullptr, *scra = nullptr;
  const bool both = nb > 1 && na > 1;
  if (nb > 1) {
    scrb = ar.get(sort_scratch_bytes(nb, npass));
    if (!scrb) return HLC_ENOMEM;
  }
  if (na > 1) {
    scra = ar.get(sort_scratch_bytes(na, npass));
    if (!scra) return HLC_ENOMEM;
  }
  if (both) {
    HLC_CUDA(cudaMemsetAsync(scrb, 0, (size_t)npass * 256 * 4, st));
    HLC_CUDA(cudaMemsetAsync(scra, 0, (size_t)npass * 256 * 4, st));
  }
  uint32_t* hist_b = both ? (uint32_t*)scrb : nullptr;
  uint32_t* hist_a = both ? (uint32_t*)scra : nullptr;
  HLC_CUDA(cudaEventRecord(eb[0], st));
  HLC_CUDA(cudaEventRecord(ea[0], st));
  HLC_CUDA(cudaStreamWaitEvent(ks, ea[0], 0));
  // 1. the two preps, side by side: each with half the blocks the GPU holds
  // at once (one wave between them; each block flushes its digit counts once)
  const unsigned prep_grid = std::max(1u, prep_resident_blocks() / 2);
  if (na) {
    k_prep_keys<true><<<grid_for(na, kThreads, prep_grid), kThreads, 0, ks>>>(
        inA->ra_deg, inA->dec_deg, inA->id, na, L, pix_const(L), XA.key,
        both ? nullptr : XA.idx, XA.rec, slow_a, P->ctr + C_SLOW_A, P->dev_err,
        P->eq4 ? inA->err_arcsec : nullptr, hist_a, shift, npass);
    HLC_LAUNCH_CHECK();
    k_prep_fallback<<<num_sms() * 4u, kThreads, 0, ks>>>(inA->ra_deg, inA->dec_deg, L, slow_a,
                                                  P->ctr + C_SLOW_A, XA.key, XA.rec, hist_a,
                                                  shift, npass);
    HLC_LAUNCH_CHECK();
  }
  HLC_CUDA(cudaEventRecord(ea[1], ks));
  if (nb) {
    k_prep_keys<true><<<grid_for(nb, kThreads, prep_grid), kThreads, 0, st>>>(
        inB->ra_deg, inB->dec_deg, inB->id, nb, L, pix_const(L), XB.key,
        both ? nullptr : XB.idx, XB.rec, slow_b, P->ctr + C_SLOW, P->dev_err,
        P->eq4 ? inB->err_arcsec : nullptr, hist_b, shift, npass);
    HLC_LAUNCH_CHECK();
    k_prep_fallback<<<num_sms() * 4u, kThreads, 0, st>>>(inB->ra_deg, inB->dec_deg, L, slow_b,
                                                  P->ctr + C_SLOW, XB.key, XB.rec, hist_b, shift,
                                                  npass);
    HLC_LAUNCH_CHECK();
  }
  HLC_CUDA(cudaEventRecord(eb[1], st));
  // 2. one sort of both arrays, after both preps
  HLC_CUDA(cudaStreamWaitEvent(st, ea[1], 0));
  ar.drop(slow_b);
  ar.drop(slow_a);
  uint32_t *tkb = nullptr, *tvb = nullptr, *tka = nullptr, *tva = nullptr;
  if (nb > 1) {
    HLC_ALLOC(ar, tkb, uint32_t, nb);
    HLC_ALLOC(ar, tvb, uint32_t, nb);
  }
  if (na > 1) {
    HLC_ALLOC(ar, tka, uint32_t, na);
    HLC_ALLOC(ar, tva, uint32_t, na);
  }
  {
    bool in_tmp = false;
    int np = 0;
    cudaEvent_t* pev = P->events ? P->ev + 7 : nullptr;
    HLC_TRY(radix_sort_pairs2<uint32_t>(XB.key, XB.idx, tkb, tvb, nb, scrb, XA.key, XA.idx, tka,
                                        tva, na, scra, bits, P->dev_err, st, shift, &in_tmp, pev,
                                        &np, both, both));
    P->sort_passes += np;
    const uint64_t ne = (nb > 1 && na > 1) ? nb + na : (nb > 1 ? nb : na);
    P->sort_entries += (uint64_t)np * ne;
    // (the one-sort form's first pass makes its values: 12 bytes, not 16)
    P->sort_bytes += (16ull * np - (both && np ? 4ull : 0ull)) * ne;
    if (pev && np) P->sort_timed[0] = true;
    if (in_tmp) {
      std::swap(XB.key, tkb);
      std::swap(XB.idx, tvb);
      std::swap(XA.key, tka);
      std::swap(XA.idx, tva);
    }
    for (void* q : {(void*)tkb, (void*)tvb, scrb, (void*)tka, (void*)tva, scra})
      if (q) ar.drop(q);
  }
  HLC_CUDA(cudaEventRecord(e_sorted, st));
  // 3. the payloads side by side (A's on ks), then B's offset table and dense cells
  HLC_CUDA(cudaStreamWaitEvent(ks, e_sorted, 0));
  if (na) {
    if (P->eq4)
      k_payload32<true><<<grid_for(na, kThreads), kThreads, 0, ks>>>(
          XA.rec, XA.idx, na, XA.v32, P->ctr + C_IDDIFF, 1.f, P->k9);
    else
      k_payload32<false><<<grid_for(na, kThreads), kThreads, 0, ks>>>(
          XA.rec, XA.idx, na, XA.v32, P->ctr + C_IDDIFF);
    HLC_LAUNCH_CHECK();
  }
  HLC_CUDA(cudaEventRecord(ea[2], ks));
  HLC_ALLOC(ar, XB.v32, float4, nb + 1);
  if (nb) {
    if (P->eq4)
      k_payload32<true><<<grid_for(nb, kThreads), kThreads, 0, st>>>(
          XB.rec, XB.idx, nb, XB.v32, nullptr, -1.f, P->k9);
    else
      k_payload32<false><<<grid_for(nb, kThreads), kThreads, 0, st>>>(
          XB.rec, XB.idx, nb, XB.v32, nullptr);
    HLC_LAUNCH_CHECK();
  }
  HLC_CUDA(cudaEventRecord(eb[2], st));
  HLC_ALLOC(ar, XB.table, uint32_t, tsize + 1);
  HLC_TRY(offset_table(P, XB.key, nb, shift, tsize, XB.table, P->ctr + C_HEADS_B, P->sparse_cell,
                       P->ctr + C_DENSE));
  if (nb > 1) {
    unsigned long long nd = 0;
    HLC_CUDA(cudaMemcpyAsync(&nd, P->ctr + C_DENSE, 8, cudaMemcpyDeviceToHost, st));
    HLC_CUDA(cudaStreamSynchronize(st));
    XB.ndense = nd;
    if (nd > 0) HLC_TRY(dense_fixup(P, XB, XB.table, shift, false));
  }
  HLC_CUDA(cudaEventRecord(eb[3], st));
  return HLC_OK;
}

// Copy one catalogue in, build its sorted entries, payload and (for B) the
// coarse offset table.  No host synchronisation in complete mode.
static int build_catalog(hlc_plan_t* P, const hlc_catalog* in, CatDev& X, bool is_b,
                         cudaEvent_t ev[4]) {
  Arena& ar = *P->arena;
  cudaStream_t st = plan_stream(P);
  // (A's id span for the output's bucketing, taken by its prep kernel)
  unsigned long long* iddiff = is_b ? nullptr : P->ctr + C_IDDIFF;
  const int L = P->p.fine_level;
  const bool quad = P->p.boundary != HLC_COMPLETE8;
  const bool fp32 = P->p.precision == HLC_FP32_GUARD;
  X.n = in->n;
  uint64_t n = X.n;
  // device inputs are read in place (only until this call returns); host
  // inputs are staged in temporary device buffers
  const double* ra = in->ra_deg;
  const double* dec = in->dec_deg;
  const uint64_t* id = in->id;
  const double* perr = P->eq4 ? in->err_arcsec : nullptr;
  double *tra = nullptr, *tdec = nullptr, *terr = nullptr;
  uint64_t* tid = nullptr;
  if (!in->on_device) {
    HLC_ALLOC(ar, tra, double, n + 1);
    HLC_ALLOC(ar, tdec, double, n + 1);
    HLC_ALLOC(ar, tid, uint64_t, n + 1);
    if (perr) HLC_ALLOC(ar, terr, double, n + 1);
    if (n) {
      HLC_CUDA(cudaMemcpyAsync(tra, in->ra_deg, n * 8, cudaMemcpyHostToDevice, st));
      HLC_CUDA(cudaMemcpyAsync(tdec, in->dec_deg, n * 8, cudaMemcpyHostToDevice, st));
      HLC_CUDA(cudaMemcpyAsync(tid, in->id, n * 8, cudaMemcpyHostToDevice, st));
      if (perr) HLC_CUDA(cudaMemcpyAsync(terr, perr, n * 8, cudaMemcpyHostToDevice, st));
    }
    ra = tra;
    dec = tdec;
    id = tid;
    if (perr) perr = terr;
  }
  cudaEventRecord(ev[0], st);
  HLC_ALLOC(ar, X.rec, SrcRec, n + 1);
  if (P->table_buckets) {
    HLC_TRY(bucket_catalog(P, X, is_b, ra, dec, id, perr, ev));
    if (tra) {
      ar.drop(tra);
      ar.drop(tdec);
      ar.drop(tid);
      if (terr) ar.drop(terr);
    }
    cudaEventRecord(ev[3], st);
    return HLC_OK;
  }
  // the sort's scratch, whose digit histograms the FP32 key writers count
  // (the guarded preps, the quad-entry emit) as they write the keys
  const int sort_bits = 2 * L + 4;
  const int sort_np = (sort_bits + 7) / 8;
  void* sscr = nullptr;
  if (!quad) {
    X.m = n;
    HLC_ALLOC(ar, X.key, uint32_t, n + 1);
    HLC_ALLOC(ar, X.idx, uint32_t, n + 1);
    if (n) {
      if (fp32) {
        uint32_t* slow = ar.get_n<uint32_t>(n + 1);
        if (!slow) return HLC_ENOMEM;
        if (n > 1) {
          sscr = ar.get(sort_scratch_bytes(n, sort_np));
          if (!sscr) return HLC_ENOMEM;
          HLC_CUDA(cudaMemsetAsync(sscr, 0, (size_t)sort_np * 256 * 4, st));
        }
        HLC_CUDA(cudaMemsetAsync(P->ctr + C_SLOW, 0, 8, st));
        k_prep_keys<true><<<grid_for(n, kThreads, prep_resident_blocks()), kThreads, 0, st>>>(
            ra, dec, id, n, L, pix_const(L), X.key, X.idx, X.rec, slow, P->ctr + C_SLOW,
            P->dev_err, nullptr, (uint32_t*)sscr, 0, sscr ? sort_np : 0, iddiff);
        HLC_LAUNCH_CHECK();
        k_prep_fallback<<<num_sms() * 4u, kThreads, 0, st>>>(ra, dec, L, slow, P->ctr + C_SLOW,
                                                              X.key, X.rec, (uint32_t*)sscr, 0,
                                                              sscr ? sort_np : 0);
        HLC_LAUNCH_CHECK();
        ar.drop(slow);
      } else {
        k_prep_keys<false><<<grid_for(n, kThreads), kThreads, 0, st>>>(
            ra, dec, id, n, L, pix_const(L), X.key, X.idx, X.rec, nullptr, nullptr, P->dev_err,
            perr, nullptr, 0, 0, iddiff);
        HLC_LAUNCH_CHECK();
      }
    }
  } else {
    HLC_ALLOC(ar, X.cells5, uint32_t, 5 * n + 5);
    uint32_t* cnt = ar.get_n<uint32_t>(n + 1);
    // entry offsets: 32-bit while the entries (at most 5 per source) fit
    const bool off32 = 5 * n < (1ull << 32);
    void* off = ar.get((n + 1) * (off32 ? 4 : 8));
    void* scr = ar.get(scan_scratch_bytes(n));
    if (!cnt || !off || !scr) return HLC_ENOMEM;
    if (n) {
      const double R = P->p.radius_arcsec / 3600.0;
      const bool cosdec = P->p.boundary == HLC_QUAD_COSDEC;
      if (fp32) {
        uint32_t* slow = ar.get_n<uint32_t>(n + 1);
        if (!slow) return HLC_ENOMEM;
        HLC_CUDA(cudaMemsetAsync(P->ctr + C_SLOW, 0, 8, st));
        k_quad_cells<true><<<grid_for(n, kThreads), kThreads, 0, st>>>(
            ra, dec, id, n, R, L, pix_const(L), X.cells5, cnt, X.rec, slow, P->ctr + C_SLOW,
            P->dev_err, cosdec, iddiff);
        HLC_LAUNCH_CHECK();
        k_quad_fallback<<<num_sms() * 4u, kThreads, 0, st>>>(ra, dec, R, L, slow, P->ctr + C_SLOW,
                                                      X.cells5, cnt, cosdec);
        HLC_LAUNCH_CHECK();
        ar.drop(slow);
      } else {
        k_quad_cells<false><<<grid_for(n, kThreads), kThreads, 0, st>>>(
            ra, dec, id, n, R, L, pix_const(L), X.cells5, cnt, X.rec, nullptr, nullptr,
            P->dev_err, cosdec, iddiff);
        HLC_LAUNCH_CHECK();
      }
    }
    if (off32)
      HLC_TRY(scan_exclusive<uint32_t>(cnt, (uint32_t*)off, n, P->ctr + C_TOTAL, scr, P->dev_err,
                                       st));
    else
      HLC_TRY(scan_exclusive<uint64_t>(cnt, (uint64_t*)off, n, P->ctr + C_TOTAL, scr,
                                       P->dev_err, st));
    unsigned long long m = 0;
    HLC_CUDA(cudaMemcpyAsync(&m, P->ctr + C_TOTAL, 8, cudaMemcpyDeviceToHost, st));
    HLC_CUDA(cudaStreamSynchronize(st));
    X.m = m;
    HLC_ALLOC(ar, X.key, uint32_t, X.m + 1);
    HLC_ALLOC(ar, X.idx, uint32_t, X.m + 1);
    if (m > 1) {
      sscr = ar.get(sort_scratch_bytes(m, sort_np));
      if (!sscr) return HLC_ENOMEM;
      HLC_CUDA(cudaMemsetAsync(sscr, 0, (size_t)sort_np * 256 * 4, st));
    }
    if (n) {
      const unsigned eg = grid_for(n, kThreads, sscr ? num_sms() * 8u : 0u);
      if (off32)
        k_quad_emit<uint32_t><<<eg, kThreads, 0, st>>>(X.cells5, cnt, (const uint32_t*)off, n,
                                                        X.key, X.idx, (uint32_t*)sscr,
                                                        sscr ? sort_np : 0);
      else
        k_quad_emit<uint64_t><<<eg, kThreads, 0, st>>>(X.cells5, cnt, (const uint64_t*)off, n,
                                                        X.key, X.idx, (uint32_t*)sscr,
                                                        sscr ? sort_np : 0);
      HLC_LAUNCH_CHECK();
    }
    ar.drop(cnt);
    ar.drop(off);
    ar.drop(scr);
  }
  cudaEventRecord(ev[1], st);
  uint64_t m = X.m;
  if (m > 1) {
    uint32_t* tk = ar.get_n<uint32_t>(m);
    uint32_t* tv = ar.get_n<uint32_t>(m);
    const bool counted = sscr != nullptr;
    void* scr = counted ? sscr : ar.get(sort_scratch_bytes(m, sort_np));
    if (!tk || !tv || !scr) return HLC_ENOMEM;
    HLC_TRY(radix_sort_pairs<uint32_t>(X.key, X.idx, tk, tv, m, sort_bits, scr, P->dev_err, st,
                                       0, nullptr, nullptr, nullptr, counted));
    ar.drop(tk);
    ar.drop(tv);
    ar.drop(scr);
  }
  cudaEventRecord(ev[2], st);
  if (!fp32) {
    HLC_ALLOC(ar, X.vx, double, m + 1);
    HLC_ALLOC(ar, X.vy, double, m + 1);
    HLC_ALLOC(ar, X.vz, double, m + 1);
    if (P->eq4) HLC_ALLOC(ar, X.ve, double, m + 1);
    if (m) {
      k_payload64<<<grid_for(m, kThreads), kThreads, 0, st>>>(X.rec, X.idx, m, X.vx, X.vy, X.vz,
                                                              X.ve);
      HLC_LAUNCH_CHECK();
    }
  } else {
    HLC_ALLOC(ar, X.v32, float4, m + 1);
    if (m) {
      k_payload32<false><<<grid_for(m, kThreads), kThreads, 0, st>>>(X.rec, X.idx, m, X.v32,
                                                                      nullptr);
      HLC_LAUNCH_CHECK();
    }
  }
  if (tra) {
    ar.drop(tra);
    ar.drop(tdec);
    ar.drop(tid);
    if (terr) ar.drop(terr);
  }
  unsigned long long* heads = P->ctr + (is_b ? C_HEADS_B : C_HEADS_A);
  if (is_b && P->p.index == HLC_INDEX_LEARNED) {
    // unique cells of B, then the per-partition models over them
    HLC_ALLOC(ar, X.uniq, uint32_t, m + 1);
    HLC_ALLOC(ar, X.start, uint32_t, m + 2);
    uint32_t* cell_of = ar.get_n<uint32_t>(m + 1);
    void* scr = ar.get(scan_scratch_bytes(m));
    if (!cell_of || !scr) return HLC_ENOMEM;
    HLC_TRY(cell_table(X.key, m, 0, cell_of, X.uniq, X.start, P->ctr + C_M, scr, P->dev_err, st));
    unsigned long long u = 0;
    HLC_CUDA(cudaMemcpyAsync(&u, P->ctr + C_M, 8, cudaMemcpyDeviceToHost, st));
    HLC_CUDA(cudaStreamSynchronize(st));
    X.u = u;
    ar.drop(cell_of);
    ar.drop(scr);
    const int Lc = P->p.coarse_level;
    X.parts = 12ull << (2 * Lc);
    HLC_TRY(build_learned(ar, X.uniq, X.u, 2 * (L - Lc), P->p.model, X.parts, P->ctr + C_TOTAL,
                          P->ctr + C_SCRATCH, P->dev_err, st, &X.learned));
    HLC_CUDA(cudaMemsetAsync(P->ctr + C_LMAXERR, 0, 8, st));
    k_max_u32<<<grid_for(X.parts, kThreads, 1024), kThreads, 0, st>>>(
        X.learned.err, X.parts, (uint32_t*)(P->ctr + C_LMAXERR));
    HLC_LAUNCH_CHECK();
  } else if (is_b) {
    X.table_order = coarse_table_order(m, L);
    X.table_shift = 2 * (L - X.table_order);
    uint64_t tsize = 12ull << (2 * X.table_order);
    HLC_ALLOC(ar, X.table, uint32_t, tsize + 1);
    HLC_TRY(offset_table(P, X.key, m, X.table_shift, tsize, X.table, heads, 0xFFFFFFFFu,
                         nullptr));
  }
  cudaEventRecord(ev[3], st);
  return HLC_OK;
}

// Eq. 4 pair radius on the host, in the same operation order as the device
// (c_pair_radius): a = e1 e1, b = e2 e2, t = a + b, r = 3 sqrt(t).
static double host_pair_radius(double e1, double e2) {
  volatile double a = e1 * e1;
  volatile double b = e2 * e2;
  volatile double t = a + b;
  return 3.0 * std::sqrt((double)t);
}

// Eq. 4 set-up of a plan: the largest error radius of each catalogue (device
// columns reduced on the device, host columns on the host; every value must
// be finite and >= 0), the largest pair radius, which complete mode needs
// within theta_L/8, and the FP32 band around s - (rho_a + rho_b).
static int eq4_setup(hlc_plan_t* P, const hlc_catalog* A, const hlc_catalog* B) {
  cudaStream_t st = plan_stream(P);
  const hlc_catalog* X[2] = {A, B};
  double emax[2] = {0.0, 0.0};
  bool dev_any = false;
  for (int i = 0; i < 2; ++i) {
    if (X[i]->n && !X[i]->err_arcsec) {
      set_error("HLC_RADIUS_EQ4: catalogue %s has no err_arcsec column", i ? "B" : "A");
      return HLC_EINVAL;
    }
    if (!X[i]->n) continue;
    if (X[i]->on_device) {
      dev_any = true;
      k_err_max<<<grid_for(X[i]->n, kThreads, num_sms() * 8u), kThreads, 0, st>>>(
          X[i]->err_arcsec, X[i]->n, P->ctr + (i ? C_EMAXB : C_EMAXA), P->dev_err);
      HLC_LAUNCH_CHECK();
    } else {
      for (uint64_t k = 0; k < X[i]->n; ++k) {
        const double v = X[i]->err_arcsec[k];
        if (!(v >= 0.0) || !std::isfinite(v)) {
          set_error("HLC_RADIUS_EQ4: catalogue %s error radius %llu is %g (must be finite "
                    "and >= 0)", i ? "B" : "A", (unsigned long long)k, v);
          return HLC_EINVAL;
        }
        emax[i] = std::max(emax[i], v);
      }
    }
  }
  if (dev_any) {
    unsigned long long hm[2] = {0, 0};
    HLC_CUDA(cudaMemcpyAsync(hm, P->ctr + C_EMAXA, 16, cudaMemcpyDeviceToHost, st));
    int rc = check_dev_err(P->dev_err, st, "hlc_plan");
    if (rc == HLC_EINVAL) {
      set_error("HLC_RADIUS_EQ4: an error radius is not finite or is negative");
      return rc;
    }
    HLC_TRY(rc);
    for (int i = 0; i < 2; ++i)
      if (X[i]->on_device) memcpy(&emax[i], &hm[i], 8);
  }
  const double pi = 3.14159265358979323846;
  P->eq4_rmax = host_pair_radius(emax[0], emax[1]);
  const int L = P->p.fine_level;
  if (P->eq4_rmax > complete_max_radius(L)) {
    set_error("HLC_RADIUS_EQ4: the largest pair radius 3 sqrt(%g^2 + %g^2) = %g arcsec exceeds "
              "theta_L/8 = %g arcsec at fine_level %d", emax[0], emax[1], P->eq4_rmax,
              complete_max_radius(L), L);
    return HLC_EINVAL;
  }
  P->k9 = 9.0 * (pi / 648000.0) * (pi / 648000.0);
  // bound on rho_a + rho_b as the FP32 payloads hold them (each rounded once)
  P->eq4_rho_max = 1.01 * P->k9 * (emax[0] * emax[0] + emax[1] * emax[1]);
  P->C = chord2_threshold(P->eq4_rmax);
  // the single-radius band at the largest threshold, plus the roundings of
  // rho_a, rho_b and their sum (3 half-ulps of C) and 4 sin^2(x/2) = x^2 -
  // x^4/12 + ... against x^2 = rho_a + rho_b
  const double u = 1.0 / 16777216.0;
  const double G = fp32_guard_band(P->C, kUnitVecErr) + 4.0 * u * P->C + 1.1 * P->C * P->C / 12.0;
  P->lo32 = (float)(-G);
  P->hi32 = (float)G;
  if ((double)P->lo32 > -G) P->lo32 = nextafterf(P->lo32, -1e30f);
  if ((double)P->hi32 < G) P->hi32 = nextafterf(P->hi32, 1e30f);
  return HLC_OK;
}

static int plan_single(const hlc_catalog* A, const hlc_catalog* B, const hlc_params* p,
                       hlc_plan_t** out) {
  HLC_TRY(validate_params(p));
  HLC_TRY(validate_catalog(A, "A"));
  HLC_TRY(validate_catalog(B, "B"));
  HLC_TRY(ensure_device_tables());
  hlc_plan_t* P = new hlc_plan_t();
  P->p = *p;
  P->al.alloc = p->alloc;
  P->al.dealloc = p->dealloc;
  P->al.ctx = p->alloc_ctx;
  P->al.stream = (cudaStream_t)p->stream;
  P->arena = new Arena(P->al);
  P->out = new Arena(P->al);
  P->join_level = p->fine_level;
  P->nslot = p->boundary != HLC_COMPLETE8 ? 1 : 9;
  P->table_buckets = p->boundary == HLC_COMPLETE8 && p->precision == HLC_FP32_GUARD &&
                     p->index != HLC_INDEX_LEARNED;
  if (p->tune) {
    for (int c = 0; c < 3; ++c) P->tile_ka[c] = p->tune->ka[c];
    P->tile_stage = p->tune->stage;
  }
  P->eq4 = p->radius_rule == HLC_RADIUS_EQ4;
  if (!P->eq4) {
    P->C = chord2_threshold(p->radius_arcsec);
    f2_sep_window(p->radius_arcsec, &P->r_lo, &P->r_hi);
    double G = fp32_guard_band(P->C, kUnitVecErr);
    P->lo32 = (float)(P->C - G);
    P->hi32 = (float)(P->C + G);
    // make the float thresholds conservative
    if ((double)P->lo32 > P->C - G) P->lo32 = nextafterf(P->lo32, 0.0f);
    if ((double)P->hi32 < P->C + G) P->hi32 = nextafterf(P->hi32, 1e30f);
    if (P->lo32 < 0) P->lo32 = -1.0f;
  }
  for (int i = 0; i < 12; ++i) pool_event(&P->ev[i], true);
  P->events = true;
  auto fail = [&](int rc) {
    hlc_free(P);
    return rc;
  };
  cudaStream_t st = plan_stream(P);
  P->dev_err = P->arena->get_n<int>(16);
  P->ctr = P->arena->get_n<unsigned long long>(C_N);
  if (!P->dev_err || !P->ctr) return fail(HLC_ENOMEM);
  if (cudaMemsetAsync(P->dev_err, 0, 64, st) != cudaSuccess ||
      cudaMemsetAsync(P->ctr, 0, C_N * 8, st) != cudaSuccess) {
    set_error("cudaMemsetAsync failed");
    return fail(HLC_ECUDA);
  }
  ev_record(P, 0);
  P->launches0 = g_launches.load();
  if (P->eq4) {
    const int rc = eq4_setup(P, A, B);
    if (rc != HLC_OK) return fail(rc);
  }
  cudaEvent_t ea[4], eb[4];
  for (int i = 0; i < 4; ++i) {
    pool_event(&ea[i], true);
    pool_event(&eb[i], true);
  }
  // (the FP32 complete form orders A by B's table cells: B first)
  const hlc_catalog* first = P->table_buckets ? B : A;
  const hlc_catalog* second = P->table_buckets ? A : B;
  // host inputs: both catalogues are copied in on a side stream in build
  // order, so that building the first overlaps the copy of the second
  hlc_catalog dv[2] = {*first, *second};
  void* stage[2][4] = {{nullptr, nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr, nullptr}};
  const int ncol = P->eq4 ? 4 : 3;  // ra, dec, id (+ Eq. 4 error radius)
  cudaStream_t cs = nullptr;
  cudaEvent_t cev[3] = {nullptr, nullptr, nullptr};
  int rc = HLC_OK;
  if (!first->on_device || !second->on_device) {
    if (pool_stream(&cs) != cudaSuccess) rc = HLC_ECUDA;
    for (int i = 0; i < 3 && rc == HLC_OK; ++i)
      if (pool_event(&cev[i], false) != cudaSuccess) rc = HLC_ECUDA;
    for (int i = 0; i < 2 && rc == HLC_OK; ++i) {
      if (dv[i].on_device) continue;
      const uint64_t n = dv[i].n;
      for (int k = 0; k < ncol; ++k) {
        stage[i][k] = P->arena->get((n + 1) * 8);
        if (!stage[i][k]) rc = HLC_ENOMEM;
      }
    }
    if (rc == HLC_OK && (cudaEventRecord(cev[2], st) != cudaSuccess ||  // allocations done
                         cudaStreamWaitEvent(cs, cev[2], 0) != cudaSuccess))
      rc = HLC_ECUDA;
    for (int i = 0; i < 2 && rc == HLC_OK; ++i) {
      if (!dv[i].on_device && dv[i].n) {
        const uint64_t n = dv[i].n;
        if (cudaMemcpyAsync(stage[i][0], dv[i].ra_deg, n * 8, cudaMemcpyHostToDevice, cs) !=
                cudaSuccess ||
            cudaMemcpyAsync(stage[i][1], dv[i].dec_deg, n * 8, cudaMemcpyHostToDevice, cs) !=
                cudaSuccess ||
            cudaMemcpyAsync(stage[i][2], dv[i].id, n * 8, cudaMemcpyHostToDevice, cs) !=
                cudaSuccess ||
            (ncol == 4 && cudaMemcpyAsync(stage[i][3], dv[i].err_arcsec, n * 8,
                                          cudaMemcpyHostToDevice, cs) != cudaSuccess))
          rc = HLC_ECUDA;
      }
      if (rc == HLC_OK && cudaEventRecord(cev[i], cs) != cudaSuccess) rc = HLC_ECUDA;
      if (!dv[i].on_device) {
        dv[i].ra_deg = (const double*)stage[i][0];
        dv[i].dec_deg = (const double*)stage[i][1];
        dv[i].id = (const uint64_t*)stage[i][2];
        if (ncol == 4) dv[i].err_arcsec = (const double*)stage[i][3];
        dv[i].on_device = 1;
      }
    }
  }
  // FP32 complete form: both catalogues built at once, A's kernels on a side
  // stream (bucket_pair), joined before A's dense cells are ordered.
  // (With host inputs A's build waits for its copy, which ends after B's
  // build anyway, so it stays on the plan stream.)
  const bool side = P->table_buckets && !cs;
  cudaStream_t ks = nullptr;
  cudaEvent_t esorted = nullptr;  // both sorts done
  if (side && rc == HLC_OK) {
    if (pool_stream(&ks) != cudaSuccess) {
      ks = nullptr;
      rc = HLC_ECUDA;
    } else if (pool_event(&esorted, false) != cudaSuccess) {
      rc = HLC_ECUDA;
    } else {
      rc = bucket_pair(P, &dv[0], &dv[1], ks, eb, ea, esorted);
    }
  }
  for (int i = 0; i < (side ? 0 : 2) && rc == HLC_OK; ++i) {
    if (cs && cudaStreamWaitEvent(st, cev[i], 0) != cudaSuccess) rc = HLC_ECUDA;
    const bool is_b = (i == 0) == P->table_buckets;
    if (rc == HLC_OK)
      rc = build_catalog(P, &dv[i], is_b ? P->B : P->A, is_b, is_b ? eb : ea);
  }
  cudaEvent_t ej = nullptr;  // (side form) the join: A's index stage starts here
  if (side) {
    if (rc == HLC_OK && (cudaStreamWaitEvent(st, ea[2], 0) != cudaSuccess ||
                         pool_event(&ej, true) != cudaSuccess || cudaEventRecord(ej, st) != cudaSuccess))
      rc = HLC_ECUDA;
    if (rc == HLC_OK) {
      if (P->A.n > 1 && P->B.ndense > 0)
        rc = dense_fixup(P, P->A, P->B.table, P->A.table_shift, true);
      if (rc == HLC_OK && cudaEventRecord(ea[3], st) != cudaSuccess) rc = HLC_ECUDA;
    }
    if (ks) {
      if (rc != HLC_OK) cudaStreamSynchronize(ks);  // nothing of A's still runs when freed
      pool_stream_back(ks);
    }
    pool_event_back(esorted, false);
  }
  if (cs) {
    cudaStreamSynchronize(cs);
    pool_stream_back(cs);
    for (int i = 0; i < 3; ++i) pool_event_back(cev[i], false);
    for (int i = 0; i < 2; ++i)
      for (int k = 0; k < 4; ++k)
        if (stage[i][k]) P->arena->drop(stage[i][k]);
  }
  unsigned long long hc[C_N] = {0};
  if (rc == HLC_OK && cudaMemcpyAsync(hc, P->ctr, sizeof(hc), cudaMemcpyDeviceToHost, st) !=
                          cudaSuccess)
    rc = HLC_ECUDA;
  if (rc == HLC_OK) rc = check_dev_err(P->dev_err, st, "hlc_plan");
  float t[6] = {0};
  if (rc == HLC_OK) {
    cudaEventElapsedTime(&t[0], ea[0], ea[1]);
    cudaEventElapsedTime(&t[1], eb[0], eb[1]);
    cudaEventElapsedTime(&t[2], ea[1], ea[2]);
    cudaEventElapsedTime(&t[3], eb[1], eb[2]);
    cudaEventElapsedTime(&t[4], ej ? ej : ea[2], ea[3]);
    cudaEventElapsedTime(&t[5], eb[2], eb[3]);
  }
  for (int i = 0; i < 4; ++i) {
    pool_event_back(ea[i], true);
    pool_event_back(eb[i], true);
  }
  pool_event_back(ej, true);
  if (rc != HLC_OK) return fail(rc);
  ev_record(P, 1);
  unsigned long long diff = hc[C_IDDIFF];
  P->id_high_bit = diff ? 63 - __builtin_clzll(diff) : -1;
  memset(&P->stats, 0, sizeof(P->stats));
  P->stats.n_a = P->A.n;
  P->stats.n_b = P->B.n;
  P->stats.entries_a = P->A.m;
  P->stats.entries_b = P->B.m;
  P->stats.cells_b = P->p.index == HLC_INDEX_LEARNED ? P->B.u : hc[C_HEADS_B];
  P->stats.learned_models = P->p.index == HLC_INDEX_LEARNED ? P->B.parts : 0;
  P->stats.dense_entries_b = P->B.ndense;
  if (P->A.tile_n) {
    unsigned long long tn[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(tn, P->A.tile_n, 32, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail(HLC_ECUDA);
    P->stats.tile_items = tn[1];
    P->stats.tile_entries_a = tn[2];
  }
  P->stats.learned_max_err = (uint32_t)hc[C_LMAXERR];
  P->stats.join_level = P->join_level;
  P->stats.ms_prep = t[0] + t[1];
  P->stats.ms_sort = t[2] + t[3];
  P->stats.ms_index = t[4] + t[5];
  P->stats.sort_passes = P->sort_passes;
  P->stats.sort_entries = P->sort_entries;
  P->stats.sort_bytes = P->sort_bytes;
  for (int i = 0; i < 2; ++i)
    if (P->sort_timed[i]) P->stats.ms_sort_passes += ev_ms(P, 7 + 2 * i, 8 + 2 * i);
  if (side && P->sort_timed[0]) P->stats.ms_plan_presort = ev_ms(P, 0, 7);
  P->plan_launches = g_launches.load() - P->launches0;
  *out = P;
  return HLC_OK;
}

// Orders M packed rows by (job, id_a, id_b, sep) into result columns: the
// bucket scatter + per-bucket sorts, or two or three stable radix sorts when
// a bucket would not fit in shared memory.  jbk null: single job; else the
// batched plan's per-job bucket table (row_bucket).
// Mdev (bucketed form only): the rows are counted on the device, M being the
// bound the buffers are sized by.
static int order_rows(hlc_plan_t* P, OutRow* rows32, uint64_t M, uint32_t* bhist,
                      uint32_t* boff, uint64_t nbk, const uint4* jbk, int bshift, uint32_t bmask,
                      bool bucketed, bool want_sep, uint64_t** oa, uint64_t** ob, double** os,
                      uint32_t** oj, const unsigned long long* Mdev = nullptr) {
  Arena& ar = *P->out;
  cudaStream_t st = plan_stream(P);
  const bool batched = jbk != nullptr;
  uint64_t* a = ar.get_n<uint64_t>(M + 1);
  uint64_t* b = ar.get_n<uint64_t>(M + 1);
  double* sp = want_sep ? ar.get_n<double>(M + 1) : nullptr;
  uint32_t* jb = batched ? ar.get_n<uint32_t>(M + 1) : nullptr;
  if (!a || !b || (want_sep && !sp) || (batched && !jb)) return HLC_ENOMEM;
  *oa = a;
  *ob = b;
  *os = sp;
  *oj = jb;
  if (M == 0) return HLC_OK;
  unsigned g = grid_for(M, kThreads);
  if (Mdev && !(bucketed && nbk < (1ull << 31))) {
    set_error("row ordering: a device row count needs the bucketed form");
    return HLC_EINVAL;
  }
  if (M == 1 && !Mdev) {
    k_rows_split<<<1, 32, 0, st>>>(rows32, M, a, b, sp, jb);
    HLC_LAUNCH_CHECK();
    return HLC_OK;
  }
  if (bucketed && nbk < (1ull << 31)) {
    // no host round trip: buckets above kSmallBucket rows are listed by
    // k_bucket_small for k_bucket_sort; one above kBucketCap raises
    // DERR_BUCKET and order_rows_checked re-orders with the radix sorts
    void* scr = ar.get(scan_scratch_bytes(nbk + 1));
    OutRow* t = ar.get_n<OutRow>(M + 1);
    uint32_t* big = ar.get_n<uint32_t>(nbk + 1);
    uint32_t* mid = ar.get_n<uint32_t>(nbk + 1);
    if (!scr || !t || !big || !mid) return HLC_ENOMEM;
    HLC_TRY(scan_exclusive<uint32_t>(bhist, boff, nbk + 1, P->ctr + C_TOTAL, scr, P->dev_err, st));
    uint32_t* nlist = (uint32_t*)(P->ctr + C_MAXB);  // [0] big buckets, [1] mid ones
    HLC_CUDA(cudaMemsetAsync(nlist, 0, 8, st));
    k_bucket_scatter<<<g, kThreads, 0, st>>>(rows32, M, bshift, bmask, jbk, boff, t, Mdev);
    HLC_LAUNCH_CHECK();
    k_bucket_small<<<g, kThreads, 0, st>>>(t, M, bshift, bmask, jbk, boff, a, b, sp, jb, big,
                                           nlist, mid, P->dev_err, Mdev);
    HLC_LAUNCH_CHECK();
    k_bucket_sort<kBucketMid><<<num_sms() * 12u, kBucketThreads, 0, st>>>(
        t, boff, mid, nlist + 1, want_sep ? 1 : 0, a, b, sp, jb);
    HLC_LAUNCH_CHECK();
    k_bucket_sort<kBucketCap><<<num_sms() * 4u, kBucketThreads, 0, st>>>(
        t, boff, big, nlist, want_sep ? 1 : 0, a, b, sp, jb);
    HLC_LAUNCH_CHECK();
    ar.drop(scr);
    ar.drop(t);
    ar.drop(big);
    ar.drop(mid);
    return HLC_OK;
  }
  // fallback: stable LSD radix sorts by id_b, id_a (and job)
  uint64_t* ua = ar.get_n<uint64_t>(M + 1);
  uint64_t* ub = ar.get_n<uint64_t>(M + 1);
  double* us = want_sep ? ar.get_n<double>(M + 1) : nullptr;
  uint32_t* uj = batched ? ar.get_n<uint32_t>(M + 1) : nullptr;
  uint32_t* perm = ar.get_n<uint32_t>(M + 1);
  uint64_t* tk = ar.get_n<uint64_t>(M + 1);
  uint32_t* tv = ar.get_n<uint32_t>(M + 1);
  void* scr = ar.get(sort_scratch_bytes(M + 1, 8));
  if (!ua || !ub || (want_sep && !us) || (batched && !uj) || !perm || !tk || !tv || !scr)
    return HLC_ENOMEM;
  k_rows_split<<<g, kThreads, 0, st>>>(rows32, M, ua, ub, us, uj);
  k_iota<<<g, kThreads, 0, st>>>(perm, M);
  HLC_LAUNCH_CHECK();
  HLC_CUDA(cudaMemcpyAsync(a, ub, M * 8, cudaMemcpyDeviceToDevice, st));
  HLC_TRY(radix_sort_pairs<uint64_t>(a, perm, tk, tv, M, 64, scr, P->dev_err, st));
  k_gather<uint64_t><<<g, kThreads, 0, st>>>(ua, perm, M, a);
  HLC_LAUNCH_CHECK();
  HLC_TRY(radix_sort_pairs<uint64_t>(a, perm, tk, tv, M, 64, scr, P->dev_err, st));
  if (batched) {
    k_gather<uint32_t><<<g, kThreads, 0, st>>>(uj, perm, M, jb);
    HLC_LAUNCH_CHECK();
    HLC_TRY(radix_sort_pairs<uint32_t>(jb, perm, (uint32_t*)tk, (uint32_t*)tk + M + 1, M, 16, scr,
                                       P->dev_err, st));
    k_gather<uint32_t><<<g, kThreads, 0, st>>>(uj, perm, M, jb);
  }
  k_gather<uint64_t><<<g, kThreads, 0, st>>>(ua, perm, M, a);
  k_gather<uint64_t><<<g, kThreads, 0, st>>>(ub, perm, M, b);
  if (want_sep) k_gather<double><<<g, kThreads, 0, st>>>(us, perm, M, sp);
  HLC_LAUNCH_CHECK();
  return HLC_OK;
}

// order_rows, then (after the stream has drained) a repeat with the radix
// sorts when a bucket was too large for the in-block sort.  With Mdev the
// stream is not drained here: the caller checks DERR_BUCKET at its own final
// synchronisation (see redo_order_rows).
static int order_rows_checked(hlc_plan_t* P, OutRow* rows32, uint64_t M, uint32_t* bhist,
                              uint32_t* boff, uint64_t nbk, const uint4* jbk, int bshift,
                              uint32_t bmask, bool bucketed, bool want_sep, uint64_t** oa,
                              uint64_t** ob, double** os, uint32_t** oj,
                              const unsigned long long* Mdev = nullptr) {
  cudaStream_t st = plan_stream(P);
  HLC_TRY(order_rows(P, rows32, M, bhist, boff, nbk, jbk, bshift, bmask, bucketed, want_sep,
                     oa, ob, os, oj, Mdev));
  if (Mdev) return HLC_OK;
  int h = 0;
  HLC_CUDA(cudaMemcpyAsync(&h, P->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  HLC_CUDA(cudaStreamSynchronize(st));
  if (!(h & DERR_BUCKET)) return HLC_OK;
  Arena& ar = *P->out;
  for (void* q : {(void*)*oa, (void*)*ob, (void*)*os, (void*)*oj})
    if (q) ar.drop(q);
  h &= ~DERR_BUCKET;
  HLC_CUDA(cudaMemcpyAsync(P->dev_err, &h, sizeof(int), cudaMemcpyHostToDevice, st));
  HLC_TRY(order_rows(P, rows32, M, bhist, boff, nbk, jbk, bshift, bmask, false, want_sep, oa,
                     ob, os, oj));
  HLC_CUDA(cudaStreamSynchronize(st));
  return HLC_OK;
}

static int match_single(hlc_plan_t* P, hlc_result* res, hlc_stats* stats) {
  cudaStream_t st = plan_stream(P);
  Arena& ar = *P->out;
  ar.release();
  CatDev& A = P->A;
  CatDev& B = P->B;
  const bool fp32 = P->p.precision == HLC_FP32_GUARD;
  const bool quad = P->p.boundary != HLC_COMPLETE8;
  const unsigned long long launches_match0 = g_launches.load();
  HLC_CUDA(cudaMemsetAsync(P->dev_err, 0, 64, st));
  ev_record(P, 2);
  ev_record(P, 3);
  bool tile_timed = false;  // (ev 11 .. ev 4: the tile kernel, the last pair launch)
  CellIndex bix;
  bix.keys = B.key;
  bix.table = B.table;
  bix.shift = B.table_shift;
  uint64_t cap = P->row_cap ? P->row_cap : std::max<uint64_t>(1u << 20, A.n + B.n);
  uint64_t bcap = fp32 ? std::max<uint64_t>(1u << 16, cap / 4) : 1;
  uint2* rows = nullptr;
  uint2* band = nullptr;
  unsigned long long h[C_N];
  for (int attempt = 0; attempt < 3; ++attempt) {
    rows = ar.get_n<uint2>(cap);
    band = ar.get_n<uint2>(bcap);
    if (!rows || !band) return HLC_ENOMEM;
    HLC_CUDA(cudaMemsetAsync(P->ctr, 0, C_N * 8, st));
    PairSink sink{rows, P->ctr + C_ROWS, cap, band, P->ctr + C_BAND, bcap,
                  P->ctr + C_TESTS, P->ctr + C_DUPS,
                  P->table_buckets ? nullptr : P->ctr + C_HEADS_A, P->dev_err};
    if (A.m && B.m) {
      unsigned grid = grid_for(A.m, kThreads, num_sms() * 16u);
      PairArgs pa;
      pa.mA = A.m;
      pa.keyA = A.key;
      pa.bix = bix;
      pa.lix = B.learned;
      pa.uniqB = B.uniq;
      pa.startB = B.start;
      pa.uB = B.u;
      pa.order = P->join_level;
      pa.axv = A.vx; pa.ayv = A.vy; pa.azv = A.vz;
      pa.bxv = B.vx; pa.byv = B.vy; pa.bzv = B.vz;
      pa.a32 = A.v32;
      pa.b32 = B.v32;
      pa.C = P->C;
      pa.lo32 = P->lo32;
      pa.hi32 = P->hi32;
      pa.idxA = A.idx;
      pa.idxB = B.idx;
      pa.cellsA = A.cells5;
      pa.cellsB = B.cells5;
      pa.sparse_cell = P->sparse_cell;
      pa.lhits = P->ctr + C_LHITS;
      pa.llook = P->ctr + C_LLOOK;
      pa.tiled = A.tiled;
      pa.aev = A.ve;
      pa.bev = B.ve;
      pa.k9 = P->k9;
      const bool learned = P->p.index == HLC_INDEX_LEARNED;
#define HLC_PAIR(F, Q, LR) k_pair<F, Q, LR, false><<<grid, kThreads, 0, st>>>(pa, sink)
      if (P->table_buckets && P->eq4) {
        k_pair<true, false, false, true, true><<<grid, kThreads, 0, st>>>(pa, sink);
      } else if (P->table_buckets) {
        k_pair<true, false, false, true><<<grid, kThreads, 0, st>>>(pa, sink);
      } else if (P->eq4) {  // (binary64, complete mode, binary-searched index)
        k_pair<false, false, false, false, true><<<grid, kThreads, 0, st>>>(pa, sink);
      } else if (fp32 && quad) {
        if (learned) HLC_PAIR(true, true, true); else HLC_PAIR(true, true, false);
      } else if (fp32) {
        if (learned) HLC_PAIR(true, false, true); else HLC_PAIR(true, false, false);
      } else if (quad) {
        if (learned) HLC_PAIR(false, true, true); else HLC_PAIR(false, true, false);
      } else {
        if (learned) HLC_PAIR(false, false, true); else HLC_PAIR(false, false, false);
      }
#undef HLC_PAIR
      HLC_LAUNCH_CHECK();
      if (P->table_buckets && A.tiled) {
        TileArgs ta{};
        ta.items = A.tile_items;
        ta.nitems = A.tile_nprep;
        ta.icap = A.tile_icap;
        ta.idxA = A.idx;
        ta.idxB = B.idx;
        ta.work = (unsigned*)(P->ctr + C_WORK);
        ta.a32 = A.v32;
        ta.b32 = B.v32;
        ta.bix = bix;
        ta.order = P->join_level;
        ta.lo32 = P->lo32;
        ta.hi32 = P->hi32;
        ta.sparse_cell = P->sparse_cell;
        for (int c = 0; c < 3; ++c) ta.ka[c] = P->tile_ka[c];
        ta.stage = P->tile_stage;
        ta.rho_max = P->eq4 ? (float)P->eq4_rho_max : 0.f;
        const int smem = kTileSmemDyn;
        PairSink tsink = sink;  // (its own test counter)
        tsink.tests = P->ctr + C_TILE_TESTS;
        ev_record(P, 11);
        if (P->eq4) {
          HLC_CUDA(cudaFuncSetAttribute(k_pair_tile<true>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
          k_pair_tile<true><<<num_sms() * 3u, kTileThreads + 32, smem, st>>>(ta, tsink);
        } else {
          HLC_CUDA(cudaFuncSetAttribute(k_pair_tile<false>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
          k_pair_tile<false><<<num_sms() * 3u, kTileThreads + 32, smem, st>>>(ta, tsink);
        }
        tile_timed = true;
        HLC_LAUNCH_CHECK();
      }
    }
    HLC_CUDA(cudaMemcpyAsync(h, P->ctr, sizeof(h), cudaMemcpyDeviceToHost, st));
    HLC_CUDA(cudaStreamSynchronize(st));
    uint64_t need = h[C_ROWS] + (fp32 ? h[C_BAND] : 0);
    if (need <= cap && h[C_BAND] <= bcap) break;
    ar.drop(rows);
    ar.drop(band);
    cap = need + need / 8 + 1024;
    bcap = std::max<uint64_t>(bcap, h[C_BAND] + 1024);
    HLC_CUDA(cudaMemsetAsync(P->dev_err, 0, 64, st));
    if (attempt == 2) {
      set_error("match rows did not fit after resizing");
      return HLC_ECUDA;
    }
  }
  P->row_cap = std::max<uint64_t>(P->row_cap, cap);
  ev_record(P, 4);
  if (fp32 && h[C_BAND]) {
    // (the table-cell form's rows already hold source indices)
    const unsigned rg = grid_for(h[C_BAND], kThreads, num_sms() * 16u);
    const uint32_t* ia = P->table_buckets ? nullptr : A.idx;
    const uint32_t* ib = P->table_buckets ? nullptr : B.idx;
    if (P->eq4)
      k_recheck<true><<<rg, kThreads, 0, st>>>(band, P->ctr + C_BAND, bcap, ia, ib, A.rec, B.rec,
                                               P->C, P->r_lo, P->r_hi, rows, P->ctr + C_ROWS,
                                               cap, P->ctr + C_BAND64, P->dev_err);
    else
      k_recheck<false><<<rg, kThreads, 0, st>>>(band, P->ctr + C_BAND, bcap, ia, ib, A.rec,
                                                B.rec, P->C, P->r_lo, P->r_hi, rows,
                                                P->ctr + C_ROWS, cap, P->ctr + C_BAND64,
                                                P->dev_err);
    HLC_LAUNCH_CHECK();
  }
  ev_record(P, 5);
  // The recheck may still add rows when the output stage is issued: with
  // bucketed output the kernels take the device's count, their buffers sized
  // by the bound M (rows before the recheck plus every band candidate), and
  // the count comes back with the final synchronisation.
  unsigned long long M = h[C_ROWS];
  int hb = P->id_high_bit;
  const unsigned long long* Mdev = nullptr;
  if (fp32 && h[C_BAND]) {
    if (M + h[C_BAND] > 1 && hb >= 0) {
      M += h[C_BAND];
      Mdev = P->ctr + C_ROWS;
    } else {
      HLC_CUDA(cudaMemcpyAsync(&M, P->ctr + C_ROWS, 8, cudaMemcpyDeviceToHost, st));
      HLC_CUDA(cudaStreamSynchronize(st));
    }
  }
  ar.drop(band);
  // rows: ids, separations, bucket histogram of id_a (about four rows per bucket)
  const bool want_sep = P->p.want_sep != 0;
  OutRow* rows32 = ar.get_n<OutRow>(M + 1);
  if (!rows32) return HLC_ENOMEM;
  int nbits = 1;
  while (nbits < 24 && (M >> (nbits + 2)) > 0) ++nbits;
  if (hb >= 0 && nbits > hb + 1) nbits = hb + 1;
  const bool bucketed = M > 1 && hb >= 0;
  const int bshift = bucketed ? hb + 1 - nbits : 0;
  const uint64_t nbk = 1ull << nbits;
  const uint32_t bmask = (uint32_t)(nbk - 1);
  uint32_t* bhist = nullptr;
  uint32_t* boff = nullptr;
  if (bucketed) {
    bhist = ar.get_n<uint32_t>(nbk + 1);
    boff = ar.get_n<uint32_t>(nbk + 1);
    if (!bhist || !boff) return HLC_ENOMEM;
    HLC_CUDA(cudaMemsetAsync(bhist, 0, (nbk + 1) * 4, st));
  }
  if (M) {
    unsigned g = grid_for(M, kThreads);
    if (fp32)
      k_rows<true><<<g, kThreads, 0, st>>>(rows, M, P->table_buckets ? nullptr : A.idx,
                                            P->table_buckets ? nullptr : B.idx, A.rec, B.rec,
                                            nullptr, nullptr,
                                            nullptr, nullptr, nullptr, nullptr, want_sep, rows32,
                                            bshift, bmask, bhist, Mdev);
    else
      k_rows<false><<<g, kThreads, 0, st>>>(rows, M, A.idx, B.idx, A.rec, B.rec, A.vx, A.vy,
                                             A.vz, B.vx, B.vy, B.vz, want_sep, rows32, bshift,
                                             bmask, bhist);
    HLC_LAUNCH_CHECK();
  }
  ar.drop(rows);
  uint64_t *oa = nullptr, *ob = nullptr;
  double* os = nullptr;
  uint32_t* oj = nullptr;
  HLC_TRY(order_rows_checked(P, rows32, M, bhist, boff, nbk, nullptr, bshift, bmask, bucketed,
                             want_sep, &oa, &ob, &os, &oj, Mdev));
  if (!Mdev) ar.drop(rows32);
  if (bhist) {
    ar.drop(bhist);
    ar.drop(boff);
  }
  ev_record(P, 6);
  // one synchronisation: binary64 band decisions, the final row count, errors
  unsigned long long fin[2] = {0, 0};
  int e = 0;
  HLC_CUDA(cudaMemcpyAsync(&fin[0], P->ctr + C_BAND64, 8, cudaMemcpyDeviceToHost, st));
  if (Mdev) HLC_CUDA(cudaMemcpyAsync(&fin[1], Mdev, 8, cudaMemcpyDeviceToHost, st));
  HLC_CUDA(cudaMemcpyAsync(&e, P->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  HLC_CUDA(cudaStreamSynchronize(st));
  HLC_TRY(dev_err_status(e, "hlc_match"));
  const unsigned long long band64 = fin[0];
  if (Mdev) {
    M = fin[1];
    if (e & DERR_BUCKET) {  // a bucket too large for the in-block sort: the radix sorts
      for (void* q : {(void*)oa, (void*)ob, (void*)os, (void*)oj})
        if (q) ar.drop(q);
      e &= ~DERR_BUCKET;
      HLC_CUDA(cudaMemcpyAsync(P->dev_err, &e, sizeof(int), cudaMemcpyHostToDevice, st));
      HLC_TRY(order_rows(P, rows32, M, nullptr, nullptr, 0, nullptr, 0, 0u, false, want_sep, &oa,
                         &ob, &os, &oj));
      HLC_CUDA(cudaStreamSynchronize(st));
    }
    ar.drop(rows32);
  }
  res->n = M;
  res->id_a = oa;
  res->id_b = ob;
  res->sep_arcsec = want_sep ? os : nullptr;
  res->job = nullptr;
  res->on_device = 1;
  P->stats.pair_tests = h[C_TESTS] + h[C_TILE_TESTS];
  P->stats.tile_tests = h[C_TILE_TESTS];
  P->stats.ms_tile = tile_timed ? ev_ms(P, 11, 4) : 0.f;
  if (!P->table_buckets) P->stats.cells_a = h[C_HEADS_A];  // counted by the pair test
  P->stats.band_candidates = fp32 ? h[C_BAND] : 0;
  P->stats.band_fp64 = fp32 ? band64 : 0;
  P->stats.matches = M;
  P->stats.quad_duplicates = h[C_DUPS];
  P->stats.learned_hit_rate = h[C_LLOOK] ? (double)h[C_LHITS] / (double)h[C_LLOOK] : 0.0;
  P->stats.ms_candidates = ev_ms(P, 2, 3);
  P->stats.ms_pair = ev_ms(P, 3, 4);
  P->stats.ms_recheck = ev_ms(P, 4, 5);
  P->stats.ms_output = ev_ms(P, 5, 6);
  P->stats.ms_plan_span = ev_ms(P, 0, 1);
  P->stats.ms_total = ev_ms(P, 0, 1) + ev_ms(P, 2, 6);
  P->stats.kernel_launches = (g_launches.load() - launches_match0) + P->plan_launches;
  if (stats) *stats = P->stats;
  return HLC_OK;
}

// ---------------------------------------------------------------------------
// Batched plans (n_jobs > 1).
// ---------------------------------------------------------------------------

// Autotuned order of a job: the finest order at which the job's B density
// (sources over the spherical cap they occupy) leaves about kTargetPerCell
// sources per cell, no finer than the completeness limit r <= theta_L / 8.
constexpr double kTargetPerCell = 2.0;

static int auto_order(double nb, double cap_one_minus_cos, double r_arcsec, double target) {
  const double pi = 3.14159265358979323846;
  double area = 2.0 * pi * std::max(cap_one_minus_cos, 1e-12);  // sr
  double density = std::max(nb, 1.0) / area;
  double cells = 4.0 * pi * density / (12.0 * target);  // 4^L
  int L = cells > 1.0 ? (int)std::floor(std::log(cells) / std::log(4.0) + 0.5) : 0;
  int Lmax = 0;
  while (Lmax < 14 && r_arcsec <= complete_max_radius(Lmax + 1)) ++Lmax;
  return std::max(0, std::min(L, Lmax));
}

static int plan_batched(const hlc_catalog* A, const hlc_catalog* B, const hlc_params* p,
                        uint32_t njobs, hlc_plan_t** out) {
  for (uint32_t j = 0; j < njobs; ++j) {
    hlc_params q = p[j];
    if (q.fine_level < 0) q.fine_level = 0;  // checked again once the order is chosen
    if (q.coarse_level > q.fine_level) q.coarse_level = q.fine_level;
    HLC_TRY(validate_params(&q));
    HLC_TRY(validate_catalog(A + j, "A"));
    HLC_TRY(validate_catalog(B + j, "B"));
    if (p[j].boundary != HLC_COMPLETE8 || p[j].index != HLC_INDEX_BSEARCH) {
      set_error("batched plans support the complete boundary with the table index");
      return HLC_EUNSUPPORTED;
    }
    if (p[j].precision != p[0].precision || p[j].stream != p[0].stream ||
        p[j].want_sep != p[0].want_sep || p[j].alloc != p[0].alloc ||
        p[j].tune != p[0].tune) {
      set_error("all jobs of a batched plan must share precision, stream, want_sep, "
                "allocator and tune");
      return HLC_EINVAL;
    }
    if (A[j].on_device != A[0].on_device || B[j].on_device != A[0].on_device) {
      set_error("all catalogues of a batched plan must be on the device or all on the host");
      return HLC_EINVAL;
    }
  }
  if (njobs > (1u << 16)) {
    set_error("at most 65536 jobs per batched plan");
    return HLC_EINVAL;
  }
  HLC_TRY(ensure_device_tables());
  hlc_plan_t* P = new hlc_plan_t();
  P->p = p[0];
  P->njobs = njobs;
  P->al.alloc = p[0].alloc;
  P->al.dealloc = p[0].dealloc;
  P->al.ctx = p[0].alloc_ctx;
  P->al.stream = (cudaStream_t)p[0].stream;
  P->arena = new Arena(P->al);
  P->out = new Arena(P->al);
  if (p[0].tune) {
    for (int c = 0; c < 3; ++c) P->tile_ka[c] = p[0].tune->ka[c];
    P->tile_stage = p[0].tune->stage;
    P->target_per_cell = p[0].tune->target_per_cell;
  }
  for (int i = 0; i < 12; ++i) pool_event(&P->ev[i], true);
  P->events = true;
  auto fail = [&](int rc) {
    hlc_free(P);
    return rc;
  };
  cudaStream_t st = plan_stream(P);
  Arena& ar = *P->arena;
  const bool fp32 = p[0].precision == HLC_FP32_GUARD;
  P->dev_err = ar.get_n<int>(16);
  P->ctr = ar.get_n<unsigned long long>(C_N);
  if (!P->dev_err || !P->ctr) return fail(HLC_ENOMEM);
  cudaMemsetAsync(P->dev_err, 0, 64, st);
  cudaMemsetAsync(P->ctr, 0, C_N * 8, st);
  ev_record(P, 0);
  P->launches0 = g_launches.load();
  // job table and offsets; host inputs are staged job by job
  std::vector<JobDev>& J = P->jobs_h;
  J.assign(njobs, JobDev{});
  std::vector<uint64_t> offA(njobs + 1, 0), offB(njobs + 1, 0);
  for (uint32_t j = 0; j < njobs; ++j) {
    offA[j + 1] = offA[j] + A[j].n;
    offB[j + 1] = offB[j] + B[j].n;
  }
  const uint64_t NA = offA[njobs], NB = offB[njobs];
  if (NA >= (1ull << 32) || NB >= (1ull << 32)) {
    set_error("a batched plan holds fewer than 2^32 sources per side");
    return fail(HLC_EINVAL);
  }
  double *sra[2] = {nullptr, nullptr}, *sdec[2] = {nullptr, nullptr};
  uint64_t* sid[2] = {nullptr, nullptr};
  if (!A[0].on_device) {
    for (int s = 0; s < 2; ++s) {
      uint64_t N = s ? NB : NA;
      sra[s] = ar.get_n<double>(N + 1);
      sdec[s] = ar.get_n<double>(N + 1);
      sid[s] = ar.get_n<uint64_t>(N + 1);
      if (!sra[s] || !sdec[s] || !sid[s]) return fail(HLC_ENOMEM);
    }
  }
  for (uint32_t j = 0; j < njobs; ++j) {
    const hlc_catalog* C2[2] = {A + j, B + j};
    const uint64_t o[2] = {offA[j], offB[j]};
    for (int s = 0; s < 2; ++s) {
      J[j].n[s] = C2[s]->n;
      J[j].off[s] = o[s];
      if (C2[s]->on_device) {
        J[j].ra[s] = C2[s]->ra_deg;
        J[j].dec[s] = C2[s]->dec_deg;
        J[j].id[s] = C2[s]->id;
      } else {
        uint64_t n = C2[s]->n;
        if (n) {
          if (cudaMemcpyAsync(sra[s] + o[s], C2[s]->ra_deg, n * 8, cudaMemcpyHostToDevice, st) !=
                  cudaSuccess ||
              cudaMemcpyAsync(sdec[s] + o[s], C2[s]->dec_deg, n * 8, cudaMemcpyHostToDevice,
                              st) != cudaSuccess ||
              cudaMemcpyAsync(sid[s] + o[s], C2[s]->id, n * 8, cudaMemcpyHostToDevice, st) !=
                  cudaSuccess) {
            set_error("host to device copy failed");
            return fail(HLC_ECUDA);
          }
        }
        // staged arrays are indexed by (global - off), so point at the job's slice
        J[j].ra[s] = sra[s] + o[s];
        J[j].dec[s] = sdec[s] + o[s];
        J[j].id[s] = sid[s] + o[s];
      }
    }
    J[j].L = p[j].fine_level;
  }
  P->jobs_d = ar.get_n<JobDev>(njobs);
  P->offA_d = ar.get_n<uint64_t>(njobs + 1);
  P->offB_d = ar.get_n<uint64_t>(njobs + 1);
  if (!P->jobs_d || !P->offA_d || !P->offB_d) return fail(HLC_ENOMEM);
  auto upload_jobs = [&]() -> int {
    HLC_CUDA(cudaMemcpyAsync(P->jobs_d, J.data(), njobs * sizeof(JobDev),
                             cudaMemcpyHostToDevice, st));
    return HLC_OK;
  };
  if (cudaMemcpyAsync(P->offA_d, offA.data(), (njobs + 1) * 8, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(P->offB_d, offB.data(), (njobs + 1) * 8, cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
    return fail(HLC_ECUDA);
  int rc = upload_jobs();
  if (rc) return fail(rc);
  // autotuned orders (jobs with fine_level < 0)
  bool need_auto = false;
  for (uint32_t j = 0; j < njobs; ++j) need_auto |= p[j].fine_level < 0;
  if (need_auto && NB) {
    float* acc = ar.get_n<float>(3 * njobs + 3);
    unsigned* cap = ar.get_n<unsigned>(njobs + 1);
    if (!acc || !cap) return fail(HLC_ENOMEM);
    cudaMemsetAsync(acc, 0, (3 * njobs + 3) * 4, st);
    cudaMemsetAsync(cap, 0, (njobs + 1) * 4, st);
    k_bjob_mean<<<grid_for(32ull * njobs, kThreads), kThreads, 0, st>>>(P->jobs_d, njobs, acc);
    std::vector<float> h(3 * njobs);
    if (cudaMemcpyAsync(h.data(), acc, 3 * njobs * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail(HLC_ECUDA);
    for (uint32_t j = 0; j < njobs; ++j) {
      double x = h[3 * j], y = h[3 * j + 1], z = h[3 * j + 2];
      double nrm = std::sqrt(x * x + y * y + z * z);
      if (nrm > 0) {
        h[3 * j] = (float)(x / nrm);
        h[3 * j + 1] = (float)(y / nrm);
        h[3 * j + 2] = (float)(z / nrm);
      }
    }
    cudaMemcpyAsync(acc, h.data(), 3 * njobs * 4, cudaMemcpyHostToDevice, st);
    k_bjob_cap<<<grid_for(32ull * njobs, kThreads), kThreads, 0, st>>>(P->jobs_d, njobs, acc,
                                                                        cap);
    std::vector<unsigned> hc(njobs);
    if (cudaMemcpyAsync(hc.data(), cap, njobs * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail(HLC_ECUDA);
    for (uint32_t j = 0; j < njobs; ++j) {
      if (p[j].fine_level >= 0) continue;
      float om;
      memcpy(&om, &hc[j], 4);
      J[j].L = auto_order((double)B[j].n, (double)om, p[j].radius_arcsec,
                          P->target_per_cell > 0 ? P->target_per_cell : kTargetPerCell);
    }
  } else {
    for (uint32_t j = 0; j < njobs; ++j)
      if (J[j].L < 0) J[j].L = 0;
  }
  int maxL = 0;
  for (uint32_t j = 0; j < njobs; ++j) {
    if (p[j].boundary == HLC_COMPLETE8 && p[j].radius_arcsec > complete_max_radius(J[j].L)) {
      set_error("job %u: radius %g arcsec exceeds theta_L/8 at order %d", j, p[j].radius_arcsec,
                J[j].L);
      return fail(HLC_EINVAL);
    }
    maxL = std::max(maxL, J[j].L);
    J[j].K = pix_const(J[j].L);
    J[j].C = chord2_threshold(p[j].radius_arcsec);
    f2_sep_window(p[j].radius_arcsec, &J[j].r_lo, &J[j].r_hi);
    double G = fp32_guard_band(J[j].C, kUnitVecErr);
    float lo = (float)(J[j].C - G), hi = (float)(J[j].C + G);
    if ((double)lo > J[j].C - G) lo = nextafterf(lo, 0.0f);
    if ((double)hi < J[j].C + G) hi = nextafterf(hi, 1e30f);
    if (lo < 0) lo = -1.0f;
    J[j].lo32 = lo;
    J[j].hi32 = hi;
  }
  P->cell_bits = 2 * maxL + 4;
  int job_bits = 0;
  while ((1u << job_bits) < njobs) ++job_bits;
  const int key_bits = P->cell_bits + job_bits;
  rc = upload_jobs();
  if (rc) return fail(rc);
  // per side: composite keys, sort, payload
  CatDev* X2[2] = {&P->A, &P->B};
  uint64_t* keys[2] = {nullptr, nullptr};
  const uint64_t N2[2] = {NA, NB};
  uint64_t* offd[2] = {P->offA_d, P->offB_d};
  cudaEvent_t ev[2][4];
  for (int s = 0; s < 2; ++s)
    for (int i = 0; i < 4; ++i) cudaEventCreate(&ev[s][i]);
  for (int s = 0; s < 2 && rc == HLC_OK; ++s) {
    CatDev& X = *X2[s];
    uint64_t n = N2[s];
    X.n = X.m = n;
    keys[s] = ar.get_n<uint64_t>(n + 1);
    X.idx = ar.get_n<uint32_t>(n + 1);
    X.rec = ar.get_n<SrcRec>(n + 1);
    uint32_t* slow = ar.get_n<uint32_t>(n + 1);
    if (!keys[s] || !X.idx || !X.rec || !slow) return fail(HLC_ENOMEM);
    // the sort's scratch first: the preps count its digit histograms
    const int np = std::min((key_bits + 7) / 8, 8);
    void* scr = n > 1 ? ar.get(sort_scratch_bytes(n, np)) : nullptr;
    if (n > 1 && !scr) return fail(HLC_ENOMEM);
    uint32_t* hist = (uint32_t*)scr;
    if (hist) cudaMemsetAsync(hist, 0, (size_t)np * 256 * 4, st);
    cudaEventRecord(ev[s][0], st);
    if (n) {
      cudaMemsetAsync(P->ctr + C_SLOW, 0, 8, st);
      if (fp32) {
        k_bprep_keys<true><<<grid_for(n, kThreads, bprep_resident_blocks(true)), kThreads, 0, st>>>(
            P->jobs_d, offd[s], njobs, s, n, P->cell_bits, keys[s], X.idx, X.rec, slow,
            P->ctr + C_SLOW, P->dev_err, hist, np);
        k_bprep_fallback<<<num_sms() * 4u, kThreads, 0, st>>>(P->jobs_d, offd[s], njobs, s, P->cell_bits,
                                                       slow, P->ctr + C_SLOW, keys[s], hist, np);
      } else {
        k_bprep_keys<false><<<grid_for(n, kThreads, bprep_resident_blocks(false)), kThreads, 0,
                              st>>>(P->jobs_d, offd[s], njobs, s, n, P->cell_bits, keys[s],
                                    X.idx, X.rec, nullptr, nullptr, P->dev_err, hist, np);
      }
      g_launches += fp32 ? 2 : 1;
    }
    ar.drop(slow);
    cudaEventRecord(ev[s][1], st);
    if (n > 1) {
      uint64_t* tk = ar.get_n<uint64_t>(n);
      uint32_t* tv = ar.get_n<uint32_t>(n);
      if (!tk || !tv) return fail(HLC_ENOMEM);
      rc = radix_sort_pairs<uint64_t>(keys[s], X.idx, tk, tv, n, key_bits, scr, P->dev_err, st,
                                      0, nullptr, nullptr, nullptr, true);
      if (rc) return fail(rc);
      ar.drop(tk);
      ar.drop(tv);
      ar.drop(scr);
    }
    cudaEventRecord(ev[s][2], st);
    X.id_s = ar.get_n<uint64_t>(n + 1);
    if (!X.id_s) return fail(HLC_ENOMEM);
    if (fp32) {
      X.v32 = ar.get_n<float4>(n + 1);
      X.rd = ar.get_n<double2>(n + 1);
      if (!X.v32 || !X.rd) return fail(HLC_ENOMEM);
      if (n)
        k_bpayload<true><<<grid_for(n, kThreads), kThreads, 0, st>>>(
            X.rec, X.idx, n, X.v32, X.rd, nullptr, nullptr, nullptr, X.id_s,
            s == 0 ? P->ctr + C_IDDIFF : nullptr);
    } else {
      X.vx = ar.get_n<double>(n + 1);
      X.vy = ar.get_n<double>(n + 1);
      X.vz = ar.get_n<double>(n + 1);
      if (!X.vx || !X.vy || !X.vz) return fail(HLC_ENOMEM);
      if (n)
        k_bpayload<false><<<grid_for(n, kThreads), kThreads, 0, st>>>(
            X.rec, X.idx, n, nullptr, nullptr, X.vx, X.vy, X.vz, X.id_s,
            s == 0 ? P->ctr + C_IDDIFF : nullptr);
    }
    if (n) ++g_launches;
    ar.drop(X.rec);  // (the later stages read the sorted payload only)
    X.rec = nullptr;
    cudaEventRecord(ev[s][3], st);
  }
  P->keyA64 = keys[0];
  P->keyB64 = keys[1];
  // per-job B tables over the occupied cell range
  if (rc == HLC_OK && NB) {
    // gather the first and last composite key of every job
    uint64_t* fl = ar.get_n<uint64_t>(2 * njobs + 2);
    if (!fl) return fail(HLC_ENOMEM);
    k_job_first_last<<<grid_for(njobs, kThreads), kThreads, 0, st>>>(keys[1], offd[1], njobs, fl);
    ++g_launches;
    std::vector<uint64_t> h(2 * njobs, 0);
    if (cudaMemcpyAsync(h.data(), fl, 2 * njobs * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail(HLC_ECUDA);
    const uint64_t cmask = (1ull << P->cell_bits) - 1;
    uint64_t toff = 0;
    for (uint32_t j = 0; j < njobs; ++j) {
      uint32_t kmin = (uint32_t)(h[2 * j] & cmask), kmax = (uint32_t)(h[2 * j + 1] & cmask);
      if (!B[j].n) kmin = kmax = 0;
      int tk = 0;
      uint64_t target = std::max<uint64_t>(2 * B[j].n, 16);
      while (tk < J[j].L && ((uint64_t)(kmax >> (2 * tk)) - (kmin >> (2 * tk)) + 1) > target) ++tk;
      J[j].tk = tk;
      J[j].tbase = kmin >> (2 * tk);
      J[j].tsize = (uint32_t)((kmax >> (2 * tk)) - J[j].tbase + 2);
      J[j].toff = toff;
      toff += J[j].tsize;
    }
    rc = upload_jobs();
    if (rc) return fail(rc);
    uint32_t* counts = ar.get_n<uint32_t>(toff + 1);
    P->btable = ar.get_n<uint32_t>(toff + 1);
    void* scr = ar.get(scan_scratch_bytes(toff + 1));
    if (!counts || !P->btable || !scr) return fail(HLC_ENOMEM);
    cudaMemsetAsync(counts, 0, (toff + 1) * 4, st);
    k_btable_hist<<<grid_for(NB, kThreads), kThreads, 0, st>>>(keys[1], NB, P->cell_bits,
                                                                P->jobs_d, counts);
    ++g_launches;
    rc = scan_exclusive<uint32_t>(counts, P->btable, toff + 1, P->ctr + C_TOTAL, scr, P->dev_err,
                                  st);
    if (rc) return fail(rc);
    ar.drop(counts);
    ar.drop(scr);
  }
  // dense cells of every job for the tile kernel: runs of at least
  // kTileMinA equal (job, cell) keys among the sorted A entries (FP32 form),
  // listed as (start, end) by one pass over the keys
  if (rc == HLC_OK && NA > 1 && NB && P->p.precision == HLC_FP32_GUARD) {
    const uint64_t rcap = NA / kTileMinA + 1;  // (the runs are disjoint)
    P->A.tile_start = ar.get_n<uint32_t>(rcap);
    uint32_t* tile_end = ar.get_n<uint32_t>(rcap);
    P->A.tile_n = ar.get_n<unsigned long long>(4);
    P->A.tiled = ar.get_n<uint8_t>(NA + 1);
    if (!P->A.tile_start || !tile_end || !P->A.tile_n || !P->A.tiled) return fail(HLC_ENOMEM);
    cudaMemsetAsync(P->A.tile_n, 0, 32, st);
    cudaMemsetAsync(P->A.tiled, 0, NA + 1, st);
    k_long_runs<<<grid_for(NA, kThreads), kThreads, 0, st>>>(keys[0], NA, P->A.tile_start,
                                                              tile_end, P->A.tile_n, rcap);
    k_mark_runs<<<num_sms() * 16u, kThreads, 0, st>>>(P->A.tile_start, tile_end, P->A.tile_n,
                                                     P->A.tiled);
    g_launches += 2;
    const uint64_t cap = NA / kTileItemDiv + 1;
    P->A.tile_icap = cap;
    P->A.tile_items = ar.get_n<TileItem>(cap);
    P->A.tile_nprep = ar.get_n<unsigned long long>(2);
    if (!P->A.tile_items || !P->A.tile_nprep) return fail(HLC_ENOMEM);
    cudaMemsetAsync(P->A.tile_nprep, 0, 16, st);
    TileArgs tp{};
    tp.start = P->A.tile_start;
    tp.end = tile_end;
    tp.nitems = P->A.tile_n;
    tp.keyA64 = keys[0];
    tp.keyB64 = keys[1];
    tp.btable = P->btable;
    tp.jobs = P->jobs_d;
    tp.cell_bits = P->cell_bits;
    k_tile_items<true><<<num_sms() * 16u, 256, 0, st>>>(tp, P->A.tile_items, P->A.tile_nprep, cap);
    ++g_launches;
  }
  unsigned long long hc[C_N] = {0};
  if (rc == HLC_OK &&
      cudaMemcpyAsync(hc, P->ctr, sizeof(hc), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    rc = HLC_ECUDA;
  if (rc == HLC_OK) rc = check_dev_err(P->dev_err, st, "hlc_plan");
  if (cudaGetLastError() != cudaSuccess && rc == HLC_OK) {
    set_error("a batched plan kernel failed to launch");
    rc = HLC_ECUDA;
  }
  float t[6] = {0};
  if (rc == HLC_OK) {
    for (int s = 0; s < 2; ++s) {
      float a = 0, b = 0, c = 0;
      cudaEventElapsedTime(&a, ev[s][0], ev[s][1]);
      cudaEventElapsedTime(&b, ev[s][1], ev[s][2]);
      cudaEventElapsedTime(&c, ev[s][2], ev[s][3]);
      t[0] += a;
      t[1] += b;
      t[2] += c;
    }
  }
  for (int s = 0; s < 2; ++s)
    for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[s][i]);
  if (rc != HLC_OK) return fail(rc);
  ev_record(P, 1);
  unsigned long long diff = hc[C_IDDIFF];
  P->id_high_bit = diff ? 63 - __builtin_clzll(diff) : -1;
  memset(&P->stats, 0, sizeof(P->stats));
  P->stats.n_a = NA;
  P->stats.n_b = NB;
  P->stats.entries_a = NA;
  P->stats.entries_b = NB;
  P->stats.join_level = maxL;
  P->stats.ms_prep = t[0];
  P->stats.ms_sort = t[1];
  P->stats.ms_index = t[2];
  if (P->A.tile_n) {
    unsigned long long tn[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(tn, P->A.tile_n, 32, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail(HLC_ECUDA);
    P->stats.tile_items = tn[1];
    P->stats.tile_entries_a = tn[2];
  }
  P->plan_launches = g_launches.load() - P->launches0;
  *out = P;
  return HLC_OK;
}

// The pair test of a batched plan as a CUDA graph (counter resets + the one
// persistent launch), captured once per output capacity and replayed.
static int batched_pair_graph(hlc_plan_t* P, uint2* rows, uint64_t cap, uint2* band,
                              uint64_t bcap) {
  cudaStream_t st = plan_stream(P);
  const bool fp32 = P->p.precision == HLC_FP32_GUARD;
  if (P->pair_graph && P->graph_rows == (void*)rows && P->graph_band == (void*)band &&
      P->graph_cap == cap && P->graph_bcap == bcap) {
    ++g_launches;
    HLC_CUDA(cudaGraphLaunch(P->pair_graph, st));
    return HLC_OK;
  }
  if (P->pair_graph) {
    cudaGraphExecDestroy(P->pair_graph);
    P->pair_graph = nullptr;
  }
  cudaStream_t cs;
  HLC_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  const int tile_smem = kTileSmemDyn;
  HLC_CUDA(cudaFuncSetAttribute(k_pair_tile<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                tile_smem));
  cudaGraph_t g;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemsetAsync(P->ctr, 0, C_N * 8, cs);
    PairSink sink{rows, P->ctr + C_ROWS, cap, band, P->ctr + C_BAND, bcap,
                  P->ctr + C_TESTS, P->ctr + C_DUPS, nullptr, P->dev_err};
    BPairArgs pa;
    pa.mA = P->A.m;
    pa.keyA = P->keyA64;
    pa.keyB = P->keyB64;
    pa.table = P->btable;
    pa.jobs = P->jobs_d;
    pa.cell_bits = P->cell_bits;
    pa.axv = P->A.vx; pa.ayv = P->A.vy; pa.azv = P->A.vz;
    pa.bxv = P->B.vx; pa.byv = P->B.vy; pa.bzv = P->B.vz;
    pa.a32 = P->A.v32;
    pa.b32 = P->B.v32;
    pa.sparse_cell = P->sparse_cell;
    pa.work = P->ctr + C_SCRATCH;
    pa.tiled = P->A.tiled;
    if (P->A.m && P->B.m) {
      if (fp32)
        k_bpair<true><<<num_sms() * 8u, kThreads, 0, cs>>>(pa, sink);
      else
        k_bpair<false><<<num_sms() * 8u, kThreads, 0, cs>>>(pa, sink);
      if (fp32 && P->A.tiled) {
        TileArgs ta{};
        ta.items = P->A.tile_items;
        ta.nitems = P->A.tile_nprep;
        ta.icap = P->A.tile_icap;
        ta.work = (unsigned*)(P->ctr + C_WORK);
        ta.a32 = P->A.v32;
        ta.b32 = P->B.v32;
        ta.sparse_cell = P->sparse_cell;
        ta.keyA64 = P->keyA64;
        ta.keyB64 = P->keyB64;
        ta.btable = P->btable;
        ta.jobs = P->jobs_d;
        ta.cell_bits = P->cell_bits;
        for (int c = 0; c < 3; ++c) ta.ka[c] = P->tile_ka[c];
        ta.stage = P->tile_stage;
        PairSink tsink = sink;  // (its own test counter)
        tsink.tests = P->ctr + C_TILE_TESTS;
        k_pair_tile<false><<<num_sms() * 3u, kTileThreads + 32, tile_smem, cs>>>(ta, tsink);
      }
    }
    e = cudaStreamEndCapture(cs, &g);
  }
  if (e == cudaSuccess) {
    e = cudaGraphInstantiate(&P->pair_graph, g, 0);
    cudaGraphDestroy(g);
  }
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    set_error("pair graph capture failed: %s", cudaGetErrorString(e));
    return HLC_ECUDA;
  }
  P->graph_rows = rows;
  P->graph_band = band;
  P->graph_cap = cap;
  P->graph_bcap = bcap;
  ++g_launches;
  HLC_CUDA(cudaGraphLaunch(P->pair_graph, st));
  return HLC_OK;
}

static int match_batched(hlc_plan_t* P, hlc_result* res, hlc_stats* stats) {
  cudaStream_t st = plan_stream(P);
  Arena& ar = *P->out;
  ar.release();
  if (P->pair_graph) {  // its buffers were released with the previous result
    cudaGraphExecDestroy(P->pair_graph);
    P->pair_graph = nullptr;
  }
  CatDev& A = P->A;
  CatDev& B = P->B;
  const bool fp32 = P->p.precision == HLC_FP32_GUARD;
  const unsigned long long launches_match0 = g_launches.load();
  HLC_CUDA(cudaMemsetAsync(P->dev_err, 0, 64, st));
  ev_record(P, 2);
  ev_record(P, 3);
  uint64_t cap = P->row_cap ? P->row_cap : std::max<uint64_t>(1u << 20, A.n + B.n);
  uint64_t bcap = fp32 ? std::max<uint64_t>(1u << 16, cap / 4) : 1;
  uint2* rows = nullptr;
  uint2* band = nullptr;
  unsigned long long h[C_N];
  for (int attempt = 0; attempt < 3; ++attempt) {
    rows = ar.get_n<uint2>(cap);
    band = ar.get_n<uint2>(bcap);
    if (!rows || !band) return HLC_ENOMEM;
    HLC_TRY(batched_pair_graph(P, rows, cap, band, bcap));
    HLC_CUDA(cudaMemcpyAsync(h, P->ctr, sizeof(h), cudaMemcpyDeviceToHost, st));
    HLC_CUDA(cudaStreamSynchronize(st));
    uint64_t need = h[C_ROWS] + (fp32 ? h[C_BAND] : 0);
    if (need <= cap && h[C_BAND] <= bcap) break;
    cudaGraphExecDestroy(P->pair_graph);
    P->pair_graph = nullptr;
    ar.drop(rows);
    ar.drop(band);
    cap = need + need / 8 + 1024;
    bcap = std::max<uint64_t>(bcap, h[C_BAND] + 1024);
    HLC_CUDA(cudaMemsetAsync(P->dev_err, 0, 64, st));
    if (attempt == 2) {
      set_error("match rows did not fit after resizing");
      return HLC_ECUDA;
    }
  }
  P->row_cap = std::max<uint64_t>(P->row_cap, cap);
  ev_record(P, 4);
  if (fp32 && h[C_BAND]) {
    k_brecheck<<<grid_for(h[C_BAND], kThreads, num_sms() * 16u), kThreads, 0, st>>>(
        band, P->ctr + C_BAND, bcap, P->keyA64, P->cell_bits, P->jobs_d, A.rd, B.rd, rows,
        P->ctr + C_ROWS, cap, P->ctr + C_BAND64, P->dev_err);
    HLC_LAUNCH_CHECK();
  }
  ev_record(P, 5);
  unsigned long long M = h[C_ROWS];
  if (fp32 && h[C_BAND]) {
    HLC_CUDA(cudaMemcpyAsync(&M, P->ctr + C_ROWS, 8, cudaMemcpyDeviceToHost, st));
    HLC_CUDA(cudaStreamSynchronize(st));
  }
  HLC_TRY(check_dev_err(P->dev_err, st, "hlc_match"));
  const bool want_sep = P->p.want_sep != 0;
  OutRow* rows32 = ar.get_n<OutRow>(M + 1);
  if (!rows32) return HLC_ENOMEM;
  // buckets: per job, bits of id_a enough for about four rows per bucket
  // (the jobs' row counts differ by orders of magnitude), but no more than
  // two to four buckets per A source of the job: a bucket cannot split the
  // rows of one id_a, so more bits only add empty buckets (and keep the
  // bucket counts out of L2)
  const int hb = P->id_high_bit;
  const uint32_t nj = P->njobs;
  std::vector<uint32_t> jrows(nj, 0u);
  if (M) {
    uint32_t* jcnt = ar.get_n<uint32_t>(nj);
    if (!jcnt) return HLC_ENOMEM;
    HLC_CUDA(cudaMemsetAsync(jcnt, 0, nj * 4ull, st));
    k_job_rows<<<grid_for(M, kThreads), kThreads, 0, st>>>(rows, M, P->keyA64, P->cell_bits,
                                                           jcnt);
    HLC_LAUNCH_CHECK();
    HLC_CUDA(cudaMemcpyAsync(jrows.data(), jcnt, nj * 4ull, cudaMemcpyDeviceToHost, st));
    HLC_CUDA(cudaStreamSynchronize(st));
    ar.drop(jcnt);
  }
  std::vector<uint4> hjb(nj);
  uint64_t nbk = 0;
  for (uint32_t j = 0; j < nj; ++j) {
    int nb = 0;
    while (nb < 24 && (jrows[j] >> (nb + 2)) > 0) ++nb;
    int na_bits = 1;
    while (na_bits < 24 && (1ull << (na_bits - 1)) < P->jobs_h[j].n[0]) ++na_bits;
    nb = std::min(nb, na_bits);
    if (nb > hb + 1) nb = std::max(hb + 1, 0);
    hjb[j] = make_uint4((uint32_t)nbk, hb >= 0 ? (uint32_t)(hb + 1 - nb) : 0u,
                        nb ? (uint32_t)((1ull << nb) - 1) : 0u, 0u);
    nbk += 1ull << nb;
  }
  if (nbk >= (1ull << 31)) {
    set_error("batched output: %llu row buckets", (unsigned long long)nbk);
    return HLC_EINVAL;
  }
  uint4* jb = ar.get_n<uint4>(nj);
  uint32_t* bhist = ar.get_n<uint32_t>(nbk + 1);
  uint32_t* boff = ar.get_n<uint32_t>(nbk + 1);
  if (!jb || !bhist || !boff) return HLC_ENOMEM;
  HLC_CUDA(cudaMemcpyAsync(jb, hjb.data(), nj * sizeof(uint4), cudaMemcpyHostToDevice, st));
  HLC_CUDA(cudaMemsetAsync(bhist, 0, (nbk + 1) * 4, st));
  if (M) {
    unsigned g = grid_for(M, kThreads);
    if (fp32)
      k_brows<true><<<g, kThreads, 0, st>>>(rows, M, P->keyA64, P->cell_bits, A.id_s, B.id_s,
                                             nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                             A.rd, B.rd, want_sep, rows32, jb, bhist);
    else
      k_brows<false><<<g, kThreads, 0, st>>>(rows, M, P->keyA64, P->cell_bits, A.id_s, B.id_s,
                                              A.vx, A.vy, A.vz, B.vx, B.vy, B.vz, nullptr,
                                              nullptr, want_sep, rows32, jb, bhist);
    HLC_LAUNCH_CHECK();
  }
  ar.drop(rows);
  ar.drop(band);
  uint64_t *oa = nullptr, *ob = nullptr;
  double* os = nullptr;
  uint32_t* oj = nullptr;
  HLC_TRY(order_rows_checked(P, rows32, M, bhist, boff, nbk, jb, 0, 0u, true, want_sep, &oa,
                             &ob, &os, &oj));
  ar.drop(rows32);
  ar.drop(jb);
  ar.drop(bhist);
  ar.drop(boff);
  ev_record(P, 6);
  unsigned long long band64 = 0;
  HLC_CUDA(cudaMemcpyAsync(&band64, P->ctr + C_BAND64, 8, cudaMemcpyDeviceToHost, st));
  HLC_CUDA(cudaStreamSynchronize(st));
  HLC_TRY(check_dev_err(P->dev_err, st, "hlc_match"));
  res->n = M;
  res->id_a = oa;
  res->id_b = ob;
  res->sep_arcsec = want_sep ? os : nullptr;
  res->job = oj;
  res->on_device = 1;
  P->stats.pair_tests = h[C_TESTS] + h[C_TILE_TESTS];
  P->stats.tile_tests = h[C_TILE_TESTS];
  P->stats.band_candidates = fp32 ? h[C_BAND] : 0;
  P->stats.band_fp64 = fp32 ? band64 : 0;
  P->stats.matches = M;
  P->stats.ms_candidates = 0;
  P->stats.ms_pair = ev_ms(P, 3, 4);
  P->stats.ms_recheck = ev_ms(P, 4, 5);
  P->stats.ms_output = ev_ms(P, 5, 6);
  P->stats.ms_plan_span = ev_ms(P, 0, 1);
  P->stats.ms_total = ev_ms(P, 0, 1) + ev_ms(P, 2, 6);
  P->stats.kernel_launches = (g_launches.load() - launches_match0) + P->plan_launches;
  if (stats) *stats = P->stats;
  return HLC_OK;
}

// ---------------------------------------------------------------------------
// Streamed plans (host inputs larger than device_mem_budget).
// ---------------------------------------------------------------------------

// Device bytes one entry costs in the in-core path (inputs, keys, sort
// buffers, payload, table, rows) -- used to size the partition groups.
constexpr uint64_t kStreamBytesPerEntry = 192;
constexpr uint64_t kStreamChunk = 8ull << 20;  // sources per streamed chunk

struct HostRows {  // one group's sorted rows, in a pooled pinned block
  PinnedBuf buf;
  const uint64_t* a = nullptr;
  const uint64_t* b = nullptr;
  const double* s = nullptr;  // null without separations
  size_t n = 0;
};

// ---------------------------------------------------------------------------
// Transfer-cost model (Sec. 4.1.1, Eq. 5): a copy of d bytes takes
// T(d) = alpha + beta d.  alpha: the time of a one-byte copy; beta: (t_s -
// alpha) / s from a large copy of s bytes (pinned host memory).
// ---------------------------------------------------------------------------
struct TransferFit {
  double a[2] = {0, 0}, b[2] = {0, 0};  // [0] host to device, [1] device to host
  bool ok = false;
  double predict(int dir, uint64_t bytes, uint64_t copies) const {
    return a[dir] * (double)copies + b[dir] * (double)bytes;
  }
};

static int measure_transfer(TransferFit* fit, hlc_transfer_fit* detail) {
  const size_t S = (size_t)256 << 20;
  void* h = nullptr;
  void* d = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = HLC_OK;
  if (cudaHostAlloc(&h, S, cudaHostAllocDefault) != cudaSuccess || cudaMalloc(&d, S) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    set_error("transfer model: allocation of the 256 MiB probe buffers failed");
    rc = HLC_ENOMEM;
  }
  // median time (s) of `reps` copies of `bytes` in direction dir
  auto time_copy = [&](int dir, size_t bytes, int reps, double* out) -> int {
    std::vector<double> t;
    for (int k = 0; k < reps + 1; ++k) {  // (the first copy warms up)
      cudaEventRecord(e0, st);
      cudaError_t e = dir == 0 ? cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, st)
                               : cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, st);
      cudaEventRecord(e1, st);
      if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
        set_error("transfer model: a probe copy failed");
        return HLC_ECUDA;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (k) t.push_back(ms * 1e-3);
    }
    std::sort(t.begin(), t.end());
    *out = t[t.size() / 2];
    return HLC_OK;
  };
  static const uint64_t kCheck[4] = {64u << 10, 1u << 20, 16u << 20, 64u << 20};
  for (int dir = 0; dir < 2 && rc == HLC_OK; ++dir) {
    double alpha = 0, ts = 0;
    rc = time_copy(dir, 1, 21, &alpha);
    if (rc == HLC_OK) rc = time_copy(dir, S, 5, &ts);
    if (rc != HLC_OK) break;
    fit->a[dir] = alpha;
    fit->b[dir] = (ts - alpha) / (double)S;
    if (detail) {
      detail->alpha_s[dir] = alpha;
      detail->beta_s_per_byte[dir] = fit->b[dir];
      detail->gbs[dir] = fit->b[dir] > 0 ? 1e-9 / fit->b[dir] : 0.0;
      for (int i = 0; i < 4 && rc == HLC_OK; ++i) {
        detail->check_bytes[i] = kCheck[i];
        rc = time_copy(dir, kCheck[i], 5, &detail->check_measured_s[dir][i]);
        detail->check_model_s[dir][i] = fit->predict(dir, kCheck[i], 1);
      }
    }
  }
  fit->ok = rc == HLC_OK && fit->b[0] > 0 && fit->b[1] > 0;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (d) cudaFree(d);
  if (h) cudaFreeHost(h);
  return rc;
}

static std::mutex g_fit_mu;
static TransferFit g_fit[64];

// The current device's fit, measured on first use and kept.
static int transfer_fit(TransferFit* out) {
  int dev = 0;
  HLC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d out of range", dev);
    return HLC_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_fit_mu);
  if (!g_fit[dev].ok) HLC_TRY(measure_transfer(&g_fit[dev], nullptr));
  *out = g_fit[dev];
  return HLC_OK;
}

// Sources per streamed chunk: the smallest multiple of 2^20 (24 bytes each
// in three copies) whose copies spend at most 1% of their time in alpha,
// at most kStreamChunk.
static uint64_t chunk_from_fit(const TransferFit& f) {
  const double a = f.a[0], b = f.b[0];
  double need = b > 0 ? 100.0 * 3.0 * a / (b * 24.0) : (double)kStreamChunk;
  uint64_t c = ((uint64_t)std::ceil(need / (double)(1u << 20))) << 20;
  return std::max<uint64_t>(1u << 20, std::min<uint64_t>(c, kStreamChunk));
}

// Streams one host catalogue through the device in chunks on two streams,
// running `fn(chunk ra, dec, id, n, stream)` on each.  Pinned inputs are
// copied directly; pageable ones through two pinned staging buffers.
template <typename Fn>
static int stream_catalog(const hlc_catalog* X, double* dra[2], double* ddec[2], uint64_t* did[2],
                          void* stage[2], cudaStream_t ss[2], cudaEvent_t done[2], float* ms_h2d,
                          uint64_t chunk, uint64_t led[4], Fn fn, bool with_id = true) {
  cudaPointerAttributes at;
  bool pinned = X->n && cudaPointerGetAttributes(&at, X->ra_deg) == cudaSuccess &&
                at.type == cudaMemoryTypeHost;
  cudaGetLastError();
  if (pinned) {
    cudaPointerAttributes a2, a3;
    pinned = cudaPointerGetAttributes(&a2, X->dec_deg) == cudaSuccess &&
             a2.type == cudaMemoryTypeHost &&
             cudaPointerGetAttributes(&a3, X->id) == cudaSuccess && a3.type == cudaMemoryTypeHost;
    cudaGetLastError();
  }
  uint64_t nchunks = (X->n + chunk - 1) / chunk;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> tev;  // H2D spans, read at the end
  for (uint64_t c = 0; c < nchunks; ++c) {
    int b = (int)(c & 1);
    uint64_t o = c * chunk;
    uint64_t n = std::min(chunk, X->n - o);
    // the buffer of this parity is free once its previous chunk is done
    HLC_CUDA(cudaEventSynchronize(done[b]));
    const double* sra = X->ra_deg + o;
    const double* sdec = X->dec_deg + o;
    const uint64_t* sid = X->id + o;
    if (!pinned) {
      char* h = (char*)stage[b];
      memcpy(h, sra, n * 8);
      memcpy(h + chunk * 8, sdec, n * 8);
      if (with_id) memcpy(h + chunk * 16, sid, n * 8);
      sra = (const double*)h;
      sdec = (const double*)(h + chunk * 8);
      sid = (const uint64_t*)(h + chunk * 16);
    }
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    tev.push_back({t0, t1});
    cudaEventRecord(t0, ss[b]);
    HLC_CUDA(cudaMemcpyAsync(dra[b], sra, n * 8, cudaMemcpyHostToDevice, ss[b]));
    HLC_CUDA(cudaMemcpyAsync(ddec[b], sdec, n * 8, cudaMemcpyHostToDevice, ss[b]));
    if (with_id) HLC_CUDA(cudaMemcpyAsync(did[b], sid, n * 8, cudaMemcpyHostToDevice, ss[b]));
    led[0] += (with_id ? 3 : 2) * n * 8;  // (the transfer ledger: bytes and copies host to device)
    led[1] += with_id ? 3 : 2;
    cudaEventRecord(t1, ss[b]);
    HLC_TRY(fn(dra[b], ddec[b], with_id ? did[b] : nullptr, n, ss[b], c, b));
    HLC_CUDA(cudaEventRecord(done[b], ss[b]));
  }
  HLC_CUDA(cudaStreamSynchronize(ss[0]));
  HLC_CUDA(cudaStreamSynchronize(ss[1]));
  for (auto& e : tev) {
    float ms = 0;
    cudaEventElapsedTime(&ms, e.first, e.second);
    *ms_h2d += ms;
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  return HLC_OK;
}

static bool row_lt(uint64_t a1, uint64_t b1, double s1, uint64_t a2, uint64_t b2, double s2) {
  if (a1 != a2) return a1 < a2;
  if (b1 != b2) return b1 < b2;
  uint64_t x, y;
  memcpy(&x, &s1, 8);
  memcpy(&y, &s2, 8);
  return x < y;
}

// Merge of sorted runs into one sorted output, in parallel: splitter rows
// taken from the largest run cut every run at the same keys (lower bounds),
// so the slices are independent; each thread merges its slice of every run
// by repeatedly taking the smallest of the runs' current heads.
static void merge_runs(const std::vector<HostRows>& runs, bool want_sep, uint64_t* oa,
                       uint64_t* ob, double* os) {
  const size_t R = runs.size();
  auto lt_at = [&](size_t r, size_t i, size_t q, size_t j) {
    const HostRows& u = runs[r];
    const HostRows& v = runs[q];
    return row_lt(u.a[i], u.b[i], u.s ? u.s[i] : 0.0, v.a[j], v.b[j], v.s ? v.s[j] : 0.0);
  };
  size_t big = 0, total = 0;
  for (size_t r = 0; r < R; ++r) {
    total += runs[r].n;
    if (runs[r].n > runs[big].n) big = r;
  }
  if (total == 0) return;
  unsigned T = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
  if (total < (1u << 20)) T = 1;
  T *= 4;  // smaller slices balance better
  // cut[t][r]: start of slice t in run r (T + 1 cuts)
  std::vector<std::vector<size_t>> cut(T + 1, std::vector<size_t>(R, 0));
  for (size_t r = 0; r < R; ++r) cut[T][r] = runs[r].n;
  for (unsigned t = 1; t < T; ++t) {
    const size_t sp = runs[big].n * t / T;  // splitter: row sp of the largest run
    for (size_t r = 0; r < R; ++r) {
      size_t lo = 0, hi = runs[r].n;
      while (lo < hi) {
        const size_t mid = (lo + hi) / 2;
        if (lt_at(r, mid, big, sp))
          lo = mid + 1;
        else
          hi = mid;
      }
      cut[t][r] = lo;
    }
  }
  std::vector<size_t> base(T + 1, 0);
  for (unsigned t = 0; t < T; ++t) {
    size_t n = 0;
    for (size_t r = 0; r < R; ++r) n += cut[t + 1][r] - cut[t][r];
    base[t + 1] = base[t] + n;
  }
  std::atomic<unsigned> next{0};
  auto work = [&]() {
    std::vector<size_t> pos(R), end(R);
    std::vector<uint64_t> ha(R);
    for (unsigned t; (t = next.fetch_add(1)) < T;) {
      size_t live = 0;
      for (size_t r = 0; r < R; ++r) {
        pos[r] = cut[t][r];
        end[r] = cut[t + 1][r];
        ha[r] = pos[r] < end[r] ? runs[r].a[pos[r]] : UINT64_MAX;
        live += pos[r] < end[r];
      }
      size_t o = base[t];
      while (live) {
        // smallest head by id_a (branch-free scan); equal id_a heads, rare
        // across runs, are ordered by the whole key
        uint64_t best = ha[0];
        size_t m = 0;
        bool tie = false;
        for (size_t r = 1; r < R; ++r) {
          const uint64_t v = ha[r];
          tie |= v == best;
          const bool lt = v < best;
          best = lt ? v : best;
          m = lt ? r : m;
          tie = lt ? false : tie;
        }
        if (tie || pos[m] >= end[m]) {
          m = R;
          for (size_t r = 0; r < R; ++r) {
            if (pos[r] >= end[r]) continue;
            if (m == R || ha[r] < ha[m] || (ha[r] == ha[m] && lt_at(r, pos[r], m, pos[m])))
              m = r;
          }
        }
        const HostRows& h = runs[m];
        const size_t i = pos[m]++;
        oa[o] = h.a[i];
        ob[o] = h.b[i];
        if (want_sep) os[o] = h.s[i];
        ++o;
        if (pos[m] < end[m]) {
          ha[m] = h.a[pos[m]];
        } else {
          ha[m] = UINT64_MAX;
          --live;
        }
      }
    }
  };
  const unsigned nth = std::min<unsigned>(T, std::max(1u, std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  for (unsigned k = 1; k < nth; ++k) th.emplace_back(work);
  work();
  for (auto& x : th) x.join();
}

static int plan_streamed(const hlc_catalog* A, const hlc_catalog* B, const hlc_params* p,
                         hlc_plan_t** out) {
  HLC_TRY(validate_params(p));
  HLC_TRY(validate_catalog(A, "A"));
  HLC_TRY(validate_catalog(B, "B"));
  if (p->boundary != HLC_COMPLETE8 || p->index != HLC_INDEX_BSEARCH) {
    set_error("streamed plans support the complete boundary with the table index");
    return HLC_EUNSUPPORTED;
  }
  HLC_TRY(ensure_device_tables());
  hlc_plan_t* P = new hlc_plan_t();
  P->p = *p;
  P->al.alloc = p->alloc;
  P->al.dealloc = p->dealloc;
  P->al.ctx = p->alloc_ctx;
  P->al.stream = (cudaStream_t)p->stream;
  P->arena = new Arena(P->al);
  P->out = new Arena(P->al);
  P->streamed = true;
  auto fail = [&](int rc) {
    hlc_free(P);
    return rc;
  };
  cudaStream_t st = plan_stream(P);
  Arena& ar = *P->arena;
  const int Lf = p->fine_level, Lc = p->coarse_level;
  // the transfer-cost model of Eq. 5 (measured once per device): chunk size,
  // and every copy below goes into the ledger it predicts the time of
  TransferFit fit;
  {
    const int frc = transfer_fit(&fit);
    if (frc != HLC_OK) return fail(frc);
  }
  const uint64_t chunk = chunk_from_fit(fit);
  uint64_t led[4] = {0, 0, 0, 0};  // bytes and copies host to device, device to host
  const uint64_t nparts = 12ull << (2 * Lc);
  const PixConst K = pix_const(Lf);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  // chunk buffers, side streams, staging
  double *dra[2], *ddec[2];
  uint64_t* did[2];
  for (int b = 0; b < 2; ++b) {
    dra[b] = ar.get_n<double>(chunk);
    ddec[b] = ar.get_n<double>(chunk);
    did[b] = ar.get_n<uint64_t>(chunk);
    if (!dra[b] || !ddec[b] || !did[b]) return fail(HLC_ENOMEM);
  }
  unsigned long long* counts = ar.get_n<unsigned long long>(2 * nparts);
  int* err = ar.get_n<int>(16);
  if (!counts || !err) return fail(HLC_ENOMEM);
  cudaStream_t ss[2];
  cudaEvent_t done[2];
  void* stage[2] = {nullptr, nullptr};
  // pageable inputs go through two pinned staging buffers
  auto is_pinned = [](const hlc_catalog* X) {
    if (!X->n) return true;
    for (const void* q : {(const void*)X->ra_deg, (const void*)X->dec_deg, (const void*)X->id}) {
      cudaPointerAttributes at;
      if (cudaPointerGetAttributes(&at, q) != cudaSuccess || at.type != cudaMemoryTypeHost) {
        cudaGetLastError();
        return false;
      }
    }
    return true;
  };
  const bool need_stage = !is_pinned(A) || !is_pinned(B);
  for (int b = 0; b < 2; ++b) {
    cudaStreamCreateWithFlags(&ss[b], cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&done[b], cudaEventDisableTiming);
    cudaEventRecord(done[b], ss[b]);
    if (need_stage &&
        cudaHostAlloc(&stage[b], chunk * 24, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      set_error("pinned staging allocation failed");
      return fail(HLC_ENOMEM);
    }
  }
  auto cleanup = [&]() {
    for (int b = 0; b < 2; ++b) {
      cudaStreamSynchronize(ss[b]);
      cudaStreamDestroy(ss[b]);
      cudaEventDestroy(done[b]);
      if (stage[b]) cudaFreeHost(stage[b]);
    }
  };
  HLC_CUDA(cudaMemsetAsync(counts, 0, 2 * nparts * 8, st));
  HLC_CUDA(cudaMemsetAsync(err, 0, 64, st));
  HLC_CUDA(cudaStreamSynchronize(st));
  float ms_h2d = 0;
  int rc = HLC_OK;
  auto wall = []() { return std::chrono::steady_clock::now(); };
  auto ms_since = [](std::chrono::steady_clock::time_point t) {
    return std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t).count();
  };
  auto tw = wall();
  float w_count = 0, w_bucket = 0, w_groups = 0, w_merge = 0;
  // pass 0: the entries each coarse cell needs
  for (int side = 0; side < 2 && rc == HLC_OK; ++side) {
    const hlc_catalog* X = side ? B : A;
    unsigned long long* cnt = counts + side * nparts;
    rc = stream_catalog(X, dra, ddec, did, stage, ss, done, &ms_h2d, chunk, led,
                        [&](double* r, double* d, uint64_t* id, uint64_t n, cudaStream_t s,
                            uint64_t, int) {
                          (void)id;
                          k_part_count<<<grid_for(n, kThreads), kThreads, 0, s>>>(
                              r, d, n, Lf, Lc, side, K, cnt, err);
                          HLC_LAUNCH_CHECK();
                          return HLC_OK;
                        },
                        false);  // (the counts need positions only)
  }
  std::vector<unsigned long long> hc(2 * nparts);
  if (rc == HLC_OK) {
    if (cudaMemcpy(hc.data(), counts, 2 * nparts * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = HLC_ECUDA;
  }
  if (rc == HLC_OK) rc = check_dev_err(err, st, "hlc_plan (streamed)");
  if (rc != HLC_OK) {
    cleanup();
    return fail(rc);
  }
  w_count = ms_since(tw);
  tw = wall();
  // groups of consecutive coarse cells that fit the budget
  uint64_t budget = p->device_mem_budget;
  uint64_t fixed = 6 * chunk * 8 + 2 * nparts * 8 + (64ull << 20);
  // (each entry of a group also has its slot in the prefetch buffers of the
  // group after it: 24 bytes)
  uint64_t cap_entries = std::max<uint64_t>(
      4096, (budget > fixed ? budget - fixed : budget) / (kStreamBytesPerEntry + 24));
  std::vector<std::pair<uint32_t, uint32_t>> groups;
  uint64_t acc = 0;
  uint32_t g0 = 0;
  for (uint32_t q = 0; q < nparts; ++q) {
    uint64_t c = hc[q] + hc[nparts + q];
    if (acc > 0 && acc + c > cap_entries) {
      groups.push_back({g0, q});
      g0 = q;
      acc = 0;
    }
    acc += c;
  }
  groups.push_back({g0, (uint32_t)nparts});
  // pass 1: every chunk bucketed by group on the device (a B source once per
  // group that needs it) and copied to pinned host runs; the per-chunk group
  // offsets are kept on the host
  const uint32_t ngroups = (uint32_t)groups.size();
  if ((uint64_t)ngroups * 8 > 48 * 1024) {
    cleanup();
    set_error("device_mem_budget too small: %u partition groups", ngroups);
    return fail(HLC_EUNSUPPORTED);
  }
  std::vector<uint32_t> c2g(nparts);
  for (uint32_t gi = 0; gi < ngroups; ++gi)
    for (uint32_t q = groups[gi].first; q < groups[gi].second; ++q) c2g[q] = gi;
  uint32_t* cell2group = ar.get_n<uint32_t>(nparts);
  uint32_t* gcnt[2];
  uint32_t* gcur[2];
  uint32_t* goff[2];
  double *bra[2], *bdec[2];
  uint64_t* bid[2];
  uint64_t bcap[2];
  uint32_t* hgoff_pin = nullptr;  // 2 x (ngroups + 1), pinned
  if (!cell2group) {
    cleanup();
    return fail(HLC_ENOMEM);
  }
  for (int b = 0; b < 2; ++b) {
    gcnt[b] = ar.get_n<uint32_t>(ngroups + 1);
    gcur[b] = ar.get_n<uint32_t>(ngroups + 1);
    goff[b] = ar.get_n<uint32_t>(ngroups + 1);
    // group-ordered chunk (grown when a chunk's B halo needs more)
    bcap[b] = std::max<uint64_t>(1024, std::min<uint64_t>(chunk,
                                                         std::max(A->n, B->n)) * 5 / 4);
    bra[b] = ar.get_n<double>(bcap[b]);
    bdec[b] = ar.get_n<double>(bcap[b]);
    bid[b] = ar.get_n<uint64_t>(bcap[b]);
    if (!gcnt[b] || !gcur[b] || !goff[b] || !bra[b] || !bdec[b] || !bid[b]) {
      cleanup();
      return fail(HLC_ENOMEM);
    }
  }
  if (cudaHostAlloc((void**)&hgoff_pin, 2 * (ngroups + 1) * 4, cudaHostAllocDefault) !=
      cudaSuccess) {
    cudaGetLastError();
    cleanup();
    set_error("pinned allocation failed");
    return fail(HLC_ENOMEM);
  }
  HLC_CUDA(cudaMemcpy(cell2group, c2g.data(), nparts * 4, cudaMemcpyHostToDevice));
  // host runs: side 0 (A) holds each source once, side 1 (B) at most its
  // per-cell count sum
  uint64_t hcap[2] = {A->n, 0};
  for (uint32_t q = 0; q < nparts; ++q) hcap[1] += hc[nparts + q];
  double *hra[2] = {nullptr, nullptr}, *hdec[2] = {nullptr, nullptr};
  uint64_t* hid[2] = {nullptr, nullptr};
  char* run_block_owned = nullptr;  // set once the runs are carved (below)
  size_t run_block_bytes = 0;
  auto free_host = [&]() {
    if (run_block_owned) pinned_release(run_block_owned, run_block_bytes);
    run_block_owned = nullptr;
    for (int sd = 0; sd < 2; ++sd) {
      hra[sd] = hdec[sd] = nullptr;
      hid[sd] = nullptr;
    }
    if (hgoff_pin) cudaFreeHost(hgoff_pin);
    hgoff_pin = nullptr;
  };
  size_t run_bytes = 0;
  char* run_block = nullptr;
  {
    const size_t b0 = (size_t)(hcap[0] + 1) * 8, b1 = (size_t)(hcap[1] + 1) * 8;
    run_bytes = 3 * (b0 + b1);
    run_block = (char*)pinned_acquire(&run_bytes);
    if (!run_block) {
      free_host();
      cleanup();
      set_error("pinned host runs (%zu bytes) could not be allocated", 3 * (b0 + b1));
      return fail(HLC_ENOMEM);
    }
    hra[0] = (double*)run_block;
    hdec[0] = (double*)(run_block + b0);
    hid[0] = (uint64_t*)(run_block + 2 * b0);
    hra[1] = (double*)(run_block + 3 * b0);
    hdec[1] = (double*)(run_block + 3 * b0 + b1);
    hid[1] = (uint64_t*)(run_block + 3 * b0 + 2 * b1);
    run_block_owned = run_block;
    run_block_bytes = run_bytes;
  }
  // hoff[side][chunk][g]: start of group g inside the chunk's run; hbase: run start
  std::vector<std::vector<std::vector<uint32_t>>> hoff(2);
  std::vector<std::vector<uint64_t>> hbase(2);
  const size_t gsmem = 2 * (size_t)ngroups * 4;
  for (int side = 0; side < 2 && rc == HLC_OK; ++side) {
    const hlc_catalog* X = side ? B : A;
    uint64_t filled = 0;
    rc = stream_catalog(
        X, dra, ddec, did, stage, ss, done, &ms_h2d, chunk, led,
        [&](double* r, double* d, uint64_t* id, uint64_t n, cudaStream_t s, uint64_t c,
            int b) {
          HLC_CUDA(cudaMemsetAsync(gcnt[b], 0, (ngroups + 1) * 4, s));
          HLC_CUDA(cudaMemsetAsync(gcur[b], 0, (ngroups + 1) * 4, s));
          k_group_hist<<<grid_for(n, kThreads, num_sms() * 4u), kThreads, gsmem / 2, s>>>(
              r, d, n, Lf, Lc, side, K, cell2group, ngroups, gcnt[b]);
          HLC_LAUNCH_CHECK();
          k_small_excl_scan<<<1, 1024, 0, s>>>(gcnt[b], ngroups, goff[b]);
          HLC_LAUNCH_CHECK();
          uint32_t* hg = hgoff_pin + b * (ngroups + 1);
          HLC_CUDA(cudaMemcpyAsync(hg, goff[b], (ngroups + 1) * 4, cudaMemcpyDeviceToHost, s));
          led[2] += (ngroups + 1) * 4;
          led[3] += 1;
          HLC_CUDA(cudaStreamSynchronize(s));
          const uint64_t tot = hg[ngroups];
          if (filled + tot > hcap[side]) {
            set_error("streamed bucketing overflowed its host runs");
            return HLC_ECUDA;
          }
          if (tot > bcap[b]) {  // this chunk's halo copies need a larger buffer
            ar.drop(bra[b]);
            ar.drop(bdec[b]);
            ar.drop(bid[b]);
            bcap[b] = tot + tot / 8;
            bra[b] = ar.get_n<double>(bcap[b]);
            bdec[b] = ar.get_n<double>(bcap[b]);
            bid[b] = ar.get_n<uint64_t>(bcap[b]);
            if (!bra[b] || !bdec[b] || !bid[b]) return HLC_ENOMEM;
            HLC_CUDA(cudaStreamSynchronize(st));  // allocations are ordered on the plan stream
          }
          k_group_scatter<<<grid_for(n, kThreads, num_sms() * 4u), kThreads, gsmem, s>>>(
              r, d, id, n, Lf, Lc, side, K, cell2group, ngroups, goff[b], gcur[b], bra[b],
              bdec[b], bid[b], err);
          HLC_LAUNCH_CHECK();
          hoff[side].push_back(std::vector<uint32_t>(hg, hg + ngroups + 1));
          hbase[side].push_back(filled);
          if (tot) {
            HLC_CUDA(cudaMemcpyAsync(hra[side] + filled, bra[b], tot * 8, cudaMemcpyDeviceToHost,
                                     s));
            HLC_CUDA(cudaMemcpyAsync(hdec[side] + filled, bdec[b], tot * 8,
                                     cudaMemcpyDeviceToHost, s));
            HLC_CUDA(cudaMemcpyAsync(hid[side] + filled, bid[b], tot * 8, cudaMemcpyDeviceToHost,
                                     s));
            led[2] += 3 * tot * 8;
            led[3] += 3;
          }
          filled += tot;
          (void)c;
          return HLC_OK;
        });
  }
  if (rc == HLC_OK) rc = check_dev_err(err, st, "hlc_plan (streamed)");
  for (int b = 0; b < 2; ++b) {
    ar.drop(bra[b]);
    ar.drop(bdec[b]);
    ar.drop(bid[b]);
  }
  w_bucket = ms_since(tw);
  tw = wall();
  // pass 2: per group, its slices of every chunk's run in, match in core, rows
  // out.  The next group's slices are copied in on a copy stream, into a
  // second set of buffers, while the current group is matched (the groups
  // are sized for that second set: kStreamBytesPerEntry + 24 bytes an entry).
  std::vector<HostRows> runs;
  hlc_stats agg{};
  struct Slot {
    double *ra[2] = {nullptr, nullptr}, *dec[2] = {nullptr, nullptr};
    uint64_t* id[2] = {nullptr, nullptr};
    uint64_t n[2] = {0, 0};
  };
  Slot slot[2];
  cudaStream_t cps = nullptr;
  cudaEvent_t cev0[2] = {nullptr, nullptr}, cev1[2] = {nullptr, nullptr}, stev = nullptr;
  bool cps_ok = cudaStreamCreateWithFlags(&cps, cudaStreamNonBlocking) == cudaSuccess &&
                cudaEventCreateWithFlags(&stev, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; k < 2 && cps_ok; ++k)
    cps_ok = cudaEventCreate(&cev0[k]) == cudaSuccess && cudaEventCreate(&cev1[k]) == cudaSuccess;
  if (!cps_ok) {
    cudaGetLastError();
    rc = HLC_ECUDA;
  }
  auto group_size = [&](uint32_t g, uint64_t gn[2]) {
    gn[0] = gn[1] = 0;
    for (int side = 0; side < 2; ++side)
      for (auto& o : hoff[side]) gn[side] += o[g + 1] - o[g];
  };
  auto next_group = [&](uint32_t from) {
    for (uint32_t g = from; g < ngroups; ++g) {
      uint64_t gn[2];
      group_size(g, gn);
      if (gn[0] && gn[1]) return g;
    }
    return ngroups;
  };
  auto release = [&](Slot& S) {
    for (int side = 0; side < 2; ++side) {
      if (S.ra[side]) ar.drop(S.ra[side]);
      if (S.dec[side]) ar.drop(S.dec[side]);
      if (S.id[side]) ar.drop(S.id[side]);
      S.ra[side] = S.dec[side] = nullptr;
      S.id[side] = nullptr;
    }
  };
  // group g's slices of every chunk's run into slot k, on the copy stream
  // (after everything issued on the plan stream so far)
  auto fetch = [&](uint32_t g, int k) -> int {
    Slot& S = slot[k];
    group_size(g, S.n);
    HLC_CUDA(cudaEventRecord(stev, st));
    HLC_CUDA(cudaStreamWaitEvent(cps, stev, 0));
    HLC_CUDA(cudaEventRecord(cev0[k], cps));
    for (int side = 0; side < 2; ++side) {
      S.ra[side] = ar.get_n<double>(S.n[side] + 1);
      S.dec[side] = ar.get_n<double>(S.n[side] + 1);
      S.id[side] = ar.get_n<uint64_t>(S.n[side] + 1);
      if (!S.ra[side] || !S.dec[side] || !S.id[side]) return HLC_ENOMEM;
      uint64_t o = 0;
      for (size_t c = 0; c < hoff[side].size(); ++c) {
        const uint64_t s0 = hbase[side][c] + hoff[side][c][g];
        const uint64_t len = hoff[side][c][g + 1] - hoff[side][c][g];
        if (!len) continue;
        HLC_CUDA(cudaMemcpyAsync(S.ra[side] + o, hra[side] + s0, len * 8,
                                 cudaMemcpyHostToDevice, cps));
        HLC_CUDA(cudaMemcpyAsync(S.dec[side] + o, hdec[side] + s0, len * 8,
                                 cudaMemcpyHostToDevice, cps));
        HLC_CUDA(cudaMemcpyAsync(S.id[side] + o, hid[side] + s0, len * 8,
                                 cudaMemcpyHostToDevice, cps));
        led[0] += 3 * len * 8;
        led[1] += 3;
        o += len;
      }
    }
    HLC_CUDA(cudaEventRecord(cev1[k], cps));
    return HLC_OK;
  };
  uint32_t gi = rc == HLC_OK ? next_group(0) : ngroups;
  int cur = 0;
  if (gi < ngroups) rc = fetch(gi, cur);
  while (gi < ngroups && rc == HLC_OK) {
    const uint32_t gnext = next_group(gi + 1);
    if (gnext < ngroups) rc = fetch(gnext, cur ^ 1);  // (behind this group's copies)
    if (rc != HLC_OK) break;
    Slot& S = slot[cur];
    const uint64_t na = S.n[0], nb = S.n[1];
    double *gra[2] = {S.ra[0], S.ra[1]}, *gdec[2] = {S.dec[0], S.dec[1]};
    uint64_t* gid[2] = {S.id[0], S.id[1]};
    if (cudaStreamWaitEvent(st, cev1[cur], 0) != cudaSuccess) {
      rc = HLC_ECUDA;
      break;
    }
    hlc_plan_t* G = nullptr;
    if (rc == HLC_OK) {
      hlc_catalog ca{gra[0], gdec[0], gid[0], na, 1}, cb{gra[1], gdec[1], gid[1], nb, 1};
      hlc_params q = *p;
      q.device_mem_budget = 0;
      rc = plan_single(&ca, &cb, &q, &G);
    }
    hlc_result r{};
    hlc_stats gs{};
    if (rc == HLC_OK) rc = match_single(G, &r, &gs);
    if (rc == HLC_OK && r.n) {
      HostRows h;
      const size_t rb = (size_t)r.n * 8;
      if (!h.buf.get((r.sep_arcsec ? 3 : 2) * rb)) {
        set_error("pinned result rows could not be allocated");
        rc = HLC_ENOMEM;
      } else {
        h.n = r.n;
        h.a = (const uint64_t*)h.buf.p;
        h.b = (const uint64_t*)(h.buf.p + rb);
        h.s = r.sep_arcsec ? (const double*)(h.buf.p + 2 * rb) : nullptr;
        cudaEvent_t d0, d1;
        cudaEventCreate(&d0);
        cudaEventCreate(&d1);
        cudaEventRecord(d0, st);
        if (cudaMemcpyAsync(h.buf.p, r.id_a, rb, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(h.buf.p + rb, r.id_b, rb, cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            (r.sep_arcsec && cudaMemcpyAsync(h.buf.p + 2 * rb, r.sep_arcsec, rb,
                                             cudaMemcpyDeviceToHost, st) != cudaSuccess))
          rc = HLC_ECUDA;
        led[2] += (r.sep_arcsec ? 3 : 2) * rb;
        led[3] += r.sep_arcsec ? 3 : 2;
        cudaEventRecord(d1, st);
        cudaStreamSynchronize(st);
        float ms = 0;
        cudaEventElapsedTime(&ms, d0, d1);
        agg.ms_d2h += ms;
        cudaEventDestroy(d0);
        cudaEventDestroy(d1);
      }
      runs.push_back(std::move(h));
    }
    if (G) {
      agg.pair_tests += gs.pair_tests;
      agg.band_candidates += gs.band_candidates;
      agg.band_fp64 += gs.band_fp64;
      agg.entries_b += gs.entries_b;
      agg.ms_prep += gs.ms_prep;
      agg.ms_sort += gs.ms_sort;
      agg.ms_index += gs.ms_index;
      agg.ms_pair += gs.ms_pair;
      agg.ms_recheck += gs.ms_recheck;
      agg.ms_output += gs.ms_output;
      agg.kernel_launches += gs.kernel_launches;
      agg.dense_entries_b += gs.dense_entries_b;
      agg.tile_items += gs.tile_items;
      agg.tile_entries_a += gs.tile_entries_a;
      hlc_free(G);
    }
    {  // this group's copy span (the copy stream ran ahead of the matches)
      float ms = 0;
      if (cudaEventElapsedTime(&ms, cev0[cur], cev1[cur]) == cudaSuccess) ms_h2d += ms;
      cudaGetLastError();
    }
    release(S);
    if (rc != HLC_OK) break;
    ++agg.partitions;
    gi = gnext;
    cur ^= 1;
  }
  if (cps) cudaStreamSynchronize(cps);
  release(slot[0]);
  release(slot[1]);
  if (cps) cudaStreamDestroy(cps);
  for (int k = 0; k < 2; ++k) {
    if (cev0[k]) cudaEventDestroy(cev0[k]);
    if (cev1[k]) cudaEventDestroy(cev1[k]);
  }
  if (stev) cudaEventDestroy(stev);
  free_host();
  cleanup();
  w_groups = ms_since(tw);
  tw = wall();
  if (rc != HLC_OK) return fail(rc);
  // k-way merge of the groups' sorted rows
  uint64_t M = 0;
  for (auto& h : runs) M += h.n;
  const bool want_sep = p->want_sep != 0;
  if (M && !P->host_buf.get((want_sep ? 3 : 2) * M * 8)) {
    set_error("pinned output rows could not be allocated");
    return fail(HLC_ENOMEM);
  }
  P->host_n = M;
  P->host_a = (uint64_t*)P->host_buf.p;
  P->host_b = M ? (uint64_t*)(P->host_buf.p + M * 8) : nullptr;
  P->host_s = want_sep && M ? (double*)(P->host_buf.p + 2 * M * 8) : nullptr;
  merge_runs(runs, want_sep, P->host_a, P->host_b, P->host_s);
  runs.clear();  // their blocks go back to the pool
  w_merge = ms_since(tw);
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float total = 0;
  cudaEventElapsedTime(&total, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  agg.n_a = A->n;
  agg.n_b = B->n;
  agg.entries_a = A->n;
  agg.matches = M;
  agg.join_level = Lf;
  agg.ms_h2d = ms_h2d;
  agg.h2d_bytes = led[0];
  agg.h2d_copies = led[1];
  agg.d2h_bytes = led[2];
  agg.d2h_copies = led[3];
  agg.ms_model_h2d = (float)(fit.predict(0, led[0], led[1]) * 1e3);
  agg.ms_model_d2h = (float)(fit.predict(1, led[2], led[3]) * 1e3);
  agg.stream_chunk = chunk;
  agg.ms_total = total;
  agg.ms_stream_count = w_count;
  agg.ms_stream_bucket = w_bucket;
  agg.ms_stream_groups = w_groups;
  agg.ms_stream_merge = w_merge;
  P->stats = agg;
  *out = P;
  return HLC_OK;
}

static int match_streamed(hlc_plan_t* P, hlc_result* res, hlc_stats* stats) {
  res->n = P->host_n;
  res->id_a = P->host_a;
  res->id_b = P->host_b;
  res->sep_arcsec = P->p.want_sep ? P->host_s : nullptr;
  res->job = nullptr;
  res->on_device = 0;
  if (stats) *stats = P->stats;
  return HLC_OK;
}

}  // namespace hlc

using namespace hlc;

// ---------------------------------------------------------------------------
// C ABI.
// ---------------------------------------------------------------------------
extern "C" {

const char* hlc_last_error(void) { return g_msg; }
const char* hlc_version(void) { return "hlc-b300 0.1 (sm_103a)"; }

extern "C" int hlc_abi_sizes(size_t* out, int n) {
  const size_t sz[8] = {sizeof(hlc_catalog), sizeof(hlc_tune), sizeof(hlc_tune_trial),
                        sizeof(hlc_tune_report), sizeof(hlc_params), sizeof(hlc_result),
                        sizeof(hlc_stats), sizeof(hlc_transfer_fit)};
  for (int i = 0; out && i < n && i < 8; ++i) out[i] = sz[i];
  return 8;
}

int hlc_canonical_coefficients(double sin_c[10], double cos_c[11]) {
  if (!sin_c || !cos_c) {
    set_error("NULL output");
    return HLC_EINVAL;
  }
  const Canon& K = canon();
  memcpy(sin_c, K.s, sizeof(K.s));
  memcpy(cos_c, K.c, sizeof(K.c));
  return HLC_OK;
}

int hlc_plan(const hlc_catalog* A, const hlc_catalog* B, const hlc_params* p, uint32_t n_jobs,
             hlc_plan_t** out) {
  clear_error();
  if (!out) {
    set_error("out is NULL");
    return HLC_EINVAL;
  }
  if (n_jobs == 0) {
    set_error("n_jobs must be >= 1");
    return HLC_EINVAL;
  }
  if (!A || !B || !p) {
    set_error("A, B or params is NULL");
    return HLC_EINVAL;
  }
  if (n_jobs > 1) {
    for (uint32_t j = 0; j < n_jobs; ++j)
      if (p[j].radius_rule != HLC_RADIUS_FIXED) {
        set_error("job %u: batched plans take one radius per job (HLC_RADIUS_FIXED)", j);
        return HLC_EUNSUPPORTED;
      }
    return plan_batched(A, B, p, n_jobs, out);
  }
  if (p->device_mem_budget && !A->on_device && !B->on_device) {
    // stream by coarse partition when the in-core footprint exceeds the budget
    uint64_t need = (A->n + B->n) * kStreamBytesPerEntry;
    if (need > p->device_mem_budget) {
      if (p->radius_rule != HLC_RADIUS_FIXED) {
        set_error("streamed plans take one radius (HLC_RADIUS_FIXED)");
        return HLC_EUNSUPPORTED;
      }
      return plan_streamed(A, B, p, out);
    }
  }
  return plan_single(A, B, p, out);
}

int hlc_match(hlc_plan_t* plan, hlc_result* out, hlc_stats* stats) {
  clear_error();
  if (!plan || !out) {
    set_error("plan or out is NULL");
    return HLC_EINVAL;
  }
  hlc_result r{};
  int rc = plan->streamed   ? match_streamed(plan, &r, stats)
           : plan->njobs > 1 ? match_batched(plan, &r, stats)
                             : match_single(plan, &r, stats);
  if (rc == HLC_OK) *out = r;
  return rc;
}

int hlc_result_to_host(const hlc_result* r, uint64_t* id_a, uint64_t* id_b, double* sep,
                       uint32_t* job) {
  clear_error();
  if (!r) {
    set_error("result is NULL");
    return HLC_EINVAL;
  }
  if (r->n == 0) return HLC_OK;
  // on the calling thread's own default stream (the result is complete once
  // hlc_match has returned): a copy on the legacy default stream would also
  // wait for, and hold up, the work other threads run on blocking streams
  HLC_TRY(hlc_result_to_host_async(r, id_a, id_b, sep, job, (void*)cudaStreamPerThread));
  HLC_CUDA(cudaStreamSynchronize(cudaStreamPerThread));
  return HLC_OK;
}

int hlc_result_to_host_async(const hlc_result* r, uint64_t* id_a, uint64_t* id_b, double* sep,
                             uint32_t* job, void* stream) {
  clear_error();
  if (!r) {
    set_error("result is NULL");
    return HLC_EINVAL;
  }
  if (r->n == 0) return HLC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemcpyKind k = r->on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
  if (id_a) HLC_CUDA(cudaMemcpyAsync(id_a, r->id_a, r->n * 8, k, st));
  if (id_b) HLC_CUDA(cudaMemcpyAsync(id_b, r->id_b, r->n * 8, k, st));
  if (sep && r->sep_arcsec) HLC_CUDA(cudaMemcpyAsync(sep, r->sep_arcsec, r->n * 8, k, st));
  if (job && r->job) HLC_CUDA(cudaMemcpyAsync(job, r->job, r->n * 4, k, st));
  return HLC_OK;
}

void hlc_free(hlc_plan_t* plan) {
  if (!plan) return;
  cudaStream_t st = (cudaStream_t)plan->p.stream;
  cudaStreamSynchronize(st);
  if (plan->pair_graph) cudaGraphExecDestroy(plan->pair_graph);
  delete plan->out;
  delete plan->arena;
  for (int i = 0; i < 12; ++i) pool_event_back(plan->ev[i], true);
  cudaStreamSynchronize(st);
  delete plan;
}

int hlc_ang2pix(const double* ra, const double* dec, uint64_t n, int order, int precision,
                uint32_t* pix, void* stream) {
  clear_error();
  if (order < 0 || order > 14 || (precision != HLC_FP64 && precision != HLC_FP32_GUARD)) {
    set_error("order must be in [0, 14] and precision HLC_FP64 or HLC_FP32_GUARD");
    return HLC_EINVAL;
  }
  if (n == 0) return HLC_OK;
  if (!ra || !dec || !pix) {
    set_error("NULL array");
    return HLC_EINVAL;
  }
  HLC_TRY(ensure_device_tables());
  cudaStream_t st = (cudaStream_t)stream;
  int* err = nullptr;
  HLC_CUDA(cudaMallocAsync(&err, sizeof(int), st));
  cudaMemsetAsync(err, 0, sizeof(int), st);
  uint32_t* idx = nullptr;
  cudaError_t e = cudaMallocAsync(&idx, n * 4, st);
  if (e != cudaSuccess) {
    cudaFreeAsync(err, st);
    set_error("cudaMallocAsync failed: %s", cudaGetErrorString(e));
    return HLC_ENOMEM;
  }
  uint32_t* slow = nullptr;
  unsigned long long* nslow = nullptr;
  if (precision == HLC_FP32_GUARD) {
    if (cudaMallocAsync(&slow, n * 4, st) != cudaSuccess ||
        cudaMallocAsync(&nslow, 8, st) != cudaSuccess) {
      cudaGetLastError();
      if (slow) cudaFreeAsync(slow, st);
      cudaFreeAsync(idx, st);
      cudaFreeAsync(err, st);
      set_error("cudaMallocAsync failed");
      return HLC_ENOMEM;
    }
    cudaMemsetAsync(nslow, 0, 8, st);
    k_prep_keys<true><<<grid_for(n, kThreads), kThreads, 0, st>>>(
        ra, dec, nullptr, n, order, pix_const(order), pix, idx, nullptr, slow, nslow, err);
    k_prep_fallback<<<num_sms() * 4u, kThreads, 0, st>>>(ra, dec, order, slow, nslow, pix);
  } else {
    k_prep_keys<false><<<grid_for(n, kThreads), kThreads, 0, st>>>(
        ra, dec, nullptr, n, order, pix_const(order), pix, idx, nullptr, nullptr, nullptr, err);
  }
  int rc = HLC_OK;
  if (cudaGetLastError() != cudaSuccess) {
    set_error("ang2pix launch failed");
    rc = HLC_ECUDA;
  }
  if (rc == HLC_OK) rc = check_dev_err(err, st, "hlc_ang2pix");
  if (slow) cudaFreeAsync(slow, st);
  if (nslow) cudaFreeAsync(nslow, st);
  cudaFreeAsync(idx, st);
  cudaFreeAsync(err, st);
  return rc;
}

}  // extern "C"

namespace hlc {
__global__ void k_neighbours(const uint32_t* __restrict__ pix, uint64_t n, int order,
                             int64_t* __restrict__ out) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    int face, ix, iy;
    nest_to_fxy(pix[i], order, &face, &ix, &iy);
    for (int d = 0; d < 8; ++d)
      out[8 * i + d] = nbr_step(face, ix, iy, d_dirs[d][0], d_dirs[d][1], order);
  }
}
__global__ void k_unitvec(const double* __restrict__ ra, const double* __restrict__ dec,
                          uint64_t n, double* __restrict__ xyz) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    double x = 0, y = 0, z = 0;
    if (c_valid(ra[i], dec[i])) c_unitvec(c_norm_ra(ra[i]), dec[i], &x, &y, &z);
    xyz[3 * i] = x;
    xyz[3 * i + 1] = y;
    xyz[3 * i + 2] = z;
  }
}
}  // namespace hlc

extern "C" {

int hlc_neighbours(const uint32_t* pix, uint64_t n, int order, int64_t* out, void* stream) {
  clear_error();
  if (order < 0 || order > 14) {
    set_error("order must be in [0, 14]");
    return HLC_EINVAL;
  }
  if (n == 0) return HLC_OK;
  if (!pix || !out) {
    set_error("NULL array");
    return HLC_EINVAL;
  }
  HLC_TRY(ensure_device_tables());
  k_neighbours<<<grid_for(n, kThreads), kThreads, 0, (cudaStream_t)stream>>>(pix, n, order, out);
  HLC_LAUNCH_CHECK();
  return HLC_OK;
}

int hlc_quad_cells(const double* ra, const double* dec, uint64_t n, double radius_arcsec,
                   int order, int precision, int boundary, uint32_t* out, int32_t* count,
                   void* stream) {
  clear_error();
  if (order < 0 || order > 14 || !(radius_arcsec > 0.0) || !(radius_arcsec <= 648000.0) ||
      (precision != HLC_FP64 && precision != HLC_FP32_GUARD) ||
      (boundary != HLC_QUAD && boundary != HLC_QUAD_COSDEC)) {
    set_error("order must be in [0, 14], radius in (0, 648000], precision HLC_FP64 or "
              "HLC_FP32_GUARD and boundary HLC_QUAD or HLC_QUAD_COSDEC");
    return HLC_EINVAL;
  }
  const bool cosdec = boundary == HLC_QUAD_COSDEC;
  if (n == 0) return HLC_OK;
  if (!ra || !dec || !out || !count) {
    set_error("NULL array");
    return HLC_EINVAL;
  }
  HLC_TRY(ensure_device_tables());
  cudaStream_t st = (cudaStream_t)stream;
  const double R = radius_arcsec / 3600.0;
  int* err = nullptr;
  HLC_CUDA(cudaMallocAsync(&err, 16, st));
  cudaMemsetAsync(err, 0, 16, st);
  int rc = HLC_OK;
  if (precision == HLC_FP32_GUARD) {
    uint32_t* slow = nullptr;
    unsigned long long* nslow = (unsigned long long*)(err + 2);
    if (cudaMallocAsync(&slow, n * 4, st) != cudaSuccess) {
      cudaFreeAsync(err, st);
      set_error("cudaMallocAsync(%llu bytes) failed", (unsigned long long)(n * 4));
      return HLC_ENOMEM;
    }
    k_quad_cells<true><<<grid_for(n, kThreads), kThreads, 0, st>>>(
        ra, dec, nullptr, n, R, order, pix_const(order), out, (uint32_t*)count, nullptr, slow,
        nslow, err, cosdec);
    k_quad_fallback<<<num_sms() * 4u, kThreads, 0, st>>>(ra, dec, R, order, slow, nslow, out,
                                                  (uint32_t*)count, cosdec);
    rc = cudaGetLastError() == cudaSuccess ? HLC_OK : HLC_ECUDA;
    cudaFreeAsync(slow, st);
  } else {
    k_quad_cells<false><<<grid_for(n, kThreads), kThreads, 0, st>>>(
        ra, dec, nullptr, n, R, order, pix_const(order), out, (uint32_t*)count, nullptr, nullptr,
        nullptr, err, cosdec);
    rc = cudaGetLastError() == cudaSuccess ? HLC_OK : HLC_ECUDA;
  }
  if (rc == HLC_OK) rc = check_dev_err(err, st, "hlc_quad_cells");
  cudaFreeAsync(err, st);
  return rc;
}

int hlc_unitvec(const double* ra, const double* dec, uint64_t n, double* xyz, void* stream) {
  clear_error();
  if (n == 0) return HLC_OK;
  if (!ra || !dec || !xyz) {
    set_error("NULL array");
    return HLC_EINVAL;
  }
  HLC_TRY(ensure_device_tables());
  k_unitvec<<<grid_for(n, kThreads), kThreads, 0, (cudaStream_t)stream>>>(ra, dec, n, xyz);
  HLC_LAUNCH_CHECK();
  return HLC_OK;
}

int hlc_sort_pairs(void* keys, uint32_t* vals, uint64_t n, int key_size, int key_bits,
                   void* stream) {
  clear_error();
  if ((key_size != 4 && key_size != 8) || key_bits < 1 || key_bits > 8 * key_size) {
    set_error("key_size must be 4 or 8 and key_bits in [1, 8*key_size]");
    return HLC_EINVAL;
  }
  if (n <= 1) return HLC_OK;
  if (!keys || !vals) {
    set_error("NULL array");
    return HLC_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int npass = (key_bits + 7) / 8;
  size_t sb = sort_scratch_bytes(n, npass);
  void* tk = nullptr;
  void* tv = nullptr;
  void* scr = nullptr;
  int* err = nullptr;
  int rc = HLC_OK;
  if (cudaMallocAsync(&tk, n * key_size, st) != cudaSuccess ||
      cudaMallocAsync(&tv, n * 4, st) != cudaSuccess ||
      cudaMallocAsync(&scr, sb, st) != cudaSuccess ||
      cudaMallocAsync(&err, 64, st) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMallocAsync failed for sort temporaries");
    rc = HLC_ENOMEM;
  }
  if (rc == HLC_OK) {
    cudaMemsetAsync(err, 0, 64, st);
    if (key_size == 4)
      rc = radix_sort_pairs<uint32_t>((uint32_t*)keys, vals, (uint32_t*)tk, (uint32_t*)tv, n,
                                      key_bits, scr, err, st);
    else
      rc = radix_sort_pairs<uint64_t>((uint64_t*)keys, vals, (uint64_t*)tk, (uint32_t*)tv, n,
                                      key_bits, scr, err, st);
    if (rc == HLC_OK) rc = check_dev_err(err, st, "hlc_sort_pairs");
  }
  if (tk) cudaFreeAsync(tk, st);
  if (tv) cudaFreeAsync(tv, st);
  if (scr) cudaFreeAsync(scr, st);
  if (err) cudaFreeAsync(err, st);
  cudaStreamSynchronize(st);
  return rc;
}

int hlc_cell_table(const uint32_t* keys, uint64_t n, uint32_t* uniq, uint32_t* start,
                   uint64_t* m_out, void* stream) {
  clear_error();
  if (!m_out || (n && (!keys || !uniq || !start))) {
    set_error("NULL argument");
    return HLC_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  void* scr = nullptr;
  uint32_t* cell_of = nullptr;
  unsigned long long* m_dev = nullptr;
  int* err = nullptr;
  int rc = HLC_OK;
  if (cudaMallocAsync(&scr, scan_scratch_bytes(n) + 64, st) != cudaSuccess ||
      cudaMallocAsync(&cell_of, (n + 1) * 4, st) != cudaSuccess ||
      cudaMallocAsync(&m_dev, 64, st) != cudaSuccess ||
      cudaMallocAsync(&err, 64, st) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMallocAsync failed");
    rc = HLC_ENOMEM;
  }
  if (rc == HLC_OK) {
    cudaMemsetAsync(err, 0, 64, st);
    rc = cell_table(keys, n, 0, cell_of, uniq, start, m_dev, scr, err, st);
    unsigned long long m = 0;
    if (rc == HLC_OK) {
      cudaMemcpyAsync(&m, m_dev, 8, cudaMemcpyDeviceToHost, st);
      rc = check_dev_err(err, st, "hlc_cell_table");
    }
    if (rc == HLC_OK) *m_out = m;
  }
  if (scr) cudaFreeAsync(scr, st);
  if (cell_of) cudaFreeAsync(cell_of, st);
  if (m_dev) cudaFreeAsync(m_dev, st);
  if (err) cudaFreeAsync(err, st);
  cudaStreamSynchronize(st);
  return rc;
}

int hlc_learned_lookup(const uint32_t* uniq, uint64_t m, int shift, int model,
                       const uint32_t* queries, uint64_t nq, uint32_t* out, hlc_stats* stats,
                       void* stream) {
  clear_error();
  if (shift < 0 || shift > 24 ||
      (model != HLC_MODEL_PLA && model != HLC_MODEL_MLP && model != HLC_MODEL_NONE)) {
    set_error("shift must be in [0, 24] and model HLC_MODEL_PLA, _MLP or _NONE");
    return HLC_EINVAL;
  }
  if ((m && !uniq) || (nq && (!queries || !out))) {
    set_error("NULL array");
    return HLC_EINVAL;
  }
  HLC_TRY(ensure_device_tables());
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t last = 0;
  if (m) {
    HLC_CUDA(cudaMemcpyAsync(&last, uniq + m - 1, 4, cudaMemcpyDeviceToHost, st));
    HLC_CUDA(cudaStreamSynchronize(st));
  }
  uint64_t P = (uint64_t)(last >> shift) + 1;
  Allocator al;
  al.stream = st;
  Arena ar(al);
  int* err = ar.get_n<int>(16);
  unsigned long long* ctr = ar.get_n<unsigned long long>(8);
  if (!err || !ctr) return HLC_ENOMEM;
  HLC_CUDA(cudaMemsetAsync(err, 0, 64, st));
  HLC_CUDA(cudaMemsetAsync(ctr, 0, 64, st));
  cudaEvent_t e0, e1, e2;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventCreate(&e2);
  cudaEventRecord(e0, st);
  LearnedIndex L;
  int rc = build_learned(ar, uniq, m, shift, model, P, ctr, ctr + 1, err, st, &L);
  cudaEventRecord(e1, st);
  if (rc == HLC_OK && nq) {
    if (model == HLC_MODEL_NONE)
      k_part_bsearch_lookup<<<grid_for(nq, kThreads), kThreads, 0, st>>>(L, queries, nq, out);
    else
      k_learned_lookup<<<grid_for(nq, kThreads), kThreads, 0, st>>>(L, queries, nq, out,
                                                                     ctr + 2);
    if (cudaGetLastError() != cudaSuccess) rc = HLC_ECUDA;
  }
  cudaEventRecord(e2, st);
  unsigned long long h[8] = {0};
  uint32_t maxerr = 0;
  if (rc == HLC_OK) {
    HLC_CUDA(cudaMemsetAsync(ctr + 3, 0, 8, st));
    k_max_u32<<<grid_for(P, kThreads, 1024), kThreads, 0, st>>>(L.err, P, (uint32_t*)(ctr + 3));
    HLC_CUDA(cudaMemcpyAsync(h, ctr, sizeof(h), cudaMemcpyDeviceToHost, st));
    rc = check_dev_err(err, st, "hlc_learned_lookup");
    maxerr = (uint32_t)h[3];
  }
  if (rc == HLC_OK && stats) {
    memset(stats, 0, sizeof(*stats));
    stats->learned_models = P;
    stats->learned_max_err = maxerr;
    stats->learned_hit_rate = (nq && model != HLC_MODEL_NONE) ? (double)h[2] / (double)nq : 1.0;
    cudaEventElapsedTime(&stats->ms_index, e0, e1);
    cudaEventElapsedTime(&stats->ms_candidates, e1, e2);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  ar.release();
  cudaStreamSynchronize(st);
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner of the batched form: times candidate order targets and tile
// shapes on a sample of the caller's jobs (coordinate descent from the rule).
// ---------------------------------------------------------------------------
extern "C" int hlc_transfer_model(hlc_transfer_fit* out) {
  clear_error();
  if (!out) {
    set_error("hlc_transfer_model: out is NULL");
    return HLC_EINVAL;
  }
  int dev = 0;
  HLC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d out of range", dev);
    return HLC_EUNSUPPORTED;
  }
  hlc_transfer_fit d;
  memset(&d, 0, sizeof(d));
  TransferFit f;
  HLC_TRY(measure_transfer(&f, &d));
  {
    std::lock_guard<std::mutex> lk(g_fit_mu);
    g_fit[dev] = f;  // later streamed plans use the newest fit
  }
  *out = d;
  return HLC_OK;
}

extern "C" int hlc_autotune(const hlc_catalog* A, const hlc_catalog* B, const hlc_params* p,
                            uint32_t n_jobs, uint32_t sample_jobs, hlc_tune_report* report) {
  clear_error();
  if (!A || !B || !p || !report || n_jobs == 0 || sample_jobs == 0) {
    set_error("hlc_autotune: NULL argument, n_jobs = 0 or sample_jobs = 0");
    return HLC_EINVAL;
  }
  // the sample: jobs ordered by B size, picked at even steps of that order
  std::vector<uint32_t> ord(n_jobs);
  for (uint32_t j = 0; j < n_jobs; ++j) ord[j] = j;
  std::stable_sort(ord.begin(), ord.end(),
                   [&](uint32_t a, uint32_t b) { return B[a].n < B[b].n; });
  const uint32_t m = std::min(n_jobs, sample_jobs);
  std::vector<hlc_catalog> sa(m), sb(m);
  std::vector<hlc_params> sp(m);
  for (uint32_t k = 0; k < m; ++k) {
    const uint32_t j = ord[(uint64_t)k * n_jobs / m];
    sa[k] = A[j];
    sb[k] = B[j];
    sp[k] = p[j];
  }
  hlc_tune_report R;
  memset(&R, 0, sizeof(R));
  R.sample_jobs = m;
  // device time of one plan + match of the sample with tune t (best of reps)
  auto timed_n = [&](const hlc_tune& t, int reps, float* ms) -> int {
    for (uint32_t k = 0; k < m; ++k) sp[k].tune = &t;
    float best = 1e30f;
    for (int rep = 0; rep < reps; ++rep) {
      hlc_plan_t* P = nullptr;
      int rc = plan_batched(sa.data(), sb.data(), sp.data(), m, &P);
      if (rc != HLC_OK) return rc;
      hlc_result r;
      hlc_stats st;
      rc = hlc_match(P, &r, &st);
      hlc_free(P);
      if (rc != HLC_OK) return rc;
      best = std::min(best, st.ms_total);
    }
    *ms = best;
    return HLC_OK;
  };
  auto timed = [&](const hlc_tune& t, float* ms) -> int {
    HLC_TRY(timed_n(t, 3, ms));
    if (R.n_trials < 32) R.trials[R.n_trials++] = hlc_tune_trial{t, *ms};
    return HLC_OK;
  };
  const hlc_tune rule{kTargetPerCell, {kTileRuleKA[0], kTileRuleKA[1], kTileRuleKA[2]},
                      (uint32_t)kTileCap};
  hlc_tune cur = rule;
  float tcur = 0;
  HLC_TRY(timed(cur, &tcur));
  auto consider = [&](const hlc_tune& c) -> int {
    float t = 0;
    HLC_TRY(timed(c, &t));
    if (t < 0.97f * tcur) {
      cur = c;
      tcur = t;
    }
    return HLC_OK;
  };
  for (double T : {0.5, 1.0, 4.0, 8.0}) {
    hlc_tune c = cur;
    c.target_per_cell = T;
    HLC_TRY(consider(c));
  }
  for (int cls = 0; cls < 3; ++cls)
    for (uint32_t ka : {1u, 2u, 4u}) {
      if (ka == cur.ka[cls]) continue;
      hlc_tune c = cur;
      c.ka[cls] = ka;
      HLC_TRY(consider(c));
    }
  for (uint32_t stg : {384u, 768u, 1536u}) {
    if (stg == cur.stage) continue;
    hlc_tune c = cur;
    c.stage = stg;
    HLC_TRY(consider(c));
  }
  // the winner against the rule, interleaved, best of four each: it is kept
  // only when at least 2% faster (timing noise on a busy GPU is ~2%)
  float tr = 1e30f, tb = 1e30f;
  for (int k = 0; k < 4; ++k) {
    float a = 0, b = 0;
    HLC_TRY(timed_n(rule, 1, &a));
    HLC_TRY(timed_n(cur, 1, &b));
    tr = std::min(tr, a);
    tb = std::min(tb, b);
  }
  R.ms_rule = tr;
  if (tb < 0.98f * tr) {
    R.best = cur;
    R.ms_best = tb;
  } else {
    R.best = rule;
    R.ms_best = tr;
  }
  *report = R;
  return HLC_OK;
}

// ---------------------------------------------------------------------------
// Test hooks: shortened spin limits, and each kind of bounded device wait run
// against a flag that nothing sets, so that tests can watch a wait give up
// and the error reach the caller without faulting or hanging the GPU.
// ---------------------------------------------------------------------------
namespace hlc {

constexpr int kTestWords = 2 * rs::kRadix;  // look-back words of tiles 0 and 1

__global__ void k_test_unset_wait(int which, unsigned long long* words, int* err) {
  if (which == 0) {
    // the radix sort's look-back: tile 1 waits for tile 0's digit counts
    (void)rs::lookback_excl(words, 1, (int)threadIdx.x, err);
  } else if (which == 1) {
    // the scan's look-back (one warp): tile 1 waits for tile 0's prefix
    if (threadIdx.x < 32) (void)sc::lookback_prefix(1, 5, words, err);
  } else {
    // the tile kernel's stage wait: an mbarrier expecting one arrival
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (!mbar_wait(&bar, 0) && (threadIdx.x & 31) == 0) atomicOr(err, DERR_TIMEOUT);
  }
}

}  // namespace hlc

extern "C" int hlc_test_spin_shift(int shift) {
  clear_error();
  if (shift < 0 || shift > 24) {
    set_error("hlc_test_spin_shift: shift must lie in [0, 24]");
    return HLC_EINVAL;
  }
  HLC_CUDA(cudaMemcpyToSymbol(d_spin_shift, &shift, sizeof(int)));
  return HLC_OK;
}

extern "C" int hlc_test_unset_wait(int which, void* stream) {
  clear_error();
  if (which < 0 || which > 2) {
    set_error("hlc_test_unset_wait: which must be 0, 1 or 2");
    return HLC_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* words = nullptr;
  int* err = nullptr;
  if (cudaMallocAsync(&words, kTestWords * 8, st) != cudaSuccess ||
      cudaMallocAsync(&err, 64, st) != cudaSuccess) {
    cudaGetLastError();
    if (words) cudaFreeAsync(words, st);
    set_error("hlc_test_unset_wait: cudaMallocAsync failed");
    return HLC_ENOMEM;
  }
  int rc = HLC_OK;
  if (cudaMemsetAsync(words, 0, kTestWords * 8, st) != cudaSuccess ||
      cudaMemsetAsync(err, 0, 64, st) != cudaSuccess) {
    set_error("hlc_test_unset_wait: %s", cudaGetErrorString(cudaGetLastError()));
    rc = HLC_ECUDA;
  }
  if (rc == HLC_OK) {
    k_test_unset_wait<<<1, rs::kRadix, 0, st>>>(which, words, err);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (cudaGetLastError() != cudaSuccess) {
      set_error("hlc_test_unset_wait: launch failed");
      rc = HLC_ECUDA;
    }
  }
  if (rc == HLC_OK) rc = check_dev_err(err, st, "hlc_test_unset_wait");
  cudaFreeAsync(words, st);
  cudaFreeAsync(err, st);
  cudaStreamSynchronize(st);
  return rc;
}

// ---------------------------------------------------------------------------
// Allocation-free radix sort: the same sort as hlc_sort_pairs, with every
// temporary (alternate key/value buffers, histograms, look-back words and the
// error word) carved out of one fixed device array compiled into the library.
// ---------------------------------------------------------------------------
namespace hlc {

constexpr uint64_t kNoAllocMaxN = 1ull << 20;  // elements per call
constexpr size_t kNoAllocKeyBytes = kNoAllocMaxN * 8;
constexpr size_t kNoAllocValBytes = kNoAllocMaxN * 4;
constexpr size_t kNoAllocSortBytes =
    kSortLookbackOffset +
    8ull * ((kNoAllocMaxN + rs::kTile - 1) / rs::kTile) * rs::kRadix * 8;
constexpr size_t kNoAllocBytes = 256 + kNoAllocKeyBytes + kNoAllocValBytes + kNoAllocSortBytes;

// Lives on every device that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the scratch array on the current device.  Looked up on
// every call (the lookup allocates nothing): after a device reset the module
// is loaded again and the array may sit at another address.
static int noalloc_scratch(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    set_error("cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
    return HLC_ECUDA;
  }
  *out = p;
  return HLC_OK;
}

}  // namespace hlc

extern "C" int hlc_sort_pairs_noalloc(void* keys, uint32_t* vals, uint64_t n, int key_size,
                                      int key_bits, void* stream) {
  clear_error();
  if ((key_size != 4 && key_size != 8) || key_bits < 1 || key_bits > 8 * key_size) {
    set_error("key_size must be 4 or 8 and key_bits in [1, 8*key_size]");
    return HLC_EINVAL;
  }
  if (n > kNoAllocMaxN) {
    set_error("hlc_sort_pairs_noalloc: n = %llu exceeds the fixed scratch capacity of %llu "
              "elements; use hlc_sort_pairs",
              (unsigned long long)n, (unsigned long long)kNoAllocMaxN);
    return HLC_EINVAL;
  }
  if (n <= 1) return HLC_OK;
  if (!keys || !vals) {
    set_error("NULL array");
    return HLC_EINVAL;
  }
  void* base = nullptr;
  HLC_TRY(noalloc_scratch(&base));
  cudaStream_t st = (cudaStream_t)stream;
  char* b = (char*)base;
  int* err = (int*)b;  // first 256 bytes: the device error word
  void* tk = b + 256;
  uint32_t* tv = (uint32_t*)(b + 256 + kNoAllocKeyBytes);
  void* scr = b + 256 + kNoAllocKeyBytes + kNoAllocValBytes;
  int rc = HLC_OK;
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) {
    set_error("hlc_sort_pairs_noalloc: %s", cudaGetErrorString(cudaGetLastError()));
    rc = HLC_ECUDA;
  }
  if (rc == HLC_OK && key_size == 4)
    rc = radix_sort_pairs<uint32_t>((uint32_t*)keys, vals, (uint32_t*)tk, tv, n, key_bits, scr,
                                    err, st);
  else if (rc == HLC_OK)
    rc = radix_sort_pairs<uint64_t>((uint64_t*)keys, vals, (uint64_t*)tk, tv, n, key_bits, scr,
                                    err, st);
  if (rc == HLC_OK) rc = check_dev_err(err, st, "hlc_sort_pairs_noalloc");
  // On every path, success or not, no queued kernel may still be using the
  // shared array when the call returns.
  cudaStreamSynchronize(st);
  return rc;
}
