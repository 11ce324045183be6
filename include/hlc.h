/*
 * hlc.h -- C ABI of the B300 (sm_103a) positional cross-match library.
 *
 * The library computes the hot path of HLC2 (Zhang et al., arXiv 2301.07331):
 * for two sky catalogues A and B, every pair (A_i, B_j) whose angular
 * separation d (Sec. 2.1, Eq. 1) is at most a radius r.  Sources are grouped
 * by HEALPix nested cell ("hp_nestid", Sec. 4.2) and only pairs in the same or
 * neighbouring cells are tested.  Two boundary rules are offered:
 *   HLC_COMPLETE8 -- the cell of each A source and its 8 (7 at the eight
 *                    three-face vertices) neighbours: the exact set of Eq. 1
 *                    whenever r <= theta_L / 8, theta_L = sqrt(pi/3) / 2^L;
 *   HLC_QUAD      -- the quad-direction strategy of Sec. 3.2, Algorithm 1:
 *                    each source is also filed under the cells of its four
 *                    copies shifted by +-r in RA and Dec, and only pairs that
 *                    share a cell are tested (an approximation, a subset of
 *                    the exact set; each pair is reported once, from the
 *                    smallest cell the two sources share).
 *
 * The radius is one r for every pair, or with HLC_RADIUS_EQ4 the paper's
 * criterion of Eq. 4 with per-source error radii: r_ij = 3 sqrt(e_i^2 +
 * e_j^2), evaluated as a = e_i e_i, b = e_j e_j, t = a + b, r = 3 sqrt(t)
 * (each step a correctly rounded binary64 operation; symmetric in i, j).
 *
 * Decision arithmetic.  A pair matches when its squared chord
 * |u_A - u_B|^2 <= 4 sin^2(r/2) (Eq. 1 in chord form), both sides evaluated
 * in a fixed sequence of IEEE binary64 operations: sin/cos in degrees by exact
 * reduction to [-45, 45] deg and Horner polynomials with the Taylor
 * coefficients (pi/180)^k/k! rounded to double; u = (cos d cos a,
 * cos d sin a, sin d); s = dx*dx, s = fma(dy,dy,s), s = fma(dz,dz,s).  With
 * HLC_FP32_GUARD the bulk test runs in FP32 with a guard band derived from
 * its error bound and only candidates inside the band are decided in that
 * binary64 arithmetic, so both precisions return the same set.
 *
 * Conventions for every entry point:
 *   - return value: HLC_OK (0) or an HLC_E* code; hlc_last_error() then holds
 *     a message (thread-local, valid until the next call on that thread);
 *   - on error nothing is written to the caller's result structures;
 *   - "device" pointers are CUDA global-memory addresses on the current
 *     device; "stream" is a cudaStream_t (NULL = legacy default stream);
 *   - RA/Dec are float64 degrees; RA is folded into [0, 360); Dec must lie in
 *     [-90, 90]; NaN or Inf anywhere is HLC_EINVAL.
 */
#ifndef HLC_H
#define HLC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define HLC_OK 0
#define HLC_EINVAL 1       /* invalid argument or input value */
#define HLC_ENOMEM 2       /* device or pinned host allocation failed */
#define HLC_ECUDA 3        /* a CUDA runtime call or kernel failed */
#define HLC_ETIMEOUT 4     /* a bounded device-side wait gave up */
#define HLC_EUNSUPPORTED 5 /* valid request the library does not implement */

/* ---- enums -------------------------------------------------------------- */
#define HLC_COMPLETE8 0
#define HLC_QUAD 1
#define HLC_QUAD_COSDEC 2 /* Algorithm 1 with the RA error radius read as an
                             angle on the sky: the RA copies are shifted by
                             R / cos(dec) (canonical cosine, at most 180 deg)
                             instead of R; Dec copies by R as in HLC_QUAD */

#define HLC_FP64 0       /* plain form: binary64 vectors and pair test */
#define HLC_FP32_GUARD 1 /* FP32 bulk test + guard band + binary64 recheck */

#define HLC_INDEX_BSEARCH 0 /* cell offsets by binary search of unique keys */
#define HLC_INDEX_LEARNED 1 /* per-partition learned model + bounded search */

#define HLC_RADIUS_FIXED 0 /* one radius r = radius_arcsec for every pair */
#define HLC_RADIUS_EQ4 1   /* per-source error radii (Sec. 2.1, Eq. 4): pair
                              (A_i, B_j) matches when its separation is at
                              most r_ij = 3 sqrt(e_i^2 + e_j^2), e from the
                              catalogues' err_arcsec columns */

#define HLC_MODEL_PLA 0 /* 256-segment monotone piecewise-linear model */
#define HLC_MODEL_MLP 1 /* 1-input 2x32 ReLU MLP, bracket-checked */
#define HLC_MODEL_NONE 2 /* hlc_learned_lookup only: no model, binary search
                            inside the partition (the baseline it replaces) */

/* ---- catalogue and parameters ------------------------------------------- */
typedef struct {
  const double* ra_deg;  /* n values */
  const double* dec_deg; /* n values */
  const uint64_t* id;    /* n user ids (need not be unique) */
  uint64_t n;            /* number of sources, < 2^31 */
  int on_device;         /* 1: the arrays are device pointers;
                            0: host pointers (pinned or pageable) */
  const double* err_arcsec; /* n per-source position error radii in arcsec
                               (finite, >= 0), read with HLC_RADIUS_EQ4 only;
                               may be NULL otherwise.  Same memory space as
                               the other arrays. */
} hlc_catalog;

/* Shape of the batched form's work (form 2): the order each job is matched
 * at and the tile kernel's tiles for dense cells.  The library's rule is
 * {2.0, {2, 4, 4}, 1536}; hlc_autotune times alternatives on a sample of the
 * caller's own jobs and returns the fastest it found. */
typedef struct {
  double target_per_cell;   /* batched jobs with fine_level < 0: the order is
                               the one leaving about this many B sources per
                               cell (capped by r <= theta_L/8); > 0 */
  uint32_t ka[3];           /* tile kernel: A sources per lane (1, 2 or 4)
                               for dense A cells of 33-64, 65-256 and more
                               than 256 sources (cells of 32 use 1) */
  uint32_t stage;           /* tile kernel: B vectors per staged round, a
                               multiple of 8 in [8, 1536] */
} hlc_tune;

/* One timed candidate of hlc_autotune. */
typedef struct {
  hlc_tune tune;
  float ms;                 /* device time of hlc_plan + hlc_match on the
                               sample (best of two runs) */
} hlc_tune_trial;

typedef struct {
  hlc_tune best;            /* the fastest candidate */
  float ms_rule, ms_best;   /* the rule's and the best candidate's time */
  uint32_t sample_jobs;     /* jobs in the calibration sample */
  uint32_t n_trials;        /* entries of trials[] used */
  hlc_tune_trial trials[32];
} hlc_tune_report;

typedef void* (*hlc_alloc_fn)(size_t bytes, void* ctx);
typedef void (*hlc_dealloc_fn)(void* ptr, void* ctx);

typedef struct {
  double radius_arcsec;       /* r > 0; COMPLETE8 needs r <= theta_L/8
                                 (HLC_RADIUS_FIXED) */
  int coarse_level;           /* HEALPix order of streaming / learned-index
                                 partitions, 0 <= coarse <= fine */
  int fine_level;             /* HEALPix order L of the cells, 0..14 */
  int boundary;               /* HLC_COMPLETE8, HLC_QUAD or HLC_QUAD_COSDEC */
  int precision;              /* HLC_FP64 or HLC_FP32_GUARD */
  int index;                  /* HLC_INDEX_BSEARCH or HLC_INDEX_LEARNED */
  int model;                  /* HLC_MODEL_PLA or HLC_MODEL_MLP (learned) */
  int want_sep;               /* 1: fill hlc_result.sep_arcsec */
  uint64_t device_mem_budget; /* 0 = no cap; else bytes of device memory the
                                 plan may hold at once (host inputs are then
                                 streamed by coarse partition) */
  void* stream;               /* cudaStream_t for all work; NULL = default */
  hlc_alloc_fn alloc;         /* optional device allocator (NULL: the
                                 library uses cudaMallocAsync on stream) */
  hlc_dealloc_fn dealloc;
  void* alloc_ctx;
  const hlc_tune* tune;       /* NULL: the library's rule; else the order
                                 target and tile shape to use (batched plans:
                                 the same pointer for every job) */
  int radius_rule;            /* HLC_RADIUS_FIXED (radius_arcsec) or
                                 HLC_RADIUS_EQ4 (per-pair radius from the
                                 catalogues' err_arcsec; radius_arcsec is then
                                 ignored).  EQ4 is implemented for single,
                                 in-core plans in complete mode with the
                                 binary-searched index, in both precisions
                                 (HLC_EUNSUPPORTED otherwise), and needs the
                                 largest pair radius 3 sqrt(max e_A^2 +
                                 max e_B^2) <= theta_L/8 (HLC_EINVAL above). */
} hlc_params;

/* Result of hlc_match: rows sorted ascending by (id_a, id_b) as unsigned
 * 64-bit values (by job first for batched plans).  The arrays belong to the
 * plan and stay valid until hlc_free or the next hlc_match on that plan. */
typedef struct {
  uint64_t n;          /* number of matched pairs */
  uint64_t* id_a;      /* n ids from catalogue A */
  uint64_t* id_b;      /* n ids from catalogue B */
  double* sep_arcsec;  /* n separations (NULL unless want_sep) */
  uint32_t* job;       /* n job indices (batched plans), else NULL */
  int on_device;       /* 1: device arrays */
} hlc_result;

/* Counters and CUDA-event timings of the last hlc_plan + hlc_match. */
typedef struct {
  uint64_t n_a, n_b;               /* sources */
  uint64_t entries_a, entries_b;   /* index entries (> n in quad mode) */
  uint64_t cells_a;                /* distinct A cells at the join level (0 in the
                                      FP32 complete form, whose A entries are
                                      grouped by offset-table cell only) */
  uint64_t cells_b;                /* non-empty cells of B's offset table (distinct
                                      B cells with the learned index) */
  uint64_t pair_tests;             /* pair tests executed (sparse regions are
                                      joined over whole table cells, a superset) */
  uint64_t band_candidates;        /* FP32 guard band: pairs rechecked */
  uint64_t matches;
  uint64_t quad_duplicates;        /* quad pairs left to a smaller shared
                                      cell */
  uint64_t partitions;             /* streamed coarse partitions */
  uint64_t learned_models;         /* learned-index partitions */
  double learned_hit_rate;         /* lookups answered inside the window */
  uint32_t learned_max_err;        /* largest stored error bound */
  int join_level;                  /* HEALPix order used for the join */
  float ms_prep, ms_sort, ms_index, ms_candidates, ms_pair, ms_recheck,
      ms_output, ms_h2d, ms_d2h, ms_total;
                                   /* stage times, summed over both catalogues
                                      (in the FP32 complete form with device
                                      inputs the two catalogues are built at
                                      once, so their stage times overlap);
                                      ms_total is the plan's and the match's
                                      own span */
  uint64_t kernel_launches;        /* library kernels launched by the plan and
                                      the match */
  uint64_t dense_entries_b;        /* FP32 complete form: B entries in dense
                                      offset-table cells (kept in fine order) */
  uint64_t tile_items;             /* dense A cells given to the tile kernel */
  uint64_t tile_entries_a;         /* A entries in those cells */
  float ms_stream_count;           /* streamed plans (host wall time): counting pass, */
  float ms_stream_bucket;          /*   bucketing pass into pinned host runs, */
  float ms_stream_groups;          /*   the groups' copies in, matches and rows out, */
  float ms_stream_merge;           /*   merge of the groups' sorted rows */
  float ms_sort_passes;            /* FP32 complete form: the radix sort's digit
                                      passes alone (both catalogues) */
  uint32_t sort_passes;            /*   and how many passes that was */
  uint64_t band_fp64;              /* FP32 forms: guard-band candidates the
                                      float-float separation left undecided,
                                      finished by the binary64 test */
  uint64_t sort_entries;           /* FP32 complete form: entries moved by the
                                      timed digit passes, summed over the
                                      launches (with device inputs one launch
                                      per pass sorts both catalogues) */
  float ms_plan_span;              /* hlc_plan's own span on the plan stream
                                      (ms_total = ms_plan_span + ms_candidates
                                      + ms_pair + ms_recheck + ms_output for
                                      single plans: consecutive intervals) */
  uint64_t h2d_bytes, h2d_copies;  /* streamed plans: host-to-device copies issued */
  uint64_t d2h_bytes, d2h_copies;  /*   and device-to-host copies */
  float ms_model_h2d, ms_model_d2h;/*   their time by the transfer model of Eq. 5,
                                      the sum over copies of alpha + beta d with
                                      the device's measured fit (hlc_transfer_model) */
  uint64_t stream_chunk;           /*   sources per streamed chunk (from the fit) */
  float ms_tile;                   /* FP32 complete form: the dense-cell pair
                                      kernel alone (inside ms_pair) */
  uint64_t tile_tests;             /*   and the pair tests it ran */
  float ms_plan_presort;           /* FP32 complete form with device inputs:
                                      from the plan's start to the first digit
                                      pass (both preps, side by side); else 0 */
  uint64_t sort_bytes;             /* FP32 complete form: algorithmic bytes of
                                      the timed digit passes, summed over the
                                      launches (a 4-byte key and a 4-byte value
                                      read and written per entry and pass; the
                                      one-sort form's first pass makes its
                                      values and reads 12 bytes) */
} hlc_stats;

typedef struct hlc_plan_s hlc_plan_t;

/* Build a plan: validate and index both catalogues (ang2pix, cell sort,
 * offset table).  n_jobs = 1 for one pair of catalogues; n_jobs > 1 makes A,
 * B and p arrays of n_jobs entries that are matched independently in one
 * batched launch sequence (every job must use the same precision, boundary
 * and stream; radius and levels may differ).  The caller's input arrays must
 * stay valid until hlc_plan returns; nothing is retained.  *out is set only
 * on success. */
int hlc_plan(const hlc_catalog* A, const hlc_catalog* B, const hlc_params* p,
             uint32_t n_jobs, hlc_plan_t** out);

/* Run the match.  out receives device arrays owned by the plan; stats may be
 * NULL.  Synchronises the plan's stream before returning. */
int hlc_match(hlc_plan_t* plan, hlc_result* out, hlc_stats* stats);

/* Copy a result to caller-owned host arrays (each may be NULL to skip) and
 * wait for the copies.  They run on the calling thread's own default stream
 * (cudaStreamPerThread), so plans matched on other threads' streams are not
 * held up.  Errors: HLC_EINVAL for a NULL result, HLC_ECUDA for a failed copy. */
int hlc_result_to_host(const hlc_result* r, uint64_t* id_a, uint64_t* id_b,
                       double* sep_arcsec, uint32_t* job);

/* The same copies, enqueued on `stream` (a cudaStream_t; NULL = the legacy
 * default stream) and not waited for: the host arrays may be read once the
 * stream has reached them (cudaStreamSynchronize, or hlc_free of the plan
 * when `stream` is the plan's stream, which synchronises it).  Page-locked
 * host arrays let the copies overlap other work on the link and the GPU;
 * with pageable ones the call returns only after the copies.  The plan must
 * not be freed on another stream before the copies are done.  Errors:
 * HLC_EINVAL for a NULL result, HLC_ECUDA when a copy cannot be enqueued. */
int hlc_result_to_host_async(const hlc_result* r, uint64_t* id_a, uint64_t* id_b,
                             double* sep_arcsec, uint32_t* job, void* stream);

/* Release the plan, its device memory and every result it returned. */
void hlc_free(hlc_plan_t* plan);

/* Message of the last failed call on this thread ("" if none). */
const char* hlc_last_error(void);

/* Library version string. */
const char* hlc_version(void);

/* sizeof of the public structs, for bindings to check their layouts against:
 * out[0..7] = hlc_catalog, hlc_tune, hlc_tune_trial, hlc_tune_report,
 * hlc_params, hlc_result, hlc_stats, hlc_transfer_fit.  Writes min(n, 8)
 * entries and returns 8 (the number of structs); out may be NULL when n is 0.
 * Host only; never fails. */
int hlc_abi_sizes(size_t* out, int n);

/* The binary64 polynomial coefficients this library uses for sin/cos in
 * degrees: sin_c[k] = (-1)^k (pi/180)^(2k+1)/(2k+1)! and
 * cos_c[k] = (-1)^k (pi/180)^(2k)/(2k)!, each the nearest double, derived at
 * load time in binary128 (host only; no device needed). */
int hlc_canonical_coefficients(double sin_c[10], double cos_c[11]);

/* ---- kernel-level entry points (device pointers, asynchronous on stream) --
 * These expose single steps of the path for testing and for callers that
 * build their own pipelines. */

/* HEALPix nested pixel of each (ra, dec) at `order` (0..14), computed in the
 * binary64 arithmetic stated above (Sec. 4.2, after Gorski et al. 2005).
 * ra, dec: n device doubles; pix: n device uint32.  precision HLC_FP32_GUARD
 * computes the same pixels through an FP32 estimate with an exact binary64
 * fallback near cell edges. */
int hlc_ang2pix(const double* ra, const double* dec, uint64_t n, int order,
                int precision, uint32_t* pix, void* stream);

/* The 8 neighbours of each nested pixel in the direction order
 * (dx,dy) = (-1,-1) (-1,0) (-1,1) (0,1) (1,1) (1,0) (1,-1) (0,-1), where x
 * grows to the north-east and y to the north-west inside a base face; a
 * missing neighbour (three-face vertices) is -1.  pix: n device uint32;
 * out: 8n device int64. */
int hlc_neighbours(const uint32_t* pix, uint64_t n, int order, int64_t* out,
                   void* stream);

/* Quad-direction cell set of each source (Algorithm 1): the distinct pixels
 * of (ra, dec), (ra +- R_A, dec), (ra, dec -+ R), R = r/3600 deg, R_A = R
 * (boundary HLC_QUAD) or R / cos(dec) capped at 180 (HLC_QUAD_COSDEC), RA
 * wrapped, Dec clamped, ascending.  out: 5n device uint32 padded with
 * 0xFFFFFFFF; count: n device int32.  precision HLC_FP32_GUARD computes the
 * same sets through the FP32 pixel estimate (the shifted coordinates in
 * float-float), each undecided position in binary64.  Returns HLC_EINVAL for
 * a bad order, radius, precision or boundary, or for non-finite RA/Dec or
 * |Dec| > 90. */
int hlc_quad_cells(const double* ra, const double* dec, uint64_t n,
                   double radius_arcsec, int order, int precision, int boundary,
                   uint32_t* out, int32_t* count, void* stream);

/* Unit vectors (3n device doubles, interleaved x,y,z) in the binary64
 * arithmetic stated above. */
int hlc_unitvec(const double* ra, const double* dec, uint64_t n, double* xyz,
                void* stream);

/* Stable ascending LSD radix sort of (key, value) pairs by the low `key_bits`
 * bits of the keys.  keys/vals: n device elements, sorted in place.  key_size
 * is 4 (uint32 keys) or 8 (uint64 keys); values are uint32.  Allocates
 * temporary device memory of about n (key_size + 4) bytes plus the look-back
 * tables with cudaMallocAsync on the stream, and frees it before returning;
 * synchronises the stream. */
int hlc_sort_pairs(void* keys, uint32_t* vals, uint64_t n, int key_size,
                   int key_bits, void* stream);

/* Allocation-free variant of hlc_sort_pairs (the paper has no counterpart;
 * this is a service for callers).  Some callers must not allocate device
 * memory on the call path: a host application that reserves all device
 * memory up front for its own allocator, or a latency-critical loop in which
 * a cudaMalloc/cudaFree (which can synchronise the device) is not acceptable.
 * This entry point performs the same stable sort, with the same arguments
 * and results, but takes every temporary buffer from one fixed device array
 * built into the library (about 16 MB, present on every device that loads
 * the library until the process exits) and never allocates or frees memory.
 *   - n is limited to 1,048,576 elements; larger n returns HLC_EINVAL with a
 *     message naming the limit (use hlc_sort_pairs instead);
 *   - every call looks up the array's address on the current device (no
 *     address is cached, so a device reset that reloads the library's module
 *     is handled); the first call on a device may load that module, so make
 *     the first call on each device before any stream capture;
 *   - all calls share the one array: calls that overlap on the GPU (other
 *     streams, other host threads) race and corrupt each other's results;
 *     the array keeps the last call's contents, and each call clears what
 *     must start at zero;
 *   - synchronises the stream before returning, on success and on every
 *     error after the array's address was taken. */
int hlc_sort_pairs_noalloc(void* keys, uint32_t* vals, uint64_t n, int key_size,
                           int key_bits, void* stream);

/* Transfer-cost model of Sec. 4.1.1, Eq. 5: a copy of d bytes between host
 * and device takes T(d) = alpha + beta d.  Measured on the current device
 * the paper's way: alpha is the time of a one-byte copy, beta = (t_s - alpha)
 * / s from the time t_s of an s = 256 MiB copy (pinned host memory, medians
 * of 21 and 5 copies, CUDA events on a stream of its own).  Four more sizes
 * are timed to check the line.  Streamed plans use the same fit, measured
 * once per device and kept: their chunk is the smallest number of sources
 * (a multiple of 2^20, at most 8 Mi) whose copy spends at most 1% of its time
 * in alpha, and hlc_stats reports their copies' predicted time beside the
 * measured one.  Allocates 256 MiB of pinned host and device memory for the
 * duration of the call and synchronises. */
typedef struct {
  double alpha_s[2];          /* [0] host to device, [1] device to host */
  double beta_s_per_byte[2];
  double gbs[2];              /* 1 / beta, GB/s */
  uint64_t check_bytes[4];    /* the sizes timed to check the line */
  double check_measured_s[2][4];
  double check_model_s[2][4];
} hlc_transfer_fit;

int hlc_transfer_model(hlc_transfer_fit* out);

/* Autotuner of the batched form (form 2; the paper's counterpart is the
 * blockDim sweep of Sec. 5.2, Fig. 8).  Takes the same arguments as a
 * batched hlc_plan (A, B, p: arrays of n_jobs) and times, on a sample of at
 * most sample_jobs of those jobs spread over their B sizes, the rule and
 * candidates changed one at a time (coordinate descent): the order target
 * in {0.5, 1, 2, 4, 8} B sources per cell, then KA in {1, 2, 4} for each
 * density class of dense A cells, then the staged round in {384, 768, 1536}
 * B vectors; a change is kept when it is at least 3% faster.  Each
 * candidate is a full batched plan + match of the sample (device time, best
 * of three).  Last, the winner and the rule are timed in turn (best of four
 * each) and the winner is reported only if it is at least 2% faster, else
 * the rule.  report->best can be passed as hlc_params.tune.  The jobs' own
 * fine_level and p[].tune are ignored for the ordering rule's trials only
 * where fine_level >= 0 (those jobs keep their order).  Synchronises the
 * stream; allocates like hlc_plan. */
int hlc_autotune(const hlc_catalog* A, const hlc_catalog* B, const hlc_params* p,
                 uint32_t n_jobs, uint32_t sample_jobs, hlc_tune_report* report);

/* ---- test hooks (no counterpart in the paper) -----------------------------
 * Every device-side wait of the library (the radix sort's and the scans'
 * look-back on a predecessor tile, the tile kernel's mbarrier waits) polls at
 * most a fixed number of times, then records HLC_ETIMEOUT and returns.  These
 * two calls let a test watch that happen without hanging or faulting a GPU. */

/* Shift every wait's poll limit right by `shift` (0..24) on the current
 * device; 0 restores the production limits.  Affects every later launch on
 * that device until changed again.  HLC_EINVAL outside 0..24. */
int hlc_test_spin_shift(int shift);

/* Run one of the library's bounded waits against a flag that nothing sets:
 * which = 0 the radix sort's look-back, 1 the scans' look-back, 2 the tile
 * kernel's mbarrier wait.  The kernel gives up after its (shifted) limit and
 * the call returns HLC_ETIMEOUT; the context stays usable.  Allocates a few
 * KB with cudaMallocAsync on the stream and synchronises it. */
int hlc_test_unset_wait(int which, void* stream);

/* Run-length table of sorted uint32 keys: unique keys uniq[0..m) and
 * start[0..m] (start[m] = n); *m_out receives m (host).  uniq and start must
 * hold n and n+1 elements.  Synchronises the stream. */
int hlc_cell_table(const uint32_t* keys, uint64_t n, uint32_t* uniq,
                   uint32_t* start, uint64_t* m_out, void* stream);

/* Learned offset index over sorted unique keys uniq[0..m) partitioned by the
 * top bits (key >> shift): per partition a model (HLC_MODEL_PLA or
 * HLC_MODEL_MLP) with a stored max error; lookup(q) returns the lower bound
 * of q in uniq exactly (bounded search in the predicted window, binary search
 * as fallback).  HLC_MODEL_NONE builds the partition offsets only and binary
 * searches the query's partition (the plain offset table, for comparison).
 * out: nq device uint32 lower-bound positions; stats may be NULL
 * (learned_hit_rate, learned_max_err, ms_index = build, ms_candidates =
 * lookups).  Synchronises the stream. */
int hlc_learned_lookup(const uint32_t* uniq, uint64_t m, int shift, int model,
                       const uint32_t* queries, uint64_t nq, uint32_t* out,
                       hlc_stats* stats, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HLC_H */
