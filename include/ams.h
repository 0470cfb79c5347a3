/*
 * ams.h -- C ABI of libams: adaptive multi-level sample sort (AMS-sort) on one GPU.
 *
 * Method: Axtmann, Bingmann, Sanders, Schulz, "Practical Massively Parallel
 * Sorting", SPAA 2015.  Problem statement: Section 1 (sort n elements; the output
 * is a sorted permutation of the input).  Tie breaking: Section 2 and Appendix D
 * (elements are ordered by (key, original position), which makes every key unique;
 * the result is therefore the stable order).  Algorithm: Section 6 (random sample,
 * sample sorted with the fast work-inefficient sort of Section 4.2, b*r-1 splitters
 * of equidistant rank, partition into b*r buckets plus equality buckets, global
 * bucket sizes, grouping of consecutive buckets with the scanning algorithm and its
 * optimal bound, delivery, recursion, sequential base case).
 *
 * Conventions shared by every call:
 *  - Pointers named d_* are device pointers (CUDA global memory of the current
 *    device); pointers named h_* are host pointers.  The caller owns every buffer it
 *    passes; the library owns its scratch memory (held by a context, see below).
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default stream.
 *    Device calls are stream ordered and asynchronous: they return once the work is
 *    enqueued.  Errors found on the host (bad arguments, allocation failure, launch
 *    failure) are returned at once.  Errors found on the device (a table capacity
 *    exceeded) are latched in the context and returned by ams_context_sync().
 *  - Keys: AMS_U32 (uint32_t), AMS_U64 (uint64_t), AMS_F32 (float, ordered through
 *    the order-preserving bit map: negative values have all bits flipped, others get
 *    the sign bit set; hence -0.0 sorts before +0.0, NaNs with the sign bit set sort
 *    first and the others last; output keys keep their input bit patterns).
 *  - Payloads (pairs) are uint64_t and move with their key.
 *  - The output is the unique permutation ordered by (key, original index).  It
 *    does not depend on `seed`, `levels`, `buckets_per_level` or the options; those
 *    only change the intermediate steps (sample, splitters, groups).
 *  - n must be below 2^32.  levels is in [1, 8]; buckets_per_level has `levels`
 *    host entries r_l >= 2 (groups per level); b * r_l (range buckets per level) must
 *    lie in [2, 2048].  More levels than requested are added when n / prod(r_l)
 *    still exceeds the base-case capacity (at most 8 levels in total).
 *  - The library never aborts, traps or prints.
 */
#ifndef AMS_H
#define AMS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define AMS_API __attribute__((visibility("default")))
#else
#define AMS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { AMS_U32 = 0, AMS_U64 = 1, AMS_F32 = 2 } ams_key_type;

typedef enum {
  AMS_OK = 0,
  AMS_ERR_INVALID = 1,      /* bad argument (null pointer, sizes, parameters) */
  AMS_ERR_OOM = 2,          /* device or pinned-host allocation failed */
  AMS_ERR_CUDA = 3,         /* a CUDA runtime call failed */
  AMS_ERR_TIMEOUT = 4,      /* a bounded device wait gave up */
  AMS_ERR_UNSUPPORTED = 5,  /* valid request outside this build's limits */
  AMS_ERR_INTERNAL = 6      /* a device table overflowed (result not valid) */
} ams_status;

/* Tuning knobs; pass NULL for all defaults.  Zero in a field selects its default. */
typedef struct ams_options {
  uint32_t oversample_a;    /* a: 0 = per segment, ceil(1.6*log10(n_g)) (Section 7.2) */
  uint32_t overpartition_b; /* b: 0 = 1 for levels == 1, else 4 (Section 6) */
  uint32_t basecase_cap;    /* C: largest group sorted in shared memory;
                               0 = 16384 for 32-bit keys, 8192 otherwise and for pairs,
                               except a sort of one segment of more than that many keys
                               whose planned leaves (n over the product of the r's,
                               plus 25%) fit half of it: pairs then use 4096, 32-bit
                               keys 8192.  Pairs with C <= 4096 use a base case that
                               fits two blocks per SM, 32-bit keys with C <= 8192 one
                               that holds half as many keys per thread. */
  uint32_t flags;           /* AMS_FLAG_* */
} ams_options;

#define AMS_FLAG_PHASE_TIMERS 0x1u  /* record CUDA events per kernel (see ams_stats) */
#define AMS_FLAG_TREE_CLASSIFIER 0x2u  /* classify by descending the implicit splitter
                                          tree (Section 2.2 multisplitter) instead of the
                                          default cell table; same bucket ids */
#define AMS_FLAG_GRAPH 0x4u  /* keys-only sorts of one array (n >= 2): replay a CUDA
                                graph per size class instead of launching every kernel.
                                The context pads the request to its class size (the next
                                power of two, at least 1024) with keys that order after
                                every key, captures the class's launch sequence once on
                                buffers of its own, and per call only updates the copy
                                in, the pad fill and the copy out.  Same result; the
                                context keeps 2 x class size keys per class in use, and
                                a graph is rebuilt when its scratch had to move.  The
                                first call of a class captures (no stream may be
                                capturing then). */

/* --------------------------------------------------------------- whole sorts */

/* Sort n keys in place (Section 1 output; Section 6 method). */
AMS_API ams_status ams_sort_keys(void* d_keys, uint64_t n, ams_key_type kt, int levels,
                         const uint32_t* buckets_per_level, uint64_t seed,
                         const ams_options* opt, void* stream);

/* Sort n (key, payload) pairs in place; payload i moves with key i. */
AMS_API ams_status ams_sort_pairs(void* d_keys, uint64_t* d_vals, uint64_t n, ams_key_type kt,
                          int levels, const uint32_t* buckets_per_level, uint64_t seed,
                          const ams_options* opt, void* stream);

/* Sort every segment [d_offsets[s], d_offsets[s+1]) independently, in place.
 * d_offsets: device array of nseg+1 non-decreasing offsets with d_offsets[0] = 0
 * and d_offsets[nseg] = n (the caller guarantees this; it is not checked).
 * d_vals may be NULL (keys only). */
AMS_API ams_status ams_sort_segmented(void* d_keys, uint64_t* d_vals, const uint64_t* d_offsets,
                              uint64_t nseg, uint64_t n, ams_key_type kt, int levels,
                              const uint32_t* buckets_per_level, uint64_t seed,
                              const ams_options* opt, void* stream);

/* Out-of-place forms: read d_in (not modified), write d_out (n elements).  d_in may
 * equal d_out.  d_vals_in / d_vals_out may be NULL together (keys only). */
AMS_API ams_status ams_sort_keys_into(const void* d_in, void* d_out, uint64_t n, ams_key_type kt,
                              int levels, const uint32_t* buckets_per_level, uint64_t seed,
                              const ams_options* opt, void* stream);
AMS_API ams_status ams_sort_pairs_into(const void* d_keys_in, void* d_keys_out,
                               const uint64_t* d_vals_in, uint64_t* d_vals_out, uint64_t n,
                               ams_key_type kt, int levels, const uint32_t* buckets_per_level,
                               uint64_t seed, const ams_options* opt, void* stream);

/* Host-buffer form: copies h_keys (and h_vals if not NULL) to the device, sorts and
 * copies the result back into the same host arrays.  Synchronous: returns after the
 * result is in host memory (device errors included).  Pinned host memory makes the
 * copies faster but is not required. */
AMS_API ams_status ams_sort_host(void* h_keys, uint64_t* h_vals, uint64_t n, ams_key_type kt,
                         int levels, const uint32_t* buckets_per_level, uint64_t seed,
                         const ams_options* opt, void* stream);
/* Asynchronous host-buffer form on a context (ctx NULL = default context): enqueues on
 * `stream` the copy of h_keys (and h_vals) into the context's device staging buffer,
 * the sort, and the copy of the result back into the same host arrays, and returns
 * once that work is enqueued.  With page-locked host arrays the copies overlap other
 * streams' work, so sorts on two contexts and two streams keep both directions of the
 * host link busy.  The host arrays must stay untouched until the stream has passed
 * the call; device errors are returned by ams_context_sync(ctx).  When the call itself
 * returns an error, the copies it had enqueued have finished.  Reusing a context is
 * ordered on its stream like every context call (one stream per context). */
AMS_API ams_status ams_sort_host_async(void* ctx, void* h_keys, uint64_t* h_vals, uint64_t n,
                               ams_key_type kt, int levels, const uint32_t* buckets_per_level,
                               uint64_t seed, const ams_options* opt, void* stream);

/* --------------------------------------------------------------- contexts */

/* A context holds the scratch memory (ping-pong buffer, per-level tables), the
 * device status word and the statistics of the last sort.  The calls above use a
 * default context per device.  A context must not be used by two host threads at
 * once, and sorts on one context must be ordered on one stream; use one context
 * per concurrent stream.  hbm_budget_bytes caps the scratch the context may hold
 * (0 = no cap); a sort that needs more returns AMS_ERR_OOM. */
AMS_API ams_status ams_context_create(uint64_t hbm_budget_bytes, void** ctx);
AMS_API ams_status ams_context_destroy(void* ctx);

typedef struct ams_request {
  const void* keys_in;          /* device */
  void* keys_out;               /* device; may equal keys_in */
  const uint64_t* vals_in;      /* device or NULL */
  uint64_t* vals_out;           /* device or NULL (NULL iff vals_in is NULL) */
  const uint64_t* d_offsets;    /* device, nseg+1 entries; NULL = one segment of n */
  uint64_t nseg;
  uint64_t n;
  ams_key_type kt;
  int levels;
  const uint32_t* buckets_per_level;  /* host, `levels` entries */
  uint64_t seed;
  ams_options opt;
} ams_request;

/* The general entry point behind all sort calls.  ctx NULL = default context. */
AMS_API ams_status ams_sort_request(void* ctx, const ams_request* req, void* stream);

/* Wait for the context's last sort and return its device status (AMS_OK or
 * AMS_ERR_INTERNAL / AMS_ERR_TIMEOUT). */
AMS_API ams_status ams_context_sync(void* ctx);

/* Bytes of device scratch the context holds now. */
AMS_API uint64_t ams_context_scratch_bytes(void* ctx);

/* Bytes of device scratch `req` needs in a context (its ping-pong buffer, bucket ids
 * and per-level tables for the plan the request implies); 0 if the request is
 * invalid or needs none. */
AMS_API uint64_t ams_request_scratch_bytes(const ams_request* req);

/* Grow the context's scratch to at least `bytes` now (one cudaMalloc, after waiting for
 * the device if the context already held scratch), so that later sorts needing at
 * most that much allocate nothing.  Respects the context's budget (AMS_ERR_OOM). */
AMS_API ams_status ams_context_reserve(void* ctx, uint64_t bytes);

typedef struct ams_stats {
  uint32_t levels_planned;       /* distribution levels launched */
  uint32_t kernel_launches;      /* kernels launched by the last sort */
  uint32_t segments[8];          /* segments processed per level */
  uint32_t basecase_items[9];    /* base-case work items per level (0 = before level 1) */
  uint32_t device_status;
  uint32_t pad;
  /* With AMS_FLAG_PHASE_TIMERS: summed device time (ms) per kernel kind and the
   * number of launches of that kind, for the last sort.  Kinds: */
#define AMS_K_INIT 0
#define AMS_K_SETUP 1
#define AMS_K_SAMPLE_SORT 2   /* sample + local tile sort (Section 4.2) */
#define AMS_K_CROSS_RANK 3    /* all-pairs tile ranking (Section 4.2) */
#define AMS_K_SPLITTERS 4
#define AMS_K_CLASSIFY 5      /* classify + count */
#define AMS_K_SCAN 6
#define AMS_K_BINPACK 7
#define AMS_K_SCATTER 8
#define AMS_K_BASECASE 9
#define AMS_K_TABLE 10        /* cell table of the splitters (classifier start) */
#define AMS_K_COUNT 11
  float kernel_ms[AMS_K_COUNT];
  uint32_t kernel_calls[AMS_K_COUNT];
  uint64_t kernel_elems[AMS_K_COUNT];  /* elements read by that kind (for bandwidth) */
} ams_stats;

/* Statistics (waits for the context's last sort).  segments, basecase_items,
 * kernel_elems and levels_planned describe the last sort; kernel_launches,
 * kernel_ms and kernel_calls add up every sort since the previous call, which
 * resets them.  ctx NULL = default context. */
AMS_API ams_status ams_get_stats(void* ctx, ams_stats* out);

/* Intermediates of the context's last sort, per distribution level (for checking the
 * steps of Section 6 against a restatement; each call waits for that sort).  Segment
 * `seg` of level `level` (1-based) is one sub-problem sorted at that level: the whole
 * input at level 1, the non-final pieces above the base-case capacity after that. */
typedef struct ams_segment_info {
  uint32_t begin, end;   /* positions [begin, end) of the segment */
  uint32_t a, S;         /* oversampling factor a and sample size S = a*b*r (Section 6) */
  uint32_t L, ngroups;   /* optimal group bound L* and groups formed at it (Section 6
                            Lemma, Appendix C) */
  uint32_t npieces;      /* delivery pieces: runs of a group's buckets between heavy
                            equality buckets, and those equality buckets (final) */
  uint32_t nbucket_ids;  /* 2*b*r - 1 bucket ids of the level */
} ams_segment_info;

/* *nseg = segments of `level`; the first min(*nseg, max_seg) descriptions go to h_segs
 * (host, may be NULL), in the device's order (the order groups were emitted in). */
AMS_API ams_status ams_get_level_segments(void* ctx, int level, uint32_t* nseg,
                                          ams_segment_info* h_segs, uint32_t max_seg);

/* Tables of segment `seg` of `level` (host arrays, any may be NULL):
 *  h_bucket_starts (nbucket_ids entries): first position of every bucket id relative to
 *    the segment's begin (exclusive prefix sum of the global bucket sizes, Section 6);
 *  h_piece_of (nbucket_ids entries): the piece that delivers each bucket id;
 *  h_piece_starts (npieces entries): first position of every piece, relative; piece p
 *    ends where piece p+1 starts (the last at the segment's end).  A piece is final --
 *    an equality bucket, delivered and never sorted again -- exactly when every id
 *    mapped to it is odd.  Empty pieces may occur. */
AMS_API ams_status ams_get_segment_tables(void* ctx, int level, uint32_t seg,
                                          uint32_t* h_bucket_starts, uint16_t* h_piece_of,
                                          uint32_t* h_piece_starts);

/* --------------------------------------------------------------- building blocks
 * Each step of one distribution level on one segment, as its own call.  They run the
 * same kernels as the whole sort (on a one-segment table) and use the default
 * context's scratch.  Sample, splitter and ordered-key arrays hold keys in order
 * form: uint32_t for AMS_U32 / AMS_F32 (float keys mapped as described above) and
 * uint64_t for AMS_U64. */

/* Section 6 random sample of a*b*r elements: d_sample[j] = key[idx_j] (ordered form) for
 * j < count, idx_j = floor(u_j * n / 2^64) where u_j is output j of SplitMix64 started
 * at mix(mix(seed + (level+1)*g) + (begin+1)*g), g the SplitMix64 increment. */
AMS_API ams_status ams_step_sample(const void* d_keys, uint64_t n, ams_key_type kt, uint32_t count,
                           uint64_t seed, uint32_t level, uint64_t begin, void* d_sample,
                           void* stream);

/* Section 4.2, fast work-inefficient sorting: d_sorted[rank_i] = d_sample[i] with
 * rank_i = #{j : s_j < s_i} + #{j < i : s_j == s_i}.  count <= 65536. */
AMS_API ams_status ams_step_rank_sort(const void* d_sample, uint32_t count, ams_key_type kt,
                              void* d_sorted, void* stream);

/* Section 6, splitters of equidistant rank: d_splitters[i] = d_sorted[(i+1)*a] for
 * i < nbuckets-1; requires count == a*nbuckets. */
AMS_API ams_status ams_step_splitters(const void* d_sorted, uint32_t a, uint32_t nbuckets,
                              ams_key_type kt, void* d_splitters, void* stream);

/* Section 6 partitioning with Appendix D equality buckets: for every key, j =
 * #{splitters < key}; id = 2j, or 2j+1 if j < nbuckets-1 and key == splitter j.
 * d_counts (2*nbuckets-1 entries, uint32) receives the bucket sizes; d_ids (n entries,
 * uint16) the ids if not NULL.  d_splitters: nbuckets-1 sorted keys (ordered form). */
AMS_API ams_status ams_step_classify(const void* d_keys, uint64_t n, ams_key_type kt,
                             const void* d_splitters, uint32_t nbuckets, uint32_t* d_counts,
                             uint16_t* d_ids, void* stream);

/* Section 6 bucket grouping / Appendix C: d_L = smallest bound L for which scanning the
 * range-bucket sizes (d_counts[0], d_counts[2], ...) forms at most r groups;
 * d_group_ends (r entries) = exclusive end bucket of each group at that bound;
 * d_ngroups = number of groups. */
AMS_API ams_status ams_step_bin_pack(const uint32_t* d_counts, uint32_t nbuckets, uint32_t r,
                             uint64_t* d_L, uint32_t* d_group_ends, uint32_t* d_ngroups,
                             void* stream);

/* Section 6 delivery: stable partition of d_in into d_out by bucket id (ids as in
 * ams_step_classify); payloads move along when d_vals_in is not NULL. */
AMS_API ams_status ams_step_partition(const void* d_in, void* d_out, const uint64_t* d_vals_in,
                              uint64_t* d_vals_out, uint64_t n, ams_key_type kt,
                              const void* d_splitters, uint32_t nbuckets, void* stream);

/* Section 6 delivery as the keys-only sorts run it: every key goes to its bucket's
 * range of d_out (the ranges in bucket-id order, as ams_step_partition places them),
 * in arrival order inside the range -- the paper fixes no order inside a group, and
 * the base case orders every group.  Keys only; same arguments, errors and stream
 * behaviour as ams_step_partition. */
AMS_API ams_status ams_step_partition_arrival(const void* d_in, void* d_out, uint64_t n, ams_key_type kt,
                                      const void* d_splitters, uint32_t nbuckets, void* stream);

/* Section 6 base case: stable sort of n <= basecase capacity keys (and payloads) in
 * place in shared memory. */
AMS_API ams_status ams_step_base_case(void* d_keys, uint64_t* d_vals, uint64_t n, ams_key_type kt,
                              void* stream);

/* --------------------------------------------------------------- RLM-sort
 * Section 5 (recurse-last multilevel multiway mergesort), the paper's other
 * algorithm, with perfect load balance.  Tiles of `run` consecutive positions play
 * the processing elements.  Level 0: every tile is sorted locally.  Level l (l = 1 ..
 * levels): every part of the previous level (level 0: the whole input) is split into
 * parts_per_level[l-1] parts whose sizes differ by at most one (part j of a part of m
 * elements starts floor(j m / r) after it) by multisequence selection over the part's
 * tiles (Section 4.1: quickselect on sorted sequences, pivots drawn from a SplitMix64
 * stream of (seed, level, part, rank)); every part receives its pieces in tile order
 * (data delivery); then every tile of the new part merges the pieces it holds (the
 * local merge, done by the shared-memory sort: the pieces are sorted, so the result is
 * their merge), which gives the sorted sequences of the next level.  The result
 * (d_keys_out, and d_vals_out when d_vals_in is not NULL) is the same as
 * ams_sort_keys_into / ams_sort_pairs_into give; d_keys_out may equal d_keys_in.
 *  - run in [2, base-case capacity] (ams_default_basecase_cap); the parts of the last
 *    level must not exceed `run` (choose the product of the part counts >= n / run);
 *    otherwise AMS_ERR_UNSUPPORTED.  levels in [0, 8]; 0 sorts tiles only (n <= run).
 *  - Scratch: n keys (and payloads) plus the part, tile and cut tables, in ctx (NULL =
 *    default context); asynchronous on `stream`; device errors are latched in the
 *    context (ams_context_sync). */
AMS_API ams_status ams_rlm_sort(void* ctx, const void* d_keys_in, void* d_keys_out,
                                const uint64_t* d_vals_in, uint64_t* d_vals_out, uint64_t n,
                                ams_key_type kt, uint32_t run, int levels,
                                const uint32_t* parts_per_level, uint64_t seed, void* stream);

/* --------------------------------------------------------------- autotuner
 * Picks the plan of a size class by measurement (Section 7 tunes a and b the same
 * way): for (key type, pairs, ceil(log2 n)) it times candidate plans on n synthetic
 * uniform keys and on n duplicate-heavy keys (P(rank k) ~ 1/k over 2^20 values) in
 * ctx's scratch (ctx NULL = default context), scoring a plan by the sum of its two
 * times.  A first pass picks the shape: 1, 2 or 3 distribution levels, groups per level r
 * a power of two near (n / t)^(1/levels) for target leaf sizes t = C/2 and C/4, at
 * the default a and b.  A second pass tries, on that shape, b = 16 with the default a
 * (Section 7.2's b = 16, a = 1.6 log10 n), a = 1 with b = 64 (the appendix's sweep),
 * a = 1 with the default b, a = 1 with b = 16 (each while b * r <= 2048) and half the
 * base-case capacity C.  The fastest plan is kept in a table shared by the process
 * (later calls for the class return it at once).  Allocates and frees 3n keys (and
 * 2n payloads) of device memory per tuning. */
typedef struct ams_tuned {
  int levels;
  uint32_t buckets_per_level[8];  /* r per level, `levels` entries */
  uint32_t overpartition_b;       /* b */
  uint32_t candidates;            /* plans timed */
  float ms;                       /* score of the chosen plan (sum of the two times) */
  uint32_t oversample_a;          /* a; 0 = the per-segment rule */
  uint32_t basecase_cap;          /* C; 0 = the default capacity */
} ams_tuned;
AMS_API ams_status ams_tune(void* ctx, uint64_t n, ams_key_type kt, int pairs, void* stream, ams_tuned* out);

/* --------------------------------------------------------------- serving loop
 * The paper sorts one input at a time; a server sorts a stream of independent
 * requests of any size and key type with continuous batching.  Requests are
 * ams_request descriptions of device buffers (the caller keeps them alive and
 * untouched until the request completes).  A host thread owned by the server
 * admits them first come first served while the scratch of the requests in flight
 * stays within hbm_budget_bytes (0 = no limit; a request larger than the whole
 * budget runs alone) and, when a worker's context would have to grow, while the
 * device's free memory (cudaMemGetInfo) covers the growth with 256 MiB to spare;
 * it runs them on `streams` worker streams (each with its own
 * context, kept between requests, so requests overlap on the device), and packs
 * consecutive keys-only requests of one key type of at most pack_max_keys keys each
 * (0 = no packing) into one segmented sort.  Each result is the one the request
 * would get alone. */
typedef struct ams_server ams_server;
AMS_API ams_status ams_server_create(uint64_t hbm_budget_bytes, int streams, uint64_t pack_max_keys,
                                     ams_server** out);
/* The server's admission rule as a pure function (the server loop calls it): with
 * `in_flight` bytes of scratch held by running requests, a request needing `scratch`
 * bytes whose worker context would have to grow by `growth` bytes is admitted (1)
 * when nothing is in flight, or when in_flight + scratch <= budget (0 = no budget)
 * and growth is 0 or fits in `free_bytes` of free device memory with 256 MiB to
 * spare; otherwise it waits (0). */
AMS_API int ams_server_admits(uint64_t in_flight, uint64_t scratch, uint64_t budget, uint64_t growth,
                              uint64_t free_bytes);
/* Size every worker context (and the packing stage) for requests up to `largest` now,
 * so that no allocation -- and no device-wide wait of a reallocation -- happens while
 * the server runs such requests.  Call before submitting. */
AMS_API ams_status ams_server_reserve(ams_server* s, const ams_request* largest);
/* Queue a request (copied; buckets_per_level is copied too); *ticket identifies it. */
AMS_API ams_status ams_server_submit(ams_server* s, const ams_request* req, uint64_t* ticket);
/* Block until the request completes; returns its status and, if not NULL, the host
 * steady-clock times (ns) of its submission and of the completion the server saw.
 * A ticket can be waited for once. */
AMS_API ams_status ams_server_wait(ams_server* s, uint64_t ticket, uint64_t* t_submit_ns, uint64_t* t_done_ns);
/* 1 if the request has completed, 0 if not, -1 for an unknown ticket. */
AMS_API int ams_server_done(ams_server* s, uint64_t ticket);
/* Launched batches and requests that were packed into shared batches. */
AMS_API ams_status ams_server_counters(ams_server* s, uint64_t* batches, uint64_t* packed_requests);
/* Finish every queued request, then release the server's streams and contexts. */
AMS_API ams_status ams_server_destroy(ams_server* s);

/* --------------------------------------------------------------- allocation-free sort
 * The paper has no counterpart to this call.  It is for callers that cannot let the
 * library allocate device memory while they call it -- for example a latency-critical
 * loop in which cudaMalloc / cudaFree would add their implicit device-wide
 * synchronisation, or a plug-in whose host application owns a fixed device-memory
 * budget.  It sorts d_keys (and d_vals if not NULL) in place, with the same result as
 * ams_sort_keys / ams_sort_pairs, using one thread block: shared-memory sorts of runs
 * and stable pairwise merges.
 *  - n must not exceed AMS_NOALLOC_MAX_KEYS; larger n returns AMS_ERR_INVALID and
 *    touches nothing.  So does a d_keys that is not aligned to its key size (4 or 8
 *    bytes) or a d_vals that is not 8-byte aligned.  It allocates nothing: the merge scratch is one file-scope
 *    device array of AMS_NOALLOC_MAX_KEYS * 16 bytes (8 MiB) that every GPU which
 *    loads the library holds until the process exits.
 *  - The first call on each device looks up that array's device address; make the
 *    first call on a device before any stream capture.
 *  - All calls on a device share the array.  Calls that overlap on the GPU (two
 *    streams, or two host threads) race and give wrong results: order them on one
 *    stream.  The array keeps the previous call's contents; the sort writes every
 *    scratch element before reading it, so nothing needs clearing.
 *  - Asynchronous on `stream` like the other device calls. */
#define AMS_NOALLOC_MAX_KEYS 524288u
AMS_API ams_status ams_sort_small_noalloc(void* d_keys, uint64_t* d_vals, uint64_t n,
                                          ams_key_type kt, void* stream);

/* --------------------------------------------------------------- misc */
AMS_API const char* ams_status_string(ams_status s);
/* Default base-case capacity for a key type (pairs != 0 for key-value sorts); a sort
 * of one segment whose planned leaves fit half of it may use half (see
 * ams_options.basecase_cap). */
AMS_API uint32_t ams_default_basecase_cap(ams_key_type kt, int pairs);
/* Library version, e.g. "0.1.0". */
AMS_API const char* ams_version(void);

#ifdef __cplusplus
}
#endif
#endif /* AMS_H */
