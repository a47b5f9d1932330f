/*
 * ed.h -- C ABI of the GB300 edit-distance library (libedgb300.so).
 *
 * The library computes the exact Levenshtein distance (unit-cost insertion,
 * deletion and substitution; Sec. 1 and Sec. 2 of "Efficient Parallel
 * Output-Sensitive Edit Distance") of byte strings with the breadth-first
 * Landau-Vishkin method of Algorithm 1 (Sec. 3.1, Appendix A), on one GPU.
 *
 * Conventions used throughout this header:
 *   - strings are arrays of uint8_t of the given length; any byte value is a
 *     symbol (NUL included); lengths 0 are legal;
 *   - a DP cell (x, y) has consumed x bytes of A and y bytes of B;
 *     diagonal d = y - x; L_t[d] is the largest x on diagonal d reachable
 *     with t edits (the paper's f_t[i] with i = -d);
 *   - n and m must each be below 2^31 - 64 (row values are 32-bit);
 *   - "host pointer" = ordinary process memory (pinned or pageable);
 *     "device pointer" = memory of the context's CUDA device;
 *   - every function returns an ed_status; negative values are failures and
 *     leave the output arguments unspecified;
 *   - a context is not thread-safe except for ed_submit / ed_poll, which may
 *     be called from any thread;
 *   - the caller keeps ownership of every buffer it passes; the library
 *     keeps no pointer to a caller buffer after the call returns, except
 *     where stated for *_dev serving calls.
 */
#ifndef ED_GB300_H
#define ED_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ed_ctx ed_ctx; /* opaque; owns device memory, streams, engine */

typedef enum {
    ED_OK = 0,         /* success */
    ED_EAGAIN = 1,     /* ed_poll: request still running */
    ED_EINVAL = -1,    /* bad argument (NULL with length > 0, size limit, ...) */
    ED_ENOMEM = -2,    /* device or host allocation failed / budget too small */
    ED_ECUDA = -3,     /* a CUDA runtime call failed (ed_last_cuda_error) */
    ED_ETIMEOUT = -4,  /* a bounded device-side wait gave up */
    ED_EBUSY = -5,     /* admission refused: no free slot or memory; retry */
    ED_ENOTFOUND = -6, /* unknown or already-collected ticket */
    ED_ELIMIT = -7     /* distance exceeds the context's frontier capacity */
} ed_status;

typedef enum {
    ED_LCP_AUTO = 0,   /* the faster on GB300 at every length and distance
                          measured: direct comparison (as ED_LCP_DIRECT) */
    ED_LCP_DIRECT = 1, /* 16-byte direct comparison (Sec. 5.1 fast path) */
    ED_LCP_HASH = 2,   /* prefix-hash doubling search, confirmed directly */
    ED_LCP_BHASH = 3   /* the same search on blocked prefix tables (Sec. 3.3,
                          Alg. 2: hashes of whole blocks only, hash_block
                          characters each), confirmed directly */
} ed_lcp_mode;

typedef struct {
    int device;               /* CUDA device ordinal; -1 = current device */
    size_t mem_budget_bytes;  /* device bytes the context may hold; 0 = 60% of free */
    int max_inflight;         /* serving slots; 0 = 1024 */
    int lcp_mode;             /* ed_lcp_mode */
    uint64_t hash_seed;       /* selects the hash base; 0 = fixed default */
    uint64_t spin_limit_ns;   /* bound of every device-side wait; 0 = 2e9 */
    int grid_ctas;            /* CTAs of the tile kernel; 0 = one per SM */
    int tile_width;           /* diagonals per CTA in the first epoch (the
                                 tiles grow with the band, by an eighth at
                                 a time); 0 = 64 */
    int block_rounds;         /* rounds between neighbour exchanges (1..64);
                                 0 = 32 */
    int64_t max_rounds;       /* frontier capacity in rounds; 0 = the larger
                                 string length (at most 2^28) */
    int hash_block;           /* block size b of ED_LCP_BHASH (1..4096);
                                 0 = 32 */
    int warp_cap;             /* bytes one warp compares before a slide
                                 goes to the whole CTA (>= 512); 0 = 4096 */
    int local_chunks;         /* 16 KiB chunks a CTA compares alone before
                                 its long slide is opened to other CTAs;
                                 0 = none (open at once) */
    int help_div;             /* while the band is narrow, 1/help_div of a
                                 group's CTAs hold no tile and serve long
                                 slides; 0 = 8, -1 = none */
    int64_t distance_hint;    /* expected distance of single pairs (0 =
                                 unknown); selects the tuning-table row */
    int tune;                 /* 1: launch parameters of single-pair calls
                                 that this configuration leaves at 0 come
                                 from the tuning table; 0 = off */
    const char *tune_table;   /* path of the tuning table; NULL = the
                                 tune_table.tsv installed beside the
                                 library.  Read by ed_create only. */
} ed_config;

typedef struct {
    uint64_t k;              /* the edit distance */
    uint64_t extensions;     /* diagonal-extensions: (t, d) cells evaluated */
    uint64_t slide_chars;    /* sum over extensions of the LCP length */
    uint64_t compared_bytes; /* 2 * (slide_chars + mismatching compares) */
    uint64_t long_slides;    /* slides handed to the job slots (helped) */
    uint64_t open_slides;    /* slides the start-row words did not finish
                                (continued by a warp), tile kernel only */
    uint64_t wide_rounds;    /* rounds run in temporal blocks */
    uint64_t hash_queries;   /* LCP queries answered by the hash search */
    uint64_t hash_collisions;/* hash answers refuted by the direct check */
    uint64_t kernel_launches;/* kernels launched by this call */
    double kernel_ms;        /* device time of the distance kernel(s) */
    double build_ms;         /* device time of the prefix-hash build */
    double phase_ms[6];      /* device time by phase, as seen by the first
                                CTA of the group: rounds, open slides,
                                neighbour waits (helping included), epoch
                                changes; [4] the CTAs' average busy time
                                (rounds + open slides); [5] the batch
                                kernel's time (batched calls) */
} ed_stats;

/* Fills *cfg with the defaults described in ed_config. */
int ed_config_default(ed_config *cfg);

/* The tuning-table row for a pair of lengths n, m with an expected
 * distance (0 = unknown, taken as an edit rate of 1e-4): sets lcp_mode,
 * block_rounds, tile_width, warp_cap, local_chunks and help_div of *cfg to
 * the row's values (the other fields are left as they are).  The table is a
 * text file (table = its path; NULL = tune_table.tsv beside the library)
 * whose rows give, for max(n, m) in [n_lo, n_hi) and distance / max(n, m) in
 * [rate_lo, rate_hi), the parameters a measured sweep found fastest:
 * columns n_lo n_hi rate_lo rate_hi lcp_mode block_rounds tile_width
 * warp_cap local_chunks help_div ('#' starts a comment); the first matching
 * row is taken.  Host only.  ED_EINVAL when the table cannot be read or a
 * row is malformed, ED_ENOTFOUND when no row matches. */
int ed_tune_lookup(const char *table, size_t n, size_t m, int64_t distance_hint, ed_config *cfg);

/* Creates a context on cfg->device (cfg may be NULL for defaults).  Sizes
 * its memory pool lazily inside the budget.  *out receives the context. */
int ed_create(ed_ctx **out, const ed_config *cfg);

/* Waits for or cancels in-flight serving work, frees everything. */
int ed_destroy(ed_ctx *ctx);

/* Static description of a status code (never NULL). */
const char *ed_strerror(int status);

/* Text of the last CUDA error seen by the context ("" if none). */
const char *ed_last_cuda_error(ed_ctx *ctx);

/* Exact distance of one pair; A and B are HOST pointers.  Copies the
 * strings to the device (inside the call), runs Algorithm 1 in one
 * persistent kernel launch and returns when *k is known.  Synchronous. */
int ed_distance(ed_ctx *ctx, const uint8_t *A, size_t n, const uint8_t *B,
                size_t m, uint64_t *k);

/* As ed_distance, but A and B are DEVICE pointers (any alignment) and the
 * work is ordered on `stream` (a cudaStream_t; NULL = legacy default).
 * Returns after the stream reaches the end of the work. */
int ed_distance_dev(ed_ctx *ctx, const uint8_t *A, size_t n,
                    const uint8_t *B, size_t m, uint64_t *k, void *stream);

/* Counters of the last ed_distance / ed_distance_dev / batch call. */
int ed_last_stats(ed_ctx *ctx, ed_stats *out);

/* Many independent pairs (Sec. 6 workloads, batched): A[p], B[p] are
 * DEVICE pointers of lengths n[p], m[p] (the pointer arrays themselves are
 * host arrays); k_out is a host array of npairs entries.  One persistent
 * launch claims pairs from a cost-ordered work queue; pairs whose band
 * outgrows one CTA continue on the single-pair kernel.  Synchronous. */
int ed_distance_batch_dev(ed_ctx *ctx, size_t npairs,
                          const uint8_t *const *A, const size_t *n,
                          const uint8_t *const *B, const size_t *m,
                          uint64_t *k_out, void *stream);

/* As ed_distance_batch_dev with HOST string pointers (copied inside). */
int ed_distance_batch(ed_ctx *ctx, size_t npairs, const uint8_t *const *A,
                      const size_t *n, const uint8_t *const *B,
                      const size_t *m, uint64_t *k_out);

/* Serving (continuous batching).  ed_submit copies the HOST strings into
 * device memory before it returns (the caller may free them at once),
 * admits the pair when a slot and its memory fit the budget, and returns a
 * ticket; ED_EBUSY means "not admitted, retry later".  Admitted pairs run
 * concurrently on the device, each keeping its frontier resident in device
 * memory between engine steps; pairs retire as soon as they finish.
 * ed_poll returns ED_OK with *k once the pair is done (the ticket is then
 * released), ED_EAGAIN while it runs, ED_ENOTFOUND for unknown tickets. */
int ed_submit(ed_ctx *ctx, const uint8_t *A, size_t n, const uint8_t *B,
              size_t m, uint64_t *ticket);
int ed_poll(ed_ctx *ctx, uint64_t ticket, uint64_t *k);

/* ed_submit for DEVICE strings A, B (memory of the context's device, any
 * alignment) produced on `stream` (a cudaStream_t; NULL = legacy default):
 * the pair is admitted like ed_submit's (a serving slot and its resident
 * frontier in the arena; ED_EBUSY when either is missing) but its strings
 * are not copied: the engine reads the caller's buffers, after the work
 * queued on `stream` before this call (an event recorded on it), so the
 * caller may submit strings that a kernel of its own is still writing.  A
 * and B must stay alive and unchanged until ed_poll returns ED_OK (or an
 * error) for the ticket.  Returns at once; results through ed_poll. */
int ed_submit_dev(ed_ctx *ctx, const uint8_t *A, size_t n, const uint8_t *B,
                  size_t m, uint64_t *ticket, void *stream);

/* Serving counters: admitted, completed, in flight, engine steps, and
 * slices (times a pair on the tile kernel was left at a sync point with its
 * band frontier saved, to be resumed at the next step).  Null pointers are
 * skipped. */
int ed_serve_counters(ed_ctx *ctx, uint64_t *admitted, uint64_t *completed,
                      uint64_t *inflight, uint64_t *steps, uint64_t *slices);

/* ---- building blocks, exported for tests and diagnostics ---------------- */

/* LCP(A, B, x[i], y[i]) of Sec. 2 for q queries; A, B device pointers;
 * x, y, out host arrays.  method: 0 = per-thread 16-byte compare, 1 = one
 * warp per query (ballot / first-set-bit), 2 = whole-grid search,
 * 3 = hash search alone (needs ed_prefix_hash tables TA, TB as device
 * pointers of n+1 and m+1 entries; may differ from the LCP on a hash
 * collision), 4 = hash search confirmed directly (exact), 5 and 6 = 3 and 4
 * on blocked tables (ed_prefix_hash_blocked_dev with the context's
 * hash_block b: n/b+1 and m/b+1 entries), 7 = 2 with each chunk staged in
 * shared memory by bulk copies.  Synchronous. */
int ed_lcp_dev(ed_ctx *ctx, const uint8_t *A, size_t n, const uint8_t *B,
               size_t m, const int64_t *x, const int64_t *y, size_t q,
               int method, const uint64_t *TA, const uint64_t *TB,
               int64_t *out, void *stream);

/* The prefix table of Sec. 3.2: T[i] = sum_{j<i} (X[j]+1) * p^(i-1-j)
 * mod 2^61-1 for i = 0..len, p = ed_hash_base(ctx).  X and T are device
 * pointers; T has len + 1 uint64 entries.  One single-pass scan launch;
 * synchronous on `stream`.  ED_ETIMEOUT when a bounded wait of the scan
 * gave up (the table is then not valid). */
int ed_prefix_hash_dev(ed_ctx *ctx, const uint8_t *X, size_t len, uint64_t *T,
                       void *stream);

/* The blocked prefix table of Sec. 3.3 (Alg. 2): T[j] = h(X[0..j*b)) for
 * j = 0..len/b, the entries of ed_prefix_hash_dev's table at multiples of
 * b (1 <= b <= 2^20).  X and T are device pointers; T has len/b + 1 uint64
 * entries.  One scan launch that writes only the block prefixes.
 * Synchronous on `stream`; ED_ETIMEOUT as for ed_prefix_hash_dev. */
int ed_prefix_hash_blocked_dev(ed_ctx *ctx, const uint8_t *X, size_t len, size_t b, uint64_t *T,
                               void *stream);

/* The hash base p used by the context (derived from hash_seed). */
uint64_t ed_hash_base(ed_ctx *ctx);

/* Largest len accepted by ed_prefix_hash_noalloc (21843 scan tiles of 4096
 * bytes: the scan's 48-byte look-back descriptors plus a 64-byte header fit
 * its 1 MiB scratch array). */
#define ED_NOALLOC_MAX_LEN ((size_t)89468928)

/* ed_prefix_hash_dev for callers that cannot allocate device memory: code
 * embedded in a host framework whose memory manager owns every device
 * allocation (a stray cudaMalloc escapes its budget and accounting, or is
 * refused), and code that cannot afford cudaMalloc / cudaFree on its path
 * (cudaFree waits for the whole device).  No context is needed and nothing
 * is allocated: the scan's working state lives in a
 * fixed 1 MiB array compiled into the library, which every GPU that loads
 * the library keeps until the process exits.  The paper has no counterpart;
 * the table computed is the same as ed_prefix_hash_dev's with the given
 * base.  X and T are device pointers (T: len + 1 uint64 entries) of the
 * CURRENT device, and `stream` belongs to it; the call must run in that
 * device's primary context (the CUDA runtime's own; the array's address is
 * looked up once per device ordinal in it).  base must lie in
 * [2, 2^61-2].  len above ED_NOALLOC_MAX_LEN returns ED_EINVAL.  The
 * first call on a device looks up the array's device address (make that
 * call before any stream capture).  Every call shares the array and clears
 * it on `stream` before use: calls whose work overlaps on the GPU (two
 * streams, or two threads) race and must be serialised by the caller.
 * Synchronous on `stream` (NULL = legacy default).  ED_ETIMEOUT when a
 * bounded wait of the scan gave up (the table is then not valid). */
int ed_prefix_hash_noalloc(const uint8_t *X, size_t len, uint64_t base, uint64_t *T,
                           void *stream);

/* Runs Algorithm 1 on DEVICE strings for rounds 0..t_max and writes the
 * frontiers to the HOST array out[t * (2*t_max+1) + (d + t_max)] (int32;
 * INT32 value -1061109568 where undefined).  *k receives the distance if
 * it is <= t_max, else UINT64_MAX.  For parity checks on small inputs. */
int ed_frontiers_dev(ed_ctx *ctx, const uint8_t *A, size_t n,
                     const uint8_t *B, size_t m, int64_t t_max, int32_t *out,
                     uint64_t *k, void *stream);

/* Edit operations of ed_edit_script_dev, and its bound on t_max. */
enum { ED_OP_SUB = 0, ED_OP_DEL = 1, ED_OP_INS = 2 };
#define ED_SCRIPT_MAX_ROUNDS 16384

/* An optimal edit script of A into B (DEVICE strings), traced back from
 * the frontiers of rounds 0..k of Algorithm 1 (Sec. 3.1): a cell on
 * diagonal d has distance at most t exactly when its row is at most L_t[d]
 * (the distance never falls along a diagonal), so walking back from (n, m)
 * each round's slide is crossed at once and one edit leads to a cell of
 * round t - 1.  ops[3*i], ops[3*i+1], ops[3*i+2] = (kind, x, y), in the
 * order they apply from the start of the strings: ED_OP_SUB puts B[y] in
 * place of A[x], ED_OP_DEL deletes A[x], ED_OP_INS inserts B[y] before A[x];
 * the characters between two operations match.  *nops = *k operations.
 * Needs k <= t_max <= ED_SCRIPT_MAX_ROUNDS.  The frontiers take (t_max+1)
 * (2 t_max+1) int32 of device memory, kept in the context, and as much host
 * memory during the call (2.1 GB each at the bound; ED_ENOMEM when either
 * cannot be had).  ED_ELIMIT with *k = UINT64_MAX when k > t_max.  ops has room for cap operations (3 int64 each); cap <
 * k returns ED_EINVAL with *k set.  Any script it returns is one of the
 * optimal ones (several may exist).  Synchronous on `stream`. */
int ed_edit_script_dev(ed_ctx *ctx, const uint8_t *A, size_t n,
                       const uint8_t *B, size_t m, int64_t t_max,
                       int64_t *ops, size_t cap, size_t *nops, uint64_t *k,
                       void *stream);

/* The walk back of ed_edit_script_dev over frontiers the caller supplies:
 * F is a HOST array F[t * (2*t_max+1) + (d + t_max)] = L_t[d] for rounds
 * 0..k (negative where undefined: the layout ed_frontiers_dev writes) for
 * strings of lengths n and m at distance k <= t_max.  Host work only.  ops,
 * cap and *nops as in ed_edit_script_dev; the characters themselves are
 * not needed.  ED_EINVAL for a null pointer, k > t_max, cap < k, or
 * frontiers that do not describe a distance-k alignment of those lengths. */
int ed_trace_script(const int32_t *F, int64_t t_max, size_t n, size_t m, uint64_t k,
                    int64_t *ops, size_t cap, size_t *nops);

#ifdef __cplusplus
}
#endif
#endif /* ED_GB300_H */
