// lv_kernels.cuh -- argument blocks and launch entry points of the
// Landau-Vishkin kernels (Algorithm 1, Sec. 3.1 / Appendix A).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace edg {

// status codes written by kernels
constexpr uint32_t ST_TIMEOUT = 4;
constexpr uint32_t ST_LIMIT = 7;  // the round cap was reached
constexpr uint32_t ST_WIDE = 8;   // per pair: the band outgrew its group's tiles
constexpr uint32_t ST_SUSPENDED = 9; // per pair: budget spent, frontier saved to keep

constexpr int CTA_THREADS = 256;   // threads of a tile CTA (up to 255 registers each)
constexpr int MAX_GRID = 1024;     // CTAs of one tile launch, at most
constexpr int HMAX = 64;           // rounds per temporal block, at most
constexpr int CHUNK_BYTES = 16 * 1024; // bytes of one job-slot claim (per string)
constexpr int SMAX_LIMIT = 16384;  // widest tile a CTA keeps in shared memory
constexpr int MAX_CLS = 12;        // group-size classes of one tile launch
// done_k of a pair that ended without a distance (status in its R_STATUS)
constexpr unsigned long long DONE_STOPPED = ~0ull - 1;

// A long slide open for help.  Each CTA owns JOB_RING slots, used in turn.
// `claim` packs the job id (high 32 bits) and the count of claims made (low
// 32 bits): every atomicAdd of 1 claims the next chunk (CHUNK_BYTES of each
// string).  The descriptor words (x, y, lim, the pair's index in the
// launch's pair table), the result (~ the least mismatch offset) and one
// answer word per chunk each carry a job id in their high half; answers are
// raised by red.max (the protocol is in lv_tiles.cu).
constexpr int JOB_RING = 2;
constexpr int JOB_MAX_CHUNKS = 4096; // chunks of one job; longer slides are cut
struct __align__(128) JobSlot {
    unsigned long long claim;
    unsigned long long pad0[15]; // the claim word alone in its 128-byte line
    unsigned long long xt, yt, lt, pt;
    unsigned long long result;
    unsigned long long pad1[11];
    unsigned long long ans[JOB_MAX_CHUNKS];
};

// One pair of a tile launch.
struct PairDesc {
    const uint8_t *A, *B;
    int64_t n, m;
    const uint64_t *TA, *TB;   // prefix-hash tables (hash LCP) or null
    unsigned long long *res;   // R_COUNT counters of this pair
    int32_t *dump;             // frontier dump (tests) or null
    int32_t dump_tmax;
    int32_t pad;
    // resident frontier across launches (serving) or null: L_{t-1}[d] at
    // keep[d + keep_r + 2] for |d| <= keep_r; the pair starts at round t0
    // with epoch radius R0 when t0 > 0
    int32_t *keep;
    int64_t keep_r, t0, R0;
};

// Per group of CTAs (zeroed before the launch).
struct __align__(64) GroupCtl {
    unsigned long long done_k; // ~0 until the tile owning d = m - n finds k
                               // (DONE_STOPPED: the pair ended without it)
    uint32_t bar_count, bar_gen;
    uint32_t epoch_req;        // epoch changes requested (for CTAs without a tile)
    uint32_t epoch_t;          // round at which the last epoch change happens
    int32_t pair;              // pair index being run (-1: none left)
    uint32_t ebar_count, ebar_gen; // epoch-change barrier (abandoned once k is known)
    uint32_t susp[2];          // epoch e ends the launch's share of the pair: susp[e & 1]
    uint32_t pad;
    // the furthest row of the band and its diagonal at epoch e's change:
    // lead[e & 1] = max over tiles of (L << 32) | (d + 2^31)
    unsigned long long lead[2];
};

// Per launch (zeroed before the launch).
struct __align__(64) LaunchCtl {
    uint32_t error;
    uint32_t queue[MAX_CLS];   // next pair of each class's queue
    uint32_t pad[3];
    // where the first failed wait gave up: site, CTA, round, awaited value,
    // values seen, done_k
    unsigned long long diag[8];
    unsigned long long active[(MAX_GRID * JOB_RING + 63) / 64]; // job slots open for help
};

// Result counters written by a launch, per pair.
enum {
    R_K = 0,
    R_SLIDE = 1,      // sum of LCP lengths
    R_MISMATCH = 2,   // slides that ended on a mismatching pair
    R_LONG = 3,       // slides given to the job slots
    R_WIDE = 4,       // temporal blocks run
    R_HASHQ = 5,
    R_HASHCOLL = 6,
    R_STATUS = 7,
    // device time (ns, seen by thread 0 of the group's first CTA): rounds,
    // open slides, halo waits (helping included), epoch changes, spare
    R_T0 = 8,
    R_RESUME_T = 14,  // suspended: the round to start from, and the radius
    R_RESUME_R = 15,
    R_OPEN = 16,      // slides continued by a warp (own diagonals)
    R_COUNT = 17
};

// The CTAs of a tile launch are cut into groups by class: class c has
// groups of cls_G[c] CTAs on CTAs [cls_c0[c], cls_c0[c+1]), numbered from
// cls_g0[c], and runs pairs [cls_p0[c], cls_p0[c+1]) of the pair list first,
// then those of the classes below it (smaller groups, narrower bands).  A
// group's re-tiling buffers (2 of 2*kc+5 entries, kc = cls_kc[c]) start at
// gf + cls_gf[c] + (its index in the class) * 2 * (2*kc+5).
struct LvArgs {
    const PairDesc *pairs;
    int32_t npairs;
    int32_t ncls;
    int32_t cls_G[MAX_CLS], cls_c0[MAX_CLS + 1], cls_g0[MAX_CLS], cls_p0[MAX_CLS + 1];
    int32_t cls_kc[MAX_CLS];
    int64_t cls_gf[MAX_CLS];
    GroupCtl *gctl;
    LaunchCtl *ctl;
    JobSlot *slots;       // gridDim.x * JOB_RING slots (CTA c owns c * JOB_RING ..)
    // tile edges: [gridDim.x][2 parity][2 sides][HMAX] words (round << 32) | L
    unsigned long long *halo;
    int32_t *gf;
    int32_t kcap;         // round cap (largest epoch radius)
    int32_t smax;         // tile width capacity (shared memory)
    int32_t h;            // rounds per temporal block (1..HMAX)
    int32_t s0;           // initial tile width
    int32_t t2_cap;       // bytes one warp examines before escalating
    int32_t use_hash;
    int32_t hash_b;       // prefix-table stride: 1 full, > 1 blocked (Alg. 2)
    uint64_t pow2[62];    // p^(2^j) mod 2^61-1 (hash LCP)
    uint64_t spin_ns;     // bound of one wait on a peer's progress
    uint64_t idle_ns;     // bound of a wait that may span other CTAs' work
    // time slicing: with budget_ns > 0, a group on a pair with a keep
    // buffer meets every sync_rounds rounds and saves and leaves the pair
    // once budget_ns have passed since the launch started
    uint64_t budget_ns;
    int32_t sync_rounds;
    // while a group's band is narrow, G / help_div of its CTAs (groups of at
    // least 2 * help_div CTAs) hold no tile and serve long slides (0: none)
    int32_t help_div;
    // chunks of a long slide its CTA scans alone before publishing the rest
    int32_t local_chunks;
    // stages of shared memory per CTA into which bulk copies bring a long
    // slide's chunks (0: loads into registers instead; 2: the owner streams
    // its first chunks with the next one's copies in flight)
    int32_t stage;
};

size_t lv_tiles_smem_bytes(int smax, int h, int stage);
cudaError_t launch_lv_tiles(const LvArgs &P, int grid, cudaStream_t s);

// ---------------------------------------------------------------- batch
// One pair of a batch / serving slot.  Frontier state lives in global
// memory between launches (serving keeps it resident across engine steps).
struct BatchPair {
    const uint8_t *A, *B;
    int64_t n, m;
    int32_t *front;    // W + 3 int32: the pair's resident frontier (round t)
    int32_t t;         // rounds completed so far (-1 = not started)
    int32_t state;     // 0 running, 1 done, 2 needs the tile kernel, 3 self-check failed
    int64_t k;
    int64_t reach;     // when parked: the furthest row of the saved frontier
    unsigned long long slide, mism;
    long long check[3]; // self-check record: round, diagonal, start row
};

struct BatchArgs {
    BatchPair *pairs;
    const int32_t *order; // claim order (cost-sorted)
    int32_t npairs;
    int32_t W;            // band capacity per pair (even)
    int32_t round_budget; // rounds per launch per pair (<=0: unlimited)
    uint32_t *next;       // work-queue head
    int32_t t2_cap;
    uint64_t spin_ns;
    uint32_t *error;
};

size_t lv_batch_smem_bytes(int W);
// budget_ns: device time after which each CTA parks its pair and stops
// claiming (0 = run every pair to the end)
cudaError_t launch_lv_batch(const BatchArgs &B, int grid, cudaStream_t s, uint64_t budget_ns);
int lv_batch_threads();
int lv_batch_ctas_per_sm(int W); // resident CTAs per SM (registers, shared memory)

// ---------------------------------------------------------------- tests
struct HashArgs {
    const uint64_t *TA, *TB;
    int32_t b;            // table stride: 1 full table, > 1 blocked (Alg. 2)
    uint64_t pow2[62];
};
// LCP queries by the building blocks: 0 per thread, 1 per warp, 2 whole
// grid (job slots), 3 hash search alone, 4 hash + direct confirmation.
// Method 2 reads queries from slots[0..q) (x, y, lim) and leaves answers in
// slots[i].result; the others use x, y, out.
cudaError_t launch_lcp_queries(const uint8_t *A, int64_t n, const uint8_t *B, int64_t m,
                               const int64_t *x, const int64_t *y, int64_t q, int method,
                               const HashArgs *hash, int64_t *out, JobSlot *slots, const PairDesc *pairs,
                               int grid, cudaStream_t s);

// ---------------------------------------------------------------- hash
// stride 1: T[i] = h(X[0..i)) for i = 0..len; stride b > 1: T[j] = h(X[0..jb))
// for j = 0..len/b (the blocked table of Sec. 3.3)
cudaError_t launch_prefix_hash(const uint8_t *X, int64_t len, uint64_t base, uint64_t *T, int64_t stride,
                               void *scan_state, size_t scan_state_bytes, cudaStream_t s);
size_t prefix_hash_state_bytes(int64_t len);
// After a launch_prefix_hash on s: waits for s and returns the scan's status
// word (0, or ST_TIMEOUT when a bounded look-back wait gave up); *e gets the
// CUDA error of the copy or the wait.
uint32_t prefix_hash_status(const void *scan_state, cudaStream_t s, cudaError_t *e);

} // namespace edg
