// lv_kernels.cuh -- argument blocks and launch entry points of the
// Landau-Vishkin kernels (Algorithm 1, Sec. 3.1 / Appendix A).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace edg {

// status codes written by kernels
constexpr uint32_t ST_TIMEOUT = 4;
constexpr uint32_t ST_LIMIT = 7;

constexpr int MAX_GRID = 1024;   // helper slots in the job block
constexpr int CTA_THREADS = 512;
constexpr int CHUNK_BYTES = CTA_THREADS * 16 * 4; // whole-grid slide chunk

// A slide that outgrew one warp, handed to the whole grid.  result starts
// at lim and is lowered with atomicMin to the first mismatch offset.
struct LongItem {
    int64_t x, y, lim;
    unsigned long long result;
    int32_t d;
    int32_t pad;
};

// Control block of one single-pair launch (zeroed before the launch).
struct LvJob {
    uint32_t epoch;     // last job published by CTA 0 (release)
    uint32_t kind;      // JOB_*
    uint32_t nitems;    // items of a JOB_LONG
    uint32_t wide_t;    // first round of the wide phase
    uint32_t error;     // kernel status (0 = ok)
    uint32_t bar_count; // grid barrier arrivals
    uint32_t bar_gen;   // grid barrier generation
    uint32_t glist[3];  // wide-phase long-item counts, by round mod 3
    uint32_t pad[6];
    uint32_t done[MAX_GRID]; // helper h: last epoch it finished
};
enum : uint32_t { JOB_NONE = 0, JOB_LONG = 1, JOB_WIDE = 2, JOB_QUIT = 3 };

// Result counters written by a launch.
enum {
    R_K = 0,
    R_SLIDE = 1,      // sum of LCP lengths
    R_MISMATCH = 2,   // slides that ended on a mismatching pair
    R_LONG = 3,       // long slides given to the grid
    R_WIDE = 4,       // rounds run in the wide phase
    R_HASHQ = 5,
    R_HASHCOLL = 6,
    R_STATUS = 7,
    R_COUNT = 8
};

struct HashArgs {
    const uint64_t *TA, *TB; // prefix tables (n+1, m+1 entries) or null
    uint64_t pow2[62];       // p^(2^j) mod 2^61-1
};

struct PairArgs {
    const uint8_t *A, *B;
    int64_t n, m;
    int32_t kcap;       // rounds the wide frontier can hold
    int32_t W0;         // narrow band capacity (even); t <= W0/2 in narrow mode
    int32_t *gf0, *gf1; // wide frontiers, 2*kcap+5 entries each (no clearing
                        // needed: every round writes its band and sentinels)
    LvJob *job;
    LongItem *items;
    int32_t item_cap;
    int32_t t1_cap;     // bytes one thread examines before escalating
    int32_t t2_cap;     // bytes one warp examines before escalating
    int32_t use_hash;
    HashArgs hash;
    unsigned long long *res; // R_COUNT counters
    int32_t *dump;           // frontier dump or null
    int32_t dump_tmax;
    uint64_t spin_ns;  // bound of one wait for a peer
    uint64_t idle_ns;  // bound of a helper's wait for the next job
};

size_t lv_single_smem_bytes(int W0);
cudaError_t launch_lv_single(const PairArgs &P, int grid, cudaStream_t s);

// ---------------------------------------------------------------- batch
// One pair of a batch / serving slot.  Frontier state lives in global
// memory between launches (serving keeps it resident across engine steps).
struct BatchPair {
    const uint8_t *A, *B;
    int64_t n, m;
    int32_t *front;    // W + 3 int32: the pair's resident frontier (round t)
    int32_t t;         // rounds completed so far (-1 = not started)
    int32_t state;     // 0 running, 1 done, 2 needs the single-pair kernel
    int64_t k;
    unsigned long long slide, mism;
};

struct BatchArgs {
    BatchPair *pairs;
    const int32_t *order; // claim order (cost-sorted)
    int32_t npairs;
    int32_t W;            // band capacity per pair (even)
    int32_t round_budget; // rounds per launch per pair (<=0: unlimited)
    uint32_t *next;       // work-queue head
    int32_t t1_cap, t2_cap;
    uint64_t spin_ns;
    uint32_t *error;
};

size_t lv_batch_smem_bytes(int W);
// budget_ns: device time after which each CTA parks its pair and stops
// claiming (0 = run every pair to the end)
cudaError_t launch_lv_batch(const BatchArgs &B, int grid, cudaStream_t s, uint64_t budget_ns);
int lv_batch_threads();

// ---------------------------------------------------------------- tests
// method 2 reads queries from items[0..q) (x, y, lim, result = lim) and
// leaves the answers in items[i].result; the others use x, y, out.
cudaError_t launch_lcp_queries(const uint8_t *A, int64_t n, const uint8_t *B, int64_t m,
                               const int64_t *x, const int64_t *y, int64_t q, int method,
                               const HashArgs *hash, int64_t *out, LongItem *items, int grid,
                               cudaStream_t s);

// ---------------------------------------------------------------- hash
cudaError_t launch_prefix_hash(const uint8_t *X, int64_t len, uint64_t base, uint64_t base_pow_tile,
                               uint64_t *T, void *scan_state, size_t scan_state_bytes,
                               cudaStream_t s);
size_t prefix_hash_state_bytes(int64_t len);

} // namespace edg
