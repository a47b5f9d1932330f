// lv_tiles.cu -- Algorithm 1 (Sec. 3.1, Appendix A) for one or several
// string pairs in ONE persistent cooperative launch.
//
// Round t sets, for every diagonal d in [-t, t] with a cell,
//     c        = max(L_{t-1}[d-1], L_{t-1}[d] + 1, L_{t-1}[d+1] + 1)
//     c        = min(c, n, m - d)           (clamp to the diagonal's last cell)
//     L_t[d]   = c + LCP(A[c..], B[c+d..])   (the slide)
// and stops at the first t with L_t[m-n] = n (then k = t).  This is the
// paper's loop with i = -d; taking the max before one slide gives the same
// row as sliding the three candidates and taking the max.
//
// GB300 mapping.
//  * The CTAs of a group split the diagonals of [-R, R] into static tiles,
//    one per CTA, each kept in shared memory.  R (the epoch radius) grows
//    by an eighth when the band [-t, t] reaches it; tiles are then re-cut
//    through a global buffer behind a group barrier (O(log k) times in all).
//    The busiest tiles are then at most 1.125 times the band's share.
//  * Temporal blocking: a CTA holds its tile plus h diagonals of halo on
//    each side and runs h rounds on the shrinking trapezoid (the halo
//    diagonals are recomputed, exactly), then trades its h edge values with
//    its two neighbours through global memory, each value in one 8-byte word
//    with its round (no fence, no flag).  There is no grid-wide barrier per
//    round, only neighbour waits every h rounds.
//  * Rounds: a narrow trapezoid (two diagonals per thread at most) runs the
//    lean form, one CTA barrier a round (run_block_lean); a wide one runs
//    pipelined rounds, six warps computing round t while two slider warps
//    finish the open slides of round t - 1 and the diagonals beside them
//    (run_block).
//  * Slides: one thread compares the two aligned 4-byte words at each start
//    row (at least five bytes; several diagonals' loads in flight together;
//    in the lean form 16 more bytes in one round trip when they all match);
//    slides still open go to one warp each (ballot / first set bit over
//    2 KiB steps), then, past t2_cap bytes, to the whole CTA, which opens a
//    job in its job slot: 16 KiB chunks (of each string), chunk 0 scanned by
//    the owner, the others claimed in order by atomicAdd by every CTA that is
//    waiting on a neighbour or has no tile, each staged in shared memory by
//    bulk copies; the first mismatch is the least over the chunks.
//  * Every wait is bounded by %globaltimer and reports ST_TIMEOUT (with the
//    place it gave up) instead of hanging.
#include "ed_device.cuh"
#include "lv_kernels.cuh"
#include "lv_round.cuh"

namespace edg {

constexpr int64_t GROW_NUM = 9, GROW_DEN = 8; // epoch radius growth factor
// Polls of the edge words by warp 0 before the CTA looks at anything else.
constexpr int HALO_SPINS = 4;
// Looks at the job slots by thread 0 of a CTA without a tile before its
// CTA meets at a barrier.
constexpr int IDLE_SPINS = 32;
// Looks at its job by the owner's warp 0 before its CTA meets at a barrier,
// and how long the claim count may stand still before the owner scans a
// chunk itself.
constexpr int WATCH_SPINS = 8;
constexpr int WATCH_WORDS = 4; // answer words a lane loads per look
constexpr uint64_t OWN_SCAN_NS = 1000;

struct Counters {
    unsigned long long slide = 0, mism = 0, hashq = 0, coll = 0, longs = 0, blocks = 0, opens = 0;
    unsigned long long tm[4] = {0, 0, 0, 0};
};
// What one call of open_slides adds to the counters.
struct SlideCounts {
    unsigned long long slide, mism, hashq, coll, longs, opens;
};

// ------------------------------------------------------------------ hash
__device__ __forceinline__ uint64_t powp(const uint64_t *pow2, int64_t e)
{
    uint64_t r = 1;
    for (int j = 0; e; j++, e >>= 1)
        if (e & 1)
            r = mulmod61(r, pow2[j]);
    return r;
}

// A prefix-hash table as the LCP search reads it: the full table (b = 1,
// T[i] = h(X[0..i))) or the blocked one of Sec. 3.3 (T[j] = h(X[0..jb))).
struct HashView {
    const uint64_t *T;
    const uint8_t *X;
    int32_t b;
};

// h(X[0..i)): the entry itself, or Alg. 2's GetHash: the prefix of the last
// whole block at or before i, extended by Horner's rule over the (< b)
// characters after it (p = pow2[0]).
__device__ __forceinline__ uint64_t prefix_at(const HashView &V, int64_t i, uint64_t p)
{
    if (V.b == 1)
        return __ldg(V.T + i);
    const int64_t r = i / V.b;
    uint64_t h = __ldg(V.T + r);
    for (int64_t j = r * V.b; j < i; j++)
        h = addmod61(mulmod61(h, p), (uint64_t)__ldg(V.X + j) + 1);
    return h;
}

// h(A[x..x+L)) == h(B[y..y+L)) with h(S2) = h([S1,S2]) - p^|S2| h(S1).
__device__ __forceinline__ bool hash_eq(const HashView &VA, const HashView &VB, uint64_t p, int64_t x,
                                        int64_t y, int64_t L, uint64_t P)
{
    const uint64_t a = submod61(prefix_at(VA, x + L, p), mulmod61(prefix_at(VA, x, p), P));
    const uint64_t b = submod61(prefix_at(VB, y + L, p), mulmod61(prefix_at(VB, y, p), P));
    return a == b;
}

// Sec. 3.2 (and Alg. 2 on blocked tables): compare chunks of length 1, 2,
// 4, ... (here: the powers of two above the l0 bytes already known equal)
// until one differs, then search the last bracket.  Returns the hash LCP
// (<= lim); the caller confirms it.
__device__ __noinline__ int64_t hash_lcp(const uint64_t *pow2, const HashView VA, const HashView VB,
                                         int64_t x, int64_t y, int64_t l0, int64_t lim)
{
    const uint64_t p = pow2[0];
    int64_t good = l0, bad;
    uint64_t pg = powp(pow2, good);
    int j = 0;
    while (j < 62 && (1ll << j) <= good)
        j++;
    for (;; j++) {
        const int64_t L = 1ll << j;
        if (L >= lim) {
            if (hash_eq(VA, VB, p, x, y, lim, powp(pow2, lim)))
                return lim;
            bad = lim;
            break;
        }
        if (hash_eq(VA, VB, p, x, y, L, pow2[j])) {
            good = L;
            pg = pow2[j];
        } else {
            bad = L;
            break;
        }
    }
    // largest length in [good, bad) whose hashes agree (binary lifting from
    // the highest bit of the bracket width)
    for (int i = 63 - __clzll((long long)(bad - good)); i >= 0; i--) {
        const int64_t cand = good + (1ll << i);
        if (cand < bad) {
            const uint64_t P = mulmod61(pg, pow2[i]);
            if (hash_eq(VA, VB, p, x, y, cand, P)) {
                good = cand;
                pg = P;
            }
        }
    }
    return good;
}

// ------------------------------------------------------------------ pair
struct Pair {
    const uint8_t *A, *B;
    int64_t n, m;
    int32_t q; // its index in the launch's pair table (job descriptors name it)
    const uint64_t *TA, *TB;
    bool hash;
};

// An open slide of diagonal d (start row c) reached row p: a mismatch at
// p < lim_abs, or none before lim_abs (p == lim_abs).  Returns the final
// row.  When the hash bound cut the search short and the direct compare
// found no mismatch at the hash answer (a collision, probability about
// l / 2^61), the slide is finished directly by this thread.
__device__ __forceinline__ int64_t finish_slide(const Pair &Q, int64_t c, int64_t d, int64_t p,
                                                int64_t lim_abs, bool own, Counters &C)
{
    const int64_t full_abs = c + min(Q.n - c, Q.m - c - d);
    if (Q.hash && lim_abs < full_abs) {
        if (own && p != lim_abs - 1)
            C.coll++;
        if (p == lim_abs) {
            bool open;
            p += slide_thread(Q.A, Q.n, Q.B, Q.m, p, p + d, full_abs - p, INT64_MAX, &open);
        }
    }
    if (own) {
        C.slide += p - c;
        C.mism += (p < full_abs);
    }
    return p;
}

// ------------------------------------------------------------------ jobs
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// Orders the relaxed loads before it ahead of every access after it (the
// acquire half of a flag handshake whose writer used a release).
__device__ __forceinline__ void fence_acquire() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void set_error(const LvArgs &P, uint32_t code)
{
    atomicCAS(&P.ctl->error, 0u, code);
}

// A wait gave up: the first one records where (for the host's error text).
__device__ __noinline__ void wait_failed(const LvArgs &P, unsigned long long site, unsigned long long t,
                                         unsigned long long want, unsigned long long s1,
                                         unsigned long long s2, unsigned long long s3)
{
    if (atomicCAS(&P.ctl->error, 0u, ST_TIMEOUT) == 0u) {
        unsigned long long *d = P.ctl->diag;
        d[0] = site;
        d[1] = blockIdx.x;
        d[2] = t;
        d[3] = want;
        d[4] = s1;
        d[5] = s2;
        d[6] = s3;
        __threadfence();
    }
}

// A helper CTA's copy of the job it claims from (read once per job).
struct JobDesc {
    const uint8_t *A, *B;
    int32_t n, m, x, y, lim; // (strings of the tile kernel are shorter than 2^31)
    uint32_t jid;
    int32_t slot;
    int32_t pq; // the pair whose strings A, B are (-1: none yet)
};
static_assert(sizeof(JobDesc) <= 64, "the job cache fills bytes 192..255 of the smem header");

// Bytes between consecutive stages (128-byte aligned).
constexpr size_t STAGE_STRIDE = (stage_bytes<CHUNK_BYTES>() + 127) & ~(size_t)127;

// The parts of a chunk's staging at p (128-byte aligned): A side, B side,
// mbarrier, phase word.
__device__ __forceinline__ Stage stage_of(unsigned char *p)
{
    Stage T;
    T.a = p;
    T.b = p + CHUNK_BYTES + 16;
    T.bar = reinterpret_cast<uint64_t *>(T.b + CHUNK_BYTES + 32);
    T.phase = reinterpret_cast<uint32_t *>(T.bar + 1);
    return T;
}

// Kept in registers: every function takes it by value (no address taken,
// no array member indexed at run time).
struct Smem {
    int32_t *F0, *F1;   // tile + halo frontier, smax + 2*HMAX + 2 entries each
    int32_t *ld;        // open slides: diagonal (lcap entries)
    // pipelined rounds: open lists by round parity (diagonal, start row;
    // OCAP entries each) and their counts, the deferred diagonals of a round
    int32_t *Ld0, *Ld1, *Lc0, *Lc1, *D;
    int *nL, *nD;       // by round parity
    int *left;          // a slider warp left a listed slide open (by round parity)
    int *kf;            // the target diagonal reached row n in the round before
    int *nR;            // deferred diagonals a slider warp computed (by round parity)
    int *n1;
    int *bc;            // 8 broadcast words
    long long *bcl;     // 4 broadcast 64-bit words
    unsigned long long *smin;
    JobDesc *jd;        // the job last claimed from
    int *jring;         // the CTA's next job slot (0 .. JOB_RING-1)
    unsigned char *stg; // bulk-copy staging of one chunk (null: none), see stage_of
    int lcap;
    uint32_t *err;             // launch status word (self-check records)
    unsigned long long *diag;
};

// Job slot protocol.  claim = (job id << 32) | count: every atomicAdd of 1
// claims chunk `count` (CHUNK_BYTES of each string) of the job the word
// names.  The job's descriptor words and every word a claimer writes back
// carry a job id in their high half: job ids grow with every job of a slot,
// and the answers are raised by red.max, so an answer of a job the slot no
// longer holds (from a claimer that fell behind) never overwrites one of the
// job it holds.  A slot is therefore reused with no wait for the claims of
// its last job, and nothing is cleared.  A claim that lands on a job
// published after the claimer looked is a claim of that job (the descriptor
// read after the atomic, and a fence, carries its id).
//   ans[c]  = (jid << 32) | job offset of the chunk's first mismatch (NOMIS: none)
//   result  = (jid << 32) | ~best  (so that red.max keeps the least offset)
constexpr uint32_t NOMIS = 0xffffffffu;

__device__ __forceinline__ bool claim_valid(unsigned long long w) { return (w >> 32) != 0; }

__device__ __forceinline__ void red_max_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("red.relaxed.gpu.global.max.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// The least mismatch offset of job jid in the result word w (lim: none
// reported, or the word is another job's).
__device__ __forceinline__ int64_t result_of(unsigned long long w, uint32_t jid, int64_t lim)
{
    return (uint32_t)(w >> 32) == jid ? min(lim, (int64_t)(uint32_t)~(uint32_t)w) : lim;
}

// Answers claim c of job jid: a mismatch at job offset r lowers the result,
// and the chunk's word records the answer (no order needed between them: the
// owner decides from the chunk words alone).
__device__ __forceinline__ void answer_claim(JobSlot *sl, uint32_t jid, int64_t c, int64_t r)
{
    const unsigned long long tg = (unsigned long long)jid << 32;
    if (r >= 0)
        red_max_u64(&sl->result, tg | (uint32_t)~(uint32_t)r);
    if (c >= 0 && c < JOB_MAX_CHUNKS)
        red_max_u64(&sl->ans[c], tg | (r >= 0 ? (uint32_t)r : NOMIS));
}

// Thread 0, after a claim w of slot s: whether its chunk is worth scanning
// (inside lim and below the best mismatch reported so far).  The job's
// descriptor is read into the CTA's cache once per job, after a fence that
// orders it behind the claim: x, y, lim and the pair (whose strings the
// launch's pair table holds), each word tagged with its job; words of
// another job mean the slot has moved on (the claim's job is over: nothing
// to scan).  best: the result word read along with the claim (~0: read it
// here).  A descriptor outside its strings is never scanned (self-check
// record 7).
__device__ __forceinline__ int claim_go(const LvArgs &P, const Smem S, JobSlot *sl, int s, unsigned long long w,
                                        unsigned long long best = ~0ull, const unsigned long long *pre = nullptr)
{
    const uint32_t jid = (uint32_t)(w >> 32);
    const int64_t c = (int64_t)(uint32_t)w;
    JobDesc *J = S.jd;
    if (J->jid != jid || J->slot != s) {
        // the words read along with the claim serve when they all carry its
        // job (each word holds its tag with its value); else read them again
        // behind a fence
        unsigned long long xt = 0, yt = 0, lt = 0, pt = 0;
        bool tags = false;
        if (pre) {
            xt = pre[0];
            yt = pre[1];
            lt = pre[2];
            pt = pre[3];
            tags = (uint32_t)(xt >> 32) == jid && (uint32_t)(yt >> 32) == jid && (uint32_t)(lt >> 32) == jid &&
                   (uint32_t)(pt >> 32) == jid;
        }
        if (!tags) {
            __threadfence();
            xt = ld_relaxed_u64(&sl->xt);
            yt = ld_relaxed_u64(&sl->yt);
            lt = ld_relaxed_u64(&sl->lt);
            pt = ld_relaxed_u64(&sl->pt);
            best = ld_relaxed_u64(&sl->result);
            if ((uint32_t)(xt >> 32) != jid || (uint32_t)(yt >> 32) != jid || (uint32_t)(lt >> 32) != jid ||
                (uint32_t)(pt >> 32) != jid) {
                J->jid = 0;
                return 0;
            }
        }
        // the pair's strings: the launch's pair table, read once per pair
        if (J->pq != (int32_t)(uint32_t)pt) {
            const PairDesc &D = P.pairs[(uint32_t)pt];
            J->A = D.A;
            J->B = D.B;
            J->n = (int32_t)D.n;
            J->m = (int32_t)D.m;
            J->pq = (int32_t)(uint32_t)pt;
        }
        J->x = (int32_t)(uint32_t)xt;
        J->y = (int32_t)(uint32_t)yt;
        J->lim = (int32_t)(uint32_t)lt;
        J->jid = jid;
        J->slot = s;
        if (J->x < 0 || J->y < 0 || J->lim < 0 || (int64_t)J->x + J->lim > J->n || (int64_t)J->y + J->lim > J->m ||
            !J->A || !J->B) {
            J->jid = 0;
            if (S.err && atomicCAS(S.err, 0u, 7u) == 0u) {
                S.diag[0] = 7;
                S.diag[1] = blockIdx.x;
                S.diag[2] = (unsigned long long)J->x;
                S.diag[3] = (unsigned long long)J->y;
                S.diag[4] = (unsigned long long)J->lim;
                S.diag[5] = (unsigned long long)J->n;
                S.diag[6] = (unsigned long long)J->m;
            }
            return 0;
        }
    } else if (best == ~0ull) {
        best = ld_relaxed_u64(&sl->result);
    }
    const int64_t cs = c * (int64_t)CHUNK_BYTES;
    return cs < result_of(best, jid, J->lim) ? 1 : 0;
}

// The first mismatch of A[x0..x0+len) vs B[y0..) (len <= CHUNK_BYTES), or
// -1: by bulk copies into the CTA's stage when it has one, else by one
// register sweep.  Whole CTA.  (A stage wait that gave up has set the launch
// status; the chunk then counts as equal and the launch reports the timeout.)
__device__ __forceinline__ int64_t chunk_scan(const LvArgs &P, const Smem S, const uint8_t *A, int64_t n,
                                              const uint8_t *B, int64_t m, int64_t x0, int64_t y0, int64_t len)
{
    if (S.stg) {
        const int64_t r = stage_scan<CHUNK_BYTES>(stage_of(S.stg), A, n, B, m, x0, y0, len, S.smin, P.spin_ns, S.err);
        return r >= 0 ? r : -1;
    }
    return sweep_scan<CHUNK_BYTES / (CTA_THREADS * 16)>(A, n, B, m, x0, y0, len, S.smin);
}

// The whole CTA scans claimed chunk c of job jid, cached in S.jd (when go),
// and answers the claim.
__device__ __forceinline__ void scan_claim(const LvArgs &P, const Smem S, JobSlot *sl, uint32_t jid, int64_t c,
                                           int go)
{
    int64_t r = -1;
    if (go) {
        const JobDesc J = *S.jd;
        const int64_t cs = c * (int64_t)CHUNK_BYTES;
        const int64_t q = chunk_scan(P, S, J.A, J.n, J.B, J.m, J.x + cs, J.y + cs,
                                     min((int64_t)CHUNK_BYTES, (int64_t)J.lim - cs));
        r = q >= 0 ? cs + q : -1;
    }
    if (threadIdx.x == 0)
        answer_claim(sl, jid, c, r);
}

// What ends a CTA's helping early: the first edge word of both neighbours
// (null: none) at round `want` or beyond, i.e. the CTA's own next block can
// (most likely) start.
struct Wake {
    const unsigned long long *lw, *rw;
    uint32_t want;
};
__device__ __forceinline__ bool wake_ready(const Wake *w)
{
    const unsigned long long a = w->lw ? ld_relaxed_u64(w->lw) : ~0ull;
    const unsigned long long b = w->rw ? ld_relaxed_u64(w->rw) : ~0ull;
    return (uint32_t)(a >> 32) >= w->want && (uint32_t)(b >> 32) >= w->want;
}

// The whole CTA claims and scans chunks of slot s's job, in order, up to
// `budget` claims: thread 0 makes the next claim before the current chunk
// is scanned, so that its round trip overlaps the scan.  w0: a claim made
// already (0: make the first one here).  Stops once a claimed chunk lies
// past the end or past the best mismatch, or its job is over (that claim is
// answered at once), or, with a Wake, once the CTA's neighbours are ready
// (checked along with each claim).  Returns the number of claims made and
// answered.
__device__ int claim_loop(const LvArgs &P, const Smem S, JobSlot *sl, int s, unsigned long long w0, int budget,
                          const Wake *wake = nullptr, unsigned long long best0 = ~0ull)
{
    const int tid = threadIdx.x;
    unsigned long long w = 0;     // thread 0: the current claim word
    unsigned long long best = best0; // thread 0: the result read with it (~0: none)
    if (tid == 0)
        w = w0 ? w0 : atomicAdd(&sl->claim, 1ull);
    int made = 0;
    for (;;) {
        if (tid == 0) {
            const bool ready = wake && wake_ready(wake);
            const int valid = claim_valid(w) ? 1 : 0;
            const int go = valid ? claim_go(P, S, sl, s, w, best) : 0;
            S.bc[0] = valid;
            S.bc[3] = go;
            S.bcl[0] = (long long)w;
            // the next claim and a look at the result, both in flight during
            // the scan below (this claim is still unanswered: the job cannot
            // change meanwhile)
            const bool next = go && !ready && made + 1 < budget;
            w = next ? atomicAdd(&sl->claim, 1ull) : 0ull;
            best = next ? ld_relaxed_u64(&sl->result) : ~0ull;
            S.bc[4] = next;
        }
        __syncthreads();
        const int valid = S.bc[0], go = S.bc[3], more = S.bc[4];
        const unsigned long long wc = (unsigned long long)S.bcl[0];
        __syncthreads();
        if (!valid)
            break;
        scan_claim(P, S, sl, (uint32_t)(wc >> 32), (int64_t)(uint32_t)wc, go);
        made++;
        if (!more)
            break;
    }
    return made;
}

// claim_loop through two shared-memory stages (budget > 1, P.stage >= 2):
// each claim's chunk is staged by bulk copies as soon as its claim word is
// back, while the chunk claimed before it is compared, and the claim after
// it is in flight meanwhile; so a helper has two chunks' bytes in flight.
// The same claims, answers and stopping rules as claim_loop.
__device__ int claim_loop2(const LvArgs &P, const Smem S, JobSlot *sl, int s, int budget, const Wake *wake)
{
    const int tid = threadIdx.x;
    const Stage T0 = stage_of(S.stg), T1 = stage_of(S.stg + STAGE_STRIDE);
    unsigned long long wn = 0, bestn = ~0ull; // thread 0: the claim in flight, the result read with it
    unsigned long long pre[4] = {0, 0, 0, 0};  // thread 0: the descriptor words read with the first claim
    if (tid == 0) {
        wn = atomicAdd(&sl->claim, 1ull);
        pre[0] = ld_relaxed_u64(&sl->xt);
        pre[1] = ld_relaxed_u64(&sl->yt);
        pre[2] = ld_relaxed_u64(&sl->lt);
        pre[3] = ld_relaxed_u64(&sl->pt);
        bestn = ld_relaxed_u64(&sl->result);
    }
    int made = 0, ps = 1;        // ps: the stage holding the pending chunk
    int pvalid = 0, pgo = 0;     // the pending claim (staged last turn)
    int64_t pc = 0;
    uint32_t pjid = 0;
    for (;;) {
        const int sn = ps ^ 1;   // the stage for the claim resolved this turn
        if (tid == 0) {
            // 1. the claim in flight: valid, worth a scan?
            const int nv = wn && claim_valid(wn) ? 1 : 0;
            const int ng = nv ? claim_go(P, S, sl, s, wn, bestn, made + pvalid == 0 ? pre : nullptr) : 0;
            const unsigned long long wc = wn;
            // 2. its copies, in flight while the pending chunk is compared
            if (ng) {
                const JobDesc &J = *S.jd;
                const int64_t cs = (int64_t)(uint32_t)wc * (int64_t)CHUNK_BYTES;
                stage_issue(sn ? T1 : T0, J.A, J.n, J.B, J.m, J.x + cs, J.y + cs,
                            min((int64_t)CHUNK_BYTES, (int64_t)J.lim - cs), true);
            }
            // 3. the claim after it, in flight meanwhile
            const bool ready = wake && wake_ready(wake);
            const bool more = ng && !ready && made + pvalid + nv < budget;
            wn = more ? atomicAdd(&sl->claim, 1ull) : 0ull;
            bestn = more ? ld_relaxed_u64(&sl->result) : ~0ull;
            S.bc[0] = nv;
            S.bc[3] = ng;
            S.bcl[0] = (long long)wc;
        }
        __syncthreads();
        const int nv = S.bc[0], ng = S.bc[3];
        const unsigned long long wcn = (unsigned long long)S.bcl[0];
        const int64_t nc = (int64_t)(uint32_t)wcn;
        __syncthreads();
        // 4. the pending chunk: compared (when worth it) and answered
        if (pvalid) {
            int64_t r = -1;
            if (pgo) {
                const JobDesc J = *S.jd;
                const int64_t cs = pc * (int64_t)CHUNK_BYTES;
                const Stage T = ps ? T1 : T0;
                const StagedChunk K = stage_issue(T, J.A, J.n, J.B, J.m, J.x + cs, J.y + cs,
                                                  min((int64_t)CHUNK_BYTES, (int64_t)J.lim - cs), false);
                if (stage_wait(T, P.spin_ns, S.err)) {
                    const int64_t q = stage_compare(T, K, S.smin);
                    r = q >= 0 ? cs + q : -1;
                }
            }
            if (tid == 0)
                answer_claim(sl, pjid, pc, r);
            made++;
        }
        // 5. the claim resolved this turn is the pending one now
        pvalid = nv;
        pgo = ng;
        pc = nc;
        pjid = (uint32_t)(wcn >> 32);
        ps = sn;
        if (!pvalid)
            break;
    }
    return made;
}

// Thread 0: an open job slot of another CTA, or -1.  The active bitmask
// over the slots (its first eight words loaded together) is read from a
// CTA-dependent bit on, so that helpers spread over jobs.
__device__ __forceinline__ int pick_slot(const LvArgs &P)
{
    int s = -1;
    const int nslot = (int)gridDim.x * JOB_RING;
    const int nw = (nslot + 63) >> 6;
    const volatile unsigned long long *act = P.ctl->active;
    unsigned long long b[8];
#pragma unroll
    for (int k = 0; k < 8; k++)
        b[k] = k < nw ? act[k] : 0ull;
    const int rot = blockIdx.x & 63;
    const int w0 = (int)(((int)blockIdx.x * JOB_RING / 64) % nw);
    for (int k = 0; k < nw && s < 0; k++) {
        const int wd = (w0 + k) % nw;
        unsigned long long v = 0ull;
#pragma unroll
        for (int q = 0; q < 8; q++)
            if (wd == q)
                v = b[q];
        if (wd >= 8)
            v = act[wd];
        v = (v >> rot) | (rot ? (v << (64 - rot)) : 0ull);
        while (v && s < 0) {
            const int j = wd * 64 + ((__ffsll((long long)v) - 1 + rot) & 63);
            v &= v - 1;
            if (j < nslot && j / JOB_RING != (int)blockIdx.x)
                s = j;
        }
    }
    return s;
}

// The whole CTA claims and scans chunks of slot s's job (s >= 0), up to
// `budget` claims.  Returns true if a claim was made.
__device__ __forceinline__ bool serve_slot(const LvArgs &P, const Smem S, int s, int budget, const Wake *wake)
{
    if (budget > 1 && S.stg && P.stage >= 2)
        return claim_loop2(P, S, &P.slots[s], s, budget, wake) > 0;
    return claim_loop(P, S, &P.slots[s], s, 0ull, budget, wake) > 0;
}

// One job of the CTA's long slide (whole CTA): the first mismatch of
// A[x..x+lim) vs B[y..), lim <= JOB_MAX_CHUNKS chunks, or lim.  The job goes
// into the CTA's next ring slot (no wait: see the protocol above), its
// chunk 0 claimed by the CTA itself; the other chunks are claimed in order by
// the CTA and by every CTA that is waiting on a neighbour or has no tile.
// The CTA watches the chunks' answer words: the job is done once every chunk
// before the first one with a mismatch (or every chunk) has answered.  It
// then takes its bit out of the active mask and returns; claims that come
// later find their chunk past the result and answer at once.
__device__ __noinline__ int64_t run_job(const LvArgs &P, const Smem S, const Pair Q, int64_t x, int64_t y,
                                        int64_t lim)
{
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t nch = (uint32_t)((lim + CHUNK_BYTES - 1) / CHUNK_BYTES);
    const int ring = *S.jring;
    const int sidx = (int)blockIdx.x * JOB_RING + ring;
    JobSlot *sl = &P.slots[sidx];
    const int word = sidx >> 6;
    const unsigned long long bit = 1ull << (sidx & 63);
    // ------------------------------------------------ publish
    if (tid == 0) {
        *S.jring = (ring + 1) % JOB_RING;
        uint32_t jid = (uint32_t)(ld_relaxed_u64(&sl->claim) >> 32) + 1u;
        jid = jid ? jid : 1u;
        const unsigned long long tg = (unsigned long long)jid << 32;
        sl->xt = tg | (uint32_t)x;
        sl->yt = tg | (uint32_t)y;
        sl->lt = tg | (uint32_t)lim;
        sl->pt = tg | (uint32_t)Q.q;
        sl->result = tg | (uint32_t)~(uint32_t)lim;
        // the CTA's own cache holds the job: no read back
        JobDesc *J = S.jd;
        J->A = Q.A;
        J->B = Q.B;
        J->n = (int32_t)Q.n;
        J->m = (int32_t)Q.m;
        J->pq = Q.q;
        J->x = (int32_t)x;
        J->y = (int32_t)y;
        J->lim = (int32_t)lim;
        J->jid = jid;
        J->slot = sidx;
        // count 1: chunk 0 is the CTA's own claim; the descriptor is visible
        // before the claim word (release), which opens the job, and before
        // the active bit (release)
        st_release_u64(&sl->claim, tg | 1ull);
        asm volatile("red.release.gpu.global.or.b64 [%0], %1;" ::"l"(&P.ctl->active[word]), "l"(bit) : "memory");
        S.bcl[2] = (long long)tg;
    }
    __syncthreads();
    const unsigned long long w0 = (unsigned long long)S.bcl[2];
    const uint32_t jid = (uint32_t)(w0 >> 32);
    __syncthreads();
    claim_loop(P, S, sl, sidx, w0, 1, nullptr, w0 | (uint32_t)~(uint32_t)lim); // chunk 0
    // ------------------------------------------------ watch
    // warp 0 loads the answer words of the next WATCH_WORDS * 32 chunks from
    // `base` on (every chunk below base has answered without a mismatch),
    // several looks before the CTA meets at a barrier.  With no progress for
    // OWN_SCAN_NS (no helper at hand), the CTA claims a chunk itself, or scans
    // the claimed chunk at base again itself.
    uint32_t base = 0, last = 1;
    uint64_t tnew = gtimer(); // lane 0: when the job last moved
    for (;;) {
        if (tid < 32) {
            int act = 0; // 0 look again, 1 claim a chunk, 2 final, 3 scan chunk base itself
            unsigned long long best = 0;
            for (int spin = 0; spin < WATCH_SPINS && act == 0; spin++) {
                const uint32_t cnt = (uint32_t)ld_relaxed_u64(&sl->claim);
                unsigned long long v[WATCH_WORDS];
#pragma unroll
                for (int i = 0; i < WATCH_WORDS; i++) {
                    const uint32_t c = base + 32u * (uint32_t)i + (uint32_t)lane;
                    v[i] = c < nch ? ld_relaxed_u64(&sl->ans[c]) : (w0 | NOMIS);
                }
                uint32_t nb = base;
#pragma unroll
                for (int i = 0; i < WATCH_WORDS; i++) {
                    if (act != 0 || nb != base + 32u * (uint32_t)i)
                        break;
                    const bool a = (uint32_t)(v[i] >> 32) == jid;
                    const bool mis = a && (uint32_t)v[i] != NOMIS;
                    const unsigned int A = __ballot_sync(0xffffffffu, a), M = __ballot_sync(0xffffffffu, mis);
                    const int fu = ~A ? __ffs((int)~A) - 1 : 32; // first unanswered
                    const int fm = M ? __ffs((int)M) - 1 : 32;   // first mismatch
                    if (fm < fu) {
                        best = __shfl_sync(0xffffffffu, (uint32_t)v[i], fm);
                        act = 2;
                    } else if (fu < 32) {
                        nb += (uint32_t)fu;
                    } else {
                        nb += 32;
                        if (nb >= nch) {
                            best = (unsigned long long)lim;
                            act = 2;
                        }
                    }
                }
                if (act == 0 && lane == 0) {
                    const uint64_t now = gtimer();
                    if (nb != base || cnt != last) {
                        last = cnt;
                        tnew = now;
                    } else if (now - tnew > OWN_SCAN_NS) {
                        // the chunk at base: claimed and slow (scan it again
                        // here), or not claimed yet (claim it)
                        act = nb < cnt ? 3 : 1;
                        tnew = now;
                    }
                }
                base = nb;
                act = __shfl_sync(0xffffffffu, act, 0);
            }
            if (lane == 0) {
                S.bc[5] = act;
                S.bcl[1] = (long long)best;
                S.bc[6] = (int)base;
            }
        }
        __syncthreads();
        const int act = S.bc[5];
        const int64_t best = S.bcl[1];
        const int64_t cb = S.bc[6];
        __syncthreads();
        if (act == 2) {
            if (tid == 0)
                asm volatile("red.relaxed.gpu.global.and.b64 [%0], %1;" ::"l"(&P.ctl->active[word]), "l"(~bit)
                             : "memory");
            return best;
        }
        if (act == 1)
            claim_loop(P, S, sl, sidx, 0ull, 1);
        if (act == 3)
            scan_claim(P, S, sl, jid, cb, 1);
    }
}

// The CTA's own long slide: the first mismatch of A[x..x+lim) vs B[y..).
// The CTA scans the first local_chunks chunks alone (after one bulk L2
// prefetch of all of them); the rest goes to jobs of at most JOB_MAX_CHUNKS
// chunks each, helped by other CTAs.  Returns the first mismatch offset, or
// lim.
__device__ __noinline__ int64_t long_slide(const LvArgs &P, const Smem S, const Pair Q, int64_t x0,
                                           int64_t y0, int64_t lim0)
{
    const int tid = threadIdx.x;
    const int64_t loc = min(lim0, (int64_t)max(0, P.local_chunks) * CHUNK_BYTES);
    if (tid == 0 && loc > CHUNK_BYTES) {
        bulk_prefetch_l2(Q.A, Q.n, x0 + CHUNK_BYTES, loc - CHUNK_BYTES);
        bulk_prefetch_l2(Q.B, Q.m, y0 + CHUNK_BYTES, loc - CHUNK_BYTES);
    }
    int64_t off = 0;
    if (S.stg && P.stage >= 2 && loc > CHUNK_BYTES) {
        // the chunks in turn through two stages, the next one's copies in flight
        const int64_t r = stream_scan<CHUNK_BYTES>(stage_of(S.stg), stage_of(S.stg + STAGE_STRIDE), Q.A, Q.n, Q.B,
                                                   Q.m, x0, y0, loc, S.smin, P.spin_ns, S.err);
        if (r < loc)
            return r >= 0 ? r : lim0; // (-2: a wait gave up; the launch reports it)
        off = loc;
    }
    for (; off < loc; off += CHUNK_BYTES) {
        const int64_t r = chunk_scan(P, S, Q.A, Q.n, Q.B, Q.m, x0 + off, y0 + off, min((int64_t)CHUNK_BYTES, lim0 - off));
        if (r >= 0)
            return off + r;
    }
    while (off < lim0) {
        const int64_t len = min(lim0 - off, (int64_t)JOB_MAX_CHUNKS * CHUNK_BYTES);
        const int64_t r = run_job(P, S, Q, x0 + off, y0 + off, len);
        if (r < len)
            return off + r;
        off += len;
    }
    return lim0;
}

// ------------------------------------------------------------------ group
// Bounded barrier over the G CTAs of a group, on (count, gen).  Returns 1
// when all arrived, 0 on error or timeout, 2 when `abandon` is set and the
// group's k became known meanwhile (the epoch-change barrier: CTAs that
// have seen k leave the pair without arriving).
__device__ int group_barrier(const LvArgs &P, GroupCtl *gc, uint32_t *count, uint32_t *gen_p, int G,
                             bool abandon, const Smem S)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint32_t gen = ld_acquire(gen_p);
        __threadfence();
        const uint32_t arrived = atomicAdd(count, 1u);
        if (arrived == (uint32_t)G - 1) {
            atomicExch(count, 0u);
            __threadfence();
            st_release(gen_p, gen + 1);
        } else {
            const uint64_t t0 = gtimer();
            while (ld_acquire(gen_p) == gen) {
                if (ld_acquire(&P.ctl->error) != 0) {
                    ok = 0;
                    break;
                }
                if (abandon && *(volatile unsigned long long *)&gc->done_k != ~0ull) {
                    ok = 2;
                    break;
                }
                if (gtimer() - t0 > P.idle_ns) {
                    wait_failed(P, abandon ? 5 : 2, 0, gen, ld_acquire(count), G, 0);
                    ok = 0;
                    break;
                }
            }
        }
        S.bc[2] = ok;
    }
    __syncthreads();
    const int ok = S.bc[2];
    __syncthreads();
    return ok;
}

__device__ bool group_sync(const LvArgs &P, GroupCtl *gc, int G, const Smem S)
{
    return group_barrier(P, gc, &gc->bar_count, &gc->bar_gen, G, false, S) == 1;
}

constexpr int OCAP = 1024;     // open slides listed per round (pipelined rounds)
constexpr int DCAP = 3 * OCAP; // deferred diagonals: neighbours of open ones

size_t lv_tiles_smem_bytes(int smax, int h, int stage)
{
    (void)h;
    // two frontier buffers and the open-slide list, each smax + 2*HMAX + 2;
    // two open lists of OCAP (diagonal, start row); DCAP deferred diagonals;
    // then, with a stage, one chunk's bulk-copy staging (128-byte aligned)
    return 256 + 3 * sizeof(int32_t) * ((size_t)smax + 2 * HMAX + 2) +
           sizeof(int32_t) * (4 * (size_t)OCAP + DCAP) + (stage ? 128 + (size_t)stage * STAGE_STRIDE : 0);
}

// The frontier of round r (buffers alternate by parity).
__device__ __forceinline__ int32_t *frontier(const Smem S, int64_t r) { return (r & 1) ? S.F1 : S.F0; }

__device__ Smem carve(const LvArgs &P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem S;
    unsigned char *p = smem_raw;
    S.smin = reinterpret_cast<unsigned long long *>(p);
    S.bcl = reinterpret_cast<long long *>(p + 16);
    S.n1 = reinterpret_cast<int *>(p + 64);
    S.bc = S.n1 + 4;
    S.nL = reinterpret_cast<int *>(p + 128);
    S.nD = S.nL + 2;
    S.left = S.nL + 4;
    S.kf = S.nL + 6;
    S.nR = S.nL + 7;
    S.jd = reinterpret_cast<JobDesc *>(p + 192);
    S.jring = reinterpret_cast<int *>(p + 48);
    // p + 176: lone (lean_slides); p + 184: the tile's lead at an epoch change
    p += 256;
    S.lcap = P.smax + 2 * HMAX + 2;
    S.ld = reinterpret_cast<int32_t *>(p);
    p += sizeof(int32_t) * S.lcap;
    S.F0 = reinterpret_cast<int32_t *>(p);
    p += sizeof(int32_t) * (P.smax + 2 * HMAX + 2);
    S.F1 = reinterpret_cast<int32_t *>(p);
    p += sizeof(int32_t) * (P.smax + 2 * HMAX + 2);
    S.Ld0 = reinterpret_cast<int32_t *>(p);
    S.Ld1 = S.Ld0 + OCAP;
    S.Lc0 = S.Ld1 + OCAP;
    S.Lc1 = S.Lc0 + OCAP;
    S.D = S.Lc1 + OCAP;
    p = reinterpret_cast<unsigned char *>(S.D + DCAP);
    S.stg = P.stage ? reinterpret_cast<unsigned char *>(((uintptr_t)p + 127) & ~(uintptr_t)127) : nullptr;
    S.err = &P.ctl->error;
    S.diag = P.ctl->diag;
    return S;
}

struct Tile {
    int64_t lo_all, hi_all, S;
    int64_t a, b; // own diagonals [a, b)
    int ntiles;
    bool has;
    int left, right; // neighbour CTA (grid index) or -1
};

// While the band is narrow (fewer than HELP_BAND diagonals per CTA), the
// last G / help_div CTAs of a group of at least 2 * help_div CTAs hold no
// tile: they serve the chunks of long slides as soon as they are published
// (the rounds of a narrow band are bound by their latency, not by the
// diagonals per CTA).
constexpr int64_t HELP_BAND = 256;

// The tiles' grid is shifted so that diagonal dp (the band's furthest row:
// the alignment path) lies in the middle of its tile, when the one more tile
// this may take is at hand: the path's long slides then run in one tile only,
// not also in its neighbour's halo.
__device__ __forceinline__ Tile partition(const Pair &Q, int64_t R, int G, int gi, int c0, int h, int help_div,
                                          int64_t smax, int64_t dp)
{
    Tile T;
    T.lo_all = max(-R, -Q.n);
    T.hi_all = min(R, Q.m);
    const int64_t N = T.hi_all - T.lo_all + 1;
    int Gt = G;
    if (help_div > 0 && G >= 2 * help_div && N < HELP_BAND * G) {
        const int g2 = G - G / help_div;
        if ((N + g2 - 1) / g2 <= smax) // the tiles still fit the shared memory
            Gt = g2;
    }
    T.S = max((int64_t)h, (N + Gt - 1) / Gt);
    int64_t sh = 0;
    if (dp >= T.lo_all && dp <= T.hi_all) {
        sh = ((T.S / 2 - (dp - T.lo_all)) % T.S + T.S) % T.S;
        if ((N + sh + T.S - 1) / T.S > G)
            sh = 0;
    }
    T.ntiles = (int)((N + sh + T.S - 1) / T.S);
    T.has = gi < T.ntiles;
    T.a = max(T.lo_all, T.lo_all + (int64_t)gi * T.S - sh);
    T.b = min(T.hi_all + 1, T.lo_all + (int64_t)(gi + 1) * T.S - sh);
    T.left = (T.has && gi > 0) ? c0 + gi - 1 : -1;
    T.right = (T.has && gi + 1 < T.ntiles) ? c0 + gi + 1 : -1;
    return T;
}

// A tile's edge values of round t - 1 for its neighbours, one word each:
// (t << 32) | L in a single 8-byte store, so that a reader that sees the
// round sees the value with it (no fence, no flag).  Parity (t / h) & 1
// alternates the buffers: a tile can be one block ahead of its neighbour at
// most, so it never overwrites a word its neighbour has still to read.
__device__ __forceinline__ unsigned long long halo_word(uint32_t t, int32_t v)
{
    return ((unsigned long long)t << 32) | (uint32_t)v;
}

__device__ __forceinline__ unsigned long long *halo_ptr(const LvArgs &P, int cta, int parity, int side)
{
    return P.halo + ((int64_t)(cta * 2 + parity) * 2 + side) * HMAX;
}

// The bound of an open slide of diagonal d from row c: the string end, or
// the hash answer + 1 (the slide confirms it directly).
__device__ __forceinline__ int64_t open_limit(const LvArgs &P, const Pair &Q, int64_t c, int64_t d, Counters &C,
                                              bool own)
{
    const int64_t full = min(Q.n - c, Q.m - c - d);
    int64_t lim = full;
    if (Q.hash && full > 0) {
        const int64_t h = hash_lcp(P.pow2, HashView{Q.TA, Q.A, P.hash_b}, HashView{Q.TB, Q.B, P.hash_b}, c,
                                   c + d, 0, full);
        C.hashq += own;
        lim = min(h + 1, full);
    }
    return c + lim;
}

// The open slides listed in Ld/Lc (diagonal, start row) for the frontier fr:
// one warp each, up to t2_cap bytes (warps w0, w0 + ws, ...); the final row
// goes to fr and the entry's diagonal becomes INT32_MIN.  Entries still open
// are left for cta_slides.
//
// nb (pipelined rounds): round tau, whose diagonals next to a slide of
// round tau - 1 wait for it (DEFER_MARK).  Once a slide is done, lanes 0..2
// claim its three neighbours in round tau and compute them (the bytes at
// the slide's end are in L1), unless another predecessor is still open;
// *nr counts those computed.
__device__ __forceinline__ void warp_slides(const LvArgs &P, const Pair &Q, int32_t *fr, int64_t off, int32_t *Ld,
                                            const int32_t *Lc, int nl, int64_t a, int64_t b, int w0, int ws,
                                            Counters &C, int *left, const RoundArgs *nb = nullptr, int *nr = nullptr)
{
    const int lane = threadIdx.x & 31;
    for (int j = w0; j < nl; j += ws) {
        const int64_t d = Ld[j], c = Lc[j];
        const bool own = d >= a && d < b;
        int64_t lim = 0;
        if (lane == 0) {
            lim = open_limit(P, Q, c, d, C, own);
            C.opens += own;
        }
        lim = __shfl_sync(0xffffffffu, lim, 0);
        bool open;
        const int64_t l = slide_warp(Q.A, Q.n, Q.B, Q.m, c, c + d, 0, lim - c, P.t2_cap, &open);
        if (!open && l >= PREFETCH_MIN) // a long slide: the next round starts past it
            prefetch_next(Q.A, Q.n, Q.B, Q.m, c + l, c + l + d);
        if (lane == 0 && !open) {
            fr[d - off] = (int32_t)finish_slide(Q, c, d, c + l, lim, own, C);
            Ld[j] = INT32_MIN; // finished
        }
        if (lane == 0 && open && left)
            *left = 1;
        if (nb && !open) {
            __syncwarp(); // the final row, written by lane 0
            const int32_t e = (int32_t)d - 1 + lane;
            if (lane < 3 && e >= nb->lo && e <= nb->hi) {
                int32_t *cp = nb->cur + (e - nb->off);
                if (atomicCAS(cp, DEFER_MARK, DEFER_CLAIM) == DEFER_MARK) {
                    RoundCount rc = {0, 0};
                    if (round_one(*nb, e, rc)) {
                        C.slide += rc.slide;
                        C.mism += rc.mism;
                        atomicAdd(nr, 1);
                    } else {
                        atomicExch(cp, DEFER_MARK); // the deferred pass takes it
                    }
                }
            }
            __syncwarp();
        }
    }
}

// The listed slides a warp left open: the whole CTA each (and beyond 128
// KiB the job slots).  Every thread must call it, after a barrier; the
// final rows are visible to every thread when it returns.
__device__ __forceinline__ void cta_slides(const LvArgs &P, const Smem S, const Pair &Q, int32_t *fr, int64_t off,
                                           const int32_t *Ld, const int32_t *Lc, int nl, int64_t a, int64_t b,
                                           Counters &C)
{
    const int tid = threadIdx.x;
    bool any = false;
    for (int j = 0; j < nl; j++) {
        const int64_t d = Ld[j];
        if (d == INT32_MIN)
            continue;
        any = true;
        const int64_t c = Lc[j];
        const bool own = d >= a && d < b;
        if (tid == 0)
            S.bcl[3] = open_limit(P, Q, c, d, C, false);
        __syncthreads();
        const int64_t lim = S.bcl[3];
        __syncthreads();
        const int64_t rr = long_slide(P, S, Q, c, c + d, lim - c);
        if (lim - c > (int64_t)max(0, P.local_chunks) * CHUNK_BYTES) // published as a job
            C.longs++;
        if (tid < 32)
            prefetch_next(Q.A, Q.n, Q.B, Q.m, c + rr, c + rr + d);
        if (tid == 0)
            fr[d - off] = (int32_t)finish_slide(Q, c, d, c + rr, lim, own, C);
    }
    if (any) // (every thread saw the same entries)
        __syncthreads();
}

// What one block of rounds adds to the counters, and whether it found k.
struct BlockOut {
    unsigned long long slide, mism, hashq, coll, longs, opens, tm_round, tm_open;
    int fin;
};

// The round arguments of round tau on the tile [a, b) with smem offset off.
__device__ __forceinline__ RoundArgs round_args(const LvArgs &P, const Smem S, const Pair &Q, int64_t tau,
                                                int64_t lo, int64_t hi, int64_t off, int64_t a, int64_t b)
{
    RoundArgs RA;
    RA.A = Q.A;
    RA.B = Q.B;
    RA.n = Q.n;
    RA.m = Q.m;
    RA.prev = frontier(S, tau - 1);
    RA.cur = frontier(S, tau);
    RA.off = off;
    RA.lo = lo;
    RA.hi = hi;
    RA.tau = tau;
    RA.a = a;
    RA.b = b;
    RA.err = &P.ctl->error;
    RA.diag = P.ctl->diag;
    RA.n1 = S.nL + (tau & 1);
    RA.open = (tau & 1) ? S.Ld1 : S.Ld0;
    RA.open_c = (tau & 1) ? S.Lc1 : S.Lc0;
    RA.ocap = OCAP;
    RA.defer = S.D;
    RA.nd = S.nD + (tau & 1);
    RA.list = nullptr;
    RA.nlist = 0;
    RA.tid = threadIdx.x;
    RA.nt = blockDim.x;
    return RA;
}

// Rounds t .. t+h-1 on the tile [a, b) and its shrinking halo trapezoid,
// pipelined: while six warps compute round tau for every diagonal whose
// predecessors are final, warps 3 and 7 finish the open slides of round
// tau - 1 (the path's slide of about n/k bytes, every round, and the
// chance matches beside it, in parallel); the diagonals
// next to those slides are deferred and computed once they are final.  A
// listed slide a warp cannot finish goes to the whole CTA.  The last round's
// open slides are finished by all warps before the block ends (its edges go
// to the neighbours).  Round tau - 1 is final after round tau's slide phase:
// the termination test and the frontier dump see only final rows.  Two
// barriers a round (three with a frontier dump): the open and deferred
// counts alternate by round parity, and thread 0 tests round tau - 1 for
// termination before the second.
__device__ __forceinline__ BlockOut run_block(const LvArgs &P, const Smem S, const Pair Q, int32_t *dump,
                                          int32_t dump_tmax, unsigned long long *res, GroupCtl *gc, int64_t t,
                                          int h, int64_t a, int64_t b)
{
    const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, nw = nt >> 5;
    // the slider warps are the last of each group of four (warps 3 and 7);
    // the other six compute the round
    const bool slider = (warp & 3) == 3;
    const int nsl = nw / 4, sli = warp >> 2;
    const int64_t n = Q.n, m = Q.m, target = m - n;
    const int64_t off = a - h - 1; // smem index = d - off
    Counters C;
    int64_t kfound = -1;
    // is row tau of the target diagonal n?  (tau's band holds it and it is this tile's)
    auto hit = [=](int64_t tau) {
        const int64_t blo = max(-tau, -n), bhi = min(tau, m);
        return target >= a && target < b && target >= blo && target <= bhi &&
               frontier(S, tau)[target - off] == n;
    };
    auto dump_row = [=](int64_t tau) {
        if (dump && tau <= dump_tmax) {
            const int64_t TT = dump_tmax;
            const int32_t *fr = frontier(S, tau);
            for (int64_t d = max(a, -TT) + tid; d < min(b, TT + 1); d += nt)
                dump[tau * (2 * TT + 1) + d + TT] = fr[d - off];
        }
    };
    if (tid == 0) {
        S.nL[0] = S.nL[1] = 0;
        S.nD[0] = S.nD[1] = 0;
        S.left[0] = S.left[1] = 0;
        S.nR[0] = S.nR[1] = 0;
    }
    __syncthreads();
    int r = 0;
    for (; r < h && kfound < 0; r++) {
        const uint64_t tr0 = clock64();
        const int64_t tau = t + r;
        const int64_t ra = a - h + 1 + r, rb = b + h - 1 - r; // computed range [ra, rb)
        const int64_t blo = max(-tau, -n), bhi = min(tau, m);
        int32_t *cur = frontier(S, tau);
        int32_t *prev = frontier(S, tau - 1);
        // outside the band (past either of its ends): minus infinity
        for (int64_t d = ra + tid; d < min(rb, blo); d += nt)
            cur[d - off] = NEG;
        for (int64_t d = max(ra, bhi + 1) + tid; d < rb; d += nt)
            cur[d - off] = NEG;
        const int pp = (int)((tau - 1) & 1);
        int32_t *Ldp = pp ? S.Ld1 : S.Ld0;
        const int32_t *Lcp = pp ? S.Lc1 : S.Lc0;
        const int nlp = r > 0 ? min(S.nL[pp], OCAP) : 0;
        // -------- phase 1: the slides of round tau - 1 || round tau
        if (slider) {
            const RoundArgs RN = round_args(P, S, Q, tau, max(ra, blo), min(rb - 1, bhi), off, a, b);
            warp_slides(P, Q, prev, off, Ldp, Lcp, nlp, a, b, sli, nsl, C, S.left + (tau & 1), &RN,
                        S.nR + (tau & 1));
        } else {
            RoundArgs RA = round_args(P, S, Q, tau, max(ra, blo), min(rb - 1, bhi), off, a, b);
            RA.tid = tid - 32 * sli;
            RA.nt = nt - 32 * nsl;
            // one diagonal per thread when the range fits (narrow bands):
            // the wide form's unrolled batch would be mostly idle slots
            const RoundCount rc = RA.hi - RA.lo < RA.nt ? tile_round<1, true>(RA)
                                                        : tile_round<2048 / CTA_THREADS, true>(RA);
            C.slide += rc.slide;
            C.mism += rc.mism;
        }
        __syncthreads();
        // -------- phase 2: slides the warp left open, then the deferred diagonals
        if (nlp > 0 && S.left[tau & 1])
            cta_slides(P, S, Q, prev, off, Ldp, Lcp, nlp, a, b, C);
        const int nd = S.nD[tau & 1];                   // deferred diagonals listed
        const bool marked = nd > S.nR[tau & 1];          // not all computed by a slider warp
        if (tid == 0) {
            // round tau - 1's list is consumed (every thread read its count
            // before the first barrier); the same parity's counts serve round
            // tau + 1 (round tau - 1's deferred count was last read before
            // the second barrier of round tau - 1)
            S.nL[pp] = 0;
            S.nD[pp] = 0;
            S.left[pp] = 0;
            S.nR[pp] = 0;
            // round tau - 1 is final here for thread 0: the slider's rows
            // before the first barrier, the CTA's slides by thread 0 itself
            *S.kf = r > 0 && hit(tau - 1);
        }
        if (marked) {
            RoundArgs RA = round_args(P, S, Q, tau, 0, -1, off, a, b);
            RA.list = S.D;
            RA.nlist = nd;
            const RoundCount rc = tile_round<1, true, true>(RA);
            C.slide += rc.slide;
            C.mism += rc.mism;
        }
        __syncthreads();
        // round tau - 1 is final now (round tau is tested in the next round,
        // or below if tau ends the block)
        if (*S.kf)
            kfound = tau - 1;
        if (dump) {
            // round tau + 1 overwrites this buffer
            if (r > 0)
                dump_row(tau - 1);
            __syncthreads();
        }
        C.tm[0] += clock64() - tr0;
    }
    // -------- the last computed round's open slides: all warps
    const uint64_t to0 = clock64();
    const int64_t tl = t + r - 1;
    if (kfound < 0 || kfound == tl) {
        const int pl = (int)(tl & 1);
        int32_t *Ldl = pl ? S.Ld1 : S.Ld0;
        const int32_t *Lcl = pl ? S.Lc1 : S.Lc0;
        const int nll = min(S.nL[pl], OCAP);
        if (nll > 0) {
            warp_slides(P, Q, frontier(S, tl), off, Ldl, Lcl, nll, a, b, warp, nw, C, nullptr);
            __syncthreads();
            cta_slides(P, S, Q, frontier(S, tl), off, Ldl, Lcl, nll, a, b, C);
            __syncthreads();
        }
        dump_row(tl);
        if (kfound < 0 && hit(tl))
            kfound = tl;
    }
    C.tm[1] += clock64() - to0;
    if (kfound >= 0 && tid == 0) {
        atomicMin(&gc->done_k, (unsigned long long)kfound);
        res[R_K] = (unsigned long long)kfound;
    }
    __syncthreads();
    return BlockOut{C.slide, C.mism, C.hashq, C.coll, C.longs, C.opens, C.tm[0], C.tm[1], kfound >= 0 ? 1 : 0};
}

// The open slides of a lean round (out of line: most rounds have none):
// one warp each, up to t2_cap bytes, then the whole CTA for those still
// open -- or, for a lone slide after a lone one that outran its warp, the
// whole CTA at once.  Every thread calls it (after a barrier); the final
// rows are visible to every thread when it returns.
__device__ __forceinline__ void lean_slides(const LvArgs &P, const Smem S, const Pair Q, int32_t *cur, int64_t off,
                                         int32_t *Ld, const int32_t *Lc, int nlo, int64_t a, int64_t b, int pr,
                                         Counters &C)
{
    // lone: whether the CTA's last lone slide outran one warp (t2_cap bytes);
    // the next lone one then goes to the whole CTA at once (its job opens
    // without the warp's step first): on the alignment path, slides long
    // and short come in runs
    int *lone = reinterpret_cast<int *>(reinterpret_cast<unsigned char *>(S.jring) + 128);
    const bool direct = nlo == 1 && *lone != 0;
    if (direct) {
        cta_slides(P, S, Q, cur, off, Ld, Lc, nlo, a, b, C);
    } else {
        const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        warp_slides(P, Q, cur, off, Ld, Lc, nlo, a, b, warp, nw, C, S.left + pr);
        __syncthreads();
        if (S.left[pr])
            cta_slides(P, S, Q, cur, off, Ld, Lc, nlo, a, b, C);
    }
    if (threadIdx.x == 0) {
        if (nlo == 1)
            *lone = direct ? (cur[Ld[0] - off] - Lc[0] > P.t2_cap) : S.left[pr];
        S.left[pr] = 0;
    }
    __syncthreads();
}

// Rounds t .. t+h-1 on a narrow tile (the trapezoid, tile and halos, fits
// two diagonals per thread): every thread computes its diagonals of the round
// (start row from the three predecessors, then the word slide); after one
// barrier the slides the words left open, if any, go to one warp each (up to
// t2_cap bytes) and then to the whole CTA; every thread then reads the
// termination test of the round itself from the final row of d = m - n.
// One barrier a round when no slide is left open, three when one is.
__device__ __forceinline__ BlockOut run_block_lean(const LvArgs &P, const Smem S, const Pair Q, int32_t *dump,
                                                int32_t dump_tmax, unsigned long long *res, GroupCtl *gc, int64_t t,
                                                int h, int64_t a, int64_t b)
{
    const int tid = threadIdx.x;
    const int64_t n = Q.n, m = Q.m, target = m - n;
    const int32_t n32 = (int32_t)n, m32 = (int32_t)m, mn = (int32_t)(m - n);
    const int64_t off = a - h - 1; // smem index = d - off
    Counters C;
    int64_t kfound = -1;
    if (tid == 0) {
        S.nL[0] = S.nL[1] = 0;
        S.left[0] = S.left[1] = 0;
    }
    __syncthreads();
    int r = 0;
    for (; r < h && kfound < 0; r++) {
        const uint64_t tr0 = clock64();
        const int64_t tau = t + r;
        const int pr = (int)(tau & 1);
        const int32_t ra = (int32_t)(a - h + 1 + r), rb = (int32_t)(b + h - 1 - r); // computed range [ra, rb)
        const int32_t blo = (int32_t)max(-tau, -n), bhi = (int32_t)min(tau, m);
        int32_t *cur = frontier(S, tau);
        const int32_t *prev = frontier(S, tau - 1);
        int32_t *Ld = pr ? S.Ld1 : S.Ld0;
        int32_t *Lc = pr ? S.Lc1 : S.Lc0;
        int *nl = S.nL + pr;
        for (int32_t d = ra + tid; d < rb; d += (int32_t)blockDim.x) {
            if (d < blo || d > bhi) {
                cur[d - off] = NEG;
            } else {
                int32_t cc = 0;
                if (tau > 0) {
                    const int32_t x1 = prev[d - 1 - off], x2 = prev[d - off], x3 = prev[d + 1 - off];
                    cc = min(max(x1, max(x2, x3) + 1), d <= mn ? n32 : m32 - d);
                }
                if (cc < 0 || cc + d < 0) {
                    record_bad_row(S.err, S.diag, tau, prev, (int32_t)off, d, cc);
                    cur[d - off] = NEG;
                } else {
                    const int32_t full = min(n32 - cc, m32 - cc - d);
                    int32_t l = 0;
                    if (full > 0) {
                        uint2 wa, wb;
                        uint32_t sh;
                        words_load(Q.A, Q.B, n32, m32, cc, d, wa, wb, sh);
                        l = words_lcp(wa, wb, sh, full);
                        if (l < 0) {
                            // every byte the words hold matched: 16 more bytes
                            // of each string in one round trip (the short runs
                            // inside a burst of edits end here) before the
                            // slide is listed for a warp
                            const int32_t k = 8 - (int32_t)max(sh & 255u, sh >> 8);
                            const uintptr_t pa = (uintptr_t)(Q.A + cc + k), pb = (uintptr_t)(Q.B + (cc + k + d));
                            const uintptr_t qa = pa & ~(uintptr_t)15, qb = pb & ~(uintptr_t)15;
                            const uint4 a0 = ld_blk_nb(Q.A, n, qa), a1 = ld_blk_nb(Q.A, n, qa + 16);
                            const uint4 b0 = ld_blk_nb(Q.B, m, qb), b1 = ld_blk_nb(Q.B, m, qb + 16);
                            const int32_t f = first_diff16(shift_bytes(a0, a1, (uint32_t)(pa & 15)),
                                                           shift_bytes(b0, b1, (uint32_t)(pb & 15)));
                            if (k + f >= full)
                                l = full;
                            else if (f < 16)
                                l = k + f;
                        }
                    }
                    if (l >= 0) {
                        cur[d - off] = cc + l;
                        if (d >= a && d < b) {
                            C.slide += (uint32_t)l;
                            C.mism += (l < full);
                        }
                    } else {
                        const int j = atomicAdd(nl, 1); // at most two per thread: the list cannot fill
                        Ld[j] = d;
                        Lc[j] = cc;
                        cur[d - off] = PENDING;
                    }
                }
            }
        }
        if (tid == 0)
            S.nL[pr ^ 1] = 0; // the other parity's list is free again
        __syncthreads();
        const int nlo = *nl;
        if (nlo > 0)
            lean_slides(P, S, Q, cur, off, Ld, Lc, nlo, a, b, pr, C);
        // the round is final: every thread reads the termination test
        if (target >= a && target < b && target >= blo && target <= bhi && cur[target - off] == n32)
            kfound = tau;
        if (dump && tau <= dump_tmax) {
            const int64_t TT = dump_tmax;
            for (int64_t e = max(a, -TT) + tid; e < min(b, TT + 1); e += blockDim.x)
                dump[tau * (2 * TT + 1) + e + TT] = cur[e - off];
        }
        C.tm[0] += clock64() - tr0;
    }
    if (kfound >= 0 && tid == 0) {
        atomicMin(&gc->done_k, (unsigned long long)kfound);
        res[R_K] = (unsigned long long)kfound;
    }
    __syncthreads();
    return BlockOut{C.slide, C.mism, C.hashq, C.coll, C.longs, C.opens, C.tm[0], C.tm[1], kfound >= 0 ? 1 : 0};
}

// Whether a CTA that is about to compute round t leaves the pair.  Once k
// is known every CTA leaves at once, except with a frontier dump: a CTA may
// lag its neighbours by a few blocks, so it first computes every round up
// to k for its tile (those rounds lie in blocks that the owner of d = m - n
// already ran at the same radius: no epoch change is needed, and its
// neighbours have published their edges for them).
__device__ __forceinline__ bool pair_over_seen(const PairDesc &D, unsigned long long v, int64_t t)
{
    if (v == ~0ull)
        return false;
    return !D.dump || v == DONE_STOPPED || (unsigned long long)t > v;
}
__device__ __forceinline__ bool pair_over(const PairDesc &D, GroupCtl *gc, int64_t t)
{
    return pair_over_seen(D, *(volatile unsigned long long *)&gc->done_k, t);
}

// The largest epoch radius whose band [max(-R, -n), min(R, m)] fits in
// cap diagonals; the band width min(R, m) + min(R, n) + 1 grows with R.
__device__ int64_t fit_radius(int64_t n, int64_t m, int64_t cap)
{
    int64_t lo = 0, hi = max(n, m);
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (min(mid, m) + min(mid, n) + 1 <= cap)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Ends the pair for the whole group without a distance: its band outgrew
// the group's tiles (ST_WIDE: the host runs it again on a larger group) or
// the round cap was reached (ST_LIMIT).  The first CTA here records the
// status; the others see done_k set at their next check or barrier.
__device__ void pair_stop(const PairDesc &D, GroupCtl *gc, uint32_t status)
{
    if (threadIdx.x == 0 && atomicCAS(&gc->done_k, ~0ull, DONE_STOPPED) == ~0ull)
        D.res[R_STATUS] = status;
}

// Runs one pair on the group; kc is the radius its re-tiling buffers hold.
// Returns false if the launch must stop.
__device__ __forceinline__ bool run_pair(const LvArgs &P, const Smem S, const PairDesc &D, int q, GroupCtl *gc, int gi, int G,
                         int c0, int32_t *gfb, int64_t kc, uint64_t deadline,
                         Counters &C)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const int h = P.h;
    Pair Q;
    Q.A = D.A;
    Q.B = D.B;
    Q.n = D.n;
    Q.m = D.m;
    Q.TA = D.TA;
    Q.TB = D.TB;
    Q.q = q;
    Q.hash = P.use_hash && D.TA && D.TB;
    const int64_t n = Q.n, m = Q.m, nm = max(n, m);
    const int64_t gstride = 2 * kc + 5;
    const bool leader = (gi == 0 && tid == 0);
    // a pair with a keep buffer may be left at a sync point and resumed
    const bool can_suspend = P.budget_ns != 0 && D.keep != nullptr;
    // epoch 0, or the saved round and radius of a resumed pair
    int64_t R = min((int64_t)P.s0 * G / 2, (int64_t)P.kcap);
    R = max(R, (int64_t)h - 1);
    R = min(R, nm);
    int64_t t = 0;
    if (D.keep && D.t0 > 0) {
        t = D.t0;
        R = D.R0;
    }
    uint32_t epoch = 0;
    Tile T = partition(Q, R, G, gi, c0, h, P.help_div, P.smax, 0);
    if (T.S > P.smax || (D.keep && R > D.keep_r)) {
        pair_stop(D, gc, ST_WIDE);
        if (tid == 0 && gi == 0 && t > 0) { // the saved state is still good
            D.res[R_RESUME_T] = (unsigned long long)t;
            D.res[R_RESUME_R] = (unsigned long long)R;
        }
        return true;
    }
    for (int i = tid; i < P.smax + 2 * HMAX + 2; i += nt) {
        S.F0[i] = NEG;
        S.F1[i] = NEG;
    }
    if (tid == 0)
        *S.n1 = 0;
    __syncthreads();
    if (t > 0 && T.has) {
        // round t - 1 of the tile and its halo from the keep buffer
        const int64_t plo = max(-(t - 1), -n), phi = min(t - 1, m);
        int32_t *dst = frontier(S, t - 1);
        for (int64_t d = T.a - h + tid; d < T.b + h; d += nt)
            dst[d - (T.a - h) + 1] = (d >= plo && d <= phi) ? D.keep[d + D.keep_r + 2] : NEG;
    }
    __syncthreads();
    int64_t t_ep = t; // round of the last epoch change (or of the start)
    for (;;) {
        // ---------------------------------------------- stop / epoch checks
        if (tid == 0) {
            int st = 0;
            if (pair_over(D, gc, t))
                st = 1;
            else if (ld_acquire(&P.ctl->error) != 0)
                st = 2;
            S.bc[1] = st;
        }
        __syncthreads();
        const int stop = S.bc[1];
        __syncthreads();
        if (stop == 1)
            return true;
        if (stop == 2)
            return false;
        const bool need_change =
            ((t + h - 1 > R) && (R < nm)) || (can_suspend && t >= t_ep + P.sync_rounds);
        if (!T.has && !need_change) {
            // no tile: help open slides until the epoch changes or k is found
            // (thread 0 looks at the group's words and the job slots together,
            // several times before the CTA meets at a barrier)
            uint64_t t0 = tid == 0 ? gtimer() : 0;
            for (;;) {
                if (tid == 0) {
                    int st = 0, sl = -1;
                    for (int spin = 0; spin < IDLE_SPINS && st == 0 && sl < 0; spin++) {
                        const unsigned long long dk = *(volatile unsigned long long *)&gc->done_k;
                        const uint32_t er = *(volatile uint32_t *)&P.ctl->error;
                        const uint32_t eq = *(volatile uint32_t *)&gc->epoch_req;
                        const uint32_t ec = *(volatile uint32_t *)&gc->ebar_count;
                        const int js = pick_slot(P);
                        // a job of the group is served even once the epoch
                        // change is asked for, until every tile is at the
                        // barrier (no job of the group opens after that)
                        const bool mine = js >= 0 && js / JOB_RING >= c0 && js / JOB_RING < c0 + G;
                        if (dk != ~0ull)
                            st = 1;
                        else if (er != 0)
                            st = 2;
                        else if (js >= 0 && (eq <= epoch || (mine && ec < (uint32_t)T.ntiles)))
                            sl = js;
                        else if (eq > epoch && ec >= (uint32_t)T.ntiles) {
                            fence_acquire(); // before epoch_t is read
                            st = 3;
                        } else if (gtimer() - t0 > P.idle_ns) {
                            wait_failed(P, 3, t, epoch, ld_acquire(&gc->epoch_req), R, T.ntiles);
                            st = 2;
                        }
                    }
                    S.bc[1] = st;
                    S.bc[2] = sl;
                    if (st == 3)
                        S.bcl[2] = *(volatile uint32_t *)&gc->epoch_t;
                }
                __syncthreads();
                const int st = S.bc[1], sl = S.bc[2];
                const int64_t et = S.bcl[2];
                __syncthreads();
                if (st == 1)
                    return true;
                if (st == 2)
                    return false;
                if (st == 3) {
                    t = et;
                    break;
                }
                if (sl >= 0)
                    serve_slot(P, S, sl, 8, nullptr);
            }
        }
        const bool grow = (t + h - 1 > R) && (R < nm);
        if (grow || (can_suspend && t >= t_ep + P.sync_rounds)) {
            // ------------------------------------------ epoch change
            // (a sync point of a time-sliced pair re-tiles at the same radius)
            const uint64_t te0 = clock64();
            int64_t Rn = R;
            bool wide = false; // the band outgrew the tiles: save it for wider ones
            // the round cap, or tiles too narrow with nowhere to save the band:
            // the pair stops here -- but only once every CTA of the group has
            // reached this round without k being found (a CTA may run blocks
            // ahead of the one that finds k), so the decision waits for the
            // barrier below
            uint32_t stop = 0;
            if (grow) {
                Rn = min(max(R * GROW_NUM / GROW_DEN, t + h - 1), min(nm, (int64_t)P.kcap));
                if (t + h - 1 > Rn && Rn < nm)
                    stop = ST_LIMIT;
                // no further than the group's tiles (and the keep buffer) hold
                Rn = min(Rn, fit_radius(n, m, (int64_t)G * P.smax));
                if (D.keep)
                    Rn = min(Rn, D.keep_r);
                if (!stop && t + h - 1 > Rn && Rn < nm) {
                    if (!D.keep)
                        stop = ST_WIDE;
                    else {
                        // every CTA of the group takes this decision at the same
                        // round: the band of round t - 1 is saved below as for a
                        // time slice, and the host resumes the pair on wider tiles
                        wide = true;
                        Rn = R;
                    }
                }
            }
            int32_t *buf = gfb + ((epoch + 1) & 1) * gstride;
            unsigned long long *lead_s = reinterpret_cast<unsigned long long *>(
                reinterpret_cast<unsigned char *>(S.jring) + 136);
            if (tid == 0)
                *lead_s = 0ull;
            __syncthreads();
            if (T.has) {
                const int32_t *src = frontier(S, t - 1);
                unsigned long long lm = 0ull; // the tile's furthest row and its diagonal
                for (int64_t d = T.a + tid; d < T.b; d += nt) {
                    const int32_t v = src[d - (T.a - h) + 1];
                    st_cg(buf + d + kc + 2, v);
                    if (v >= 0)
                        lm = max(lm, ((unsigned long long)(uint32_t)v << 32) | (uint32_t)(d + 0x80000000ll));
                }
                if (lm)
                    atomicMax(lead_s, lm);
            }
            __syncthreads();
            if (tid == 0 && *lead_s)
                atomicMax(&gc->lead[(epoch + 1) & 1], *lead_s);
            if (leader) {
                // the leader alone decides whether the launch leaves the pair here
                gc->susp[(epoch + 1) & 1] = (wide || (can_suspend && gtimer() >= deadline)) ? 1u : 0u;
                gc->epoch_t = (uint32_t)t;
                __threadfence();
                st_release(&gc->epoch_req, epoch + 1);
            }
            __threadfence();
            const int eb = group_barrier(P, gc, &gc->ebar_count, &gc->ebar_gen, G, true, S);
            if (eb == 0)
                return false;
            if (eb == 2)
                return true; // k is known: the pair is over
            if (stop) {
                pair_stop(D, gc, stop);
                return true;
            }
            epoch++;
            if (*(volatile uint32_t *)&gc->susp[epoch & 1]) {
                // save round t - 1 of the band for the next launch, then leave
                const int64_t plo = max(-(t - 1), -n), phi = min(t - 1, m);
                for (int64_t d = plo + (int64_t)gi * nt + tid; d <= phi; d += (int64_t)G * nt)
                    D.keep[d + D.keep_r + 2] = ld_cg(buf + d + kc + 2);
                if (leader) {
                    D.res[R_STATUS] = wide ? ST_WIDE : ST_SUSPENDED;
                    D.res[R_RESUME_T] = (unsigned long long)t;
                    D.res[R_RESUME_R] = (unsigned long long)Rn;
                }
                return true;
            }
            t_ep = t;
            R = Rn;
            // the band's lead (read by every CTA after the barrier: the same
            // tiles everywhere); the other word is free again for the next
            // change once every CTA has passed this barrier
            const unsigned long long lead = *(volatile unsigned long long *)&gc->lead[epoch & 1];
            if (leader)
                gc->lead[(epoch + 1) & 1] = 0ull;
            T = partition(Q, R, G, gi, c0, h, P.help_div, P.smax,
                          lead ? (int64_t)(uint32_t)lead - 0x80000000ll : 0);
            if (T.S > P.smax) {
                pair_stop(D, gc, ST_WIDE);
                return true;
            }
            if (T.has) {
                const int64_t plo = max(-(t - 1), -n), phi = min(t - 1, m);
                int32_t *dst = frontier(S, t - 1);
                for (int64_t d = T.a - h + tid; d < T.b + h; d += nt)
                    dst[d - (T.a - h) + 1] = (d >= plo && d <= phi) ? ld_cg(buf + d + kc + 2) : NEG;
            }
            __syncthreads();
            C.tm[3] += clock64() - te0;
            if (!T.has)
                continue;
        }
        const int64_t a = T.a, b = T.b, off = a - h - 1; // smem index = d - off
        // ---------------------------------------------- blocks outside the band
        // The band of round t' is [-t', t'].  A tile whose trapezoid (the
        // tile and h - 1 halo diagonals per side) lies outside it for every
        // round of a block holds minus infinity there: the block is skipped,
        // and so is every block after it until the band can reach the
        // trapezoid, an epoch change is due, or a sync point comes.  The tile
        // publishes minus-infinity edges for those rounds at once (both
        // parities: its neighbours read either) and helps long slides while
        // its inner neighbour catches up.  The neighbours' edges of those
        // rounds are minus infinity too (they lie further out than h - 1
        // diagonals inside the trapezoid).
        const int64_t dist = a > 0 ? a : (b <= 0 ? 1 - b : 0); // min |d| over the tile
        int64_t t2 = t;
        while (t2 + 2 * h - 2 < dist && !(t2 + h - 1 > R && R < nm) &&
               !(can_suspend && t2 >= t_ep + P.sync_rounds))
            t2 += h;
        if (t2 > t) {
            int32_t *f = frontier(S, t2 - 1);
            for (int64_t d = a - h + tid; d < b + h; d += nt)
                f[d - off] = NEG;
            const int op = (int)(((t2 / h) & 1) ^ 1);
            if (tid < h) {
                st_relaxed_u64(halo_ptr(P, blockIdx.x, op, 0) + tid, halo_word((uint32_t)(t2 - h), NEG));
                st_relaxed_u64(halo_ptr(P, blockIdx.x, op, 1) + tid, halo_word((uint32_t)(t2 - h), NEG));
            }
            t = t2;
        } else {
            // ------------------------------------------ h rounds
            // a trapezoid of at most two diagonals per thread: the lean rounds
            const BlockOut bo = (b - a) + 2 * h - 2 <= 2 * (int64_t)blockDim.x
                                    ? run_block_lean(P, S, Q, D.dump, D.dump_tmax, D.res, gc, t, h, a, b)
                                    : run_block(P, S, Q, D.dump, D.dump_tmax, D.res, gc, t, h, a, b);
            C.slide += bo.slide;
            C.mism += bo.mism;
            C.hashq += bo.hashq;
            C.coll += bo.coll;
            C.longs += bo.longs;
            C.opens += bo.opens;
            C.tm[0] += bo.tm_round;
            C.tm[1] += bo.tm_open;
            const bool fin = bo.fin != 0;
            if (fin)
                return true;
            t += h;
            C.blocks++;
        }
        // ---------------------------------------------- halo exchange
        // The edge words of round t - 1 (halo_word): a word of round t or
        // later is the value for round t - 1 (a later round is a tile that
        // skipped ahead with minus infinity on its edges, which holds for the
        // rounds it skipped as well).
        const uint64_t tw0 = clock64();
        const int parity = (int)((t / h) & 1);
        int32_t *edge = frontier(S, t - 1);
        const uint32_t tag = (uint32_t)t;
        if (tid < h) {
            const int64_t dl = a + tid, dr = b - h + tid;
            st_relaxed_u64(halo_ptr(P, blockIdx.x, parity, 0) + tid, halo_word(tag, dl < b ? edge[dl - off] : NEG));
            st_relaxed_u64(halo_ptr(P, blockIdx.x, parity, 1) + tid, halo_word(tag, dr >= a ? edge[dr - off] : NEG));
        }
        const unsigned long long *lw = T.left >= 0 ? halo_ptr(P, T.left, parity, 1) : nullptr;
        const unsigned long long *rw = T.right >= 0 ? halo_ptr(P, T.right, parity, 0) : nullptr;
        // wait for both neighbours' words (warp 0: lanes 0..15 the left
        // neighbour's, 16..31 the right one's; lane j reads words j, j + 16,
        // j + 32 and j + 48 of its side), helping open slides meanwhile
        const uint64_t t0 = tid == 0 ? gtimer() : 0;
        for (;;) {
            if (tid < 32) {
                const int side = tid >> 4, j = tid & 15;
                const unsigned long long *wp = side ? rw : lw;
                int st = 0, js = -1;
                for (int spin = 0; spin < HALO_SPINS; spin++) {
                    unsigned long long v[HMAX / 16];
                    bool ok = true;
#pragma unroll
                    for (int u = 0; u < HMAX / 16; u++) {
                        const int jj = j + 16 * u;
                        v[u] = (jj < h && wp) ? ld_relaxed_u64(wp + jj) : ~0ull;
                    }
                    // an open job of another CTA, looked for in the same round trip
                    int q = tid == 0 ? pick_slot(P) : -1;
#pragma unroll
                    for (int u = 0; u < HMAX / 16; u++)
                        ok = ok && (uint32_t)(v[u] >> 32) >= tag;
                    if (__all_sync(0xffffffffu, ok)) {
#pragma unroll
                        for (int u = 0; u < HMAX / 16; u++) {
                            const int jj = j + 16 * u;
                            if (jj < h)
                                edge[(side ? b + jj : a - h + jj) - off] = wp ? (int32_t)(uint32_t)v[u] : NEG;
                        }
                        st = 3;
                        break;
                    }
                    q = __shfl_sync(0xffffffffu, q, 0);
                    if (q >= 0) {
                        js = q;
                        break;
                    }
                }
                if (tid == 0 && st == 0 && js < 0) {
                    const unsigned long long dk = *(volatile unsigned long long *)&gc->done_k;
                    const uint32_t er = *(volatile uint32_t *)&P.ctl->error;
                    if (pair_over_seen(D, dk, t))
                        st = 1;
                    else if (er != 0)
                        st = 2;
                    else if (gtimer() - t0 > P.idle_ns) {
                        wait_failed(P, 4, t, tag, lw ? ld_relaxed_u64(lw) : ~0ull, rw ? ld_relaxed_u64(rw) : ~0ull,
                                    ((unsigned long long)(uint32_t)T.left << 32) | (uint32_t)T.right);
                        st = 2;
                    }
                }
                if (tid == 0) {
                    S.bc[1] = st;
                    S.bc[2] = js;
                }
            }
            __syncthreads();
            const int st = S.bc[1], js = S.bc[2];
            __syncthreads();
            if (st == 1)
                return true;
            if (st == 2)
                return false;
            if (st == 3)
                break;
            if (js >= 0) {
                // two claims at most (one pipeline fill): a tile's own next
                // block waits on the chunks it has in flight
                const Wake wk{lw, rw, tag};
                serve_slot(P, S, js, 2, &wk);
            }
        }
        C.tm[2] += clock64() - tw0;
    }
}

__device__ __forceinline__ void flush_counters(const PairDesc &D, Counters &C, bool first_cta)
{
    unsigned long long v[7] = {C.slide, C.mism, C.hashq, C.coll, C.longs, C.blocks, C.opens};
    for (int o = 16; o; o >>= 1)
        for (int i = 0; i < 7; i++)
            v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
    if ((threadIdx.x & 31) == 0) {
        if (v[6]) atomicAdd(&D.res[R_OPEN], v[6]);
        if (v[0]) atomicAdd(&D.res[R_SLIDE], v[0]);
        if (v[1]) atomicAdd(&D.res[R_MISMATCH], v[1]);
        if (v[2]) atomicAdd(&D.res[R_HASHQ], v[2]);
        if (v[3]) atomicAdd(&D.res[R_HASHCOLL], v[3]);
    }
    if (threadIdx.x == 0) {
        // counted once per CTA (the values are the CTA's, not per thread)
        if (C.longs)
            atomicAdd(&D.res[R_LONG], C.longs);
        if (first_cta)
            D.res[R_WIDE] = C.blocks;
        // phase cycles: the largest over the group's CTAs, and the sum of
        // round + slide cycles (for the average busy time)
        for (int i = 0; i < 4; i++)
            atomicMax(&D.res[R_T0 + i], C.tm[i]);
        atomicAdd(&D.res[R_T0 + 4], C.tm[0] + C.tm[1]);
        atomicAdd(&D.res[R_T0 + 5], 1ull);
    }
    C = Counters();
}

__global__ void __launch_bounds__(CTA_THREADS, 1) lv_tiles_kernel(LvArgs P)
{
    const Smem S = carve(P);
    if (threadIdx.x == 0) { // no job cached (read before the first group barrier)
        S.jd->jid = 0;
        S.jd->slot = -1;
        S.jd->pq = -1;
        *S.jring = 0;
        *reinterpret_cast<int *>(reinterpret_cast<unsigned char *>(S.jring) + 128) = 0;
        for (int i = 0; S.stg && i < P.stage; i++) {
            const Stage T = stage_of(S.stg + i * STAGE_STRIDE);
            mbar_init(T.bar, 1);
            *T.phase = 0;
        }
        if (S.stg)
            fence_mbar_init();
    }
    const uint64_t deadline = gtimer() + P.budget_ns;
    int cls = 0;
    while (cls + 1 < P.ncls && (int)blockIdx.x >= P.cls_c0[cls + 1])
        cls++;
    const int G = P.cls_G[cls];
    const int rel = (int)blockIdx.x - P.cls_c0[cls];
    const int gi = rel % G, c0 = (int)blockIdx.x - gi;
    GroupCtl *gc = &P.gctl[P.cls_g0[cls] + rel / G];
    const int64_t kc = P.cls_kc[cls];
    int32_t *gfb = P.gf + P.cls_gf[cls] + (int64_t)(rel / G) * 2 * (2 * kc + 5);
    Counters C;
    for (;;) {
        // the CTA's edge words start each pair cleared (round 0): every CTA
        // of the group has left the pair before (the barrier that ends the
        // last turn), and the barrier below orders the clear before the
        // first read of the next pair
        for (int i = threadIdx.x; i < 4 * HMAX; i += blockDim.x)
            st_relaxed_u64(P.halo + (size_t)blockIdx.x * 4 * HMAX + i, 0ull);
        if (gi == 0 && threadIdx.x == 0) {
            // the class's own queue first, then the classes below it
            int32_t q = -1;
            for (int c = cls; c >= 0 && q < 0; c--) {
                const uint32_t cnt = (uint32_t)(P.cls_p0[c + 1] - P.cls_p0[c]);
                if (*(volatile uint32_t *)&P.ctl->queue[c] >= cnt)
                    continue;
                const uint32_t i = atomicAdd(&P.ctl->queue[c], 1u);
                if (i < cnt)
                    q = P.cls_p0[c] + (int32_t)i;
            }
            gc->pair = q;
            gc->done_k = ~0ull;
            gc->epoch_req = 0;
            gc->epoch_t = 0;
            gc->lead[0] = gc->lead[1] = 0ull;
            gc->ebar_count = 0; // no CTA is inside the epoch barrier here
            __threadfence();
        }
        if (!group_sync(P, gc, G, S))
            break;
        const int q = *(volatile int32_t *)&gc->pair;
        if (q < 0)
            break;
        const PairDesc D = P.pairs[q];
        const bool ok = run_pair(P, S, D, q, gc, gi, G, c0, gfb, kc, deadline, C);
        flush_counters(D, C, gi == 0);
        if (!ok)
            break;
        if (!group_sync(P, gc, G, S))
            break;
    }
}

cudaError_t launch_lv_tiles(const LvArgs &P, int grid, cudaStream_t s)
{
    const size_t smem = lv_tiles_smem_bytes(P.smax, P.h, P.stage);
    cudaError_t e =
        cudaFuncSetAttribute(lv_tiles_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    LvArgs Pc = P;
    void *args[] = {&Pc};
    return cudaLaunchCooperativeKernel((const void *)lv_tiles_kernel, dim3(grid), dim3(CTA_THREADS), args,
                                       smem, s);
}

// ------------------------------------------------------------------ tests
__global__ void lcp_query_kernel(const uint8_t *A, int64_t n, const uint8_t *B, int64_t m,
                                 const int64_t *qx, const int64_t *qy, int64_t q, int method,
                                 HashArgs H, int64_t *out)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (method == 0 || method == 3 || method == 4) {
        for (int64_t i = tid; i < q; i += (int64_t)gridDim.x * blockDim.x) {
            const int64_t x = qx[i], y = qy[i];
            const int64_t lim = (x <= n && y <= m) ? min(n - x, m - y) : 0;
            bool open;
            if (method == 0) {
                out[i] = slide_thread(A, n, B, m, x, y, lim, INT64_MAX, &open);
            } else if (lim <= 0) {
                out[i] = 0;
            } else {
                // the leading window directly, then the doubling search
                int64_t l = slide_thread(A, n, B, m, x, y, lim, 4, &open);
                if (open) {
                    const int64_t hh = hash_lcp(H.pow2, HashView{H.TA, A, H.b}, HashView{H.TB, B, H.b}, x, y, l, lim);
                    if (method == 3) {
                        l = hh;
                    } else {
                        const int64_t cl = min(hh + 1, lim);
                        l = slide_thread(A, n, B, m, x, y, cl, INT64_MAX, &open);
                        if (l == cl && cl < lim)
                            l = slide_thread(A, n, B, m, x, y, lim, INT64_MAX, &open);
                    }
                }
                out[i] = l;
            }
        }
    } else if (method == 1) {
        const int64_t w = tid >> 5, nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
        for (int64_t i = w; i < q; i += nwarps) {
            const int64_t x = qx[i], y = qy[i];
            const int64_t lim = (x <= n && y <= m) ? min(n - x, m - y) : 0;
            bool open;
            const int64_t l = slide_warp(A, n, B, m, x, y, 0, lim, INT64_MAX / 4, &open);
            if ((threadIdx.x & 31) == 0)
                out[i] = l;
        }
    }
}

// Method 2: every CTA claims chunks of the queries' slots (published by the
// host: claim = 1 << 32, result = lim) until each slot is exhausted; the
// answers stay in the slots.
__device__ uint32_t g_lcp_grid_err; // status word of the test launches below

__global__ void __launch_bounds__(CTA_THREADS) lcp_grid_kernel(JobSlot *slots, int nslots, int stage,
                                                                const PairDesc *pairs)
{
    extern __shared__ __align__(128) unsigned char gsm[];
    __shared__ unsigned long long s_min;
    __shared__ long long s_bcl[4];
    __shared__ int s_bc[8];
    __shared__ JobDesc s_jd;
    Smem S{};
    S.smin = &s_min;
    S.bc = s_bc;
    S.bcl = s_bcl;
    S.jd = &s_jd;
    S.err = &g_lcp_grid_err;
    S.stg = stage ? gsm : nullptr;
    LvArgs P{};
    P.spin_ns = 2000000000ull;
    P.pairs = pairs;
    if (threadIdx.x == 0) {
        s_jd.jid = 0;
        s_jd.slot = -1;
        s_jd.pq = -1;
        if (stage) {
            const Stage T = stage_of(gsm);
            mbar_init(T.bar, 1);
            *T.phase = 0;
            fence_mbar_init();
        }
    }
    __syncthreads();
    for (int j = 0; j < nslots; j++) {
        const int s = (j + (int)blockIdx.x) % nslots;
        // claims until a chunk lies past the end or the best mismatch
        claim_loop(P, S, &slots[s], s, 0ull, INT32_MAX);
    }
}

cudaError_t launch_lcp_queries(const uint8_t *A, int64_t n, const uint8_t *B, int64_t m,
                               const int64_t *x, const int64_t *y, int64_t q, int method,
                               const HashArgs *hash, int64_t *out, JobSlot *slots, const PairDesc *pairs,
                               int grid, cudaStream_t s)
{
    if (q == 0)
        return cudaSuccess;
    if (method == 2 || method == 7) {
        // 2: register sweeps; 7: the same claims scanned through a bulk-copy stage
        const int stage = method == 7;
        const size_t smem = stage ? stage_bytes<CHUNK_BYTES>() : 0;
        if (stage) {
            const cudaError_t e =
                cudaFuncSetAttribute(lcp_grid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess)
                return e;
        }
        lcp_grid_kernel<<<grid, CTA_THREADS, smem, s>>>(slots, (int)q, stage, pairs);
        return cudaGetLastError();
    }
    HashArgs H{};
    if (hash)
        H = *hash;
    const int threads = 256;
    const int64_t blocks = method == 1 ? (q * 32 + threads - 1) / threads : (q + threads - 1) / threads;
    lcp_query_kernel<<<(unsigned)min(blocks, (int64_t)65535), threads, 0, s>>>(A, n, B, m, x, y, q,
                                                                              method, H, out);
    return cudaGetLastError();
}

} // namespace edg
