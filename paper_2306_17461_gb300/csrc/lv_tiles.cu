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
//    one per CTA, each kept in shared memory.  R (the epoch radius) doubles
//    when the band [-t, t] reaches it; tiles are then re-cut through a
//    global buffer behind a group barrier (O(log k) times in all).
//  * Temporal blocking: a CTA holds its tile plus h diagonals of halo on
//    each side and runs h rounds on the shrinking trapezoid (the halo
//    diagonals are recomputed, exactly), then trades its h edge values with
//    its two neighbours through global memory and a per-CTA release flag.
//    There is no grid-wide barrier per round, only neighbour waits every h
//    rounds.
//  * Slides: one thread compares the leading 4-byte words (several
//    diagonals' loads in flight together), then 16-byte windows; a slide
//    still open after t1_cap bytes goes to one warp (ballot / first set
//    bit over 512-byte steps); one still open after t2_cap bytes becomes a
//    job in the CTA's job slot, split into 64 KiB chunks that the owner and
//    every CTA waiting on a neighbour (or without a tile) claim by CAS;
//    the first mismatch is the atomicMin over chunks.
//  * Every wait is bounded by %globaltimer and reports ST_TIMEOUT instead
//    of hanging.
#include "ed_device.cuh"
#include "lv_kernels.cuh"

namespace edg {

struct Counters {
    unsigned long long slide = 0, mism = 0, hashq = 0, coll = 0, longs = 0, blocks = 0;
    unsigned long long tm[4] = {0, 0, 0, 0};
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

// h(A[x..x+L)) == h(B[y..y+L)) with h(S2) = h([S1,S2]) - p^|S2| h(S1).
__device__ __forceinline__ bool hash_eq(const uint64_t *TA, const uint64_t *TB, int64_t x, int64_t y,
                                        int64_t L, uint64_t P)
{
    const uint64_t a = submod61(__ldg(TA + x + L), mulmod61(__ldg(TA + x), P));
    const uint64_t b = submod61(__ldg(TB + y + L), mulmod61(__ldg(TB + y), P));
    return a == b;
}

// Sec. 3.2: compare chunks of length 1, 2, 4, ... (here: the powers of two
// above the l0 bytes already known equal) until one differs, then search
// the last bracket.  Returns the hash LCP (<= lim); the caller confirms it.
__device__ __noinline__ int64_t hash_lcp(const uint64_t *pow2, const uint64_t *TA, const uint64_t *TB,
                                         int64_t x, int64_t y, int64_t l0, int64_t lim)
{
    int64_t good = l0, bad;
    uint64_t pg = powp(pow2, good);
    int j = 0;
    while (j < 62 && (1ll << j) <= good)
        j++;
    for (;; j++) {
        const int64_t L = 1ll << j;
        if (L >= lim) {
            if (hash_eq(TA, TB, x, y, lim, powp(pow2, lim)))
                return lim;
            bad = lim;
            break;
        }
        if (hash_eq(TA, TB, x, y, L, pow2[j])) {
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
            if (hash_eq(TA, TB, x, y, cand, P)) {
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
    const uint64_t *TA, *TB;
    bool hash;
};

// ------------------------------------------------------------------ phase A
constexpr int DPT = 4; // diagonals per thread per batch

// One round over diagonals [lo, hi] (strided over the CTA): the start row
// c = getc(d), then the per-thread slide.  DPT diagonals per thread are
// handled together so that their first loads are in flight together.
// done(d, c, l, full) receives finished slides (row c + l); open_(d, c, pos,
// lim_abs) receives slides still open after t1_cap bytes (A[c..pos) matched,
// the first mismatch lies in [pos, lim_abs], lim_abs possibly lowered to
// the hash answer + 1).
template <class GetC, class Done, class Open>
__device__ __forceinline__ void phase_a(const LvArgs &P, const Pair &Q, int64_t lo, int64_t hi,
                                        GetC getc, Done done, Open open_, Counters &C)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int64_t base = lo; base <= hi; base += (int64_t)nt * DPT) {
        int64_t c[DPT];
        uint32_t wa[DPT], wb[DPT];
#pragma unroll
        for (int u = 0; u < DPT; u++) {
            const int64_t d = base + (int64_t)u * nt + tid;
            c[u] = 0;
            wa[u] = wb[u] = 0;
            if (d <= hi) {
                c[u] = getc(d);
                if (min(Q.n - c[u], Q.m - c[u] - d) > 0)
                    word_load(Q.A, Q.B, c[u], c[u] + d, wa[u], wb[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < DPT; u++) {
            const int64_t d = base + (int64_t)u * nt + tid;
            if (d <= hi) {
                const int64_t cc = c[u];
                const int64_t full = min(Q.n - cc, Q.m - cc - d);
                bool op;
                const int64_t l = slide_thread_w(Q.A, Q.n, Q.B, Q.m, cc, cc + d, full, P.t1_cap,
                                                 wa[u], wb[u], &op);
                if (!op) {
                    done(d, cc, l, full);
                } else {
                    int64_t lim = full;
                    if (Q.hash) {
                        const int64_t h = hash_lcp(P.pow2, Q.TA, Q.TB, cc, cc + d, l, full);
                        C.hashq++;
                        lim = min(h + 1, full);
                    }
                    open_(d, cc, cc + l, cc + lim);
                }
            }
        }
    }
}

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

// Claim the next chunk of slot sl (thread 0).  Returns the chunk index, -1
// when there is nothing left to claim (closed, past the end, or past the
// first mismatch found so far), -2 when the CAS lost a race.
__device__ int64_t try_claim(JobSlot *sl)
{
    const unsigned long long w = ld_acquire_u64(&sl->claim);
    const uint32_t c = (uint32_t)w;
    if (c == CLAIM_CLOSED || (w >> 32) == 0)
        return -1;
    const uint32_t nch = *(volatile unsigned int *)&sl->nchunks;
    const unsigned long long res = *(volatile unsigned long long *)&sl->result;
    if (c >= nch || (unsigned long long)c * CHUNK_BYTES >= res)
        return -1;
    if (atomicCAS(&sl->claim, w, w + 1) != w)
        return -2;
    __threadfence();
    return (int64_t)c;
}

struct Smem {
    int32_t *F[2];      // tile + halo frontier, smax + 2h + 2 entries each
    int32_t *ld, *lc;   // open slides: diagonal, start row
    int64_t *lpos, *llim;
    int *n1;
    int *bc;            // 8 broadcast words
    long long *bcl;     // 4 broadcast 64-bit words
    unsigned long long *smin;
    int lcap;
};

// Scan chunk c of slot sl with the whole CTA, lower its result, count it.
__device__ __noinline__ void scan_chunk(const Smem &S, JobSlot *sl, int64_t c)
{
    // the slot is rewritten for every job: read it past the L1
    const uint8_t *A = (const uint8_t *)__ldcg((const unsigned long long *)&sl->A);
    const uint8_t *B = (const uint8_t *)__ldcg((const unsigned long long *)&sl->B);
    const int64_t n = __ldcg(&sl->n), m = __ldcg(&sl->m), x = __ldcg(&sl->x), y = __ldcg(&sl->y),
                  lim = __ldcg(&sl->lim);
    const int64_t cs = c * (int64_t)CHUNK_BYTES;
    const int64_t r = cta_scan<CHUNK_UNROLL>(A, n, B, m, x, y, cs, min((int64_t)CHUNK_BYTES, lim - cs),
                                             S.smin);
    if (threadIdx.x == 0) {
        if (r >= 0)
            atomicMin(&sl->result, (unsigned long long)r);
        __threadfence();
        atomicAdd(&sl->done, 1u);
    }
}

// Help one open job of any CTA (whole CTA).  Returns true if a chunk was
// scanned.
__device__ bool help_one(const LvArgs &P, const Smem &S)
{
    const int tid = threadIdx.x;
    if (tid == 0) {
        int slot = -1;
        long long chunk = -1;
        const int nw = (gridDim.x + 63) >> 6;
        for (int k = 0; k < nw && slot < 0; k++) {
            const int w = (int)((blockIdx.x / 64 + k) % nw);
            unsigned long long bits = *(volatile unsigned long long *)&P.ctl->active[w];
            // start from a CTA-dependent bit so helpers spread over jobs
            const int rot = blockIdx.x & 63;
            bits = (bits >> rot) | (rot ? (bits << (64 - rot)) : 0ull);
            while (bits && slot < 0) {
                const int b = (__ffsll((long long)bits) - 1 + rot) & 63;
                bits &= bits - 1;
                const int s = w * 64 + b;
                if (s >= (int)gridDim.x)
                    continue;
                int64_t c = try_claim(&P.slots[s]);
                if (c == -2)
                    c = try_claim(&P.slots[s]);
                if (c >= 0) {
                    slot = s;
                    chunk = c;
                }
            }
        }
        S.bc[0] = slot;
        S.bcl[0] = chunk;
    }
    __syncthreads();
    const int slot = S.bc[0];
    const int64_t chunk = S.bcl[0];
    __syncthreads();
    if (slot < 0)
        return false;
    scan_chunk(S, &P.slots[slot], chunk);
    return true;
}

// The CTA's own long slide: A[x..x+lim) vs B[y..).  Published in the CTA's
// slot when it spans more than one chunk; the owner claims chunks like any
// helper, then closes the slot and waits for the claims still running.
// Returns the first mismatch offset, or lim.
__device__ __noinline__ int64_t long_slide(const LvArgs &P, const Smem &S, const Pair &Q, int64_t x,
                                           int64_t y, int64_t lim)
{
    const int tid = threadIdx.x;
    JobSlot *sl = &P.slots[blockIdx.x];
    const uint32_t nch = (uint32_t)((lim + CHUNK_BYTES - 1) / CHUNK_BYTES);
    const int word = blockIdx.x >> 6;
    const unsigned long long bit = 1ull << (blockIdx.x & 63);
    if (tid == 0) {
        sl->A = Q.A;
        sl->B = Q.B;
        sl->n = Q.n;
        sl->m = Q.m;
        sl->x = x;
        sl->y = y;
        sl->lim = lim;
        sl->result = (unsigned long long)lim;
        sl->done = 0;
        sl->nchunks = nch;
        const uint32_t jid = (uint32_t)(sl->claim >> 32) + 1u;
        __threadfence();
        atomicExch(&sl->claim, ((unsigned long long)(jid ? jid : 1u) << 32));
        if (nch > 1)
            atomicOr(&P.ctl->active[word], bit);
    }
    __syncthreads();
    for (;;) {
        if (tid == 0) {
            int64_t c;
            while ((c = try_claim(sl)) == -2) {
            }
            S.bcl[1] = c;
        }
        __syncthreads();
        const int64_t c = S.bcl[1];
        __syncthreads();
        if (c < 0)
            break;
        scan_chunk(S, sl, c);
    }
    if (tid == 0) {
        if (nch > 1)
            atomicAnd(&P.ctl->active[word], ~bit);
        unsigned long long w = ld_acquire_u64(&sl->claim);
        uint32_t nclaimed = 0;
        for (;;) {
            nclaimed = (uint32_t)w;
            if (nclaimed == CLAIM_CLOSED) { // not reachable: only the owner closes
                nclaimed = 0;
                break;
            }
            const unsigned long long nw = (w & 0xffffffff00000000ull) | CLAIM_CLOSED;
            const unsigned long long old = atomicCAS(&sl->claim, w, nw);
            if (old == w)
                break;
            w = old;
        }
        const uint64_t t0 = gtimer();
        while (*(volatile unsigned int *)&sl->done < nclaimed) {
            if (gtimer() - t0 > P.spin_ns) {
                wait_failed(P, 1, 0, nclaimed, *(volatile unsigned int *)&sl->done, 0, 0);
                break;
            }
        }
        __threadfence();
        S.bcl[1] = (long long)*(volatile unsigned long long *)&sl->result;
    }
    __syncthreads();
    const int64_t r = S.bcl[1];
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------ group
// Bounded barrier over the G CTAs of a group, on (count, gen).  Returns 1
// when all arrived, 0 on error or timeout, 2 when `abandon` is set and the
// group's k became known meanwhile (the epoch-change barrier: CTAs that
// have seen k leave the pair without arriving).
__device__ int group_barrier(const LvArgs &P, GroupCtl *gc, uint32_t *count, uint32_t *gen_p, int G,
                             bool abandon, const Smem &S)
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

__device__ bool group_sync(const LvArgs &P, GroupCtl *gc, int G, const Smem &S)
{
    return group_barrier(P, gc, &gc->bar_count, &gc->bar_gen, G, false, S) == 1;
}

size_t lv_tiles_smem_bytes(int smax, int h)
{
    (void)h;
    const int lcap = 512;
    return 128 + (size_t)lcap * (2 * sizeof(int64_t) + 2 * sizeof(int32_t)) +
           2 * sizeof(int32_t) * ((size_t)smax + 2 * HMAX + 2);
}

__device__ Smem carve(const LvArgs &P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem S;
    unsigned char *p = smem_raw;
    S.smin = reinterpret_cast<unsigned long long *>(p);
    S.bcl = reinterpret_cast<long long *>(p + 16);
    S.n1 = reinterpret_cast<int *>(p + 64);
    S.bc = S.n1 + 4;
    p += 128;
    S.lcap = 512;
    S.lpos = reinterpret_cast<int64_t *>(p);
    p += sizeof(int64_t) * S.lcap;
    S.llim = reinterpret_cast<int64_t *>(p);
    p += sizeof(int64_t) * S.lcap;
    S.ld = reinterpret_cast<int32_t *>(p);
    p += sizeof(int32_t) * S.lcap;
    S.lc = reinterpret_cast<int32_t *>(p);
    p += sizeof(int32_t) * S.lcap;
    S.F[0] = reinterpret_cast<int32_t *>(p);
    p += sizeof(int32_t) * (P.smax + 2 * HMAX + 2);
    S.F[1] = reinterpret_cast<int32_t *>(p);
    return S;
}

struct Tile {
    int64_t lo_all, hi_all, S;
    int64_t a, b; // own diagonals [a, b)
    int ntiles;
    bool has;
    int left, right; // neighbour CTA (grid index) or -1
};

__device__ Tile partition(const Pair &Q, int64_t R, int G, int gi, int c0, int h)
{
    Tile T;
    T.lo_all = max(-R, -Q.n);
    T.hi_all = min(R, Q.m);
    const int64_t N = T.hi_all - T.lo_all + 1;
    T.S = max((int64_t)h, (N + G - 1) / G);
    T.ntiles = (int)((N + T.S - 1) / T.S);
    T.has = gi < T.ntiles;
    T.a = T.lo_all + (int64_t)gi * T.S;
    T.b = min(T.hi_all + 1, T.a + T.S);
    T.left = (T.has && gi > 0) ? c0 + gi - 1 : -1;
    T.right = (T.has && gi + 1 < T.ntiles) ? c0 + gi + 1 : -1;
    return T;
}

__device__ __forceinline__ int32_t *halo_ptr(const LvArgs &P, int cta, int parity, int side)
{
    return P.halo + ((int64_t)(cta * 2 + parity) * 2 + side) * HMAX;
}

// Runs one pair on the group.  Returns false if the launch must stop.
__device__ bool run_pair(const LvArgs &P, const Smem &S, const PairDesc &D, GroupCtl *gc, int gi, int G,
                         int c0, int32_t *gfb, unsigned long long iter, Counters &C)
{
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int h = P.h;
    Pair Q;
    Q.A = D.A;
    Q.B = D.B;
    Q.n = D.n;
    Q.m = D.m;
    Q.TA = D.TA;
    Q.TB = D.TB;
    Q.hash = P.use_hash && D.TA && D.TB;
    const int64_t n = Q.n, m = Q.m, target = m - n, nm = max(n, m);
    const int64_t gstride = 2 * (int64_t)P.kcap + 5;
    const bool leader = (gi == 0 && tid == 0);
    // epoch 0
    int64_t R = min((int64_t)P.s0 * G / 2, (int64_t)P.kcap);
    R = max(R, (int64_t)h - 1);
    R = min(R, nm);
    uint32_t epoch = 0;
    Tile T = partition(Q, R, G, gi, c0, h);
    if (T.S > P.smax) {
        if (tid == 0)
            set_error(P, ST_LIMIT);
        return false;
    }
    for (int i = tid; i < P.smax + 2 * HMAX + 2; i += nt) {
        S.F[0][i] = NEG;
        S.F[1][i] = NEG;
    }
    if (tid == 0)
        *S.n1 = 0;
    __syncthreads();
    int64_t t = 0;
    for (;;) {
        // ---------------------------------------------- stop / epoch checks
        if (tid == 0) {
            int st = 0;
            if (*(volatile unsigned long long *)&gc->done_k != ~0ull)
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
        const bool need_change = (t + h - 1 > R) && (R < nm);
        if (!T.has && !need_change) {
            // no tile: help open slides until the epoch changes or k is found
            uint64_t t0 = tid == 0 ? gtimer() : 0;
            for (;;) {
                if (tid == 0) {
                    int st = 0;
                    if (*(volatile unsigned long long *)&gc->done_k != ~0ull)
                        st = 1;
                    else if (ld_acquire(&P.ctl->error) != 0)
                        st = 2;
                    else if (ld_acquire(&gc->epoch_req) > epoch)
                        st = 3;
                    else if (gtimer() - t0 > P.idle_ns) {
                        wait_failed(P, 3, t, epoch, ld_acquire(&gc->epoch_req), R, T.ntiles);
                        st = 2;
                    }
                    S.bc[1] = st;
                    if (st == 3)
                        S.bcl[2] = *(volatile uint32_t *)&gc->epoch_t;
                }
                __syncthreads();
                const int st = S.bc[1];
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
                if (!help_one(P, S))
                    __nanosleep(256);
            }
        }
        if ((t + h - 1 > R) && (R < nm)) {
            // ------------------------------------------ epoch change
            const uint64_t te0 = gtimer();
            const int64_t Rn = min(max(2 * R, t + h - 1), min(nm, (int64_t)P.kcap));
            if (t + h - 1 > Rn && Rn < nm) {
                if (tid == 0)
                    set_error(P, ST_LIMIT);
                return false;
            }
            int32_t *buf = gfb + ((epoch + 1) & 1) * gstride;
            if (T.has) {
                const int32_t *src = S.F[(t - 1) & 1];
                for (int64_t d = T.a + tid; d < T.b; d += nt)
                    st_cg(buf + d + P.kcap + 2, src[d - (T.a - h) + 1]);
            }
            if (leader) {
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
            epoch++;
            R = Rn;
            T = partition(Q, R, G, gi, c0, h);
            if (T.S > P.smax) {
                if (tid == 0)
                    set_error(P, ST_LIMIT);
                return false;
            }
            if (T.has) {
                const int64_t plo = max(-(t - 1), -n), phi = min(t - 1, m);
                int32_t *dst = S.F[(t - 1) & 1];
                for (int64_t d = T.a - h + tid; d < T.b + h; d += nt)
                    dst[d - (T.a - h) + 1] = (d >= plo && d <= phi) ? ld_cg(buf + d + P.kcap + 2) : NEG;
            }
            __syncthreads();
            C.tm[3] += gtimer() - te0;
            if (!T.has)
                continue;
        }
        // ---------------------------------------------- h rounds
        const int64_t a = T.a, b = T.b, off = a - h - 1; // smem index = d - off
        bool fin = false;
        for (int r = 0; r < h && !fin; r++) {
            const uint64_t tr0 = gtimer();
            const int64_t tau = t + r;
            const int64_t ra = a - h + 1 + r, rb = b + h - 1 - r; // computed range [ra, rb)
            const int64_t blo = max(-tau, -n), bhi = min(tau, m);
            const int32_t *prev = S.F[(tau - 1) & 1];
            int32_t *cur = S.F[tau & 1];
            // outside the band: minus infinity
            for (int64_t d = ra + tid; d < rb; d += nt)
                if (d < blo || d > bhi)
                    cur[d - off] = NEG;
            const int64_t lo = max(ra, blo), hi = min(rb - 1, bhi);
            phase_a(
                P, Q, lo, hi,
                [&](int64_t d) -> int64_t {
                    if (tau == 0)
                        return 0;
                    const int64_t x1 = prev[d - 1 - off];
                    const int64_t x2 = (int64_t)prev[d - off] + 1;
                    const int64_t x3 = (int64_t)prev[d + 1 - off] + 1;
                    return min(max(x1, max(x2, x3)), min(n, m - d));
                },
                [&](int64_t d, int64_t c, int64_t l, int64_t full) {
                    cur[d - off] = (int32_t)(c + l);
                    if (d >= a && d < b) {
                        C.slide += l;
                        C.mism += (l < full);
                    }
                },
                [&](int64_t d, int64_t c, int64_t pos, int64_t lim) {
                    const int s = atomicAdd(S.n1, 1);
                    if (s < S.lcap) {
                        S.ld[s] = (int32_t)d;
                        S.lc[s] = (int32_t)c;
                        S.lpos[s] = pos;
                        S.llim[s] = lim;
                    } else {
                        bool o;
                        const int64_t p = pos + slide_thread(Q.A, n, Q.B, m, pos, pos + d, lim - pos,
                                                             INT64_MAX, &o);
                        cur[d - off] = (int32_t)finish_slide(Q, c, d, p, lim, d >= a && d < b, C);
                    }
                },
                C);
            __syncthreads();
            const uint64_t tr1 = gtimer();
            C.tm[0] += tr1 - tr0;
            const int n1 = min(*S.n1, S.lcap);
            if (n1 > 0) {
                // one warp per open slide
                for (int j = warp; j < n1; j += nw) {
                    const int64_t d = S.ld[j], c = S.lc[j], pos = S.lpos[j], lim = S.llim[j];
                    bool open;
                    const int64_t l =
                        slide_warp(Q.A, n, Q.B, m, pos, pos + d, 0, lim - pos, P.t2_cap, &open);
                    if (lane == 0) {
                        if (!open) {
                            cur[d - off] = (int32_t)finish_slide(Q, c, d, pos + l, lim, d >= a && d < b, C);
                            S.llim[j] = -1; // finished
                        } else {
                            S.lpos[j] = pos + l;
                        }
                    }
                }
                __syncthreads();
                // still open: a job for the whole CTA, helped by waiting CTAs
                for (int j = 0; j < n1; j++) {
                    const int64_t lim = S.llim[j];
                    if (lim < 0)
                        continue;
                    const int64_t d = S.ld[j], pos = S.lpos[j];
                    const int64_t rr = long_slide(P, S, Q, pos, pos + d, lim - pos);
                    if (tid == 0) {
                        const int64_t c = S.lc[j];
                        const bool own = d >= a && d < b;
                        cur[d - off] = (int32_t)finish_slide(Q, c, d, pos + rr, lim, own, C);
                        C.longs += own;
                    }
                }
                __syncthreads();
                if (tid == 0)
                    *S.n1 = 0;
                C.tm[1] += gtimer() - tr1;
            }
            // termination: the tile owning the target diagonal reports k
            if (target >= a && target < b && target >= blo && target <= bhi && cur[target - off] == n) {
                fin = true;
                if (tid == 0) {
                    atomicMin(&gc->done_k, (unsigned long long)tau);
                    D.res[R_K] = (unsigned long long)tau;
                }
            }
            if (D.dump && tau <= D.dump_tmax) {
                const int64_t TT = D.dump_tmax;
                for (int64_t d = max(a, -TT) + tid; d < min(b, TT + 1); d += nt)
                    D.dump[tau * (2 * TT + 1) + d + TT] = cur[d - off];
            }
            __syncthreads();
        }
        if (fin)
            return true;
        t += h;
        C.blocks++;
        // ---------------------------------------------- halo exchange
        const uint64_t tw0 = gtimer();
        const int parity = (int)((t / h) & 1);
        const int32_t *last = S.F[(t - 1) & 1];
        int32_t *hl = halo_ptr(P, blockIdx.x, parity, 0), *hr = halo_ptr(P, blockIdx.x, parity, 1);
        if (tid < h) {
            const int64_t dl = a + tid, dr = b - h + tid;
            st_cg(hl + tid, dl < b ? last[dl - off] : NEG);
            st_cg(hr + tid, dr >= a ? last[dr - off] : NEG);
        }
        __threadfence();
        __syncthreads();
        const unsigned long long want = (iter << 32) | (unsigned long long)t;
        if (tid == 0)
            st_release_u64(&P.ctl->flags[blockIdx.x], want);
        // wait for both neighbours, helping open slides meanwhile
        const uint64_t t0 = tid == 0 ? gtimer() : 0;
        for (;;) {
            if (tid == 0) {
                int st = 0;
                const bool lok = T.left < 0 || ld_acquire_u64(&P.ctl->flags[T.left]) >= want;
                const bool rok = T.right < 0 || ld_acquire_u64(&P.ctl->flags[T.right]) >= want;
                if (lok && rok)
                    st = 3;
                else if (*(volatile unsigned long long *)&gc->done_k != ~0ull)
                    st = 1;
                else if (ld_acquire(&P.ctl->error) != 0)
                    st = 2;
                else if (gtimer() - t0 > P.idle_ns) {
                    wait_failed(P, 4, t, want, T.left >= 0 ? ld_acquire_u64(&P.ctl->flags[T.left]) : ~0ull,
                                T.right >= 0 ? ld_acquire_u64(&P.ctl->flags[T.right]) : ~0ull,
                                ((unsigned long long)(uint32_t)T.left << 32) | (uint32_t)T.right);
                    st = 2;
                }
                S.bc[1] = st;
            }
            __syncthreads();
            const int st = S.bc[1];
            __syncthreads();
            if (st == 1)
                return true;
            if (st == 2)
                return false;
            if (st == 3)
                break;
            help_one(P, S);
        }
        int32_t *edge = S.F[(t - 1) & 1];
        if (tid < h) {
            edge[a - h + tid - off] = T.left >= 0 ? ld_cg(halo_ptr(P, T.left, parity, 1) + tid) : NEG;
            edge[b + tid - off] = T.right >= 0 ? ld_cg(halo_ptr(P, T.right, parity, 0) + tid) : NEG;
        }
        __syncthreads();
        C.tm[2] += gtimer() - tw0;
    }
}

__device__ void flush_counters(const PairDesc &D, Counters &C, bool first_cta)
{
    unsigned long long v[6] = {C.slide, C.mism, C.hashq, C.coll, C.longs, C.blocks};
    for (int o = 16; o; o >>= 1)
        for (int i = 0; i < 6; i++)
            v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
    if ((threadIdx.x & 31) == 0) {
        if (v[0]) atomicAdd(&D.res[R_SLIDE], v[0]);
        if (v[1]) atomicAdd(&D.res[R_MISMATCH], v[1]);
        if (v[2]) atomicAdd(&D.res[R_HASHQ], v[2]);
        if (v[3]) atomicAdd(&D.res[R_HASHCOLL], v[3]);
        if (v[4]) atomicAdd(&D.res[R_LONG], v[4]);
    }
    if (first_cta && threadIdx.x == 0) {
        D.res[R_WIDE] = C.blocks;
        for (int i = 0; i < 4; i++)
            D.res[R_T0 + i] = C.tm[i];
    }
    C = Counters();
}

__global__ void __launch_bounds__(CTA_THREADS, 1) lv_tiles_kernel(LvArgs P)
{
    const Smem S = carve(P);
    const int G = P.group_size;
    const int grp = blockIdx.x / G, gi = blockIdx.x % G, c0 = grp * G;
    GroupCtl *gc = &P.gctl[grp];
    int32_t *gfb = P.gf + (int64_t)grp * P.gf_stride;
    Counters C;
    for (unsigned long long iter = 1;; iter++) {
        if (gi == 0 && threadIdx.x == 0) {
            const uint32_t q = atomicAdd(&P.ctl->queue, 1u);
            gc->pair = q < (uint32_t)P.npairs ? (int32_t)q : -1;
            gc->done_k = ~0ull;
            gc->epoch_req = 0;
            gc->epoch_t = 0;
            gc->ebar_count = 0; // no CTA is inside the epoch barrier here
            __threadfence();
        }
        if (!group_sync(P, gc, G, S))
            break;
        const int q = *(volatile int32_t *)&gc->pair;
        if (q < 0)
            break;
        const PairDesc D = P.pairs[q];
        const bool ok = run_pair(P, S, D, gc, gi, G, c0, gfb, iter, C);
        flush_counters(D, C, gi == 0);
        if (!ok)
            break;
        if (!group_sync(P, gc, G, S))
            break;
    }
}

cudaError_t launch_lv_tiles(const LvArgs &P, int grid, cudaStream_t s)
{
    const size_t smem = lv_tiles_smem_bytes(P.smax, P.h);
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
                    const int64_t hh = hash_lcp(H.pow2, H.TA, H.TB, x, y, l, lim);
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

// Method 2: each CTA claims chunks of the queries' slots (published by the
// host, claim = (1 << 32)) until none is left; the results stay in slots.
__global__ void __launch_bounds__(CTA_THREADS) lcp_grid_kernel(JobSlot *slots, int nslots)
{
    __shared__ unsigned long long s_min;
    __shared__ long long s_c;
    Smem S{};
    S.smin = &s_min;
    for (int j = 0; j < nslots; j++) {
        JobSlot *sl = &slots[(j + blockIdx.x) % nslots];
        for (;;) {
            if (threadIdx.x == 0) {
                int64_t c;
                while ((c = try_claim(sl)) == -2) {
                }
                s_c = c;
            }
            __syncthreads();
            const int64_t c = s_c;
            __syncthreads();
            if (c < 0)
                break;
            scan_chunk(S, sl, c);
        }
    }
}

cudaError_t launch_lcp_queries(const uint8_t *A, int64_t n, const uint8_t *B, int64_t m,
                               const int64_t *x, const int64_t *y, int64_t q, int method,
                               const HashArgs *hash, int64_t *out, JobSlot *slots, int grid,
                               cudaStream_t s)
{
    if (q == 0)
        return cudaSuccess;
    if (method == 2) {
        lcp_grid_kernel<<<grid, CTA_THREADS, 0, s>>>(slots, (int)q);
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
