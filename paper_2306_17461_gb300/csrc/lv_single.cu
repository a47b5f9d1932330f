// lv_single.cu -- one string pair, all k rounds of Algorithm 1 (Sec. 3.1,
// Appendix A) in ONE persistent cooperative launch.
//
// Round t sets, for every diagonal d in [-t, t] with a cell,
//     c        = max(L_{t-1}[d-1], L_{t-1}[d] + 1, L_{t-1}[d+1] + 1)
//     c        = min(c, n, m - d)           (clamp to the diagonal's last cell)
//     L_t[d]   = c + LCP(A[c..], B[c+d..])   (the slide)
// and stops at the first t with L_t[m-n] = n (then k = t).  This is the
// paper's loop with i = -d; taking the max before one slide gives the same
// row as sliding the three candidates and taking the max.
//
// Phases of the launch (all CTAs resident: cooperative launch):
//   narrow  -- while the band fits W0 diagonals, CTA 0 alone runs the rounds
//              with the frontier in shared memory (one __syncthreads per
//              round).  A slide still open after one thread (t1_cap bytes)
//              goes to one warp (t2_cap bytes, ballot/ffs); one still open
//              after that is published to the other CTAs, which wait idle
//              for such jobs and split it into 64 KiB chunks (atomicMin of
//              the first mismatch).
//   wide    -- once the band outgrows W0, every CTA takes an equal share of
//              the band each round; frontiers live in L2-resident global
//              memory; rounds are separated by a bounded grid barrier; long
//              slides of the round are split over the whole grid.
// Every wait is bounded by %globaltimer and reports ST_TIMEOUT instead of
// hanging.
#include "ed_device.cuh"
#include "lv_kernels.cuh"

namespace edg {

struct Counters {
    unsigned long long slide = 0, mism = 0, hashq = 0, coll = 0;
};

// ------------------------------------------------------------------ hash
__device__ __forceinline__ uint64_t powp(const HashArgs &H, int64_t e)
{
    uint64_t r = 1;
    for (int j = 0; e; j++, e >>= 1)
        if (e & 1)
            r = mulmod61(r, H.pow2[j]);
    return r;
}

// h(A[x..x+L)) == h(B[y..y+L)) with h(S2) = h([S1,S2]) - p^|S2| h(S1).
__device__ __forceinline__ bool hash_eq(const HashArgs &H, int64_t x, int64_t y, int64_t L,
                                        uint64_t P)
{
    const uint64_t a = submod61(__ldg(H.TA + x + L), mulmod61(__ldg(H.TA + x), P));
    const uint64_t b = submod61(__ldg(H.TB + y + L), mulmod61(__ldg(H.TB + y), P));
    return a == b;
}

// Sec. 3.2: compare chunks of length 1, 2, 4, ... (here: the powers of two
// above the l0 bytes already known equal) until one differs, then search
// the last bracket.  Returns the hash LCP (< = lim); the caller confirms it.
__device__ __noinline__ int64_t hash_lcp(const HashArgs &H, int64_t x, int64_t y, int64_t l0, int64_t lim)
{
    int64_t good = l0, bad;
    uint64_t pg = powp(H, good);
    int j = 0;
    while (j < 62 && (1ll << j) <= good)
        j++;
    for (;; j++) {
        const int64_t L = 1ll << j;
        if (L >= lim) {
            if (hash_eq(H, x, y, lim, powp(H, lim)))
                return lim;
            bad = lim;
            break;
        }
        if (hash_eq(H, x, y, L, H.pow2[j])) {
            good = L;
            pg = H.pow2[j];
        } else {
            bad = L;
            break;
        }
    }
    // largest length in [good, bad) whose hashes agree (binary lifting)
    for (int i = 62 - __clzll((long long)(bad - good)); i >= 0; i--) {
        const int64_t cand = good + (1ll << i);
        if (cand < bad) {
            const uint64_t P = mulmod61(pg, H.pow2[i]);
            if (hash_eq(H, x, y, cand, P)) {
                good = cand;
                pg = P;
            }
        }
    }
    return good;
}

// ------------------------------------------------------------------ slides
constexpr int DPT = 4; // diagonals per thread per batch in phase A

// Phase A of a round over diagonals [lo, hi] (strided over the CTA): the
// start row c = getc(d), then the slide by one thread.  DPT diagonals per
// thread are handled together so that their first loads overlap.  done(d,
// row) receives finished slides; open(d, c, pos, lim_abs) receives slides
// still open after t1_cap bytes (A[c..pos) matched; the first mismatch lies
// in [pos, lim_abs], lim_abs possibly lowered by the hash answer).
template <class GetC, class Done, class Open>
__device__ __forceinline__ void phase_a(const PairArgs &P, int64_t lo, int64_t hi, GetC getc, Done done,
                                        Open open_, Counters &C)
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
                if (min(P.n - c[u], P.m - c[u] - d) > 0)
                    word_load(P.A, P.B, c[u], c[u] + d, wa[u], wb[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < DPT; u++) {
            const int64_t d = base + (int64_t)u * nt + tid;
            if (d <= hi) {
                const int64_t cc = c[u];
                const int64_t full = min(P.n - cc, P.m - cc - d);
                bool op;
                const int64_t l = slide_thread_w(P.A, P.n, P.B, P.m, cc, cc + d, full, P.t1_cap,
                                                 wa[u], wb[u], &op);
                if (!op) {
                    done(d, cc + l);
                    C.slide += l;
                    C.mism += (l < full);
                } else {
                    int64_t lim = full;
                    if (P.use_hash) {
                        const int64_t h = hash_lcp(P.hash, cc, cc + d, l, full);
                        C.hashq++;
                        lim = min(h + 1, full);
                    }
                    open_(d, cc, cc + l, cc + lim);
                }
            }
        }
    }
}

// An open slide of diagonal d (start row c) reached row p: either a
// mismatch at p < lim_abs, or no mismatch before lim_abs (p == lim_abs).
// Returns the final row.  When the hash bound cut the search short and the
// direct compare found no mismatch at the hash answer (a collision), the
// slide is finished directly by this thread (a path taken with probability
// about l / 2^61).
__device__ __forceinline__ int64_t finish_slide(const PairArgs &P, int64_t c, int64_t d, int64_t p,
                                                int64_t lim_abs, Counters &C)
{
    const int64_t full_abs = c + min(P.n - c, P.m - c - d);
    if (P.use_hash && lim_abs < full_abs) {
        // hash answer h = lim_abs - 1 - c; any other outcome is a collision
        if (p != lim_abs - 1)
            C.coll++;
        if (p == lim_abs) {
            bool open;
            p += slide_thread(P.A, P.n, P.B, P.m, p, p + d, full_abs - p, INT64_MAX, &open);
        }
    }
    C.slide += p - c;
    C.mism += (p < full_abs);
    return p;
}

// The calling CTA's share (chunks h, h+G, ...) of every long item.
__device__ __noinline__ void grid_share(const PairArgs &P, LongItem *items, int nitems, int h, int G,
                           unsigned long long *s_min, int *s_stop)
{
    const int tid = threadIdx.x;
    for (int j = 0; j < nitems; j++) {
        const int64_t x = __ldcg(&items[j].x), y = __ldcg(&items[j].y),
                      lim = __ldcg(&items[j].lim);
        for (int64_t c = h;; c += G) {
            const int64_t cs = c * (int64_t)CHUNK_BYTES;
            if (tid == 0)
                *s_stop = (cs >= lim) ||
                          (cs >= (int64_t)(*(volatile unsigned long long *)&items[j].result));
            __syncthreads();
            const int stop = *s_stop;
            __syncthreads();
            if (stop)
                break;
            const int64_t r = cta_scan(P.A, P.n, P.B, P.m, x, y, cs,
                                       min((int64_t)CHUNK_BYTES, lim - cs), s_min);
            if (r >= 0) {
                if (tid == 0)
                    atomicMin(&items[j].result, (unsigned long long)r);
                break;
            }
        }
    }
}

__device__ __forceinline__ void set_error(LvJob *job, uint32_t code)
{
    atomicCAS(&job->error, 0u, code);
}

// Bounded grid barrier (sense by generation counter).  Returns false on
// timeout or when another CTA reported an error.
__device__ bool grid_sync(const PairArgs &P, int *s_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        LvJob *job = P.job;
        int ok = 1;
        const uint32_t gen = ld_acquire(&job->bar_gen);
        __threadfence();
        const uint32_t arrived = atomicAdd(&job->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&job->bar_count, 0u);
            __threadfence();
            st_release(&job->bar_gen, gen + 1);
        } else {
            const uint64_t t0 = gtimer();
            while (ld_acquire(&job->bar_gen) == gen) {
                if (ld_acquire(&job->error) != 0) {
                    ok = 0;
                    break;
                }
                if (gtimer() - t0 > P.spin_ns) {
                    set_error(job, ST_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        *s_flag = ok;
    }
    __syncthreads();
    const int ok = *s_flag;
    __syncthreads();
    return ok != 0;
}

struct Smem {
    int32_t *f[2];      // narrow frontiers
    int32_t *ld, *lc;   // open-slide list: diagonal, start row
    int64_t *lpos, *llim;
    int *n1, *n2, *flag, *stop;
    unsigned long long *smin;
    uint32_t *kind, *nitems, *epoch;
    int lcap;
};

__device__ Smem carve(int W0)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem S;
    unsigned char *p = smem_raw;
    S.smin = reinterpret_cast<unsigned long long *>(p);
    p += 16;
    S.n1 = reinterpret_cast<int *>(p);
    S.n2 = S.n1 + 1;
    S.flag = S.n1 + 2;
    S.stop = S.n1 + 3;
    S.kind = reinterpret_cast<uint32_t *>(S.n1 + 4);
    S.nitems = S.kind + 1;
    S.epoch = S.kind + 2;
    p += 64;
    S.lcap = W0 + 1;
    S.lpos = reinterpret_cast<int64_t *>(p);
    p += sizeof(int64_t) * S.lcap;
    S.llim = reinterpret_cast<int64_t *>(p);
    p += sizeof(int64_t) * S.lcap;
    S.f[0] = reinterpret_cast<int32_t *>(p);
    p += sizeof(int32_t) * (W0 + 3);
    S.f[1] = reinterpret_cast<int32_t *>(p);
    p += sizeof(int32_t) * (W0 + 3);
    S.ld = reinterpret_cast<int32_t *>(p);
    p += sizeof(int32_t) * S.lcap;
    S.lc = reinterpret_cast<int32_t *>(p);
    return S;
}

size_t lv_single_smem_bytes(int W0)
{
    const size_t lcap = (size_t)W0 + 1;
    return 16 + 64 + 2 * sizeof(int64_t) * lcap + 2 * sizeof(int32_t) * (W0 + 3) +
           2 * sizeof(int32_t) * lcap + 16;
}

__device__ void flush_counters(const PairArgs &P, Counters &C)
{
    // warp-reduce, then one atomic per warp
    for (int o = 16; o; o >>= 1) {
        C.slide += __shfl_down_sync(0xffffffffu, C.slide, o);
        C.mism += __shfl_down_sync(0xffffffffu, C.mism, o);
        C.hashq += __shfl_down_sync(0xffffffffu, C.hashq, o);
        C.coll += __shfl_down_sync(0xffffffffu, C.coll, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (C.slide) atomicAdd(&P.res[R_SLIDE], C.slide);
        if (C.mism) atomicAdd(&P.res[R_MISMATCH], C.mism);
        if (C.hashq) atomicAdd(&P.res[R_HASHQ], C.hashq);
        if (C.coll) atomicAdd(&P.res[R_HASHCOLL], C.coll);
    }
}

// ------------------------------------------------------------------ wide
// wide frontier index: d in [-kcap-2, kcap+2] -> [0, 2*kcap+4]
__device__ __forceinline__ int64_t gidx(const PairArgs &P, int64_t d) { return d + P.kcap + 2; }

// The entries just outside the band of round t must read as minus
// infinity in round t+1 (the buffers are never cleared): write them.
__device__ __forceinline__ void wide_sentinels(const PairArgs &P, int32_t *buf, int64_t lo, int64_t hi)
{
    st_cg(buf + gidx(P, lo - 1), NEG);
    st_cg(buf + gidx(P, lo - 2), NEG);
    st_cg(buf + gidx(P, hi + 1), NEG);
    st_cg(buf + gidx(P, hi + 2), NEG);
}

__device__ __noinline__ void wide_loop(const PairArgs &P, const Smem &S, int64_t t, Counters &C)
{
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5,
              nw = nt >> 5;
    const int g = blockIdx.x, G = gridDim.x;
    LvJob *job = P.job;
    const int64_t target = P.m - P.n;
    for (;; t++) {
        if (t > P.kcap) {
            if (g == 0 && tid == 0)
                set_error(job, ST_LIMIT);
            break;
        }
        const int32_t *prev = ((t - 1) & 1) ? P.gf1 : P.gf0;
        int32_t *cur = (t & 1) ? P.gf1 : P.gf0;
        const int64_t lo = max(-t, -P.n), hi = min(t, P.m);
        const int64_t cnt = hi - lo + 1, per = (cnt + G - 1) / G;
        const int64_t mlo = lo + (int64_t)g * per, mhi = min(hi, mlo + per - 1);
        if (g == 0 && tid == 0)
            wide_sentinels(P, cur, lo, hi);
        // phase A: one thread per diagonal
        phase_a(
            P, mlo, mhi,
            [&](int64_t d) {
                const int64_t a = ld_cg(prev + gidx(P, d - 1));
                const int64_t b = (int64_t)ld_cg(prev + gidx(P, d)) + 1;
                const int64_t e = (int64_t)ld_cg(prev + gidx(P, d + 1)) + 1;
                return min(max(a, max(b, e)), min(P.n, P.m - d));
            },
            [&](int64_t d, int64_t row) { st_cg(cur + gidx(P, d), (int32_t)row); },
            [&](int64_t d, int64_t c, int64_t pos, int64_t lim) {
                const int s = atomicAdd(S.n1, 1);
                if (s < S.lcap) {
                    S.ld[s] = (int32_t)d;
                    S.lc[s] = (int32_t)c;
                    S.lpos[s] = pos;
                    S.llim[s] = lim;
                } else {
                    bool open;
                    const int64_t p = pos + slide_thread(P.A, P.n, P.B, P.m, pos, pos + d, lim - pos,
                                                         INT64_MAX, &open);
                    st_cg(cur + gidx(P, d), (int32_t)finish_slide(P, c, d, p, lim, C));
                }
            },
            C);
        __syncthreads();
        const int n1 = min(*S.n1, S.lcap);
        if (n1 > 0) {
            // phase B: one warp per open slide
            for (int j = warp; j < n1; j += nw) {
                const int64_t d = S.ld[j], c = S.lc[j], pos = S.lpos[j], lim = S.llim[j];
                bool open;
                const int64_t l =
                    slide_warp(P.A, P.n, P.B, P.m, pos, pos + d, 0, lim - pos, P.t2_cap, &open);
                if (!open) {
                    if (lane == 0)
                        st_cg(cur + gidx(P, d), (int32_t)finish_slide(P, c, d, pos + l, lim, C));
                } else {
                    int slot = 0;
                    if (lane == 0)
                        slot = (int)atomicAdd(&job->glist[t % 3], 1u);
                    slot = __shfl_sync(0xffffffffu, slot, 0);
                    if (slot < P.item_cap) {
                        if (lane == 0) {
                            LongItem &it = P.items[slot];
                            it.x = pos + l;
                            it.y = pos + l + d;
                            it.lim = lim - pos - l;
                            it.result = (unsigned long long)(lim - pos - l);
                            it.d = (int32_t)d;
                            it.pad = (int32_t)c;
                            __threadfence();
                        }
                    } else {
                        // item list full: finish with this warp alone
                        bool o2;
                        const int64_t l2 = slide_warp(P.A, P.n, P.B, P.m, pos, pos + d, l, lim - pos,
                                                      INT64_MAX / 4, &o2);
                        if (lane == 0)
                            st_cg(cur + gidx(P, d), (int32_t)finish_slide(P, c, d, pos + l2, lim, C));
                    }
                }
            }
            __syncthreads();
            if (tid == 0)
                *S.n1 = 0;
        }
        if (!grid_sync(P, S.flag))
            break;
        if (g == 0 && tid == 0)
            job->glist[(t + 2) % 3] = 0;
        const int ng = (int)min((uint32_t)P.item_cap, ld_acquire(&job->glist[t % 3]));
        if (ng > 0) {
            if (g == 0 && tid == 0)
                atomicAdd(&P.res[R_LONG], (unsigned long long)ng);
            grid_share(P, P.items, ng, g, G, S.smin, S.stop);
            if (!grid_sync(P, S.flag))
                break;
            for (int j = g * nt + tid; j < ng; j += G * nt) {
                const LongItem &it = P.items[j];
                const int64_t d = __ldcg(&it.d), c = __ldcg(&it.pad);
                const int64_t r = (int64_t)atomicAdd(&P.items[j].result, 0ull);
                const int64_t x = __ldcg(&it.x);
                const int64_t lim_abs = x + __ldcg(&it.lim);
                st_cg(cur + gidx(P, d), (int32_t)finish_slide(P, c, d, x + r, lim_abs, C));
            }
            if (!grid_sync(P, S.flag))
                break;
        }
        if (g == 0 && tid == 0)
            atomicAdd(&P.res[R_WIDE], 1ull);
        if (P.dump && t <= P.dump_tmax) {
            const int64_t T = P.dump_tmax;
            for (int64_t d = mlo + tid; d <= mhi; d += nt)
                if (d >= -T && d <= T)
                    P.dump[t * (2 * T + 1) + d + T] = ld_cg(cur + gidx(P, d));
        }
        bool fin = false;
        if (target >= -t && target <= t)
            fin = (ld_cg(cur + gidx(P, target)) == P.n);
        if (fin) {
            if (g == 0 && tid == 0)
                P.res[R_K] = (unsigned long long)t;
            break;
        }
    }
}

// ------------------------------------------------------------------ narrow
__device__ __forceinline__ int nidx(int H, int64_t d) { return (int)(d + H + 1); }

// CTA 0: the round loop while the band fits W0.  Returns the round to start
// the wide phase from, or -1 when finished (or failed).
__device__ __noinline__ int64_t narrow_loop(const PairArgs &P, const Smem &S, Counters &C)
{
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5,
              nw = nt >> 5;
    const int G = gridDim.x;
    const int H = P.W0 / 2;
    LvJob *job = P.job;
    const int64_t target = P.m - P.n;
    for (int i = tid; i < P.W0 + 3; i += nt) {
        S.f[0][i] = NEG;
        S.f[1][i] = NEG;
    }
    if (tid == 0) {
        *S.n1 = 0;
        *S.n2 = 0;
        *S.epoch = 0;
    }
    __syncthreads();
    for (int64_t t = 0;; t++) {
        const int64_t lo = max(-t, -P.n), hi = min(t, P.m);
        if (lo < -H || hi > H) {
            // hand over to the whole grid: publish round t-1 to global memory
            int32_t *g = ((t - 1) & 1) ? P.gf1 : P.gf0;
            const int32_t *src = S.f[(t - 1) & 1];
            const int64_t plo = max(-(t - 1), -P.n), phi = min(t - 1, P.m);
            for (int64_t d = plo + tid; d <= phi; d += nt)
                st_cg(g + gidx(P, d), src[nidx(H, d)]);
            if (tid == 0)
                wide_sentinels(P, g, plo, phi);
            __threadfence();
            __syncthreads();
            if (tid == 0) {
                job->wide_t = (uint32_t)t;
                job->kind = JOB_WIDE;
                __threadfence();
                st_release(&job->epoch, *S.epoch + 1);
            }
            __syncthreads();
            return t;
        }
        const int32_t *prev = S.f[(t - 1) & 1];
        int32_t *cur = S.f[t & 1];
        phase_a(
            P, lo, hi,
            [&](int64_t d) -> int64_t {
                if (t == 0)
                    return 0;
                const int64_t a = prev[nidx(H, d - 1)];
                const int64_t b = (int64_t)prev[nidx(H, d)] + 1;
                const int64_t e = (int64_t)prev[nidx(H, d + 1)] + 1;
                return min(max(a, max(b, e)), min(P.n, P.m - d));
            },
            [&](int64_t d, int64_t row) { cur[nidx(H, d)] = (int32_t)row; },
            [&](int64_t d, int64_t c, int64_t pos, int64_t lim) {
                const int s = atomicAdd(S.n1, 1); // < lcap: band <= W0 + 1
                S.ld[s] = (int32_t)d;
                S.lc[s] = (int32_t)c;
                S.lpos[s] = pos;
                S.llim[s] = lim;
            },
            C);
        __syncthreads();
        const int n1 = *S.n1;
        if (n1 > 0) {
            for (int j = warp; j < n1; j += nw) {
                const int64_t d = S.ld[j], c = S.lc[j], pos = S.lpos[j], lim = S.llim[j];
                bool open;
                const int64_t l =
                    slide_warp(P.A, P.n, P.B, P.m, pos, pos + d, 0, lim - pos, P.t2_cap, &open);
                if (!open) {
                    if (lane == 0)
                        cur[nidx(H, d)] = (int32_t)finish_slide(P, c, d, pos + l, lim, C);
                } else if (lane == 0) {
                    const int s = atomicAdd(S.n2, 1); // < item_cap >= W0 + 1
                    LongItem &it = P.items[s];
                    it.x = pos + l;
                    it.y = pos + l + d;
                    it.lim = lim - pos - l;
                    it.result = (unsigned long long)(lim - pos - l);
                    it.d = (int32_t)d;
                    it.pad = (int32_t)c;
                    __threadfence();
                }
            }
            __syncthreads();
            const int n2 = *S.n2;
            if (tid == 0)
                *S.n1 = 0;
            if (n2 > 0) {
                // publish the long slides to the helper CTAs and take share 0
                if (tid == 0) {
                    job->nitems = (uint32_t)n2;
                    job->kind = JOB_LONG;
                    *S.epoch += 1;
                    __threadfence();
                    st_release(&job->epoch, *S.epoch);
                    atomicAdd(&P.res[R_LONG], (unsigned long long)n2);
                }
                __syncthreads();
                const uint32_t ep = *S.epoch;
                grid_share(P, P.items, n2, 0, G, S.smin, S.stop);
                int ok = 1;
                for (int h = 1 + tid; h < G; h += nt) {
                    const uint64_t t0 = gtimer();
                    while (ld_acquire(&job->done[h]) != ep) {
                        if (gtimer() - t0 > P.spin_ns) {
                            set_error(job, ST_TIMEOUT);
                            ok = 0;
                            break;
                        }
                    }
                    if (!ok)
                        break;
                }
                if (!__syncthreads_and(ok))
                    return -1;
                for (int j = tid; j < n2; j += nt) {
                    const LongItem &it = P.items[j];
                    const int64_t d = __ldcg(&it.d), c = __ldcg(&it.pad), x = __ldcg(&it.x);
                    const int64_t r = (int64_t)atomicAdd(&P.items[j].result, 0ull);
                    cur[nidx(H, d)] = (int32_t)finish_slide(P, c, d, x + r, x + __ldcg(&it.lim), C);
                }
                __syncthreads();
                if (tid == 0)
                    *S.n2 = 0;
            }
        }
        if (P.dump && t <= P.dump_tmax) {
            const int64_t T = P.dump_tmax;
            for (int64_t d = lo + tid; d <= hi; d += nt)
                if (d >= -T && d <= T)
                    P.dump[t * (2 * T + 1) + d + T] = cur[nidx(H, d)];
        }
        const bool fin = (target >= lo && target <= hi) && cur[nidx(H, target)] == P.n;
        __syncthreads();
        if (fin) {
            if (tid == 0)
                P.res[R_K] = (unsigned long long)t;
            return -1;
        }
    }
}

// ------------------------------------------------------------------ kernel
__global__ void __launch_bounds__(CTA_THREADS, 1) lv_single_kernel(PairArgs P)
{
    const Smem S = carve(P.W0);
    const int tid = threadIdx.x;
    Counters C;
    LvJob *job = P.job;
    if (blockIdx.x == 0) {
        const int64_t tw = narrow_loop(P, S, C);
        if (tw >= 0)
            wide_loop(P, S, tw, C);
        __syncthreads();
        if (tid == 0) {
            // release the helpers (those already in the wide phase have left)
            job->kind = JOB_QUIT;
            __threadfence();
            st_release(&job->epoch, 0xffffffffu);
        }
    } else {
        uint32_t my = 0;
        for (;;) {
            if (tid == 0) {
                const uint64_t t0 = gtimer();
                uint32_t e;
                int ok = 1;
                while ((e = ld_acquire(&job->epoch)) == my) {
                    if (ld_acquire(&job->error) != 0 || gtimer() - t0 > P.idle_ns) {
                        set_error(job, ST_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
                *S.epoch = e;
                *S.kind = ok ? ld_acquire(&job->kind) : JOB_QUIT;
                *S.nitems = ld_acquire(&job->nitems);
                *S.n1 = 0;
            }
            __syncthreads();
            const uint32_t kind = *S.kind, e = *S.epoch;
            const int nitems = (int)*S.nitems;
            __syncthreads();
            if (kind == JOB_QUIT || e == 0xffffffffu)
                break;
            my = e;
            if (kind == JOB_WIDE) {
                wide_loop(P, S, (int64_t)ld_acquire(&job->wide_t), C);
                break;
            }
            if (kind == JOB_LONG) {
                grid_share(P, P.items, nitems, blockIdx.x, gridDim.x, S.smin, S.stop);
                __syncthreads();
                if (tid == 0) {
                    __threadfence();
                    st_release(&job->done[blockIdx.x], my);
                }
            }
        }
    }
    flush_counters(P, C);
    if (blockIdx.x == 0 && tid == 0) {
        __threadfence();
        P.res[R_STATUS] = ld_acquire(&job->error);
    }
}

cudaError_t launch_lv_single(const PairArgs &P, int grid, cudaStream_t s)
{
    const size_t smem = lv_single_smem_bytes(P.W0);
    cudaError_t e =
        cudaFuncSetAttribute(lv_single_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    PairArgs Pc = P;
    void *args[] = {&Pc};
    return cudaLaunchCooperativeKernel((const void *)lv_single_kernel, dim3(grid), dim3(CTA_THREADS),
                                       args, smem, s);
}


// ------------------------------------------------------------------ tests
// LCP(A, B, x[i], y[i]) by the building blocks above, one query per thread
// (method 0), per warp (1), per whole grid (2: every CTA takes its chunks of
// every query), by the hash search alone (3) or hash + direct confirmation
// (4).
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
                    const int64_t h = hash_lcp(H, x, y, l, lim);
                    if (method == 3) {
                        l = h;
                    } else {
                        const int64_t cl = min(h + 1, lim);
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

__global__ void __launch_bounds__(CTA_THREADS) lcp_grid_kernel(PairArgs P, int nitems)
{
    __shared__ unsigned long long s_min;
    __shared__ int s_stop;
    grid_share(P, P.items, nitems, blockIdx.x, gridDim.x, &s_min, &s_stop);
}

cudaError_t launch_lcp_queries(const uint8_t *A, int64_t n, const uint8_t *B, int64_t m,
                               const int64_t *x, const int64_t *y, int64_t q, int method,
                               const HashArgs *hash, int64_t *out, LongItem *items, int grid,
                               cudaStream_t s)
{
    if (q == 0)
        return cudaSuccess;
    if (method == 2) {
        PairArgs P{};
        P.A = A;
        P.B = B;
        P.n = n;
        P.m = m;
        P.items = items;
        lcp_grid_kernel<<<grid, CTA_THREADS, 0, s>>>(P, (int)q);
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
