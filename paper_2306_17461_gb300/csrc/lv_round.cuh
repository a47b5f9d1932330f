// lv_round.cuh -- one round of Algorithm 1 (Sec. 3.1, Appendix A) over a
// contiguous range of diagonals held in shared memory, shared by the tile
// kernel and the batch kernel.
//
// For each diagonal d of [lo, hi]:
//     c      = max(L_{t-1}[d-1], L_{t-1}[d] + 1, L_{t-1}[d+1] + 1), clamped
//              to the diagonal's last cell min(n, m - d)
//     L_t[d] = c + LCP(A[c..], B[c+d..])
// The slide is taken here as far as the aligned words at the start row
// decide it (one load per string and word, all of a thread's diagonals in
// flight together); slides that match all the bytes those words hold are
// listed for the caller, which continues them a warp each.
#pragma once
#include "ed_device.cuh"

namespace edg {

// The frontier value of a diagonal whose slide a warp is still finishing
// (pipelined rounds): below the minus infinity of undefined diagonals.
constexpr int32_t PENDING = INT32_MIN;
// The frontier value of a diagonal of the round being computed that waits
// for a PENDING predecessor, and of one a slider warp is computing (it
// claimed it from DEFER_MARK); neither survives the round.
constexpr int32_t DEFER_MARK = INT32_MIN + 1;
constexpr int32_t DEFER_CLAIM = INT32_MIN + 2;

struct RoundArgs {
    const uint8_t *A, *B;
    int64_t n, m;
    const int32_t *prev;     // round tau-1, indexed d - off
    int32_t *cur;            // round tau
    int64_t off, lo, hi, tau, a, b;
    int *n1;
    int32_t *open;           // diagonals whose slide is still open
    uint32_t *err;           // launch status word (self-check records)
    unsigned long long *diag;
    int tid, nt;             // this thread among the nt that run the round
    // pipelined rounds only: the start rows of the open list (ocap entries at
    // most), and the diagonals deferred because a predecessor is PENDING
    int32_t *open_c;
    int ocap;
    int32_t *defer;
    int *nd;
    // list mode: the diagonals list[0..nlist) instead of [lo, hi]
    const int32_t *list;
    int nlist;
};
struct RoundCount {
    unsigned long long slide, mism;
};

// The start row of diagonal d in round tau from the three predecessors,
// clamped to the diagonal's last cell.
__device__ __forceinline__ int64_t start_row(const int32_t *prev, int64_t off, int64_t d, int64_t tau,
                                             int64_t n, int64_t m)
{
    if (tau == 0)
        return 0;
    const int64_t x1 = prev[d - 1 - off];
    const int64_t x2 = (int64_t)prev[d - off] + 1;
    const int64_t x3 = (int64_t)prev[d + 1 - off] + 1;
    return min(max(x1, max(x2, x3)), min(n, m - d));
}

// One round over diagonals [lo, hi] of the tile (strided over the CTA): the
// start row, then the word slide.  DPT diagonals per thread are handled
// together so that their loads are in flight together.  Diagonals whose
// slide is still open are listed; the list holds one entry per computed
// diagonal at most, so it cannot fill.  Counts only diagonals of [a, b).
//
// Rows, diagonals and lengths are below 2^31 (strings are shorter than
// 2^31 bytes), so the round works in 32-bit integers; the one quantity that
// can exceed that, m - d (up to n + m), appears only in the clamp, which
// takes n whenever d <= m - n.
// An open slide that found the open list full finishes here, one thread,
// 16-byte windows: only for inputs where more than ocap slides of a round
// stay open (long common runs on every diagonal).
static __device__ __noinline__ int32_t slide_alone(const uint8_t *A, int64_t n, const uint8_t *B, int64_t m, int32_t c,
                                            int32_t d, int32_t full)
{
    bool open;
    return (int32_t)slide_thread(A, n, B, m, c, (int64_t)c + d, full, INT64_MAX, &open);
}

// The aligned 4-byte word holding A[c] and the next one (only while it still
// holds a byte of A: then it cannot fault), the same for B[c + d], and the
// byte offsets of A[c] and B[c + d] in their words (sa | sb << 8).  Needs
// min(n - c, m - c - d) > 0.
__device__ __forceinline__ void words_load(const uint8_t *A, const uint8_t *B, int32_t n, int32_t m, int32_t c,
                                           int32_t d, uint2 &wa, uint2 &wb, uint32_t &sh)
{
    const int32_t ya = c, yb = c + d;
    const uint32_t sa = ((uint32_t)(uintptr_t)A + (uint32_t)ya) & 3u, sb = ((uint32_t)(uintptr_t)B + (uint32_t)yb) & 3u;
    const uint32_t *qa = reinterpret_cast<const uint32_t *>(A + (ya - (int32_t)sa));
    const uint32_t *qb = reinterpret_cast<const uint32_t *>(B + (yb - (int32_t)sb));
    wa.x = __ldg(qa);
    wb.x = __ldg(qb);
    wa.y = ya - (int32_t)sa + 4 < n ? __ldg(qa + 1) : 0u;
    wb.y = yb - (int32_t)sb + 4 < m ? __ldg(qb + 1) : 0u;
    sh = sa | (sb << 8);
}

// The slide from the words of words_load, at most full bytes: the bytes
// from A[c] and B[c + d] the words hold, 8 - max(sa, sb) (at least five),
// the first four by funnel shift, the rest after.  -1: every byte the words
// hold matched and the slide may go on (a warp continues it).
__device__ __forceinline__ int32_t words_lcp(uint2 wa, uint2 wb, uint32_t sh, int32_t full)
{
    const uint32_t sa = sh & 255u, sb = sh >> 8;
    const uint32_t smax = max(sa, sb);
    const uint32_t m1 = __funnelshift_r(wa.x, wa.y, 8 * sa) ^ __funnelshift_r(wb.x, wb.y, 8 * sb);
    const uint32_t m2 = ((wa.y >> (8 * sa)) ^ (wb.y >> (8 * sb))) & (0xffffffffu >> (8 * smax));
    const int32_t av = 8 - (int32_t)smax;
    int32_t l = m1 ? (__ffs((int)m1) - 1) >> 3 : (m2 ? 4 + ((__ffs((int)m2) - 1) >> 3) : av);
    if (full <= 0)
        l = 0;
    else if (l >= full)
        l = full;
    else if (l == av)
        l = -1;
    return l;
}

// A start row outside the grid (a broken invariant): recorded once in the
// launch status, never loaded.
static __device__ __noinline__ void record_bad_row(uint32_t *err, unsigned long long *diag, int64_t tau,
                                                   const int32_t *prev, int32_t off, int32_t d, int32_t cc)
{
    if (atomicCAS(err, 0u, 6u) == 0u) {
        diag[0] = 6;
        diag[1] = blockIdx.x;
        diag[2] = (unsigned long long)tau;
        diag[3] = (unsigned long long)(int64_t)d;
        diag[4] = (unsigned long long)(int64_t)cc;
        diag[5] = ((unsigned long long)(uint32_t)prev[d - 1 - off] << 32) | (uint32_t)prev[d + 1 - off];
        diag[6] = (unsigned long long)(int64_t)off;
    }
}

// PIPE: the pipelined form of the tile kernel.  A diagonal with a PENDING
// predecessor is deferred (listed in R.defer, its value DEFER_MARK) instead
// of computed; an open slide is listed with its start row (R.open,
// R.open_c) and its value set to PENDING until a warp finishes it.  LIST:
// the deferred diagonals R.list[0..nlist) still marked DEFER_MARK (a slider
// warp may have computed the others).
template <int DPT, bool PIPE = false, bool LIST = false> // DPT: diagonals per thread per batch
__device__ __forceinline__ RoundCount tile_round(const RoundArgs &R)
{
    RoundCount out = {0, 0};
    const int tid = R.tid, nt = R.nt;
    const int32_t n = (int32_t)R.n, m = (int32_t)R.m, mn = (int32_t)(R.m - R.n);
    const int32_t off = (int32_t)R.off, lo = (int32_t)R.lo, hi = (int32_t)R.hi;
    const int32_t a = (int32_t)R.a, b = (int32_t)R.b;
    const bool first = R.tau == 0;
    const int32_t *prev = R.prev;
    int32_t *cur = R.cur;
    uint32_t slide = 0, mism = 0;
    const int32_t first_slot = LIST ? 0 : lo, last_slot = LIST ? R.nlist - 1 : hi;
    for (int32_t base = first_slot; base <= last_slot; base += nt * DPT) {
        int32_t c[DPT];
        uint32_t sh[DPT]; // byte offsets of A[c] and B[c+d] in their words: sa | sb << 8
        uint2 wa[DPT], wb[DPT];
#pragma unroll
        for (int u = 0; u < DPT; u++) {
            const int32_t slot = base + u * nt + tid;
            const int32_t d = LIST ? (slot <= last_slot ? R.list[slot] : 0) : slot;
            c[u] = -1;
            sh[u] = 0;
            wa[u] = wb[u] = make_uint2(0u, 0u);
            if (slot <= last_slot && (!LIST || cur[d - off] == DEFER_MARK)) {
                int32_t cc = 0;
                bool blocked = false;
                if (!first) {
                    const int32_t x1 = prev[d - 1 - off];
                    const int32_t x2 = prev[d - off];
                    const int32_t x3 = prev[d + 1 - off];
                    if (PIPE && min(x1, min(x2, x3)) == PENDING) {
                        R.defer[atomicAdd(R.nd, 1)] = d;
                        cur[d - off] = DEFER_MARK;
                        blocked = true;
                    }
                    cc = min(max(x1, max(x2, x3) + 1), d <= mn ? n : m - d);
                }
                if (blocked) {
                    // computed later, from the finished value
                } else if (cc < 0 || cc + d < 0) {
                    record_bad_row(R.err, R.diag, R.tau, prev, off, d, cc);
                } else {
                    c[u] = cc;
                    if (min(n - cc, m - cc - d) > 0)
                        words_load(R.A, R.B, n, m, cc, d, wa[u], wb[u], sh[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < DPT; u++) {
            const int32_t slot = base + u * nt + tid;
            const int32_t d = LIST ? (slot <= last_slot ? R.list[slot] : 0) : slot;
            if (slot <= last_slot && c[u] >= 0) {
                const int32_t cc = c[u];
                const int32_t full = min(n - cc, m - cc - d);
                const int32_t l = words_lcp(wa[u], wb[u], sh[u], full);
                if (l >= 0) {
                    cur[d - off] = cc + l;
                    if (d >= a && d < b) {
                        slide += (uint32_t)l;
                        mism += (l < full);
                    }
                } else if (!PIPE) {
                    R.open[atomicAdd(R.n1, 1)] = d;
                } else {
                    const int j = atomicAdd(R.n1, 1);
                    if (j < R.ocap) {
                        R.open[j] = d;
                        R.open_c[j] = cc;
                        cur[d - off] = PENDING;
                    } else {
                        const int32_t l2 = slide_alone(R.A, n, R.B, m, cc, d, full);
                        cur[d - off] = cc + l2;
                        if (d >= a && d < b) {
                            slide += (uint32_t)l2;
                            mism += (l2 < full);
                        }
                    }
                }
            }
        }
    }
    out.slide = slide;
    out.mism = mism;
    return out;
}

// One diagonal d of round R.tau (pipelined form), for a slider warp's lane
// that claimed it (its value DEFER_CLAIM): the start row from the three
// predecessors, the word slide, the open list, as tile_round computes it.
// Returns false, computing nothing, while a predecessor is still PENDING.
__device__ __forceinline__ bool round_one(const RoundArgs &R, int32_t d, RoundCount &rc)
{
    const int32_t n = (int32_t)R.n, m = (int32_t)R.m, mn = (int32_t)(R.m - R.n), off = (int32_t)R.off;
    const int32_t x1 = R.prev[d - 1 - off], x2 = R.prev[d - off], x3 = R.prev[d + 1 - off];
    if (min(x1, min(x2, x3)) == PENDING)
        return false;
    const int32_t cc = R.tau == 0 ? 0 : min(max(x1, max(x2, x3) + 1), d <= mn ? n : m - d);
    int32_t *cur = R.cur;
    if (cc < 0 || cc + d < 0) {
        record_bad_row(R.err, R.diag, R.tau, R.prev, off, d, cc);
        cur[d - off] = NEG;
        return true;
    }
    const int32_t full = min(n - cc, m - cc - d);
    int32_t l = 0;
    if (full > 0) {
        uint2 wa, wb;
        uint32_t sh;
        words_load(R.A, R.B, n, m, cc, d, wa, wb, sh);
        l = words_lcp(wa, wb, sh, full);
    }
    const bool own = d >= R.a && d < R.b;
    if (l < 0) {
        const int j = atomicAdd(R.n1, 1);
        if (j < R.ocap) {
            R.open[j] = d;
            R.open_c[j] = cc;
            cur[d - off] = PENDING;
            return true;
        }
        l = slide_alone(R.A, n, R.B, m, cc, d, full);
    }
    cur[d - off] = cc + l;
    if (own) {
        rc.slide += (unsigned long long)l;
        rc.mism += (l < full);
    }
    return true;
}

} // namespace edg
