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

// PIPE: the pipelined form of the tile kernel.  A diagonal with a PENDING
// predecessor is deferred (listed in R.defer) instead of computed; an open
// slide is listed with its start row (R.open, R.open_c) and its value set to
// PENDING until a warp finishes it.
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
    // byte phases of the two strings' bases within a 4-byte word
    const uint32_t pa0 = (uint32_t)(uintptr_t)R.A, pb0 = (uint32_t)(uintptr_t)R.B;
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
            if (slot <= last_slot) {
                int32_t cc = 0;
                bool blocked = false;
                if (!first) {
                    const int32_t x1 = prev[d - 1 - off];
                    const int32_t x2 = prev[d - off];
                    const int32_t x3 = prev[d + 1 - off];
                    if (PIPE && min(x1, min(x2, x3)) == PENDING) {
                        R.defer[atomicAdd(R.nd, 1)] = d;
                        blocked = true;
                    }
                    cc = min(max(x1, max(x2, x3) + 1), d <= mn ? n : m - d);
                }
                if (blocked) {
                    // computed later, from the finished value
                } else if (cc < 0 || cc + d < 0) {
                    // a start row outside the grid: record it, never load it
                    if (atomicCAS(R.err, 0u, 6u) == 0u) {
                        R.diag[0] = 6;
                        R.diag[1] = blockIdx.x;
                        R.diag[2] = (unsigned long long)R.tau;
                        R.diag[3] = (unsigned long long)(int64_t)d;
                        R.diag[4] = (unsigned long long)(int64_t)cc;
                        R.diag[5] = ((unsigned long long)(uint32_t)prev[d - 1 - off] << 32) |
                                    (uint32_t)prev[d + 1 - off];
                        R.diag[6] = (unsigned long long)R.off;
                    }
                } else {
                    c[u] = cc;
                    if (min(n - cc, m - cc - d) > 0) {
                        // the aligned word holding A[cc] and the next one (only
                        // while it still holds a byte of A: then it cannot
                        // fault); the same for B[cc + d]
                        const int32_t ya = cc, yb = cc + d;
                        const uint32_t sa = (pa0 + (uint32_t)ya) & 3u, sb = (pb0 + (uint32_t)yb) & 3u;
                        const uint32_t *qa = reinterpret_cast<const uint32_t *>(R.A + (ya - (int32_t)sa));
                        const uint32_t *qb = reinterpret_cast<const uint32_t *>(R.B + (yb - (int32_t)sb));
                        wa[u].x = __ldg(qa);
                        wb[u].x = __ldg(qb);
                        wa[u].y = ya - (int32_t)sa + 4 < n ? __ldg(qa + 1) : 0u;
                        wb[u].y = yb - (int32_t)sb + 4 < m ? __ldg(qb + 1) : 0u;
                        sh[u] = sa | (sb << 8);
                    }
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
                // the bytes from A[cc] and B[cc + d] the two words hold: 8 - max(sa, sb)
                // (at least five); the first four by funnel shift, the rest after
                const uint32_t sa = sh[u] & 255u, sb = sh[u] >> 8;
                const uint32_t smax = max(sa, sb);
                const uint32_t m1 = __funnelshift_r(wa[u].x, wa[u].y, 8 * sa) ^ __funnelshift_r(wb[u].x, wb[u].y, 8 * sb);
                const uint32_t m2 = ((wa[u].y >> (8 * sa)) ^ (wb[u].y >> (8 * sb))) & (0xffffffffu >> (8 * smax));
                const int32_t av = 8 - (int32_t)smax;
                int32_t l = m1 ? (__ffs((int)m1) - 1) >> 3 : (m2 ? 4 + ((__ffs((int)m2) - 1) >> 3) : av);
                if (full <= 0)
                    l = 0;
                else if (l >= full)
                    l = full;
                else if (l == av)
                    l = -1; // every byte the words hold matched: a warp goes on
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

} // namespace edg
