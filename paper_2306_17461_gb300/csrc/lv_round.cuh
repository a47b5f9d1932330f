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
template <int DPT> // diagonals per thread per batch
__device__ __forceinline__ RoundCount tile_round(const RoundArgs &R)
{
    RoundCount out = {0, 0};
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int64_t base = R.lo; base <= R.hi; base += (int64_t)nt * DPT) {
        int64_t c[DPT];
        uint2 wa[DPT], wb[DPT];
#pragma unroll
        for (int u = 0; u < DPT; u++) {
            const int64_t d = base + (int64_t)u * nt + tid;
            c[u] = 0;
            wa[u] = wb[u] = make_uint2(0u, 0u);
            if (d <= R.hi) {
                c[u] = start_row(R.prev, R.off, d, R.tau, R.n, R.m);
                if (c[u] < 0 || c[u] + d < 0) {
                    // a start row outside the grid: record it, never load it
                    if (atomicCAS(R.err, 0u, 6u) == 0u) {
                        R.diag[0] = 6;
                        R.diag[1] = blockIdx.x;
                        R.diag[2] = (unsigned long long)R.tau;
                        R.diag[3] = (unsigned long long)d;
                        R.diag[4] = (unsigned long long)c[u];
                        R.diag[5] = ((unsigned long long)(uint32_t)R.prev[d - 1 - R.off] << 32) |
                                    (uint32_t)R.prev[d + 1 - R.off];
                        R.diag[6] = (unsigned long long)R.off;
                    }
                    c[u] = -1; // skipped below: no load at a bad row
                } else if (min(R.n - c[u], R.m - c[u] - d) > 0) {
                    word_load2(R.A, R.n, R.B, R.m, c[u], c[u] + d, wa[u], wb[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < DPT; u++) {
            const int64_t d = base + (int64_t)u * nt + tid;
            if (d <= R.hi && c[u] >= 0) {
                const int64_t cc = c[u];
                const int64_t full = min(R.n - cc, R.m - cc - d);
                const int64_t l = word_slide2(R.A, R.B, cc, cc + d, full, wa[u], wb[u]);
                if (l >= 0) {
                    R.cur[d - R.off] = (int32_t)(cc + l);
                    if (d >= R.a && d < R.b) {
                        out.slide += l;
                        out.mism += (l < full);
                    }
                } else {
                    R.open[atomicAdd(R.n1, 1)] = (int32_t)d;
                }
            }
        }
    }
    return out;
}

} // namespace edg
