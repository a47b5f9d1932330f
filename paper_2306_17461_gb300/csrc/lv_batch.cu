// lv_batch.cu -- many independent pairs in one persistent launch.
//
// Each CTA claims pairs from a work queue (atomicAdd on a head index over a
// cost-sorted order) and runs Algorithm 1 (Sec. 3.1) on its pair with the
// frontier in shared memory: per round, the shared round function (several
// diagonals' loads in flight per thread), then the open slides, one warp
// each, then the whole CTA for those still open.  A pair whose band outgrows
// W diagonals is parked (state 2) for the tile kernel.  With a time budget
// (serving), a CTA stops a pair at a round boundary once the budget is
// spent, saves the round's frontier in the pair's resident buffer, and the
// next launch resumes it.
#include "ed_device.cuh"
#include "lv_kernels.cuh"
#include "lv_round.cuh"

namespace edg {

constexpr int BT = 256; // threads per batch CTA

struct BSmem {
    int32_t *f0, *f1; // frontiers by round parity, W + 3 entries each (index d + W/2 + 1)
    int32_t *ld;     // open slides: diagonal (W + 1 entries)
    int *n1, *flag, *claim, *reach;
    uint32_t *err;   // self-check status of the round function
    unsigned long long *diag;
    unsigned long long *smin;
    long long *bcl;
};

size_t lv_batch_smem_bytes(int W)
{
    return 256 + sizeof(int32_t) * ((size_t)W + 1) + 2 * sizeof(int32_t) * ((size_t)W + 3);
}

__device__ BSmem bcarve(int W)
{
    extern __shared__ __align__(16) unsigned char bsmem_raw[];
    BSmem S;
    unsigned char *p = bsmem_raw;
    S.smin = reinterpret_cast<unsigned long long *>(p);
    S.diag = S.smin + 1;                            // 8 words
    S.bcl = reinterpret_cast<long long *>(p + 80);  // 4 words
    S.n1 = reinterpret_cast<int *>(p + 128);
    S.flag = S.n1 + 1;
    S.claim = S.n1 + 2;
    S.err = reinterpret_cast<uint32_t *>(S.n1 + 3);
    S.reach = S.n1 + 4;
    p += 256;
    S.ld = reinterpret_cast<int32_t *>(p);
    p += sizeof(int32_t) * (W + 1);
    S.f0 = reinterpret_cast<int32_t *>(p);
    p += sizeof(int32_t) * (W + 3);
    S.f1 = reinterpret_cast<int32_t *>(p);
    return S;
}

__device__ __forceinline__ int32_t *bfront(const BSmem S, int64_t r) { return (r & 1) ? S.f1 : S.f0; }

// The whole CTA finishes one open slide: the first mismatch of
// A[pos..lim_abs) vs B[pos+d..), 32 KiB per step with every load in flight.
__device__ __noinline__ int64_t cta_slide(const uint8_t *A, int64_t n, const uint8_t *B, int64_t m, int64_t d,
                                          int64_t pos, int64_t lim_abs, unsigned long long *s_min)
{
    constexpr int64_t STEP = (int64_t)BT * 16 * 4;
    for (int64_t off = 0; pos + off < lim_abs; off += STEP) {
        const int64_t len = min(STEP, lim_abs - pos - off);
        const int64_t r = cta_scan<4>(A, n, B, m, pos, pos + d, off, len, s_min);
        if (r >= 0)
            return pos + r;
    }
    return lim_abs;
}

// One warp's attempt at an open slide, out of line so that the round loop
// keeps its registers: the first mismatch within cap bytes of the start, or
// *open when there is none.
__device__ __forceinline__ int64_t warp_slide(const uint8_t *A, int64_t n, const uint8_t *B, int64_t m, int64_t c,
                                           int64_t d, int64_t len, int64_t cap, bool *open)
{
    return slide_warp(A, n, B, m, c, c + d, 0, len, cap, open);
}

__global__ void __launch_bounds__(BT, 2) lv_batch_kernel(BatchArgs Bg, uint64_t budget_ns)
{
    const BSmem S = bcarve(Bg.W);
    // 0 = no time budget; otherwise this CTA stops claiming and parks its
    // pair once budget_ns have passed since it started (thread 0 decides)
    const uint64_t deadline_ns = budget_ns ? gtimer() + budget_ns : 0;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int H = Bg.W / 2;
    const int64_t off = -(int64_t)H - 1; // smem index = d - off
    for (;;) {
        if (tid == 0) {
            int c = -1;
            if (deadline_ns == 0 || gtimer() < deadline_ns) {
                const uint32_t q = atomicAdd(Bg.next, 1u);
                if (q < (uint32_t)Bg.npairs)
                    c = Bg.order[q];
            }
            *S.claim = c;
            *S.n1 = 0;
            *S.err = 0;
            *S.reach = 0;
        }
        __syncthreads();
        const int pi = *S.claim;
        __syncthreads();
        if (pi < 0)
            break;
        BatchPair &Pr = Bg.pairs[pi];
        if (Pr.state != 0) // finished or parked: nothing to do
            continue;
        const uint8_t *A = Pr.A, *B = Pr.B;
        const int64_t n = Pr.n, m = Pr.m, target = m - n;
        // restore the resident frontier (round t0) or start at round 0
        const int64_t t0 = Pr.t;
        for (int i = tid; i < Bg.W + 3; i += nt) {
            S.f0[i] = NEG;
            S.f1[i] = NEG;
        }
        __syncthreads();
        if (t0 >= 0) {
            const int32_t *src = Pr.front;
            int32_t *dst = bfront(S, t0);
            for (int i = tid; i < Bg.W + 3; i += nt)
                dst[i] = src[i];
        }
        __syncthreads();
        unsigned long long slide = 0, mism = 0;
        int64_t t = t0 + 1;
        int outcome = 0; // 0 budget spent, 1 done, 2 band too wide, 3 self-check failed
        int rounds_here = 0;
        for (;; t++) {
            const int64_t lo = max(-t, -n), hi = min(t, m);
            if (lo < -H || hi > H) {
                outcome = 2;
                break;
            }
            // the budget decision is taken by one thread for the whole CTA:
            // threads reading the timer apart must not leave the loop apart
            if (tid == 0)
                *S.flag = rounds_here > 0 && ((Bg.round_budget > 0 && rounds_here >= Bg.round_budget) ||
                                              (deadline_ns != 0 && gtimer() >= deadline_ns));
            __syncthreads();
            const int spent = *S.flag;
            __syncthreads();
            if (spent) {
                outcome = 0;
                break;
            }
            rounds_here++;
            const int32_t *prev = bfront(S, t - 1);
            int32_t *cur = bfront(S, t);
            RoundArgs RA;
            RA.A = A;
            RA.B = B;
            RA.n = n;
            RA.m = m;
            RA.prev = prev;
            RA.cur = cur;
            RA.off = off;
            RA.lo = lo;
            RA.hi = hi;
            RA.tau = t;
            RA.a = lo;
            RA.b = hi + 1;
            RA.n1 = S.n1;
            RA.open = S.ld;
            RA.err = S.err;
            RA.diag = S.diag;
            RA.tid = tid;
            RA.nt = nt;
            RA.open_c = nullptr;
            RA.ocap = 0;
            RA.defer = nullptr;
            RA.nd = nullptr;
            const RoundCount rc = tile_round<4>(RA);
            slide += rc.slide;
            mism += rc.mism;
            __syncthreads();
            if (*S.err != 0) {
                outcome = 3;
                break;
            }
            const int n1 = *S.n1;
            if (n1 > 0) {
                // one warp per open slide; those still open get the whole CTA
                for (int j = warp; j < n1; j += nw) {
                    const int64_t d = S.ld[j];
                    const int64_t c = start_row(prev, off, d, t, n, m);
                    const int64_t lim = c + min(n - c, m - c - d);
                    bool open;
                    const int64_t l = warp_slide(A, n, B, m, c, d, lim - c, Bg.t2_cap, &open);
                    if (!open && l >= PREFETCH_MIN)
                        prefetch_next(A, n, B, m, c + l, c + l + d);
                    if (lane == 0) {
                        if (!open) {
                            cur[d - off] = (int32_t)(c + l);
                            slide += l;
                            mism += (c + l < lim);
                            S.ld[j] = INT32_MIN; // finished
                        }
                    }
                }
                __syncthreads();
                for (int j = 0; j < n1; j++) {
                    const int64_t d = S.ld[j];
                    if (d == INT32_MIN)
                        continue;
                    const int64_t c = start_row(prev, off, d, t, n, m);
                    const int64_t lim = c + min(n - c, m - c - d);
                    const int64_t row = cta_slide(A, n, B, m, d, c, lim, S.smin);
                    if (tid < 32)
                        prefetch_next(A, n, B, m, row, row + d);
                    if (tid == 0) {
                        cur[d - off] = (int32_t)row;
                        slide += row - c;
                        mism += (row < lim);
                    }
                }
                __syncthreads();
                if (tid == 0)
                    *S.n1 = 0;
            }
            const bool fin = (target >= lo && target <= hi) && cur[target - off] == n;
            __syncthreads();
            if (fin) {
                outcome = 1;
                break;
            }
        }
        // counters
        for (int o = 16; o; o >>= 1) {
            slide += __shfl_down_sync(0xffffffffu, slide, o);
            mism += __shfl_down_sync(0xffffffffu, mism, o);
        }
        if (lane == 0) {
            if (slide)
                atomicAdd(&Pr.slide, slide);
            if (mism)
                atomicAdd(&Pr.mism, mism);
        }
        if (outcome == 3) {
            // a start row outside the grid was recorded, never loaded
            if (tid == 0) {
                Pr.check[0] = (long long)S.diag[2];
                Pr.check[1] = (long long)S.diag[3];
                Pr.check[2] = (long long)S.diag[4];
                Pr.state = 3;
            }
        } else if (outcome == 1) {
            if (tid == 0) {
                Pr.k = t;
                Pr.t = (int32_t)t;
                Pr.state = 1;
            }
        } else {
            // save the last completed round (t - 1) as the resident frontier;
            // its furthest row tells the host how far along the pair is
            const int32_t *src = bfront(S, t - 1);
            int r = 0;
            for (int i = tid; i < Bg.W + 3; i += nt) {
                Pr.front[i] = src[i];
                r = max(r, src[i]);
            }
            atomicMax(S.reach, r);
            __syncthreads();
            if (tid == 0) {
                Pr.t = (int32_t)(t - 1);
                Pr.reach = *S.reach;
                Pr.state = outcome == 2 ? 2 : 0;
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_lv_batch(const BatchArgs &B, int grid, cudaStream_t s, uint64_t budget_ns)
{
    const size_t smem = lv_batch_smem_bytes(B.W);
    cudaError_t e =
        cudaFuncSetAttribute(lv_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    lv_batch_kernel<<<grid, BT, smem, s>>>(B, budget_ns);
    return cudaGetLastError();
}

int lv_batch_threads() { return BT; }

int lv_batch_ctas_per_sm(int W)
{
    const size_t smem = lv_batch_smem_bytes(W);
    if (cudaFuncSetAttribute(lv_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 1;
    int nb = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, lv_batch_kernel, BT, smem) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

} // namespace edg
