// lv_batch.cu -- many independent pairs in one persistent launch.
//
// Each CTA claims pairs from a work queue (atomicAdd on a head index over a
// cost-sorted order) and runs Algorithm 1 (Sec. 3.1) on its pair with the
// frontier in shared memory, one __syncthreads per round.  Slides escalate
// from one thread to one warp to the whole CTA (64 KiB chunks).  A pair
// whose band outgrows W diagonals is parked (state 2) with its frontier
// saved, for the single-pair kernel.  With a time budget (serving), a CTA
// stops a pair when the budget is spent, saves the round-t frontier to the
// pair's resident buffer, and the next launch resumes it.
#include "ed_device.cuh"
#include "lv_kernels.cuh"

namespace edg {

constexpr int BT = 256;      // threads per batch CTA
constexpr int LB = 256;      // open-slide list entries per CTA

struct BSmem {
    int32_t *f[2];
    int32_t *ld, *lc;
    int64_t *lpos, *llim;
    int *n1, *flag, *claim;
    unsigned long long *smin;
};

size_t lv_batch_smem_bytes(int W)
{
    return 16 + 64 + (size_t)LB * (2 * sizeof(int64_t) + 2 * sizeof(int32_t)) +
           2 * sizeof(int32_t) * ((size_t)W + 3);
}

__device__ BSmem bcarve(int W)
{
    extern __shared__ __align__(16) unsigned char bsmem_raw[];
    BSmem S;
    unsigned char *p = bsmem_raw;
    S.smin = reinterpret_cast<unsigned long long *>(p);
    p += 16;
    S.n1 = reinterpret_cast<int *>(p);
    S.flag = S.n1 + 1;
    S.claim = S.n1 + 2;
    p += 64;
    S.lpos = reinterpret_cast<int64_t *>(p);
    p += sizeof(int64_t) * LB;
    S.llim = reinterpret_cast<int64_t *>(p);
    p += sizeof(int64_t) * LB;
    S.ld = reinterpret_cast<int32_t *>(p);
    p += sizeof(int32_t) * LB;
    S.lc = reinterpret_cast<int32_t *>(p);
    p += sizeof(int32_t) * LB;
    S.f[0] = reinterpret_cast<int32_t *>(p);
    p += sizeof(int32_t) * (W + 3);
    S.f[1] = reinterpret_cast<int32_t *>(p);
    return S;
}

// The whole CTA finishes one open slide: A[pos..lim_abs) vs B[pos+d..).
__device__ int64_t cta_slide(const BatchPair &Pr, int64_t d, int64_t pos, int64_t lim_abs,
                             unsigned long long *s_min)
{
    for (int64_t off = 0; pos + off < lim_abs; off += CHUNK_BYTES / 4) {
        const int64_t len = min((int64_t)CHUNK_BYTES / 4, lim_abs - pos - off);
        const int64_t r = cta_scan<1>(Pr.A, Pr.n, Pr.B, Pr.m, pos, pos + d, off, len, s_min);
        if (r >= 0)
            return pos + r;
    }
    return lim_abs;
}

__global__ void __launch_bounds__(BT) lv_batch_kernel(BatchArgs Bg, uint64_t budget_ns)
{
    const BSmem S = bcarve(Bg.W);
    // 0 = no time budget; otherwise this CTA stops claiming and parks its
    // pair once budget_ns have passed since it started
    const uint64_t deadline_ns = budget_ns ? gtimer() + budget_ns : 0;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int H = Bg.W / 2;
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
        }
        __syncthreads();
        const int pi = *S.claim;
        __syncthreads();
        if (pi < 0)
            break;
        BatchPair &Pr = Bg.pairs[pi];
        if (Pr.state != 0) // finished or parked: nothing to do
            continue;
        const int64_t n = Pr.n, m = Pr.m, target = m - n;
        // restore the resident frontier (round t0) or start at round 0
        const int64_t t0 = Pr.t;
        for (int i = tid; i < Bg.W + 3; i += nt) {
            S.f[0][i] = NEG;
            S.f[1][i] = NEG;
        }
        __syncthreads();
        if (t0 >= 0) {
            const int32_t *src = Pr.front;
            int32_t *dst = S.f[t0 & 1];
            for (int i = tid; i < Bg.W + 3; i += nt)
                dst[i] = src[i];
        }
        __syncthreads();
        unsigned long long slide = 0, mism = 0;
        int64_t t = t0 + 1;
        int outcome = 0; // 0 budget spent, 1 done, 2 band too wide
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
            const int32_t *prev = S.f[(t - 1) & 1];
            int32_t *cur = S.f[t & 1];
            for (int64_t d = lo + tid; d <= hi; d += nt) {
                int64_t c;
                if (t == 0) {
                    c = 0;
                } else {
                    const int64_t a = prev[d + H + 1 - 1];
                    const int64_t b = (int64_t)prev[d + H + 1] + 1;
                    const int64_t e = (int64_t)prev[d + H + 1 + 1] + 1;
                    c = max(a, max(b, e));
                    c = min(c, min(n, m - d));
                }
                if (c < 0 || c + d < 0) {
                    // a start row outside the grid: record it, never load it
                    Pr.check[0] = t;
                    Pr.check[1] = d;
                    Pr.check[2] = c;
                    Pr.state = 3;
                    cur[d + H + 1] = NEG;
                    continue;
                }
                const int64_t full = min(n - c, m - c - d);
                bool open;
                const int64_t l = slide_thread(Pr.A, n, Pr.B, m, c, c + d, full, Bg.t1_cap, &open);
                if (!open) {
                    cur[d + H + 1] = (int32_t)(c + l);
                    slide += l;
                    mism += (l < full);
                } else {
                    const int s = atomicAdd(S.n1, 1);
                    if (s < LB) {
                        S.ld[s] = (int32_t)d;
                        S.lc[s] = (int32_t)c;
                        S.lpos[s] = c + l;
                        S.llim[s] = c + full;
                    } else {
                        bool o2;
                        const int64_t l2 =
                            slide_thread(Pr.A, n, Pr.B, m, c, c + d, full, INT64_MAX, &o2);
                        cur[d + H + 1] = (int32_t)(c + l2);
                        slide += l2;
                        mism += (l2 < full);
                    }
                }
            }
            __syncthreads();
            const int n1 = min(*S.n1, LB);
            if (n1 > 0) {
                // one warp per open slide; still-open ones get the whole CTA
                for (int j = warp; j < n1; j += nw) {
                    const int64_t d = S.ld[j], pos = S.lpos[j], lim = S.llim[j];
                    bool open;
                    const int64_t l = slide_warp(Pr.A, n, Pr.B, m, pos, pos + d, 0, lim - pos,
                                                 Bg.t2_cap, &open);
                    if (lane == 0) {
                        if (!open) {
                            S.llim[j] = -(pos + l) - 1; // negative: final row, encoded
                        } else {
                            S.lpos[j] = pos + l;
                        }
                    }
                }
                __syncthreads();
                for (int j = 0; j < n1; j++) {
                    const int64_t ll = S.llim[j];
                    int64_t row;
                    if (ll < 0) {
                        row = -ll - 1;
                    } else {
                        row = cta_slide(Pr, S.ld[j], S.lpos[j], ll, S.smin);
                    }
                    if (tid == 0) {
                        const int64_t d = S.ld[j], c = S.lc[j];
                        cur[d + H + 1] = (int32_t)row;
                        const int64_t full_abs = c + min(n - c, m - c - d);
                        slide += row - c;
                        mism += (row < full_abs);
                    }
                }
                __syncthreads();
                if (tid == 0)
                    *S.n1 = 0;
            }
            const bool fin = ((target >= lo && target <= hi) && cur[target + H + 1] == n) ||
                             *(volatile int32_t *)&Pr.state == 3;
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
            if (slide) atomicAdd(&Pr.slide, slide);
            if (mism) atomicAdd(&Pr.mism, mism);
        }
        __syncthreads();
        const bool failed = *(volatile int32_t *)&Pr.state == 3;
        __syncthreads();
        if (failed) {
            // leave the self-check record for the host
        } else if (outcome == 1) {
            if (tid == 0) {
                Pr.k = t;
                Pr.t = (int32_t)t;
                Pr.state = 1;
            }
        } else {
            // save the last completed round (t - 1) as the resident frontier
            const int32_t *src = S.f[(t - 1) & 1];
            for (int i = tid; i < Bg.W + 3; i += nt)
                Pr.front[i] = src[i];
            if (tid == 0) {
                Pr.t = (int32_t)(t - 1);
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

} // namespace edg
