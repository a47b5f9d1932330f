// ed_device.cuh -- device building blocks shared by the GB300 kernels.
//
// Notation (the paper's diagonal i = x - y, mirrored):
//   cell (x, y) = x bytes of A and y bytes of B consumed; diagonal d = y - x;
//   L_t[d] = furthest row x on diagonal d reachable with t edits.
// LCP(x, y) (Sec. 2) = length of the longest common prefix of A[x..n) and
// B[y..m).  The slides below compute it by direct comparison in 16-byte
// windows (Sec. 5.1 checks a few leading characters before a query; here
// that check is a 16-byte vector compare).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace edg {

// "Minus infinity" for frontier entries: a byte pattern so that a memset
// with 0xC0 initialises a buffer, far enough from 0 that +1 stays negative.
constexpr int32_t NEG = (int32_t)0xC0C0C0C0;

constexpr uint64_t Q61 = (1ull << 61) - 1;


// ---------------------------------------------------------------- timing
__device__ __forceinline__ uint64_t gtimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------- memory ordering
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int32_t ld_cg(const int32_t *p) { return __ldcg(p); }
__device__ __forceinline__ void st_cg(int32_t *p, int32_t v) { __stcg(p, v); }
__device__ __forceinline__ int64_t ld_vol64(const int64_t *p)
{
    return *(const volatile int64_t *)p;
}

// ------------------------------------------------------- string windows
// A 16-byte aligned block is loaded only if it overlaps the string
// [base, base+len): such a block lies in the same page as a valid byte, so
// the load cannot fault whatever the alignment of base.  Bytes outside the
// string are garbage and are always masked by the caller's bound.
__device__ __forceinline__ uint4 ld_blk(const uint8_t *base, int64_t len, uintptr_t blk)
{
    const uintptr_t b = (uintptr_t)base;
    if (blk + 16 > b && blk < b + (uintptr_t)len)
        return __ldg(reinterpret_cast<const uint4 *>(blk));
    return make_uint4(0u, 0u, 0u, 0u);
}

// Branch-free form of ld_blk for len > 0, so that a thread's loads all
// issue before any is used: a block that does not overlap the string is
// replaced by the block holding the string's last byte (always valid).
// Its bytes lie outside the window asked for and are masked by the
// caller's bound like any byte past the string.
__device__ __forceinline__ uint4 ld_blk_nb(const uint8_t *base, int64_t len, uintptr_t blk)
{
    const uintptr_t b = (uintptr_t)base;
    const bool in = blk + 16 > b && blk < b + (uintptr_t)len;
    const uintptr_t safe = (b + (uintptr_t)len - 1) & ~(uintptr_t)15;
    return __ldg(reinterpret_cast<const uint4 *>(in ? blk : safe));
}

// 16 bytes of the 32-byte concatenation lo|hi starting at byte s (0..15).
__device__ __forceinline__ uint4 shift_bytes(uint4 lo, uint4 hi, uint32_t s)
{
    const uint32_t q = s >> 2, r = (s & 3u) * 8u;
    const uint32_t w0 = lo.x, w1 = lo.y, w2 = lo.z, w3 = lo.w;
    const uint32_t w4 = hi.x, w5 = hi.y, w6 = hi.z, w7 = hi.w;
    const uint32_t a0 = q == 0 ? w0 : q == 1 ? w1 : q == 2 ? w2 : w3;
    const uint32_t a1 = q == 0 ? w1 : q == 1 ? w2 : q == 2 ? w3 : w4;
    const uint32_t a2 = q == 0 ? w2 : q == 1 ? w3 : q == 2 ? w4 : w5;
    const uint32_t a3 = q == 0 ? w3 : q == 1 ? w4 : q == 2 ? w5 : w6;
    const uint32_t a4 = q == 0 ? w4 : q == 1 ? w5 : q == 2 ? w6 : w7;
    uint4 o;
    o.x = __funnelshift_r(a0, a1, r);
    o.y = __funnelshift_r(a1, a2, r);
    o.z = __funnelshift_r(a2, a3, r);
    o.w = __funnelshift_r(a3, a4, r);
    return o;
}

// The 16 bytes base[pos .. pos+16) (two aligned loads and a byte shift).
__device__ __forceinline__ uint4 load16(const uint8_t *base, int64_t len, int64_t pos)
{
    const uintptr_t a = (uintptr_t)(base + pos);
    const uintptr_t al = a & ~(uintptr_t)15;
    const uint32_t s = (uint32_t)(a & 15);
    const uint4 lo = ld_blk(base, len, al);
    if (s == 0)
        return lo;
    const uint4 hi = ld_blk(base, len, al + 16);
    return shift_bytes(lo, hi, s);
}

// Index of the first differing byte of two 16-byte windows, 16 if equal.
__device__ __forceinline__ int first_diff16(uint4 a, uint4 b)
{
    const uint64_t d0 = ((uint64_t)(a.y ^ b.y) << 32) | (uint64_t)(a.x ^ b.x);
    const uint64_t d1 = ((uint64_t)(a.w ^ b.w) << 32) | (uint64_t)(a.z ^ b.z);
    if (d0)
        return (__ffsll((long long)d0) - 1) >> 3;
    if (d1)
        return 8 + ((__ffsll((long long)d1) - 1) >> 3);
    return 16;
}

// ------------------------------------------------------- per-thread slide
// The aligned 4-byte words holding A[x] and B[y], shifted so that byte 0 is
// A[x] (resp. B[y]).  Requires x < n and y < m: the words then hold a valid
// byte and cannot fault.  Issued apart from their use so that several
// diagonals' loads are in flight together.
__device__ __forceinline__ void word_load(const uint8_t *A, const uint8_t *B, int64_t x, int64_t y,
                                          uint32_t &wa, uint32_t &wb)
{
    const uintptr_t pa = (uintptr_t)(A + x), pb = (uintptr_t)(B + y);
    wa = __ldg(reinterpret_cast<const uint32_t *>(pa & ~(uintptr_t)3));
    wb = __ldg(reinterpret_cast<const uint32_t *>(pb & ~(uintptr_t)3));
}

// LCP from (x, y) up to `lim` bytes (lim <= min(n-x, m-y)), examining at
// most `cap` bytes, given the words of word_load (unshifted).  Returns the
// matched length l (l == lim: no mismatch before lim); *open is set when the
// first `cap` bytes all matched and lim was not reached (the slide must
// continue elsewhere).  The words decide most slides; then 16-byte windows.
__device__ __forceinline__ int64_t slide_thread_w(const uint8_t *A, int64_t n, const uint8_t *B,
                                                  int64_t m, int64_t x, int64_t y, int64_t lim,
                                                  int64_t cap, uint32_t wa, uint32_t wb, bool *open)
{
    *open = false;
    if (lim <= 0)
        return 0;
    const uint32_t sa = (uint32_t)((uintptr_t)(A + x) & 3), sb = (uint32_t)((uintptr_t)(B + y) & 3);
    wa >>= 8 * sa;
    wb >>= 8 * sb;
    int64_t avail = (int64_t)(4 - max(sa, sb));
    if (avail > lim)
        avail = lim;
    const uint32_t mask = avail >= 4 ? 0xffffffffu : ((1u << (8 * avail)) - 1u);
    const uint32_t dif = (wa ^ wb) & mask;
    if (dif)
        return (__ffs((int)dif) - 1) >> 3;
    int64_t l = avail;
    const int64_t stop = min(lim, cap);
    while (l < stop) {
        const uint4 va = load16(A, n, x + l);
        const uint4 vb = load16(B, m, y + l);
        const int f = first_diff16(va, vb);
        if (f < 16)
            return min(l + f, lim);
        l += 16;
    }
    if (l >= lim)
        return lim;
    *open = true;
    return l;
}

// The word part of slide_thread_w alone: returns the matched length when
// the words decide the slide (a mismatch within them, or lim reached), else
// -1 with *avail = the bytes they showed equal.
__device__ __forceinline__ int64_t word_slide(const uint8_t *A, const uint8_t *B, int64_t x, int64_t y,
                                              int64_t lim, uint32_t wa, uint32_t wb, int64_t *avail)
{
    if (lim <= 0)
        return 0;
    const uint32_t sa = (uint32_t)((uintptr_t)(A + x) & 3), sb = (uint32_t)((uintptr_t)(B + y) & 3);
    wa >>= 8 * sa;
    wb >>= 8 * sb;
    int64_t av = (int64_t)(4 - max(sa, sb));
    if (av > lim)
        av = lim;
    const uint32_t mask = av >= 4 ? 0xffffffffu : ((1u << (8 * av)) - 1u);
    const uint32_t dif = (wa ^ wb) & mask;
    if (dif)
        return (__ffs((int)dif) - 1) >> 3;
    if (av >= lim)
        return lim;
    *avail = av;
    return -1;
}

// The aligned 4-byte word holding A[x] and the one after it, and the same
// for B[y]: at least five bytes from each start row whatever its
// alignment.  The second word is loaded only while it still holds a byte of
// the string (an aligned word holding a valid byte cannot fault); else 0.
__device__ __forceinline__ void word_load2(const uint8_t *A, int64_t n, const uint8_t *B, int64_t m,
                                           int64_t x, int64_t y, uint2 &wa, uint2 &wb)
{
    const uintptr_t pa = (uintptr_t)(A + x) & ~(uintptr_t)3, pb = (uintptr_t)(B + y) & ~(uintptr_t)3;
    wa.x = __ldg(reinterpret_cast<const uint32_t *>(pa));
    wb.x = __ldg(reinterpret_cast<const uint32_t *>(pb));
    wa.y = pa + 4 < (uintptr_t)(A + n) ? __ldg(reinterpret_cast<const uint32_t *>(pa + 4)) : 0u;
    wb.y = pb + 4 < (uintptr_t)(B + m) ? __ldg(reinterpret_cast<const uint32_t *>(pb + 4)) : 0u;
}

// The LCP from (x, y) as far as the words of word_load2 decide it: the
// matched length when a mismatch shows within them or `lim` is reached,
// else -1 (every byte they hold matched; the slide goes on elsewhere).
__device__ __forceinline__ int64_t word_slide2(const uint8_t *A, const uint8_t *B, int64_t x, int64_t y,
                                               int64_t lim, uint2 wa, uint2 wb)
{
    if (lim <= 0)
        return 0;
    const uint32_t sa = (uint32_t)((uintptr_t)(A + x) & 3), sb = (uint32_t)((uintptr_t)(B + y) & 3);
    const uint64_t va = (((uint64_t)wa.y << 32) | wa.x) >> (8 * sa);
    const uint64_t vb = (((uint64_t)wb.y << 32) | wb.x) >> (8 * sb);
    int64_t av = (int64_t)(8 - max(sa, sb));
    if (av > lim)
        av = lim;
    const uint64_t mask = av >= 8 ? ~0ull : ((1ull << (8 * av)) - 1ull);
    const uint64_t dif = (va ^ vb) & mask;
    if (dif)
        return (__ffsll((long long)dif) - 1) >> 3;
    return av >= lim ? lim : -1;
}

// The 16-byte window part of slide_thread_w, from l bytes already equal:
// four windows (64 bytes) per step, their loads in flight together.
static __device__ __noinline__ int64_t slide_more(const uint8_t *A, int64_t n, const uint8_t *B, int64_t m,
                                           int64_t x, int64_t y, int64_t l, int64_t lim, int64_t cap,
                                           bool *open)
{
    *open = false;
    const int64_t stop = min(lim, cap);
    while (l < stop) {
        uint4 va[4], vb[4];
#pragma unroll
        for (int w = 0; w < 4; w++) {
            if (l + 16 * w < stop) {
                va[w] = load16(A, n, x + l + 16 * w);
                vb[w] = load16(B, m, y + l + 16 * w);
            }
        }
#pragma unroll
        for (int w = 0; w < 4; w++) {
            if (l + 16 * w < stop) {
                const int f = first_diff16(va[w], vb[w]);
                if (f < 16)
                    return min(l + 16 * w + f, lim);
            }
        }
        l = min(l + 64, stop);
    }
    if (l >= lim)
        return lim;
    *open = true;
    return l;
}

// Asks L2 for len bytes of X from byte x on (clipped to the string), by the
// copy engine: one bulk prefetch, no load issued by the calling thread.  It
// covers whole 16-byte blocks, never past the one that holds the string's
// last byte.
__device__ __forceinline__ void bulk_prefetch_l2(const uint8_t *X, int64_t len_x, int64_t x, int64_t len)
{
    if (x < 0 || x >= len_x || len <= 0)
        return;
    const uintptr_t lo = (uintptr_t)(X + x) & ~(uintptr_t)15;
    const uintptr_t end = ((uintptr_t)(X + len_x) + 15) & ~(uintptr_t)15;
    const uintptr_t hi = min((((uintptr_t)(X + x) + (uintptr_t)len) + 15) & ~(uintptr_t)15, end);
    uint64_t g;
    asm("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(lo));
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(g), "r"((uint32_t)(hi - lo)) : "memory");
}

// Slides at least this long are followed by a prefetch of what follows
// them (shorter ones are chance matches off the alignment path).
constexpr int64_t PREFETCH_MIN = 256;

// Asks L2 for the 4 KiB of each string that follow rows x (of A) and y (of
// B), one 128-byte line per lane of the calling warp: a diagonal that just
// ended a long slide starts its next round there.  Only addresses inside
// the strings are touched; a line never crosses a page.
__device__ __forceinline__ void prefetch_next(const uint8_t *A, int64_t n, const uint8_t *B, int64_t m,
                                              int64_t x, int64_t y)
{
    const int64_t o = (int64_t)(threadIdx.x & 31) * 128;
    if (x + o < n)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(A + x + o));
    if (y + o < m)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(B + y + o));
}

__device__ __forceinline__ int64_t slide_thread(const uint8_t *A, int64_t n, const uint8_t *B,
                                                int64_t m, int64_t x, int64_t y, int64_t lim,
                                                int64_t cap, bool *open)
{
    if (lim <= 0) {
        *open = false;
        return 0;
    }
    uint32_t wa, wb;
    word_load(A, B, x, y, wa, wb);
    return slide_thread_w(A, n, B, m, x, y, lim, cap, wa, wb, open);
}

// ------------------------------------------------------- per-warp slide
// All 32 lanes of the calling warp compare 512 consecutive bytes per step
// (16 per lane), UNROLL steps in flight; __ballot_sync + __ffs pick the
// first lane holding a mismatch.  Starts at offset l0 (bytes already known
// equal), up to `lim` bytes from (x, y), examining at most `cap` further
// bytes.  Must be called by a whole warp with identical arguments.  Returns
// the matched length from (x, y); *open as for slide_thread.
template <int UNROLL = 4>
__device__ __forceinline__ int64_t slide_warp(const uint8_t *A, int64_t n, const uint8_t *B,
                                              int64_t m, int64_t x, int64_t y, int64_t l0,
                                              int64_t lim, int64_t cap, bool *open)
{
    const int lane = threadIdx.x & 31;
    const int64_t stop = min(lim, l0 + cap);
    *open = false;
    for (int64_t base = l0; base < stop; base += 512 * UNROLL) {
        // every aligned block first (windows past lim read a valid block and
        // are ignored below), then the compares
        uint4 alo[UNROLL], ahi[UNROLL], blo[UNROLL], bhi[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; u++) {
            const int64_t o = min(base + u * 512 + lane * 16, lim - 1);
            const uintptr_t pa = ((uintptr_t)(A + x + o)) & ~(uintptr_t)15;
            const uintptr_t pb = ((uintptr_t)(B + y + o)) & ~(uintptr_t)15;
            alo[u] = ld_blk_nb(A, n, pa);
            ahi[u] = ld_blk_nb(A, n, pa + 16);
            blo[u] = ld_blk_nb(B, m, pb);
            bhi[u] = ld_blk_nb(B, m, pb + 16);
        }
#pragma unroll
        for (int u = 0; u < UNROLL; u++) {
            const int64_t o = base + u * 512 + lane * 16;
            int64_t cand = -1;
            if (o < lim) {
                const uint32_t sa = (uint32_t)((uintptr_t)(A + x + o) & 15), sb = (uint32_t)((uintptr_t)(B + y + o) & 15);
                const int f = first_diff16(shift_bytes(alo[u], ahi[u], sa), shift_bytes(blo[u], bhi[u], sb));
                if (f < 16 || o + 16 >= lim)
                    cand = min(o + f, lim);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, cand >= 0);
            if (bal) {
                const int src = __ffs((int)bal) - 1;
                return __shfl_sync(0xffffffffu, cand, src);
            }
        }
    }
    if (stop >= lim)
        return lim;
    *open = true;
    return stop;
}

// ------------------------------------------------------- CTA chunk scan
// The calling CTA compares A[x+off .. x+off+len) with B[y+off ..) and
// returns the first mismatching offset (>= off), or -1 if all equal.
// Every thread must call it; s_min is a shared int64 scratch word.
template <int UNROLL = 4>
__device__ __forceinline__ int64_t cta_scan(const uint8_t *A, int64_t n, const uint8_t *B,
                                            int64_t m, int64_t x, int64_t y, int64_t off,
                                            int64_t len, unsigned long long *s_min)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0)
        *s_min = ~0ull;
    __syncthreads();
    int64_t best = -1;
    for (int64_t base = 0; base < len; base += (int64_t)nt * 16 * UNROLL) {
        // every aligned block first (windows past len read a valid block and
        // are ignored below), then the compares
        uint4 alo[UNROLL], ahi[UNROLL], blo[UNROLL], bhi[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; u++) {
            const int64_t o = min(base + ((int64_t)u * nt + tid) * 16, len - 1);
            const uintptr_t pa = ((uintptr_t)(A + x + off + o)) & ~(uintptr_t)15;
            const uintptr_t pb = ((uintptr_t)(B + y + off + o)) & ~(uintptr_t)15;
            alo[u] = ld_blk_nb(A, n, pa);
            ahi[u] = ld_blk_nb(A, n, pa + 16);
            blo[u] = ld_blk_nb(B, m, pb);
            bhi[u] = ld_blk_nb(B, m, pb + 16);
        }
#pragma unroll
        for (int u = 0; u < UNROLL; u++) {
            const int64_t o = base + ((int64_t)u * nt + tid) * 16;
            if (best < 0 && o < len) {
                const uint32_t sa = (uint32_t)((uintptr_t)(A + x + off + o) & 15),
                               sb = (uint32_t)((uintptr_t)(B + y + off + o) & 15);
                const int f = first_diff16(shift_bytes(alo[u], ahi[u], sa), shift_bytes(blo[u], bhi[u], sb));
                if (f < 16 && o + f < len)
                    best = off + o + f;
            }
        }
        // the whole CTA stops after the first step with a mismatch
        if (__syncthreads_or(best >= 0))
            break;
    }
    if (best >= 0)
        atomicMin(s_min, (unsigned long long)best);
    __syncthreads();
    const unsigned long long r = *s_min;
    __syncthreads();
    return r == ~0ull ? -1 : (int64_t)r;
}

// ------------------------------------------------------- CTA sweep
// An aligned 16-byte block loaded past the L1 (the bytes of a long slide are
// read once; the L1 keeps the lines the rounds' start rows reuse).
__device__ __forceinline__ uint4 ld_stream16(uintptr_t p)
{
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
    return v;
}

// The aligned block at blk if it overlaps [base, base + len) (len > 0),
// else the block holding the string's first or last byte: a block that
// overlaps the string lies in the same page as a valid byte and cannot
// fault.  Bytes outside the window a caller asked for are masked by it.
__device__ __forceinline__ uintptr_t safe_blk(uintptr_t base, int64_t len, uintptr_t blk)
{
    const uintptr_t first = base & ~(uintptr_t)15, last = (base + (uintptr_t)len - 1) & ~(uintptr_t)15;
    return blk < first ? first : (blk > last ? last : blk);
}

// The calling CTA compares A[x0 .. x0+len) with B[y0 .. y0+len) for
// len <= blockDim.x * 16 * U (32 KiB per string at 256 threads, U = 8) and
// returns the first mismatching offset, or -1 if all are equal.  Needs
// x0 + len <= n and y0 + len <= m.  Every load is issued before the first
// compare: one memory round trip per call.
//
// The A side is read in aligned 16-byte blocks: block j starts sa bytes
// before A[x0] (sa = the misalignment of A + x0) and holds offsets
// 16j - sa .. 16j - sa + 15.  The B bytes paired with them are bytes
// qb .. qb + 15 of the 32-byte run made of B's aligned blocks j and j + 1
// (counted from the block holding B[y0 - sa]); block j + 1 belongs to the
// next lane, so it comes by shuffle (lane 31 takes the next row of blocks,
// or one extra load after the last).  Warp w reads 32 * U consecutive
// blocks.  Every thread must call it; s_min is a shared 64-bit scratch word.
template <int U>
__device__ __forceinline__ int64_t sweep_scan(const uint8_t *A, int64_t n, const uint8_t *B, int64_t m, int64_t x0,
                                              int64_t y0, int64_t len, unsigned long long *s_min)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0)
        *s_min = ~0ull;
    const uintptr_t pa = (uintptr_t)(A + x0);
    const uint32_t sa = (uint32_t)(pa & 15);
    const uintptr_t a0 = pa - sa;
    const uintptr_t pbs = (uintptr_t)(B + y0) - sa; // B address paired with a0
    const uint32_t qb = (uint32_t)(pbs & 15);
    const uintptr_t b0 = pbs - qb;
    const uintptr_t Ab = (uintptr_t)A, Bb = (uintptr_t)B;
    const int64_t jw = (int64_t)warp * 32 * U; // this warp's first block
    uint4 va[U], vb[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int64_t j = jw + u * 32 + lane;
        va[u] = ld_stream16(safe_blk(Ab, n, a0 + 16 * j));
        vb[u] = ld_stream16(safe_blk(Bb, m, b0 + 16 * j));
    }
    const uint4 vx = ld_stream16(safe_blk(Bb, m, b0 + 16 * (jw + 32 * U)));
    int64_t best = -1;
#pragma unroll
    for (int u = 0; u < U; u++) {
        // the B block after this lane's: the next lane's, or for lane 31 the
        // first of the next row (the extra block after the last row)
        const uint4 nb = u + 1 < U ? vb[u + 1] : vx;
        uint4 nx;
        nx.x = __shfl_down_sync(0xffffffffu, vb[u].x, 1);
        nx.y = __shfl_down_sync(0xffffffffu, vb[u].y, 1);
        nx.z = __shfl_down_sync(0xffffffffu, vb[u].z, 1);
        nx.w = __shfl_down_sync(0xffffffffu, vb[u].w, 1);
        const uint4 f0 = make_uint4(__shfl_sync(0xffffffffu, nb.x, 0), __shfl_sync(0xffffffffu, nb.y, 0),
                                    __shfl_sync(0xffffffffu, nb.z, 0), __shfl_sync(0xffffffffu, nb.w, 0));
        if (lane == 31)
            nx = f0;
        const uint4 bs = shift_bytes(vb[u], nx, qb);
        const int64_t j = jw + u * 32 + lane;
        // valid bytes of this block: offsets 16j - sa + i in [0, len)
        const int64_t o0 = 16 * j - (int64_t)sa;
        const int lo = o0 < 0 ? (int)-o0 : 0;
        const int64_t hi64 = len - o0;
        const int hi = hi64 >= 16 ? 16 : (hi64 <= 0 ? 0 : (int)hi64);
        if (best < 0 && lo < hi) {
            uint64_t d0 = ((uint64_t)(va[u].y ^ bs.y) << 32) | (uint64_t)(va[u].x ^ bs.x);
            uint64_t d1 = ((uint64_t)(va[u].w ^ bs.w) << 32) | (uint64_t)(va[u].z ^ bs.z);
            // keep bytes lo .. hi-1
            const uint64_t k0lo = lo >= 8 ? 0ull : (~0ull << (8 * lo));
            const uint64_t k1lo = lo <= 8 ? ~0ull : (~0ull << (8 * (lo - 8)));
            const uint64_t k0hi = hi >= 8 ? ~0ull : ((1ull << (8 * hi)) - 1ull);
            const uint64_t k1hi = hi <= 8 ? 0ull : (hi >= 16 ? ~0ull : ((1ull << (8 * (hi - 8))) - 1ull));
            d0 &= k0lo & k0hi;
            d1 &= k1lo & k1hi;
            if (d0)
                best = o0 + ((__ffsll((long long)d0) - 1) >> 3);
            else if (d1)
                best = o0 + 8 + ((__ffsll((long long)d1) - 1) >> 3);
        }
    }
    if (__syncthreads_or(best >= 0)) {
        if (best >= 0)
            atomicMin(s_min, (unsigned long long)best);
        __syncthreads();
        const int64_t r = (int64_t)*s_min;
        __syncthreads(); // read by all before the next call resets it
        return r;
    }
    return -1;
}

// ------------------------------------------------------- bulk copies
// Shared-memory address of a generic pointer into shared memory.
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Orders an mbarrier's initialisation before its use by the bulk-copy
// (async) proxy.
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// The calling thread's arrival on bar, announcing `bytes` of bulk copies
// that will complete on it.
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// A bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global memory into this CTA's shared memory, completing on bar.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    uint64_t g;
    asm("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(src));
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(g), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// True once bar's phase `parity` has completed.
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// Orders this thread's earlier shared-memory reads before later bulk copies
// (async proxy) into the same bytes.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Shared-memory staging of one chunk for stage_scan: the A side (chunk +
// 16 bytes), the B side (chunk + 32 bytes), the mbarrier the copies
// complete on, and the phase to wait for next.
struct Stage {
    unsigned char *a, *b;
    uint64_t *bar;
    uint32_t *phase;
};
template <int CH>
constexpr size_t stage_bytes()
{
    return (size_t)CH + 16 + (size_t)CH + 32 + 16 + 16;
}

// A staged chunk: A[x0 .. x0+len) against B[y0 .. y0+len), len <= CH, with
// x0 + len <= n and y0 + len <= m.  The A side is held in aligned 16-byte
// blocks, block j starting sa bytes before A[x0] (offsets 16j - sa ..
// 16j - sa + 15); the B bytes paired with block j are bytes qb .. qb + 15 of
// the stage's B blocks j and j + 1.
struct StagedChunk {
    uint32_t sa, qb;
    int64_t nblk, len;
};

// Thread 0: copies the chunk's aligned blocks into stage T by two bulk
// copies completing on T's mbarrier (clipped to the blocks that overlap
// each string: such a block lies in the same page as a valid byte).  Bytes
// copied from outside a string, or not copied at all, pair only with
// offsets outside [0, len).
__device__ __forceinline__ StagedChunk stage_issue(const Stage T, const uint8_t *A, int64_t n, const uint8_t *B,
                                                   int64_t m, int64_t x0, int64_t y0, int64_t len, bool issue)
{
    StagedChunk K;
    const uintptr_t pa = (uintptr_t)(A + x0);
    K.sa = (uint32_t)(pa & 15);
    const uintptr_t a0 = pa - K.sa;
    const uintptr_t pbs = (uintptr_t)(B + y0) - K.sa; // B address paired with a0
    K.qb = (uint32_t)(pbs & 15);
    const uintptr_t b0 = pbs - K.qb;
    K.nblk = (K.sa + len + 15) >> 4; // A blocks holding offsets [0, len)
    K.len = len;
    if (issue) {
        const uintptr_t aend = (((uintptr_t)A + (uintptr_t)n - 1) & ~(uintptr_t)15) + 16;
        const uint32_t la = (uint32_t)(min(a0 + 16 * (uintptr_t)K.nblk, aend) - a0);
        const uintptr_t bfirst = (uintptr_t)B & ~(uintptr_t)15;
        const uintptr_t bend = (((uintptr_t)B + (uintptr_t)m - 1) & ~(uintptr_t)15) + 16;
        const uintptr_t bs = max(b0, bfirst);
        const uintptr_t be = min(b0 + 16 * (uintptr_t)(K.nblk + 1), bend);
        const uint32_t lb = (uint32_t)(be - bs);
        mbar_arrive_tx(T.bar, la + lb);
        bulk_g2s(T.a, (const void *)a0, la, T.bar);
        bulk_g2s(T.b + (bs - b0), (const void *)bs, lb, T.bar);
    }
    return K;
}

// Every thread: waits for stage T's copies (phase *T.phase), bounded by
// spin_ns.  On expiry *err is set, thread 0 gives the copies one more
// bounded wait, the phase is passed and false is returned (to every
// thread).
__device__ __forceinline__ bool stage_wait(const Stage T, uint64_t spin_ns, uint32_t *err)
{
    const uint32_t parity = *T.phase;
    bool ok = mbar_test(T.bar, parity);
    if (!ok) {
        const uint64_t t0 = gtimer();
        while (!(ok = mbar_test(T.bar, parity))) {
            if (gtimer() - t0 > spin_ns)
                break;
        }
    }
    if (__syncthreads_and(ok))
        return true;
    if (threadIdx.x == 0) {
        atomicCAS(err, 0u, 4u);
        const uint64_t t1 = gtimer();
        while (!mbar_test(T.bar, parity) && gtimer() - t1 < spin_ns) {
        }
        *T.phase = parity ^ 1u;
    }
    __syncthreads();
    return false;
}

// Every thread, after stage_wait: the first mismatching offset of the
// staged chunk, or -1.  Each thread compares its 16-byte blocks of A with
// the B bytes paired with them (two aligned 16-byte reads and a byte shift).
// The stage is released (phase passed, reads ordered before later bulk
// copies into it) before the result is combined.  s_min: a shared 64-bit
// scratch word.
__device__ __forceinline__ int64_t stage_compare(const Stage T, const StagedChunk K, unsigned long long *s_min)
{
    const int tid = threadIdx.x;
    int64_t best = -1;
    for (int64_t j = tid; j < K.nblk && best < 0; j += blockDim.x) {
        const uint4 va = *reinterpret_cast<const uint4 *>(T.a + 16 * j);
        const uint4 lo = *reinterpret_cast<const uint4 *>(T.b + 16 * j);
        const uint4 hi = *reinterpret_cast<const uint4 *>(T.b + 16 * j + 16);
        const uint4 bs = shift_bytes(lo, hi, K.qb);
        const int64_t o0 = 16 * j - (int64_t)K.sa;
        const int lo_i = o0 < 0 ? (int)-o0 : 0;
        const int64_t hi64 = K.len - o0;
        const int hi_i = hi64 >= 16 ? 16 : (hi64 <= 0 ? 0 : (int)hi64);
        if (lo_i < hi_i) {
            uint64_t d0 = ((uint64_t)(va.y ^ bs.y) << 32) | (uint64_t)(va.x ^ bs.x);
            uint64_t d1 = ((uint64_t)(va.w ^ bs.w) << 32) | (uint64_t)(va.z ^ bs.z);
            const uint64_t k0lo = lo_i >= 8 ? 0ull : (~0ull << (8 * lo_i));
            const uint64_t k1lo = lo_i <= 8 ? ~0ull : (~0ull << (8 * (lo_i - 8)));
            const uint64_t k0hi = hi_i >= 8 ? ~0ull : ((1ull << (8 * hi_i)) - 1ull);
            const uint64_t k1hi = hi_i <= 8 ? 0ull : (hi_i >= 16 ? ~0ull : ((1ull << (8 * (hi_i - 8))) - 1ull));
            d0 &= k0lo & k0hi;
            d1 &= k1lo & k1hi;
            if (d0)
                best = o0 + ((__ffsll((long long)d0) - 1) >> 3);
            else if (d1)
                best = o0 + 8 + ((__ffsll((long long)d1) - 1) >> 3);
        }
    }
    fence_proxy_async_smem();
    if (tid == 0)
        *s_min = ~0ull;
    const int any = __syncthreads_or(best >= 0);
    if (tid == 0)
        *T.phase ^= 1u;
    if (any) {
        if (best >= 0)
            atomicMin(s_min, (unsigned long long)best);
        __syncthreads();
        const int64_t r = (int64_t)*s_min;
        __syncthreads(); // read by all before the next use resets it
        return r;
    }
    __syncthreads(); // the phase update is seen by all before the next use
    return -1;
}

// One chunk through one stage: issue, wait, compare.  Whole CTA.  Returns
// the first mismatching offset, -1 if none, or -2 when the wait gave up
// (*err set).
template <int CH>
__device__ __noinline__ int64_t stage_scan(const Stage T, const uint8_t *A, int64_t n, const uint8_t *B, int64_t m,
                                           int64_t x0, int64_t y0, int64_t len, unsigned long long *s_min,
                                           uint64_t spin_ns, uint32_t *err)
{
    const StagedChunk K = stage_issue(T, A, n, B, m, x0, y0, len, threadIdx.x == 0);
    if (!stage_wait(T, spin_ns, err))
        return -2;
    return stage_compare(T, K, s_min);
}

// A[x0 .. x0+lim) against B[y0 ..) chunk by chunk through two stages, the
// next chunk's copies in flight while the current one is compared.  Whole
// CTA.  Returns the first mismatching offset, lim if none, or -2 when a
// wait gave up (*err set).  Before returning it waits for the copies still
// in flight, so that both stages are idle.
template <int CH>
__device__ __noinline__ int64_t stream_scan(const Stage T0, const Stage T1, const uint8_t *A, int64_t n,
                                            const uint8_t *B, int64_t m, int64_t x0, int64_t y0, int64_t lim,
                                            unsigned long long *s_min, uint64_t spin_ns, uint32_t *err)
{
    const bool lead = threadIdx.x == 0;
    const int64_t nch = (lim + CH - 1) / CH;
    StagedChunk K0 = stage_issue(T0, A, n, B, m, x0, y0, min((int64_t)CH, lim), lead);
    StagedChunk K1{};
    if (nch > 1)
        K1 = stage_issue(T1, A, n, B, m, x0 + CH, y0 + CH, min((int64_t)CH, lim - CH), lead);
    for (int64_t c = 0; c < nch; c++) {
        const Stage T = (c & 1) ? T1 : T0;
        const StagedChunk K = (c & 1) ? K1 : K0;
        if (!stage_wait(T, spin_ns, err))
            return -2;
        const int64_t r = stage_compare(T, K, s_min);
        if (r >= 0) {
            // the other stage may still be receiving chunk c + 1
            if (c + 1 < nch && !stage_wait((c & 1) ? T0 : T1, spin_ns, err))
                return -2;
            if (c + 1 < nch && lead)
                *((c & 1) ? T0 : T1).phase ^= 1u;
            __syncthreads();
            return c * CH + r;
        }
        // this stage is free again: chunk c + 2 goes into it
        if (c + 2 < nch) {
            const StagedChunk Kn = stage_issue(T, A, n, B, m, x0 + (c + 2) * CH, y0 + (c + 2) * CH,
                                               min((int64_t)CH, lim - (c + 2) * CH), lead);
            if (c & 1)
                K1 = Kn;
            else
                K0 = Kn;
        }
    }
    return lim;
}

// ------------------------------------------------------- mod 2^61 - 1
// a * b mod q for a, b < q: the 122-bit product hi:lo splits as
// (hi << 3 | lo >> 61) * 2^61 + (lo & q), and 2^61 = 1 (mod q).
__device__ __forceinline__ uint64_t mulmod61(uint64_t a, uint64_t b)
{
    const uint64_t lo = a * b;
    const uint64_t hi = __umul64hi(a, b);
    uint64_t r = (lo & Q61) + ((hi << 3) | (lo >> 61));
    r = (r & Q61) + (r >> 61);
    return r >= Q61 ? r - Q61 : r;
}
__device__ __forceinline__ uint64_t addmod61(uint64_t a, uint64_t b)
{
    const uint64_t r = a + b;
    return r >= Q61 ? r - Q61 : r;
}
__device__ __forceinline__ uint64_t submod61(uint64_t a, uint64_t b)
{
    return a >= b ? a - b : a + Q61 - b;
}

} // namespace edg
