// hash.cu -- the prefix-hash table of Sec. 3.2 built by one single-pass
// scan on the device.
//
//   T[i] = h(X[0..i)) = sum_{j<i} (X[j] + 1) * p^(i-1-j)   mod q = 2^61 - 1
//
// Prefix hashes compose by the concatenation rule of Sec. 2,
//   (h1, P1) (+) (h2, P2) = (h1 * P2 + h2, P1 * P2),  P = p^length,
// which is associative, so T is an inclusive scan of per-character pairs
// (X[j] + 1, p).  Each CTA owns a tile of TILE_CHARS characters: a thread
// folds 16 characters with Horner's rule, the CTA scans the 256 thread pairs
// in shared memory, and tiles chain through a decoupled look-back on tile
// descriptors (aggregate first, inclusive prefix when known), with tile ids
// handed out in launch order by an atomic counter.  Reads 1 byte and writes
// 8 bytes per character; with an output stride b > 1 it writes only the
// prefixes of whole blocks, T[j] = h(X[0..jb)), the blocked table of
// Sec. 3.3 (Alg. 2), 8/b bytes per character.
#include <cstddef>

#include "ed_device.cuh"
#include "lv_kernels.cuh"

namespace edg {

constexpr int HT = 256;                 // threads per scan CTA
constexpr int HITEMS = 16;              // characters per thread
constexpr int TILE_CHARS = HT * HITEMS; // 4096

struct TileDesc {
    unsigned long long agg_h, agg_p; // the tile's own pair
    unsigned long long inc_h, inc_p; // pair of X[0 .. tile end)
    uint32_t flag;                   // 0 none, 1 aggregate, 2 inclusive
    uint32_t pad[3];
};

struct ScanState {
    uint32_t next_tile;
    uint32_t error;
    uint32_t pad[14];
    // TileDesc tiles[] follows (64-byte header)
};

size_t prefix_hash_state_bytes(int64_t len)
{
    const int64_t tiles = (len + TILE_CHARS - 1) / TILE_CHARS + 1;
    return 64 + sizeof(TileDesc) * (size_t)tiles;
}

struct HPair {
    uint64_t h, p;
};
__device__ __forceinline__ HPair hcat(HPair a, HPair b)
{
    return {addmod61(mulmod61(a.h, b.p), b.h), mulmod61(a.p, b.p)};
}

__global__ void __launch_bounds__(HT) prefix_hash_kernel(const uint8_t *X, int64_t len, uint64_t base,
                                                         uint64_t *T, int64_t stride,
                                                         ScanState *st, uint64_t spin_ns)
{
    __shared__ HPair s_pair[HT];
    __shared__ HPair s_prefix;
    __shared__ uint32_t s_tile;
    TileDesc *tiles = reinterpret_cast<TileDesc *>(reinterpret_cast<unsigned char *>(st) + 64);
    const int tid = threadIdx.x;
    if (tid == 0)
        s_tile = atomicAdd(&st->next_tile, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t t0 = tile * TILE_CHARS;
    if (t0 >= len && !(len == 0 && tile == 0))
        return;
    // 1. this thread's 16 characters, folded with Horner's rule
    const int64_t s0 = t0 + (int64_t)tid * HITEMS;
    uint8_t c[HITEMS];
    int cnt = 0;
    if (s0 + HITEMS <= len && ((((uintptr_t)(X + s0)) & 15) == 0)) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(X + s0));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < HITEMS; i++)
            c[i] = (uint8_t)(w[i >> 2] >> (8 * (i & 3)));
        cnt = HITEMS;
    } else {
#pragma unroll
        for (int i = 0; i < HITEMS; i++) {
            const int64_t j = s0 + i;
            c[i] = j < len ? __ldg(X + j) : 0;
        }
        cnt = (int)max((int64_t)0, min((int64_t)HITEMS, len - s0));
    }
    HPair mine = {0, 1};
    for (int i = 0; i < cnt; i++) {
        mine.h = addmod61(mulmod61(mine.h, base), (uint64_t)c[i] + 1);
        mine.p = mulmod61(mine.p, base);
    }
    // 2. inclusive scan of the thread pairs across the CTA (Hillis-Steele)
    s_pair[tid] = mine;
    __syncthreads();
    for (int off = 1; off < HT; off <<= 1) {
        HPair v = s_pair[tid];
        if (tid >= off)
            v = hcat(s_pair[tid - off], v);
        __syncthreads();
        s_pair[tid] = v;
        __syncthreads();
    }
    const HPair tile_agg = s_pair[HT - 1];
    // 3. decoupled look-back for the prefix of everything before this tile
    if (tid == 0) {
        TileDesc &me = tiles[tile];
        HPair prefix = {0, 1};
        if (tile == 0) {
            __stcg(&me.inc_h, tile_agg.h);
            __stcg(&me.inc_p, tile_agg.p);
            __threadfence();
            st_release(&me.flag, 2u);
        } else {
            __stcg(&me.agg_h, tile_agg.h);
            __stcg(&me.agg_p, tile_agg.p);
            __threadfence();
            st_release(&me.flag, 1u);
            HPair run = {0, 1}; // pair of tiles (j, tile) exclusive, built right to left
            int64_t j = tile - 1;
            const uint64_t tstart = gtimer();
            for (;;) {
                uint32_t f;
                while ((f = ld_acquire(&tiles[j].flag)) == 0) {
                    if (gtimer() - tstart > spin_ns) {
                        atomicCAS(&st->error, 0u, ST_TIMEOUT);
                        break;
                    }
                }
                if (f == 0) {
                    prefix = {0, 1};
                    break;
                }
                if (f == 2) {
                    const HPair inc = {__ldcg(&tiles[j].inc_h), __ldcg(&tiles[j].inc_p)};
                    prefix = hcat(inc, run);
                    break;
                }
                const HPair agg = {__ldcg(&tiles[j].agg_h), __ldcg(&tiles[j].agg_p)};
                run = hcat(agg, run);
                j--;
            }
            const HPair inc = hcat(prefix, tile_agg);
            __stcg(&me.inc_h, inc.h);
            __stcg(&me.inc_p, inc.p);
            __threadfence();
            st_release(&me.flag, 2u);
        }
        s_prefix = prefix;
    }
    __syncthreads();
    // 4. the exclusive prefix of this thread's segment, then T for each char
    HPair excl = s_prefix;
    if (tid > 0)
        excl = hcat(excl, s_pair[tid - 1]);
    uint64_t h = excl.h;
    if (tile == 0 && tid == 0)
        T[0] = 0;
    if (stride == 1) {
        for (int i = 0; i < cnt; i++) {
            h = addmod61(mulmod61(h, base), (uint64_t)c[i] + 1);
            T[s0 + i + 1] = h;
        }
    } else {
        // only the prefixes that end a whole block
        int64_t next = (s0 / stride + 1) * stride; // first block end after s0
        for (int i = 0; i < cnt; i++) {
            h = addmod61(mulmod61(h, base), (uint64_t)c[i] + 1);
            if (s0 + i + 1 == next) {
                T[next / stride] = h;
                next += stride;
            }
        }
    }

}

uint32_t prefix_hash_status(const void *scan_state, cudaStream_t s, cudaError_t *e)
{
    // the scan's status word (ST_TIMEOUT when a look-back wait gave up and
    // the table after that tile is wrong), copied to the host stack
    uint32_t st = 0;
    *e = cudaMemcpyAsync(&st, static_cast<const unsigned char *>(scan_state) + offsetof(ScanState, error),
                         sizeof(st), cudaMemcpyDeviceToHost, s);
    if (*e == cudaSuccess)
        *e = cudaStreamSynchronize(s);
    return st;
}

cudaError_t launch_prefix_hash(const uint8_t *X, int64_t len, uint64_t base, uint64_t *T, int64_t stride,
                               void *scan_state, size_t scan_state_bytes, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(scan_state, 0, scan_state_bytes, s);
    if (e != cudaSuccess)
        return e;
    const int64_t tiles = len == 0 ? 1 : (len + TILE_CHARS - 1) / TILE_CHARS;
    prefix_hash_kernel<<<(unsigned)tiles, HT, 0, s>>>(X, len, base, T, stride < 1 ? 1 : stride,
                                                      reinterpret_cast<ScanState *>(scan_state),
                                                      2000000000ull);
    return cudaGetLastError();
}

} // namespace edg

// ---------------------------------------------------------------------------
// Allocation-free prefix hash (see ed_prefix_hash_noalloc in include/ed.h).
//
// The scan's look-back descriptors live in this file-scope device array
// instead of memory the caller or a context allocates.  Every GPU that loads
// the library holds it until the process exits.  Host code only ever uses
// the array's device address, obtained once per device with
// cudaGetSymbolAddress (the name itself is a host-side stand-in).
#include <mutex>

#include "../../include/ed.h"

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 1u << 20; // 1 MiB
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scan[NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void *g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

} // namespace

extern "C" int ed_prefix_hash_noalloc(const uint8_t *X, size_t len, uint64_t base, uint64_t *T,
                                      void *stream)
{
    if (!T || (len && !X) || base < 2 || base >= ((1ull << 61) - 1))
        return ED_EINVAL;
    const size_t need = edg::prefix_hash_state_bytes((int64_t)len);
    if (len > (size_t)INT64_MAX || need > NOALLOC_SCRATCH_BYTES)
        return ED_EINVAL; // beyond the fixed scratch: at most ED_NOALLOC_MAX_LEN bytes
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return ED_ECUDA;
    void *scratch = nullptr;
    {
        // first call on this device: look up the array's device address
        std::lock_guard<std::mutex> g(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scan) != cudaSuccess || !p) {
                cudaGetLastError();
                return ED_ECUDA;
            }
            g_noalloc_addr[dev] = p;
        }
        scratch = g_noalloc_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the look-back descriptors must start at zero: cleared on every call
    if (edg::launch_prefix_hash(X, (int64_t)len, base, T, 1, scratch, need, s) != cudaSuccess)
        return ED_ECUDA;
    cudaError_t e = cudaSuccess;
    const uint32_t st = edg::prefix_hash_status(scratch, s, &e);
    if (e != cudaSuccess)
        return ED_ECUDA;
    return st == 0 ? ED_OK : (st == edg::ST_TIMEOUT ? ED_ETIMEOUT : ED_ECUDA);
}
