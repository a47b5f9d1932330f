// ed_api.cu -- host runtime and C ABI of libedgb300 (declared in include/ed.h).
//
// The context owns: one CUDA stream, a pool of device buffers grown on demand
// inside the memory budget, a pinned result block, and (when serving is
// used) a continuous-batching engine thread with a device arena.  Every
// compute step runs in the kernels of lv_tiles.cu, lv_batch.cu and hash.cu;
// this file only validates, plans, allocates and launches.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <dlfcn.h>
#include <fstream>
#include <sstream>
#include <map>
#include <memory>
#include <new>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ed.h"
#include "lv_kernels.cuh"

using namespace edg;

namespace {

constexpr int64_t MAX_LEN = (1ll << 31) - 64;
constexpr uint64_t Q61H = (1ull << 61) - 1;
constexpr int BATCH_W = 4096; // band capacity of one batch CTA
constexpr int START_TILE = 2048; // diagonals per CTA a single pair starts with

// host mod 2^61-1 (exact 128-bit product), for the hash base powers
uint64_t hmul(uint64_t a, uint64_t b)
{
    const unsigned __int128 p = (unsigned __int128)a * b;
    uint64_t r = (uint64_t)(p & Q61H) + (uint64_t)(p >> 61);
    r = (r & Q61H) + (r >> 61);
    return r >= Q61H ? r - Q61H : r;
}

uint64_t splitmix(uint64_t x)
{
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// First-fit arena over one device allocation (serving strings and frontiers).
struct Arena {
    char *base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_; // offset -> length
    std::mutex mu;
    void init(char *b, size_t s)
    {
        base = b;
        size = s;
        free_.clear();
        free_[0] = s;
    }
    char *alloc(size_t n)
    {
        n = (n + 255) & ~(size_t)255;
        std::lock_guard<std::mutex> g(mu);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > n)
                    free_[off + n] = len - n;
                return base + off;
            }
        }
        return nullptr;
    }
    void release(char *p, size_t n)
    {
        if (!p)
            return;
        n = (n + 255) & ~(size_t)255;
        std::lock_guard<std::mutex> g(mu);
        size_t off = (size_t)(p - base);
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + n == nx->first) {
            n += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                pv->second += n;
                return;
            }
        }
        free_[off] = n;
    }
};

struct Request {
    uint64_t ticket = 0;
    char *dA = nullptr, *dB = nullptr, *front = nullptr;
    size_t bytesA = 0, bytesB = 0, bytesF = 0;
    // ed_submit_dev: the strings are the caller's (not in the arena), ready
    // once `ready` (recorded on the caller's stream) has completed
    bool caller_strings = false;
    cudaEvent_t ready = nullptr;
    int64_t n = 0, m = 0;
    int32_t t = -1;
    // on the tile kernel (band wider than one batch CTA): its group size,
    // resident frontier (keep, radius keep_r) and the round / radius to
    // resume from (t0 = 0: from the start)
    int tile_G = 0;
    double cost = 0.0;
    char *keep = nullptr;
    size_t bytesK = 0;
    int64_t keep_r = 0, t0 = 0, R0 = 0;
};

// One pair handed to the tile kernel.
struct TileJob {
    const uint8_t *A, *B;
    int64_t n, m;
    const uint64_t *TA, *TB;
    int32_t *dump;
    int64_t dump_tmax;
    int G;       // CTAs of the group the pair runs on (1 .. grid)
    double cost; // estimated run time (any unit), to share CTAs among classes
    // resident frontier (time slicing, resuming on wider tiles), or null
    int32_t *keep = nullptr;
    int64_t keep_r = 0, t0 = 0, R0 = 0;
    // tile width to start from (diagonals per CTA; 0: what the longest
    // string could need).  Narrow tiles leave most of the SM's unified
    // L1/shared memory to the L1, which holds the rows' string bytes.
    int64_t smax_want = 0;
};

// What a tile launch left for one pair: its distance (st 0), or ST_WIDE,
// ST_LIMIT, or ST_SUSPENDED with the round and radius to resume from.
struct TileOut {
    uint64_t k = 0;
    uint32_t st = 0;
    int64_t rt = 0, rr = 0;
};

// Launch parameters of one call, resolved from the context's
// configuration, the tuning table and the built-in defaults.
struct Eff {
    int lcp_mode = ED_LCP_DIRECT; // AUTO resolved
    int hash_block = 32;
    int block_rounds = 32;
    int tile_width = 64;
    int warp_cap = 4096;
    int local_chunks = 0;
    int help_div = 8;
};

// One row of a tuning table: the launch parameters measured best for
// max(n, m) in [n_lo, n_hi) and expected edit rate (distance / max(n, m))
// in [r_lo, r_hi).
struct TuneRow {
    double n_lo, n_hi, r_lo, r_hi;
    int lcp_mode, block_rounds, tile_width, warp_cap, local_chunks, help_div;
};

// Reads a tuning table (whitespace-separated columns n_lo n_hi r_lo r_hi
// lcp block_rounds tile_width warp_cap local_chunks help_div; '#' starts a
// comment).  Returns false if the file cannot be read or a row is malformed.
bool read_tune_table(const char *path, std::vector<TuneRow> &rows)
{
    std::ifstream f(path);
    if (!f)
        return false;
    rows.clear();
    std::string line;
    while (std::getline(f, line)) {
        const size_t h = line.find('#');
        if (h != std::string::npos)
            line.resize(h);
        std::istringstream ss(line);
        TuneRow r{};
        if (!(ss >> r.n_lo))
            continue; // blank
        if (!(ss >> r.n_hi >> r.r_lo >> r.r_hi >> r.lcp_mode >> r.block_rounds >> r.tile_width >> r.warp_cap >>
              r.local_chunks >> r.help_div))
            return false;
        if (r.lcp_mode < ED_LCP_DIRECT || r.lcp_mode > ED_LCP_BHASH || r.block_rounds < 1 || r.block_rounds > HMAX ||
            r.tile_width < 1 || r.tile_width > SMAX_LIMIT || r.warp_cap < 512 || r.local_chunks < 0 ||
            r.help_div < 0)
            return false;
        rows.push_back(r);
    }
    return true;
}

// The table installed beside the library (tune_table.tsv in the directory
// of libedgb300.so).
std::string default_tune_path()
{
    Dl_info info{};
    if (dladdr((void *)&read_tune_table, &info) && info.dli_fname) {
        std::string p(info.dli_fname);
        const size_t s = p.rfind('/');
        return (s == std::string::npos ? std::string(".") : p.substr(0, s)) + "/tune_table.tsv";
    }
    return "tune_table.tsv";
}

// The row for a pair of lengths n, m with an expected distance hint (0:
// unknown, taken as an edit rate of 1e-4), or null.
const TuneRow *tune_lookup(const std::vector<TuneRow> &rows, int64_t n, int64_t m, int64_t hint)
{
    const double nm = (double)std::max<int64_t>(std::max(n, m), 1);
    const double rate = hint > 0 ? (double)hint / nm : 1e-4;
    for (const TuneRow &r : rows)
        if (nm >= r.n_lo && nm < r.n_hi && rate >= r.r_lo && rate < r.r_hi)
            return &r;
    return nullptr;
}

} // namespace

struct ed_ctx {
    ed_config cfg{};
    Eff eff;                     // parameters of the call in progress
    std::vector<TuneRow> tune;   // the tuning table (cfg.tune)
    int device = 0;
    int num_sms = 0;
    int grid = 0; // CTAs of the tile kernel
    int clock_khz = 1;
    int smem_optin = 0; // largest dynamic shared memory of one CTA
    cudaStream_t stream = nullptr;
    std::string last_err;
    size_t budget = 0;
    size_t held = 0;
    // pool
    DevBuf strA, strB, gf, ctl, gctl, slots, halo, pdesc, res, dump, hashA, hashB, scan, qx, qy, qo, bpairs,
        border, bnext, bfront, keep;
    unsigned long long *h_res = nullptr; // pinned result block
    size_t h_res_cap = 0;
    uint64_t hash_base = 0;
    uint64_t pow2[62]{};
    ed_stats last{};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
    std::mutex api_mu; // serialises the synchronous calls and the engine's steps
    // serving
    std::thread engine;
    std::mutex smu;
    std::condition_variable scv;
    bool stop = false;
    std::atomic<bool> engine_on{false};
    Arena arena;
    DevBuf arena_buf;
    std::deque<Request *> pending;
    std::vector<Request *> live;
    std::map<uint64_t, int64_t> results; // ticket -> k (or negative status)
    std::map<uint64_t, bool> known;
    uint64_t next_ticket = 1;
    uint64_t n_admitted = 0, n_completed = 0, n_steps = 0, n_slices = 0;
    cudaStream_t sstream = nullptr, cstream = nullptr;
    DevBuf s_pairs, s_order, s_next;
};

namespace {

int cuda_fail(ed_ctx *c, cudaError_t e, const char *what)
{
    if (c)
        c->last_err = std::string(what) + ": " + cudaGetErrorString(e);
    return ED_ECUDA;
}
#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return cuda_fail(ctx, e_, #call);                                                      \
    } while (0)

int ensure(ed_ctx *ctx, DevBuf &b, size_t bytes)
{
    if (b.bytes >= bytes)
        return ED_OK;
    if (b.p) {
        cudaFree(b.p);
        ctx->held -= b.bytes;
        b.p = nullptr;
        b.bytes = 0;
    }
    const size_t want = std::max(bytes, (size_t)4096);
    if (ctx->held + want > ctx->budget)
        return ED_ENOMEM;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        ctx->last_err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        return ED_ENOMEM;
    }
    b.bytes = want;
    ctx->held += want;
    return ED_OK;
}

void release(ed_ctx *ctx, DevBuf &b)
{
    if (b.p) {
        cudaFree(b.p);
        ctx->held -= b.bytes;
    }
    b.p = nullptr;
    b.bytes = 0;
}

int status_from_kernel(uint32_t st)
{
    if (st == 0)
        return ED_OK;
    if (st == ST_TIMEOUT)
        return ED_ETIMEOUT;
    if (st == ST_LIMIT)
        return ED_ELIMIT;
    return ED_ECUDA;
}

// sum over t = 0..k of the diagonals of [-t, t] inside [-n, m]
uint64_t count_extensions(int64_t n, int64_t m, int64_t k)
{
    auto S = [](int64_t a, int64_t b) -> uint64_t { // sum_{t=0}^{b} min(t, a)
        if (b < 0)
            return 0;
        if (b <= a)
            return (uint64_t)b * (uint64_t)(b + 1) / 2;
        return (uint64_t)a * (uint64_t)(a + 1) / 2 + (uint64_t)(b - a) * (uint64_t)a;
    };
    return (uint64_t)(k + 1) + S(n, k) + S(m, k);
}

bool bad_len(size_t n) { return n > (size_t)MAX_LEN; }

bool hash_mode(const ed_ctx *ctx) { return ctx->eff.lcp_mode == ED_LCP_HASH || ctx->eff.lcp_mode == ED_LCP_BHASH; }

// Stride of the call's prefix tables: 1 (full, Sec. 3.2) or the block size
// of Sec. 3.3 (blocked, Alg. 2).
int64_t hash_stride(const ed_ctx *ctx)
{
    return ctx->eff.lcp_mode == ED_LCP_BHASH ? (int64_t)ctx->eff.hash_block : 1;
}

// The call's launch parameters: built-in defaults, then (with cfg.tune and a
// single pair of lengths n, m) the tuning table's row, then every field the
// configuration sets explicitly.
void resolve(ed_ctx *ctx, int64_t n, int64_t m, bool single)
{
    Eff e;
    const ed_config &c = ctx->cfg;
    e.hash_block = c.hash_block;
    if (single && c.tune) {
        if (const TuneRow *r = tune_lookup(ctx->tune, n, m, c.distance_hint)) {
            e.lcp_mode = r->lcp_mode;
            e.block_rounds = r->block_rounds;
            e.tile_width = r->tile_width;
            e.warp_cap = r->warp_cap;
            e.local_chunks = r->local_chunks;
            e.help_div = r->help_div;
        }
    }
    if (c.lcp_mode != ED_LCP_AUTO)
        e.lcp_mode = c.lcp_mode;
    if (c.block_rounds > 0)
        e.block_rounds = std::min(c.block_rounds, HMAX);
    if (c.tile_width > 0)
        e.tile_width = c.tile_width;
    if (c.warp_cap > 0)
        e.warp_cap = c.warp_cap;
    if (c.local_chunks != 0)
        e.local_chunks = std::max(0, c.local_chunks);
    if (c.help_div != 0)
        e.help_div = std::max(0, c.help_div);
    ctx->eff = e;
}

// Waits for the prefix-hash scan last launched on s with the context's scan
// state and maps its status word: a look-back wait that gave up leaves a
// wrong table, reported as ED_ETIMEOUT.
int scan_result(ed_ctx *ctx, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    const uint32_t st = prefix_hash_status(ctx->scan.p, s, &e);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "prefix hash scan");
    if (st != 0) {
        ctx->last_err = "prefix hash scan: a look-back wait gave up";
        return status_from_kernel(st);
    }
    return ED_OK;
}

int run_hash_tables(ed_ctx *ctx, const uint8_t *dA, int64_t n, const uint8_t *dB, int64_t m,
                    cudaStream_t s)
{
    int r;
    const int64_t b = hash_stride(ctx);
    if ((r = ensure(ctx, ctx->hashA, sizeof(uint64_t) * (n / b + 1))) != ED_OK)
        return r;
    if ((r = ensure(ctx, ctx->hashB, sizeof(uint64_t) * (m / b + 1))) != ED_OK)
        return r;
    const size_t sb = std::max(prefix_hash_state_bytes(n), prefix_hash_state_bytes(m));
    if ((r = ensure(ctx, ctx->scan, sb)) != ED_OK)
        return r;
    CK(launch_prefix_hash(dA, n, ctx->hash_base, (uint64_t *)ctx->hashA.p, b, ctx->scan.p,
                          prefix_hash_state_bytes(n), s));
    if ((r = scan_result(ctx, s)) != ED_OK)
        return r;
    CK(launch_prefix_hash(dB, m, ctx->hash_base, (uint64_t *)ctx->hashB.p, b, ctx->scan.p,
                          prefix_hash_state_bytes(m), s));
    if ((r = scan_result(ctx, s)) != ED_OK)
        return r;
    ctx->last.kernel_launches += 2;
    return ED_OK;
}

// One tile launch over the jobs, CTA groups by class (one class per group
// size wanted).  Every class that fits gets one group, largest first; the
// remaining CTAs go, one group at a time, to the class whose estimated run
// time per group is highest.  out[i] receives each pair's outcome; the
// counters of pairs that finished or were suspended are summed into
// ctx->last.  budget_ns > 0 time-slices the pairs that have a keep buffer.
static int run_tiles_once(ed_ctx *ctx, const std::vector<TileJob> &jobs, cudaStream_t s, uint64_t budget_ns,
                          std::vector<TileOut> &out)
{
    int r;
    const int np = (int)jobs.size();
    const int h = ctx->eff.block_rounds;
    const int s0 = ctx->eff.tile_width;
    // classes, ascending group size; pairs by class, then cost, largest first
    std::vector<int> sizes;
    for (const TileJob &j : jobs)
        sizes.push_back(std::max(1, std::min(j.G, ctx->grid)));
    std::vector<int> Gs = sizes;
    std::sort(Gs.begin(), Gs.end());
    Gs.erase(std::unique(Gs.begin(), Gs.end()), Gs.end());
    if ((int)Gs.size() > MAX_CLS) { // merge the smallest classes upwards
        const int drop = (int)Gs.size() - MAX_CLS;
        for (int &g : sizes)
            if (g < Gs[drop])
                g = Gs[drop];
        Gs.erase(Gs.begin(), Gs.begin() + drop);
    }
    const int ncls = (int)Gs.size();
    auto cls_of = [&](int g) { return (int)(std::lower_bound(Gs.begin(), Gs.end(), g) - Gs.begin()); };
    std::vector<int> ord(np);
    for (int i = 0; i < np; i++)
        ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
        const int ca = cls_of(sizes[a]), cb = cls_of(sizes[b]);
        return ca != cb ? ca < cb : jobs[a].cost > jobs[b].cost;
    });
    std::vector<int> npc(ncls, 0), ng(ncls, 0);
    std::vector<double> wc(ncls, 0.0);
    std::vector<int64_t> nmc(ncls, 0), wantc(ncls, 0);
    for (int i = 0; i < np; i++) {
        const int c = cls_of(sizes[i]);
        npc[c]++;
        wc[c] += std::max(jobs[i].cost, 1.0);
        nmc[c] = std::max(nmc[c], std::max(jobs[i].n, jobs[i].m));
        wantc[c] = std::max<int64_t>(wantc[c], jobs[i].smax_want > 0 ? jobs[i].smax_want : SMAX_LIMIT);
    }
    int used = 0;
    for (int c = ncls - 1; c >= 0; c--)
        if (used + Gs[c] <= ctx->grid) {
            ng[c] = 1;
            used += Gs[c];
        }
    for (;;) {
        int best = -1;
        double bw = -1.0;
        for (int c = 0; c < ncls; c++)
            if (ng[c] > 0 && ng[c] < npc[c] && used + Gs[c] <= ctx->grid && wc[c] / ng[c] > bw) {
                bw = wc[c] / ng[c];
                best = c;
            }
        if (best < 0)
            break;
        ng[best]++;
        used += Gs[best];
    }
    int64_t nm = 0;
    for (const TileJob &j : jobs)
        nm = std::max(nm, std::max(j.n, j.m));
    int64_t kcap = nm + 1;
    if (ctx->cfg.max_rounds > 0)
        kcap = std::min<int64_t>(kcap, ctx->cfg.max_rounds);
    kcap = std::min<int64_t>(kcap, (int64_t)1 << 28);
    kcap = std::max<int64_t>(kcap, h);
    // tile capacity: what the widest band of any class needs, at most SMAX_LIMIT
    // (a group also runs pairs of the classes below its own)
    int64_t smax = std::max(h, s0), nm_below = 0, want_below = 0;
    for (int c = 0; c < ncls; c++) {
        nm_below = std::max(nm_below, nmc[c]);
        want_below = std::max(want_below, wantc[c]);
        if (ng[c] > 0)
            smax = std::max<int64_t>(
                smax, std::min<int64_t>(std::min<int64_t>(SMAX_LIMIT, want_below),
                                        (2 * std::min(kcap, nm_below) + 1 + Gs[c] - 1) / Gs[c] + 1));
    }
    LvArgs P{};
    int ngroups = 0;
    int64_t gf_total = 0;
    int cta = 0;
    int pi = 0;
    for (int c = 0; c < ncls; c++) {
        P.cls_G[c] = Gs[c];
        P.cls_c0[c] = cta;
        P.cls_g0[c] = ngroups;
        P.cls_p0[c] = pi;
        P.cls_kc[c] = (int32_t)std::min<int64_t>(kcap, (int64_t)Gs[c] * smax);
        P.cls_gf[c] = gf_total;
        cta += ng[c] * Gs[c];
        ngroups += ng[c];
        pi += npc[c];
        gf_total += (int64_t)ng[c] * 2 * (2 * (int64_t)P.cls_kc[c] + 5);
    }
    P.cls_c0[ncls] = cta;
    P.cls_p0[ncls] = pi;
    P.ncls = ncls;
    const int grid = cta;
    if ((r = ensure(ctx, ctx->gf, sizeof(int32_t) * (size_t)std::max<int64_t>(gf_total, 1))) != ED_OK ||
        (r = ensure(ctx, ctx->ctl, sizeof(LaunchCtl))) != ED_OK ||
        (r = ensure(ctx, ctx->gctl, sizeof(GroupCtl) * ngroups)) != ED_OK ||
        (r = ensure(ctx, ctx->slots, sizeof(JobSlot) * grid * JOB_RING)) != ED_OK ||
        (r = ensure(ctx, ctx->halo, sizeof(unsigned long long) * (size_t)grid * 4 * HMAX)) != ED_OK ||
        (r = ensure(ctx, ctx->pdesc, sizeof(PairDesc) * np)) != ED_OK ||
        (r = ensure(ctx, ctx->res, sizeof(unsigned long long) * R_COUNT * np)) != ED_OK)
        return r;
    const size_t hres = sizeof(unsigned long long) * R_COUNT * np + 64;
    if (ctx->h_res_cap < hres) {
        if (ctx->h_res)
            cudaFreeHost(ctx->h_res);
        ctx->h_res = nullptr;
        ctx->h_res_cap = 0;
        CK(cudaMallocHost((void **)&ctx->h_res, hres));
        ctx->h_res_cap = hres;
    }
    // pair slot q runs job ord[q]; its counters land in row q
    std::vector<PairDesc> pd(np);
    for (int q = 0; q < np; q++) {
        const TileJob &j = jobs[ord[q]];
        pd[q] = PairDesc{};
        pd[q].A = j.A;
        pd[q].B = j.B;
        pd[q].n = j.n;
        pd[q].m = j.m;
        pd[q].TA = j.TA;
        pd[q].TB = j.TB;
        pd[q].res = (unsigned long long *)ctx->res.p + (size_t)R_COUNT * q;
        pd[q].dump = j.dump;
        pd[q].dump_tmax = (int32_t)j.dump_tmax;
        pd[q].keep = j.keep;
        pd[q].keep_r = j.keep_r;
        pd[q].t0 = j.t0;
        pd[q].R0 = j.R0;
    }
    P.pairs = (const PairDesc *)ctx->pdesc.p;
    P.npairs = np;
    P.gctl = (GroupCtl *)ctx->gctl.p;
    P.ctl = (LaunchCtl *)ctx->ctl.p;
    P.slots = (JobSlot *)ctx->slots.p;
    P.halo = (unsigned long long *)ctx->halo.p;
    P.gf = (int32_t *)ctx->gf.p;
    P.kcap = (int32_t)kcap;
    P.smax = (int32_t)smax;
    P.h = h;
    P.s0 = s0;
    P.t2_cap = ctx->eff.warp_cap;
    P.use_hash = jobs[0].TA != nullptr;
    P.hash_b = (int32_t)hash_stride(ctx);
    std::memcpy(P.pow2, ctx->pow2, sizeof(P.pow2));
    P.spin_ns = ctx->cfg.spin_limit_ns;
    P.idle_ns = ctx->cfg.spin_limit_ns * 60;
    P.budget_ns = budget_ns;
    P.sync_rounds = 16 * h;
    P.help_div = ctx->eff.help_div;
    P.local_chunks = ctx->eff.local_chunks;
    // bulk-copy staging of long-slide chunks (two stages: the owner streams
    // its first chunks with the next one's copies in flight) when the tiles
    // leave room for it
    P.stage = lv_tiles_smem_bytes((int)smax, h, 2) <= (size_t)ctx->smem_optin
                  ? 2
                  : (lv_tiles_smem_bytes((int)smax, h, 1) <= (size_t)ctx->smem_optin ? 1 : 0);
    CK(cudaMemcpyAsync(ctx->pdesc.p, pd.data(), sizeof(PairDesc) * np, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(ctx->ctl.p, 0, sizeof(LaunchCtl), s));
    CK(cudaMemsetAsync(ctx->gctl.p, 0, sizeof(GroupCtl) * ngroups, s));
    CK(cudaMemsetAsync(ctx->slots.p, 0, sizeof(JobSlot) * grid * JOB_RING, s));
    CK(cudaMemsetAsync(ctx->res.p, 0, sizeof(unsigned long long) * R_COUNT * np, s));
    CK(cudaEventRecord(ctx->ev0, s));
    CK(launch_lv_tiles(P, grid, s));
    CK(cudaEventRecord(ctx->ev1, s));
    CK(cudaMemcpyAsync(ctx->h_res, ctx->res.p, sizeof(unsigned long long) * R_COUNT * np,
                       cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ctx->h_res + (size_t)R_COUNT * np, ctx->ctl.p, sizeof(uint32_t),
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ctx->last.kernel_launches += 1;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    ctx->last.kernel_ms += ms;
    const int lst = status_from_kernel(*(uint32_t *)(ctx->h_res + (size_t)R_COUNT * np));
    if (lst != ED_OK) {
        unsigned long long dg[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        cudaMemcpy(dg, (char *)ctx->ctl.p + offsetof(LaunchCtl, diag), sizeof(dg), cudaMemcpyDeviceToHost);
        char buf[256];
        std::snprintf(buf, sizeof(buf), "kernel check failed: site %llu cta %llu t %llu want %llx seen %llx %llx %llx",
                      dg[0], dg[1], dg[2], dg[3], dg[4], dg[5], dg[6]);
        ctx->last_err = buf;
        return lst;
    }
    out.assign(np, TileOut{});
    for (int q = 0; q < np; q++) {
        const int i = ord[q];
        const unsigned long long *R = ctx->h_res + (size_t)R_COUNT * q;
        TileOut &o = out[i];
        o.st = (uint32_t)R[R_STATUS];
        if (o.st == ST_SUSPENDED || (o.st == ST_WIDE && R[R_RESUME_T] > 0)) {
            o.rt = (int64_t)R[R_RESUME_T];
            o.rr = (int64_t)R[R_RESUME_R];
            // rounds t0 .. rt - 1 done in this launch
            ctx->last.extensions += count_extensions(jobs[i].n, jobs[i].m, o.rt - 1) -
                                    (jobs[i].t0 > 0 ? count_extensions(jobs[i].n, jobs[i].m, jobs[i].t0 - 1) : 0);
        } else if (o.st != 0) {
            continue;
        } else {
            o.k = R[R_K];
            ctx->last.extensions += count_extensions(jobs[i].n, jobs[i].m, (int64_t)R[R_K]) -
                                    (jobs[i].t0 > 0 ? count_extensions(jobs[i].n, jobs[i].m, jobs[i].t0 - 1) : 0);
        }
        ctx->last.slide_chars += R[R_SLIDE];
        ctx->last.compared_bytes += 2ull * (R[R_SLIDE] + R[R_MISMATCH]);
        ctx->last.long_slides += R[R_LONG];
        ctx->last.open_slides += R[R_OPEN];
        ctx->last.wide_rounds += R[R_WIDE] * (uint64_t)h;
        ctx->last.hash_queries += R[R_HASHQ];
        ctx->last.hash_collisions += R[R_HASHCOLL];
        // SM cycles -> ms at the device's nominal clock
        const double per_ms = (double)ctx->clock_khz;
        for (int j = 0; j < 4; j++)
            ctx->last.phase_ms[j] += (double)R[R_T0 + j] / per_ms;
        if (R[R_T0 + 5])
            ctx->last.phase_ms[4] += (double)R[R_T0 + 4] / (double)R[R_T0 + 5] / per_ms;
    }
    return ED_OK;
}

// Runs pairs on the tile kernel until each has its distance: a pair whose
// band outgrew its group runs again on a group twice as large; a pair
// that needs more than the whole grid, or more rounds than the cap, fails
// the call with ED_ELIMIT.
int run_tiles(ed_ctx *ctx, const std::vector<TileJob> &jobs, cudaStream_t s, std::vector<uint64_t> &k)
{
    k.assign(jobs.size(), 0);
    std::vector<TileJob> cur = jobs;
    std::vector<size_t> idx(jobs.size());
    for (size_t i = 0; i < idx.size(); i++)
        idx[i] = i;
    while (!cur.empty()) {
        std::vector<TileOut> o;
        int r = run_tiles_once(ctx, cur, s, 0, o);
        if (r != ED_OK)
            return r;
        std::vector<TileJob> next;
        std::vector<size_t> nidx;
        for (size_t i = 0; i < cur.size(); i++) {
            if (o[i].st == 0) {
                k[idx[i]] = o[i].k;
            } else if (o[i].st == ST_WIDE &&
                       (cur[i].G < ctx->grid || (cur[i].smax_want > 0 && cur[i].smax_want < SMAX_LIMIT))) {
                // wider tiles first, then a larger group; from the saved
                // round when the kernel left one in the pair's keep buffer
                TileJob j = cur[i];
                if (j.smax_want > 0 && j.smax_want < SMAX_LIMIT)
                    j.smax_want = std::min<int64_t>(SMAX_LIMIT, 4 * j.smax_want);
                else
                    j.G = std::min(ctx->grid, 2 * std::max(1, j.G));
                const bool resume = j.keep && o[i].rt > 0;
                j.t0 = resume ? o[i].rt : 0;
                j.R0 = resume ? o[i].rr : 0;
                next.push_back(j);
                nidx.push_back(idx[i]);
            } else {
                char buf[160];
                std::snprintf(buf, sizeof(buf), "pair %zu: %s", idx[i],
                              o[i].st == ST_WIDE ? "band wider than the whole grid's tiles hold"
                                                 : "more rounds than the configured cap");
                ctx->last_err = buf;
                return ED_ELIMIT;
            }
        }
        cur.swap(next);
        idx.swap(nidx);
    }
    return ED_OK;
}

// One pair, device strings, on stream s (the whole grid as one group).
int run_pair(ed_ctx *ctx, const uint8_t *dA, int64_t n, const uint8_t *dB, int64_t m,
             cudaStream_t s, int32_t *dump, int64_t dump_tmax, uint64_t *k_out)
{
    int r;
    TileJob j{dA, dB, n, m, nullptr, nullptr, dump, dump_tmax, ctx->grid, 1.0};
    // narrow tiles first (a large L1), saved and resumed on wider ones when
    // the band outgrows them
    j.smax_want = START_TILE;
    j.keep_r = std::min<int64_t>(std::max(n, m), (int64_t)ctx->grid * SMAX_LIMIT);
    if ((r = ensure(ctx, ctx->keep, sizeof(int32_t) * (size_t)(2 * j.keep_r + 5))) != ED_OK)
        return r;
    j.keep = (int32_t *)ctx->keep.p;
    if (hash_mode(ctx)) {
        CK(cudaEventRecord(ctx->ev2, s));
        if ((r = run_hash_tables(ctx, dA, n, dB, m, s)) != ED_OK)
            return r;
        j.TA = (const uint64_t *)ctx->hashA.p;
        j.TB = (const uint64_t *)ctx->hashB.p;
    }
    std::vector<uint64_t> k;
    if ((r = run_tiles(ctx, {j}, s, k)) != ED_OK)
        return r;
    if (hash_mode(ctx)) {
        float bms = 0.f;
        cudaEventElapsedTime(&bms, ctx->ev2, ctx->ev0);
        ctx->last.build_ms += bms;
    }
    ctx->last.k = k[0];
    *k_out = k[0];
    return ED_OK;
}

} // namespace

// =====================================================================
extern "C" {

const char *ed_strerror(int s)
{
    switch (s) {
    case ED_OK: return "ok";
    case ED_EAGAIN: return "not ready";
    case ED_EINVAL: return "invalid argument";
    case ED_ENOMEM: return "out of memory or over the memory budget";
    case ED_ECUDA: return "CUDA error";
    case ED_ETIMEOUT: return "a bounded device-side wait timed out";
    case ED_EBUSY: return "busy: no free slot or memory, retry";
    case ED_ENOTFOUND: return "unknown ticket";
    case ED_ELIMIT: return "distance exceeds the frontier capacity";
    default: return "unknown status";
    }
}

int ed_tune_lookup(const char *table, size_t n, size_t m, int64_t distance_hint, ed_config *cfg)
{
    if (!cfg || distance_hint < 0)
        return ED_EINVAL;
    std::vector<TuneRow> rows;
    const std::string path = table ? std::string(table) : default_tune_path();
    if (!read_tune_table(path.c_str(), rows))
        return ED_EINVAL;
    const TuneRow *r = tune_lookup(rows, (int64_t)n, (int64_t)m, distance_hint);
    if (!r)
        return ED_ENOTFOUND;
    cfg->lcp_mode = r->lcp_mode;
    cfg->block_rounds = r->block_rounds;
    cfg->tile_width = r->tile_width;
    cfg->warp_cap = r->warp_cap;
    cfg->local_chunks = r->local_chunks > 0 ? r->local_chunks : -1;
    cfg->help_div = r->help_div > 0 ? r->help_div : -1;
    return ED_OK;
}

int ed_config_default(ed_config *cfg)
{
    if (!cfg)
        return ED_EINVAL;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->device = -1;
    cfg->max_inflight = 1024;
    cfg->lcp_mode = ED_LCP_AUTO;
    cfg->spin_limit_ns = 2000000000ull;
    return ED_OK;
}

const char *ed_last_cuda_error(ed_ctx *ctx) { return ctx ? ctx->last_err.c_str() : ""; }

int ed_create(ed_ctx **out, const ed_config *cfg)
{
    if (!out)
        return ED_EINVAL;
    *out = nullptr;
    std::unique_ptr<ed_ctx> c(new ed_ctx());
    ed_ctx *ctx = c.get();
    if (cfg)
        c->cfg = *cfg;
    else
        ed_config_default(&c->cfg);
    if (c->cfg.spin_limit_ns == 0)
        c->cfg.spin_limit_ns = 2000000000ull;
    if (c->cfg.max_inflight <= 0)
        c->cfg.max_inflight = 1024;
    if (c->cfg.hash_block == 0)
        c->cfg.hash_block = 32;
    if (c->cfg.lcp_mode < 0 || c->cfg.lcp_mode > 3 || c->cfg.tile_width < 0 || c->cfg.block_rounds < 0 ||
        c->cfg.tile_width > SMAX_LIMIT || c->cfg.hash_block < 1 || c->cfg.hash_block > 4096 ||
        c->cfg.warp_cap < 0 || (c->cfg.warp_cap > 0 && c->cfg.warp_cap < 512) || c->cfg.local_chunks < -1 ||
        c->cfg.help_div < -1 || c->cfg.distance_hint < 0)
        return ED_EINVAL;
    if (c->cfg.tune) {
        const std::string path = c->cfg.tune_table ? std::string(c->cfg.tune_table) : default_tune_path();
        if (!read_tune_table(path.c_str(), c->tune))
            return ED_EINVAL;
        c->cfg.tune_table = nullptr; // the caller's string is not kept
    }
    int dev = c->cfg.device;
    if (dev < 0)
        CK(cudaGetDevice(&dev));
    CK(cudaSetDevice(dev));
    c->device = dev;
    CK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaDeviceGetAttribute(&c->clock_khz, cudaDevAttrClockRate, dev));
    CK(cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    c->clock_khz = std::max(c->clock_khz, 1);
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    c->budget = c->cfg.mem_budget_bytes ? c->cfg.mem_budget_bytes : (size_t)(fr * 0.6);
    // co-resident grid for the cooperative tile kernel: one 512-thread CTA per SM
    c->grid = c->cfg.grid_ctas > 0 ? std::min(c->cfg.grid_ctas, c->num_sms) : c->num_sms;
    c->grid = std::min(c->grid, MAX_GRID);
    CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    CK(cudaEventCreate(&c->ev0));
    CK(cudaEventCreate(&c->ev1));
    CK(cudaEventCreate(&c->ev2));
    // hash base: seeded, in [2^8, q-2]
    const uint64_t seed = c->cfg.hash_seed ? c->cfg.hash_seed : 0x5eed2306174610ull;
    c->hash_base = 256 + splitmix(seed) % (Q61H - 2 - 256);
    c->pow2[0] = c->hash_base;
    for (int j = 1; j < 62; j++)
        c->pow2[j] = hmul(c->pow2[j - 1], c->pow2[j - 1]);
    *out = c.release();
    return ED_OK;
}

static void engine_stop(ed_ctx *ctx);

int ed_destroy(ed_ctx *ctx)
{
    if (!ctx)
        return ED_EINVAL;
    engine_stop(ctx);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    DevBuf *bufs[] = {&ctx->strA,  &ctx->strB,   &ctx->gf,    &ctx->ctl,    &ctx->gctl,      &ctx->slots,
                      &ctx->halo,  &ctx->pdesc,  &ctx->res,   &ctx->dump,   &ctx->hashA,     &ctx->hashB,
                      &ctx->scan,  &ctx->qx,     &ctx->qy,    &ctx->qo,     &ctx->bpairs,    &ctx->border,
                      &ctx->bnext, &ctx->bfront, &ctx->arena_buf, &ctx->s_pairs, &ctx->s_order, &ctx->s_next,
                      &ctx->keep};
    for (DevBuf *b : bufs)
        release(ctx, *b);
    if (ctx->h_res)
        cudaFreeHost(ctx->h_res);
    if (ctx->ev0)
        cudaEventDestroy(ctx->ev0);
    if (ctx->ev1)
        cudaEventDestroy(ctx->ev1);
    if (ctx->ev2)
        cudaEventDestroy(ctx->ev2);
    if (ctx->stream)
        cudaStreamDestroy(ctx->stream);
    delete ctx;
    return ED_OK;
}

uint64_t ed_hash_base(ed_ctx *ctx) { return ctx ? ctx->hash_base : 0; }

int ed_last_stats(ed_ctx *ctx, ed_stats *out)
{
    if (!ctx || !out)
        return ED_EINVAL;
    *out = ctx->last;
    return ED_OK;
}

int ed_distance_dev(ed_ctx *ctx, const uint8_t *A, size_t n, const uint8_t *B, size_t m, uint64_t *k,
                    void *stream)
{
    if (!ctx || !k || (n && !A) || (m && !B) || bad_len(n) || bad_len(m))
        return ED_EINVAL;
    std::lock_guard<std::mutex> g(ctx->api_mu);
    CK(cudaSetDevice(ctx->device));
    ctx->last = ed_stats{};
    resolve(ctx, (int64_t)n, (int64_t)m, true);
    return run_pair(ctx, A, (int64_t)n, B, (int64_t)m, (cudaStream_t)stream, nullptr, 0, k);
}

int ed_distance(ed_ctx *ctx, const uint8_t *A, size_t n, const uint8_t *B, size_t m, uint64_t *k)
{
    if (!ctx || !k || (n && !A) || (m && !B) || bad_len(n) || bad_len(m))
        return ED_EINVAL;
    std::lock_guard<std::mutex> g(ctx->api_mu);
    CK(cudaSetDevice(ctx->device));
    ctx->last = ed_stats{};
    resolve(ctx, (int64_t)n, (int64_t)m, true);
    int r;
    if ((r = ensure(ctx, ctx->strA, n + 64)) != ED_OK || (r = ensure(ctx, ctx->strB, m + 64)) != ED_OK)
        return r;
    if (n)
        CK(cudaMemcpyAsync(ctx->strA.p, A, n, cudaMemcpyHostToDevice, ctx->stream));
    if (m)
        CK(cudaMemcpyAsync(ctx->strB.p, B, m, cudaMemcpyHostToDevice, ctx->stream));
    return run_pair(ctx, (const uint8_t *)ctx->strA.p, (int64_t)n, (const uint8_t *)ctx->strB.p, (int64_t)m,
                    ctx->stream, nullptr, 0, k);
}

// The frontiers of rounds 0..t_max into the host array out (ed_frontiers_dev
// up to t_max_limit rounds).
static int frontiers_to_host(ed_ctx *ctx, const uint8_t *A, size_t n, const uint8_t *B, size_t m, int64_t t_max,
                             int32_t *out, uint64_t *k, void *stream, int64_t t_max_limit)
{
    if (!ctx || !k || !out || t_max < 0 || t_max > t_max_limit || (n && !A) || (m && !B) || bad_len(n) ||
        bad_len(m))
        return ED_EINVAL;
    std::lock_guard<std::mutex> g(ctx->api_mu);
    CK(cudaSetDevice(ctx->device));
    ctx->last = ed_stats{};
    resolve(ctx, (int64_t)n, (int64_t)m, true);
    const size_t cnt = (size_t)(t_max + 1) * (size_t)(2 * t_max + 1);
    int r;
    if ((r = ensure(ctx, ctx->dump, cnt * sizeof(int32_t))) != ED_OK)
        return r;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemsetAsync(ctx->dump.p, 0xC0, cnt * sizeof(int32_t), s));
    uint64_t kk = 0;
    r = run_pair(ctx, A, (int64_t)n, B, (int64_t)m, s, (int32_t *)ctx->dump.p, t_max, &kk);
    if (r != ED_OK)
        return r;
    CK(cudaMemcpy(out, ctx->dump.p, cnt * sizeof(int32_t), cudaMemcpyDeviceToHost));
    // tiles that had not yet seen k may have gone on past round k: the
    // frontiers after round k are not part of the answer
    for (int64_t t = (int64_t)kk + 1; t <= t_max; t++)
        for (int64_t i = 0; i < 2 * t_max + 1; i++)
            out[t * (2 * t_max + 1) + i] = (int32_t)0xC0C0C0C0;
    *k = kk <= (uint64_t)t_max ? kk : UINT64_MAX;
    return ED_OK;
}

int ed_frontiers_dev(ed_ctx *ctx, const uint8_t *A, size_t n, const uint8_t *B, size_t m, int64_t t_max,
                     int32_t *out, uint64_t *k, void *stream)
{
    return frontiers_to_host(ctx, A, n, B, m, t_max, out, k, stream, 4096);
}

// The walk back of ed_edit_script_dev over the frontiers F (rows 0..k of
// a dump with bound T).  ops receives (kind, x, y) triples from the end of
// the strings backwards.  Returns false if the frontiers contradict
// themselves (a device error).
static bool trace_script(const int32_t *F, int64_t T, int64_t n, int64_t m, int64_t k, std::vector<int64_t> &ops)
{
    constexpr int64_t NONE = INT64_MIN;
    const int64_t W = 2 * T + 1;
    auto L = [&](int64_t t, int64_t d) -> int64_t {
        if (t < 0 || d < -t || d > t)
            return NONE;
        const int32_t v = F[t * W + d + T];
        return v < 0 ? NONE : (int64_t)v;
    };
    int64_t x = n, y = m, t = k;
    if (L(k, m - n) != n) // (n, m) is not reached in round k
        return false;
    while (x > 0 || y > 0) {
        const int64_t d = y - x;
        if (t == 0) // the slide of round 0 from (0, 0)
            return d == 0 && x <= L(0, 0);
        const int64_t a1 = L(t - 1, d - 1), a2 = L(t - 1, d), a3 = L(t - 1, d + 1);
        if (a2 != NONE && x <= a2) { // distance at most t - 1 already
            t--;
            continue;
        }
        // the start row of round t's slide on diagonal d
        int64_t c = NONE;
        if (a1 != NONE)
            c = std::max(c, a1);
        if (a2 != NONE)
            c = std::max(c, a2 + 1);
        if (a3 != NONE)
            c = std::max(c, a3 + 1);
        if (c == NONE)
            return false;
        c = std::min(c, d <= m - n ? n : m - d);
        if (x > c) { // back along the slide: matches
            x = c;
            y = c + d;
            continue;
        }
        if (x < c)
            return false;
        // one edit from a cell of distance t - 1
        if (x >= 1 && y >= 1 && a2 != NONE && x - 1 <= a2) {
            ops.insert(ops.end(), {(int64_t)ED_OP_SUB, x - 1, y - 1});
            x--, y--;
        } else if (x >= 1 && a3 != NONE && x - 1 <= a3) {
            ops.insert(ops.end(), {(int64_t)ED_OP_DEL, x - 1, y});
            x--;
        } else if (y >= 1 && a1 != NONE && x <= a1) {
            ops.insert(ops.end(), {(int64_t)ED_OP_INS, x, y - 1});
            y--;
        } else {
            return false;
        }
        t--;
    }
    return true;
}

int ed_edit_script_dev(ed_ctx *ctx, const uint8_t *A, size_t n, const uint8_t *B, size_t m, int64_t t_max,
                       int64_t *ops, size_t cap, size_t *nops, uint64_t *k, void *stream)
{
    if (!ctx || !k || !nops || (cap && !ops) || t_max < 0 || t_max > ED_SCRIPT_MAX_ROUNDS || (n && !A) ||
        (m && !B) || bad_len(n) || bad_len(m))
        return ED_EINVAL;
    std::vector<int32_t> F;
    try {
        F.resize((size_t)(t_max + 1) * (size_t)(2 * t_max + 1));
    } catch (const std::bad_alloc &) {
        return ED_ENOMEM;
    }
    uint64_t kk = 0;
    int r = frontiers_to_host(ctx, A, n, B, m, t_max, F.data(), &kk, stream, ED_SCRIPT_MAX_ROUNDS);
    if (r != ED_OK)
        return r;
    *k = kk;
    *nops = 0;
    if (kk == UINT64_MAX)
        return ED_ELIMIT;
    if (cap < kk)
        return ED_EINVAL;
    // frontiers that contradict themselves would be a device fault
    return ed_trace_script(F.data(), t_max, n, m, kk, ops, cap, nops) == ED_OK ? ED_OK : ED_ECUDA;
}

int ed_trace_script(const int32_t *F, int64_t t_max, size_t n, size_t m, uint64_t k, int64_t *ops, size_t cap,
                    size_t *nops)
{
    if (!F || !nops || (cap && !ops) || t_max < 0 || k > (uint64_t)t_max || cap < k || bad_len(n) || bad_len(m))
        return ED_EINVAL;
    *nops = 0;
    std::vector<int64_t> back;
    back.reserve(3 * (size_t)k);
    if (!trace_script(F, t_max, (int64_t)n, (int64_t)m, (int64_t)k, back) || back.size() != 3 * k)
        return ED_EINVAL;
    for (size_t i = 0; i < k; i++)
        for (int j = 0; j < 3; j++)
            ops[3 * i + j] = back[3 * (k - 1 - i) + j];
    *nops = (size_t)k;
    return ED_OK;
}

int ed_prefix_hash_dev(ed_ctx *ctx, const uint8_t *X, size_t len, uint64_t *T, void *stream)
{
    if (!ctx || !T || (len && !X) || bad_len(len))
        return ED_EINVAL;
    std::lock_guard<std::mutex> g(ctx->api_mu);
    CK(cudaSetDevice(ctx->device));
    int r;
    const size_t sb = prefix_hash_state_bytes((int64_t)len);
    if ((r = ensure(ctx, ctx->scan, sb)) != ED_OK)
        return r;
    cudaStream_t s = (cudaStream_t)stream;
    CK(launch_prefix_hash(X, (int64_t)len, ctx->hash_base, T, 1, ctx->scan.p, sb, s));
    return scan_result(ctx, s);
}

int ed_prefix_hash_blocked_dev(ed_ctx *ctx, const uint8_t *X, size_t len, size_t b, uint64_t *T, void *stream)
{
    if (!ctx || !T || (len && !X) || bad_len(len) || b < 1 || b > (size_t)1 << 20)
        return ED_EINVAL;
    std::lock_guard<std::mutex> g(ctx->api_mu);
    CK(cudaSetDevice(ctx->device));
    int r;
    const size_t sb = prefix_hash_state_bytes((int64_t)len);
    if ((r = ensure(ctx, ctx->scan, sb)) != ED_OK)
        return r;
    cudaStream_t s = (cudaStream_t)stream;
    CK(launch_prefix_hash(X, (int64_t)len, ctx->hash_base, T, (int64_t)b, ctx->scan.p, sb, s));
    return scan_result(ctx, s);
}

int ed_lcp_dev(ed_ctx *ctx, const uint8_t *A, size_t n, const uint8_t *B, size_t m, const int64_t *x,
               const int64_t *y, size_t q, int method, const uint64_t *TA, const uint64_t *TB, int64_t *out,
               void *stream)
{
    if (!ctx || (q && (!x || !y || !out)) || method < 0 || method > 7 || bad_len(n) || bad_len(m))
        return ED_EINVAL;
    if (method >= 3 && method <= 6 && (!TA || !TB))
        return ED_EINVAL;
    for (size_t i = 0; i < q; i++)
        if (x[i] < 0 || y[i] < 0 || x[i] > (int64_t)n || y[i] > (int64_t)m)
            return ED_EINVAL;
    std::lock_guard<std::mutex> g(ctx->api_mu);
    CK(cudaSetDevice(ctx->device));
    if (q == 0)
        return ED_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int r;
    if (method == 2 || method == 7) {
        // one job per query (job id 1, pair 0 of a one-entry pair table)
        if (n >= (1ull << 31) || m >= (1ull << 31))
            return ED_EINVAL;
        if ((r = ensure(ctx, ctx->slots, sizeof(JobSlot) * q)) != ED_OK ||
            (r = ensure(ctx, ctx->pdesc, sizeof(PairDesc))) != ED_OK)
            return r;
        PairDesc pd{};
        pd.A = A;
        pd.B = B;
        pd.n = (int64_t)n;
        pd.m = (int64_t)m;
        CK(cudaMemcpyAsync(ctx->pdesc.p, &pd, sizeof(pd), cudaMemcpyHostToDevice, s));
        const unsigned long long tg = 1ull << 32;
        std::vector<JobSlot> it(q);
        std::vector<int64_t> lim(q);
        for (size_t i = 0; i < q; i++) {
            JobSlot &j = it[i];
            j = JobSlot{};
            lim[i] = std::min<int64_t>((int64_t)n - x[i], (int64_t)m - y[i]);
            j.xt = tg | (uint32_t)x[i];
            j.yt = tg | (uint32_t)y[i];
            j.lt = tg | (uint32_t)lim[i];
            j.pt = tg;
            j.result = tg | (uint32_t)~(uint32_t)lim[i];
            j.claim = tg;
        }
        CK(cudaMemcpyAsync(ctx->slots.p, it.data(), sizeof(JobSlot) * q, cudaMemcpyHostToDevice, s));
        CK(launch_lcp_queries(A, (int64_t)n, B, (int64_t)m, nullptr, nullptr, (int64_t)q, method, nullptr,
                              nullptr, (JobSlot *)ctx->slots.p, (const PairDesc *)ctx->pdesc.p, ctx->grid, s));
        CK(cudaMemcpyAsync(it.data(), ctx->slots.p, sizeof(JobSlot) * q, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (size_t i = 0; i < q; i++)
            out[i] = std::min<int64_t>(lim[i], (int64_t)(uint32_t)~(uint32_t)it[i].result);
        return ED_OK;
    }
    if ((r = ensure(ctx, ctx->qx, 8 * q)) != ED_OK || (r = ensure(ctx, ctx->qy, 8 * q)) != ED_OK ||
        (r = ensure(ctx, ctx->qo, 8 * q)) != ED_OK)
        return r;
    CK(cudaMemcpyAsync(ctx->qx.p, x, 8 * q, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->qy.p, y, 8 * q, cudaMemcpyHostToDevice, s));
    HashArgs H{};
    H.TA = TA;
    H.TB = TB;
    // methods 5, 6: 3, 4 on blocked tables with the context's block size
    H.b = method >= 5 ? ctx->cfg.hash_block : 1;
    std::memcpy(H.pow2, ctx->pow2, sizeof(H.pow2));
    CK(launch_lcp_queries(A, (int64_t)n, B, (int64_t)m, (const int64_t *)ctx->qx.p, (const int64_t *)ctx->qy.p,
                          (int64_t)q, method >= 5 ? method - 2 : method, &H, (int64_t *)ctx->qo.p, nullptr,
                          nullptr, ctx->grid, s));
    CK(cudaMemcpyAsync(out, ctx->qo.p, 8 * q, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return ED_OK;
}

// ------------------------------------------------------------------ batch
static int batch_launch(ed_ctx *ctx, std::vector<BatchPair> &hp, const std::vector<int32_t> &order,
                        DevBuf &dpairs, DevBuf &dorder, DevBuf &dnext, cudaStream_t s, uint64_t budget_ns)
{
    const size_t np = hp.size();
    int r;
    if ((r = ensure(ctx, dpairs, sizeof(BatchPair) * np)) != ED_OK ||
        (r = ensure(ctx, dorder, sizeof(int32_t) * np)) != ED_OK || (r = ensure(ctx, dnext, 64)) != ED_OK)
        return r;
    CK(cudaMemcpyAsync(dpairs.p, hp.data(), sizeof(BatchPair) * np, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dorder.p, order.data(), sizeof(int32_t) * np, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(dnext.p, 0, 64, s));
    BatchArgs Bg{};
    Bg.pairs = (BatchPair *)dpairs.p;
    Bg.order = (const int32_t *)dorder.p;
    Bg.npairs = (int32_t)np;
    Bg.W = BATCH_W;
    Bg.round_budget = 0;
    Bg.next = (uint32_t *)dnext.p;
    Bg.t2_cap = 8192;
    Bg.spin_ns = ctx->cfg.spin_limit_ns;
    const int occ = lv_batch_ctas_per_sm(BATCH_W);
    CK(cudaEventRecord(ctx->ev0, s));
    CK(launch_lv_batch(Bg, ctx->num_sms * occ, s, budget_ns));
    CK(cudaEventRecord(ctx->ev1, s));
    CK(cudaMemcpyAsync(hp.data(), dpairs.p, sizeof(BatchPair) * np, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    ctx->last.kernel_ms += ms;
    ctx->last.kernel_launches += 1;
    for (size_t i = 0; i < np; i++)
        if (hp[i].state == 3) {
            char buf[200];
            std::snprintf(buf, sizeof(buf), "batch self-check: pair %zu round %lld diagonal %lld start row %lld", i,
                          (long long)hp[i].check[0], (long long)hp[i].check[1], (long long)hp[i].check[2]);
            ctx->last_err = buf;
            return ED_ECUDA;
        }
    return ED_OK;
}

// A tile job for a pair parked by the batch kernel after t rounds with its
// furthest row at `reach`.  Its distance is estimated by extrapolating the
// rounds per row so far (t * n / reach, between t and max(n, m)); its group
// is the smallest power of two of CTAs whose tiles hold that band with a
// quarter to spare.  The estimate only places the pair: one whose band
// outgrows its group runs again on a larger group.
static TileJob parked_job(ed_ctx *ctx, const BatchPair &b)
{
    const int64_t nm = std::max(b.n, b.m);
    const int64_t t = std::max<int64_t>(b.t, 1);
    int64_t kest = b.reach > 0 ? (int64_t)((double)t * (double)b.n / (double)b.reach) : nm;
    kest = std::min(std::max(kest, t), nm);
    TileJob j{b.A, b.B, b.n, b.m, nullptr, nullptr, nullptr, 0, 1, (double)kest};
    const int64_t band = std::min<int64_t>(2 * (kest + kest / 4) + 1, b.n + b.m + 1);
    while (j.G < ctx->grid && (int64_t)j.G * SMAX_LIMIT < band)
        j.G *= 2;
    j.G = std::min(j.G, ctx->grid);
    return j;
}

// While the groups the jobs ask for fill at most half of the grid, doubles
// them: with few pairs, more CTAs per pair shorten each round; a single job
// takes the whole grid.  The cost of a job (for sharing CTAs among classes)
// is its estimated distance times the round time, which grows with the band
// per CTA.
static void spread_jobs(ed_ctx *ctx, std::vector<TileJob> &jobs)
{
    if (jobs.size() == 1)
        jobs[0].G = ctx->grid;
    for (;;) {
        int64_t sum = 0;
        bool room = false;
        for (const TileJob &j : jobs) {
            sum += j.G;
            room |= j.G < ctx->grid;
        }
        if (!room || 2 * sum > ctx->grid)
            break;
        for (TileJob &j : jobs)
            j.G = std::min(ctx->grid, 2 * j.G);
    }
    for (TileJob &j : jobs) {
        const double band = std::min(2.0 * j.cost + 1.0, (double)(j.n + j.m + 1));
        j.cost = j.cost * (1.0 + band / ((double)j.G * 4096.0));
    }
}

static int batch_core(ed_ctx *ctx, size_t np, const uint8_t *const *A, const size_t *n,
                      const uint8_t *const *B, const size_t *m, uint64_t *k_out, cudaStream_t s)
{
    int r;
    const size_t fb = sizeof(int32_t) * (BATCH_W + 3);
    if ((r = ensure(ctx, ctx->bfront, fb * np)) != ED_OK)
        return r;
    std::vector<BatchPair> hp(np);
    std::vector<int32_t> order(np);
    for (size_t p = 0; p < np; p++) {
        BatchPair &b = hp[p];
        b = BatchPair{};
        b.A = A[p];
        b.B = B[p];
        b.n = (int64_t)n[p];
        b.m = (int64_t)m[p];
        b.front = (int32_t *)((char *)ctx->bfront.p + fb * p);
        b.t = -1;
        b.k = -1;
        order[p] = (int32_t)p;
    }
    // longest-processing-time first: longer pairs are claimed first
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return std::max(n[a], m[a]) > std::max(n[b], m[b]); });
    if ((r = batch_launch(ctx, hp, order, ctx->bpairs, ctx->border, ctx->bnext, s, 0)) != ED_OK)
        return r;
    const double batch_ms = ctx->last.kernel_ms;
    uint64_t ext = 0, slide = 0, mism = 0;
    std::vector<size_t> parked;
    for (size_t p = 0; p < np; p++) {
        const BatchPair &b = hp[p];
        if (b.state == 1) {
            k_out[p] = (uint64_t)b.k;
            ext += count_extensions(b.n, b.m, b.k);
            slide += b.slide;
            mism += b.mism;
        } else {
            parked.push_back(p);
        }
    }
    ed_stats keep = ctx->last;
    if (!parked.empty()) {
        // pairs whose band outgrew one CTA: CTA groups of the tile kernel,
        // sized by each pair's estimated distance, in one launch
        std::vector<TileJob> jobs;
        for (size_t p : parked)
            jobs.push_back(parked_job(ctx, hp[p]));
        spread_jobs(ctx, jobs);
        ctx->last = ed_stats{};
        std::vector<uint64_t> kk;
        if ((r = run_tiles(ctx, jobs, s, kk)) != ED_OK)
            return r;
        for (size_t i = 0; i < parked.size(); i++)
            k_out[parked[i]] = kk[i];
        ext += ctx->last.extensions;
        slide += ctx->last.slide_chars;
        mism += ctx->last.compared_bytes / 2 - ctx->last.slide_chars;
        keep.kernel_ms += ctx->last.kernel_ms;
        keep.kernel_launches += ctx->last.kernel_launches;
        keep.long_slides += ctx->last.long_slides;
        keep.open_slides += ctx->last.open_slides;
        keep.wide_rounds += ctx->last.wide_rounds;
    }
    ctx->last = keep;
    ctx->last.extensions = ext;
    ctx->last.slide_chars = slide;
    ctx->last.compared_bytes = 2 * (slide + mism);
    ctx->last.phase_ms[5] = batch_ms;
    return ED_OK;
}

int ed_distance_batch_dev(ed_ctx *ctx, size_t np, const uint8_t *const *A, const size_t *n,
                          const uint8_t *const *B, const size_t *m, uint64_t *k_out, void *stream)
{
    if (!ctx || (np && (!A || !B || !n || !m || !k_out)))
        return ED_EINVAL;
    for (size_t p = 0; p < np; p++)
        if ((n[p] && !A[p]) || (m[p] && !B[p]) || bad_len(n[p]) || bad_len(m[p]))
            return ED_EINVAL;
    std::lock_guard<std::mutex> g(ctx->api_mu);
    CK(cudaSetDevice(ctx->device));
    ctx->last = ed_stats{};
    resolve(ctx, 0, 0, false);
    if (np == 0)
        return ED_OK;
    return batch_core(ctx, np, A, n, B, m, k_out, (cudaStream_t)stream);
}

int ed_distance_batch(ed_ctx *ctx, size_t np, const uint8_t *const *A, const size_t *n,
                      const uint8_t *const *B, const size_t *m, uint64_t *k_out)
{
    if (!ctx || (np && (!A || !B || !n || !m || !k_out)))
        return ED_EINVAL;
    size_t total = 0;
    for (size_t p = 0; p < np; p++) {
        if ((n[p] && !A[p]) || (m[p] && !B[p]) || bad_len(n[p]) || bad_len(m[p]))
            return ED_EINVAL;
        total += ((n[p] + 15) & ~(size_t)15) + ((m[p] + 15) & ~(size_t)15);
    }
    std::lock_guard<std::mutex> g(ctx->api_mu);
    CK(cudaSetDevice(ctx->device));
    ctx->last = ed_stats{};
    resolve(ctx, 0, 0, false);
    if (np == 0)
        return ED_OK;
    int r;
    if ((r = ensure(ctx, ctx->strA, total + 64)) != ED_OK)
        return r;
    std::vector<const uint8_t *> dA(np), dB(np);
    size_t off = 0;
    for (size_t p = 0; p < np; p++) {
        char *base = (char *)ctx->strA.p;
        dA[p] = (const uint8_t *)(base + off);
        if (n[p])
            CK(cudaMemcpyAsync(base + off, A[p], n[p], cudaMemcpyHostToDevice, ctx->stream));
        off += (n[p] + 15) & ~(size_t)15;
        dB[p] = (const uint8_t *)(base + off);
        if (m[p])
            CK(cudaMemcpyAsync(base + off, B[p], m[p], cudaMemcpyHostToDevice, ctx->stream));
        off += (m[p] + 15) & ~(size_t)15;
    }
    return batch_core(ctx, np, dA.data(), n, dB.data(), m, k_out, ctx->stream);
}

// ------------------------------------------------------------------ serving
// Device time per engine step: the batch kernel (pairs within one CTA's
// band), then the tile kernel (pairs whose band outgrew it).
constexpr uint64_t SERVE_BATCH_NS = 2000000;
constexpr uint64_t SERVE_TILE_NS = 4000000;

static void release_request(ed_ctx *ctx, Request *q)
{
    if (!q->caller_strings) {
        ctx->arena.release(q->dA, q->bytesA);
        ctx->arena.release(q->dB, q->bytesB);
    }
    ctx->arena.release(q->front, q->bytesF);
    ctx->arena.release(q->keep, q->bytesK);
    if (q->ready)
        cudaEventDestroy(q->ready);
    q->ready = nullptr;
}

// Moves a request to the tile kernel on a group of G CTAs, with a resident
// frontier as wide as the whole grid's tiles (so that the pair can change
// groups between steps; none if the arena is full: the pair then runs to
// its end in one launch).
static void to_tiles(ed_ctx *ctx, Request *q, int G)
{
    ctx->arena.release(q->keep, q->bytesK);
    q->tile_G = G;
    q->keep_r = std::min<int64_t>(std::max(q->n, q->m), (int64_t)ctx->grid * SMAX_LIMIT);
    q->bytesK = sizeof(int32_t) * (size_t)(2 * q->keep_r + 5);
    q->keep = ctx->arena.alloc(q->bytesK);
    q->t0 = 0;
    q->R0 = 0;
}

// One engine step: the live pairs not yet on the tile kernel get up to
// SERVE_BATCH_NS in one launch of the batch kernel (frontiers resident in
// the arena); those whose band outgrew a CTA move to the tile kernel, where
// every such pair gets up to SERVE_TILE_NS per step and its band frontier
// stays resident between steps.
static void engine_loop(ed_ctx *ctx)
{
    cudaSetDevice(ctx->device);
    std::vector<BatchPair> hp;
    std::vector<int32_t> order;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(ctx->smu);
            while (!ctx->stop && ctx->pending.empty() && ctx->live.empty())
                ctx->scv.wait_for(lk, std::chrono::milliseconds(50));
            if (ctx->stop)
                break;
            while (!ctx->pending.empty()) {
                Request *q = ctx->pending.front();
                // device strings of the caller: the engine's stream waits for
                // the work the caller queued before submitting them
                if (q->ready)
                    cudaStreamWaitEvent(ctx->sstream, q->ready, 0);
                ctx->live.push_back(q);
                ctx->pending.pop_front();
            }
        }
        std::unique_lock<std::mutex> api(ctx->api_mu);
        resolve(ctx, 0, 0, false);
        const size_t L = ctx->live.size();
        std::vector<int64_t> result(L, 0);
        std::vector<char> done(L, 0);
        // (1) the batch kernel
        std::vector<size_t> bidx;
        for (size_t i = 0; i < L; i++)
            if (!ctx->live[i]->tile_G)
                bidx.push_back(i);
        hp.resize(bidx.size());
        order.resize(bidx.size());
        for (size_t j = 0; j < bidx.size(); j++) {
            Request *q = ctx->live[bidx[j]];
            BatchPair &b = hp[j];
            b = BatchPair{};
            b.A = (const uint8_t *)q->dA;
            b.B = (const uint8_t *)q->dB;
            b.n = q->n;
            b.m = q->m;
            b.front = (int32_t *)q->front;
            b.t = q->t;
            b.k = -1;
            order[j] = (int32_t)j;
        }
        if (!bidx.empty()) {
            const uint64_t grid = (uint64_t)ctx->num_sms * lv_batch_ctas_per_sm(BATCH_W);
            std::rotate(order.begin(), order.begin() + (ctx->n_steps * grid) % bidx.size(), order.end());
            const int rc = batch_launch(ctx, hp, order, ctx->s_pairs, ctx->s_order, ctx->s_next, ctx->sstream,
                                        SERVE_BATCH_NS);
            for (size_t j = 0; j < bidx.size(); j++) {
                Request *q = ctx->live[bidx[j]];
                const BatchPair &b = hp[j];
                if (rc != ED_OK) {
                    result[bidx[j]] = rc;
                    done[bidx[j]] = 1;
                } else if (b.state == 1) {
                    result[bidx[j]] = b.k;
                    done[bidx[j]] = 1;
                } else if (b.state == 2) {
                    // group from the distance estimate, doubled while the
                    // tile pairs would fill at most half of the grid
                    // the group its estimated band needs; each step spreads
                    // the groups over the grid
                    const TileJob pj = parked_job(ctx, b);
                    q->cost = pj.cost;
                    to_tiles(ctx, q, pj.G);
                } else {
                    q->t = b.t;
                }
            }
        }
        ctx->n_steps++;
        // (2) the tile kernel, time-sliced
        std::vector<size_t> tidx;
        std::vector<TileJob> jobs;
        for (size_t i = 0; i < L; i++) {
            Request *q = ctx->live[i];
            if (!q->tile_G || done[i])
                continue;
            TileJob j{(const uint8_t *)q->dA, (const uint8_t *)q->dB, q->n, q->m, nullptr, nullptr, nullptr, 0,
                      q->tile_G, q->cost};
            j.keep = (int32_t *)q->keep;
            j.keep_r = q->keep ? q->keep_r : 0;
            j.t0 = q->keep ? q->t0 : 0;
            j.R0 = q->R0;
            tidx.push_back(i);
            jobs.push_back(j);
        }
        if (!jobs.empty()) {
            // each pair's group at least what its band needs (tile_G), all of
            // them spread over the grid (a single pair takes all of it: its
            // resident frontier holds any group's band)
            if (std::all_of(jobs.begin(), jobs.end(), [](const TileJob &j) { return j.keep != nullptr; }))
                spread_jobs(ctx, jobs);
            std::vector<TileOut> o;
            const int rt = run_tiles_once(ctx, jobs, ctx->sstream, SERVE_TILE_NS, o);
            for (size_t j = 0; j < tidx.size(); j++) {
                Request *q = ctx->live[tidx[j]];
                if (rt != ED_OK) {
                    result[tidx[j]] = rt;
                    done[tidx[j]] = 1;
                } else if (o[j].st == 0) {
                    result[tidx[j]] = (int64_t)o[j].k;
                    done[tidx[j]] = 1;
                } else if (o[j].st == ST_SUSPENDED) {
                    q->t0 = o[j].rt;
                    q->R0 = o[j].rr;
                    ctx->n_slices++;
                } else if (o[j].st == ST_WIDE && q->keep && o[j].rt > 0 && jobs[j].G < ctx->grid) {
                    // a larger group from the saved round
                    q->tile_G = std::min(ctx->grid, 2 * jobs[j].G);
                    q->t0 = o[j].rt;
                    q->R0 = o[j].rr;
                } else if (o[j].st == ST_WIDE && q->tile_G < ctx->grid) {
                    to_tiles(ctx, q, std::min(ctx->grid, 2 * q->tile_G)); // again, from round 0
                } else {
                    result[tidx[j]] = ED_ELIMIT;
                    done[tidx[j]] = 1;
                }
            }
        }
        api.unlock();
        std::vector<Request *> still;
        for (size_t i = 0; i < L; i++) {
            Request *q = ctx->live[i];
            if (done[i]) {
                release_request(ctx, q);
                std::lock_guard<std::mutex> lk(ctx->smu);
                ctx->results[q->ticket] = result[i];
                ctx->n_completed++;
                delete q;
            } else {
                still.push_back(q);
            }
        }
        std::lock_guard<std::mutex> lk(ctx->smu);
        ctx->live.swap(still);
    }
}

static int engine_start(ed_ctx *ctx)
{
    // checked before the lock too: the engine holds api_mu through each
    // step, and submitters must not queue behind it once it runs
    if (ctx->engine_on.load(std::memory_order_acquire))
        return ED_OK;
    std::lock_guard<std::mutex> g(ctx->api_mu);
    if (ctx->engine_on)
        return ED_OK;
    CK(cudaSetDevice(ctx->device));
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    size_t want = std::min(ctx->budget > ctx->held ? (ctx->budget - ctx->held) / 2 : 0, fr / 2);
    want = std::max<size_t>(want, 64ull << 20);
    int r = ensure(ctx, ctx->arena_buf, want);
    if (r != ED_OK)
        return r;
    ctx->arena.init((char *)ctx->arena_buf.p, ctx->arena_buf.bytes);
    CK(cudaStreamCreateWithFlags(&ctx->sstream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&ctx->cstream, cudaStreamNonBlocking));
    ctx->stop = false;
    ctx->engine = std::thread(engine_loop, ctx);
    ctx->engine_on = true;
    return ED_OK;
}

static void engine_stop(ed_ctx *ctx)
{
    if (!ctx->engine_on)
        return;
    {
        std::lock_guard<std::mutex> lk(ctx->smu);
        ctx->stop = true;
    }
    ctx->scv.notify_all();
    ctx->engine.join();
    ctx->engine_on = false;
    for (Request *q : ctx->live) {
        if (q->ready)
            cudaEventDestroy(q->ready);
        delete q;
    }
    for (Request *q : ctx->pending) {
        if (q->ready)
            cudaEventDestroy(q->ready);
        delete q;
    }
    ctx->live.clear();
    ctx->pending.clear();
    if (ctx->sstream)
        cudaStreamDestroy(ctx->sstream);
    if (ctx->cstream)
        cudaStreamDestroy(ctx->cstream);
    ctx->sstream = ctx->cstream = nullptr;
}

int ed_submit(ed_ctx *ctx, const uint8_t *A, size_t n, const uint8_t *B, size_t m, uint64_t *ticket)
{
    if (!ctx || !ticket || (n && !A) || (m && !B) || bad_len(n) || bad_len(m))
        return ED_EINVAL;
    int r = engine_start(ctx);
    if (r != ED_OK)
        return r;
    {
        std::lock_guard<std::mutex> lk(ctx->smu);
        if (ctx->live.size() + ctx->pending.size() >= (size_t)ctx->cfg.max_inflight)
            return ED_EBUSY;
    }
    Request *q = new Request();
    q->n = (int64_t)n;
    q->m = (int64_t)m;
    q->bytesA = n + 64;
    q->bytesB = m + 64;
    q->bytesF = sizeof(int32_t) * (BATCH_W + 3);
    q->dA = ctx->arena.alloc(q->bytesA);
    q->dB = q->dA ? ctx->arena.alloc(q->bytesB) : nullptr;
    q->front = q->dB ? ctx->arena.alloc(q->bytesF) : nullptr;
    if (!q->front) {
        ctx->arena.release(q->dA, q->bytesA);
        ctx->arena.release(q->dB, q->bytesB);
        delete q;
        return ED_EBUSY;
    }
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaSuccess;
    if (n)
        e = cudaMemcpyAsync(q->dA, A, n, cudaMemcpyHostToDevice, ctx->cstream);
    if (e == cudaSuccess && m)
        e = cudaMemcpyAsync(q->dB, B, m, cudaMemcpyHostToDevice, ctx->cstream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(ctx->cstream);
    if (e != cudaSuccess) {
        ctx->arena.release(q->dA, q->bytesA);
        ctx->arena.release(q->dB, q->bytesB);
        ctx->arena.release(q->front, q->bytesF);
        delete q;
        return cuda_fail(ctx, e, "ed_submit copy");
    }
    {
        std::lock_guard<std::mutex> lk(ctx->smu);
        q->ticket = ctx->next_ticket++;
        ctx->known[q->ticket] = true;
        ctx->pending.push_back(q);
        ctx->n_admitted++;
        *ticket = q->ticket;
    }
    ctx->scv.notify_all();
    return ED_OK;
}

int ed_submit_dev(ed_ctx *ctx, const uint8_t *A, size_t n, const uint8_t *B, size_t m, uint64_t *ticket,
                  void *stream)
{
    if (!ctx || !ticket || (n && !A) || (m && !B) || bad_len(n) || bad_len(m))
        return ED_EINVAL;
    int r = engine_start(ctx);
    if (r != ED_OK)
        return r;
    {
        std::lock_guard<std::mutex> lk(ctx->smu);
        if (ctx->live.size() + ctx->pending.size() >= (size_t)ctx->cfg.max_inflight)
            return ED_EBUSY;
    }
    Request *q = new Request();
    q->n = (int64_t)n;
    q->m = (int64_t)m;
    q->caller_strings = true;
    q->dA = (char *)A;
    q->dB = (char *)B;
    q->bytesF = sizeof(int32_t) * (BATCH_W + 3);
    q->front = ctx->arena.alloc(q->bytesF);
    if (!q->front) {
        delete q;
        return ED_EBUSY;
    }
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaEventCreateWithFlags(&q->ready, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventRecord(q->ready, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        release_request(ctx, q);
        delete q;
        return cuda_fail(ctx, e, "ed_submit_dev event");
    }
    {
        std::lock_guard<std::mutex> lk(ctx->smu);
        q->ticket = ctx->next_ticket++;
        ctx->known[q->ticket] = true;
        ctx->pending.push_back(q);
        ctx->n_admitted++;
        *ticket = q->ticket;
    }
    ctx->scv.notify_all();
    return ED_OK;
}

int ed_poll(ed_ctx *ctx, uint64_t ticket, uint64_t *k)
{
    if (!ctx || !k)
        return ED_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->smu);
    auto it = ctx->results.find(ticket);
    if (it == ctx->results.end())
        return ctx->known.count(ticket) ? ED_EAGAIN : ED_ENOTFOUND;
    const int64_t v = it->second;
    ctx->results.erase(it);
    ctx->known.erase(ticket);
    if (v < 0)
        return (int)v;
    *k = (uint64_t)v;
    return ED_OK;
}

int ed_serve_counters(ed_ctx *ctx, uint64_t *admitted, uint64_t *completed, uint64_t *inflight,
                      uint64_t *steps, uint64_t *slices)
{
    if (!ctx)
        return ED_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->smu);
    if (admitted)
        *admitted = ctx->n_admitted;
    if (completed)
        *completed = ctx->n_completed;
    if (inflight)
        *inflight = ctx->live.size() + ctx->pending.size();
    if (steps)
        *steps = ctx->n_steps;
    if (slices)
        *slices = ctx->n_slices;
    return ED_OK;
}

} // extern "C"
