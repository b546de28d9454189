// muca_api.cu -- host runtime behind include/muca.h.  It owns the context,
// lays out the device arena, turns every C call into kernel launches on the
// context's stream, and maps CUDA errors onto MUCA_ERR_* codes with a
// thread-local message.  No compute happens on the host.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "muca.h"
#include "muca_internal.h"

using namespace muca;

namespace {

// NVTX range for the duration of a C call (visible in profilers; free otherwise).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define MUCA_CUDA(expr)                                                                         \
    do {                                                                                        \
        cudaError_t e_ = (expr);                                                                \
        if (e_ != cudaSuccess) return fail(MUCA_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

constexpr size_t kAlign = 256;
constexpr size_t kMaxSmem = 227u * 1024u;  // dynamic shared memory a block can have
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
    size_t lat, bin, T, lnW, lnW_sampled, G, lnR, H, Hpart, rlist, reach, state, out, Eq, lnWq, obs, metrics, tun, total;
};

}  // namespace

struct muca_ctx {
    int system = 0, L = 0, q = 2, p = 0, N = 0, B = 0, C = 0, nreach = 0;
    uint64_t seed = 0;
    double beta = 0.0, flat_ratio = 0.5;
    int record = 0, block = 64, walker_offset = 0;
    bool block_small_p = false;  // q-Potts: 32 walkers a block because every block has an SM to itself
    int lanes = 0;     // polymer: lanes per walker in the sweep (8, 16, 32; 0 = chosen by N)
    int model = 0;     // polymer: 0 benchmark parameters, 1 the paper's (Eq. 7)
    int moves = 0;     // polymer: 0 single-bead shifts, 1 shifts and spherical rotations
    int debug_drop_row = -1;  // test hook for the bounded waits (next spin iterate only)
    int spin_limit = 0;       // tries of one bounded hand-over wait (0: the kernels' default)
    int debug_check = 0;      // checked build: every table bounds check of the next iterate fails
    int recursion = 0;        // weight update: 0 accumulated statistics, 1 plain W/H
    int flush_cap = 0;        // spins: most sweeps between histogram flushes (0: the counters' own bound)
    PolyTraceRec *trace = nullptr;  // polymer: attempt records of the next iterate (device), or null
    int64_t trace_n = 0;            // records the trace buffer holds
    int observables = 0;      // Ising: per-sweep sums of 1, |M|, M^2 per bin
    unsigned long long *obs = nullptr;  // [0, 3B): sums being filled, [3B, 6B): of the last update
    unsigned long long *metrics = nullptr;  // kMetricWords counters, see UpdateArgs::metrics
    uint8_t *tun = nullptr;                 // [p] tunnelling state per walker
    int pipeline = 2;  // spins: code form (2), producer/consumer (1) or one warp per walker group (0)
    int pstride = 0, wpw = 0, nblk_max = 0;
    cudaStream_t stream = nullptr;
    bool owns_arena = false, started = false;
    bool open = false;  // sweeps since the last merge (their partial histograms sit in Hpart)
    void *arena = nullptr;
    size_t arena_bytes = 0;
    uint32_t *lat = nullptr;
    int32_t *bin = nullptr;
    uint32_t *T = nullptr;
    double *lnW = nullptr, *lnW_sampled = nullptr, *G = nullptr, *lnR = nullptr;
    unsigned long long *H = nullptr, *Hpart = nullptr;
    int32_t *rlist = nullptr;
    uint8_t *reach = nullptr;
    DevState *state = nullptr;
    double *out = nullptr;  // reweight outputs: 4 + B doubles
    // polymer: energies and ln W in fixed point, window and FENE parameters
    long long *Eq = nullptr, *lnWq = nullptr;
    double e_lo = 0.0, e_hi = 0.0, fene_K = 40.0, fene_R = 1.5;
    int bin_k = 10;            // polymer: bins per unit energy (width 1 / bin_k)
    long long step_q = kPolyStepQ;  // polymer: move grid units per unit of (u - 2^31) (cube side step_q / 4096)
    std::vector<uint8_t> h_reach;
    std::vector<int32_t> h_rlist;
};

namespace {

bool valid_config(int system, int L, int q, int p, std::string &why)
{
    if (p < 1) { why = "p must be >= 1"; return false; }
    if (system == kPolymer) {
        if (!polymer_supported(L)) { why = "polymer bead count must be in [2, 128]"; return false; }
        return true;
    }
    if (system != kIsing && system != kPotts && system != kMuma) { why = "unknown system"; return false; }
    if (system == kPotts && (q < 2 || q > 16)) { why = "Potts q must be in [2, 16]"; return false; }
    if (!spin_sweep_supported(system, L)) {
        why = "lattice size not supported (L in {4,8,12,16,24,32,48,64})";
        return false;
    }
    return true;
}

// Polymer bins of width 1 / k over [e_lo, e_hi).
int polymer_bins(double e_lo, double e_hi, int k) { return (int)((e_hi - e_lo) * (double)k + 0.5); }

void fill_shape(muca_ctx *c, int system, int L, int q, int p)
{
    if (system == kPolymer) {
        c->system = system;
        c->L = L;
        c->N = L;  // beads
        c->q = 0;
        c->p = p;
        c->e_lo = 2.0 * L;  // default window; set "e_lo"/"e_hi" for the run's own
        c->e_hi = 6.0 * L;
        c->B = polymer_bins(c->e_lo, c->e_hi, c->bin_k);
        c->C = 0;
        c->pstride = p;
        c->wpw = 0;
        c->nblk_max = 1;
        c->block = 256;
        return;
    }
    c->system = system;
    c->L = L;
    c->q = (system == kPotts) ? q : 2;
    c->p = p;
    c->N = L * L;
    c->B = (system == kPotts) ? 2 * c->N + 1 : c->N + 1;
    c->C = num_cols(system);
    c->pstride = (p + 31) / 32 * 32;
    c->wpw = words_per_walker(system, L);
    c->nblk_max = (p + 31) / 32;  // smallest allowed block is one warp
    // default walkers per block: 64, or 32 where only that fits the code form (e.g. q = 10 Potts,
    // L = 48, whose threshold table alone takes 184 KB of shared memory)
    if (!spin_sweep_tn_fits(system, L, c->B, 64) && spin_sweep_tn_fits(system, L, c->B, 32)) c->block = 32;
    // without the code form, the global-table Potts form (L = 64) hides more of its L2 latency
    // with four warps a block
    if (system == kPotts && L == 64 && !spin_sweep_tn_fits(system, L, c->B, 32)) c->block = 128;
}

// Reachable bins of the periodic L x L lattice (L even): the Ising model has
// no state with exactly 2 or 2N-2 broken bonds; the q >= 3 Potts model none
// with 1, 2, 3 or 5; the q = 2 Potts model follows Ising (even counts only);
// every magnetisation is reachable.
void reachable_bins(muca_ctx *c)
{
    const int N = c->N, B = c->B;
    c->h_reach.assign(B, 1);
    if (c->system == kPolymer) {
        // every bin of the window
    } else if (c->system == kIsing) {
        c->h_reach[1] = 0;
        c->h_reach[N - 1] = 0;
    } else if (c->system == kPotts) {
        if (c->q == 2) {
            for (int b = 0; b < B; ++b)
                if ((b & 1) || b == 2 || b == 2 * N - 2) c->h_reach[b] = 0;
        } else {
            for (int b : {1, 2, 3, 5}) c->h_reach[b] = 0;
        }
    }
    c->h_rlist.clear();
    for (int b = 0; b < B; ++b)
        if (c->h_reach[b]) c->h_rlist.push_back(b);
    c->nreach = (int)c->h_rlist.size();
}

Layout plan(const muca_ctx *c)
{
    Layout l{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align_up(bytes);
        return o;
    };
    if (c->system == kPolymer) {
        const size_t Bc = kPolyMaxBins;
        l.lat = take(sizeof(long long) * 3 * (size_t)c->N * c->p);
        l.bin = take(sizeof(int32_t) * (size_t)c->p);
        l.Eq = take(sizeof(long long) * (size_t)c->p);
        l.T = take(0);
        l.lnW = take(sizeof(double) * Bc);
        l.lnW_sampled = take(sizeof(double) * Bc);
        l.G = take(sizeof(double) * Bc);
        l.lnR = take(sizeof(double) * Bc);
        l.H = take(sizeof(unsigned long long) * Bc);
        l.Hpart = take(sizeof(unsigned long long) * Bc);
        l.lnWq = take(sizeof(long long) * Bc);
        l.rlist = take(sizeof(int32_t) * Bc);
        l.reach = take(Bc);
        l.state = take(sizeof(DevState));
        l.out = take(sizeof(double) * (4 + Bc));
        l.metrics = take(sizeof(unsigned long long) * kMetricWords);
        l.tun = take((size_t)c->p);
        l.total = off;
        return l;
    }
    l.lat = take(sizeof(uint32_t) * (size_t)c->wpw * c->pstride);
    l.bin = take(sizeof(int32_t) * (size_t)c->pstride);
    l.T = take(sizeof(uint32_t) * (size_t)c->B * c->C);
    l.lnW = take(sizeof(double) * c->B);
    l.lnW_sampled = take(sizeof(double) * c->B);
    l.G = take(sizeof(double) * c->B);
    l.lnR = take(sizeof(double) * c->B);
    l.H = take(sizeof(unsigned long long) * c->B);
    l.Hpart = take(sizeof(unsigned long long) * (size_t)c->nblk_max * c->B);
    l.rlist = take(sizeof(int32_t) * c->B);
    l.reach = take((size_t)c->B);
    l.state = take(sizeof(DevState));
    l.out = take(sizeof(double) * (4 + (size_t)c->B));
    l.obs = take(sizeof(unsigned long long) * 6 * (size_t)c->B);
    l.metrics = take(sizeof(unsigned long long) * kMetricWords);
    l.tun = take((size_t)c->p);
    l.total = off;
    return l;
}

UpdateArgs update_args(const muca_ctx *c)
{
    UpdateArgs a{};
    a.system = c->system;
    a.B = c->B;
    a.nreach = c->nreach;
    a.nblocks = (c->p + c->block - 1) / c->block;
    a.N = c->N;
    a.q = c->q;
    a.p = c->p;
    a.pstride = c->pstride;
    a.L = c->L;
    a.beta = c->beta;
    a.flat_ratio = c->flat_ratio;
    a.e_lo = c->e_lo;
    a.bin_w = 1.0 / (double)c->bin_k;
    a.recursion = c->recursion;
    a.metrics = c->metrics;
    if (c->system == kPolymer) a.nblocks = 1;  // the open histogram is one global slot
    a.reach = c->reach;
    a.rlist = c->rlist;
    a.Hpart = c->Hpart;
    a.H = c->H;
    a.lnW = c->lnW;
    a.lnW_sampled = c->lnW_sampled;
    a.G = c->G;
    a.lnR = c->lnR;
    a.T = c->T;
    a.state = c->state;
    return a;
}

// Arguments of a spin sweep launch of `sweeps` sweeps with `block` walkers a block.
SpinSweepArgs sweep_args(const muca_ctx *c, int64_t sweeps, int block)
{
    SpinSweepArgs a{};
    a.T = c->T;
    a.lattice = c->lat;
    a.bin = c->bin;
    a.Hpart = c->Hpart;
    a.state = c->state;
    a.p = c->p;
    a.pstride = c->pstride;
    a.B = c->B;
    a.q = c->q;
    a.sweeps = sweeps;
    const unsigned long long per_sweep = (unsigned long long)block * (c->record == 0 ? (unsigned)c->N : 1u);
    unsigned long long fe = 0xFFFFFFFFull / per_sweep;
    if (fe < 1) fe = 1;
    if (c->flush_cap > 0 && fe > (unsigned long long)c->flush_cap) fe = (unsigned long long)c->flush_cap;
    if (fe > (unsigned long long)sweeps) fe = (unsigned long long)sweeps;
    a.flush_every = (int)(fe > 0x7fffffffull ? 0x7fffffffull : fe);
    fill_round_keys(a, c->seed);
    a.record = c->record;
    a.walker_offset = c->walker_offset;
    a.kind = sweep_kind(c->system, c->L);
    a.metrics = c->metrics;
    a.tun = c->tun;
    a.bin_lo = c->h_rlist.front();
    a.bin_hi = c->h_rlist.back();
    a.spin_limit = c->spin_limit;
    a.debug_check = c->debug_check;
    return a;
}

// The context's sweep in its configured form (code form, producer/consumer or one warp), falling
// back to the next lower form where one does not fit the system, L, bin count or block.
cudaError_t launch_system_sweep(const muca_ctx *c, const SpinSweepArgs &a, cudaStream_t s, int block = 0)
{
    if (block <= 0) block = c->block;
    if (c->pipeline >= 2 && spin_sweep_tn_fits(c->system, c->L, c->B, block))
        return launch_spin_sweep_tn(c->system, c->L, a, block, s);
    if (c->pipeline >= 1 && spin_sweep_pc_fits(c->system, c->L, c->B, block))
        return launch_spin_sweep_pc(c->system, c->L, a, block, s);
    return launch_spin_sweep(c->system, c->L, a, block, s);
}

PolyArgs poly_args(const muca_ctx *c, int64_t sweeps)
{
    PolyArgs a{};
    a.X = (long long *)c->lat;
    a.E = c->Eq;
    a.bin = c->bin;
    a.lnWq = c->lnWq;
    a.H = c->Hpart;
    a.state = c->state;
    a.p = c->p;
    a.N = c->N;
    a.B = c->B;
    a.record = c->record;
    a.walker_offset = c->walker_offset;
    a.lanes = c->lanes;
    a.flush_every = c->flush_cap;
    a.bin_k = c->bin_k;
    a.step_q = (int)c->step_q;
    a.elo_q = llrint(c->e_lo * 4294967296.0);                                          // e_lo * 2^32
    a.ehi_q = a.elo_q + ((long long)c->B * 4294967296LL + c->bin_k - 1) / c->bin_k;  // first energy with bin >= B
    a.model = c->model;
    a.moves = c->moves;
    if (c->model == 1) {  // the paper's parameters of Eq. 7: K = 40, r0 = 0.7, r_max = 1, no LJ cutoff
        const double K = 40.0, r0 = 0.7, R = 0.3;
        a.fene_KR2_half = (float)(0.5 * K * R * R);
        a.fene_invR2 = (float)(1.0 / (R * R));
        a.fene_r0 = (float)r0;
        a.fene_invR = (float)(1.0 / R);
        a.lj_sigma2 = (float)(r0 * r0 * std::pow(2.0, -1.0 / 3.0));
        a.lj_rc2 = INFINITY;
        a.lj_shift = 0.0f;
        a.init_bond = r0;
        a.init_d2min = 0.3969;  // (0.9 r0)^2
    } else {
        a.fene_KR2_half = (float)(0.5 * c->fene_K * c->fene_R * c->fene_R);
        a.fene_invR2 = (float)(1.0 / (c->fene_R * c->fene_R));
        a.fene_r0 = 0.0f;
        a.fene_invR = (float)(1.0 / c->fene_R);
        a.lj_sigma2 = 1.0f;
        a.lj_rc2 = 6.25f;
        const double irc6 = 1.0 / (6.25 * 6.25 * 6.25);
        a.lj_shift = (float)(4.0 * (irc6 * irc6 - irc6));
        a.init_bond = 1.0;
        a.init_d2min = 0.81;  // (0.9 b0)^2
    }
    a.sweeps = sweeps;
    a.metrics = c->metrics;
    a.tun = c->tun;
    SpinSweepArgs keys{};
    fill_round_keys(keys, c->seed);
    a.key0 = keys.key0;
    a.key1 = keys.key1;
    for (int i = 0; i < 20; ++i) a.rk[i] = keys.rk[i];
    return a;
}

// Upload the reachable list and reset the weights; for the polymer also
// recompute every walker's energy and bin for the current window.
int reset_weights(muca_ctx *c)
{
    reachable_bins(c);
    MUCA_CUDA(cudaMemcpyAsync(c->reach, c->h_reach.data(), c->B, cudaMemcpyHostToDevice, c->stream));
    MUCA_CUDA(cudaMemcpyAsync(c->rlist, c->h_rlist.data(), sizeof(int32_t) * c->nreach, cudaMemcpyHostToDevice,
                              c->stream));
    UpdateArgs a = update_args(c);
    MUCA_CUDA(launch_init_lnW(a, c->stream));
    if (c->system == kPolymer) {
        PolyArgs pa = poly_args(c, 0);
        MUCA_CUDA(launch_poly_energy(pa, 0, c->stream));
        MUCA_CUDA(launch_poly_lnwq(c->lnW, c->lnWq, c->B, c->stream));
    } else {
        MUCA_CUDA(launch_thresholds(a, c->stream));
    }
    MUCA_CUDA(cudaStreamSynchronize(c->stream));
    return MUCA_OK;
}

int init_walkers(muca_ctx *c)
{
    // new walkers: no tunnelling history, no counts
    MUCA_CUDA(cudaMemsetAsync(c->tun, 0, (size_t)c->p, c->stream));
    MUCA_CUDA(cudaMemsetAsync(c->metrics, 0, sizeof(unsigned long long) * kMetricWords, c->stream));
    if (c->system == kPolymer) {
        PolyArgs pa = poly_args(c, 0);
        MUCA_CUDA(launch_poly_init(pa, c->stream));
        MUCA_CUDA(launch_poly_energy(pa, 0, c->stream));
        return MUCA_OK;
    }
    MUCA_CUDA(launch_init_spins(c->system, c->L, c->q, c->p, c->pstride, (uint32_t)(c->seed & 0xffffffffu),
                                (uint32_t)(c->seed >> 32), c->walker_offset, c->lat, c->bin, c->stream));
    return MUCA_OK;
}

int setup(muca_ctx *c)
{
    Layout l = plan(c);
    char *base = (char *)c->arena;
    c->lat = (uint32_t *)(base + l.lat);
    c->bin = (int32_t *)(base + l.bin);
    c->T = (uint32_t *)(base + l.T);
    c->lnW = (double *)(base + l.lnW);
    c->lnW_sampled = (double *)(base + l.lnW_sampled);
    c->G = (double *)(base + l.G);
    c->lnR = (double *)(base + l.lnR);
    c->H = (unsigned long long *)(base + l.H);
    c->Hpart = (unsigned long long *)(base + l.Hpart);
    c->rlist = (int32_t *)(base + l.rlist);
    c->reach = (uint8_t *)(base + l.reach);
    c->state = (DevState *)(base + l.state);
    c->out = (double *)(base + l.out);
    c->metrics = (unsigned long long *)(base + l.metrics);
    c->tun = (uint8_t *)(base + l.tun);
    if (c->system == kPolymer) {
        c->Eq = (long long *)(base + l.Eq);
        c->lnWq = (long long *)(base + l.lnWq);
    } else {
        c->obs = (unsigned long long *)(base + l.obs);
    }
    MUCA_CUDA(cudaMemsetAsync(c->arena, 0, l.total, c->stream));
    int rc = init_walkers(c);
    if (rc) return rc;
    return reset_weights(c);
}

int create(muca_ctx **out, int system, int L, int q, int p, uint64_t seed, void *arena, size_t arena_bytes)
{
    if (!out) return fail(MUCA_ERR_ARG, "out is NULL");
    *out = nullptr;
    std::string why;
    if (!valid_config(system, L, q, p, why)) return fail(MUCA_ERR_ARG, "muca_init: %s", why.c_str());
    muca_ctx *c = new (std::nothrow) muca_ctx();
    if (!c) return fail(MUCA_ERR_OOM, "host allocation failed");
    fill_shape(c, system, L, q, p);
    // q-Potts with few walkers: when every 32-walker block has an SM to itself, one consumer warp
    // an SM decides faster than two (measured at p = 2048: 71 against 92 cycles an attempt at
    // L = 16, 60 against 72 at L = 32)
    if (system == kPotts && c->block == 64 && spin_sweep_tn_fits(system, L, c->B, 32)) {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && (p + 31) / 32 <= nsm) {
            c->block = 32;
            c->block_small_p = true;
        }
    }
    c->seed = seed;
    if (const char *env = std::getenv("MUCA_SPIN_LIMIT")) {  // bound of the hand-over waits
        const long v = std::strtol(env, nullptr, 10);
        if (v > 0 && v <= 0x7fffffffL) c->spin_limit = (int)v;
    }
    const size_t need = plan(c).total;
    if (arena) {
        if (arena_bytes < need || ((uintptr_t)arena % kAlign) != 0) {
            delete c;
            return fail(MUCA_ERR_OOM, "arena too small or misaligned: need %zu bytes, 256-byte aligned", need);
        }
        c->arena = arena;
        c->arena_bytes = arena_bytes;
        c->owns_arena = false;
    } else {
        cudaError_t e = cudaMalloc(&c->arena, need);
        if (e != cudaSuccess) {
            delete c;
            return fail(MUCA_ERR_OOM, "cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
        }
        c->arena_bytes = need;
        c->owns_arena = true;
    }
    int rc = setup(c);
    if (rc) {
        if (c->owns_arena) cudaFree(c->arena);
        delete c;
        return rc;
    }
    *out = c;
    return MUCA_OK;
}

int check_ctx(const muca_ctx *c)
{
    if (!c) return fail(MUCA_ERR_ARG, "context is NULL");
    return MUCA_OK;
}

// Device-side checks (bounded waits) leave a flag in the device state; every
// call that synchronises reports it.
int check_device_flag(muca_ctx *c)
{
    int err = 0;
    MUCA_CUDA(cudaMemcpyAsync(&err, &c->state->err, sizeof err, cudaMemcpyDeviceToHost, c->stream));
    MUCA_CUDA(cudaStreamSynchronize(c->stream));
    if (err & 2) return fail(MUCA_ERR_CHECK, "a device bounds check failed (checked build); the last iterations are invalid");
    if (err) return fail(MUCA_ERR_TIMEOUT, "a bounded device wait gave up; the last iterations are invalid");
    return MUCA_OK;
}

int d2h(muca_ctx *c, void *host, const void *dev, size_t bytes)
{
    MUCA_CUDA(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, c->stream));
    MUCA_CUDA(cudaStreamSynchronize(c->stream));
    return check_device_flag(c);
}

// Checkpoint blob: fixed header, then the device sections in this order.
struct StateHeader {
    char magic[8];
    int32_t version, system, L, q, p, B, C, wpw, pstride, record, walker_offset, model, bin_k, pad;
    uint64_t seed;
    int64_t step_q;
    double beta, e_lo, e_hi, fene_K, fene_R;
    DevState dev;
};

// Device sections of a checkpoint, in order: walkers, bins, [polymer energies],
// ln W, ln W sampled, G, lnR, merged H, open histogram, thresholds / ln W fixed point.
struct Section {
    void *dev;
    size_t bytes;
};

// A spin state read from a buffer must be one the sweeps can run: every Potts colour below q,
// no bits past the last site of a row, and each walker's bin equal to the bin of its lattice
// (the sweeps move the bin by each accepted move's change, so a bin that disagrees with its
// lattice could walk off the shared-memory tables).  `lat` is the lattice section, unaligned.
bool spin_state_consistent(const muca_ctx *c, const char *lat, const char *bins, std::string &why)
{
    const int L = c->L, N = c->N, bits = (c->system == kPotts) ? 4 : 1;
    const int WR = (c->system == kPotts) ? potts_words_per_row(L) : ising_words_per_row(L);
    std::vector<uint32_t> rows((size_t)L * WR);
    std::vector<uint8_t> col((size_t)N);  // Potts colours
    std::vector<uint64_t> r64((size_t)L);  // Ising / MUMA rows (L <= 64 bits)
    const uint64_t mask = (L == 64) ? ~0ull : ((1ull << L) - 1ull);
    for (int w = 0; w < c->p; ++w) {
        for (int k = 0; k < L * WR; ++k)
            memcpy(&rows[k], lat + ((size_t)k * c->pstride + w) * sizeof(uint32_t), sizeof(uint32_t));
        for (int y = 0; y < L; ++y)
            for (int j = 0; j < WR; ++j) {
                const int used = std::min(32, L * bits - 32 * j);  // bits of sites in word j
                if (used < 32 && (rows[(size_t)y * WR + j] >> used) != 0u) {
                    why = "walker " + std::to_string(w) + ": bits past the last site of a row";
                    return false;
                }
            }
        int want;
        if (c->system == kPotts) {
            for (int i = 0; i < N; ++i) {
                const int y = i / L, x = i - y * L;
                const uint32_t v = (rows[(size_t)y * WR + (4 * x) / 32] >> ((4 * x) & 31)) & 15u;
                if (v >= (uint32_t)c->q) {
                    why = "walker " + std::to_string(w) + ": colour " + std::to_string(v) + " >= q";
                    return false;
                }
                col[i] = (uint8_t)v;
            }
            int E = 0;
            for (int y = 0; y < L; ++y) {
                const uint8_t *r = &col[(size_t)y * L], *d = &col[(size_t)((y + 1) % L) * L];
                for (int x = 0; x < L; ++x) E -= (r[x] == r[(x + 1) % L]) + (r[x] == d[x]);
            }
            want = E + 2 * N;
        } else {  // bit 1 = spin -1; a bond is broken where the bits differ
            int broken = 0, minus = 0;
            for (int y = 0; y < L; ++y)
                r64[y] = rows[(size_t)y * WR] | (WR > 1 ? (uint64_t)rows[(size_t)y * WR + 1] << 32 : 0ull);
            for (int y = 0; y < L; ++y) {
                const uint64_t r = r64[y], right = ((r >> 1) | (r << (L - 1))) & mask;  // bit x: site x+1
                broken += __builtin_popcountll(r ^ right) + __builtin_popcountll(r ^ r64[(y + 1) % L]);
                minus += __builtin_popcountll(r);
            }
            want = (c->system == kIsing) ? broken / 2 : N - minus;  // (E + 2N) / 4 with E = 2 broken - 2N
        }
        int32_t b;
        memcpy(&b, bins + (size_t)w * sizeof(int32_t), sizeof b);
        if (b != want) {
            why = "walker " + std::to_string(w) + " has bin " + std::to_string(b) + ", its lattice bin " +
                  std::to_string(want);
            return false;
        }
    }
    return true;
}

std::vector<Section> state_sections(const muca_ctx *c)
{
    std::vector<Section> v;
    const size_t B = (size_t)c->B;
    if (c->system == kPolymer) {
        v.push_back({c->lat, sizeof(long long) * 3 * (size_t)c->N * c->p});
        v.push_back({c->bin, sizeof(int32_t) * (size_t)c->p});
        v.push_back({c->Eq, sizeof(long long) * (size_t)c->p});
    } else {
        v.push_back({c->lat, sizeof(uint32_t) * (size_t)c->wpw * c->pstride});
        v.push_back({c->bin, sizeof(int32_t) * (size_t)c->p});
    }
    v.push_back({c->lnW, sizeof(double) * B});
    v.push_back({c->lnW_sampled, sizeof(double) * B});
    v.push_back({c->G, sizeof(double) * B});
    v.push_back({c->lnR, sizeof(double) * B});
    v.push_back({c->H, sizeof(unsigned long long) * B});
    v.push_back({nullptr, sizeof(unsigned long long) * B});  // open histogram (summed over block slots)
    if (c->system == kPolymer) {
        v.push_back({c->lnWq, sizeof(long long) * B});
    } else {
        v.push_back({c->T, sizeof(uint32_t) * B * c->C});
        v.push_back({c->obs, sizeof(unsigned long long) * 6 * B});  // observable sums (open, last)
    }
    v.push_back({c->metrics, sizeof(unsigned long long) * kMetricWords});  // metrics counters
    v.push_back({c->tun, (size_t)c->p});                                    // tunnelling states
    return v;
}

size_t state_bytes(const muca_ctx *c)
{
    size_t n = sizeof(StateHeader);
    for (const Section &s : state_sections(c)) n += s.bytes;
    return n;
}

}  // namespace

extern "C" {

const char *muca_last_error(void) { return g_err.c_str(); }

int muca_workspace_size(int system, int L_or_N, int q, int p, size_t *bytes)
{
    if (!bytes) return fail(MUCA_ERR_ARG, "bytes is NULL");
    std::string why;
    if (!valid_config(system, L_or_N, q, p, why)) return fail(MUCA_ERR_ARG, "muca_workspace_size: %s", why.c_str());
    muca_ctx c;
    fill_shape(&c, system, L_or_N, q, p);
    *bytes = plan(&c).total;
    return MUCA_OK;
}

int muca_init(muca_ctx **out, int system, int L_or_N, int q, int p, uint64_t seed)
{
    return create(out, system, L_or_N, q, p, seed, nullptr, 0);
}

int muca_init_ex(muca_ctx **out, int system, int L_or_N, int q, int p, uint64_t seed, void *device_arena,
                 size_t arena_bytes)
{
    if (!device_arena) return fail(MUCA_ERR_ARG, "device_arena is NULL");
    return create(out, system, L_or_N, q, p, seed, device_arena, arena_bytes);
}

int muca_set_param(muca_ctx *c, const char *key, double v)
{
    if (int rc = check_ctx(c)) return rc;
    if (!key) return fail(MUCA_ERR_ARG, "key is NULL");
    const std::string k(key);
    if (k == "flat_ratio") {
        if (!(v > 0.0 && v <= 1.0)) return fail(MUCA_ERR_ARG, "flat_ratio must be in (0, 1]");
        c->flat_ratio = v;
        return MUCA_OK;
    }
    const bool locked = c->started;
    if (k == "beta") {
        if (locked) return fail(MUCA_ERR_STATE, "beta must be set before the first iterate");
        if (!(v == v) || v < 0.0) return fail(MUCA_ERR_ARG, "beta must be >= 0");
        c->beta = v;
        if (c->system == kPolymer) return MUCA_OK;  // reweighting only
        UpdateArgs a = update_args(c);
        MUCA_CUDA(launch_thresholds(a, c->stream));
        return MUCA_OK;
    }
    if (k == "e_lo" || k == "e_hi" || k == "fene_K" || k == "fene_R" || k == "bin_width") {
        if (c->system != kPolymer) return fail(MUCA_ERR_ARG, "'%s' applies to the polymer only", key);
        if (locked) return fail(MUCA_ERR_STATE, "%s must be set before the first iterate", key);
        if (!(v == v) || v > 1e6 || v < -1e6) return fail(MUCA_ERR_ARG, "bad value for %s", key);
        double lo = c->e_lo, hi = c->e_hi, K = c->fene_K, R = c->fene_R;
        int bk = c->bin_k;
        if (k == "e_lo") lo = v;
        if (k == "e_hi") hi = v;
        if (k == "fene_K") K = v;
        if (k == "fene_R") R = v;
        if (k == "bin_width") {  // 1 / k for a whole k, so that a bin is an exact fixed-point product
            const double kk = (v > 0.0) ? std::nearbyint(1.0 / v) : 0.0;
            if (!(kk >= 1.0 && kk <= 1000.0) || std::fabs(1.0 / kk - v) > 1e-12 * v)
                return fail(MUCA_ERR_ARG, "bin_width must be 1/k for a whole k in 1..1000");
            bk = (int)kk;
        }
        if (!(K > 0.0) || !(R > 0.0)) return fail(MUCA_ERR_ARG, "fene_K and fene_R must be > 0");
        const int B = (hi > lo) ? polymer_bins(lo, hi, bk) : 0;
        if (B < 2 || B > kPolyMaxBins)
            return fail(MUCA_ERR_RANGE, "window [%g, %g) gives %d bins of 1/%d; need 2..%d", lo, hi, B, bk, kPolyMaxBins);
        c->e_lo = lo;
        c->e_hi = hi;
        c->fene_K = K;
        c->fene_R = R;
        c->bin_k = bk;
        c->B = B;
        return reset_weights(c);
    }
    if (k == "step") {  // the side of the move cube, on the grid: step_q = round(side * 4096)
        if (c->system != kPolymer) return fail(MUCA_ERR_ARG, "'step' applies to the polymer only");
        if (locked) return fail(MUCA_ERR_STATE, "step must be set before the first iterate");
        const double q = std::nearbyint(v * 4096.0);
        if (!(q >= 1.0 && q <= 8192.0)) return fail(MUCA_ERR_ARG, "step must be in [1/4096, 2]");
        c->step_q = (long long)q;
        return MUCA_OK;
    }
    if (k == "record") {
        if (locked) return fail(MUCA_ERR_STATE, "record must be set before the first iterate");
        if (v != 0.0 && v != 1.0) return fail(MUCA_ERR_ARG, "record must be 0 or 1");
        c->record = (int)v;
        return MUCA_OK;
    }
    if (k == "block") {
        if (locked) return fail(MUCA_ERR_STATE, "block must be set before the first iterate");
        const int b = (int)v;
        if ((double)b != v || b < 32 || b > kMaxSweepBlock || (b % 32) != 0)
            return fail(MUCA_ERR_ARG, "block must be a multiple of 32 in [32, %d]", kMaxSweepBlock);
        c->block = b;
        c->block_small_p = false;
        return MUCA_OK;
    }
    if (k == "debug_check") {
#ifdef MUCA_CHECKED
        if (v != 0.0 && v != 1.0) return fail(MUCA_ERR_ARG, "debug_check must be 0 or 1");
        c->debug_check = (int)v;
        return MUCA_OK;
#else
        return fail(MUCA_ERR_ARG, "debug_check needs the checked build (MUCA_DEBUG=1)");
#endif
    }
    if (k == "spin_limit") {
        const long long lim = (long long)v;
        if ((double)lim != v || lim < 0 || lim > 0x7fffffffLL)
            return fail(MUCA_ERR_ARG, "spin_limit must be an integer in [0, 2^31)");
        c->spin_limit = (int)lim;
        return MUCA_OK;
    }
    if (k == "flush_every") {
        const long long n = (long long)v;
        if ((double)n != v || n < 0 || n > 0x7fffffffLL) return fail(MUCA_ERR_ARG, "flush_every must be an integer >= 0");
        c->flush_cap = (int)n;
        return MUCA_OK;
    }
    if (k == "pipeline") {
        if (v != 0.0 && v != 1.0 && v != 2.0) return fail(MUCA_ERR_ARG, "pipeline must be 0, 1 or 2");
        c->pipeline = (int)v;
        return MUCA_OK;
    }
    if (k == "observables") {
        if (c->system != kIsing) return fail(MUCA_ERR_ARG, "observables are recorded for the Ising system only");
        if (locked) return fail(MUCA_ERR_STATE, "observables must be set before the first iterate");
        if (v != 0.0 && v != 1.0) return fail(MUCA_ERR_ARG, "observables must be 0 or 1");
        c->observables = (int)v;
        return MUCA_OK;
    }
    if (k == "recursion") {
        if (c->system == kPolymer) return fail(MUCA_ERR_ARG, "recursion applies to lattice systems only");
        if (locked) return fail(MUCA_ERR_STATE, "recursion must be set before the first iterate");
        if (v != 0.0 && v != 1.0) return fail(MUCA_ERR_ARG, "recursion must be 0 or 1");
        c->recursion = (int)v;
        return MUCA_OK;
    }
    if (k == "debug_drop_row") {
        if (c->system == kPolymer) return fail(MUCA_ERR_ARG, "debug_drop_row applies to lattice systems only");
        const long long r = (long long)v;
        if ((double)r != v || r < 0 || r > 0x7fffffffLL) return fail(MUCA_ERR_ARG, "debug_drop_row must be >= 0");
        c->debug_drop_row = (int)r;
        return MUCA_OK;
    }
    if (k == "moves") {
        if (c->system != kPolymer) return fail(MUCA_ERR_ARG, "moves applies to the polymer only");
        if (locked) return fail(MUCA_ERR_STATE, "moves must be set before the first iterate");
        if (v != 0.0 && v != 1.0) return fail(MUCA_ERR_ARG, "moves must be 0 or 1");
        c->moves = (int)v;
        return MUCA_OK;
    }
    if (k == "model") {
        if (c->system != kPolymer) return fail(MUCA_ERR_ARG, "model applies to the polymer only");
        if (locked) return fail(MUCA_ERR_STATE, "model must be set before the first iterate");
        if (v != 0.0 && v != 1.0) return fail(MUCA_ERR_ARG, "model must be 0 or 1");
        c->model = (int)v;
        if (int rc = init_walkers(c)) return rc;  // the initial chains depend on the bond length
        return reset_weights(c);
    }
    if (k == "lanes") {
        if (c->system != kPolymer) return fail(MUCA_ERR_ARG, "lanes applies to the polymer only");
        if (v != 0.0 && v != 1.0 && v != 2.0 && v != 4.0 && v != 8.0 && v != 16.0 && v != 32.0)
            return fail(MUCA_ERR_ARG, "lanes must be 0, 1, 2, 4, 8, 16 or 32");
        c->lanes = (int)v;
        return MUCA_OK;
    }
    if (k == "walker_offset") {
        if (locked) return fail(MUCA_ERR_STATE, "walker_offset must be set before the first iterate");
        const long long o = (long long)v;
        if ((double)o != v || o < 0 || o + c->p > 0x7fffffffLL) return fail(MUCA_ERR_ARG, "bad walker_offset");
        c->walker_offset = (int)o;
        if (int rc = init_walkers(c)) return rc;
        return c->system == kPolymer ? reset_weights(c) : MUCA_OK;
    }
    return fail(MUCA_ERR_ARG, "unknown parameter '%s'", key);
}

int muca_set_stream(muca_ctx *c, void *stream)
{
    if (int rc = check_ctx(c)) return rc;
    MUCA_CUDA(cudaStreamSynchronize(c->stream));
    c->stream = (cudaStream_t)stream;
    return MUCA_OK;
}

int muca_iterate(muca_ctx *c, int64_t sweeps)
{
    NvtxRange nvtx("muca_iterate");
    if (int rc = check_ctx(c)) return rc;
    if (sweeps < 1) return fail(MUCA_ERR_ARG, "sweeps must be >= 1");
    if (c->system == kPolymer) {
        if (sweeps > 0x7fffffffLL / c->N) return fail(MUCA_ERR_RANGE, "too many sweeps in one call");
        PolyArgs pa = poly_args(c, sweeps);
        if (c->trace) {  // one-shot: this iterate only
            const int64_t need = (int64_t)c->p * sweeps * c->N;
            pa.trace = c->trace;
            c->trace = nullptr;
            if (c->trace_n < need)
                return fail(MUCA_ERR_ARG, "trace buffer holds %lld records; this iterate makes %lld",
                            (long long)c->trace_n, (long long)need);
        }
        MUCA_CUDA(launch_poly_sweep(pa, c->block, c->stream));
        MUCA_CUDA(launch_advance(c->state, sweeps, c->stream));
        // refresh the running energies from scratch; the largest change is recorded
        MUCA_CUDA(launch_poly_energy(pa, 1, c->stream));
        c->started = true;
        c->open = true;
        return MUCA_OK;
    }
    SpinSweepArgs a = sweep_args(c, sweeps, c->block);
    a.obs = (c->observables && c->system == kIsing) ? c->obs : nullptr;
    a.debug_drop_row = c->debug_drop_row;
    c->debug_drop_row = -1;
    MUCA_CUDA(launch_system_sweep(c, a, c->stream));
    MUCA_CUDA(launch_advance(c->state, sweeps, c->stream));
    c->started = true;
    c->open = true;
    return MUCA_OK;
}

int muca_merge_and_update(muca_ctx *c, int *is_flat)
{
    NvtxRange nvtx("muca_merge_and_update");
    if (int rc = check_ctx(c)) return rc;
    UpdateArgs a = update_args(c);
    MUCA_CUDA(launch_merge(a, c->stream));
    MUCA_CUDA(launch_recursion(a, c->stream));
    if (c->system == kPolymer) {
        MUCA_CUDA(launch_poly_lnwq(c->lnW, c->lnWq, c->B, c->stream));
    } else {
        MUCA_CUDA(launch_thresholds(a, c->stream));
        if (c->observables) {  // the sums just filled belong to the weights of this update
            const size_t bytes = sizeof(unsigned long long) * 3 * (size_t)c->B;
            MUCA_CUDA(cudaMemcpyAsync(c->obs + 3 * (size_t)c->B, c->obs, bytes, cudaMemcpyDeviceToDevice, c->stream));
            MUCA_CUDA(cudaMemsetAsync(c->obs, 0, bytes, c->stream));
        }
    }
    c->started = true;
    c->open = false;
    if (is_flat) {
        int f = 0;
        if (int rc = d2h(c, &f, &c->state->flat, sizeof(int))) return rc;
        *is_flat = f;
    }
    return MUCA_OK;
}

int muca_merge_open(muca_ctx *c, uint64_t *dev_H_out)
{
    NvtxRange nvtx("muca_merge_open");
    if (int rc = check_ctx(c)) return rc;
    if (!dev_H_out) return fail(MUCA_ERR_ARG, "dev_H_out is NULL");
    UpdateArgs a = update_args(c);
    a.H = (unsigned long long *)dev_H_out;  // block slots summed (and cleared) into the caller's buffer
    MUCA_CUDA(launch_merge(a, c->stream));
    return MUCA_OK;
}

int muca_update_with(muca_ctx *c, const uint64_t *dev_H, int *is_flat)
{
    NvtxRange nvtx("muca_update_with");
    if (int rc = check_ctx(c)) return rc;
    if (!dev_H) return fail(MUCA_ERR_ARG, "dev_H is NULL");
    MUCA_CUDA(cudaMemcpyAsync(c->H, dev_H, sizeof(unsigned long long) * c->B, cudaMemcpyDeviceToDevice, c->stream));
    UpdateArgs a = update_args(c);
    MUCA_CUDA(launch_recursion(a, c->stream));
    if (c->system == kPolymer) {
        MUCA_CUDA(launch_poly_lnwq(c->lnW, c->lnWq, c->B, c->stream));
    } else {
        MUCA_CUDA(launch_thresholds(a, c->stream));
        if (c->observables) {  // this shard's own sums (observables are not exchanged)
            const size_t bytes = sizeof(unsigned long long) * 3 * (size_t)c->B;
            MUCA_CUDA(cudaMemcpyAsync(c->obs + 3 * (size_t)c->B, c->obs, bytes, cudaMemcpyDeviceToDevice, c->stream));
            MUCA_CUDA(cudaMemsetAsync(c->obs, 0, bytes, c->stream));
        }
    }
    c->started = true;
    c->open = false;
    if (is_flat) {
        int f = 0;
        if (int rc = d2h(c, &f, &c->state->flat, sizeof(int))) return rc;
        *is_flat = f;
    }
    return MUCA_OK;
}

int muca_set_lnW(muca_ctx *c, const double *host_lnW, int nbins)
{
    if (int rc = check_ctx(c)) return rc;
    if (!host_lnW || nbins != c->B) return fail(MUCA_ERR_ARG, "need a host buffer of %d doubles", c->B);
    std::vector<double> v(host_lnW, host_lnW + c->B);
    for (int b = 0; b < c->B; ++b) {
        if (!c->h_reach[b]) {
            v[b] = -INFINITY;  // unreachable bins keep ln W = -inf
        } else if (!(std::fabs(v[b]) <= 1e300)) {
            return fail(MUCA_ERR_ARG, "ln W of reachable bin %d is not finite", b);
        }
    }
    MUCA_CUDA(cudaMemcpyAsync(c->lnW, v.data(), sizeof(double) * c->B, cudaMemcpyHostToDevice, c->stream));
    if (c->system == kPolymer) {
        MUCA_CUDA(launch_poly_lnwq(c->lnW, c->lnWq, c->B, c->stream));
    } else {
        UpdateArgs a = update_args(c);
        MUCA_CUDA(launch_thresholds(a, c->stream));
    }
    MUCA_CUDA(cudaStreamSynchronize(c->stream));  // the host buffer may go away after the call
    return MUCA_OK;
}

int muca_poly_trace(muca_ctx *c, void *dev_records, int64_t n_records)
{
    if (int rc = check_ctx(c)) return rc;
    if (c->system != kPolymer) return fail(MUCA_ERR_ARG, "muca_poly_trace: polymer contexts only");
    if (!dev_records || n_records < 1) return fail(MUCA_ERR_ARG, "muca_poly_trace: need a device buffer");
    if (((uintptr_t)dev_records % 16) != 0) return fail(MUCA_ERR_ARG, "muca_poly_trace: buffer not 16-byte aligned");
    c->trace = (PolyTraceRec *)dev_records;
    c->trace_n = n_records;
    return MUCA_OK;
}

int muca_num_bins(const muca_ctx *c, int *nbins)
{
    if (int rc = check_ctx(c)) return rc;
    if (!nbins) return fail(MUCA_ERR_ARG, "nbins is NULL");
    *nbins = c->B;
    return MUCA_OK;
}

int muca_get_lnW(muca_ctx *c, double *host_out, int nbins)
{
    if (int rc = check_ctx(c)) return rc;
    if (!host_out || nbins != c->B) return fail(MUCA_ERR_ARG, "need a host buffer of %d doubles", c->B);
    return d2h(c, host_out, c->lnW, sizeof(double) * c->B);
}

int muca_get_lnW_sampled(muca_ctx *c, double *host_out, int nbins)
{
    if (int rc = check_ctx(c)) return rc;
    if (!host_out || nbins != c->B) return fail(MUCA_ERR_ARG, "need a host buffer of %d doubles", c->B);
    return d2h(c, host_out, c->lnW_sampled, sizeof(double) * c->B);
}

int muca_get_histogram(muca_ctx *c, uint64_t *host_out, int nbins)
{
    if (int rc = check_ctx(c)) return rc;
    if (!host_out || nbins != c->B) return fail(MUCA_ERR_ARG, "need a host buffer of %d uint64", c->B);
    return d2h(c, host_out, c->H, sizeof(uint64_t) * c->B);
}

int muca_get_flatness(muca_ctx *c, double host_stats[3])
{
    if (int rc = check_ctx(c)) return rc;
    if (!host_stats) return fail(MUCA_ERR_ARG, "stats is NULL");
    DevState st;
    if (int rc = d2h(c, &st, c->state, sizeof st)) return rc;
    host_stats[0] = st.flat_min;
    host_stats[1] = st.flat_mean;
    host_stats[2] = st.flat_max;
    return MUCA_OK;
}

int muca_get_reweight(muca_ctx *c, double beta, double host_out[4], double *host_lnP)
{
    if (int rc = check_ctx(c)) return rc;
    if (!host_out) return fail(MUCA_ERR_ARG, "out is NULL");
    if (!(beta == beta)) return fail(MUCA_ERR_ARG, "beta is NaN");
    UpdateArgs a = update_args(c);
    MUCA_CUDA(launch_reweight(a, beta, c->out, c->out + 4, c->stream));
    if (int rc = d2h(c, host_out, c->out, sizeof(double) * 4)) return rc;
    if (host_lnP) return d2h(c, host_lnP, c->out + 4, sizeof(double) * c->B);
    return MUCA_OK;
}

int muca_get_metrics(muca_ctx *c, uint64_t host_out[6])
{
    if (int rc = check_ctx(c)) return rc;
    if (!host_out) return fail(MUCA_ERR_ARG, "host_out is NULL");
    unsigned long long m[kMetricWords], it = 0;
    MUCA_CUDA(cudaMemcpyAsync(&it, &c->state->iteration, sizeof it, cudaMemcpyDeviceToHost, c->stream));
    if (int rc = d2h(c, m, c->metrics, sizeof m)) return rc;
    for (int k = 0; k < 5; ++k) host_out[k] = m[2 + k];
    host_out[5] = it;
    return MUCA_OK;
}

int muca_get_observables(muca_ctx *c, double beta, double host_out[3], uint64_t *host_sums, int nbins)
{
    if (int rc = check_ctx(c)) return rc;
    if (c->system != kIsing || !c->observables)
        return fail(MUCA_ERR_STATE, "observables are not recorded (set \"observables\" = 1 on an Ising context)");
    if (!host_out) return fail(MUCA_ERR_ARG, "out is NULL");
    if (!(beta == beta)) return fail(MUCA_ERR_ARG, "beta is NaN");
    if (host_sums && nbins != c->B) return fail(MUCA_ERR_ARG, "need a host buffer of 3 x %d uint64", c->B);
    const unsigned long long *last = c->obs + 3 * (size_t)c->B;
    MUCA_CUDA(launch_reweight_obs(last, c->lnW_sampled, c->B, c->N, beta, c->out, c->stream));
    if (int rc = d2h(c, host_out, c->out, sizeof(double) * 3)) return rc;
    if (host_sums) return d2h(c, host_sums, last, sizeof(unsigned long long) * 3 * (size_t)c->B);
    return MUCA_OK;
}

int muca_get_spins(muca_ctx *c, int8_t *host_out, int64_t n)
{
    if (int rc = check_ctx(c)) return rc;
    if (c->system == kPolymer) return fail(MUCA_ERR_ARG, "the polymer has no spins; use muca_get_coords");
    if (!host_out || n != (int64_t)c->p * c->N) return fail(MUCA_ERR_ARG, "need p*L*L = %lld bytes",
                                                              (long long)c->p * c->N);
    int8_t *tmp = nullptr;
    MUCA_CUDA(cudaMalloc(&tmp, (size_t)n));
    cudaError_t e = launch_unpack_spins(c->system, c->L, c->p, c->pstride, c->lat, tmp, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, tmp, (size_t)n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return fail(MUCA_ERR_CUDA, "muca_get_spins: %s", cudaGetErrorString(e));
    return MUCA_OK;
}

int muca_get_walker_bins(muca_ctx *c, int32_t *host_out, int p)
{
    if (int rc = check_ctx(c)) return rc;
    if (!host_out || p != c->p) return fail(MUCA_ERR_ARG, "need a host buffer of p = %d int32", c->p);
    return d2h(c, host_out, c->bin, sizeof(int32_t) * c->p);
}

int muca_get_thresholds(muca_ctx *c, uint32_t *host_out, int64_t n)
{
    if (int rc = check_ctx(c)) return rc;
    if (c->system == kPolymer) return fail(MUCA_ERR_ARG, "the polymer has no threshold table");
    if (!host_out || n != (int64_t)c->B * c->C) return fail(MUCA_ERR_ARG, "need B*C = %lld uint32",
                                                              (long long)c->B * c->C);
    return d2h(c, host_out, c->T, sizeof(uint32_t) * (size_t)n);
}

int muca_get_coords(muca_ctx *c, double *host_coords, int64_t n, double *host_energies, int p)
{
    if (int rc = check_ctx(c)) return rc;
    if (c->system != kPolymer) return fail(MUCA_ERR_ARG, "coordinates exist for the polymer only");
    if (!host_coords || n != (int64_t)c->p * c->N * 3) return fail(MUCA_ERR_ARG, "need p*N*3 = %lld doubles",
                                                                      (long long)c->p * c->N * 3);
    if (host_energies && p != c->p) return fail(MUCA_ERR_ARG, "need p = %d energies", c->p);
    double *tmp = nullptr;
    MUCA_CUDA(cudaMalloc(&tmp, sizeof(double) * ((size_t)n + c->p)));
    PolyArgs pa = poly_args(c, 0);
    cudaError_t e = launch_poly_unpack(pa, tmp, tmp + n, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_coords, tmp, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && host_energies)
        e = cudaMemcpyAsync(host_energies, tmp + n, sizeof(double) * c->p, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return fail(MUCA_ERR_CUDA, "muca_get_coords: %s", cudaGetErrorString(e));
    return MUCA_OK;
}

int muca_get_drift(muca_ctx *c, double *host_out)
{
    if (int rc = check_ctx(c)) return rc;
    if (!host_out) return fail(MUCA_ERR_ARG, "out is NULL");
    DevState st;
    if (int rc = d2h(c, &st, c->state, sizeof st)) return rc;
    *host_out = (double)st.drift_max_q * 0x1p-32;
    return MUCA_OK;
}

int muca_get_sweep_counter(muca_ctx *c, int64_t *host_out)
{
    if (int rc = check_ctx(c)) return rc;
    if (!host_out) return fail(MUCA_ERR_ARG, "out is NULL");
    unsigned long long v = 0;
    if (int rc = d2h(c, &v, &c->state->sweep_counter, sizeof v)) return rc;
    *host_out = (int64_t)v;
    return MUCA_OK;
}

int muca_get_state(muca_ctx *c, void *host_buf, size_t *bytes)
{
    if (int rc = check_ctx(c)) return rc;
    if (!bytes) return fail(MUCA_ERR_ARG, "bytes is NULL");
    const size_t need = state_bytes(c);
    if (!host_buf) {
        *bytes = need;
        return MUCA_OK;
    }
    if (*bytes < need) return fail(MUCA_ERR_ARG, "state buffer too small: need %zu bytes", need);
    char *p = (char *)host_buf;
    StateHeader h{};
    memcpy(h.magic, "MUCAST5", 8);
    h.version = 5;
    h.system = c->system;
    h.L = c->L;
    h.q = c->q;
    h.p = c->p;
    h.B = c->B;
    h.C = c->C;
    h.wpw = c->wpw;
    h.pstride = c->pstride;
    h.record = c->record;
    h.walker_offset = c->walker_offset;
    h.model = c->model;
    h.seed = c->seed;
    h.beta = c->beta;
    h.e_lo = c->e_lo;
    h.e_hi = c->e_hi;
    h.fene_K = c->fene_K;
    h.fene_R = c->fene_R;
    h.bin_k = c->bin_k;
    h.step_q = c->step_q;
    if (int rc = d2h(c, &h.dev, c->state, sizeof h.dev)) return rc;
    memcpy(p, &h, sizeof h);
    p += sizeof h;
    for (const Section &sec : state_sections(c)) {
        if (sec.dev) {
            cudaError_t e = cudaMemcpyAsync(p, sec.dev, sec.bytes, cudaMemcpyDeviceToHost, c->stream);
            if (e != cudaSuccess) return fail(MUCA_ERR_CUDA, "muca_get_state: %s", cudaGetErrorString(e));
        } else {
            // open histogram: sum of the block slots (integer, exact)
            const int slots = (c->system == kPolymer) ? 1 : c->nblk_max;
            std::vector<unsigned long long> part((size_t)slots * c->B), open(c->B, 0ull);
            cudaError_t e = cudaMemcpyAsync(part.data(), c->Hpart, sizeof(unsigned long long) * part.size(),
                                            cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) return fail(MUCA_ERR_CUDA, "muca_get_state: %s", cudaGetErrorString(e));
            for (int k = 0; k < slots; ++k)
                for (int b = 0; b < c->B; ++b) open[b] += part[(size_t)k * c->B + b];
            memcpy(p, open.data(), sec.bytes);
        }
        p += sec.bytes;
    }
    MUCA_CUDA(cudaStreamSynchronize(c->stream));
    *bytes = need;
    return MUCA_OK;
}

int muca_set_state(muca_ctx *c, const void *host_buf, size_t bytes)
{
    if (int rc = check_ctx(c)) return rc;
    if (!host_buf) return fail(MUCA_ERR_ARG, "buffer is NULL");
    if (bytes < sizeof(StateHeader)) return fail(MUCA_ERR_ARG, "not a muca state buffer");
    StateHeader h;
    memcpy(&h, host_buf, sizeof h);
    if (memcmp(h.magic, "MUCAST5", 8) != 0 || h.version != 5) return fail(MUCA_ERR_ARG, "not a muca state buffer");
    if (h.system != c->system || h.L != c->L || h.q != c->q || h.p != c->p || h.C != c->C || h.wpw != c->wpw ||
        h.pstride != c->pstride || h.seed != c->seed)
        return fail(MUCA_ERR_ARG, "state buffer was written by a different configuration");
    if (c->system == kPolymer) {
        if (h.bin_k < 1 || h.bin_k > 1000 || h.step_q < 1 || h.step_q > 8192 || h.B < 2 || h.B > kPolyMaxBins ||
            h.B != polymer_bins(h.e_lo, h.e_hi, h.bin_k))
            return fail(MUCA_ERR_ARG, "state buffer: bad polymer window");
    } else if (h.B != c->B) {
        return fail(MUCA_ERR_ARG, "state buffer was written by a different configuration");
    }
    if (h.record != 0 && h.record != 1) return fail(MUCA_ERR_ARG, "state buffer: bad record mode");
    if (h.model != 0 && h.model != 1) return fail(MUCA_ERR_ARG, "state buffer: bad polymer model");
    const int oldB = c->B;
    c->B = h.B;  // the polymer window travels with the state
    const size_t need = state_bytes(c);
    if (bytes != need) {
        c->B = oldB;
        return fail(MUCA_ERR_ARG, "state size %zu does not match this context (%zu)", bytes, need);
    }
    {
        // every walker's bin indexes shared-memory tables of the sweep kernels: check them here
        const size_t off = sizeof h + state_sections(c)[0].bytes;
        const int32_t *bins = (const int32_t *)((const char *)host_buf + off);
        for (int w = 0; w < c->p; ++w) {
            int32_t b;
            memcpy(&b, bins + w, sizeof b);
            const bool ok = (c->system == kPolymer) ? (b >= -1 && b <= c->B)
                                                    : (b >= 0 && b < c->B && c->h_reach[b]);
            if (!ok) {
                c->B = oldB;
                return fail(MUCA_ERR_ARG, "state buffer: walker %d has bin %d", w, b);
            }
        }
        std::string why;
        if (c->system != kPolymer &&
            !spin_state_consistent(c, (const char *)host_buf + sizeof h, (const char *)bins, why)) {
            c->B = oldB;
            return fail(MUCA_ERR_ARG, "state buffer: %s", why.c_str());
        }
    }
    c->record = h.record;
    c->walker_offset = h.walker_offset;
    c->beta = h.beta;
    c->e_lo = h.e_lo;
    c->e_hi = h.e_hi;
    c->fene_K = h.fene_K;
    c->fene_R = h.fene_R;
    if (c->system == kPolymer) {
        c->bin_k = h.bin_k;
        c->step_q = h.step_q;
    }
    c->model = h.model;
    if (c->system == kPolymer) {
        reachable_bins(c);
        MUCA_CUDA(cudaMemcpyAsync(c->reach, c->h_reach.data(), c->B, cudaMemcpyHostToDevice, c->stream));
        MUCA_CUDA(cudaMemcpyAsync(c->rlist, c->h_rlist.data(), sizeof(int32_t) * c->nreach, cudaMemcpyHostToDevice,
                                  c->stream));
    }
    const int slots = (c->system == kPolymer) ? 1 : c->nblk_max;
    MUCA_CUDA(cudaMemsetAsync(c->Hpart, 0, sizeof(unsigned long long) * (size_t)slots * c->B, c->stream));
    const char *p = (const char *)host_buf + sizeof h;
    bool open_counts = false;  // the buffer carries sweeps not merged yet
    for (const Section &sec : state_sections(c)) {
        void *dst = sec.dev ? sec.dev : (void *)c->Hpart;  // open histogram -> slot 0
        if (!sec.dev)
            for (size_t i = 0; i < sec.bytes && !open_counts; ++i) open_counts = p[i] != 0;
        cudaError_t e = cudaMemcpyAsync(dst, p, sec.bytes, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return fail(MUCA_ERR_CUDA, "muca_set_state: %s", cudaGetErrorString(e));
        p += sec.bytes;
    }
    MUCA_CUDA(cudaMemcpyAsync(c->state, &h.dev, sizeof h.dev, cudaMemcpyHostToDevice, c->stream));
    MUCA_CUDA(cudaStreamSynchronize(c->stream));
    c->started = true;
    c->open = open_counts;
    return MUCA_OK;
}

int muca_det_math(int fn, const double *host_in, double *host_out, int64_t n)
{
    if (fn != 0 && fn != 1) return fail(MUCA_ERR_ARG, "fn must be 0 (exp) or 1 (log)");
    if (n < 0 || (n > 0 && (!host_in || !host_out))) return fail(MUCA_ERR_ARG, "bad buffers");
    if (n == 0) return MUCA_OK;
    double *d = nullptr;
    MUCA_CUDA(cudaMalloc(&d, sizeof(double) * 2 * (size_t)n));
    cudaError_t e = cudaMemcpy(d, host_in, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_det_math(fn, d, d + n, (long long)n, 0);
    if (e == cudaSuccess) e = cudaMemcpy(host_out, d + n, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(MUCA_ERR_CUDA, "muca_det_math: %s", cudaGetErrorString(e));
    return MUCA_OK;
}

int muca_synchronize(muca_ctx *c)
{
    if (int rc = check_ctx(c)) return rc;
    MUCA_CUDA(cudaStreamSynchronize(c->stream));
    return check_device_flag(c);
}

int muca_free(muca_ctx *c)
{
    if (!c) return MUCA_OK;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (c->owns_arena && c->arena) cudaFree(c->arena);
    delete c;
    if (e != cudaSuccess) return fail(MUCA_ERR_CUDA, "muca_free: %s", cudaGetErrorString(e));
    return MUCA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batching: several systems (different models, lattice sizes, walker counts)
// advance together.  One iteration is five launches for the whole batch -- a
// persistent sweep over a tile list (system, first walker), the sweep-counter
// advance, and the merge, recursion and threshold kernels over all systems --
// and muca_batch_run can capture all n_iter iterations as one CUDA graph.
// Small systems alone leave most of the GPU idle (2048 walkers are 64 warps
// for 608 schedulers); in one launch they fill it together.
struct muca_batch {
    std::vector<muca_ctx *> sys;
    int block = 128;
    size_t smem = 0;
    int ntiles = 0, max_bins = 0, max_nreach = 0, max_cells = 0;
    void *dmem = nullptr;
    SpinSweepArgs *d_sys = nullptr;
    int2 *d_tiles = nullptr;
    UpdateArgs *d_upd = nullptr;
    DevState **d_states = nullptr;
    std::vector<SpinSweepArgs> h_sys;
    cudaStream_t ctx_stream = nullptr;  // the systems' stream (may be the legacy default stream)
    cudaStream_t stream = nullptr;      // the batch's own stream (capturable)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t exec = nullptr;
    int g_iter = 0;
    int64_t g_sweeps = 0;
    // form 1: every system's own sweep launch on a stream of its own, forked from and joined
    // back into the batch stream (captured as parallel graph branches)
    int form = 0;  // set to 1 (the default) by muca_batch_create
    std::vector<cudaStream_t> sub;
    std::vector<cudaEvent_t> ev_join;
    cudaEvent_t ev_fork = nullptr;
    std::vector<SpinSweepArgs> h_own;  // form 1: per-system launch arguments
    std::vector<int> order;            // systems, heaviest first (tile order; form 1 launch order)
    bool tiles_fit = true;             // every system's table fits the form-0 kernel's shared memory
    std::vector<int64_t> sw;           // per-system sweeps of an iteration (empty: the run's argument)
    std::vector<int> blk;              // form 1: each system's walkers per block in this batch
    std::vector<int64_t> g_sw;         // per-system sweeps the captured graph was made with
};

namespace {

// Systems heaviest first (sites x sweeps, Potts sites counted 2.5 times), so that their
// blocks or tiles start in the first wave.
std::vector<int> batch_order(const muca_batch *b)
{
    const int n = (int)b->sys.size();
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    auto cost = [&](int i) {  // a polymer bead attempt counted as ~40 spin attempts (its pair terms)
        const muca_ctx *c = b->sys[i];
        const double w = c->system == kPotts ? 2.5 : (c->system == kPolymer ? 40.0 : 1.0);
        return (double)c->N * w * (b->sw.empty() ? 1.0 : (double)b->sw[i]);
    };
    for (int i = 1; i < n; ++i)
        for (int j = i; j > 0 && cost(order[j]) > cost(order[j - 1]); --j) std::swap(order[j], order[j - 1]);
    return order;
}

int batch_enqueue_iteration(muca_batch *b, int64_t sweeps)
{
    const int n = (int)b->sys.size();
    if (b->form == 1) {
        MUCA_CUDA(cudaEventRecord(b->ev_fork, b->stream));
        // heaviest first, so that their blocks take the SMs before the light systems' blocks
        for (int i : b->order) {
            MUCA_CUDA(cudaStreamWaitEvent(b->sub[i], b->ev_fork, 0));
            muca_ctx *c = b->sys[i];
            if (c->system == kPolymer) {  // as muca_iterate: the sweeps, then the energies from scratch
                const PolyArgs pa = poly_args(c, b->h_sys[i].sweeps);
                MUCA_CUDA(launch_poly_sweep(pa, c->block, b->sub[i]));
                MUCA_CUDA(launch_poly_energy(pa, 1, b->sub[i]));
            } else {
                MUCA_CUDA(launch_system_sweep(c, b->h_own[i], b->sub[i], b->blk[i]));
            }
            MUCA_CUDA(cudaEventRecord(b->ev_join[i], b->sub[i]));
        }
        for (int i = 0; i < n; ++i) MUCA_CUDA(cudaStreamWaitEvent(b->stream, b->ev_join[i], 0));
    } else {
        MUCA_CUDA(launch_sweep_batch(b->d_sys, b->d_tiles, b->ntiles, b->block, b->smem, b->stream));
    }
    (void)sweeps;
    MUCA_CUDA(launch_advance_batch(b->d_states, b->d_sys, n, b->stream));
    MUCA_CUDA(launch_merge_batch(b->d_upd, n, b->max_bins, b->stream));
    MUCA_CUDA(launch_recursion_batch(b->d_upd, n, b->max_nreach, b->stream));
    if (b->max_cells > 0)  // (polymers skip it)
        MUCA_CUDA(launch_thresholds_batch(b->d_upd, n, b->max_cells, b->stream));
    for (int i = 0; i < n; ++i)
        if (b->sys[i]->system == kPolymer)
            MUCA_CUDA(launch_poly_lnwq(b->sys[i]->lnW, b->sys[i]->lnWq, b->sys[i]->B, b->stream));
    return MUCA_OK;
}

}  // namespace

extern "C" {

int muca_batch_create(muca_ctx *const *systems, int n, muca_batch **out)
{
    if (!out) return fail(MUCA_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!systems || n < 1) return fail(MUCA_ERR_ARG, "need at least one system");
    for (int i = 0; i < n; ++i) {
        if (!systems[i]) return fail(MUCA_ERR_ARG, "system %d is NULL", i);
        if (systems[i]->stream != systems[0]->stream)
            return fail(MUCA_ERR_ARG, "all systems of a batch must use the same stream");
        if (systems[i]->observables)
            return fail(MUCA_ERR_ARG, "system %d records observables, which batches do not support", i);
        for (int j = 0; j < i; ++j)
            if (systems[j] == systems[i]) return fail(MUCA_ERR_ARG, "system %d appears twice", i);
    }
    muca_batch *b = new (std::nothrow) muca_batch();
    if (!b) return fail(MUCA_ERR_OOM, "host allocation failed");
    b->sys.assign(systems, systems + n);
    b->ctx_stream = systems[0]->stream;
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        if (b->stream) cudaStreamDestroy(b->stream);
        if (b->ev_in) cudaEventDestroy(b->ev_in);
        delete b;
        return fail(MUCA_ERR_CUDA, "muca_batch_create: cannot create stream/events");
    }
    const std::vector<int> order = batch_order(b);
    // Form 1 runs each system in its own block size, except that q-Potts systems given 32-walker
    // blocks because every block would have an SM to itself go back to 64 when the batch's
    // systems together have more such blocks than the GPU has SMs (they share the SMs then).
    {
        int dev = 0, nsm = 0;
        long long blocks32 = 0;
        for (int i = 0; i < n; ++i) blocks32 += (b->sys[i]->p + 31) / 32;
        const bool shared = cudaGetDevice(&dev) == cudaSuccess &&
                            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                            blocks32 > nsm;
        b->blk.resize(n);
        for (int i = 0; i < n; ++i) {
            const muca_ctx *c = b->sys[i];
            b->blk[i] = (shared && c->block_small_p && spin_sweep_tn_fits(c->system, c->L, c->B, 64)) ? 64 : c->block;
        }
    }
    std::vector<int2> tiles;
    std::vector<UpdateArgs> upd(n);
    std::vector<DevState *> states(n);
    for (int i = 0; i < n; ++i) {
        muca_ctx *c = b->sys[i];
        if (c->system == kPolymer) {
            b->tiles_fit = false;  // the tile launch is for lattices: polymers run in form 1
        } else {
            const size_t sm = spin_sweep_smem_bytes(c->system, c->B);
            if (sm <= kMaxSmem) b->smem = std::max(b->smem, sm);
            else b->tiles_fit = false;  // e.g. q-Potts at L = 64: only form 1 runs it
            b->max_cells = std::max(b->max_cells, c->B * c->C);
        }
        b->max_bins = std::max(b->max_bins, c->B);
        b->max_nreach = std::max(b->max_nreach, c->nreach);
        upd[i] = update_args(c);
        upd[i].nblocks = (c->p + b->block - 1) / b->block;
        states[i] = c->state;
    }
    for (int i : order)
        if (b->sys[i]->system != kPolymer)
            for (int w0 = 0; w0 < b->sys[i]->p; w0 += b->block) tiles.push_back(make_int2(i, w0));
    b->order = order;
    b->ntiles = (int)tiles.size();
    b->h_sys.resize(n);
    const size_t sz_sys = align_up(sizeof(SpinSweepArgs) * n), sz_tiles = align_up(sizeof(int2) * tiles.size()),
                 sz_upd = align_up(sizeof(UpdateArgs) * n), sz_st = align_up(sizeof(DevState *) * n);
    cudaError_t e = cudaMalloc(&b->dmem, sz_sys + sz_tiles + sz_upd + sz_st);
    if (e != cudaSuccess) {
        cudaStreamDestroy(b->stream);
        cudaEventDestroy(b->ev_in);
        cudaEventDestroy(b->ev_out);
        delete b;
        return fail(MUCA_ERR_OOM, "muca_batch_create: %s", cudaGetErrorString(e));
    }
    char *base = (char *)b->dmem;
    b->d_sys = (SpinSweepArgs *)base;
    b->d_tiles = (int2 *)(base + sz_sys);
    b->d_upd = (UpdateArgs *)(base + sz_sys + sz_tiles);
    b->d_states = (DevState **)(base + sz_sys + sz_tiles + sz_upd);
    e = cudaMemcpy(b->d_tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_upd, upd.data(), sizeof(UpdateArgs) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_states, states.data(), sizeof(DevState *) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && b->tiles_fit) e = prepare_sweep_batch(b->smem);
    if (e == cudaSuccess) e = prepare_recursion_batch(b->max_nreach);
    if (e != cudaSuccess) {
        cudaFree(b->dmem);
        cudaStreamDestroy(b->stream);
        cudaEventDestroy(b->ev_in);
        cudaEventDestroy(b->ev_out);
        delete b;
        return fail(MUCA_ERR_CUDA, "muca_batch_create: %s", cudaGetErrorString(e));
    }
    if (int rc = muca_batch_set_form(b, 1)) {  // default: the systems' own kernels side by side
        muca_batch_free(b);
        return rc;
    }
    *out = b;
    return MUCA_OK;
}

int muca_batch_run(muca_batch *b, int n_iter, int64_t sweeps, int use_graph)
{
    NvtxRange nvtx(use_graph ? "muca_batch_run (graph)" : "muca_batch_run");
    if (!b) return fail(MUCA_ERR_ARG, "batch is NULL");
    if (n_iter < 1 || sweeps < 1) return fail(MUCA_ERR_ARG, "n_iter and sweeps must be >= 1");
    const int n = (int)b->sys.size();
    for (int i = 0; i < n; ++i)
        if (b->sys[i]->open)
            return fail(MUCA_ERR_STATE, "system %d has unmerged sweeps; call muca_merge_and_update first", i);
    auto sweeps_of = [&](int i) { return b->sw.empty() ? sweeps : b->sw[i]; };
    for (int i = 0; i < n; ++i)
        if (b->sys[i]->system == kPolymer && sweeps_of(i) > 0x7fffffffLL / b->sys[i]->N)
            return fail(MUCA_ERR_RANGE, "system %d: too many sweeps in one iteration", i);
    b->h_own.resize(n);
    for (int i = 0; i < n; ++i) {
        if (b->sys[i]->system == kPolymer) {  // only the sweep count and the state (counter advance)
            SpinSweepArgs z{};
            z.sweeps = sweeps_of(i);
            z.state = b->sys[i]->state;
            b->h_sys[i] = b->h_own[i] = z;
        } else {
            b->h_sys[i] = sweep_args(b->sys[i], sweeps_of(i), b->block);
            b->h_own[i] = sweep_args(b->sys[i], sweeps_of(i), b->blk[i]);
        }
    }
    // order the batch's own stream after the systems' earlier work
    MUCA_CUDA(cudaEventRecord(b->ev_in, b->ctx_stream));
    MUCA_CUDA(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    MUCA_CUDA(cudaMemcpyAsync(b->d_sys, b->h_sys.data(), sizeof(SpinSweepArgs) * n, cudaMemcpyHostToDevice,
                              b->stream));
    // the flatness ratio may change between runs
    std::vector<UpdateArgs> upd(n);
    for (int i = 0; i < n; ++i) {
        upd[i] = update_args(b->sys[i]);
        if (b->sys[i]->system != kPolymer) {  // (a polymer's open histogram is one slot)
            const int blk = (b->form == 0) ? b->block : b->blk[i];  // form 1: each system's block in the batch
            upd[i].nblocks = (b->sys[i]->p + blk - 1) / blk;
        }
    }
    MUCA_CUDA(cudaMemcpyAsync(b->d_upd, upd.data(), sizeof(UpdateArgs) * n, cudaMemcpyHostToDevice, b->stream));
    if (use_graph) {
        if (!b->exec || b->g_iter != n_iter || b->g_sweeps != sweeps || b->g_sw != b->sw) {
            if (b->exec) {
                cudaGraphExecDestroy(b->exec);
                b->exec = nullptr;
            }
            // the host-side copies above stay outside the captured region
            MUCA_CUDA(cudaStreamSynchronize(b->stream));
            MUCA_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            int rc = MUCA_OK;
            for (int it = 0; it < n_iter && rc == MUCA_OK; ++it) rc = batch_enqueue_iteration(b, sweeps);
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
            if (rc != MUCA_OK) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (e != cudaSuccess) return fail(MUCA_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
            e = cudaGraphInstantiate(&b->exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                b->exec = nullptr;
                return fail(MUCA_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
            }
            b->g_iter = n_iter;
            b->g_sweeps = sweeps;
            b->g_sw = b->sw;
        }
        MUCA_CUDA(cudaGraphLaunch(b->exec, b->stream));
    } else {
        for (int it = 0; it < n_iter; ++it)
            if (int rc = batch_enqueue_iteration(b, sweeps)) return rc;
    }
    // and the systems' later work after the batch
    MUCA_CUDA(cudaEventRecord(b->ev_out, b->stream));
    MUCA_CUDA(cudaStreamWaitEvent(b->ctx_stream, b->ev_out, 0));
    for (int i = 0; i < n; ++i) b->sys[i]->started = true;
    return MUCA_OK;
}

int muca_batch_free(muca_batch *b)
{
    if (!b) return MUCA_OK;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->dmem) cudaFree(b->dmem);
    for (cudaStream_t st : b->sub) {
        if (cudaStreamSynchronize(st) != cudaSuccess && e == cudaSuccess) e = cudaErrorUnknown;
        cudaStreamDestroy(st);
    }
    for (cudaEvent_t ev : b->ev_join) cudaEventDestroy(ev);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    cudaStreamDestroy(b->stream);
    cudaEventDestroy(b->ev_in);
    cudaEventDestroy(b->ev_out);
    delete b;
    if (e != cudaSuccess) return fail(MUCA_ERR_CUDA, "muca_batch_free: %s", cudaGetErrorString(e));
    return MUCA_OK;
}

int muca_batch_set_sweeps(muca_batch *b, const int64_t *sweeps, int n)
{
    if (!b) return fail(MUCA_ERR_ARG, "batch is NULL");
    std::vector<int64_t> sw;
    if (sweeps) {
        if (n != (int)b->sys.size()) return fail(MUCA_ERR_ARG, "need %d sweep counts, got %d", (int)b->sys.size(), n);
        for (int i = 0; i < n; ++i)
            if (sweeps[i] < 1) return fail(MUCA_ERR_ARG, "system %d: sweeps must be >= 1", i);
        sw.assign(sweeps, sweeps + n);
    }
    MUCA_CUDA(cudaStreamSynchronize(b->stream));  // the tile list may be in use
    b->sw = sw;
    b->order = batch_order(b);
    std::vector<int2> tiles;
    for (int i : b->order)
        if (b->sys[i]->system != kPolymer)
            for (int w0 = 0; w0 < b->sys[i]->p; w0 += b->block) tiles.push_back(make_int2(i, w0));
    if (!tiles.empty())
        MUCA_CUDA(cudaMemcpy(b->d_tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice));
    return MUCA_OK;
}

int muca_batch_set_form(muca_batch *b, int form)
{
    if (!b) return fail(MUCA_ERR_ARG, "batch is NULL");
    if (form != 0 && form != 1) return fail(MUCA_ERR_ARG, "batch form must be 0 or 1");
    if (form == 0 && !b->tiles_fit)
        return fail(MUCA_ERR_ARG, "batch form 0 needs every system's table in shared memory (not q-Potts at L = 64)");
    if (form == 1 && b->sub.empty()) {
        const int n = (int)b->sys.size();
        for (int i = 0; i < n; ++i) {
            cudaStream_t st = nullptr;
            cudaEvent_t ev = nullptr;
            if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
                return fail(MUCA_ERR_CUDA, "muca_batch_set_form: cannot create a stream");
            b->sub.push_back(st);
            if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
                return fail(MUCA_ERR_CUDA, "muca_batch_set_form: cannot create an event");
            b->ev_join.push_back(ev);
        }
        if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess)
            return fail(MUCA_ERR_CUDA, "muca_batch_set_form: cannot create an event");
    }
    if (form != b->form && b->exec) {  // the captured graph belongs to the other form
        MUCA_CUDA(cudaStreamSynchronize(b->stream));
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    b->form = form;
    return MUCA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// No-allocation variant of one iteration's sweeps + histogram merge.
//
// Some callers cannot call cudaMalloc at the point where they run an iteration:
// code that must not allocate while a CUDA graph is being captured, hosts whose
// memory pools forbid raw driver allocations, or processes that run the GPU at
// its memory limit and cannot risk an allocation failure mid-run.  For them this
// entry point keeps the per-block partial histograms of the sweep kernel in a
// fixed array that is part of the library image instead of in memory allocated
// at run time.  The array is a file-scope __device__ array: every GPU that loads
// the library holds it (4 MiB) until the process exits.
namespace {

constexpr size_t kStaticHistSlots = size_t(1) << 19;  // 524288 uint64 bins = 4 MiB
static __device__ __align__(256) unsigned long long g_static_hist[kStaticHistSlots];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
unsigned long long *g_static_ptr[kMaxDevices] = {};

// Device address of g_static_hist on the current device, looked up once per
// device (host code cannot use the symbol itself: in host code its name is a
// host-side stand-in, not a device address).
int static_hist_ptr(unsigned long long **out)
{
    int dev = 0;
    MUCA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(MUCA_ERR_RANGE, "device %d beyond the supported %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_hist);
        if (e != cudaSuccess)
            return fail(MUCA_ERR_CUDA, "cudaGetSymbolAddress(g_static_hist): %s", cudaGetErrorString(e));
        g_static_ptr[dev] = (unsigned long long *)p;
    }
    *out = g_static_ptr[dev];
    return MUCA_OK;
}

}  // namespace

extern "C" int muca_iterate_noalloc(muca_ctx *c, int64_t sweeps, uint64_t *dev_H_out)
{
    if (int rc = check_ctx(c)) return rc;
    if (sweeps < 1) return fail(MUCA_ERR_ARG, "sweeps must be >= 1");
    if (!dev_H_out) return fail(MUCA_ERR_ARG, "dev_H_out is NULL");
    if (c->system == kPolymer) return fail(MUCA_ERR_ARG, "muca_iterate_noalloc: spin systems only");
    const size_t nblocks = (size_t)((c->p + c->block - 1) / c->block);
    const size_t need = nblocks * (size_t)c->B;
    if (need > kStaticHistSlots)
        return fail(MUCA_ERR_RANGE,
                    "muca_iterate_noalloc: %zu thread blocks x %d bins = %zu partial-histogram slots exceed the "
                    "static maximum of %zu (use fewer walkers, a larger block, or muca_iterate)",
                    nblocks, c->B, need, kStaticHistSlots);
    unsigned long long *scratch = nullptr;
    if (int rc = static_hist_ptr(&scratch)) return rc;
    // The array keeps whatever the previous call left in it: clear the slots used here.
    MUCA_CUDA(cudaMemsetAsync(scratch, 0, need * sizeof(unsigned long long), c->stream));
    SpinSweepArgs a = sweep_args(c, sweeps, c->block);
    a.Hpart = scratch;
    // the context's configured sweep form, as muca_iterate runs it: every form writes its block
    // histograms to slots 0 .. ceil(p / block) - 1 of a.Hpart
    MUCA_CUDA(launch_system_sweep(c, a, c->stream));
    MUCA_CUDA(launch_advance(c->state, sweeps, c->stream));
    UpdateArgs u = update_args(c);
    u.Hpart = scratch;
    u.H = (unsigned long long *)dev_H_out;
    MUCA_CUDA(launch_merge(u, c->stream));
    c->started = true;
    return MUCA_OK;
}
