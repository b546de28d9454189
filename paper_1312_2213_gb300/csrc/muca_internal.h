// muca_internal.h -- host-side context and the launch interfaces between the
// C ABI (muca_api.cu) and the kernels (sweep_spin.cu, update.cu).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace muca {

enum System { kIsing = 0, kPotts = 1, kMuma = 2, kPolymer = 3 };

// Largest thread block of the sweep kernels (keeps up to 128 registers a thread).
constexpr int kMaxSweepBlock = 512;
constexpr int kMetricWords = 8;  // per-context metrics counters (see UpdateArgs::metrics)

// Threshold meaning "always accept"; any other value t accepts iff u < t.
constexpr uint32_t kAlways = 0xFFFFFFFFu;

// Device-resident loop state: the sweep counter lives on the device so that a
// captured iterate -> merge -> update sequence can be replayed unchanged.
struct DevState {
    unsigned long long sweep_counter;  // global sweep index of the next sweep
    unsigned long long iteration;      // completed merge+update steps
    double flat_min, flat_mean, flat_max;
    int flat;
    int err;                           // non-zero: a device-side check failed
    unsigned long long drift_max_q;    // polymer: largest |E_running - E_scratch| at a refresh (2^-32 units)
};

// Everything one spin sweep launch needs.  All pointers are device pointers.
struct SpinSweepArgs {
    const uint32_t *T;       // [B][C] thresholds
    uint32_t *lattice;       // packed rows, word j of walker w at lattice[j * pstride + w]
    int32_t *bin;            // [p] current bin
    unsigned long long *Hpart;  // [nblocks][B] per-block histograms (uint64)
    const DevState *state;   // sweep counter
    int p, pstride, B, q;
    int64_t sweeps;
    int flush_every;         // sweeps between smem -> global histogram flushes
    uint32_t key0, key1;
    int record;
    int walker_offset;       // global id of walker 0 (for sharding)
    uint32_t rk[20];         // Philox round keys (k0 + r*W0, k1 + r*W1), r = 0..9
    int kind;                // system * 16 + L / 4 (dispatch key of the batched sweep)
    unsigned long long *obs = nullptr;  // Ising observables: per bin (samples, sum |M|, sum M^2), or null
    int debug_drop_row = -1; // test hook: row hand-over (count within the launch) that the first
                             // producer warp of block 0 skips, so the consumer's wait runs out; -1 = off
    unsigned long long *metrics = nullptr;  // open counters {accepted moves, tunnelling events}
    uint8_t *tun = nullptr;  // [p] tunnelling state per walker (0 none, 1 lowest bin last, 2 highest)
    int bin_lo = 0, bin_hi = 0;  // lowest and highest reachable bins
    int spin_limit = 0;          // tries a bounded hand-over wait makes before it gives up (0: default)
    int debug_check = 0;         // checked build only: every table bounds check fails (test hook)
};

// Philox round keys for a seed: round r uses (lo + r*W0, hi + r*W1).
inline void fill_round_keys(SpinSweepArgs &a, uint64_t seed)
{
    uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    a.key0 = k0;
    a.key1 = k1;
    for (int r = 0; r < 10; ++r) {
        a.rk[2 * r] = k0;
        a.rk[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Layout helpers shared by host and kernels.
__host__ __device__ constexpr int ising_words_per_row(int L) { return (L + 31) / 32; }
__host__ __device__ constexpr int potts_words_per_row(int L) { return (4 * L + 31) / 32; }
__host__ __device__ constexpr int words_per_walker(int system, int L)
{
    return L * (system == kPotts ? potts_words_per_row(L) : ising_words_per_row(L));
}
__host__ __device__ constexpr int num_cols(int system) { return system == kPotts ? 9 : (system == kMuma ? 10 : 5); }

// Launchers (return cudaSuccess or the launch error; cudaErrorInvalidValue for
// an unsupported lattice size).
bool spin_sweep_supported(int system, int L);
size_t spin_sweep_smem_bytes(int system, int B);
cudaError_t launch_spin_sweep(int system, int L, const SpinSweepArgs &a, int block, cudaStream_t s);
int sweep_kind(int system, int L);
// Producer/consumer form: `block` walkers a block, run by 2*block threads.
bool spin_sweep_pc_fits(int system, int L, int B, int walkers_per_block);
size_t spin_sweep_pc_smem_bytes(int system, int L, int B, int walkers_per_block);
cudaError_t launch_spin_sweep_pc(int system, int L, const SpinSweepArgs &a, int block, cudaStream_t s);
// Producer/consumer form with precomputed site codes (Ising, MUMA).
bool spin_sweep_tn_fits(int system, int L, int B, int walkers_per_block);
size_t spin_sweep_tn_smem_bytes(int system, int L, int B, int walkers_per_block);
cudaError_t launch_spin_sweep_tn(int system, int L, const SpinSweepArgs &a, int block, cudaStream_t s);
// Batched sweep: tiles[k] = (system index, first walker); all tiles use `block` threads.
cudaError_t prepare_sweep_batch(size_t smem);
cudaError_t launch_sweep_batch(const SpinSweepArgs *d_sys, const int2 *d_tiles, int ntiles, int block, size_t smem,
                               cudaStream_t s);

// Polymer (bead-spring chain, Eq. 7 reading).  Master coordinates are int64 on a
// 2^-44 grid, walker-major and axis-major: X[(w*3 + a)*N + j]; energies are int64
// in units of 2^-32; the window is [elo_q, elo_q + B/10) in the same units.
constexpr int kPolyMaxBins = 12288;  // the recursion stages 2 doubles a bin in shared memory
constexpr int kPolyMaxN = 128;
constexpr long long kPolyStepQ = 1229;  // displacement grid units per unit of (u - 2^31)

// One attempt of a polymer sweep, recorded for parity checks (muca_poly_trace):
// the energy change and the energy after the decision (2^-32 units), the bin of
// the proposed energy and the bin after the decision, flags 1 accepted, 2 a bond
// broke (or a rotation found no point), 4 a lane sum too large (rejected).
struct PolyTraceRec {
    long long dq, E;
    int32_t bn, b, flags, pad;
};

struct PolyArgs {
    long long *X;
    long long *E;
    int32_t *bin;
    const long long *lnWq;         // ln W in units of 2^-32
    unsigned long long *H;         // open histogram (B counters)
    DevState *state;
    int p, N, B, record, walker_offset;
    int lanes;                     // lanes per walker in the sweep (8, 16, 32; 0 = by N)
    long long elo_q, ehi_q;        // window [elo_q, ehi_q): bins 0..B-1
    float fene_KR2_half, fene_invR2, lj_rc2, lj_shift;
    int model;                     // 0: benchmark parameters, 1: the paper's (Eq. 7)
    int moves;                     // 0: single-bead shifts, 1: shifts and spherical rotations
    float fene_r0, fene_invR, lj_sigma2;  // model 1: rest length, 1/R, sigma^2 (model 0: 0, -, 1)
    double init_bond, init_d2min;  // initial bond length b0 and (0.9 b0)^2
    int64_t sweeps;
    uint32_t key0, key1;
    uint32_t rk[20];
    unsigned long long *metrics = nullptr;  // open counters {accepted moves, tunnelling events}
    uint8_t *tun = nullptr;                 // [p] tunnelling state per walker
    PolyTraceRec *trace = nullptr;          // [p][sweeps][N] attempt records, or null
    int flush_every = 0;  // most sweeps between flushes of the block's counters (0: their own bound)
    int bin_k = 10;               // bins per unit energy (width 1 / bin_k)
    int step_q = 1229;            // move grid units per unit of (u - 2^31): cube side step_q / 4096
    int64_t sweep_base = 0;    // this launch's first sweep within the iterate (launch_poly_sweep chunks)
    int64_t trace_sweeps = 0;  // sweeps of the traced iterate
};
bool polymer_supported(int N);
cudaError_t launch_poly_init(const PolyArgs &a, cudaStream_t s);
cudaError_t launch_poly_energy(const PolyArgs &a, int track_drift, cudaStream_t s);
cudaError_t launch_poly_sweep(const PolyArgs &a, int block, cudaStream_t s);
int poly_lanes(const PolyArgs &a, int requested);
cudaError_t launch_poly_lnwq(const double *lnW, long long *lnWq, int B, cudaStream_t s);
cudaError_t launch_poly_unpack(const PolyArgs &a, double *coords, double *energies, cudaStream_t s);

struct UpdateArgs {
    int system, B, nreach, nblocks, N, q, p, pstride, L;
    double beta, flat_ratio;
    double e_lo;  // polymer: energy of the window's lower edge
    double bin_w = 0.1;  // polymer: bin width
    int recursion;  // 0: accumulated statistics, 1: plain W/H
    const uint8_t *reach;
    const int32_t *rlist;
    unsigned long long *Hpart, *H;
    double *lnW, *lnW_sampled, *G, *lnR;
    uint32_t *T;
    DevState *state;
    // metrics counters {open accepted, open tunnelling events, last accepted, last events,
    // total accepted, total events, sweeps of the last iteration, sweep counter at the last
    // update}; the recursion launch closes them (null: none)
    unsigned long long *metrics;
};
cudaError_t launch_merge(const UpdateArgs &a, cudaStream_t s);
// Batched update kernels over n systems (argument arrays in device memory).
cudaError_t launch_merge_batch(const UpdateArgs *d_args, int n, int max_bins, cudaStream_t s);
cudaError_t launch_recursion_batch(const UpdateArgs *d_args, int n, int max_nreach, cudaStream_t s);
cudaError_t prepare_recursion_batch(int max_nreach);
cudaError_t launch_thresholds_batch(const UpdateArgs *d_args, int n, int max_cells, cudaStream_t s);
cudaError_t launch_advance_batch(DevState *const *d_states, const SpinSweepArgs *d_sys, int n, cudaStream_t s);
cudaError_t launch_recursion(const UpdateArgs &a, cudaStream_t s);
cudaError_t launch_thresholds(const UpdateArgs &a, cudaStream_t s);
cudaError_t launch_advance(DevState *st, int64_t sweeps, cudaStream_t s);
cudaError_t launch_init_lnW(const UpdateArgs &a, cudaStream_t s);
cudaError_t launch_init_spins(int system, int L, int q, int p, int pstride, uint32_t key0, uint32_t key1,
                              int walker_offset, uint32_t *lattice, int32_t *bin, cudaStream_t s);
cudaError_t launch_unpack_spins(int system, int L, int p, int pstride, const uint32_t *lattice, int8_t *out,
                                cudaStream_t s);
cudaError_t launch_det_math(int fn, const double *in, double *out, long long n, cudaStream_t s);
cudaError_t launch_reweight(const UpdateArgs &a, double beta, double *out4, double *lnP, cudaStream_t s);
cudaError_t launch_reweight_obs(const unsigned long long *sums, const double *lnW_sampled, int B, int N, double beta,
                                double *out3, cudaStream_t s);

}  // namespace muca
