/*
 * muca.h -- C ABI of a GB300 (sm_103a) implementation of the parallel
 * multicanonical (MUCA) method of Zierenberg, Marenz and Janke,
 * "Scaling Properties of Parallelized Multicanonical Simulations"
 * (arXiv:1312.2213).
 *
 * The method (paper, Fig. 1 and the paragraph before it): p independent
 * Markov chains ("walkers") share one weight function W; each iteration they
 * sweep and fill histograms, the histograms are merged, a new W is computed
 * from the merged histogram and handed back to all walkers; this repeats until
 * the histogram is flat.  Here all p walkers of a system live on one GPU, the
 * merge is an integer reduction on the device and the weight recursion runs on
 * the device, so nothing crosses the host inside the loop.
 *
 * Conventions for every function:
 *   - Return value: MUCA_OK (0) or a negative MUCA_ERR_* code.  No function
 *     aborts or exits; on error muca_last_error() returns a message (storage
 *     owned by the library, valid until the next call on the same host thread).
 *   - Pointers named host_* are caller-owned HOST memory of the stated length;
 *     the call copies synchronously and returns when the data is there.
 *   - Device work is enqueued on the context's stream (muca_set_stream) and is
 *     asynchronous unless the call returns data to the host.
 *   - A context is used by one host thread at a time.
 *   - Lengths that do not match the context (nbins, p, ...) give MUCA_ERR_ARG.
 */
#ifndef MUCA_H
#define MUCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MUCA_OK 0
#define MUCA_ERR_ARG (-1)         /* bad argument or unsupported combination */
#define MUCA_ERR_CUDA (-2)        /* a CUDA runtime call or kernel launch failed */
#define MUCA_ERR_OOM (-3)         /* device allocation failed / arena too small */
#define MUCA_ERR_TIMEOUT (-4)     /* a bounded device wait gave up */
#define MUCA_ERR_STATE (-5)       /* call not allowed in the context's current state */
#define MUCA_ERR_RANGE (-6)       /* value outside the supported range */
#define MUCA_ERR_CHECK (-7)       /* checked build: a device bounds check failed */

/* Systems (paper: Ising paragraph, Potts paragraph, multimagnetic ensemble
 * Eq. 3, bead-spring polymer Eq. 7). */
enum {
    MUCA_ISING2D = 0,      /* H = -J sum_<ij> s_i s_j, L x L periodic, MUCA in E   */
    MUCA_POTTS2D = 1,      /* H = -J sum_<ij> delta(s_i,s_j), q states, MUCA in E  */
    MUCA_ISING2D_MUMA = 2, /* Ising at fixed beta, weight exp(-beta E) W(M), Eq. 3 */
    MUCA_POLYMER3D = 3     /* FENE + Lennard-Jones chain, Eq. 7, MUCA in E (see muca_set_param) */
};

typedef struct muca_ctx muca_ctx;     /* opaque, library-owned */
typedef struct muca_batch muca_batch; /* opaque, library-owned */

/* Message of the last failed call on this host thread ("" if none). */
const char *muca_last_error(void);

/* Create a simulation of p walkers of one system sharing one ln W table
 * (Fig. 1: "initialized in p independent realizations with the same weight
 * function").  L_or_N is the lattice side L (spins) or the bead count N
 * (polymer); q is the number of Potts states (ignored otherwise).
 * Spins: L in {4, 8, 12, 16, 24, 32, 48, 64}; Potts 2 <= q <= 16 (at L = 64
 * the Potts threshold table is split, see "pipeline").
 * Polymer: 2 <= N <= 128 beads; the walkers start as random walks of unit
 * bonds and walk into the energy window before anything is recorded.
 * The walkers' initial states are drawn from the counter-based generator
 * keyed by `seed` (ln W = 0 everywhere, so the first iteration samples
 * beta = 0, where a random state is already in equilibrium: the paper
 * thermalises only at the start).  The library allocates its device memory
 * with cudaMalloc on the current device; the context uses the legacy default
 * stream until muca_set_stream.  *out receives the context. */
int muca_init(muca_ctx **out, int system, int L_or_N, int q, int p, uint64_t seed);

/* Same, but every device buffer is carved from a caller-provided device arena
 * (e.g. a torch uint8 tensor) of at least muca_workspace_size() bytes, 256-byte
 * aligned.  The caller keeps the arena alive until muca_free. */
int muca_workspace_size(int system, int L_or_N, int q, int p, size_t *bytes);
int muca_init_ex(muca_ctx **out, int system, int L_or_N, int q, int p, uint64_t seed,
                 void *device_arena, size_t arena_bytes);

/* Set a parameter.  Keys:
 *   "beta"        MUMA inverse temperature (Eq. 3); before the first iterate.
 *   "record"      0 = count the current bin after every attempt (default),
 *                 1 = once per sweep; before the first iterate.
 *   "flat_ratio"  flatness criterion min H / mean H (default 0.5); any time.
 *   "block"       spins: walkers per thread block of the sweep kernel (32..512,
 *                 multiple of 32; default 64, or 32 where only that fits the
 *                 code form, and 32 for q-Potts when p <= 32 x the SM count;
 *                 the code form runs for 32 or 64);
 *                 polymer: threads per block (default 256).  Before the first
 *                 iterate.
 *   "pipeline"    spins: 2 (default) pairs every warp of walkers with
 *                 producer warps (two; three for Potts) that compute their
 *                 random numbers and each site's neighbour code (Potts: also
 *                 the proposal) into a shared-memory ring; 1 does the same
 *                 with random numbers only, one producer warp; 0 runs one
 *                 warp per 32 walkers.  q-Potts at L = 64: the code form keeps
 *                 the upper 16 bits of its 295 KB threshold table in shared
 *                 memory beside 16-bit visit counters (64 walkers a block)
 *                 and decides equal upper halves on the full words; 0 reads
 *                 the full table from global memory.  A form that does not
 *                 fit the system, L, bin count or block falls back to the next
 *                 lower one.  Ring hand-overs are bounded waits; a wait that
 *                 gives up makes the next synchronising call return
 *                 MUCA_ERR_TIMEOUT.  Results are identical in every form.
 *   "walker_offset" global id of this context's walker 0 when one system's
 *                 walkers are split over several contexts (e.g. one per GPU):
 *                 walker w draws from the stream of walker w + offset, so the
 *                 union of the shards equals one context of all walkers;
 *                 re-draws the initial states; before the first iterate.
 *   "observables" Ising, before the first iterate: 1 records per-sweep sums of
 *                 |M| and M^2 per energy bin (see muca_get_observables).
 *   "recursion"   lattice systems, before the first iterate: the weight update,
 *                 0 (default) = accumulated statistics in log form (the paper's
 *                 method), 1 = the paper's simple rule W(n+1)(E) = W(n)(E)/H(n)(E)
 *                 in log form over the reachable bins (an unvisited bin keeps
 *                 its weight, ln W(r_0) = 0).
 *   "debug_drop_row"  test hook for the bounded waits (lattice systems): in the
 *                 next muca_iterate only, the first producer warp of thread
 *                 block 0 leaves out its hand-over of row r (counted from 0
 *                 over the sweeps of that call), so the consumer's wait runs
 *                 out; its warp then stops computing and the next synchronising
 *                 call returns MUCA_ERR_TIMEOUT.  The context's walker state is
 *                 invalid afterwards (restore a checkpoint with muca_set_state).
 *                 No effect with pipeline = 0 or a row past the call's sweeps.
 *   "debug_check" checked build only (libmuca_checked.so, -DMUCA_CHECKED, which
 *                 bounds-checks every shared-memory table access of the spin
 *                 sweeps, clamps an index outside the table to its first entry
 *                 and makes the next synchronising call return MUCA_ERR_CHECK):
 *                 1 makes every check of the following iterates fail, to test
 *                 that path (all accesses then read the table's first entry).
 *                 The regular build refuses the key with MUCA_ERR_ARG.
 *   "spin_limit"  tries (of mbarrier.try_wait, each suspending the warp for a
 *                 few microseconds) one row hand-over of the producer/consumer
 *                 forms makes before it gives up; 0 (default) = 2^17, about a
 *                 second on GB300.  The environment variable MUCA_SPIN_LIMIT
 *                 sets it at muca_init.  A limit too small for a healthy run
 *                 only makes the next synchronising call report
 *                 MUCA_ERR_TIMEOUT.  Any time.
 *   "flush_every" at most this many sweeps between two flushes of a thread
 *                 block's shared-memory uint32 histogram counters to its
 *                 uint64 slot (the polymer: to the uint64 histogram); 0
 *                 (default) = the largest count that cannot overflow a
 *                 counter (floor((2^32 - 1) / (block walkers * N)), or
 *                 / block with "record" = 1).  Results do not depend on it;
 *                 a small value makes short runs cross the flush between
 *                 chunks of sweeps (tests).  Any time.
 *   "model"       polymer, before the first iterate: 0 (default) = the benchmark
 *                 parameters (FENE K = 40, R = 1.5, rest length 0; LJ sigma = 1 cut
 *                 at 2.5 and shifted), 1 = the paper's own parameters of Eq. (7)
 *                 (FENE with K = 40, r0 = 0.7, r_max = 1; LJ sigma = 2^(-1/6) r0,
 *                 no cutoff).  Redraws the initial chains (bond length r0 in
 *                 model 1); travels with muca_get_state.
 *   "moves"       polymer, before the first iterate: 0 (default) = single-bead
 *                 shifts; 1 = the paper's combination of shifts with spherical
 *                 rotations (each attempt picks one with probability 1/2; a
 *                 rotation puts the bead on a uniform point of the sphere about a
 *                 bonded neighbour, keeping that bond's length, computed in
 *                 correctly rounded binary64 and rounded to the coordinate grid).
 *   "lanes"       polymer: lanes of a warp per walker in the sweep, 1, 2, 4, 8, 16 or
 *                 32 (32/lanes walkers share a warp; with 1 lane a walker's lane takes
 *                 both bonds of the moved bead); 0 (default) means 16.  A grouping whose
 *                 warp does not fit a block's shared memory falls back to the next larger
 *                 one, and the block shrinks to the warps that fit.  The pair terms are
 *                 FP32 and their grouping over lanes changes their rounding, so
 *                 runs with different values agree within the FP32 tolerance,
 *                 not bit for bit.  Any time.
 *   Polymer only (before the first iterate): "e_lo", "e_hi" (the energy
 *   window, at most 12288 bins; default [2N, 6N)), "bin_width" (1/k for a
 *   whole k in 1..1000; default 0.1), "step" (the side of the move cube,
 *   rounded to a multiple of 1/4096 in [1/4096, 2]; default 1229/4096 =
 *   0.30005), "fene_K", "fene_R" (default 40, 1.5).  Fixed: LJ eps = sigma = 1
 *   cut at 2.5 and shifted, acting on beads |i-j| >= 2; FENE on bonds;
 *   single-bead moves uniform in the cube on a 2^-44 grid.
 * Unknown key or bad value: MUCA_ERR_ARG; too late: MUCA_ERR_STATE. */
int muca_set_param(muca_ctx *ctx, const char *key, double value);

/* Use `cuda_stream` (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream)
 * for all later device work of this context. */
int muca_set_stream(muca_ctx *ctx, void *cuda_stream);

/* Run `sweeps` sweeps of every walker under the current weights (one
 * iteration's worth of independent equilibrium simulation, Fig. 1), filling
 * the histogram of the open iteration.  Asynchronous. sweeps >= 1. */
int muca_iterate(muca_ctx *ctx, int64_t sweeps);

/* Merge the walkers' histograms into H^(n), compute W^(n+1) with the
 * accumulated-statistics recursion in log form (paper: "use the full
 * statistics of previous iterations ... implemented with logarithmic
 * weights") and rebuild the acceptance thresholds ("distributed to all p
 * cores").  If is_flat is non-NULL the call synchronises and stores 1 when
 * every reachable bin of H^(n) is non-zero and min/mean >= flat_ratio. */
int muca_merge_and_update(muca_ctx *ctx, int *is_flat);

/* Sharded runs: one system's walkers split over processes (typically one per
 * GPU), the paper's Fig. 1 scheme with the histogram exchange as an all-reduce.
 * Each shard is a context with the same system, L, q and seed, holding p_k
 * walkers and "walker_offset" = the global id of its first walker.  After
 * muca_iterate, muca_merge_open sums this shard's open histogram (its walkers'
 * counts since the last update) into the caller's DEVICE buffer dev_H_out (B
 * uint64, overwritten) and clears it in the context; the caller adds the
 * buffers of all shards (e.g. torch.distributed.all_reduce) and muca_update_with
 * closes the iteration on every shard with the summed histogram dev_H (the same
 * recursion and thresholds as muca_merge_and_update), so all shards keep
 * identical weights and together equal one context that holds all walkers.
 * Observable sums (if recorded) stay per shard.  is_flat as in
 * muca_merge_and_update.  Errors: MUCA_ERR_ARG on a NULL buffer. */
int muca_merge_open(muca_ctx *ctx, uint64_t *dev_H_out);
int muca_update_with(muca_ctx *ctx, const uint64_t *dev_H, int *is_flat);

/* Replace the current weights ln W^(n) with host_lnW (B doubles; unreachable
 * bins are set to -inf whatever the buffer holds; reachable bins must be
 * finite) and rebuild what the sweeps read from them (thresholds, or the
 * polymer's fixed-point table).  Use: a production run at fixed weights, e.g.
 * converged weights of an earlier run (the paper's last step: simulate with the
 * final W and reweight, Eq. 2).  The accumulated statistics of the recursion
 * are not touched, so the next muca_merge_and_update computes W^(n+1) from
 * them as before; the histogram it merges is reweighted with the weights set
 * here.  Synchronous.  Errors: MUCA_ERR_ARG on a wrong length or a non-finite
 * reachable bin. */
int muca_set_lnW(muca_ctx *ctx, const double *host_lnW, int nbins);

/* Polymer parity inspection (no counterpart in the paper): the next
 * muca_iterate of this context writes one 32-byte record per attempt of every
 * walker into the caller's DEVICE buffer dev_records (16-byte aligned; index
 * (walker * sweeps + sweep) * N + bead, sweep counted within that call):
 *   int64 dq     energy change of the attempt in units of 2^-32 (0 if a lane
 *                sum was too large),
 *   int64 E      the walker's energy after the decision (2^-32 units),
 *   int32 bn     bin of the proposed energy (-1 below, B above the window),
 *   int32 b      bin after the decision,
 *   int32 flags  1 accepted, 2 a bond broke (or a rotation found no point),
 *                4 a lane sum too large (move rejected),
 *   int32 pad.
 * n_records is the buffer's capacity; that iterate returns MUCA_ERR_ARG if it
 * makes more than n_records attempts.  Only that one iterate records.  Errors:
 * MUCA_ERR_ARG for a spin context, a NULL or misaligned buffer. */
int muca_poly_trace(muca_ctx *ctx, void *dev_records, int64_t n_records);

/* Number of histogram bins B of the context. */
int muca_num_bins(const muca_ctx *ctx, int *nbins);

/* ln W^(n) (the current weights), B doubles; unreachable bins hold -inf. */
int muca_get_lnW(muca_ctx *ctx, double *host_out, int nbins);
/* The weights the last merged histogram was sampled with (ln W^(n-1)). */
int muca_get_lnW_sampled(muca_ctx *ctx, double *host_out, int nbins);
/* Last merged histogram H^(n), B counts. */
int muca_get_histogram(muca_ctx *ctx, uint64_t *host_out, int nbins);
/* {min, mean, max} of the last merged histogram over reachable bins. */
int muca_get_flatness(muca_ctx *ctx, double host_stats[3]);

/* Reweighting, Eq. (2), of the last merged histogram with the weights it was
 * sampled with: ln Omega(b) = ln H(b) - ln W(b).
 * Ising / Potts: host_out = {<E>, <E^2>, C_V per site, ln Z} at beta, with
 *   ln Z normalised by the ground-state degeneracy (2, resp. q); NaN if the
 *   ground state was never visited.
 * MUMA (at its own beta; `beta` is ignored): {<|M|>/N, <M^2>/N^2,
 *   susceptibility per site, ln P(M=0) - ln P(M=N)}.
 * host_lnP (nullable, B doubles) receives ln P(b). */
int muca_get_reweight(muca_ctx *ctx, double beta, double host_out[4], double *host_lnP);

/* Observables (Ising with "observables" = 1; the paper's Eq. (2) for an
 * observable O that is not a function of the energy): after every sweep each
 * walker adds one sample, |M| and M^2 to three uint64 sums of its current
 * energy bin; each muca_merge_and_update closes the sums with the weights they
 * were sampled with.  host_out = {<|M|>/N, <M^2>/N^2, beta N (<M^2>/N^2 -
 * (<|M|>/N)^2)} at beta (NaN if no samples); host_sums (nullable, 3*nbins
 * uint64: samples, sum |M|, sum M^2 per bin) receives the sums.
 * Not recorded by muca_iterate_noalloc or in batches.
 * Errors: MUCA_ERR_STATE if observables are off, MUCA_ERR_ARG on bad lengths. */
int muca_get_observables(muca_ctx *ctx, double beta, double host_out[3], uint64_t *host_sums, int nbins);

/* Per-iteration metrics (no counterpart in the paper; the acceptance rate and
 * the walkers' round trips between the energy extremes are the usual figures of
 * merit of a multicanonical run).  Every sweep kernel counts the moves it
 * accepts, and samples each walker's bin at the end of every sweep: a
 * tunnelling event is an arrival at the lowest reachable bin when the highest
 * was the last of the two visited, or the reverse (polymer: bins 0 and B-1 of
 * the window).  Each update closes the counts of its iteration.  host_out =
 * {accepted moves of the last closed iteration, its tunnelling events,
 * accepted moves of all closed iterations, their tunnelling events, sweeps of
 * the last closed iteration, closed iterations}; acceptance rate = out[0] /
 * (p N out[4]).  A sharded context counts its own walkers.  Sweeps run by
 * muca_iterate_noalloc count toward the next closed iteration like any other.
 * Synchronises the context's stream. */
int muca_get_metrics(muca_ctx *ctx, uint64_t host_out[6]);

/* Checkpoint: the complete state (walkers, weights, recursion state, counters).
 * Call with host_buf == NULL to get the size in *bytes.  muca_set_state
 * restores a buffer produced by a context of the same configuration; resuming
 * is bit-exact because the random numbers are keyed by (seed, walker, sweep). */
int muca_get_state(muca_ctx *ctx, void *host_buf, size_t *bytes);
int muca_set_state(muca_ctx *ctx, const void *host_buf, size_t bytes);

/* Inspection (parity checks).  Spins unpacked to one int8 per site, walker-major
 * (Ising/MUMA: +1/-1, Potts: 0..q-1), n = p*L*L; current bin of each walker;
 * threshold table T[b][c] (B*C uint32, C = 5 Ising, 9 Potts, 10 MUMA);
 * the global sweep counter. */
int muca_get_spins(muca_ctx *ctx, int8_t *host_out, int64_t n);
int muca_get_walker_bins(muca_ctx *ctx, int32_t *host_out, int p);
int muca_get_thresholds(muca_ctx *ctx, uint32_t *host_out, int64_t n);
int muca_get_sweep_counter(muca_ctx *ctx, int64_t *host_out);

/* Batching.  A batch advances several contexts together -- different systems,
 * lattice sizes, polymer lengths and walker counts, e.g. Ising L in {16..64} and
 * q = 10 Potts L in {16..48} with 2048 walkers each, or polymers of N = 13..128
 * beads -- so that systems too small to fill the GPU alone fill it together
 * (polymers in form 1 only).  Each iteration of muca_batch_run is the paper's
 * Fig. 1 step for every system at once: sweeps of all walkers of all systems
 * (side by side, or in one persistent launch: see muca_batch_set_form), then the merge, the
 * accumulated-statistics recursion and the threshold rebuild for all systems
 * (one launch each).  With use_graph != 0 all n_iter iterations are captured
 * once into a CUDA graph (re-captured when n_iter or sweeps change) and
 * launched as one graph.  Results are bit-identical to running each context on
 * its own with muca_iterate + muca_merge_and_update: a walker's random stream
 * depends only on (seed, walker, sweep).
 * muca_batch_create: the contexts must use the same stream and stay alive
 * until muca_batch_free; the batch owns a small device descriptor table.
 * muca_batch_run: every context must have no unmerged sweeps (MUCA_ERR_STATE). */
int muca_batch_create(muca_ctx *const *systems, int n, muca_batch **out);
int muca_batch_run(muca_batch *batch, int n_iter, int64_t sweeps, int use_graph);
int muca_batch_free(muca_batch *batch);
/* How a batch runs its sweeps.  form 1 (default): each context's own sweep
 * kernel in its configured form ("pipeline", "block"; a q-Potts context whose
 * 32-walker default came from small p runs 64-walker blocks when the batch's
 * contexts together have more 32-walker blocks than the GPU has SMs), one
 * stream per context, forked from and joined back into the batch's stream, heaviest
 * system first, so the launches run side by side (in a graph: as parallel
 * branches); the merge, recursion and threshold launches stay batched.
 * form 0: the one persistent launch over a tile list described above (one
 * warp per 32 walkers, 128 walkers a tile).  Same results either way.
 * Changing the form drops a captured graph.  Errors: MUCA_ERR_ARG for another
 * value. */
int muca_batch_set_form(muca_batch *batch, int form);
/* Sweeps per context and iteration: sweeps[i] >= 1 for context i (e.g. each
 * system's own optimal iteration length M_opt of Eq. 4, so that short and long
 * lattices iterate at their own pace), or sweeps = NULL to give every context
 * the `sweeps` argument of muca_batch_run again (the default).  The systems'
 * launch order and tile list follow the new work, heaviest first; a captured
 * graph is re-captured on the next run.  Synchronises the batch's stream.
 * Errors: MUCA_ERR_ARG for n != the number of contexts or a count < 1. */
int muca_batch_set_sweeps(muca_batch *batch, const int64_t *sweeps, int n);

/* Diagnostics: evaluate the library's deterministic binary64 exp (fn = 0) or
 * log (fn = 1) -- the functions the weight recursion and the threshold build
 * use -- on n host values, on the current device.  Synchronous. */
int muca_det_math(int fn, const double *host_in, double *host_out, int64_t n);

/* No-allocation variant of one iteration's sweeps and histogram merge.
 * The paper has no counterpart: this serves callers that cannot call cudaMalloc
 * when they run an iteration (code that must not allocate during CUDA graph
 * capture, hosts whose memory pools forbid raw driver allocations, processes at
 * their device-memory limit).  It runs `sweeps` sweeps of every walker of `ctx`
 * (like muca_iterate) and writes the merged histogram of exactly these sweeps to
 * the caller's DEVICE buffer dev_H_out (B uint64, overwritten; the context's own
 * open histogram and H are not touched, the weights are not updated).  Walkers,
 * bins and the sweep counter advance as with muca_iterate, and the sweeps run
 * in the context's configured form ("pipeline", "block"), so they are as fast
 * as muca_iterate's; a bounded hand-over wait that gives up shows as
 * MUCA_ERR_TIMEOUT at the next synchronising call (muca_synchronize).  The
 * accepted moves and tunnelling events of these sweeps are added to the
 * context's open metrics counters (muca_get_metrics reports them with the next
 * closed iteration, whose sweep count includes these sweeps); observables are
 * not recorded.
 * Scratch: the per-block partial histograms live in one static device array of
 * 2^19 uint64 slots (4 MiB) that every GPU loading the library holds until the
 * process exits; a call needs ceil(p/block) * B slots and returns MUCA_ERR_RANGE
 * beyond that.  The call allocates nothing: no cudaMalloc, no cudaFree.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) for the device that is current; make that first call
 * before any stream capture.  Every call uses the same array (it clears the
 * slots it needs first), so calls whose GPU work overlaps -- on two streams, or
 * two contexts on the same device from two threads -- race and give wrong
 * histograms; serialise them. */
int muca_iterate_noalloc(muca_ctx *ctx, int64_t sweeps, uint64_t *dev_H_out);

/* Polymer: bead coordinates (p*N*3 doubles, walker-major, then bead, then
 * x/y/z; exact values of the 2^-44 grid the moves live on) and, if host_energies
 * is not NULL, the walkers' running energies (p doubles). */
int muca_get_coords(muca_ctx *ctx, double *host_coords, int64_t n, double *host_energies, int p);
/* Polymer: the largest difference between a running energy and its from-scratch
 * recomputation seen at the refresh after each muca_iterate. */
int muca_get_drift(muca_ctx *ctx, double *host_out);

/* Wait for the context's stream; MUCA_ERR_TIMEOUT if a device-side bounded
 * wait gave up since the context was created. */
int muca_synchronize(muca_ctx *ctx);

/* Release the context and (unless it came from muca_init_ex) its device memory. */
int muca_free(muca_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* MUCA_H */
