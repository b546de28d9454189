/*
 * muca_oracle.h -- plain, slow CPU oracle for the parallel multicanonical (MUCA)
 * method of Zierenberg, Marenz and Janke, "Scaling Properties of Parallelized
 * Multicanonical Simulations" (arXiv:1312.2213).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load
 * this code; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no source with the CUDA library: every formula here
 * is written out from the paper (and, where the paper is silent, from the
 * readings listed at the top of muca_oracle.c).
 *
 * All floating point is IEEE binary64, built with -ffp-contract=off so that
 * a*b+c is always two roundings.
 */
#ifndef MUCA_ORACLE_H
#define MUCA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_ISING = 0, ORC_POTTS = 1, ORC_MUMA = 2, ORC_POLYMER = 3 };

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): out = Philox(ctr, key). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Deterministic binary64 exp / log (Cody-Waite reduction + Taylor / atanh series). */
double orc_det_exp(double x);
double orc_det_log(double x);

typedef struct orc_run orc_run;

/* One MUCA (or multimagnetic) simulation of p independent walkers sharing one
 * weight table, as in the paper's Fig. 1 scheme.  Returns NULL on bad args. */
orc_run *orc_create(int system, int L, int q, int p, uint64_t seed, double beta, int record);
void orc_free(orc_run *r);

int orc_num_bins(const orc_run *r);
int orc_num_cols(const orc_run *r);
int orc_num_sites(const orc_run *r);
void orc_reachable(const orc_run *r, uint8_t *out /* B */);

/* a1: random initial lattices from the INIT Philox stream; ln W = 0; thresholds. */
void orc_init(orc_run *r);
/* a2+a3+a4: `sweeps` sweeps of walkers [w0, w1); their histograms are summed into
 * the open histogram of the current iteration.  The global sweep counter
 * advances by `sweeps` (call with the full range once per chunk, or use
 * orc_iterate_range + orc_advance for sampled walkers). */
void orc_iterate(orc_run *r, int64_t sweeps, int nthreads);
void orc_iterate_range(orc_run *r, int64_t sweeps, int w0, int w1, int nthreads);
void orc_advance(orc_run *r, int64_t sweeps);
/* a5+a6: merge -> accumulated-statistics recursion in log form -> new thresholds. */
void orc_update(orc_run *r);
/* Select the weight update: 0 = accumulated statistics (R5, default),
 * 1 = the plain W/H rule (R5'). */
void orc_set_recursion(orc_run *r, int mode);
/* Fixed weights (a production run at given ln W, Eq. 1): ln W of the reachable bins
 * from lnW[B], -inf elsewhere, then the thresholds (a6). */
void orc_set_lnW(orc_run *r, const double *lnW);
/* Observables (Ising, reading R9): per-sweep sums of 1, |M|, M^2 per bin. */
void orc_set_observables(orc_run *r, int on);
void orc_get_observables(const orc_run *r, uint64_t *out); /* 3*B, last update */
void orc_reweight_obs(int B, int N, const uint64_t *sums, const double *lnW_sampled, double beta, double out[3]);
void orc_reweight_observables(const orc_run *r, double beta, double out[3]);
/* Metrics of the last update: {accepted moves of the closed iteration, its
 * tunnelling events (a walker's bin sampled at the end of every sweep arrives at
 * the lowest reachable bin after the highest was the last end visited, or the
 * reverse), accepted moves of all closed iterations, their tunnelling events,
 * sweeps of the closed iteration}. */
void orc_get_metrics(const orc_run *r, uint64_t out[5]);
/* Replace the open histogram (for recursion tests on hand-made histograms). */
void orc_set_open_histogram(orc_run *r, const uint64_t *H);
void orc_get_open_histogram(const orc_run *r, uint64_t *out);
/* a7: 1 if every reachable bin of the last merged histogram is > 0 and
 * min/mean >= ratio.  stats = {min, mean, max} over reachable bins. */
int orc_is_flat(const orc_run *r, double ratio, double stats[3]);
/* a8: reweighting (Eq. 2) of the last merged histogram to inverse temperature beta.
 * out = {<E>, <E^2>, C_V per site, ln Z} (spin MUCA) or
 *       {<|M|>/N, <M^2>/N^2, chi per site, ln P(0)-ln P(max)} (MUMA, at its own beta). */
void orc_reweight(const orc_run *r, double beta, double out[4], double *lnP /* nullable, B */);

void orc_get_lnW(const orc_run *r, double *out);
void orc_get_lnW_sampled(const orc_run *r, double *out);
void orc_get_histogram(const orc_run *r, uint64_t *out);
void orc_get_thresholds(const orc_run *r, uint32_t *out /* B*K */);
void orc_get_spins(const orc_run *r, int8_t *out /* p*N */);
void orc_get_bins(const orc_run *r, int32_t *out /* p */);
int64_t orc_get_sweep_counter(const orc_run *r);

/* Exact tools, used to pin the above: brute-force enumeration of all states. */
int orc_bruteforce_ising(int L, uint64_t *omega /* N+1, index (E+2N)/4 */);
int orc_bruteforce_ising_EM(int L, uint64_t *omega /* (N+1)*(N+1), [(E+2N)/4][(M+N)/2] */);
int orc_bruteforce_potts(int L, int q, uint64_t *omega /* 2N+1, index E+2N */);
/* Exact tools: transfer matrices, counts as (lo, hi) 64-bit pairs.
 * orc_tm_ising: index (E+2N)/4, or [(E+2N)/4][(M+N)/2] when track_m != 0. */
int orc_tm_ising(int L, int track_m, uint64_t *out);
int orc_tm_potts(int L, int q, uint64_t *out /* index E+2N */);

/* Polymer (Eq. 7 reading, see polymer_oracle.c).  Handles are opaque. */
void *orc_poly_create(int N, int p, uint64_t seed, double e_lo, double e_hi, double K, double R, int record);
void orc_poly_free(void *h);
int orc_poly_num_bins(void *h);
void orc_poly_set_beta(void *h, double beta);
void orc_poly_set_model(void *h, int model); /* 1: the paper's parameters (Eq. 7); before init */
void orc_poly_set_moves(void *h, int moves); /* 1: shifts and spherical rotations */
int orc_poly_set_grid(void *h, int bin_k, double step_q); /* bin width 1/bin_k, cube side step_q/4096; before init */
void orc_poly_init(void *h);
void orc_poly_iterate(void *h, int64_t sweeps, int nthreads);
void orc_poly_iterate_range(void *h, int64_t sweeps, int w0, int w1, int nthreads);
void orc_poly_advance(void *h, int64_t sweeps);
void orc_poly_update(void *h);
double orc_poly_refresh_energy(void *h);
void orc_poly_get_lnW(void *h, double *out);
void orc_poly_get_lnW_sampled(void *h, double *out);
void orc_poly_get_histogram(void *h, uint64_t *out);
void orc_poly_get_coords(void *h, double *out /* p*N*3 */);
void orc_poly_get_energy(void *h, double *out /* p */);
void orc_poly_get_bins(void *h, int32_t *out /* p */);
void orc_poly_get_counters(void *h, int64_t *out /* {near-tie acceptances, bin-edge events} */);
void orc_poly_reweight(void *h, double beta, double out[4], double *lnP /* nullable, B */);
void orc_poly_get_walker_events(void *h, int64_t *out /* p*2 */);
void orc_poly_get_metrics(void *h, uint64_t out[5]); /* as orc_get_metrics; ends: bins 0 and B-1 */
double orc_poly_energy(int N, const double *X, int model); /* model 0 benchmark, 1 paper */
/* One attempt of the polymer trace: energy change (NaN if a bond broke or a
 * rotation found no point), its error scale S, the energy after the decision
 * and the bound delta after it, bins of the proposed and of the kept energy,
 * flags (1 accepted, 2 broken, 4 event, 8 started inside the window). */
typedef struct {
    double dE, scale, E, delta;
    int32_t bin_new, bin_after, flags, pad;
} orc_poly_trace_rec;
void orc_poly_get_first_events(void *h, int64_t *out /* p */);
double orc_poly_get_drift(void *h);
void orc_poly_get_delta(void *h, double *out /* p */);
void orc_poly_set_trace(void *h, orc_poly_trace_rec *buf);
void orc_poly_set_tau(void *h, double tau);
void orc_poly_set_perturbation(void *h, double perturb, uint64_t seed); /* tests of the event rule */
void orc_poly_set_lnW(void *h, const double *lnW);
double orc_poly_pair_scale(double r, int sep, int model);
double orc_poly_pair(double r, int sep, int model);

#ifdef __cplusplus
}
#endif
#endif
