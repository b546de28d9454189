/*
 * polymer_oracle.c -- plain CPU oracle of the multicanonical simulation of a
 * single flexible bead-spring polymer (paper: polymer paragraph, Eq. 7).
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the bench).
 *
 * Hamiltonian (reading of Eq. 7 with the benchmark's parameters):
 *   E = sum_{|i-j| >= 2} V_LJ(r_ij) + sum_i V_FENE(r_{i,i+1})
 *   V_LJ(r)   = 4 [(1/r)^12 - (1/r)^6] - V_LJ(rc),  r < rc = 2.5, else 0
 *               (eps = sigma = 1, truncated and shifted)
 *   V_FENE(r) = -(K/2) R^2 ln(1 - (r/R)^2),  r < R, else +infinity (move rejected)
 *               (K = 40, R = 1.5, bond rest length 0)
 * Move: beads i = 0..N-1 in order; bead i is displaced by
 *   delta_a = (u_a - 2^31) * Q * 2^-44,  a = x, y, z,  Q = 1229 by default,
 * i.e. uniform in a cube of side Q/4096 (0.30005) on a dyadic grid of
 * spacing Q * 2^-44, so every coordinate stays an exact binary64 value and
 * any implementation that adds the same integers lands on the same bits.
 * orc_poly_set_grid takes another cube side (as Q = round(side * 4096)).
 * Random words: Philox4x32-10, counter (bead, global sweep, walker, tag 1),
 * words 0..2 the displacement, word 3 the acceptance.
 * Energy bins: b = floor((E - e_lo) * k), width 1/k (k = 10 by default, any
 * integer k >= 1 through orc_poly_set_grid); the window is
 * 0 <= b < B.  Inside the window a move to E' is accepted iff b' is inside and
 * (d >= 0 or u_3 < floor(2^32 exp(d))), d = ln W(b') - ln W(b); outside the
 * window (walk-in after the start) a move is accepted iff it does not increase
 * the distance of E to the window, and nothing is recorded.  In canonical mode
 * (beta > 0) the weight is exp(-beta E) and there is no window.
 * After each call that runs sweeps, every chain is shifted so that bead 0 sits
 * at the origin (an exact shift by a grid vector, so coordinates stay well
 * inside the range where binary64 holds the grid exactly).
 * Initial chain: bead 0 at the origin; bead k = bead k-1 + b0 u_hat, with u_hat
 * a unit vector from Marsaglia's (1972) method on Philox tag-2 words, rounded
 * to the 2^-44 grid; redrawn (up to 64 times) while any earlier bead lies
 * closer than 0.9 b0 (b0 = 1 here, the rest length 0.7 in model 1).
 *
 * Model 1 (the paper's own parameters of Eq. 7): the same sums with
 *   V_LJ(r)   = 4 [(sigma/r)^12 - (sigma/r)^6], sigma = 2^(-1/6) r0, no cutoff,
 *   V_FENE(r) = -(K/2) R^2 ln(1 - ((r - r0)/R)^2), |r - r0| < R, else +infinity,
 *   K = 40, r0 = 0.7, R = r_max - r0 = 0.3 (r_max = 1).
 *
 * Move set 1 (the paper combines single-bead shifts with spherical rotations):
 * at bead i a second Philox block (counter (i, sweep, walker, tag 3)) picks the
 * move: word 0 < 2^31 the shift above, else a spherical rotation.  The pivot is
 * bead i+1 (i = 0), i-1 (i = N-1), otherwise i+1 if word 1 is odd, else i-1;
 * bead i goes to pivot + d n, d = |r_i - r_pivot|, n a unit vector from
 * Marsaglia's method on (word 2, word 3) and, after a rejected pair, on the
 * words of blocks (64 i + t, sweep, walker, tag 4), two pairs a block, at most
 * 64 pairs (none accepted: the move is rejected).  Every step is a correctly
 * rounded binary64 operation, and the offset is rounded to the grid.
 *
 * Energy refresh: after each call that runs sweeps, every walker's energy is
 * recomputed from scratch (the largest change is kept as the drift), so a
 * running sum carries its rounding only within one call.
 *
 * Events (trajectory parity with an implementation whose pair terms are FP32):
 * the oracle's decisions are exact functions of binary64 energies, so an
 * implementation that evaluates the pair terms in lower precision can decide
 * differently only where a decision is within its error of a boundary.  Its
 * error is bounded per pair term by tau * sigma(r), with the first-order error
 * scale sigma(r) = |v(r)| + |r v'(r)| (rounding of the value plus the error of
 * the separation carried through the potential), tau = 1e-6 by default (the
 * tolerance of the energy change, relative to the size of its terms).  Per
 * walker the oracle keeps delta, a bound on |E_impl - E|: tau * sum over all
 * pairs of sigma at the start and after each refresh, plus tau * S + rho for
 * every accepted move (S = sum of sigma over the move's old and new pair
 * terms, rho = 32 * 2^-32 for the rounding of a fixed-point energy change
 * summed over at most 32 lanes).  An attempt is an event when
 *   - its acceptance test is a near tie, |u_3 2^-32 - p_acc| < 1e-6;
 *   - its new energy lies within delta + tau * S + rho of a bin edge of the
 *     window (edges 0 .. B), so the new bin may differ;
 *   - outside the window, the two distances to the window differ by less than
 *     2 delta + tau * S + rho (the walk-in decision may differ);
 *   - a bond of the move is within 1e-5 (relative) of breaking, or the move's
 *     terms are so large (S > 2^21) that a lower-precision sum may overflow;
 * and the refresh at the end of a call is an event when the refreshed energy
 * lies within the new delta of a bin edge.  The oracle records each walker's
 * first event of a call (attempt index sweep * N + bead, N * sweeps for the
 * refresh) and, on request, a trace of every attempt.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "muca_oracle.h"

#define POLY_TAG_SWEEP 1u
#define POLY_TAG_INIT 2u
#define POLY_TAG_MOVE 3u
#define POLY_TAG_SPHERE 4u
#define POLY_STEP_Q 1229.0 /* default cube side 1229/4096 */
#define POLY_BIN_K 10      /* default bins per unit energy (width 0.1) */
#define POLY_GRID 0x1p-44
#define POLY_RC 2.5
#define POLY_PAPER_R0 0.7
#define POLY_PAPER_R 0.3

typedef struct {
    int N, p, B, record;
    uint64_t seed;
    double e_lo, e_hi, K, R, beta;
    int bin_k;        /* bins per unit energy (width 1/bin_k) */
    double step_q;    /* displacement grid units per unit of (u - 2^31) */
    int model;        /* 0: benchmark parameters, 1: the paper's (Eq. 7) */
    int moves;        /* 0: single-bead shifts, 1: shifts and spherical rotations */
    double r0, sigma2; /* model 1: FENE rest length, LJ sigma^2 */
    int64_t sweep_counter;
    double *X;       /* p*N*3 */
    double *E;       /* p */
    double *lnW, *lnW_sampled, *G, *lnR;
    uint64_t *H_open, *H_last;
    int64_t *events; /* p*2: [near-tie acceptances, bin-edge events] */
    /* metrics, as in the spin oracle: per walker accepted moves and tunnelling
     * events (bins 0 and B-1, sampled at the end of every sweep) of the open
     * iteration, and the end visited last (0 none, 1 bin 0, 2 bin B-1) */
    uint64_t *acc_w, *ev_w;
    uint8_t *tun;
    uint64_t m_last[2], m_total[2];
    int64_t sweeps_last, sweep_at_update;
    /* events: tolerance per unit of error scale, per-walker energy bounds, first event of the
     * last call, largest refresh change; optional per-attempt trace of the next call */
    double tau;
    double *delta;
    int64_t *first;
    double *drift;
    orc_poly_trace_rec *trace;
    int trace_w0; /* walker whose records start the trace buffer (ranged calls) */
    /* planted error for the tests of the event rule: every pair term of a move and
     * of a from-scratch energy is changed by perturb * sigma * xi, xi in [-1, 1)
     * from a Philox word (tag 7, key perturb_seed); 0 = off */
    double perturb;
    uint64_t perturb_seed;
} orc_poly;

#define POLY_TAG_PERTURB 7u

#define POLY_RHO (32.0 * 0x1p-32)

static double poly_lj(double r2)
{
    if (r2 >= POLY_RC * POLY_RC) return 0.0;
    double ir2 = 1.0 / r2;
    double ir6 = ir2 * ir2 * ir2;
    double irc2 = 1.0 / (POLY_RC * POLY_RC);
    double irc6 = irc2 * irc2 * irc2;
    return 4.0 * (ir6 * ir6 - ir6) - 4.0 * (irc6 * irc6 - irc6);
}

static double poly_fene(double r2, double K, double R)
{
    if (r2 >= R * R) return INFINITY;
    return -0.5 * K * R * R * log(1.0 - r2 / (R * R));
}

/* Model 1 (Eq. 7 with the paper's parameters). */
static double poly_paper_sigma2(void) { return POLY_PAPER_R0 * POLY_PAPER_R0 * pow(2.0, -1.0 / 3.0); }

static double poly_lj_paper(double r2, double sigma2)
{
    double s2 = sigma2 / r2;
    double s6 = s2 * s2 * s2;
    return 4.0 * (s6 * s6 - s6);
}

static double poly_fene_paper(double r2, double K, double R, double r0)
{
    double x = (sqrt(r2) - r0) / R;
    if (!(fabs(x) < 1.0)) return INFINITY;
    return -0.5 * K * R * R * log(1.0 - x * x);
}

static double poly_pair_model(double r2, int sep, int model)
{
    if (model == 1)
        return sep == 1 ? poly_fene_paper(r2, 40.0, POLY_PAPER_R, POLY_PAPER_R0) : poly_lj_paper(r2, poly_paper_sigma2());
    return sep == 1 ? poly_fene(r2, 40.0, 1.5) : poly_lj(r2);
}

/* Pair energy at distance r for index separation sep (1 = bond, >= 2 = LJ);
 * model 0 benchmark, 1 the paper's parameters. */
double orc_poly_pair(double r, int sep, int model) { return poly_pair_model(r * r, sep, model); }

static double poly_pair2(const orc_poly *P, double r2, int sep)
{
    if (P->model == 1) return sep == 1 ? poly_fene_paper(r2, P->K, P->R, P->r0) : poly_lj_paper(r2, P->sigma2);
    return sep == 1 ? poly_fene(r2, P->K, P->R) : poly_lj(r2);
}

static double poly_dist2(const double *a, const double *b)
{
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return dx * dx + dy * dy + dz * dz;
}

/* First-order error scale sigma(r) = |v(r)| + |r v'(r)| of a pair term at squared
 * distance r2 (0 for an LJ pair beyond the cutoff, +inf for a broken bond). */
static double poly_pair_scale(const orc_poly *P, double r2, int sep)
{
    if (sep == 1) {
        const double c = 0.5 * P->K * P->R * P->R;
        if (P->model == 1) {
            const double r = sqrt(r2), y = (r - P->r0) / P->R, g = 1.0 - y * y;
            if (!(g > 0.0)) return INFINITY;
            return c * (fabs(log(g)) + 2.0 * fabs(y) * r / (P->R * g));
        }
        const double x = r2 / (P->R * P->R), g = 1.0 - x;
        if (!(g > 0.0)) return INFINITY;
        return c * (fabs(log(g)) + 2.0 * x / g);
    }
    if (P->model == 1) {
        const double s2 = P->sigma2 / r2, s6 = s2 * s2 * s2;
        return 4.0 * (13.0 * s6 * s6 + 7.0 * s6);
    }
    if (r2 >= POLY_RC * POLY_RC) return 0.0;
    const double i2 = 1.0 / r2, i6 = i2 * i2 * i2;
    const double irc2 = 1.0 / (POLY_RC * POLY_RC), irc6 = irc2 * irc2 * irc2;
    return 4.0 * (13.0 * i6 * i6 + 7.0 * i6) + 4.0 * fabs(irc6 * irc6 - irc6);
}

/* Planted error of a pair term (tests of the event rule only): perturb * sigma * xi with
 * xi = u 2^-31 - 1 from the Philox word of counter (c0, c1, c2, tag 7). */
static double poly_perturbation(const orc_poly *P, double sigma, uint32_t c0, uint32_t c1, uint32_t c2)
{
    if (P->perturb == 0.0 || !(sigma < INFINITY)) return 0.0;
    uint32_t key[2] = {(uint32_t)(P->perturb_seed & 0xffffffffu), (uint32_t)(P->perturb_seed >> 32)};
    uint32_t ctr[4] = {c0, c1, c2, POLY_TAG_PERTURB}, u[4];
    orc_philox4x32_10(ctr, key, u);
    return P->perturb * sigma * ((double)u[0] * 0x1p-31 - 1.0);
}

/* Sum of sigma over all pairs of a configuration. */
static double poly_scale_all(const orc_poly *P, const double *X)
{
    double S = 0.0;
    for (int i = 0; i < P->N; ++i)
        for (int j = i + 1; j < P->N; ++j) S += poly_pair_scale(P, poly_dist2(X + 3 * i, X + 3 * j), j - i);
    return S;
}

/* Is E within m of a bin edge of the window (e_lo + k / bin_k, k = 0 .. B)? */
static int poly_near_edge(const orc_poly *P, double E, double m)
{
    const double t = (E - P->e_lo) * (double)P->bin_k, k = nearbyint(t);
    return k >= 0.0 && k <= (double)P->B && fabs(t - k) < (double)P->bin_k * m;
}

/* A bond of squared length r2 within 1e-5 (relative) of breaking. */
static int poly_bond_near_break(const orc_poly *P, double r2)
{
    if (P->model == 1) return fabs(fabs(sqrt(r2) - P->r0) / P->R - 1.0) < 1e-5;
    return fabs(r2 / (P->R * P->R) - 1.0) < 1e-5;
}

/* Energy of one configuration from scratch, pairs i < j in order. */
double orc_poly_energy(int N, const double *X, int model)
{
    double E = 0.0;
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) E += poly_pair_model(poly_dist2(X + 3 * i, X + 3 * j), j - i, model);
    return E;
}

static double poly_energy_P(const orc_poly *P, const double *X)
{
    double E = 0.0;
    for (int i = 0; i < P->N; ++i)
        for (int j = i + 1; j < P->N; ++j) E += poly_pair2(P, poly_dist2(X + 3 * i, X + 3 * j), j - i);
    return E;
}

/* The same with the planted error of the tests of the event rule (tag word 2^31 + pair index,
 * sweep counter g, walker w). */
static double poly_energy_perturbed(const orc_poly *P, const double *X, uint32_t g, int w)
{
    double E = poly_energy_P(P, X);
    if (P->perturb == 0.0) return E;
    for (int i = 0; i < P->N; ++i)
        for (int j = i + 1; j < P->N; ++j) {
            const double r2 = poly_dist2(X + 3 * i, X + 3 * j);
            E += poly_perturbation(P, poly_pair_scale(P, r2, j - i), 0x80000000u + (uint32_t)(i * P->N + j), g,
                                   (uint32_t)w);
        }
    return E;
}

/* Bin of E, clamped to [-1, B] (below / above the window) so that energies far
 * outside it (overlapping beads) cannot overflow the conversion. */
static int poly_bin(const orc_poly *P, double E)
{
    double t = floor((E - P->e_lo) * (double)P->bin_k);
    if (!(t >= -1.0)) return -1;
    if (t > (double)P->B) return P->B;
    return (int)t;
}

void *orc_poly_create(int N, int p, uint64_t seed, double e_lo, double e_hi, double K, double R, int record)
{
    if (N < 2 || p < 1 || !(e_hi > e_lo) || !(K > 0) || !(R > 0)) return NULL;
    orc_poly *P = (orc_poly *)calloc(1, sizeof *P);
    P->N = N;
    P->p = p;
    P->seed = seed;
    P->e_lo = e_lo;
    P->e_hi = e_hi;
    P->K = K;
    P->R = R;
    P->record = record;
    P->bin_k = POLY_BIN_K;
    P->step_q = POLY_STEP_Q;
    P->B = (int)floor((e_hi - e_lo) * (double)P->bin_k + 0.5);
    if (P->B < 2) { free(P); return NULL; }
    P->X = (double *)calloc((size_t)p * N * 3, sizeof(double));
    P->E = (double *)calloc((size_t)p, sizeof(double));
    P->lnW = (double *)calloc((size_t)P->B, sizeof(double));
    P->lnW_sampled = (double *)calloc((size_t)P->B, sizeof(double));
    P->G = (double *)calloc((size_t)P->B, sizeof(double));
    P->lnR = (double *)calloc((size_t)P->B, sizeof(double));
    P->H_open = (uint64_t *)calloc((size_t)P->B, sizeof(uint64_t));
    P->H_last = (uint64_t *)calloc((size_t)P->B, sizeof(uint64_t));
    P->events = (int64_t *)calloc((size_t)p * 2, sizeof(int64_t));
    P->acc_w = (uint64_t *)calloc((size_t)p, sizeof(uint64_t));
    P->ev_w = (uint64_t *)calloc((size_t)p, sizeof(uint64_t));
    P->tun = (uint8_t *)calloc((size_t)p, 1);
    P->tau = 1e-6;
    P->delta = (double *)calloc((size_t)p, sizeof(double));
    P->first = (int64_t *)calloc((size_t)p, sizeof(int64_t));
    P->drift = (double *)calloc((size_t)p, sizeof(double));
    for (int w = 0; w < p; ++w) P->first[w] = -1;
    return P;
}

void orc_poly_free(void *h)
{
    orc_poly *P = (orc_poly *)h;
    if (!P) return;
    free(P->X); free(P->E); free(P->lnW); free(P->lnW_sampled); free(P->G); free(P->lnR);
    free(P->H_open); free(P->H_last); free(P->events);
    free(P->acc_w); free(P->ev_w); free(P->tun);
    free(P->delta); free(P->first); free(P->drift);
    free(P);
}

int orc_poly_num_bins(void *h) { return ((orc_poly *)h)->B; }

/* Canonical mode for the window pilot: weight exp(-beta E), no window. */
void orc_poly_set_beta(void *h, double beta) { ((orc_poly *)h)->beta = beta; }

void orc_poly_set_moves(void *h, int moves) { ((orc_poly *)h)->moves = moves; }

/* Bins of width 1/bin_k and a cube of side step_q/4096 for the moves (before init).  The
 * window keeps its edges; the bin count and every per-bin array follow.  Returns the new bin
 * count, or -1 for bin_k < 1, step_q < 1 or a window of fewer than 2 bins. */
int orc_poly_set_grid(void *h, int bin_k, double step_q)
{
    orc_poly *P = (orc_poly *)h;
    if (bin_k < 1 || !(step_q >= 1.0) || step_q != floor(step_q)) return -1;
    const int B = (int)floor((P->e_hi - P->e_lo) * (double)bin_k + 0.5);
    if (B < 2) return -1;
    P->bin_k = bin_k;
    P->step_q = step_q;
    if (B != P->B) {
        P->B = B;
        double **d[4] = {&P->lnW, &P->lnW_sampled, &P->G, &P->lnR};
        for (int i = 0; i < 4; ++i) {
            free(*d[i]);
            *d[i] = (double *)calloc((size_t)B, sizeof(double));
        }
        free(P->H_open);
        free(P->H_last);
        P->H_open = (uint64_t *)calloc((size_t)B, sizeof(uint64_t));
        P->H_last = (uint64_t *)calloc((size_t)B, sizeof(uint64_t));
    }
    return B;
}

/* Spherical rotation of bead i of walker w (move set 1): the new position on
 * the grid in xn, or 0 if Marsaglia's method found no point in 64 pairs. */
static int poly_rotation(const orc_poly *P, const double *X, int i, int w, uint32_t g, const uint32_t m[4],
                         double xn[3])
{
    const int N = P->N;
    uint32_t key[2] = {(uint32_t)(P->seed & 0xffffffffu), (uint32_t)(P->seed >> 32)};
    int pv = (i == 0) ? 1 : (i == N - 1) ? N - 2 : ((m[1] & 1u) ? i + 1 : i - 1);
    double v1 = 0.0, v2 = 0.0, s = 0.0;
    int found = 0;
    uint32_t blk[4] = {0, 0, m[2], m[3]};
    for (int t = 0; t < 64 && !found; ++t) {
        if (t > 0 && (t & 1) == 1) {
            uint32_t ctr[4] = {(uint32_t)(64 * i + (t >> 1)), g, (uint32_t)w, POLY_TAG_SPHERE};
            orc_philox4x32_10(ctr, key, blk);
        }
        uint32_t a = (t == 0) ? m[2] : blk[(t & 1) ? 0 : 2];
        uint32_t b = (t == 0) ? m[3] : blk[(t & 1) ? 1 : 3];
        v1 = (double)a * 0x1p-31 - 1.0;
        v2 = (double)b * 0x1p-31 - 1.0;
        s = v1 * v1 + v2 * v2;
        found = (s < 1.0 && s > 0.0);
    }
    if (!found) return 0;
    double f = 2.0 * sqrt(1.0 - s);
    double n[3] = {v1 * f, v2 * f, 1.0 - 2.0 * s};
    const double *xp = X + 3 * pv, *xi = X + 3 * i;
    double dx = xi[0] - xp[0], dy = xi[1] - xp[1], dz = xi[2] - xp[2];
    double d = sqrt((dx * dx + dy * dy) + dz * dz);
    for (int a = 0; a < 3; ++a) xn[a] = xp[a] + nearbyint((n[a] * d) * 0x1p44) * POLY_GRID;
    return 1;
}

/* Model 1: the paper's parameters (K = 40, r0 = 0.7, r_max = 1, LJ without cutoff);
 * before orc_poly_init. */
void orc_poly_set_model(void *h, int model)
{
    orc_poly *P = (orc_poly *)h;
    P->model = model;
    if (model == 1) {
        P->K = 40.0;
        P->R = POLY_PAPER_R;
        P->r0 = POLY_PAPER_R0;
        P->sigma2 = poly_paper_sigma2();
    }
}

void orc_poly_init(void *h)
{
    orc_poly *P = (orc_poly *)h;
    const int N = P->N;
    const double b0 = (P->model == 1) ? POLY_PAPER_R0 : 1.0;  /* initial bond length */
    const double d2min = (P->model == 1) ? 0.3969 : 0.81;      /* (0.9 b0)^2 */
    uint32_t key[2] = {(uint32_t)(P->seed & 0xffffffffu), (uint32_t)(P->seed >> 32)};
    for (int w = 0; w < P->p; ++w) {
        double *X = P->X + (size_t)w * N * 3;
        X[0] = X[1] = X[2] = 0.0;
        uint32_t draw = 0; /* counts Philox blocks drawn for this walker */
        for (int k = 1; k < N; ++k) {
            double cand[3] = {0, 0, 0};
            for (int attempt = 0; attempt < 64; ++attempt) {
                /* Marsaglia: v1, v2 uniform in [-1, 1) with s = v1^2 + v2^2 < 1 */
                double v1, v2, s;
                for (;;) {
                    uint32_t ctr[4] = {draw++, 0u, (uint32_t)w, POLY_TAG_INIT}, u[4];
                    orc_philox4x32_10(ctr, key, u);
                    v1 = (double)u[0] * 0x1p-31 - 1.0;
                    v2 = (double)u[1] * 0x1p-31 - 1.0;
                    s = v1 * v1 + v2 * v2;
                    if (s < 1.0 && s > 0.0) break;
                }
                double f = 2.0 * sqrt(1.0 - s);
                double uh[3] = {v1 * f, v2 * f, 1.0 - 2.0 * s};
                for (int a = 0; a < 3; ++a)
                    cand[a] = X[3 * (k - 1) + a] + nearbyint((uh[a] * b0) * 0x1p44) * POLY_GRID;
                int ok = 1;
                for (int j = 0; j < k - 1 && ok; ++j)
                    if (poly_dist2(cand, X + 3 * j) < d2min) ok = 0;
                if (ok) break;
            }
            for (int a = 0; a < 3; ++a) X[3 * k + a] = cand[a];
        }
        P->E[w] = poly_energy_perturbed(P, X, 0u, w);
        P->delta[w] = P->tau * poly_scale_all(P, X) + POLY_RHO;
        P->first[w] = -1;
        P->drift[w] = 0.0;
    }
    for (int b = 0; b < P->B; ++b) {
        P->lnW[b] = P->lnW_sampled[b] = P->G[b] = P->lnR[b] = 0.0;
        P->H_open[b] = P->H_last[b] = 0;
    }
    P->sweep_counter = 0;
    for (int w = 0; w < P->p; ++w) {
        P->acc_w[w] = P->ev_w[w] = 0;
        P->tun[w] = 0;
    }
    P->m_last[0] = P->m_last[1] = P->m_total[0] = P->m_total[1] = 0;
    P->sweeps_last = P->sweep_at_update = 0;
}

static double poly_window_dist(const orc_poly *P, double E)
{
    int b = poly_bin(P, E);
    if (b >= 0 && b < P->B) return 0.0;
    return (b < 0) ? (P->e_lo - E) : (E - P->e_hi);
}

static void poly_walker_sweeps(orc_poly *P, int w, int64_t g0, int64_t sweeps, uint64_t *hist)
{
    const int N = P->N;
    double *X = P->X + (size_t)w * N * 3;
    double E = P->E[w];
    int64_t *ev = P->events + 2 * (size_t)w;
    const int muca = P->beta <= 0.0;
    int64_t first = -1; /* first event of this call (attempt index) */
    uint32_t key[2] = {(uint32_t)(P->seed & 0xffffffffu), (uint32_t)(P->seed >> 32)};
    for (int64_t sw = 0; sw < sweeps; ++sw) {
        uint32_t g = (uint32_t)(g0 + sw);
        for (int i = 0; i < N; ++i) {
            uint32_t ctr[4] = {(uint32_t)i, g, (uint32_t)w, POLY_TAG_SWEEP}, u[4];
            orc_philox4x32_10(ctr, key, u);
            double xn[3] = {X[3 * i], X[3 * i + 1], X[3 * i + 2]};
            int rotation = 0, broken = 0, event = 0;
            if (P->moves == 1) {
                uint32_t mc[4] = {(uint32_t)i, g, (uint32_t)w, POLY_TAG_MOVE}, mw[4];
                orc_philox4x32_10(mc, key, mw);
                rotation = mw[0] >= 0x80000000u;
                if (rotation && !poly_rotation(P, X, i, w, g, mw, xn)) broken = 1; /* no point: rejected */
            }
            if (!rotation)
                for (int a = 0; a < 3; ++a)
                    xn[a] = X[3 * i + a] + (double)((int64_t)u[a] - 2147483648LL) * P->step_q * POLY_GRID;
            /* energy change and its error scale S (old and new pair terms) */
            double dE = 0.0, S = 0.0;
            for (int j = 0; j < N; ++j) {
                if (j == i) continue;
                int sep = abs(i - j);
                double r2n = poly_dist2(xn, X + 3 * j), r2o = poly_dist2(X + 3 * i, X + 3 * j);
                double vn = poly_pair2(P, r2n, sep);
                double vo = poly_pair2(P, r2o, sep);
                if (isinf(vn)) broken = 1;
                if (sep == 1 && poly_bond_near_break(P, r2n)) event = 1;
                const double so = poly_pair_scale(P, r2o, sep), sn = isinf(vn) ? 0.0 : poly_pair_scale(P, r2n, sep);
                S += so + sn;
                if (P->perturb != 0.0 && !isinf(vn)) {
                    const uint32_t pj = (uint32_t)(2 * (i * N + j));
                    vo += poly_perturbation(P, so, pj, g, (uint32_t)w);
                    vn += poly_perturbation(P, sn, pj + 1u, g, (uint32_t)w);
                }
                dE += vn - vo;
            }
            int accept = 0;
            double En = E + dE;
            const int b = muca ? poly_bin(P, E) : 0, inside = muca && b >= 0 && b < P->B;
            const double m = P->delta[w] + P->tau * S + POLY_RHO;
            if (muca && !broken && S > 0x1p21) event = 1;
            if (!broken) {
                if (!muca) {
                    double d = -P->beta * dE;
                    accept = d >= 0.0 || (double)u[3] < floor(ldexp(orc_det_exp(d), 32));
                } else {
                    int bn = poly_bin(P, En);
                    if (poly_near_edge(P, En, m)) {
                        /* the new energy is within the implementation's error of a bin edge */
                        event = 1;
                        ev[1] += 1;
                    }
                    if (inside) {
                        if (bn >= 0 && bn < P->B) {
                            double d = P->lnW[bn] - P->lnW[b];
                            if (d >= 0.0) {
                                accept = 1;
                            } else {
                                double pa = orc_det_exp(d);
                                accept = (double)u[3] < floor(ldexp(pa, 32));
                                if (fabs((double)u[3] * 0x1p-32 - pa) < 1e-6) {
                                    event = 1;
                                    ev[0] += 1;
                                }
                            }
                        }
                    } else {
                        double dn = poly_window_dist(P, En), dd = poly_window_dist(P, E);
                        accept = dn <= dd;
                        if (fabs(dn - dd) < P->delta[w] + m) event = 1;
                    }
                }
            }
            if (event && first < 0) first = sw * N + i;
            if (accept) {
                for (int a = 0; a < 3; ++a) X[3 * i + a] = xn[a];
                E = En;
                P->acc_w[w] += 1;
                if (muca) P->delta[w] += P->tau * S + POLY_RHO;
            }
            if (P->trace) {
                orc_poly_trace_rec *t =
                    P->trace + ((size_t)(w - P->trace_w0) * (size_t)sweeps + (size_t)sw) * (size_t)N + i;
                t->dE = broken ? NAN : dE;
                t->scale = S;
                t->E = E;
                t->delta = P->delta[w];
                t->bin_new = muca ? poly_bin(P, En) : 0;
                t->bin_after = muca ? poly_bin(P, E) : 0;
                t->flags = (accept ? 1 : 0) | (broken ? 2 : 0) | (event ? 4 : 0) | (inside ? 8 : 0);
                t->pad = 0;
            }
            if (P->record == 0 && muca) {
                int bb = poly_bin(P, E);
                if (bb >= 0 && bb < P->B) hist[bb] += 1;
            }
        }
        if (P->record == 1 && muca) {
            int bb = poly_bin(P, E);
            if (bb >= 0 && bb < P->B) hist[bb] += 1;
        }
        {
            const int bb = poly_bin(P, E);
            if (bb == 0) {
                if (P->tun[w] == 2) P->ev_w[w] += 1;
                P->tun[w] = 1;
            } else if (bb == P->B - 1) {
                if (P->tun[w] == 1) P->ev_w[w] += 1;
                P->tun[w] = 2;
            }
        }
    }
    /* recentre on bead 0 (an exact shift by a grid vector: energies are unchanged) */
    double c[3] = {X[0], X[1], X[2]};
    for (int j = 0; j < N; ++j)
        for (int a = 0; a < 3; ++a) X[3 * j + a] -= c[a];
    /* refresh the running energy from scratch; the new bound is that of a from-scratch sum */
    if (sweeps > 0) {
        const double e = poly_energy_perturbed(P, X, (uint32_t)(g0 + sweeps), w);
        if (fabs(e - E) > P->drift[w]) P->drift[w] = fabs(e - E);
        E = e;
        P->delta[w] = P->tau * poly_scale_all(P, X) + POLY_RHO;
        if (muca && first < 0 && poly_near_edge(P, E, P->delta[w])) first = sweeps * N;
    }
    P->E[w] = E;
    P->first[w] = first;
}

typedef struct {
    orc_poly *P;
    int w0, w1;
    int64_t g0, sweeps;
    uint64_t *hist;
} poly_job;

static void *poly_job_main(void *arg)
{
    poly_job *j = (poly_job *)arg;
    for (int w = j->w0; w < j->w1; ++w) poly_walker_sweeps(j->P, w, j->g0, j->sweeps, j->hist);
    return NULL;
}

void orc_poly_iterate_range(void *h, int64_t sweeps, int w0, int w1, int nthreads)
{
    orc_poly *P = (orc_poly *)h;
    if (w0 < 0) w0 = 0;
    if (w1 > P->p) w1 = P->p;
    if (w1 <= w0 || sweeps <= 0) return;
    P->trace_w0 = w0; /* a trace of this call holds walkers w0 .. w1-1 */
    int nw = w1 - w0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nw) nthreads = nw;
    poly_job *jobs = (poly_job *)calloc((size_t)nthreads, sizeof *jobs);
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof *th);
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].P = P;
        jobs[t].w0 = w0 + (int)((int64_t)nw * t / nthreads);
        jobs[t].w1 = w0 + (int)((int64_t)nw * (t + 1) / nthreads);
        jobs[t].g0 = P->sweep_counter;
        jobs[t].sweeps = sweeps;
        jobs[t].hist = (uint64_t *)calloc((size_t)P->B, sizeof(uint64_t));
    }
    if (nthreads == 1) {
        poly_job_main(&jobs[0]);
    } else {
        for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, poly_job_main, &jobs[t]);
        for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    }
    for (int t = 0; t < nthreads; ++t) {
        for (int b = 0; b < P->B; ++b) P->H_open[b] += jobs[t].hist[b];
        free(jobs[t].hist);
    }
    free(jobs);
    free(th);
}

void orc_poly_advance(void *h, int64_t sweeps) { ((orc_poly *)h)->sweep_counter += sweeps; }

void orc_poly_iterate(void *h, int64_t sweeps, int nthreads)
{
    orc_poly_iterate_range(h, sweeps, 0, ((orc_poly *)h)->p, nthreads);
    orc_poly_advance(h, sweeps);
}

/* Same accumulated-statistics recursion as the spin oracle, over all B bins. */
void orc_poly_get_metrics(void *h, uint64_t out[5])
{
    orc_poly *P = (orc_poly *)h;
    out[0] = P->m_last[0];
    out[1] = P->m_last[1];
    out[2] = P->m_total[0];
    out[3] = P->m_total[1];
    out[4] = (uint64_t)P->sweeps_last;
}

void orc_poly_update(void *h)
{
    orc_poly *P = (orc_poly *)h;
    const int B = P->B;
    {
        uint64_t a = 0, e = 0;
        for (int w = 0; w < P->p; ++w) {
            a += P->acc_w[w];
            e += P->ev_w[w];
            P->acc_w[w] = P->ev_w[w] = 0;
        }
        P->m_last[0] = a;
        P->m_last[1] = e;
        P->m_total[0] += a;
        P->m_total[1] += e;
        P->sweeps_last = P->sweep_counter - P->sweep_at_update;
        P->sweep_at_update = P->sweep_counter;
    }
    memcpy(P->lnW_sampled, P->lnW, sizeof(double) * B);
    for (int k = 0; k + 1 < B; ++k) {
        uint64_t h0 = P->H_open[k], h1 = P->H_open[k + 1];
        if (h0 > 0 && h1 > 0) {
            double a = (double)h0, c = (double)h1;
            double g = (a * c) / (a + c);
            P->G[k] = P->G[k] + g;
            double kappa = g / P->G[k];
            double diff = orc_det_log(a) - orc_det_log(c);
            P->lnR[k] = P->lnR[k] + kappa * diff;
        }
    }
    double acc = 0.0;
    P->lnW[0] = acc;
    for (int k = 0; k + 1 < B; ++k) {
        acc = acc + P->lnR[k];
        P->lnW[k + 1] = acc;
    }
    memcpy(P->H_last, P->H_open, sizeof(uint64_t) * B);
    memset(P->H_open, 0, sizeof(uint64_t) * B);
}

/* Recompute every walker's energy from scratch (removes accumulated rounding);
 * returns the largest |E_running - E_scratch|. */
double orc_poly_refresh_energy(void *h)
{
    orc_poly *P = (orc_poly *)h;
    double worst = 0.0;
    for (int w = 0; w < P->p; ++w) {
        double e = poly_energy_P(P, P->X + (size_t)w * P->N * 3);
        double d = fabs(e - P->E[w]);
        if (d > worst) worst = d;
        P->E[w] = e;
    }
    return worst;
}

void orc_poly_get_lnW(void *h, double *out) { memcpy(out, ((orc_poly *)h)->lnW, sizeof(double) * ((orc_poly *)h)->B); }
void orc_poly_get_lnW_sampled(void *h, double *out)
{
    memcpy(out, ((orc_poly *)h)->lnW_sampled, sizeof(double) * ((orc_poly *)h)->B);
}
void orc_poly_get_histogram(void *h, uint64_t *out)
{
    memcpy(out, ((orc_poly *)h)->H_last, sizeof(uint64_t) * ((orc_poly *)h)->B);
}
void orc_poly_get_coords(void *h, double *out)
{
    orc_poly *P = (orc_poly *)h;
    memcpy(out, P->X, sizeof(double) * (size_t)P->p * P->N * 3);
}
void orc_poly_get_energy(void *h, double *out) { memcpy(out, ((orc_poly *)h)->E, sizeof(double) * ((orc_poly *)h)->p); }
void orc_poly_get_bins(void *h, int32_t *out)
{
    orc_poly *P = (orc_poly *)h;
    for (int w = 0; w < P->p; ++w) out[w] = poly_bin(P, P->E[w]);
}
void orc_poly_get_counters(void *h, int64_t *out)
{
    orc_poly *P = (orc_poly *)h;
    out[0] = out[1] = 0;
    for (int w = 0; w < P->p; ++w) {
        out[0] += P->events[2 * w];
        out[1] += P->events[2 * w + 1];
    }
}

/* Eq. (2) for the polymer with E at bin centres: out = {<E>, <E^2>, C_V per bead,
 * ln of <exp(-beta E)> over the estimated density of states normalised to 1}. */
void orc_poly_reweight(void *h, double beta, double out[4], double *lnP)
{
    orc_poly *P = (orc_poly *)h;
    const int B = P->B;
    double *x = (double *)malloc(sizeof(double) * B), *lo = (double *)malloc(sizeof(double) * B);
    double m = -INFINITY, m2 = -INFINITY;
    for (int b = 0; b < B; ++b) {
        x[b] = lo[b] = -INFINITY;
        if (P->H_last[b] == 0) continue;
        lo[b] = log((double)P->H_last[b]) - P->lnW_sampled[b];
        x[b] = lo[b] - beta * (P->e_lo + (b + 0.5) / (double)P->bin_k);
        if (x[b] > m) m = x[b];
        if (lo[b] > m2) m2 = lo[b];
    }
    double z = 0.0, z2 = 0.0;
    for (int b = 0; b < B; ++b)
        if (x[b] > -INFINITY) {
            z += exp(x[b] - m);
            z2 += exp(lo[b] - m2);
        }
    double lse = m + log(z), a1 = 0.0, a2 = 0.0;
    for (int b = 0; b < B; ++b) {
        double lp = (x[b] > -INFINITY) ? x[b] - lse : -INFINITY;
        if (lnP) lnP[b] = lp;
        if (x[b] == -INFINITY) continue;
        double E = P->e_lo + (b + 0.5) / (double)P->bin_k, pr = exp(lp);
        a1 += pr * E;
        a2 += pr * E * E;
    }
    out[0] = a1;
    out[1] = a2;
    out[2] = beta * beta * (a2 - a1 * a1) / P->N;
    out[3] = lse - (m2 + log(z2));
    free(x);
    free(lo);
}

void orc_poly_get_walker_events(void *h, int64_t *out)
{
    orc_poly *P = (orc_poly *)h;
    memcpy(out, P->events, sizeof(int64_t) * 2 * (size_t)P->p);
}

/* First event of each walker in the last call that ran sweeps (attempt index
 * sweep * N + bead within the call, sweeps * N for the refresh, -1 none). */
void orc_poly_get_first_events(void *h, int64_t *out)
{
    orc_poly *P = (orc_poly *)h;
    memcpy(out, P->first, sizeof(int64_t) * (size_t)P->p);
}

/* Largest change of a running energy at a refresh since init. */
double orc_poly_get_drift(void *h)
{
    orc_poly *P = (orc_poly *)h;
    double d = 0.0;
    for (int w = 0; w < P->p; ++w)
        if (P->drift[w] > d) d = P->drift[w];
    return d;
}

/* Per-walker energy bounds delta (see the header). */
void orc_poly_get_delta(void *h, double *out)
{
    orc_poly *P = (orc_poly *)h;
    memcpy(out, P->delta, sizeof(double) * (size_t)P->p);
}

/* Trace of every attempt of the next calls ((w1 - w0) * sweeps * N records for a
 * call over walkers [w0, w1), walker-major, then sweep, then bead), or NULL to
 * stop tracing. */
void orc_poly_set_trace(void *h, orc_poly_trace_rec *buf) { ((orc_poly *)h)->trace = buf; }

/* Tolerance of the pair terms per unit of error scale (default 1e-6); before init. */
void orc_poly_set_tau(void *h, double tau) { ((orc_poly *)h)->tau = tau; }

/* Planted error of the pair terms (tests of the event rule only), see orc_poly. */
void orc_poly_set_perturbation(void *h, double perturb, uint64_t seed)
{
    orc_poly *P = (orc_poly *)h;
    P->perturb = perturb;
    P->perturb_seed = seed;
}

/* Replace ln W (B doubles), e.g. to give two runs the same weights. */
void orc_poly_set_lnW(void *h, const double *lnW)
{
    orc_poly *P = (orc_poly *)h;
    memcpy(P->lnW, lnW, sizeof(double) * (size_t)P->B);
}

/* First-order error scale sigma(r) = |v| + |r v'| of a pair term (see the header). */
double orc_poly_pair_scale(double r, int sep, int model)
{
    orc_poly P;
    memset(&P, 0, sizeof P);
    P.K = 40.0;
    P.R = 1.5;
    P.model = model;
    if (model == 1) {
        P.R = POLY_PAPER_R;
        P.r0 = POLY_PAPER_R0;
        P.sigma2 = poly_paper_sigma2();
    }
    return poly_pair_scale(&P, r * r, sep);
}
