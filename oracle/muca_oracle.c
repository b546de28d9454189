/*
 * muca_oracle.c -- plain CPU oracle of the parallel multicanonical method
 * (Zierenberg, Marenz, Janke, arXiv:1312.2213).  TEST INFRASTRUCTURE ONLY:
 * only tests, the smoke check and the benchmark's CPU-baseline leg use it.
 *
 * What it follows, passage by passage:
 *   - MUCA ensemble, Eq. (1): states are sampled with weight W(E) instead of
 *     exp(-beta E); a move E -> E' is accepted with min(1, W(E')/W(E)).
 *   - Multimagnetic ensemble, Eq. (3): weight exp(-beta E) W(M).
 *   - Parallel scheme, Fig. 1 and the paragraph before it: p independent
 *     realisations share one W; after each iteration the p histograms are
 *     merged, a new W is computed and handed back to all p chains.
 *   - Weight recursion: the accumulated-statistics update in log form that the
 *     paper says all its runs use (paragraph after Eq. 2).
 *   - Ising Hamiltonian H = -J sum s_i s_j and q-state Potts Hamiltonian
 *     H = -J sum delta(s_i, s_j) (Ising / Potts paragraphs), J = 1, periodic.
 *   - Reweighting, Eq. (2).
 *
 * Readings where the paper is silent (each is also stated where it is used):
 *   R1 site order: sites i = y*L + x are visited in order 0..N-1 every sweep.
 *   R2 random numbers: Philox4x32-10, key = (seed lo, seed hi), counter =
 *      (word group, global sweep index, walker id, tag); tag 0 = init,
 *      tag 1 = sweep.  Ising/MUMA use one 32-bit word per attempt (group =
 *      site/4, word = site%4); Potts two (group = site/2, words 2*(site%2) for
 *      the proposal and 2*(site%2)+1 for the acceptance).
 *   R3 acceptance: accept iff T == 0xFFFFFFFF or u < T, with the integer
 *      threshold T = floor(2^32 * exp(d)) for d < 0 and 0xFFFFFFFF for d >= 0,
 *      d = ln W(target) - ln W(current) (MUMA: minus beta*dE as well).
 *   R4 histogram: after every attempt (accepted or not) the current bin is
 *      counted once (record = 0), or once per sweep after its last site
 *      (record = 1).
 *   R5 recursion (accumulated statistics in log form, over the ordered list of
 *      reachable bins r_0 < ... < r_{K-1}): for each neighbouring pair with
 *      h0 = H(r_k) > 0 and h1 = H(r_{k+1}) > 0,
 *         g = h0*h1/(h0+h1);  G_k += g;  kappa = g/G_k;
 *         lnR_k += kappa * (ln h0 - ln h1);
 *      then ln W(r_0) = 0, ln W(r_{k+1}) = ln W(r_k) + lnR_k summed in order.
 *      The first iteration with data has kappa = 1: the plain W/H update.
 *   R5' plain update (selectable, recursion = 1), the paper's simple rule
 *      W(n+1)(E) = W(n)(E) / H(n)(E) in log form over the reachable bins:
 *         x_k = ln W(r_k) - ln max(H(r_k), 1),  ln W(r_k) <- x_k - x_0,
 *      so an unvisited bin keeps its weight (H = 0 is taken as H = 1) and
 *      ln W(r_0) = 0 as in R5.
 *   R9 observables (Ising, optional): after each sweep every walker adds 1,
 *      |M| and M^2 (M = sum of its spins) to three sums of its current bin;
 *      Eq. (2) then reweights them with the weights they were sampled with.
 *   R6 reachable bins (even L >= 4, periodic): Ising has no state with
 *      exactly 2 or 2N-2 broken bonds; Potts (q >= 3) none with 1, 2, 3 or 5
 *      broken bonds; q = 2 Potts follows Ising.  Unreachable bins get
 *      ln W = -inf and are skipped by the recursion.
 *   R7 thermalisation: none for spins (the paper thermalises only at the
 *      start, and with ln W = 0 the first iteration samples beta = 0, where a
 *      uniformly random configuration is already an equilibrium sample).
 *   R8 Potts proposal: new = (old + 1 + mulhi32(u, q-1)) mod q, uniform over
 *      the q-1 other states.
 */
#include "muca_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, as published by Salmon et al. (SC'11): ten rounds of two
 * 32x32->64 multiplications with the Weyl key schedule between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------- */
/* Deterministic exp and log.  Both are written from the textbook methods
 * named below, with a fixed operation order (this file is compiled with
 * -ffp-contract=off), so that any other implementation that performs the same
 * IEEE operations in the same order returns the same bits.
 *
 * Constants: ln 2 split Cody-Waite style into HI (ln 2 truncated to 32
 * significant bits, so k*HI is exact for |k| < 2^20) and LO = ln 2 - HI
 * rounded; 1/j! and 1/(2j+1) rounded to nearest.  All were derived from a
 * 300-bit evaluation of ln 2 and are written as hexadecimal literals. */
static const double ORC_LN2_HI = 0x1.62e42fee00000p-1;
static const double ORC_LN2_LO = 0x1.a39ef35793c76p-33;
static const double ORC_INV_LN2 = 0x1.71547652b82fep+0;
static const double ORC_SQRT2 = 0x1.6a09e667f3bcdp+0;

static double orc_pow2i(int k) /* 2^k for -1022 <= k <= 1023 */
{
    uint64_t bits = (uint64_t)(k + 1023) << 52;
    double r;
    memcpy(&r, &bits, sizeof r);
    return r;
}

/* exp(x): x = k ln2 + r with k = nearest integer to x/ln2, |r| <= ln2/2 (+tiny);
 * exp(r) by its Taylor series through r^13/13! in Horner form; times 2^k. */
double orc_det_exp(double x)
{
    static const double C[14] = {
        0x1.0000000000000p+0,  0x1.0000000000000p+0,  0x1.0000000000000p-1,
        0x1.5555555555555p-3,  0x1.5555555555555p-5,  0x1.1111111111111p-7,
        0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13, 0x1.a01a01a01a01ap-16,
        0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22, 0x1.ae64567f544e4p-26,
        0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33};
    if (x != x) return x;
    if (x > 709.0) return INFINITY;
    if (x < -745.0) return 0.0;
    double kd = floor(x * ORC_INV_LN2 + 0.5);
    int k = (int)kd;
    double r = (x - kd * ORC_LN2_HI) - kd * ORC_LN2_LO;
    double poly = C[13];
    for (int j = 12; j >= 0; --j) poly = poly * r + C[j];
    if (k >= -1022) {
        if (k > 1023) return (poly * orc_pow2i(k - 1)) * 2.0;
        return poly * orc_pow2i(k);
    }
    /* result below the normal range: scale in two steps (one rounding) */
    return (poly * orc_pow2i(k + 64)) * orc_pow2i(-64);
}

/* log(x): x = 2^e m with m in [sqrt(1/2), sqrt(2)); with s = (m-1)/(m+1),
 * ln m = 2 atanh(s) = 2 s sum_{j>=0} s^{2j}/(2j+1), truncated after s^22;
 * ln x = e*HI + (e*LO + ln m). */
double orc_det_log(double x)
{
    static const double D[12] = {
        0x1.0000000000000p+0,  0x1.5555555555555p-2, 0x1.999999999999ap-3,
        0x1.2492492492492p-3,  0x1.c71c71c71c71cp-4, 0x1.745d1745d1746p-4,
        0x1.3b13b13b13b14p-4,  0x1.1111111111111p-4, 0x1.e1e1e1e1e1e1ep-5,
        0x1.af286bca1af28p-5,  0x1.8618618618618p-5, 0x1.642c8590b2164p-5};
    if (x != x || x < 0.0) return NAN;
    if (x == 0.0) return -INFINITY;
    if (x == INFINITY) return INFINITY;
    int e_adj = 0;
    if (x < 0x1p-1022) { /* subnormal: scale into the normal range */
        x = x * 0x1p54;
        e_adj = -54;
    }
    uint64_t bits;
    memcpy(&bits, &x, sizeof bits);
    int e = (int)((bits >> 52) & 0x7ff) - 1023 + e_adj;
    bits = (bits & 0x000fffffffffffffull) | 0x3ff0000000000000ull;
    double m;
    memcpy(&m, &bits, sizeof m);
    if (m > ORC_SQRT2) {
        m = m * 0.5;
        e = e + 1;
    }
    double s = (m - 1.0) / (m + 1.0);
    double z = s * s;
    double poly = D[11];
    for (int j = 10; j >= 0; --j) poly = poly * z + D[j];
    double lnm = (s + s) * poly;
    double ed = (double)e;
    return ed * ORC_LN2_HI + (ed * ORC_LN2_LO + lnm);
}

/* ------------------------------------------------------------------------- */
#define ORC_TAG_INIT 0u
#define ORC_TAG_SWEEP 1u
#define ORC_T_ALWAYS 0xFFFFFFFFu

struct orc_run {
    int system, L, q, p, N, B, K;
    uint64_t seed;
    double beta;
    int record;
    int recursion; /* 0: R5 accumulated statistics, 1: R5' plain W/H */
    int observables;            /* R9 on/off (Ising) */
    uint64_t *O_open, *O_last;  /* 3 per bin: samples, sum |M|, sum M^2 */
    int64_t sweep_counter;
    int8_t *spin;       /* p*N: Ising/MUMA +-1, Potts 0..q-1 */
    int32_t *bin;       /* p: current bin of each walker */
    uint8_t *reach;     /* B */
    int *rlist, nreach; /* ordered reachable bins */
    double *lnW, *lnW_sampled, *G, *lnR;
    uint64_t *H_open, *H_last;
    uint32_t *T; /* B*K */
    /* metrics (no counterpart in the paper): per walker, accepted moves and
     * tunnelling events of the open iteration, and which end of the reachable
     * bins it visited last (0 none, 1 lowest, 2 highest), the bin sampled at
     * the end of every sweep */
    uint64_t *acc_w, *ev_w;
    uint8_t *tun;
    uint64_t m_last[2], m_total[2];
    int64_t sweeps_last, sweep_at_update;
};

static int orc_valid(int system, int L, int q, int p)
{
    if (p < 1 || L < 4 || (L & 1)) return 0;
    if (system == ORC_ISING || system == ORC_MUMA) return L * L <= (1 << 20);
    if (system == ORC_POTTS) return q >= 2 && q <= 16 && L * L <= (1 << 20);
    return 0;
}

int orc_num_bins(const orc_run *r) { return r->B; }
int orc_num_cols(const orc_run *r) { return r->K; }
int orc_num_sites(const orc_run *r) { return r->N; }

/* Reading R6 (see header comment). */
static void orc_compute_reachable(orc_run *r)
{
    int N = r->N;
    for (int b = 0; b < r->B; ++b) r->reach[b] = 1;
    if (r->system == ORC_ISING) {
        /* bin b = (E+2N)/4 = number of broken bonds / 2 */
        r->reach[1] = 0;
        r->reach[N - 1] = 0;
    } else if (r->system == ORC_POTTS) {
        /* bin b = E + 2N = number of broken bonds */
        if (r->q == 2) {
            for (int b = 0; b < r->B; ++b)
                if ((b & 1) || b == 2 || b == 2 * N - 2) r->reach[b] = 0;
        } else {
            r->reach[1] = r->reach[2] = r->reach[3] = r->reach[5] = 0;
        }
    }
    r->nreach = 0;
    for (int b = 0; b < r->B; ++b)
        if (r->reach[b]) r->rlist[r->nreach++] = b;
}

void orc_reachable(const orc_run *r, uint8_t *out) { memcpy(out, r->reach, (size_t)r->B); }

orc_run *orc_create(int system, int L, int q, int p, uint64_t seed, double beta, int record)
{
    if (!orc_valid(system, L, q, p)) return NULL;
    orc_run *r = (orc_run *)calloc(1, sizeof *r);
    r->system = system;
    r->L = L;
    r->q = (system == ORC_POTTS) ? q : 2;
    r->p = p;
    r->N = L * L;
    r->seed = seed;
    r->beta = beta;
    r->record = record;
    if (system == ORC_ISING) { r->B = r->N + 1; r->K = 5; }
    else if (system == ORC_MUMA) { r->B = r->N + 1; r->K = 10; }
    else { r->B = 2 * r->N + 1; r->K = 9; }
    r->spin = (int8_t *)calloc((size_t)p * r->N, 1);
    r->bin = (int32_t *)calloc((size_t)p, sizeof(int32_t));
    r->reach = (uint8_t *)calloc((size_t)r->B, 1);
    r->rlist = (int *)calloc((size_t)r->B, sizeof(int));
    r->lnW = (double *)calloc((size_t)r->B, sizeof(double));
    r->lnW_sampled = (double *)calloc((size_t)r->B, sizeof(double));
    r->G = (double *)calloc((size_t)r->B, sizeof(double));
    r->lnR = (double *)calloc((size_t)r->B, sizeof(double));
    r->H_open = (uint64_t *)calloc((size_t)r->B, sizeof(uint64_t));
    r->H_last = (uint64_t *)calloc((size_t)r->B, sizeof(uint64_t));
    r->O_open = (uint64_t *)calloc((size_t)r->B * 3, sizeof(uint64_t));
    r->O_last = (uint64_t *)calloc((size_t)r->B * 3, sizeof(uint64_t));
    r->T = (uint32_t *)calloc((size_t)r->B * r->K, sizeof(uint32_t));
    r->acc_w = (uint64_t *)calloc((size_t)p, sizeof(uint64_t));
    r->ev_w = (uint64_t *)calloc((size_t)p, sizeof(uint64_t));
    r->tun = (uint8_t *)calloc((size_t)p, 1);
    orc_compute_reachable(r);
    return r;
}

void orc_free(orc_run *r)
{
    if (!r) return;
    free(r->spin); free(r->bin); free(r->reach); free(r->rlist);
    free(r->lnW); free(r->lnW_sampled); free(r->G); free(r->lnR);
    free(r->H_open); free(r->H_last); free(r->T);
    free(r->O_open); free(r->O_last);
    free(r->acc_w); free(r->ev_w); free(r->tun);
    free(r);
}

static uint32_t orc_mulhi(uint32_t a, uint32_t b) { return (uint32_t)(((uint64_t)a * b) >> 32); }

static void orc_key(const orc_run *r, uint32_t key[2])
{
    key[0] = (uint32_t)(r->seed & 0xffffffffu);
    key[1] = (uint32_t)(r->seed >> 32);
}

/* Energy of walker w from scratch: E = -sum over the 2N bonds (right, down). */
static int orc_energy(const orc_run *r, int w)
{
    const int8_t *s = r->spin + (size_t)w * r->N;
    int L = r->L, E = 0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int i = y * L + x, rt = y * L + (x + 1) % L, dn = ((y + 1) % L) * L + x;
            if (r->system == ORC_POTTS) E -= (s[i] == s[rt]) + (s[i] == s[dn]);
            else E -= s[i] * s[rt] + s[i] * s[dn];
        }
    return E;
}

static int orc_magnetisation(const orc_run *r, int w)
{
    const int8_t *s = r->spin + (size_t)w * r->N;
    int M = 0;
    for (int i = 0; i < r->N; ++i) M += s[i];
    return M;
}

static int orc_bin_of_walker(const orc_run *r, int w)
{
    if (r->system == ORC_ISING) return (orc_energy(r, w) + 2 * r->N) / 4;
    if (r->system == ORC_POTTS) return orc_energy(r, w) + 2 * r->N;
    return (orc_magnetisation(r, w) + r->N) / 2;
}

/* a6: thresholds from ln W (reading R3). */
static void orc_build_thresholds(orc_run *r)
{
    for (int b = 0; b < r->B; ++b)
        for (int c = 0; c < r->K; ++c) {
            uint32_t t = 0;
            int b2 = -1, dE = 0;
            if (r->system == ORC_ISING) { b2 = b + (c - 2); }
            else if (r->system == ORC_POTTS) { dE = c - 4; b2 = b + dE; }
            else { int sidx = c / 5, k = c % 5; dE = 4 * (k - 2); b2 = b - 1 + 2 * sidx; }
            if (r->reach[b] && b2 >= 0 && b2 < r->B && r->reach[b2]) {
                double d = r->lnW[b2] - r->lnW[b];
                if (r->system == ORC_MUMA) d = d - r->beta * (double)dE;
                if (d >= 0.0) {
                    t = ORC_T_ALWAYS;
                } else {
                    double scaled = orc_det_exp(d) * 4294967296.0;
                    t = (scaled >= 4294967296.0) ? ORC_T_ALWAYS : (uint32_t)floor(scaled);
                }
            }
            r->T[(size_t)b * r->K + c] = t;
        }
}

/* a1: initial states from the INIT stream (reading R2, R7). */
void orc_init(orc_run *r)
{
    uint32_t key[2], ctr[4], u[4];
    orc_key(r, key);
    for (int w = 0; w < r->p; ++w) {
        int8_t *s = r->spin + (size_t)w * r->N;
        for (int i = 0; i < r->N; ++i) {
            if ((i & 3) == 0) {
                ctr[0] = (uint32_t)(i / 4); ctr[1] = 0; ctr[2] = (uint32_t)w; ctr[3] = ORC_TAG_INIT;
                orc_philox4x32_10(ctr, key, u);
            }
            uint32_t word = u[i & 3];
            if (r->system == ORC_POTTS) s[i] = (int8_t)orc_mulhi(word, (uint32_t)r->q);
            else s[i] = (word >> 31) ? -1 : +1;
        }
        r->bin[w] = orc_bin_of_walker(r, w);
    }
    for (int b = 0; b < r->B; ++b) {
        r->lnW[b] = r->reach[b] ? 0.0 : -INFINITY;
        r->lnW_sampled[b] = r->lnW[b];
        r->G[b] = 0.0;
        r->lnR[b] = 0.0;
        r->H_open[b] = 0;
        r->H_last[b] = 0;
    }
    r->sweep_counter = 0;
    for (int w = 0; w < r->p; ++w) {
        r->acc_w[w] = 0;
        r->ev_w[w] = 0;
        r->tun[w] = 0;
    }
    r->m_last[0] = r->m_last[1] = r->m_total[0] = r->m_total[1] = 0;
    r->sweeps_last = 0;
    r->sweep_at_update = 0;
    orc_build_thresholds(r);
}

/* a2 + a3 for one walker: `sweeps` sweeps starting at global sweep g0. */
static void orc_walker_sweeps(const orc_run *r, int w, int64_t g0, int64_t sweeps, uint64_t *hist, uint64_t *obs)
{
    const int L = r->L, N = r->N, K = r->K;
    int8_t *s = r->spin + (size_t)w * N;
    int b = r->bin[w];
    uint32_t key[2], ctr[4], u[4];
    orc_key(r, key);
    for (int64_t sw = 0; sw < sweeps; ++sw) {
        uint32_t g = (uint32_t)(g0 + sw);
        for (int i = 0; i < N; ++i) {
            int x = i % L, y = i / L;
            int nb[4] = {y * L + (x + 1) % L, y * L + (x + L - 1) % L,
                         ((y + 1) % L) * L + x, ((y + L - 1) % L) * L + x};
            uint32_t u_acc;
            int col, db;
            int8_t new_s;
            if (r->system == ORC_POTTS) {
                if ((i & 1) == 0) {
                    ctr[0] = (uint32_t)(i / 2); ctr[1] = g; ctr[2] = (uint32_t)w; ctr[3] = ORC_TAG_SWEEP;
                    orc_philox4x32_10(ctr, key, u);
                }
                uint32_t u_prop = u[2 * (i & 1)];
                u_acc = u[2 * (i & 1) + 1];
                int old = s[i];
                int nw = (old + 1 + (int)orc_mulhi(u_prop, (uint32_t)(r->q - 1))) % r->q;
                int eq_old = 0, eq_new = 0;
                for (int j = 0; j < 4; ++j) {
                    eq_old += (s[nb[j]] == old);
                    eq_new += (s[nb[j]] == nw);
                }
                int dE = eq_old - eq_new; /* E = -sum delta */
                col = dE + 4;
                db = dE;
                new_s = (int8_t)nw;
            } else {
                if ((i & 3) == 0) {
                    ctr[0] = (uint32_t)(i / 4); ctr[1] = g; ctr[2] = (uint32_t)w; ctr[3] = ORC_TAG_SWEEP;
                    orc_philox4x32_10(ctr, key, u);
                }
                u_acc = u[i & 3];
                int sum_nn = s[nb[0]] + s[nb[1]] + s[nb[2]] + s[nb[3]];
                int dE = 2 * s[i] * sum_nn; /* in {-8,-4,0,4,8} */
                int k = dE / 4 + 2;
                if (r->system == ORC_ISING) {
                    col = k;
                    db = dE / 4;
                } else { /* MUMA: bin over M, dM = -2 s_i */
                    int sidx = (s[i] == 1) ? 0 : 1;
                    col = sidx * 5 + k;
                    db = -s[i];
                }
                new_s = (int8_t)(-s[i]);
            }
            uint32_t t = r->T[(size_t)b * K + col];
            if (t == ORC_T_ALWAYS || u_acc < t) {
                s[i] = new_s;
                b += db;
                r->acc_w[w] += 1;
            }
            if (r->record == 0) hist[b] += 1;
        }
        if (r->record == 1) hist[b] += 1;
        /* tunnelling: the walker's bin at the end of the sweep against the two ends */
        if (b == r->rlist[0]) {
            if (r->tun[w] == 2) r->ev_w[w] += 1;
            r->tun[w] = 1;
        } else if (b == r->rlist[r->nreach - 1]) {
            if (r->tun[w] == 1) r->ev_w[w] += 1;
            r->tun[w] = 2;
        }
        if (obs) { /* R9 */
            int64_t M = 0;
            for (int i = 0; i < N; ++i) M += s[i];
            obs[3 * (size_t)b] += 1;
            obs[3 * (size_t)b + 1] += (uint64_t)(M < 0 ? -M : M);
            obs[3 * (size_t)b + 2] += (uint64_t)(M * M);
        }
    }
    r->bin[w] = b;
}

typedef struct {
    const orc_run *r;
    int w0, w1;
    int64_t g0, sweeps;
    uint64_t *hist, *obs;
} orc_job;

static void *orc_job_main(void *arg)
{
    orc_job *j = (orc_job *)arg;
    for (int w = j->w0; w < j->w1; ++w) orc_walker_sweeps(j->r, w, j->g0, j->sweeps, j->hist, j->obs);
    return NULL;
}

void orc_iterate_range(orc_run *r, int64_t sweeps, int w0, int w1, int nthreads)
{
    if (w0 < 0) w0 = 0;
    if (w1 > r->p) w1 = r->p;
    if (w1 <= w0 || sweeps <= 0) return;
    int nw = w1 - w0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nw) nthreads = nw;
    orc_job *jobs = (orc_job *)calloc((size_t)nthreads, sizeof *jobs);
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof *th);
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].r = r;
        jobs[t].w0 = w0 + (int)((int64_t)nw * t / nthreads);
        jobs[t].w1 = w0 + (int)((int64_t)nw * (t + 1) / nthreads);
        jobs[t].g0 = r->sweep_counter;
        jobs[t].sweeps = sweeps;
        jobs[t].hist = (uint64_t *)calloc((size_t)r->B, sizeof(uint64_t));
        jobs[t].obs = (r->observables && r->system == ORC_ISING) ? (uint64_t *)calloc((size_t)r->B * 3, sizeof(uint64_t))
                                                                  : NULL;
    }
    if (nthreads == 1) {
        orc_job_main(&jobs[0]);
    } else {
        for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, orc_job_main, &jobs[t]);
        for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    }
    /* a4: merge the per-walker-group histograms (an integer sum). */
    for (int t = 0; t < nthreads; ++t) {
        for (int b = 0; b < r->B; ++b) r->H_open[b] += jobs[t].hist[b];
        free(jobs[t].hist);
        if (jobs[t].obs) {
            for (size_t i = 0; i < (size_t)r->B * 3; ++i) r->O_open[i] += jobs[t].obs[i];
            free(jobs[t].obs);
        }
    }
    free(jobs);
    free(th);
}

void orc_advance(orc_run *r, int64_t sweeps) { r->sweep_counter += sweeps; }

void orc_iterate(orc_run *r, int64_t sweeps, int nthreads)
{
    orc_iterate_range(r, sweeps, 0, r->p, nthreads);
    orc_advance(r, sweeps);
}

void orc_set_open_histogram(orc_run *r, const uint64_t *H) { memcpy(r->H_open, H, sizeof(uint64_t) * r->B); }
void orc_get_open_histogram(const orc_run *r, uint64_t *out) { memcpy(out, r->H_open, sizeof(uint64_t) * r->B); }

void orc_set_recursion(orc_run *r, int mode) { r->recursion = mode; }
void orc_set_lnW(orc_run *r, const double *lnW)
{
    for (int b = 0; b < r->B; ++b) r->lnW[b] = r->reach[b] ? lnW[b] : -INFINITY;
    orc_build_thresholds(r);
}
void orc_set_observables(orc_run *r, int on) { r->observables = on; }
void orc_get_observables(const orc_run *r, uint64_t *out) { memcpy(out, r->O_last, sizeof(uint64_t) * 3 * r->B); }

/* Eq. (2) with per-bin sums (R9): <O>_beta = sum_b S_O(b) e^{-beta E_b} / W(b) over
 * sum_b n(b) e^{-beta E_b} / W(b), W the weights the samples were taken with, E_b
 * the Ising energy of bin b (4b - 2N).  out = {<|M|>/N, <M^2>/N^2, beta N
 * (<M^2>/N^2 - (<|M|>/N)^2)}; NaN if no bin has samples. */
void orc_reweight_obs(int B, int N, const uint64_t *sums, const double *lnW_sampled, double beta, double out[3])
{
    double m = -INFINITY;
    for (int b = 0; b < B; ++b)
        if (sums[3 * b] > 0) {
            double x = -beta * (double)(4 * b - 2 * N) - lnW_sampled[b];
            if (x > m) m = x;
        }
    if (m == -INFINITY) { out[0] = out[1] = out[2] = NAN; return; }
    double z = 0.0, a1 = 0.0, a2 = 0.0;
    for (int b = 0; b < B; ++b) {
        if (sums[3 * b] == 0) continue;
        double f = exp(-beta * (double)(4 * b - 2 * N) - lnW_sampled[b] - m);
        z += f * (double)sums[3 * b];
        a1 += f * (double)sums[3 * b + 1];
        a2 += f * (double)sums[3 * b + 2];
    }
    out[0] = a1 / z / N;
    out[1] = a2 / z / ((double)N * N);
    out[2] = beta * N * (out[1] - out[0] * out[0]);
}

void orc_reweight_observables(const orc_run *r, double beta, double out[3])
{
    orc_reweight_obs(r->B, r->N, r->O_last, r->lnW_sampled, beta, out);
}

/* a5 (reading R5, or R5' when selected) followed by a6. */
/* Close the metrics of the iteration that the update ends. */
static void orc_close_metrics(orc_run *r)
{
    uint64_t a = 0, e = 0;
    for (int w = 0; w < r->p; ++w) {
        a += r->acc_w[w];
        e += r->ev_w[w];
        r->acc_w[w] = 0;
        r->ev_w[w] = 0;
    }
    r->m_last[0] = a;
    r->m_last[1] = e;
    r->m_total[0] += a;
    r->m_total[1] += e;
    r->sweeps_last = r->sweep_counter - r->sweep_at_update;
    r->sweep_at_update = r->sweep_counter;
}

void orc_get_metrics(const orc_run *r, uint64_t out[5])
{
    out[0] = r->m_last[0];
    out[1] = r->m_last[1];
    out[2] = r->m_total[0];
    out[3] = r->m_total[1];
    out[4] = (uint64_t)r->sweeps_last;
}

void orc_update(orc_run *r)
{
    const int Kr = r->nreach;
    orc_close_metrics(r);
    memcpy(r->lnW_sampled, r->lnW, sizeof(double) * r->B);
    memcpy(r->O_last, r->O_open, sizeof(uint64_t) * 3 * r->B);
    memset(r->O_open, 0, sizeof(uint64_t) * 3 * r->B);
    if (r->recursion == 1) {
        /* R5': x_k = ln W(r_k) - ln max(H(r_k), 1); ln W(r_k) = x_k - x_0 */
        double x0 = 0.0;
        for (int k = 0; k < Kr; ++k) {
            uint64_t h = r->H_open[r->rlist[k]];
            double lh = h > 0 ? orc_det_log((double)h) : 0.0;
            double x = r->lnW_sampled[r->rlist[k]] - lh;
            if (k == 0) x0 = x;
            r->lnW[r->rlist[k]] = x - x0;
        }
        memcpy(r->H_last, r->H_open, sizeof(uint64_t) * r->B);
        memset(r->H_open, 0, sizeof(uint64_t) * r->B);
        orc_build_thresholds(r);
        return;
    }
    for (int k = 0; k + 1 < Kr; ++k) {
        uint64_t h0 = r->H_open[r->rlist[k]], h1 = r->H_open[r->rlist[k + 1]];
        if (h0 > 0 && h1 > 0) {
            double a = (double)h0, c = (double)h1;
            double g = (a * c) / (a + c);
            r->G[k] = r->G[k] + g;
            double kappa = g / r->G[k];
            double diff = orc_det_log(a) - orc_det_log(c);
            r->lnR[k] = r->lnR[k] + kappa * diff;
        }
    }
    for (int b = 0; b < r->B; ++b) r->lnW[b] = -INFINITY;
    double acc = 0.0;
    r->lnW[r->rlist[0]] = acc;
    for (int k = 0; k + 1 < Kr; ++k) {
        acc = acc + r->lnR[k];
        r->lnW[r->rlist[k + 1]] = acc;
    }
    memcpy(r->H_last, r->H_open, sizeof(uint64_t) * r->B);
    memset(r->H_open, 0, sizeof(uint64_t) * r->B);
    orc_build_thresholds(r);
}

int orc_is_flat(const orc_run *r, double ratio, double stats[3])
{
    uint64_t mn = UINT64_MAX, mx = 0, sum = 0;
    for (int k = 0; k < r->nreach; ++k) {
        uint64_t h = r->H_last[r->rlist[k]];
        if (h < mn) mn = h;
        if (h > mx) mx = h;
        sum += h;
    }
    double mean = (double)sum / (double)r->nreach;
    if (stats) { stats[0] = (double)mn; stats[1] = mean; stats[2] = (double)mx; }
    return mn > 0 && (double)mn / mean >= ratio;
}

/* a8: Eq. (2) with O a function of the binned variable.  ln Omega_hat(b) =
 * ln H(b) - ln W(b), with W the weights the histogram was sampled with. */
void orc_reweight(const orc_run *r, double beta, double out[4], double *lnP)
{
    const int B = r->B, N = r->N;
    double *x = (double *)malloc(sizeof(double) * B);
    double m = -INFINITY;
    for (int b = 0; b < B; ++b) {
        x[b] = -INFINITY;
        if (!r->reach[b] || r->H_last[b] == 0) continue;
        double lnOmega = log((double)r->H_last[b]) - r->lnW_sampled[b];
        if (r->system == ORC_MUMA) {
            x[b] = lnOmega; /* exp(-beta E) is already in the ensemble, Eq. (3) */
        } else {
            double E = (r->system == ORC_ISING) ? (double)(4 * b - 2 * N) : (double)(b - 2 * N);
            x[b] = lnOmega - beta * E;
        }
        if (x[b] > m) m = x[b];
    }
    double z = 0.0;
    for (int b = 0; b < B; ++b)
        if (x[b] > -INFINITY) z += exp(x[b] - m);
    double lse = m + log(z);
    double a1 = 0.0, a2 = 0.0;
    for (int b = 0; b < B; ++b) {
        double lp = (x[b] > -INFINITY) ? x[b] - lse : -INFINITY;
        if (lnP) lnP[b] = lp;
        if (x[b] == -INFINITY) continue;
        double P = exp(lp);
        double v;
        if (r->system == ORC_MUMA) v = fabs((double)(2 * b - N));
        else v = (r->system == ORC_ISING) ? (double)(4 * b - 2 * N) : (double)(b - 2 * N);
        a1 += P * v;
        a2 += P * v * v;
    }
    if (r->system == ORC_MUMA) {
        out[0] = a1 / N;
        out[1] = a2 / ((double)N * N);
        out[2] = r->beta * N * (out[1] - out[0] * out[0]);
        int b0 = N / 2, bm = N;
        out[3] = (x[b0] > -INFINITY && x[bm] > -INFINITY) ? (x[b0] - x[bm]) : NAN;
    } else {
        out[0] = a1;
        out[1] = a2;
        out[2] = beta * beta * (a2 - a1 * a1) / N;
        double g0 = (r->system == ORC_ISING) ? 2.0 : (double)r->q;
        if (x[0] > -INFINITY) {
            double lnOmega0 = x[0] - beta * (double)(2 * N); /* x[0] = lnOmega0 + 2N beta */
            out[3] = lse + log(g0) - lnOmega0;
        } else {
            out[3] = NAN;
        }
    }
    free(x);
}

void orc_get_lnW(const orc_run *r, double *out) { memcpy(out, r->lnW, sizeof(double) * r->B); }
void orc_get_lnW_sampled(const orc_run *r, double *out) { memcpy(out, r->lnW_sampled, sizeof(double) * r->B); }
void orc_get_histogram(const orc_run *r, uint64_t *out) { memcpy(out, r->H_last, sizeof(uint64_t) * r->B); }
void orc_get_thresholds(const orc_run *r, uint32_t *out) { memcpy(out, r->T, sizeof(uint32_t) * r->B * r->K); }
void orc_get_spins(const orc_run *r, int8_t *out) { memcpy(out, r->spin, (size_t)r->p * r->N); }
void orc_get_bins(const orc_run *r, int32_t *out) { memcpy(out, r->bin, sizeof(int32_t) * r->p); }
int64_t orc_get_sweep_counter(const orc_run *r) { return r->sweep_counter; }

/* ------------------------------------------------------------------------- */
/* Exact tools: enumerate every state of a small periodic lattice. */
int orc_bruteforce_ising(int L, uint64_t *omega)
{
    int N = L * L;
    if (L < 2 || N > 30) return -1;
    memset(omega, 0, sizeof(uint64_t) * (N + 1));
    for (uint64_t st = 0; st < (1ull << N); ++st) {
        int E = 0;
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int i = y * L + x, rt = y * L + (x + 1) % L, dn = ((y + 1) % L) * L + x;
                int si = (st >> i & 1) ? -1 : 1, sr = (st >> rt & 1) ? -1 : 1, sd = (st >> dn & 1) ? -1 : 1;
                E -= si * sr + si * sd;
            }
        omega[(E + 2 * N) / 4] += 1;
    }
    return 0;
}

int orc_bruteforce_ising_EM(int L, uint64_t *omega)
{
    int N = L * L;
    if (L < 2 || N > 30) return -1;
    memset(omega, 0, sizeof(uint64_t) * (N + 1) * (N + 1));
    for (uint64_t st = 0; st < (1ull << N); ++st) {
        int E = 0, M = 0;
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int i = y * L + x, rt = y * L + (x + 1) % L, dn = ((y + 1) % L) * L + x;
                int si = (st >> i & 1) ? -1 : 1, sr = (st >> rt & 1) ? -1 : 1, sd = (st >> dn & 1) ? -1 : 1;
                E -= si * sr + si * sd;
                M += si;
            }
        omega[(size_t)((E + 2 * N) / 4) * (N + 1) + (M + N) / 2] += 1;
    }
    return 0;
}

int orc_bruteforce_potts(int L, int q, uint64_t *omega)
{
    int N = L * L;
    if (L < 2 || q < 2 || N > 40) return -1;
    double states = pow((double)q, (double)N);
    if (states > 2e9) return -1;
    memset(omega, 0, sizeof(uint64_t) * (2 * N + 1));
    int *s = (int *)calloc((size_t)N, sizeof(int));
    for (;;) {
        int E = 0;
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int i = y * L + x, rt = y * L + (x + 1) % L, dn = ((y + 1) % L) * L + x;
                E -= (s[i] == s[rt]) + (s[i] == s[dn]);
            }
        omega[E + 2 * N] += 1;
        int i = 0;
        while (i < N && ++s[i] == q) s[i++] = 0;
        if (i == N) break;
    }
    free(s);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Exact density of states by a site-by-site ("helical window") transfer
 * matrix on the periodic L x L lattice.  The window holds the last L spins
 * added: bit/digit 0 is the up neighbour of the next site, the top one its left
 * neighbour, and at the end of a row digit 1 is the row's first site (the
 * right neighbour through the periodic boundary).  The first row is fixed by
 * an outer sum, which closes the lattice in the vertical direction.  Counts
 * are kept as unsigned 128-bit integers and returned as (lo, hi) pairs. */
typedef unsigned __int128 orc_u128;

int orc_tm_ising(int L, int track_m, uint64_t *out)
{
    if (L < 2 || L > 10) return -1;
    const int N = L * L, W = 1 << L, NE = 4 * N + 1, NM = track_m ? 2 * N + 1 : 1;
    const size_t S = (size_t)W * NE * NM;
    orc_u128 *cur = (orc_u128 *)calloc(S, sizeof(orc_u128));
    orc_u128 *nxt = (orc_u128 *)calloc(S, sizeof(orc_u128));
    orc_u128 *tot = (orc_u128 *)calloc((size_t)(N + 1) * (track_m ? N + 1 : 1), sizeof(orc_u128));
    if (!cur || !nxt || !tot) { free(cur); free(nxt); free(tot); return -2; }
#define ORC_SPIN(w, j) ((((w) >> (j)) & 1) ? -1 : 1)
    for (int r0 = 0; r0 < W; ++r0) {
        memset(cur, 0, S * sizeof(orc_u128));
        int E0 = 0, M0 = 0;
        for (int x = 0; x < L; ++x) {
            E0 -= ORC_SPIN(r0, x) * ORC_SPIN(r0, (x + 1) % L);
            M0 += ORC_SPIN(r0, x);
        }
        cur[((size_t)r0 * NE + (E0 + 2 * N)) * NM + (track_m ? M0 + N : 0)] = 1;
        for (int y = 1; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                memset(nxt, 0, S * sizeof(orc_u128));
                for (int w = 0; w < W; ++w)
                    for (int e = 0; e < NE; ++e)
                        for (int m = 0; m < NM; ++m) {
                            orc_u128 c = cur[((size_t)w * NE + e) * NM + m];
                            if (!c) continue;
                            for (int sn = 0; sn < 2; ++sn) {
                                int sv = sn ? -1 : 1;
                                int dE = -sv * ORC_SPIN(w, 0);
                                if (x >= 1) dE -= sv * ORC_SPIN(w, L - 1);
                                if (x == L - 1) dE -= sv * ORC_SPIN(w, 1);
                                if (y == L - 1) dE -= sv * ORC_SPIN(r0, x);
                                int nw = (w >> 1) | (sn << (L - 1));
                                int nm = track_m ? m + sv : 0;
                                nxt[((size_t)nw * NE + (e + dE)) * NM + nm] += c;
                            }
                        }
                orc_u128 *t = cur; cur = nxt; nxt = t;
            }
        for (int w = 0; w < W; ++w)
            for (int e = 0; e < NE; ++e)
                for (int m = 0; m < NM; ++m) {
                    orc_u128 c = cur[((size_t)w * NE + e) * NM + m];
                    if (!c) continue;
                    /* e = E + 2N and E = -2N + 4j, so e is a multiple of 4 */
                    size_t idx = (size_t)(e / 4) * (track_m ? N + 1 : 1) + (track_m ? (m / 2) : 0);
                    tot[idx] += c;
                }
    }
#undef ORC_SPIN
    size_t n = (size_t)(N + 1) * (track_m ? N + 1 : 1);
    for (size_t i = 0; i < n; ++i) {
        out[2 * i] = (uint64_t)tot[i];
        out[2 * i + 1] = (uint64_t)(tot[i] >> 64);
    }
    free(cur); free(nxt); free(tot);
    return 0;
}

int orc_tm_potts(int L, int q, uint64_t *out /* 2*(2N+1): index E+2N */)
{
    if (L < 2 || q < 2) return -1;
    double wd = pow((double)q, (double)L);
    if (wd > 70000.0) return -1;
    const int N = L * L, W = (int)wd, NE = 2 * N + 1;
    int qtop = 1;
    for (int j = 0; j < L - 1; ++j) qtop *= q;
    const size_t S = (size_t)W * NE;
    orc_u128 *cur = (orc_u128 *)calloc(S, sizeof(orc_u128));
    orc_u128 *nxt = (orc_u128 *)calloc(S, sizeof(orc_u128));
    orc_u128 *tot = (orc_u128 *)calloc((size_t)NE, sizeof(orc_u128));
    int *dig = (int *)calloc((size_t)W * L, sizeof(int));
    if (!cur || !nxt || !tot || !dig) { free(cur); free(nxt); free(tot); free(dig); return -2; }
    for (int w = 0; w < W; ++w) {
        int v = w;
        for (int j = 0; j < L; ++j) { dig[w * L + j] = v % q; v /= q; }
    }
    for (int r0 = 0; r0 < W; ++r0) {
        memset(cur, 0, S * sizeof(orc_u128));
        const int *d0 = dig + (size_t)r0 * L;
        int nsat = 0;
        for (int x = 0; x < L; ++x) nsat += (d0[x] == d0[(x + 1) % L]);
        cur[(size_t)r0 * NE + nsat] = 1;
        for (int y = 1; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                memset(nxt, 0, S * sizeof(orc_u128));
                for (int w = 0; w < W; ++w) {
                    const int *dw = dig + (size_t)w * L;
                    for (int e = 0; e < NE; ++e) {
                        orc_u128 c = cur[(size_t)w * NE + e];
                        if (!c) continue;
                        for (int sn = 0; sn < q; ++sn) {
                            int ds = (sn == dw[0]);
                            if (x >= 1) ds += (sn == dw[L - 1]);
                            if (x == L - 1) ds += (sn == dw[1]);
                            if (y == L - 1) ds += (sn == d0[x]);
                            int nw = w / q + sn * qtop;
                            nxt[(size_t)nw * NE + e + ds] += c;
                        }
                    }
                }
                orc_u128 *t = cur; cur = nxt; nxt = t;
            }
        for (int w = 0; w < W; ++w)
            for (int e = 0; e < NE; ++e) tot[2 * N - e] += cur[(size_t)w * NE + e]; /* E = -nsat */
    }
    for (int i = 0; i < NE; ++i) {
        out[2 * i] = (uint64_t)tot[i];
        out[2 * i + 1] = (uint64_t)(tot[i] >> 64);
    }
    free(cur); free(nxt); free(tot); free(dig);
    return 0;
}
