// sweep_spin.cu -- the hot loop of the parallel multicanonical method for
// lattice spins (paper: Ising and Potts paragraphs, multimagnetic Eq. 3, and
// the Fig. 1 scheme of p independent chains sharing one weight function).
//
// One walker per thread.  A MUCA acceptance depends on the walker's global
// energy, so the sites of one walker are updated strictly in order
// (i = y*L + x, every sweep) and no checkerboard split is possible; the
// parallelism is across walkers.  Per attempt:
//   random word(s) from Philox(counter = (site group, sweep, walker, tag))
//   -> neighbour count -> column c of the threshold table
//   -> accept iff T[b][c] == always or u < T[b][c]   (integer compare)
//   -> flip / recolour, move the bin
//   -> count the current bin in the block's shared-memory histogram.
//
// Latency structure.  With p = 8192 walkers there is one warp per scheduler,
// so nothing hides a walker's serial chain: the shared-memory threshold load
// would sit between two consecutive accept decisions.  The sweep therefore
// loads, for site x+1, both thresholds it can need -- the one for "site x
// rejected" (same bin, left neighbour unchanged) and the one for "site x
// accepted" (bin moved by site x's energy change, left neighbour flipped) --
// while site x is being decided, and then selects one.  Every such index is the
// bin of a configuration that can occur, so it is always inside the table.
// Philox blocks are computed one group ahead (the block after a sweep's last
// group is computed and discarded, which keeps the row one basic block), with
// the round keys read from the kernel parameters; the recording mode is a
// template parameter for the same reason.
//
// Shared memory holds one row of RS = C+1 words per bin: the C thresholds and
// the bin's histogram counter, so one row offset addresses both.
// Lattice rows live in HBM/L2 walker-interleaved (coalesced) and stream through
// registers: the row above (final), the current row and the row below (old),
// with the next row prefetched one row ahead.
#include "muca_device.cuh"
#include "muca_internal.h"

namespace muca {

template <int WR>
__device__ __forceinline__ int bit_at(const uint32_t (&r)[WR], int pos)
{
    return (int)((r[pos >> 5] >> (pos & 31)) & 1u);
}

template <int WR>
__device__ __forceinline__ uint32_t nib_at(const uint32_t (&r)[WR], int x)
{
    return (r[(4 * x) >> 5] >> ((4 * x) & 31)) & 15u;
}

__device__ __forceinline__ uint32_t word_of(const uint4 &u, int j)
{
    return j == 0 ? u.x : (j == 1 ? u.y : (j == 2 ? u.z : u.w));
}

// One sweep of an Ising (MUCA in E) or multimagnetic (weight in M) walker.
// Spin bit 1 means s = -1.  k = 4 - (number of anti-aligned neighbours), so
// dE = 4(k-2); Ising column c = k and the bin moves by k-2; MUMA column
// c = 5*bit + k and the bin (M+N)/2 moves by 2*bit-1.
template <int SYS, int L, int RECORD>
__device__ __forceinline__ void ising_sweep(uint32_t *__restrict__ lat, int ps, int &bR,
                                            uint32_t *__restrict__ sTH, uint32_t g, uint32_t wid,
                                            const uint32_t (&rk)[20])
{
    constexpr int WR = ising_words_per_row(L);
    constexpr int C = (SYS == kMuma) ? 10 : 5;
    constexpr int RS = C + 1;
    uint32_t up[WR], cur[WR], dn[WR], first[WR], nxt[WR], old[WR];
#pragma unroll
    for (int j = 0; j < WR; ++j) {
        up[j] = lat[((L - 1) * WR + j) * ps];
        cur[j] = lat[j * ps];
        dn[j] = lat[(WR + j) * ps];
        first[j] = 0u;
        nxt[j] = 0u;
    }
    uint4 u_next = philox4x32_10_rk(make_uint4(0u, g, wid, kTagSweep), rk);
#pragma unroll 1
    for (int y = 0; y < L; ++y) {
        if (y + 2 < L) {
#pragma unroll
            for (int j = 0; j < WR; ++j) nxt[j] = lat[((y + 2) * WR + j) * ps];
        }
#pragma unroll
        for (int j = 0; j < WR; ++j) old[j] = cur[j];
        // Columns and bin-row moves of site x for "left neighbour as it was"
        // (c0, d0) and "left neighbour flipped" (c1, d1), from the row's old
        // values; the right neighbour of the last site is site 0 of this row,
        // already final.
        auto site = [&](int x, int &c0, int &c1, int &d0, int &d1) {
            const int s = bit_at<WR>(old, x);
            const int l = bit_at<WR>(old, (x + L - 1) % L);
            const int r = (x == L - 1) ? bit_at<WR>(cur, 0) : bit_at<WR>(old, x + 1);
            const int n1 = l + r + bit_at<WR>(up, x) + bit_at<WR>(dn, x);
            const int k0 = s ? n1 : 4 - n1;
            const int k1 = k0 - 1 + 2 * (l ^ s);
            if (SYS == kMuma) {
                c0 = 5 * s + k0;
                c1 = 5 * s + k1;
                d0 = d1 = (2 * s - 1) * RS;
            } else {
                c0 = k0;
                c1 = k1;
                d0 = (k0 - 2) * RS;
                d1 = (k1 - 2) * RS;
            }
        };
        int c0, c1, d0, d1;
        site(0, c0, c1, d0, d1);
        uint32_t T0 = sTH[bR + c0], T1 = 0u;
        bool accP = false;
        int dRp = 0;
        uint4 u = u_next;
#pragma unroll
        for (int x = 0; x < L; ++x) {
            if ((x & 3) == 0) {
                u = u_next;
                u_next = philox4x32_10_rk(make_uint4((uint32_t)((y * L + x) / 4 + 1), g, wid, kTagSweep), rk);
            }
            const uint32_t uw = word_of(u, x & 3);
            bR = accP ? bR + dRp : bR;
            const int dR = accP ? d1 : d0;
            const uint32_t T = accP ? T1 : T0;
            if (x + 1 < L) {
                int n0, n1c, e0, e1;
                site(x + 1, n0, n1c, e0, e1);
                T0 = sTH[bR + n0];
                T1 = sTH[bR + dR + n1c];
                d0 = e0;
                d1 = e1;
            }
            const bool acc = (T == kAlways) || (uw < T);
            if (acc) cur[x >> 5] ^= 1u << (x & 31);
            if (RECORD == 0) atomicAdd(&sTH[(acc ? bR + dR : bR) + C], 1u);
            accP = acc;
            dRp = dR;
        }
        bR = accP ? bR + dRp : bR;
#pragma unroll
        for (int j = 0; j < WR; ++j) lat[(y * WR + j) * ps] = cur[j];
        if (y == 0) {
#pragma unroll
            for (int j = 0; j < WR; ++j) first[j] = cur[j];
        }
#pragma unroll
        for (int j = 0; j < WR; ++j) {
            up[j] = cur[j];
            cur[j] = dn[j];
            dn[j] = (y + 2 < L) ? nxt[j] : first[j];
        }
    }
    if (RECORD == 1) atomicAdd(&sTH[bR + C], 1u);
}

// One sweep of a q-state Potts walker (4-bit spins).  Proposal: a uniform new
// state different from the old one, new = (old + 1 + mulhi(u, q-1)) mod q.
// dE = n_eq(old) - n_eq(new) in [-4, 4]; column dE+4; bin E+2N moves by dE.
// The "left neighbour changed" candidate uses the left site's proposed colour.
template <int L, int RECORD>
__device__ __forceinline__ void potts_sweep(uint32_t *__restrict__ lat, int ps, int &bR,
                                            uint32_t *__restrict__ sTH, uint32_t g, uint32_t wid,
                                            const uint32_t (&rk)[20], uint32_t q)
{
    constexpr int WR = potts_words_per_row(L);
    constexpr int RS = 10;
    uint32_t up[WR], cur[WR], dn[WR], first[WR], nxt[WR], old[WR];
#pragma unroll
    for (int j = 0; j < WR; ++j) {
        up[j] = lat[((L - 1) * WR + j) * ps];
        cur[j] = lat[j * ps];
        dn[j] = lat[(WR + j) * ps];
        first[j] = 0u;
        nxt[j] = 0u;
    }
    const uint32_t qm1 = q - 1u;
    uint4 u_next = philox4x32_10_rk(make_uint4(0u, g, wid, kTagSweep), rk);
#pragma unroll 1
    for (int y = 0; y < L; ++y) {
        if (y + 2 < L) {
#pragma unroll
            for (int j = 0; j < WR; ++j) nxt[j] = lat[((y + 2) * WR + j) * ps];
        }
#pragma unroll
        for (int j = 0; j < WR; ++j) old[j] = cur[j];
        // Proposal and energy change of site x, for the left neighbour as it was
        // (c0, d0) and recoloured to the left site's proposal lnw (c1, d1).
        auto site = [&](int x, uint32_t uprop, uint32_t lnw, uint32_t &nw, int &c0, int &c1, int &d0, int &d1) {
            const uint32_t o = nib_at<WR>(old, x);
            const uint32_t nl = nib_at<WR>(old, (x + L - 1) % L);
            const uint32_t nr = (x == L - 1) ? nib_at<WR>(cur, 0) : nib_at<WR>(old, x + 1);
            const uint32_t nu = nib_at<WR>(up, x), nd = nib_at<WR>(dn, x);
            uint32_t v = o + 1u + __umulhi(uprop, qm1);
            v = (v >= q) ? v - q : v;
            nw = v;
            const int rest = (int)(nr == o) + (int)(nu == o) + (int)(nd == o) - (int)(nr == v) - (int)(nu == v) -
                             (int)(nd == v);
            const int dE0 = rest + (int)(nl == o) - (int)(nl == v);
            const int dE1 = rest + (int)(lnw == o) - (int)(lnw == v);
            c0 = dE0 + 4;
            c1 = dE1 + 4;
            d0 = dE0 * RS;
            d1 = dE1 * RS;
        };
        uint4 u = u_next;
        uint32_t nwc;
        int c0, c1, d0, d1;
        site(0, u.x, 0u, nwc, c0, c1, d0, d1);
        uint32_t T0 = sTH[bR + c0], T1 = 0u;
        bool accP = false;
        int dRp = 0;
#pragma unroll
        for (int x = 0; x < L; ++x) {
            if ((x & 1) == 0) {
                u = u_next;
                u_next = philox4x32_10_rk(make_uint4((uint32_t)((y * L + x) / 2 + 1), g, wid, kTagSweep), rk);
            }
            const uint32_t u_acc = (x & 1) ? u.w : u.y;
            bR = accP ? bR + dRp : bR;
            const int dR = accP ? d1 : d0;
            const uint32_t T = accP ? T1 : T0;
            const uint32_t nw = nwc;
            if (x + 1 < L) {
                const uint32_t uprop = ((x + 1) & 1) ? u.z : u_next.x;
                int n0, n1c, e0, e1;
                site(x + 1, uprop, nw, nwc, n0, n1c, e0, e1);
                T0 = sTH[bR + n0];
                T1 = sTH[bR + dR + n1c];
                d0 = e0;
                d1 = e1;
            }
            const bool acc = (T == kAlways) || (u_acc < T);
            if (acc) {
                const int wi = (4 * x) >> 5, sh = (4 * x) & 31;
                cur[wi] = (cur[wi] & ~(15u << sh)) | (nw << sh);
            }
            if (RECORD == 0) atomicAdd(&sTH[(acc ? bR + dR : bR) + 9], 1u);
            accP = acc;
            dRp = dR;
        }
        bR = accP ? bR + dRp : bR;
#pragma unroll
        for (int j = 0; j < WR; ++j) lat[(y * WR + j) * ps] = cur[j];
        if (y == 0) {
#pragma unroll
            for (int j = 0; j < WR; ++j) first[j] = cur[j];
        }
#pragma unroll
        for (int j = 0; j < WR; ++j) {
            up[j] = cur[j];
            cur[j] = dn[j];
            dn[j] = (y + 2 < L) ? nxt[j] : first[j];
        }
    }
    if (RECORD == 1) atomicAdd(&sTH[bR + 9], 1u);
}

// ---------------------------------------------------------------------------
// Producer/consumer form.  With one warp per scheduler a walker's Philox rounds
// (long dependent multiply/xor chains) and its serial accept chain share one
// instruction stream.  Here each consumer warp (the walkers' chains) is paired
// with a producer warp that computes the same walkers' Philox blocks, one lattice
// row at a time, into a ring of kRing row slots in shared memory; the two run on
// different schedulers.  Hand-over uses mbarriers: FULL[slot] (32 producer
// arrivals) and EMPTY[slot] (32 consumer arrivals).  Every wait is bounded: a
// warp that gives up sets the error flag, skips its remaining waits but keeps
// arriving, so both sides always finish the same number of rows and every block
// barrier is reached (the results of such a launch are invalid and the host
// reports MUCA_ERR_TIMEOUT).
constexpr int kRing = 4;
constexpr int kSpinLimit = 1 << 20;

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Bounded wait; returns false (and leaves the barrier alone) after kSpinLimit tries.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity)
{
    for (int i = 0; i < kSpinLimit; ++i)
        if (mbar_try(bar, parity)) return true;
    return false;
}

// Consumer side of one Ising / MUMA sweep: as ising_sweep, with the random words
// of row y read from ring slot (k % kRing).
template <int SYS, int L, int RECORD>
__device__ __forceinline__ void ising_sweep_pc(uint32_t *__restrict__ lat, int ps, int &bR,
                                               uint32_t *__restrict__ sTH, const uint4 *__restrict__ ring,
                                               unsigned long long *full, unsigned long long *empty, int &k,
                                               bool &bad)
{
    constexpr int WR = ising_words_per_row(L);
    constexpr int C = (SYS == kMuma) ? 10 : 5;
    constexpr int RS = C + 1;
    constexpr int G = L / 4;  // Philox blocks per row
    uint32_t up[WR], cur[WR], dn[WR], first[WR], nxt[WR], old[WR];
#pragma unroll
    for (int j = 0; j < WR; ++j) {
        up[j] = lat[((L - 1) * WR + j) * ps];
        cur[j] = lat[j * ps];
        dn[j] = lat[(WR + j) * ps];
        first[j] = 0u;
        nxt[j] = 0u;
    }
#pragma unroll 1
    for (int y = 0; y < L; ++y) {
        if (y + 2 < L) {
#pragma unroll
            for (int j = 0; j < WR; ++j) nxt[j] = lat[((y + 2) * WR + j) * ps];
        }
#pragma unroll
        for (int j = 0; j < WR; ++j) old[j] = cur[j];
        const int slot = k % kRing;
        if (!bad && !mbar_wait(&full[slot], (unsigned)((k / kRing) & 1))) bad = true;
        const uint4 *ru = ring + (size_t)slot * G * 32;
        auto site = [&](int x, int &c0, int &c1, int &d0, int &d1) {
            const int s = bit_at<WR>(old, x);
            const int l = bit_at<WR>(old, (x + L - 1) % L);
            const int r = (x == L - 1) ? bit_at<WR>(cur, 0) : bit_at<WR>(old, x + 1);
            const int n1 = l + r + bit_at<WR>(up, x) + bit_at<WR>(dn, x);
            const int k0 = s ? n1 : 4 - n1;
            const int k1 = k0 - 1 + 2 * (l ^ s);
            if (SYS == kMuma) {
                c0 = 5 * s + k0;
                c1 = 5 * s + k1;
                d0 = d1 = (2 * s - 1) * RS;
            } else {
                c0 = k0;
                c1 = k1;
                d0 = (k0 - 2) * RS;
                d1 = (k1 - 2) * RS;
            }
        };
        int c0, c1, d0, d1;
        site(0, c0, c1, d0, d1);
        uint32_t T0 = sTH[bR + c0], T1 = 0u;
        bool accP = false;
        int dRp = 0;
        uint4 u = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int x = 0; x < L; ++x) {
            if ((x & 3) == 0) u = ru[(x / 4) * 32];
            const uint32_t uw = word_of(u, x & 3);
            bR = accP ? bR + dRp : bR;
            const int dR = accP ? d1 : d0;
            const uint32_t T = accP ? T1 : T0;
            if (x + 1 < L) {
                int n0, n1c, e0, e1;
                site(x + 1, n0, n1c, e0, e1);
                T0 = sTH[bR + n0];
                T1 = sTH[bR + dR + n1c];
                d0 = e0;
                d1 = e1;
            }
            const bool acc = (T == kAlways) || (uw < T);
            if (acc) cur[x >> 5] ^= 1u << (x & 31);
            if (RECORD == 0) atomicAdd(&sTH[(acc ? bR + dR : bR) + C], 1u);
            accP = acc;
            dRp = dR;
        }
        bR = accP ? bR + dRp : bR;
#pragma unroll
        for (int j = 0; j < WR; ++j) lat[(y * WR + j) * ps] = cur[j];
        mbar_arrive(&empty[slot]);
        ++k;
        if (y == 0) {
#pragma unroll
            for (int j = 0; j < WR; ++j) first[j] = cur[j];
        }
#pragma unroll
        for (int j = 0; j < WR; ++j) {
            up[j] = cur[j];
            cur[j] = dn[j];
            dn[j] = (y + 2 < L) ? nxt[j] : first[j];
        }
    }
    if (RECORD == 1) atomicAdd(&sTH[bR + C], 1u);
}

// Consumer side of one Potts sweep (two words a site: proposal, acceptance).
template <int L, int RECORD>
__device__ __forceinline__ void potts_sweep_pc(uint32_t *__restrict__ lat, int ps, int &bR,
                                               uint32_t *__restrict__ sTH, const uint4 *__restrict__ ring,
                                               unsigned long long *full, unsigned long long *empty, int &k,
                                               bool &bad, uint32_t q)
{
    constexpr int WR = potts_words_per_row(L);
    constexpr int RS = 10;
    constexpr int G = L / 2;
    uint32_t up[WR], cur[WR], dn[WR], first[WR], nxt[WR], old[WR];
#pragma unroll
    for (int j = 0; j < WR; ++j) {
        up[j] = lat[((L - 1) * WR + j) * ps];
        cur[j] = lat[j * ps];
        dn[j] = lat[(WR + j) * ps];
        first[j] = 0u;
        nxt[j] = 0u;
    }
    const uint32_t qm1 = q - 1u;
#pragma unroll 1
    for (int y = 0; y < L; ++y) {
        if (y + 2 < L) {
#pragma unroll
            for (int j = 0; j < WR; ++j) nxt[j] = lat[((y + 2) * WR + j) * ps];
        }
#pragma unroll
        for (int j = 0; j < WR; ++j) old[j] = cur[j];
        const int slot = k % kRing;
        if (!bad && !mbar_wait(&full[slot], (unsigned)((k / kRing) & 1))) bad = true;
        const uint4 *ru = ring + (size_t)slot * G * 32;
        auto site = [&](int x, uint32_t uprop, uint32_t lnw, uint32_t &nw, int &c0, int &c1, int &d0, int &d1) {
            const uint32_t o = nib_at<WR>(old, x);
            const uint32_t nl = nib_at<WR>(old, (x + L - 1) % L);
            const uint32_t nr = (x == L - 1) ? nib_at<WR>(cur, 0) : nib_at<WR>(old, x + 1);
            const uint32_t nu = nib_at<WR>(up, x), nd = nib_at<WR>(dn, x);
            uint32_t v = o + 1u + __umulhi(uprop, qm1);
            v = (v >= q) ? v - q : v;
            nw = v;
            const int rest = (int)(nr == o) + (int)(nu == o) + (int)(nd == o) - (int)(nr == v) - (int)(nu == v) -
                             (int)(nd == v);
            const int dE0 = rest + (int)(nl == o) - (int)(nl == v);
            const int dE1 = rest + (int)(lnw == o) - (int)(lnw == v);
            c0 = dE0 + 4;
            c1 = dE1 + 4;
            d0 = dE0 * RS;
            d1 = dE1 * RS;
        };
        uint4 u = ru[0];
        uint4 u_next = ru[32];
        uint32_t nwc;
        int c0, c1, d0, d1;
        site(0, u.x, 0u, nwc, c0, c1, d0, d1);
        uint32_t T0 = sTH[bR + c0], T1 = 0u;
        bool accP = false;
        int dRp = 0;
#pragma unroll
        for (int x = 0; x < L; ++x) {
            if ((x & 1) == 0) {
                u = (x == 0) ? u : u_next;
                if (x + 2 < L) u_next = ru[(x / 2 + 1) * 32];
            }
            const uint32_t u_acc = (x & 1) ? u.w : u.y;
            bR = accP ? bR + dRp : bR;
            const int dR = accP ? d1 : d0;
            const uint32_t T = accP ? T1 : T0;
            const uint32_t nw = nwc;
            if (x + 1 < L) {
                const uint32_t uprop = ((x + 1) & 1) ? u.z : u_next.x;
                int n0, n1c, e0, e1;
                site(x + 1, uprop, nw, nwc, n0, n1c, e0, e1);
                T0 = sTH[bR + n0];
                T1 = sTH[bR + dR + n1c];
                d0 = e0;
                d1 = e1;
            }
            const bool acc = (T == kAlways) || (u_acc < T);
            if (acc) {
                const int wi = (4 * x) >> 5, sh = (4 * x) & 31;
                cur[wi] = (cur[wi] & ~(15u << sh)) | (nw << sh);
            }
            if (RECORD == 0) atomicAdd(&sTH[(acc ? bR + dR : bR) + 9], 1u);
            accP = acc;
            dRp = dR;
        }
        bR = accP ? bR + dRp : bR;
#pragma unroll
        for (int j = 0; j < WR; ++j) lat[(y * WR + j) * ps] = cur[j];
        mbar_arrive(&empty[slot]);
        ++k;
        if (y == 0) {
#pragma unroll
            for (int j = 0; j < WR; ++j) first[j] = cur[j];
        }
#pragma unroll
        for (int j = 0; j < WR; ++j) {
            up[j] = cur[j];
            cur[j] = dn[j];
            dn[j] = (y + 2 < L) ? nxt[j] : first[j];
        }
    }
    if (RECORD == 1) atomicAdd(&sTH[bR + 9], 1u);
}

// Producer side: the Philox blocks of one sweep, row by row, for the walkers of
// the paired consumer warp.  G blocks a row: L/4 (one word a site) or L/2 (two).
template <int SYS, int L>
__device__ __forceinline__ void produce_sweep(uint32_t g, uint32_t wid, const uint32_t (&rk)[20], uint4 *ring,
                                              unsigned long long *full, unsigned long long *empty, int &k, bool &bad)
{
    constexpr int G = (SYS == kPotts) ? L / 2 : L / 4;
#pragma unroll 1
    for (int y = 0; y < L; ++y) {
        const int slot = k % kRing;
        if (!bad && !mbar_wait(&empty[slot], (unsigned)(((k / kRing) & 1) ^ 1))) bad = true;
        uint4 *wu = ring + (size_t)slot * G * 32;
#pragma unroll
        for (int gq = 0; gq < G; ++gq)
            wu[gq * 32] = philox4x32_10_rk(make_uint4((uint32_t)(y * G + gq), g, wid, kTagSweep), rk);
        mbar_arrive(&full[slot]);
        ++k;
    }
}

// Shared memory of the producer/consumer block: thresholds + histogram rows,
// then one ring per consumer warp, then the mbarriers.
__host__ __device__ constexpr size_t pc_ring_bytes(int system, int L)
{
    return (size_t)kRing * ((system == kPotts) ? L / 2 : L / 4) * 32 * 16;
}

template <int SYS, int L>
__device__ __forceinline__ void sweep_block_pc(const SpinSweepArgs &a, int w0, int slot_id, uint32_t *smem)
{
    constexpr int C = num_cols(SYS);
    constexpr int RS = C + 1;
    constexpr int G = (SYS == kPotts) ? L / 2 : L / 4;
    const int ncw = blockDim.x / 64;  // consumer warps (= producer warps)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool producer = warp >= ncw;
    const int pair = producer ? warp - ncw : warp;
    uint32_t *sTH = smem;
    const size_t th_bytes = ((size_t)a.B * RS * 4 + 15) / 16 * 16;
    uint4 *ring = (uint4 *)((char *)smem + th_bytes) + (size_t)pair * kRing * G * 32 + lane;
    unsigned long long *bars =
        (unsigned long long *)((char *)smem + th_bytes + (size_t)ncw * pc_ring_bytes(SYS, L));
    unsigned long long *full = bars + (size_t)pair * 2 * kRing, *empty = full + kRing;

    const int tid = threadIdx.x;
    for (int i = tid; i < a.B * RS; i += blockDim.x) {
        const int b = i / RS, c = i - (i / RS) * RS;
        sTH[i] = (c < C) ? a.T[b * C + c] : 0u;
    }
    if (tid == 0)
        for (int i = 0; i < ncw * 2 * kRing; ++i) mbar_init(bars + i, 32);
    __syncthreads();

    const int w = w0 + pair * 32 + lane;
    const bool active = w < a.p;
    const uint32_t wid = (uint32_t)(w + a.walker_offset);
    const uint32_t g0 = (uint32_t)a.state->sweep_counter;
    uint32_t *lat = a.lattice + (active ? w : 0);
    int bR = (active ? a.bin[w] : 0) * RS;
    unsigned long long *Hb = a.Hpart + (size_t)slot_id * a.B;
    int k = 0;
    bool bad = false;
    // Inactive lanes (w >= p) run the same rows on walker 0's lattice copy in
    // registers only: they read but never store, so every lane arrives on every
    // barrier phase.
    for (int64_t s0 = 0; s0 < a.sweeps; s0 += a.flush_every) {
        const int64_t s1 = (a.sweeps < s0 + a.flush_every) ? a.sweeps : s0 + a.flush_every;
#pragma unroll 1
        for (int64_t sw = s0; sw < s1; ++sw) {
            const uint32_t g = g0 + (uint32_t)sw;
            if (producer) {
                produce_sweep<SYS, L>(g, wid, a.rk, ring, full, empty, k, bad);
            } else if (active) {
                if (a.record == 0) {
                    if (SYS == kPotts)
                        potts_sweep_pc<L, 0>(lat, a.pstride, bR, sTH, ring, full, empty, k, bad, (uint32_t)a.q);
                    else
                        ising_sweep_pc<SYS, L, 0>(lat, a.pstride, bR, sTH, ring, full, empty, k, bad);
                } else {
                    if (SYS == kPotts)
                        potts_sweep_pc<L, 1>(lat, a.pstride, bR, sTH, ring, full, empty, k, bad, (uint32_t)a.q);
                    else
                        ising_sweep_pc<SYS, L, 1>(lat, a.pstride, bR, sTH, ring, full, empty, k, bad);
                }
            } else {
                // inactive consumer lane: keep the barrier protocol, do no work
#pragma unroll 1
                for (int y = 0; y < L; ++y) {
                    const int slot = k % kRing;
                    if (!bad && !mbar_wait(&full[slot], (unsigned)((k / kRing) & 1))) bad = true;
                    mbar_arrive(&empty[slot]);
                    ++k;
                }
            }
        }
        __syncthreads();
        for (int b = tid; b < a.B; b += blockDim.x) {
            const uint32_t c = sTH[b * RS + C];
            if (c) {
                Hb[b] += c;
                sTH[b * RS + C] = 0u;
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(const_cast<int *>(&a.state->err), 1);
    if (!producer && active) a.bin[w] = bR / RS;
}

// ---------------------------------------------------------------------------
// Producer/consumer form with precomputed site codes (Ising and MUMA).
// Shared memory holds the same threshold + histogram rows as above.  The
// producer warp writes, per row, the walkers' random
// words, their old row and, for every site, two column bytes: c0 for "left
// neighbour as it was" and c1 for "left neighbour flipped", both without the up
// neighbour (which only the consumer knows: the row above is final only after
// the consumer has swept it) and, for the last site, without its right
// neighbour (site 0 of the same row).  Four sites are handled at once with
// bytewise arithmetic.  The consumer subtracts the up term (and the right term of
// the last site), derives the bin moves from the two columns and runs the same
// speculative chain as above.  (A variant that stored (threshold, next-row) pairs
// to save the moves was slower: its 8-byte random loads doubled the bank
// conflicts on the critical chain.)
__device__ __forceinline__ uint32_t nib_to_bytes(uint32_t n)  // 4 bits -> 4 bytes of 0/1
{
    return (n * 0x00204081u) & 0x01010101u;
}

template <int L, int WR>
__device__ __forceinline__ uint32_t row_nibble(const uint32_t (&r)[WR], int x)  // bits x..x+3 (x % 4 == 0)
{
    return (r[x >> 5] >> (x & 31)) & 15u;
}

template <int L, int WR>
__device__ __forceinline__ uint32_t row_bit(const uint32_t (&r)[WR], int x)
{
    return (r[x >> 5] >> (x & 31)) & 1u;
}

template <int SYS, int L>
__device__ __forceinline__ void produce_sweep_tn(uint32_t g, uint32_t wid, const uint32_t (&rk)[20],
                                                 const uint32_t *__restrict__ lat, int ps, uint4 *ring_u,
                                                 uint2 *ring_c, uint32_t *ring_r, unsigned long long *full,
                                                 unsigned long long *empty, int &k, bool &bad)
{
    constexpr int WR = ising_words_per_row(L);
    constexpr int G = L / 4;
    constexpr size_t SU = (size_t)G * 32, SC = (size_t)G * 32, SR = (size_t)WR * 32;
    // Rolling rows: o = row y (old), d = row y+1 (old; row 0 final for y = L-1), nn = row y+2
    // prefetched one row ahead.  The producer runs at most kRing rows ahead of the
    // consumer and L >= 2 kRing, so every row it reads has its value for this sweep
    // (rows y, y+1, y+2 not yet swept; row 0 already swept when it is the last row's
    // down neighbour).  The first two rows of a sweep are read after the first wait.
    uint32_t o[WR], d[WR], nn[WR];
#pragma unroll 1
    for (int y = 0; y < L; ++y) {
        const int slot = k % kRing;
        if (!bad && !mbar_wait(&empty[slot], (unsigned)(((k / kRing) & 1) ^ 1))) bad = true;
        if (y == 0) {
#pragma unroll
            for (int j = 0; j < WR; ++j) {
                o[j] = lat[j * ps];
                d[j] = lat[(WR + j) * ps];
            }
        }
        const int y2 = (y + 2 < L) ? y + 2 : y + 2 - L;
        if (y + 1 < L) {
#pragma unroll
            for (int j = 0; j < WR; ++j) nn[j] = lat[(y2 * WR + j) * ps];
        }
        uint4 *wu = ring_u + slot * SU;
        uint2 *wc = ring_c + slot * SC;
        uint32_t *wr = ring_r + slot * SR;
#pragma unroll
        for (int j = 0; j < WR; ++j) wr[j * 32] = o[j];
#pragma unroll
        for (int gq = 0; gq < G; ++gq) {
            wu[gq * 32] = philox4x32_10_rk(make_uint4((uint32_t)(y * G + gq), g, wid, kTagSweep), rk);
            const int x = 4 * gq;
            const uint32_t s4 = row_nibble<L, WR>(o, x);
            // left neighbours x-1..x+2 and right neighbours x+1..x+4 (periodic in x)
            uint32_t l4 = (s4 << 1) & 15u, r4 = s4 >> 1;
            l4 |= row_bit<L, WR>(o, (x + L - 1) % L);
            if (x + 4 < L) r4 |= row_bit<L, WR>(o, x + 4) << 3;
            else r4 |= ((s4 >> 3) & 1u) << 3;  // last site: right neighbour left out (anti = 0)
            const uint32_t S = nib_to_bytes(s4);
            const uint32_t A = nib_to_bytes(l4) ^ S;  // left anti-aligned
            const uint32_t Bq = nib_to_bytes(r4) ^ S;
            const uint32_t D = nib_to_bytes(row_nibble<L, WR>(d, x)) ^ S;
            const uint32_t k0 = 0x04040404u - (A + Bq + D);  // 4 - anti-aligned (without up), per byte
            const uint32_t k1 = k0 + 2u * A - 0x01010101u;   // left neighbour flipped
            if (SYS == kMuma) {
                const uint32_t s5 = S * 5u;
                wc[gq * 32] = make_uint2(s5 + k0, s5 + k1);
            } else {
                wc[gq * 32] = make_uint2(k0, k1);
            }
        }
        mbar_arrive(&full[slot]);
        ++k;
#pragma unroll
        for (int j = 0; j < WR; ++j) {
            o[j] = d[j];
            d[j] = nn[j];
        }
    }
}

template <int SYS, int L, int RECORD>
__device__ __forceinline__ void ising_sweep_tc(uint32_t *__restrict__ lat, int ps, int &bR, uint32_t *__restrict__ sTH,
                                               const uint4 *__restrict__ ring_u, const uint2 *__restrict__ ring_c,
                                               const uint32_t *__restrict__ ring_r, unsigned long long *full,
                                               unsigned long long *empty, int &k, bool &bad)
{
    constexpr int WR = ising_words_per_row(L);
    constexpr int C = (SYS == kMuma) ? 10 : 5;
    constexpr int RS = C + 1;
    constexpr int G = L / 4;
    constexpr size_t SU = (size_t)G * 32, SC = (size_t)G * 32, SR = (size_t)WR * 32;
    // bin-row move of an accepted flip, from its column: Ising (c - 2) rows,
    // MUMA one row down for s = +1 (c < 5) and one up for s = -1
    auto move = [](uint32_t c) -> int {
        return (SYS == kMuma) ? ((c >= 5u) ? RS : -RS) : ((int)c - 2) * RS;
    };
    uint32_t up[WR], cur[WR];
#pragma unroll
    for (int j = 0; j < WR; ++j) up[j] = lat[((L - 1) * WR + j) * ps];
#pragma unroll 1
    for (int y = 0; y < L; ++y) {
        const int slot = k % kRing;
        if (!bad && !mbar_wait(&full[slot], (unsigned)((k / kRing) & 1))) bad = true;
        const uint4 *ru = ring_u + slot * SU;
        const uint2 *rc = ring_c + slot * SC;
        const uint32_t *rr = ring_r + slot * SR;
        uint32_t ua[WR];
#pragma unroll
        for (int j = 0; j < WR; ++j) {
            cur[j] = rr[j * 32];
            ua[j] = up[j] ^ cur[j];  // up neighbour anti-aligned
        }
        const uint32_t sLast = row_bit<L, WR>(cur, L - 1);
        uint2 cd = rc[0];
        {
            const uint32_t u4 = nib_to_bytes(row_nibble<L, WR>(ua, 0));
            cd.x -= u4;
            cd.y -= u4;
        }
        uint2 cdn = cd;
        const uint32_t c00 = cd.x & 0xffu;
        uint32_t T0 = sTH[bR + (int)c00], T1 = 0u;
        int d0 = move(c00), d1 = 0;
        bool accP = false;
        int dRp = 0;
        uint4 u = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int x = 0; x < L; ++x) {
            const int j4 = x & 3;
            if (j4 == 0) {
                u = ru[(x / 4) * 32];
                cd = cdn;
                if (x + 4 < L) {
                    cdn = rc[(x / 4 + 1) * 32];
                    const uint32_t u4 = nib_to_bytes(row_nibble<L, WR>(ua, x + 4));
                    cdn.x -= u4;
                    cdn.y -= u4;
                }
            }
            const uint32_t uw = word_of(u, j4);
            bR = accP ? bR + dRp : bR;
            const int dR = accP ? d1 : d0;
            const uint32_t T = accP ? T1 : T0;
            if (x + 1 < L) {
                const int jn = (x + 1) & 3;
                const uint32_t wx = (jn == 0) ? cdn.x : cd.x, wy = (jn == 0) ? cdn.y : cd.y;
                uint32_t c0 = (wx >> (8 * jn)) & 0xffu, c1 = (wy >> (8 * jn)) & 0xffu;
                if (x + 1 == L - 1) {
                    // the last site's right neighbour is site 0 of this row, final by now
                    const uint32_t ra = row_bit<L, WR>(cur, 0) ^ sLast;
                    c0 -= ra;
                    c1 -= ra;
                }
                T0 = sTH[bR + (int)c0];
                T1 = sTH[bR + dR + (int)c1];
                d0 = move(c0);
                d1 = move(c1);
            }
            const bool acc = (T == kAlways) || (uw < T);
            if (acc) cur[x >> 5] ^= 1u << (x & 31);
            if (RECORD == 0) atomicAdd(&sTH[(acc ? bR + dR : bR) + C], 1u);
            accP = acc;
            dRp = dR;
        }
        bR = accP ? bR + dRp : bR;
#pragma unroll
        for (int j = 0; j < WR; ++j) {
            lat[(y * WR + j) * ps] = cur[j];
            up[j] = cur[j];
        }
        mbar_arrive(&empty[slot]);  // after the row is stored: the producer reads it later
        ++k;
    }
    if (RECORD == 1) atomicAdd(&sTH[bR + C], 1u);
}

__host__ __device__ constexpr size_t tn_ring_bytes(int L)
{
    return (size_t)kRing * ((size_t)(L / 4) * 32 * 16 + (size_t)(L / 4) * 32 * 8 + (size_t)((L + 31) / 32) * 32 * 4);
}

template <int SYS, int L>
__device__ __forceinline__ void sweep_block_tn(const SpinSweepArgs &a, int w0, int slot_id, uint32_t *smem)
{
    constexpr int C = num_cols(SYS);
    constexpr int RS = C + 1;
    constexpr int G = L / 4;
    const int ncw = blockDim.x / 64;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool producer = warp >= ncw;
    const int pair = producer ? warp - ncw : warp;
    uint32_t *sTH = smem;
    const size_t th_bytes = ((size_t)a.B * RS * 4 + 15) / 16 * 16;
    char *rbase = (char *)smem + th_bytes + (size_t)pair * tn_ring_bytes(L);
    uint4 *ring_u = (uint4 *)rbase + lane;
    uint2 *ring_c = (uint2 *)(rbase + (size_t)kRing * G * 32 * 16) + lane;
    uint32_t *ring_r = (uint32_t *)(rbase + (size_t)kRing * (G * 32 * 16 + G * 32 * 8)) + lane;
    unsigned long long *bars = (unsigned long long *)((char *)smem + th_bytes + (size_t)ncw * tn_ring_bytes(L));
    unsigned long long *full = bars + (size_t)pair * 2 * kRing, *empty = full + kRing;

    const int tid = threadIdx.x;
    for (int i = tid; i < a.B * RS; i += blockDim.x) {
        const int b = i / RS, c = i - (i / RS) * RS;
        sTH[i] = (c < C) ? a.T[b * C + c] : 0u;
    }
    if (tid == 0)
        for (int i = 0; i < ncw * 2 * kRing; ++i) mbar_init(bars + i, 32);
    __syncthreads();

    const int w = w0 + pair * 32 + lane;
    const bool active = w < a.p;
    const uint32_t wid = (uint32_t)(w + a.walker_offset);
    const uint32_t g0 = (uint32_t)a.state->sweep_counter;
    uint32_t *lat = a.lattice + (active ? w : 0);
    int bR = (active ? a.bin[w] : 0) * RS;
    unsigned long long *Hb = a.Hpart + (size_t)slot_id * a.B;
    int k = 0;
    bool bad = false;
    for (int64_t s0 = 0; s0 < a.sweeps; s0 += a.flush_every) {
        const int64_t s1 = (a.sweeps < s0 + a.flush_every) ? a.sweeps : s0 + a.flush_every;
#pragma unroll 1
        for (int64_t sw = s0; sw < s1; ++sw) {
            const uint32_t g = g0 + (uint32_t)sw;
            if (producer) {
                produce_sweep_tn<SYS, L>(g, wid, a.rk, lat, a.pstride, ring_u, ring_c, ring_r, full, empty, k, bad);
            } else if (active) {
                if (a.record == 0)
                    ising_sweep_tc<SYS, L, 0>(lat, a.pstride, bR, sTH, ring_u, ring_c, ring_r, full, empty, k, bad);
                else
                    ising_sweep_tc<SYS, L, 1>(lat, a.pstride, bR, sTH, ring_u, ring_c, ring_r, full, empty, k, bad);
            } else {
#pragma unroll 1
                for (int y = 0; y < L; ++y) {
                    const int slot = k % kRing;
                    if (!bad && !mbar_wait(&full[slot], (unsigned)((k / kRing) & 1))) bad = true;
                    mbar_arrive(&empty[slot]);
                    ++k;
                }
            }
        }
        __syncthreads();
        for (int b = tid; b < a.B; b += blockDim.x) {
            const uint32_t c = sTH[b * RS + C];
            if (c) {
                Hb[b] += c;
                sTH[b * RS + C] = 0u;
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(const_cast<int *>(&a.state->err), 1);
    if (!producer && active) a.bin[w] = bR / RS;
}

template <int SYS, int L>
__global__ void __launch_bounds__(kMaxSweepBlock, 1) k_sweep_spin_tn(const SpinSweepArgs a)
{
    extern __shared__ __align__(16) uint32_t smem[];
    sweep_block_tn<SYS, L>(a, blockIdx.x * (blockDim.x / 2), blockIdx.x, smem);
}

size_t spin_sweep_tn_smem_bytes(int system, int L, int B, int walkers_per_block)
{
    const int ncw = walkers_per_block / 32;
    return ((size_t)B * (num_cols(system) + 1) * 4 + 15) / 16 * 16 + (size_t)ncw * tn_ring_bytes(L) +
           (size_t)ncw * 2 * kRing * sizeof(unsigned long long);
}

template <int SYS, int L>
__global__ void __launch_bounds__(kMaxSweepBlock, 1) k_sweep_spin_pc(const SpinSweepArgs a)
{
    extern __shared__ __align__(16) uint32_t smem[];
    sweep_block_pc<SYS, L>(a, blockIdx.x * (blockDim.x / 2), blockIdx.x, smem);
}

size_t spin_sweep_pc_smem_bytes(int system, int L, int B, int walkers_per_block)
{
    const int ncw = walkers_per_block / 32;
    return ((size_t)B * (num_cols(system) + 1) * 4 + 15) / 16 * 16 + (size_t)ncw * pc_ring_bytes(system, L) +
           (size_t)ncw * 2 * kRing * sizeof(unsigned long long);
}

// One thread block's share of a sweep launch: stage the threshold table in
// shared memory (rows of C thresholds + 1 histogram counter), run walkers
// [w0, w0 + blockDim.x) of the system, flush the block histogram to its
// own uint64 slot `slot` every `flush_every` sweeps (so no uint32 counter can
// overflow) and at the end.
template <int SYS, int L>
__device__ __forceinline__ void sweep_block(const SpinSweepArgs &a, int w0, int slot, uint32_t *smem)
{
    constexpr int C = num_cols(SYS);
    constexpr int RS = C + 1;
    uint32_t *sTH = smem;
    const int tid = threadIdx.x;
    for (int i = tid; i < a.B * RS; i += blockDim.x) {
        const int b = i / RS, c = i - (i / RS) * RS;
        sTH[i] = (c < C) ? a.T[b * C + c] : 0u;
    }
    __syncthreads();

    const int w = w0 + tid;
    const bool active = w < a.p;
    const uint32_t wid = (uint32_t)(w + a.walker_offset);
    const uint32_t g0 = (uint32_t)a.state->sweep_counter;
    uint32_t *lat = a.lattice + (active ? w : 0);
    int bR = (active ? a.bin[w] : 0) * RS;
    unsigned long long *Hb = a.Hpart + (size_t)slot * a.B;

    for (int64_t s0 = 0; s0 < a.sweeps; s0 += a.flush_every) {
        const int64_t s1 = (a.sweeps < s0 + a.flush_every) ? a.sweeps : s0 + a.flush_every;
        if (active) {
            if (a.record == 0) {
#pragma unroll 1
                for (int64_t sw = s0; sw < s1; ++sw) {
                    const uint32_t g = g0 + (uint32_t)sw;
                    if (SYS == kPotts)
                        potts_sweep<L, 0>(lat, a.pstride, bR, sTH, g, wid, a.rk, (uint32_t)a.q);
                    else
                        ising_sweep<SYS, L, 0>(lat, a.pstride, bR, sTH, g, wid, a.rk);
                }
            } else {
#pragma unroll 1
                for (int64_t sw = s0; sw < s1; ++sw) {
                    const uint32_t g = g0 + (uint32_t)sw;
                    if (SYS == kPotts)
                        potts_sweep<L, 1>(lat, a.pstride, bR, sTH, g, wid, a.rk, (uint32_t)a.q);
                    else
                        ising_sweep<SYS, L, 1>(lat, a.pstride, bR, sTH, g, wid, a.rk);
                }
            }
        }
        __syncthreads();
        for (int b = tid; b < a.B; b += blockDim.x) {
            const uint32_t c = sTH[b * RS + C];
            if (c) {
                Hb[b] += c;
                sTH[b * RS + C] = 0u;
            }
        }
        __syncthreads();
    }
    if (active) a.bin[w] = bR / RS;
}

// One system per launch: block k runs walkers [k*blockDim.x, (k+1)*blockDim.x).
template <int SYS, int L>
__global__ void __launch_bounds__(kMaxSweepBlock) k_sweep_spin(const SpinSweepArgs a)
{
    extern __shared__ __align__(16) uint32_t smem[];
    sweep_block<SYS, L>(a, blockIdx.x * blockDim.x, blockIdx.x, smem);
}

// Every system of a batch in one launch: block k runs the tile (system,
// first walker) tiles[k]; the per-system arguments live in device memory.
// The switch dispatches to the same block function as the one-system kernel,
// so a walker's trajectory does not depend on how the launch is grouped.
__global__ void __launch_bounds__(kMaxSweepBlock) k_sweep_batch(const SpinSweepArgs *__restrict__ sys,
                                                                const int2 *__restrict__ tiles)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int2 t = tiles[blockIdx.x];
    const SpinSweepArgs a = sys[t.x];
    const int slot = t.y / blockDim.x;
    switch (a.kind) {
#define MUCA_CASE(S, LL) \
    case (S) * 16 + (LL) / 4: sweep_block<(S), (LL)>(a, t.y, slot, smem); break;
#define MUCA_CASES(S) \
    MUCA_CASE(S, 4) MUCA_CASE(S, 8) MUCA_CASE(S, 12) MUCA_CASE(S, 16) MUCA_CASE(S, 24) MUCA_CASE(S, 32) \
    MUCA_CASE(S, 48) MUCA_CASE(S, 64)
        MUCA_CASES(kIsing)
        MUCA_CASES(kMuma)
        MUCA_CASE(kPotts, 4) MUCA_CASE(kPotts, 8) MUCA_CASE(kPotts, 12) MUCA_CASE(kPotts, 16)
        MUCA_CASE(kPotts, 24) MUCA_CASE(kPotts, 32) MUCA_CASE(kPotts, 48)
#undef MUCA_CASES
#undef MUCA_CASE
    default: break;
    }
}

int sweep_kind(int system, int L) { return system * 16 + L / 4; }

cudaError_t launch_sweep_batch(const SpinSweepArgs *d_sys, const int2 *d_tiles, int ntiles, int block, size_t smem,
                               cudaStream_t s)
{
    k_sweep_batch<<<ntiles, block, smem, s>>>(d_sys, d_tiles);
    return cudaGetLastError();
}

cudaError_t prepare_sweep_batch(size_t smem)
{
    return cudaFuncSetAttribute(k_sweep_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

size_t spin_sweep_smem_bytes(int system, int B) { return (size_t)B * (num_cols(system) + 1) * sizeof(uint32_t); }

static bool supported_L(int L)
{
    return L == 4 || L == 8 || L == 12 || L == 16 || L == 24 || L == 32 || L == 48 || L == 64;
}

bool spin_sweep_supported(int system, int L)
{
    if (system != kIsing && system != kPotts && system != kMuma) return false;
    if (!supported_L(L)) return false;
    const int N = L * L;
    const int B = (system == kPotts) ? 2 * N + 1 : N + 1;
    return spin_sweep_smem_bytes(system, B) <= 227u * 1024u;
}

template <int SYS, int L>
static cudaError_t launch_one(const SpinSweepArgs &a, int block, cudaStream_t s)
{
    const size_t smem = spin_sweep_smem_bytes(SYS, a.B);
    cudaError_t e = cudaFuncSetAttribute(k_sweep_spin<SYS, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nblk = (a.p + block - 1) / block;
    k_sweep_spin<SYS, L><<<nblk, block, smem, s>>>(a);
    return cudaGetLastError();
}

template <int SYS, int L>
static cudaError_t launch_one_pc(const SpinSweepArgs &a, int block, cudaStream_t s)
{
    const size_t smem = spin_sweep_pc_smem_bytes(SYS, L, a.B, block);
    cudaError_t e = cudaFuncSetAttribute(k_sweep_spin_pc<SYS, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nblk = (a.p + block - 1) / block;
    k_sweep_spin_pc<SYS, L><<<nblk, 2 * block, smem, s>>>(a);
    return cudaGetLastError();
}

template <int SYS>
static cudaError_t launch_sys_pc(int L, const SpinSweepArgs &a, int block, cudaStream_t s)
{
    switch (L) {
    case 4: return launch_one_pc<SYS, 4>(a, block, s);
    case 8: return launch_one_pc<SYS, 8>(a, block, s);
    case 12: return launch_one_pc<SYS, 12>(a, block, s);
    case 16: return launch_one_pc<SYS, 16>(a, block, s);
    case 24: return launch_one_pc<SYS, 24>(a, block, s);
    case 32: return launch_one_pc<SYS, 32>(a, block, s);
    case 48: return launch_one_pc<SYS, 48>(a, block, s);
    case 64: return launch_one_pc<SYS, 64>(a, block, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int SYS, int L>
static cudaError_t launch_one_tn(const SpinSweepArgs &a, int block, cudaStream_t s)
{
    const size_t smem = spin_sweep_tn_smem_bytes(SYS, L, a.B, block);
    cudaError_t e = cudaFuncSetAttribute(k_sweep_spin_tn<SYS, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nblk = (a.p + block - 1) / block;
    k_sweep_spin_tn<SYS, L><<<nblk, 2 * block, smem, s>>>(a);
    return cudaGetLastError();
}

template <int SYS>
static cudaError_t launch_sys_tn(int L, const SpinSweepArgs &a, int block, cudaStream_t s)
{
    switch (L) {
    case 4: return launch_one_tn<SYS, 4>(a, block, s);
    case 8: return launch_one_tn<SYS, 8>(a, block, s);
    case 12: return launch_one_tn<SYS, 12>(a, block, s);
    case 16: return launch_one_tn<SYS, 16>(a, block, s);
    case 24: return launch_one_tn<SYS, 24>(a, block, s);
    case 32: return launch_one_tn<SYS, 32>(a, block, s);
    case 48: return launch_one_tn<SYS, 48>(a, block, s);
    case 64: return launch_one_tn<SYS, 64>(a, block, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int SYS>
static cudaError_t launch_sys(int L, const SpinSweepArgs &a, int block, cudaStream_t s)
{
    switch (L) {
    case 4: return launch_one<SYS, 4>(a, block, s);
    case 8: return launch_one<SYS, 8>(a, block, s);
    case 12: return launch_one<SYS, 12>(a, block, s);
    case 16: return launch_one<SYS, 16>(a, block, s);
    case 24: return launch_one<SYS, 24>(a, block, s);
    case 32: return launch_one<SYS, 32>(a, block, s);
    case 48: return launch_one<SYS, 48>(a, block, s);
    case 64: return launch_one<SYS, 64>(a, block, s);
    default: return cudaErrorInvalidValue;
    }
}

bool spin_sweep_pc_fits(int system, int L, int B, int walkers_per_block)
{
    return walkers_per_block % 32 == 0 && 2 * walkers_per_block <= kMaxSweepBlock &&
           spin_sweep_pc_smem_bytes(system, L, B, walkers_per_block) <= 227u * 1024u;
}

bool spin_sweep_tn_fits(int system, int L, int B, int walkers_per_block)
{
    return (system == kIsing || system == kMuma) && L >= 2 * kRing && walkers_per_block % 32 == 0 &&
           2 * walkers_per_block <= kMaxSweepBlock &&
           spin_sweep_tn_smem_bytes(system, L, B, walkers_per_block) <= 227u * 1024u;
}

cudaError_t launch_spin_sweep_tn(int system, int L, const SpinSweepArgs &a, int block, cudaStream_t s)
{
    if (!spin_sweep_supported(system, L) || !spin_sweep_tn_fits(system, L, a.B, block)) return cudaErrorInvalidValue;
    switch (system) {
    case kIsing: return launch_sys_tn<kIsing>(L, a, block, s);
    case kMuma: return launch_sys_tn<kMuma>(L, a, block, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_spin_sweep_pc(int system, int L, const SpinSweepArgs &a, int block, cudaStream_t s)
{
    if (!spin_sweep_supported(system, L) || !spin_sweep_pc_fits(system, L, a.B, block)) return cudaErrorInvalidValue;
    switch (system) {
    case kIsing: return launch_sys_pc<kIsing>(L, a, block, s);
    case kMuma: return launch_sys_pc<kMuma>(L, a, block, s);
    case kPotts: return launch_sys_pc<kPotts>(L, a, block, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_spin_sweep(int system, int L, const SpinSweepArgs &a, int block, cudaStream_t s)
{
    if (!spin_sweep_supported(system, L)) return cudaErrorInvalidValue;
    switch (system) {
    case kIsing: return launch_sys<kIsing>(L, a, block, s);
    case kMuma: return launch_sys<kMuma>(L, a, block, s);
    case kPotts: return launch_sys<kPotts>(L, a, block, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace muca
