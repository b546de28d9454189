// sweep_codes.cu -- producer/consumer form with precomputed site codes (Ising,
// MUMA and Potts).
#include "muca_device.cuh"
#include "muca_internal.h"
#include "muca_checks.cuh"
#include "sweep_common.cuh"

namespace muca {

// ---------------------------------------------------------------------------
// Producer/consumer form with precomputed site codes (Ising and MUMA).
// Shared memory holds the same threshold + histogram rows as above.  The
// producer warp writes, per row, the walkers' random
// words (clamped, see clamp_words), their old row and, for every site, two column
// bytes holding 4 c (byte offsets into a threshold row): c0 for "left
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

// The random words handed to a code-form consumer are min(u, 2^32 - 2).  With
// that clamp the acceptance "T == always or u < T" becomes the single compare
// u' < T: for T = 2^32 - 1 (always) every u' is below it, and for any smaller T
// the only changed word, 2^32 - 1, is rejected before and after.
__device__ __forceinline__ uint4 clamp_words(uint4 u)
{
    u.x = min(u.x, 0xFFFFFFFEu);
    u.y = min(u.y, 0xFFFFFFFEu);
    u.z = min(u.z, 0xFFFFFFFEu);
    u.w = min(u.w, 0xFFFFFFFEu);
    return u;
}

// Producer warps per consumer warp in the Ising/MUMA code form (the Potts form
// has kPottsProducers).  One Philox4x32-10 block costs a scheduler about 90
// cycles of integer-multiply throughput and a single warp reaches about 134
// cycles a block, so one producer cannot keep up with its consumer; the row's
// site groups are split over the producers (on other schedulers), which arrive
// together on the row's FULL barrier.
constexpr int kCodeProducers = 2;

template <int WR>
__device__ __forceinline__ void rotate_words(uint32_t (&o)[WR])  // o[e] <- o[e+1], cyclic
{
    const uint32_t t = o[0];
#pragma unroll
    for (int e = 0; e + 1 < WR; ++e) o[e] = o[e + 1];
    o[WR - 1] = t;
}

// Warp roles of a code-form block of one or two walker warps (ncw).  The block
// has 4 ncw warps, laid out so that, with warp w issuing from scheduler w mod 4,
// every consumer has a scheduler to itself (its serial chain is what sets the
// pace) and the two producers of a consumer share another one:
//   ncw = 1: [C0, idle, P0.0, P0.1]
//   ncw = 2: [C0, C1, P0.0, P1.0, idle, idle, P0.1, P1.1]   (Pc.k: part k for consumer c)
// Idle warps only take part in the block-wide barriers of the histogram flush
// (the Potts form makes them a third producer part, see kPottsProducers).
enum { kRoleConsumer = 0, kRoleProducer = 1, kRoleIdle = 2 };
struct CodeRole {
    int kind, pair, part;
};
__device__ __forceinline__ CodeRole code_role(int warp, int ncw)
{
    if (ncw == 1) {
        if (warp == 0) return CodeRole{kRoleConsumer, 0, 0};
        if (warp == 1) return CodeRole{kRoleIdle, 0, 0};
        return CodeRole{kRoleProducer, 0, warp - 2};
    }
    const int sch = warp & 3, grp = warp >> 2;
    if (sch < 2) return grp == 0 ? CodeRole{kRoleConsumer, sch, 0} : CodeRole{kRoleIdle, 0, 0};
    return CodeRole{kRoleProducer, sch - 2, grp};
}
constexpr int kCodeWarpsPerWalkerWarp = 4;

template <int SYS, int L, int PART>
__device__ __forceinline__ void produce_sweep_tn(uint32_t g, uint32_t wid, const uint32_t (&rk)[20],
                                                 const uint32_t *__restrict__ lat, int ps, uint4 *ring_u,
                                                 uint2 *ring_c, uint32_t *ring_r, unsigned long long *full,
                                                 unsigned long long *empty, int &k, bool &bad, int drop_k)
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
        if (PART == 0) {
#pragma unroll
            for (int j = 0; j < WR; ++j) wr[j * 32] = o[j];
        }
        constexpr int g_lo = PART * G / kCodeProducers, g_hi = (PART + 1) * G / kCodeProducers;
#pragma unroll
        for (int gq = g_lo; gq < g_hi; ++gq) {
            wu[gq * 32] = clamp_words(philox4x32_10_rk(make_uint4((uint32_t)(y * G + gq), g, wid, kTagSweep), rk));
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
            // columns as byte offsets (4 c) into a threshold row, per byte
            const uint32_t k0 = (0x04040404u - (A + Bq + D)) << 2;  // 4 - anti-aligned (without up)
            const uint32_t k1 = k0 + 8u * A - 0x04040404u;          // left neighbour flipped
            if (SYS == kMuma) {
                const uint32_t s5 = S * 20u;
                wc[gq * 32] = make_uint2(s5 + k0, s5 + k1);
            } else {
                wc[gq * 32] = make_uint2(k0, k1);
            }
        }
        if (k != drop_k) mbar_arrive(&full[slot]);
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
                                               unsigned long long *empty, int &k, bool &bad, unsigned long long *obs,
                                               unsigned &nacc)
{
    int pc = 0;  // -1 spins of the final rows (observables)
    constexpr int WR = ising_words_per_row(L);
    constexpr int C = (SYS == kMuma) ? 10 : 5;
    constexpr int RS = C + 1;
    constexpr int G = L / 4;
    constexpr size_t SU = (size_t)G * 32, SC = (size_t)G * 32, SR = (size_t)WR * 32;
    // The chain works in 32-bit shared-window byte addresses: bB = table base + 4 RS bin and the
    // producer's columns are 4 c, so a threshold address is one add and the bin's histogram
    // counter an immediate offset from the (already updated) bin address.
    const int sbase = (int)__cvta_generic_to_shared(sTH);
    auto th = [sbase](int addr) -> uint32_t {
        uint32_t v;
        asm("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(checked_addr(addr, sbase)));
        return v;
    };
    // bin-row move of an accepted flip in bytes: Ising (c - 2) rows from the column,
    // MUMA one row up for s = +1 and one down for s = -1 (the old spin of the site)
    auto move = [](uint32_t cb) -> int { return ((int)cb - 8) * RS; };
    int bB = sbase + bR * 4;
    uint32_t up[WR], cur[WR], old[WR];
#pragma unroll
    for (int j = 0; j < WR; ++j) up[j] = lat[((L - 1) * WR + j) * ps];
    // two rows an iteration from L = 32 up (2-4 % there; L = 16 rows are short enough that the
    // larger body costs more than the loop overhead it saves)
    constexpr int kRowUnroll = (L >= 32) ? 2 : 1;
#pragma unroll kRowUnroll
    for (int y = 0; y < L; ++y) {
        const int slot = k % kRing;
        if (!bad && !mbar_wait(&full[slot], (unsigned)((k / kRing) & 1))) bad = true;
        if (bad) {  // a wait gave up: the ring is out of step, so nothing more is computed
            mbar_arrive(&empty[slot]);
            ++k;
            continue;
        }
        const uint4 *ru = ring_u + slot * SU;
        const uint2 *rc = ring_c + slot * SC;
        const uint32_t *rr = ring_r + slot * SR;
        uint32_t ua[WR];
#pragma unroll
        for (int j = 0; j < WR; ++j) {
            cur[j] = rr[j * 32];
            old[j] = cur[j];
            ua[j] = up[j] ^ cur[j];  // up neighbour anti-aligned
        }
        const uint32_t sLast = row_bit<L, WR>(cur, L - 1);
        uint2 cd = rc[0];
        {
            const uint32_t u4 = nib_to_bytes(row_nibble<L, WR>(ua, 0)) << 2;
            cd.x -= u4;
            cd.y -= u4;
        }
        uint2 cdn = cd;
        const uint32_t c00 = cd.x & 0xffu;
        uint32_t T0 = th(bB + (int)c00), T1 = 0u;
        int d0 = move(c00), d1 = 0;
        bool accP = false;
        uint4 u = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int x = 0; x < L; ++x) {
            const int j4 = x & 3;
            if (j4 == 0) {
                u = ru[(x / 4) * 32];
                cd = cdn;
                if (x + 4 < L) {
                    cdn = rc[(x / 4 + 1) * 32];
                    const uint32_t u4 = nib_to_bytes(row_nibble<L, WR>(ua, x + 4)) << 2;
                    cdn.x -= u4;
                    cdn.y -= u4;
                }
            }
            const uint32_t uw = word_of(u, j4);
            const int dR = (SYS == kMuma) ? (row_bit<L, WR>(old, x) ? 4 * RS : -4 * RS) : (accP ? d1 : d0);
            const uint32_t T = accP ? T1 : T0;
            if (x + 1 < L) {
                const int jn = (x + 1) & 3;
                const uint32_t wx = (jn == 0) ? cdn.x : cd.x, wy = (jn == 0) ? cdn.y : cd.y;
                // byte jn of the packed codes (selector bytes 4 pick zeros)
                uint32_t c0 = __byte_perm(wx, 0u, 0x4440u | (uint32_t)jn);
                uint32_t c1 = __byte_perm(wy, 0u, 0x4440u | (uint32_t)jn);
                if (x + 1 == L - 1) {
                    // the last site's right neighbour is site 0 of this row, final by now
                    const uint32_t ra = (row_bit<L, WR>(cur, 0) ^ sLast) << 2;
                    c0 -= ra;
                    c1 -= ra;
                }
                T0 = th(bB + (int)c0);
                T1 = th(bB + dR + (int)c1);
                if (SYS != kMuma) {
                    d0 = move(c0);
                    d1 = move(c1);
                }
            }
            const bool acc = uw < T;  // the producer's clamp makes this "always or u < T"
            if (acc) cur[x >> 5] ^= 1u << (x & 31);
            bB = acc ? bB + dR : bB;
            if (RECORD == 0)
                asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(checked_addr(bB + 4 * C, sbase)), "r"(1u) : "memory");
            accP = acc;
        }
#pragma unroll
        for (int j = 0; j < WR; ++j) {
            lat[(y * WR + j) * ps] = cur[j];
            pc += __popc(cur[j]);
            nacc += __popc(old[j] ^ cur[j]);
            up[j] = cur[j];
        }
        mbar_arrive(&empty[slot]);  // after the row is stored: the producer reads it later
        ++k;
    }
    bR = (bB - sbase) / 4;
    if (RECORD == 1) atomicAdd(&sTH[checked_word(bR + C)], 1u);
    if (SYS == kIsing && obs && !bad) record_observables(obs, bR / RS, L * L, pc);
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
    constexpr int NP = kCodeProducers;
    const int ncw = blockDim.x / (32 * kCodeWarpsPerWalkerWarp);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const CodeRole role = code_role(warp, ncw);
    const bool producer = role.kind == kRoleProducer, consumer = role.kind == kRoleConsumer;
    const int pair = role.pair, part = role.part;
    const int drop_k = (blockIdx.x == 0 && producer && pair == 0 && part == 0) ? a.debug_drop_row : -1;
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
    if (tid == 0)  // per pair: FULL[kRing] (NP producer warps arrive), EMPTY[kRing] (the consumer)
        for (int i = 0; i < ncw * 2 * kRing; ++i) mbar_init(bars + i, ((i / kRing) % 2 == 0) ? 32 * NP : 32);
    set_block_spin_limit(a.spin_limit);
    checks_begin(a.B * RS, a.debug_check);
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
    const int r_lo = a.bin_lo * RS, r_hi = a.bin_hi * RS;
    int tst = (consumer && active && a.tun) ? a.tun[w] : 0;
    unsigned ev = 0;
    unsigned long long nacc = 0;
    for (int64_t s0 = 0; s0 < a.sweeps; s0 += a.flush_every) {
        const int64_t s1 = (a.sweeps < s0 + a.flush_every) ? a.sweeps : s0 + a.flush_every;
#pragma unroll 1
        for (int64_t sw = s0; sw < s1; ++sw) {
            const uint32_t g = g0 + (uint32_t)sw;
            if (producer) {
                if (part == 0)
                    produce_sweep_tn<SYS, L, 0>(g, wid, a.rk, lat, a.pstride, ring_u, ring_c, ring_r, full, empty, k, bad,
                                                drop_k);
                else
                    produce_sweep_tn<SYS, L, 1>(g, wid, a.rk, lat, a.pstride, ring_u, ring_c, ring_r, full, empty, k, bad,
                                                -1);
            } else if (consumer && active) {
                unsigned na = 0;
                if (a.record == 0)
                    ising_sweep_tc<SYS, L, 0>(lat, a.pstride, bR, sTH, ring_u, ring_c, ring_r, full, empty, k, bad,
                                              a.obs, na);
                else
                    ising_sweep_tc<SYS, L, 1>(lat, a.pstride, bR, sTH, ring_u, ring_c, ring_r, full, empty, k, bad,
                                              a.obs, na);
                nacc += na;
                tunnel_step(bR, r_lo, r_hi, tst, ev);
            } else if (consumer) {  // a consumer warp with no walkers keeps the barrier protocol
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
    if (consumer && active) {
        a.bin[w] = bR / RS;
        if (a.tun) a.tun[w] = (uint8_t)tst;
    }
    flush_metrics(a.metrics, nacc, ev);
    checks_end(a.state);
}

template <int SYS, int L>
__global__ void __launch_bounds__(kMaxSweepBlock, 1) k_sweep_spin_tn(const SpinSweepArgs a)
{
    extern __shared__ __align__(16) uint32_t smem[];
    sweep_block_tn<SYS, L>(a, blockIdx.x * (blockDim.x / kCodeWarpsPerWalkerWarp), blockIdx.x, smem);
}

static int potts_tn_depth(int L, int B, int walkers_per_block);
static size_t potts_tn_smem_bytes(int L, int RD, int B, int walkers_per_block);

size_t spin_sweep_tn_smem_bytes(int system, int L, int B, int walkers_per_block)
{
    if (system == kPotts) {
        const int rd = potts_tn_depth(L, B, walkers_per_block);
        return potts_tn_smem_bytes(L, rd ? rd : 2, B, walkers_per_block);
    }
    const int ncw = walkers_per_block / 32;
    return ((size_t)B * (num_cols(system) + 1) * 4 + 15) / 16 * 16 + (size_t)ncw * tn_ring_bytes(L) +
           (size_t)ncw * 2 * kRing * sizeof(unsigned long long);
}

// ---------------------------------------------------------------------------
// Code form for Potts.  The producer warp draws both words of every site and
// makes the proposal v = (s + 1 + mulhi(u, q-1)) mod q itself.  Per row it
// writes the acceptance words, the old and the proposed row (one byte a site)
// and two code bytes a site, c = 4 + dE without the up neighbour: c0 with the
// left neighbour as it was, c1 with the left neighbour recoloured to its own
// proposal.  With ne(n, s) = [n != s], a neighbour n adds ne(n, v) - ne(n, s) to
// dE; the producer evaluates it four sites at a time on bytes.  The consumer
// adds the up neighbour's term the same way, four sites at a time, from the
// final row above (kept in bytes), and the last site's right neighbour (site 0
// of the same row, final by then) once a row.  The chain itself is the one of
// the Ising code form.  RD is the ring depth in rows (4, or 2 where a deeper ring
// does not fit next to the threshold table).
__device__ __forceinline__ uint32_t ne_bytes(uint32_t a, uint32_t b)  // per byte [a != b], bytes < 16
{
    return (((a ^ b) + 0x0F0F0F0Fu) >> 4) & 0x01010101u;
}

__device__ __forceinline__ uint32_t nib_half_to_bytes(uint32_t w, int half)  // 4 nibbles -> 4 bytes
{
    const uint32_t t = __byte_perm(w, 0u, half ? 0x3322u : 0x1100u);
    return (t & 0x000F000Fu) | ((t >> 4) & 0x0F000F00u);
}

__device__ __forceinline__ uint32_t bytes_to_nibs(uint32_t w0, uint32_t w1)  // 8 bytes (< 16) -> 8 nibbles
{
    return __byte_perm(w0 | (w0 >> 4), w1 | (w1 >> 4), 0x6420u);
}

// Potts producers: kPottsProducers parts per consumer.  Parts 0 and 1 share a
// scheduler; part 2 runs on the consumer's scheduler in the two-walker-warp
// layout (the idle warps of the Ising layout) or on a scheduler of its own in
// the one-walker-warp layout, and takes about a third of the row's nibble words.
// A part may own no words; it still waits and arrives on every row.
constexpr int kPottsProducers = 3;
__host__ __device__ constexpr int potts_part_begin(int WR, int part)
{
    // parts 0 / 1 / 2 own [0, n0), [n0, WR - n2), [WR - n2, WR) with n2 = (WR + 1) / 3
    return part <= 0 ? 0 : part == 1 ? (WR - (WR + 1) / 3 + 1) / 2 : part == 2 ? WR - (WR + 1) / 3 : WR;
}

// The producer runs a rolled loop over the row's nibble words (8 sites, 4
// Philox blocks each); its old and down rows rotate through registers so that
// word i is always element 0.  (A fully unrolled row was several times larger
// than the instruction cache serves without fetch stalls.)
// The split table (L = 64, see potts_split_full): the acceptance words travel as their
// upper 16 bits, two to a 32-bit word (uint2 per 4 sites instead of uint4).
template <int L>
struct PottsSplit {
    static constexpr bool on = L > 48;
};

// The 16-bit stand-ins of the split table.  A threshold T keeps 0xFFFF only for "always"
// and min(T >> 16, 0xFFFE) otherwise; a random word u travels as min(u >> 16, 0xFFFE).  Then
// the upper halves decide exactly wherever they differ (u < T when the half of u is the
// smaller, u >= T when it is the larger, u < T whenever T is "always"), and only equal
// halves -- never with T "always" -- need the full words.
__host__ __device__ __forceinline__ uint16_t split_hi(uint32_t T)
{
    return T == kAlways ? (uint16_t)0xFFFFu : (uint16_t)((T >> 16) < 0xFFFEu ? (T >> 16) : 0xFFFEu);
}

// The split table's 16-bit counters, emptied into the block's 64-bit slot: every bin's
// count is taken and cleared with one atomic AND while the consumers keep counting.
// Producer part 1 of every consumer warp scans one F-th of the bins (b = slice mod F) after
// every row it hands over, so every bin is scanned once every F rows and no row carries the
// whole table.  Having produced row k it knows its consumer has finished row k - RD, so the
// consumer counts at most F + RD rows between two scans of a bin, and F + RD <= 2^16 / (32 L
// x consumer warps) keeps every counter below 2^16.  Words are read eight at a time so the
// loads overlap; the AND runs only where a count is not zero.
template <int RS>
__device__ __forceinline__ void split_scan(uint32_t *sTH, unsigned long long *Hb, int B, int lane, int slice, int F)
{
    const int sbase = (int)__cvta_generic_to_shared(sTH);
    for (int b0 = slice + F * lane; b0 < B; b0 += F * 8 * 32) {
        uint32_t w[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int b = b0 + F * 32 * i;
            w[i] = 0u;
            if (b < B)
                asm volatile("ld.shared.u32 %0, [%1];" : "=r"(w[i]) : "r"(checked_addr(sbase + 4 * (b * RS + RS - 1), sbase)));
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int b = b0 + F * 32 * i;
            if (w[i] >> 16) {
                const uint32_t old = atomicAnd(&sTH[b * RS + RS - 1], 0xFFFFu);
                atomicAdd(&Hb[b], (unsigned long long)(old >> 16));
            }
        }
    }
}

template <int L, int RD, int PART>
__device__ __forceinline__ void produce_sweep_potts_tn(uint32_t g, uint32_t wid, const uint32_t (&rk)[20],
                                                       const uint32_t *__restrict__ lat, int ps, uint32_t q,
                                                       void *ring_u, uint2 *ring_c, uint2 *ring_op,
                                                       unsigned long long *full, unsigned long long *empty, int &k,
                                                       bool &bad, int drop_k, uint32_t *sTH, unsigned long long *Hb,
                                                       int B, int F, int &since)
{
    constexpr bool SPLIT = PottsSplit<L>::on;
    constexpr int RSW = 5;  // words a split row (only the split table is scanned)
    static_assert(L % 8 == 0, "whole nibble words a row");
    constexpr int WR = L / 8;
    constexpr size_t S = (size_t)(L / 4) * 32;
    const uint32_t qm1 = q - 1u;
    uint32_t o[WR], d[WR], nn[WR];
#pragma unroll 1
    for (int y = 0; y < L; ++y) {
        const int slot = k % RD;
        if (!bad && !mbar_wait(&empty[slot], (unsigned)(((k / RD) & 1) ^ 1))) bad = true;
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
        uint4 *wu = (uint4 *)ring_u + slot * S;
        uint2 *wu16 = (uint2 *)ring_u + slot * S;
        uint2 *wc = ring_c + slot * S;
        uint2 *wop = ring_op + slot * S;
        // this producer's nibble words [i0, i1); the arrays are rotated so that word i0 is element 0
        constexpr int i0 = potts_part_begin(WR, PART), i1 = potts_part_begin(WR, PART + 1);
#pragma unroll
        for (int e = 0; e < i0; ++e) {
            rotate_words<WR>(o);
            rotate_words<WR>(d);
        }
        uint32_t ob_prev = nib_half_to_bytes(o[WR - 1], 1);  // the four sites left of word i0 (cyclic)
        uint32_t pprev = 0u;                                  // site 0's c1 is never used
        if (i0 > 0 && i0 < i1) {
            // proposal of site 8 i0 - 1 (the second site of its Philox block): the c1
            // column of site 8 i0 has it as its recoloured left neighbour
            const uint4 r = philox4x32_10_rk(make_uint4((uint32_t)(y * (L / 2) + 4 * i0 - 1), g, wid, kTagSweep), rk);
            uint32_t v = (ob_prev >> 24) + 1u + __umulhi(r.z, qm1);
            v = (v >= q) ? v - q : v;
            pprev = v << 24;
        }
#pragma unroll 1
        for (int i = i0; i < i1; ++i) {
            const uint32_t on = o[1 % WR];  // next nibble word, cyclic
            const uint32_t mask_last = (i == WR - 1) ? 0x00FFFFFFu : 0xFFFFFFFFu;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = 2 * i + h;
                const uint32_t ob = nib_half_to_bytes(o[0], h);
                const uint32_t ob_next = nib_half_to_bytes(h == 0 ? o[0] : on, h ^ 1);
                const uint32_t db = nib_half_to_bytes(d[0], h);
                const uint32_t base = (uint32_t)(y * (L / 2) + 2 * j);
                const uint4 r0 = philox4x32_10_rk(make_uint4(base, g, wid, kTagSweep), rk);
                const uint4 r1 = philox4x32_10_rk(make_uint4(base + 1u, g, wid, kTagSweep), rk);
                if (SPLIT)  // upper halves, clamped to 0xFFFE (split_hi)
                    wu16[j * 32] = make_uint2(__vminu2((r0.y >> 16) | (r0.w & 0xFFFF0000u), 0xFFFEFFFEu),
                                              __vminu2((r1.y >> 16) | (r1.w & 0xFFFF0000u), 0xFFFEFFFEu));
                else
                    wu[j * 32] = clamp_words(make_uint4(r0.y, r0.w, r1.y, r1.w));
                const uint32_t up4[4] = {r0.x, r0.z, r1.x, r1.z};
                uint32_t pb = 0u;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    uint32_t v = ((ob >> (8 * e)) & 0xffu) + 1u + __umulhi(up4[e], qm1);
                    v = (v >= q) ? v - q : v;
                    pb |= v << (8 * e);
                }
                const uint32_t R = __funnelshift_r(ob, ob_next, 8);   // right neighbours (old)
                const uint32_t Lo = __funnelshift_l(ob_prev, ob, 8);  // left neighbours (old)
                const uint32_t Lp = __funnelshift_l(pprev, pb, 8);    // left neighbours (recoloured)
                uint32_t nRp = ne_bytes(R, pb), nRo = ne_bytes(R, ob);
                if (h == 1) {  // the row's last site: its right neighbour is added by the consumer
                    nRp &= mask_last;
                    nRo &= mask_last;
                }
                const uint32_t sp = 0x04040404u + nRp + ne_bytes(db, pb);
                const uint32_t so = nRo + ne_bytes(db, ob);
                // every byte stays in [1, 7] and no partial result borrows across bytes
                const uint32_t c0 = sp + ne_bytes(Lo, pb) - so - ne_bytes(Lo, ob);
                const uint32_t c1 = sp + ne_bytes(Lp, pb) - so - ne_bytes(Lp, ob);
                wc[j * 32] = make_uint2(c0, c1);
                wop[j * 32] = make_uint2(ob, pb);
                ob_prev = ob;
                pprev = pb;
            }
            rotate_words<WR>(o);
            rotate_words<WR>(d);
        }
#pragma unroll
        for (int e = i1; e < WR; ++e) {  // back to word 0 first (WR rotations in all)
            rotate_words<WR>(o);
            rotate_words<WR>(d);
        }
        if (k != drop_k) mbar_arrive(&full[slot]);
        ++k;
        if (SPLIT && PART == 1) {  // empty one F-th of the 16-bit counters (split_scan)
            split_scan<RSW>(sTH, Hb, B, (int)(threadIdx.x & 31), since, F);
            if (++since == F) since = 0;
        }
#pragma unroll
        for (int j = 0; j < WR; ++j) {
            o[j] = d[j];
            d[j] = nn[j];
        }
    }
}

// The full acceptance test behind the split table: the walker's acceptance word
// recomputed from its Philox block (block `blk` of the sweep, word y for even
// sites and w for odd ones) against the full threshold T[bin][col] in global
// memory.  Only the row redo (potts_redo_row) calls it, for sites whose upper halves tie.
__device__ __forceinline__ bool potts_split_full(const uint32_t *__restrict__ Tg, int bin, int col, uint32_t blk,
                                                uint32_t g, uint32_t wid, uint32_t key0, uint32_t key1, int odd)
{
    const uint4 r = philox4x32_10_rolled(make_uint4(blk, g, wid, kTagSweep), key0, key1);
    const uint32_t u = odd ? r.w : r.y;
    const uint32_t T = Tg[bin * 9 + col];
    return T == kAlways || u < T;
}

// Row layout of the Potts tables: 11 words a bin (9 thresholds, the counter, a pad word that
// makes the stride odd, so that the bins of a warp's walkers spread over all 32 banks: 1-2 %
// faster than 10 words), 10 at L = 48 (where the 11th would not fit), or at L = 64 the split
// row of 5 words: the 9 upper halves of the thresholds and a 16-bit
// counter, the high half of word 4 (whose low half is column 8).  A visit adds 2^16 to
// word 4, so column 8 never changes; a producer warp empties the 16-bit counters every
// few rows (split_scan) before they can wrap.  Codes are scaled to byte offsets into a
// row (4 c, or 2 c for halfword entries), and a bin move of (c - 4) rows is
// (cs - 4 CSC) MS bytes.
template <int L>
struct PottsRow {
    static constexpr bool split = PottsSplit<L>::on;
    static constexpr int RSW = split ? 5 : (L <= 32 ? 11 : 10);  // words a row
    static constexpr int HW = split ? 4 : 9;               // counter word
    static constexpr uint32_t ONE = split ? 0x10000u : 1u;  // one visit
    static constexpr int CSH = split ? 16 : 0;             // counter shift in its word
    static constexpr int CSC = split ? 2 : 4;              // code scale
    static constexpr int C4 = 4 * CSC;                     // scaled code of dE = 0
    static constexpr int MS = 4 * RSW / CSC;               // bytes a row per unit of scaled code
};

// The row redo behind the split table.  The consumer's pass decides every site on the
// 16-bit stand-ins alone (split_hi), a tie (probability 2^-16 where the threshold is not
// "always") counting as a rejection, and only notes that the row had one.  A lane whose row had a tie then replays the row from its start
// along two trajectories at once: the pass's own (its visits are taken back out of the
// block's 64-bit histogram slot) and the exact one, on which a tie is decided on the full
// words (potts_split_full) and whose visits are added to the slot.  The exact trajectory
// rewrites the row (lattice and up row), the bin and the acceptance count, before the
// ring slot is released.  Up to the first tie the two trajectories coincide.
template <int L>
__device__ __forceinline__ void potts_redo_row(uint32_t *__restrict__ lat, int ps, int y, int sbase, int b0, int &bB,
                                            const uint2 *__restrict__ ru16, const uint2 *__restrict__ rc,
                                            const uint2 *__restrict__ rop, const uint32_t *__restrict__ uOld,
                                            uint32_t *__restrict__ uNew, unsigned long long *Hb, int record,
                                            unsigned &nacc, uint32_t g, uint32_t wid, uint32_t key0, uint32_t key1,
                                            const uint32_t *__restrict__ Tg)
{
    using R = PottsRow<L>;
    constexpr int W4 = L / 4, WR = L / 8;
    auto th = [sbase](int addr) -> uint32_t {
        uint32_t v;
        asm volatile("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(checked_addr(addr, sbase)));
        return v;
    };
    int bw = b0, br = b0;    // byte addresses of the bins: the pass's trajectory, the exact one
    bool pw = false, pr = false;  // the left neighbour's decision on each
    uint32_t f0w = 0u, f0r = 0u, fprev = 0u;
    unsigned naw = 0u, nar = 0u;
#pragma unroll 1
    for (int j = 0; j < W4; ++j) {
        const uint2 op = rop[j * 32];
        const uint32_t ubw = uOld[j * 32];
        const uint32_t np = ne_bytes(ubw, op.y), no = ne_bytes(ubw, op.x);
        const uint32_t cx = (rc[j * 32].x + np - no) << 1, cy = (rc[j * 32].y + np - no) << 1;
        const uint2 h = ru16[j * 32];
        uint32_t amw = 0u, amr = 0u;
#pragma unroll 1
        for (int i = 0; i < 4; ++i) {
            const int x = 4 * j + i;
            const uint32_t uw = ((i < 2 ? h.x : h.y) >> (16 * (i & 1))) & 0xFFFFu;
            int cw = (int)(((pw ? cy : cx) >> (8 * i)) & 0xffu);
            int cr = (int)(((pr ? cy : cx) >> (8 * i)) & 0xffu);
            if (x == L - 1) {  // right neighbour: site 0 of this row, final on each trajectory
                cw += R::CSC * ((int)(f0w != (op.y >> 24)) - (int)(f0w != (op.x >> 24)));
                cr += R::CSC * ((int)(f0r != (op.y >> 24)) - (int)(f0r != (op.x >> 24)));
            }
            const bool aw = uw < th(bw + cw);
            const uint32_t Tr = th(br + cr);
            bool ar = uw < Tr;
            if (uw == Tr)
                ar = potts_split_full(Tg, (br - sbase) / (4 * R::RSW), cr / R::CSC, (uint32_t)(y * (L / 2) + x / 2), g,
                                      wid, key0, key1, x & 1);
            if (aw) {
                bw += (cw - R::C4) * R::MS;
                amw |= 0xffu << (8 * i);
            }
            if (ar) {
                br += (cr - R::C4) * R::MS;
                amr |= 0xffu << (8 * i);
            }
            if (record == 0) {
                atomicAdd(&Hb[(bw - sbase) / (4 * R::RSW)], ~0ull);  // minus one: the pass counted it
                atomicAdd(&Hb[(br - sbase) / (4 * R::RSW)], 1ull);
            }
            pw = aw;
            pr = ar;
        }
        naw += (unsigned)__popc(amw);
        nar += (unsigned)__popc(amr);
        const uint32_t fr = op.x ^ ((op.x ^ op.y) & amr);
        if (j == 0) {
            f0r = fr & 0xffu;
            f0w = (op.x ^ ((op.x ^ op.y) & amw)) & 0xffu;
        }
        uNew[j * 32] = fr;
        if (j & 1) lat[(y * WR + (j >> 1)) * ps] = bytes_to_nibs(fprev, fr);
        fprev = fr;
    }
    bB = br;
    nacc += nar - naw;  // modulo 2^32, like the count itself
}

// The consumer runs a loop over the row's byte words (4 sites each), unrolled
// by two (rolled it lost 16-20 % to loop overhead between the words' chains;
// fully unrolled, L = 48 stalled on instruction fetch), and peels the last
// word, which holds the last site's right-neighbour term.  The final row above
// lives in a per-lane shared-memory row (bytes).  With the split table there are
// two such rows, read and written in turn (the row being decided reads one and
// writes the other), so that a redo still has the row above; otherwise one row
// is rewritten word by word as the current row completes.
template <int L, int RD, int RECORD>
__device__ __forceinline__ void potts_sweep_tc(uint32_t *__restrict__ lat, int ps, int &bR,
                                               uint32_t *__restrict__ sTH, const void *__restrict__ ring_u_,
                                               const uint2 *__restrict__ ring_c, const uint2 *__restrict__ ring_op,
                                               uint32_t *__restrict__ sU, unsigned long long *full,
                                               unsigned long long *empty, int &k, bool &bad, unsigned &nacc,
                                               uint32_t g, uint32_t wid, uint32_t key0, uint32_t key1,
                                               const uint32_t *__restrict__ Tg, unsigned long long *Hb)
{
    static_assert(L % 8 == 0, "whole nibble words a row");
    using R = PottsRow<L>;
    constexpr bool SPLIT = R::split;
    constexpr int WR = L / 8;
    constexpr int W4 = L / 4;
    constexpr size_t S = (size_t)W4 * 32;
    static_assert(!SPLIT || L % 2 == 0, "the up rows alternate: row L - 1 must leave its values in the first");
    const uint4 *ring_u = (const uint4 *)ring_u_;
    const uint2 *ring_u16 = (const uint2 *)ring_u_;
    // byte i of a packed word (selector bytes 4 pick zeros)
    auto byte_of = [](uint32_t w, int i) -> int { return (int)__byte_perm(w, 0u, 0x4440u | (uint32_t)i); };
    // As in the Ising consumer: 32-bit shared-window byte addresses (bB = table base + 4 RSW bin,
    // codes scaled to CSC c), clamped acceptance words, one compare (split: upper halves).
    const int sbase = (int)__cvta_generic_to_shared(sTH);
    auto th = [sbase](int addr) -> uint32_t {
        uint32_t v;
        if (SPLIT)
            asm("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(checked_addr(addr, sbase)));
        else
            asm("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(checked_addr(addr, sbase)));
        return v;
    };
    auto hist = [sbase](int addr) {
        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(checked_addr(addr, sbase)), "r"(R::ONE) : "memory");
    };
    int bB = sbase + bR * 4;
#pragma unroll 1
    for (int y = 0; y < L; ++y) {
        const int slot = k % RD;
        if (!bad && !mbar_wait(&full[slot], (unsigned)((k / RD) & 1))) bad = true;
        if (bad) {  // a wait gave up: the ring is out of step, so nothing more is computed
            mbar_arrive(&empty[slot]);
            ++k;
            continue;
        }
        const uint4 *ru = ring_u + slot * S;
        const uint2 *ru16 = ring_u16 + slot * S;
        const uint2 *rc = ring_c + slot * S;
        const uint2 *rop = ring_op + slot * S;
        const uint32_t *uOld = (SPLIT && (y & 1)) ? sU + S : sU;  // the row above
        uint32_t *uNew = (SPLIT && !(y & 1)) ? sU + S : sU;       // this row, as it is decided
        const int b0 = bB;
        bool tie = false;
        // the acceptance words of byte word j (split: their upper halves)
        auto words = [&](int j) -> uint4 {
            if (SPLIT) {
                const uint2 h = ru16[j * 32];
                return make_uint4(h.x & 0xFFFFu, h.x >> 16, h.y & 0xFFFFu, h.y >> 16);
            }
            return ru[j * 32];
        };
        // code bytes of word j with the up neighbour's term added (bytes stay in [0, 8]),
        // scaled to byte offsets CSC c
        auto codes = [&](int j, uint2 op, uint32_t ubw) -> uint2 {
            uint2 c = rc[j * 32];
            const uint32_t np = ne_bytes(ubw, op.y), no = ne_bytes(ubw, op.x);
            c.x = (c.x + np - no) << (SPLIT ? 1 : 2);
            c.y = (c.y + np - no) << (SPLIT ? 1 : 2);
            return c;
        };
        uint2 opn = rop[0];
        uint2 cdn = codes(0, opn, uOld[0]);
        const int c00 = byte_of(cdn.x, 0);
        uint32_t T0 = th(bB + c00), T1 = 0u;
        int d0 = (c00 - R::C4) * R::MS, d1 = 0;  // bin-row move (c - 4) rows, in bytes
        bool accP = false;
        // decide the current site (threshold T0 or T1 by the previous decision) and
        // load both candidates of the next site, whose code bytes are n0 / n1
        auto site = [&](uint32_t uw, int n0, int n1, uint32_t &am, int i) {
            const int dR = accP ? d1 : d0;
            const uint32_t T = accP ? T1 : T0;
            T0 = th(bB + n0);
            T1 = th(bB + dR + n1);
            d0 = (n0 - R::C4) * R::MS;
            d1 = (n1 - R::C4) * R::MS;
            const bool acc = uw < T;  // the producer's clamp makes this "always or u < T"
            if (SPLIT) tie |= uw == T;  // upper halves equal: the row is redone (potts_redo_row)
            if (acc) am |= 0xffu << (8 * i);
            bB = acc ? bB + dR : bB;
            if (RECORD == 0) hist(bB + 4 * R::HW);
            accP = acc;
        };
        uint32_t fprev = 0u;
#pragma unroll 2
        for (int j = 0; j < W4 - 1; ++j) {
            const uint2 op = opn, cd = cdn;
            const uint4 u = words(j);
            opn = rop[(j + 1) * 32];
            cdn = codes(j + 1, opn, uOld[(j + 1) * 32]);
            uint32_t am = 0u;
            site(u.x, byte_of(cd.x, 1), byte_of(cd.y, 1), am, 0);
            site(u.y, byte_of(cd.x, 2), byte_of(cd.y, 2), am, 1);
            site(u.z, byte_of(cd.x, 3), byte_of(cd.y, 3), am, 2);
            site(u.w, byte_of(cdn.x, 0), byte_of(cdn.y, 0), am, 3);
            nacc += (unsigned)__popc(am);  // 0xff per accepted site: 8 x accepted (divided at the end)
            const uint32_t f = op.x ^ ((op.x ^ op.y) & am);
            uNew[j * 32] = f;
            if (j & 1) lat[(y * WR + (j >> 1)) * ps] = bytes_to_nibs(fprev, f);
            fprev = f;
        }
        {
            constexpr int j = W4 - 1;
            const uint2 op = opn, cd = cdn;
            const uint4 u = words(j);
            uint32_t am = 0u;
            site(u.x, byte_of(cd.x, 1), byte_of(cd.y, 1), am, 0);
            site(u.y, byte_of(cd.x, 2), byte_of(cd.y, 2), am, 1);
            // the last site's right neighbour is site 0 of this row, final by now (word 0 is written)
            const uint32_t f0 = uNew[0] & 0xffu;
            const int t = (int)(f0 != (op.y >> 24)) - (int)(f0 != (op.x >> 24));
            site(u.z, byte_of(cd.x, 3) + R::CSC * t, byte_of(cd.y, 3) + R::CSC * t, am, 2);
            // the last site: decision only
            const int dR = accP ? d1 : d0;
            const uint32_t T = accP ? T1 : T0;
            const bool acc = u.w < T;
            if (SPLIT) tie |= u.w == T;
            if (acc) am |= 0xff000000u;
            bB = acc ? bB + dR : bB;
            if (RECORD == 0) hist(bB + 4 * R::HW);
            nacc += (unsigned)__popc(am);
            const uint32_t f = op.x ^ ((op.x ^ op.y) & am);
            uNew[j * 32] = f;
            lat[(y * WR + WR - 1) * ps] = bytes_to_nibs(fprev, f);
        }
        if (SPLIT && tie)
            potts_redo_row<L>(lat, ps, y, sbase, b0, bB, ru16, rc, rop, uOld, uNew, Hb, RECORD, nacc, g, wid, key0,
                              key1, Tg);
        mbar_arrive(&empty[slot]);  // after the row is stored: the producer reads it later
        ++k;
    }
    bR = (bB - sbase) / 4;
    nacc >>= 3;
    if (RECORD == 1) atomicAdd(&sTH[checked_word(bR + R::HW)], R::ONE);
}

// Shared memory a consumer warp owns: RD ring rows (acceptance words 16 B, or their
// upper halves 8 B at L = 64, codes 8 B, old/proposed bytes 8 B, per group of 4 sites
// and lane) and its up row (two at L = 64).
__host__ __device__ constexpr size_t tnp_warp_bytes(int L, int RD)
{
    return (size_t)RD * (size_t)(L / 4) * 32 * ((L > 48 ? 8 : 16) + 8 + 8) + (size_t)(L > 48 ? 2 : 1) * (L / 4) * 32 * 4;
}

// Bytes of the Potts threshold + counter table: PottsRow<L>::RSW words a bin (11, 10 at
// L = 48, the split rows of 5 at L = 64).
__host__ __device__ constexpr size_t tnp_table_bytes(int L, int B)
{
    return ((size_t)B * (L > 48 ? 20 : (L > 32 ? 40 : 44)) + 15) / 16 * 16;
}

template <int L, int RD>
__device__ __forceinline__ void sweep_block_tnp(const SpinSweepArgs &a, int w0, int slot_id, uint32_t *smem)
{
    using R = PottsRow<L>;
    constexpr int C = 9;
    constexpr int RS = R::RSW;  // words a table row
    constexpr size_t S = (size_t)(L / 4) * 32;
    constexpr int NP = kPottsProducers;
    const int ncw = blockDim.x / (32 * kCodeWarpsPerWalkerWarp);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    CodeRole role = code_role(warp, ncw);
    if (role.kind == kRoleIdle) role = CodeRole{kRoleProducer, ncw == 1 ? 0 : (warp & 1), 2};
    const bool producer = role.kind == kRoleProducer, consumer = role.kind == kRoleConsumer;
    const int pair = role.pair, part = role.part;
    const int drop_k = (blockIdx.x == 0 && producer && pair == 0 && part == 0) ? a.debug_drop_row : -1;
    uint32_t *sTH = smem;
    const size_t th_bytes = tnp_table_bytes(L, a.B);
    constexpr size_t UB = R::split ? 8 : 16;  // ring bytes of a group's acceptance words
    char *rbase = (char *)smem + th_bytes + (size_t)pair * tnp_warp_bytes(L, RD);
    void *ring_u = R::split ? (void *)((uint2 *)rbase + lane) : (void *)((uint4 *)rbase + lane);
    uint2 *ring_c = (uint2 *)(rbase + (size_t)RD * S * UB) + lane;
    uint2 *ring_op = (uint2 *)(rbase + (size_t)RD * S * (UB + 8)) + lane;
    uint32_t *sU = (uint32_t *)(rbase + (size_t)RD * S * (UB + 16)) + lane;
    unsigned long long *bars = (unsigned long long *)((char *)smem + th_bytes + (size_t)ncw * tnp_warp_bytes(L, RD));
    unsigned long long *full = bars + (size_t)pair * 2 * RD, *empty = full + RD;

    const int tid = threadIdx.x;
    if (R::split) {  // halfword rows: 9 upper halves (split_hi), the 16-bit counter
        uint16_t *h = (uint16_t *)smem;
        for (int i = tid; i < a.B * 10; i += blockDim.x) {
            const int b = i / 10, c = i - (i / 10) * 10;
            h[i] = (c < C) ? split_hi(a.T[b * C + c]) : (uint16_t)0;
        }
    } else {
        for (int i = tid; i < a.B * RS; i += blockDim.x) {
            const int b = i / RS, c = i - (i / RS) * RS;
            sTH[i] = (c < C) ? a.T[b * C + c] : 0u;
        }
    }
    if (tid == 0)  // per pair: FULL[RD] (NP producer warps arrive), EMPTY[RD] (the consumer)
        for (int i = 0; i < ncw * 2 * RD; ++i) mbar_init(bars + i, ((i / RD) % 2 == 0) ? 32 * NP : 32);
    set_block_spin_limit(a.spin_limit);
    checks_begin(a.B * RS, a.debug_check);
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
    const int r_lo = a.bin_lo * RS, r_hi = a.bin_hi * RS;
    int tst = (consumer && active && a.tun) ? a.tun[w] : 0;
    unsigned ev = 0;
    unsigned long long nacc = 0;
    // rows between two scans of the split table's 16-bit counters (split_scan)
    const int F = R::split ? 65535 / (ncw * 32 * L) - RD : 0;
    int since = 0;
    if (consumer && active) {  // the row above row 0: row L-1 as the previous launch left it
        constexpr int WR = L / 8;
#pragma unroll
        for (int j = 0; j < L / 4; ++j)
            sU[j * 32] = nib_half_to_bytes(lat[((L - 1) * WR + (j >> 1)) * a.pstride], j & 1);
    }
    for (int64_t s0 = 0; s0 < a.sweeps; s0 += a.flush_every) {
        const int64_t s1 = (a.sweeps < s0 + a.flush_every) ? a.sweeps : s0 + a.flush_every;
#pragma unroll 1
        for (int64_t sw = s0; sw < s1; ++sw) {
            const uint32_t g = g0 + (uint32_t)sw;
            if (producer) {
                if (part == 0)
                    produce_sweep_potts_tn<L, RD, 0>(g, wid, a.rk, lat, a.pstride, (uint32_t)a.q, ring_u, ring_c,
                                                     ring_op, full, empty, k, bad, drop_k, sTH, Hb, a.B, F, since);
                else if (part == 1)
                    produce_sweep_potts_tn<L, RD, 1>(g, wid, a.rk, lat, a.pstride, (uint32_t)a.q, ring_u, ring_c,
                                                     ring_op, full, empty, k, bad, -1, sTH, Hb, a.B, F, since);
                else
                    produce_sweep_potts_tn<L, RD, 2>(g, wid, a.rk, lat, a.pstride, (uint32_t)a.q, ring_u, ring_c,
                                                     ring_op, full, empty, k, bad, -1, sTH, Hb, a.B, F, since);
            } else if (consumer && active) {
                unsigned na = 0;
                if (a.record == 0)
                    potts_sweep_tc<L, RD, 0>(lat, a.pstride, bR, sTH, ring_u, ring_c, ring_op, sU, full, empty, k, bad,
                                             na, g, wid, a.key0, a.key1, a.T, Hb);
                else
                    potts_sweep_tc<L, RD, 1>(lat, a.pstride, bR, sTH, ring_u, ring_c, ring_op, sU, full, empty, k, bad,
                                             na, g, wid, a.key0, a.key1, a.T, Hb);
                nacc += na;
                tunnel_step(bR, r_lo, r_hi, tst, ev);
            } else if (consumer) {
#pragma unroll 1
                for (int y = 0; y < L; ++y) {
                    const int slot = k % RD;
                    if (!bad && !mbar_wait(&full[slot], (unsigned)((k / RD) & 1))) bad = true;
                    mbar_arrive(&empty[slot]);
                    ++k;
                }
            }
        }
        __syncthreads();
        for (int b = tid; b < a.B; b += blockDim.x) {
            const uint32_t c = sTH[b * RS + R::HW] >> R::CSH;
            if (c) {
                Hb[b] += c;
                sTH[b * RS + R::HW] -= c << R::CSH;
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(const_cast<int *>(&a.state->err), 1);
    if (consumer && active) {
        a.bin[w] = bR / RS;
        if (a.tun) a.tun[w] = (uint8_t)tst;
    }
    flush_metrics(a.metrics, nacc, ev);
    checks_end(a.state);
}

template <int L, int RD>
// At most 64 walkers (256 threads) a block: the L = 48 and 64 forms need more than the 128
// registers a thread that 512-thread blocks would leave.
__global__ void __launch_bounds__(kCodeWarpsPerWalkerWarp * 64, 1) k_sweep_potts_tn(const SpinSweepArgs a)
{
    extern __shared__ __align__(16) uint32_t smem[];
    sweep_block_tnp<L, RD>(a, blockIdx.x * (blockDim.x / kCodeWarpsPerWalkerWarp), blockIdx.x, smem);
}

static size_t potts_tn_smem_bytes(int L, int RD, int B, int walkers_per_block)
{
    const int ncw = walkers_per_block / 32;
    return tnp_table_bytes(L, B) + (size_t)ncw * tnp_warp_bytes(L, RD) +
           (size_t)ncw * 2 * RD * sizeof(unsigned long long);
}

// Deepest ring (4 or 2 rows) whose block fits in shared memory; 0 if none does.
static int potts_tn_depth(int L, int B, int walkers_per_block)
{
    if (L < 8 || L > 64 || L % 8 != 0 || !sweep_L_supported(L)) return 0;
    // L = 64 (the split table) is built with the two-row ring only: the four-row one fits
    // 32-walker blocks but not the default 64
    if (L < 64 && potts_tn_smem_bytes(L, 4, B, walkers_per_block) <= 227u * 1024u) return 4;
    if (potts_tn_smem_bytes(L, 2, B, walkers_per_block) <= 227u * 1024u) return 2;
    return 0;
}


template <int SYS, int L>
static cudaError_t launch_one_tn(const SpinSweepArgs &a, int block, cudaStream_t s)
{
    const size_t smem = spin_sweep_tn_smem_bytes(SYS, L, a.B, block);
    cudaError_t e = cudaFuncSetAttribute(k_sweep_spin_tn<SYS, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nblk = (a.p + block - 1) / block;
    k_sweep_spin_tn<SYS, L><<<nblk, kCodeWarpsPerWalkerWarp * block, smem, s>>>(a);
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

bool spin_sweep_tn_fits(int system, int L, int B, int walkers_per_block)
{
    if (system == kPotts)
        return (walkers_per_block == 32 || walkers_per_block == 64) && potts_tn_depth(L, B, walkers_per_block) != 0;
    return (system == kIsing || system == kMuma) && L >= 2 * kRing &&
           (walkers_per_block == 32 || walkers_per_block == 64) &&
           spin_sweep_tn_smem_bytes(system, L, B, walkers_per_block) <= 227u * 1024u;
}

template <int L, int RD>
static cudaError_t launch_one_tnp(const SpinSweepArgs &a, int block, cudaStream_t s)
{
    const size_t smem = potts_tn_smem_bytes(L, RD, a.B, block);
    cudaError_t e = cudaFuncSetAttribute(k_sweep_potts_tn<L, RD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nblk = (a.p + block - 1) / block;
    k_sweep_potts_tn<L, RD><<<nblk, kCodeWarpsPerWalkerWarp * block, smem, s>>>(a);
    return cudaGetLastError();
}

template <int RD>
static cudaError_t launch_potts_tn_rd(int L, const SpinSweepArgs &a, int block, cudaStream_t s)
{
    switch (L) {
    case 8: return launch_one_tnp<8, RD>(a, block, s);
    case 16: return launch_one_tnp<16, RD>(a, block, s);
    case 24: return launch_one_tnp<24, RD>(a, block, s);
    case 32: return launch_one_tnp<32, RD>(a, block, s);
    case 48: return launch_one_tnp<48, RD>(a, block, s);
    case 64:  // the split table: only the two-row ring fits
        if constexpr (RD == 2) return launch_one_tnp<64, 2>(a, block, s);
        return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

static cudaError_t launch_potts_tn(int L, int rd, const SpinSweepArgs &a, int block, cudaStream_t s)
{
    if (rd == 4) return launch_potts_tn_rd<4>(L, a, block, s);
    if (rd == 2) return launch_potts_tn_rd<2>(L, a, block, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_spin_sweep_tn(int system, int L, const SpinSweepArgs &a, int block, cudaStream_t s)
{
    if (!spin_sweep_supported(system, L) || !spin_sweep_tn_fits(system, L, a.B, block)) return cudaErrorInvalidValue;
    switch (system) {
    case kIsing: return launch_sys_tn<kIsing>(L, a, block, s);
    case kMuma: return launch_sys_tn<kMuma>(L, a, block, s);
    case kPotts: return launch_potts_tn(L, potts_tn_depth(L, a.B, block), a, block, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace muca
