// sweep_pc.cu -- producer/consumer form of the spin sweep (Ising, MUMA, Potts).
#include "muca_device.cuh"
#include "muca_internal.h"
#include "muca_checks.cuh"
#include "sweep_common.cuh"

namespace muca {

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

template <int SYS, int L, int RECORD>
__device__ __forceinline__ void ising_sweep_pc(uint32_t *__restrict__ lat, int ps, int &bR,
                                               uint32_t *__restrict__ sTH, const uint4 *__restrict__ ring,
                                               unsigned long long *full, unsigned long long *empty, int &k,
                                               bool &bad, unsigned long long *obs, unsigned &nacc)
{
    int pc = 0;  // -1 spins of the final rows (observables)
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
        if (bad) {  // a wait gave up: the ring is out of step, so nothing more is computed
            mbar_arrive(&empty[slot]);
            ++k;
            continue;
        }
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
        uint32_t T0 = sTH[checked_word(bR + c0)], T1 = 0u;
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
                T0 = sTH[checked_word(bR + n0)];
                T1 = sTH[checked_word(bR + dR + n1c)];
                d0 = e0;
                d1 = e1;
            }
            const bool acc = (T == kAlways) || (uw < T);
            if (acc) cur[x >> 5] ^= 1u << (x & 31);
            if (RECORD == 0) atomicAdd(&sTH[checked_word((acc ? bR + dR : bR) + C)], 1u);
            accP = acc;
            dRp = dR;
        }
        bR = accP ? bR + dRp : bR;
#pragma unroll
        for (int j = 0; j < WR; ++j) {
            lat[(y * WR + j) * ps] = cur[j];
            pc += __popc(cur[j]);
            nacc += __popc(old[j] ^ cur[j]);
        }
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
    if (RECORD == 1) atomicAdd(&sTH[checked_word(bR + C)], 1u);
    if (SYS == kIsing && obs && !bad) record_observables(obs, bR / RS, L * L, pc);
}

// Consumer side of one Potts sweep (two words a site: proposal, acceptance).
template <int L, int RECORD>
__device__ __forceinline__ void potts_sweep_pc(uint32_t *__restrict__ lat, int ps, int &bR,
                                               uint32_t *__restrict__ sTH, const uint4 *__restrict__ ring,
                                               unsigned long long *full, unsigned long long *empty, int &k,
                                               bool &bad, uint32_t q, unsigned &nacc)
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
        if (bad) {  // a wait gave up: the ring is out of step, so nothing more is computed
            mbar_arrive(&empty[slot]);
            ++k;
            continue;
        }
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
        uint32_t T0 = sTH[checked_word(bR + c0)], T1 = 0u;
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
                T0 = sTH[checked_word(bR + n0)];
                T1 = sTH[checked_word(bR + dR + n1c)];
                d0 = e0;
                d1 = e1;
            }
            const bool acc = (T == kAlways) || (u_acc < T);
            if (acc) {
                const int wi = (4 * x) >> 5, sh = (4 * x) & 31;
                cur[wi] = (cur[wi] & ~(15u << sh)) | (nw << sh);
            }
            if (RECORD == 0) atomicAdd(&sTH[checked_word((acc ? bR + dR : bR) + 9)], 1u);
            accP = acc;
            dRp = dR;
        }
        bR = accP ? bR + dRp : bR;
#pragma unroll
        for (int j = 0; j < WR; ++j) {
            lat[(y * WR + j) * ps] = cur[j];
            nacc += changed_nibbles(old[j], cur[j]);
        }
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
    if (RECORD == 1) atomicAdd(&sTH[checked_word(bR + 9)], 1u);
}

// Producer side: the Philox blocks of one sweep, row by row, for the walkers of
// the paired consumer warp.  G blocks a row: L/4 (one word a site) or L/2 (two).
template <int SYS, int L>
__device__ __forceinline__ void produce_sweep(uint32_t g, uint32_t wid, const uint32_t (&rk)[20], uint4 *ring,
                                              unsigned long long *full, unsigned long long *empty, int &k, bool &bad,
                                              int drop_k)
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
        if (k != drop_k) mbar_arrive(&full[slot]);
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
    const int drop_k = (blockIdx.x == 0 && producer && pair == 0) ? a.debug_drop_row : -1;
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
    int tst = (!producer && active && a.tun) ? a.tun[w] : 0;
    unsigned ev = 0;
    unsigned long long nacc = 0;
    // Inactive lanes (w >= p) run the same rows on walker 0's lattice copy in
    // registers only: they read but never store, so every lane arrives on every
    // barrier phase.
    for (int64_t s0 = 0; s0 < a.sweeps; s0 += a.flush_every) {
        const int64_t s1 = (a.sweeps < s0 + a.flush_every) ? a.sweeps : s0 + a.flush_every;
#pragma unroll 1
        for (int64_t sw = s0; sw < s1; ++sw) {
            const uint32_t g = g0 + (uint32_t)sw;
            if (producer) {
                produce_sweep<SYS, L>(g, wid, a.rk, ring, full, empty, k, bad, drop_k);
            } else if (active) {
                unsigned na = 0;
                if (a.record == 0) {
                    if (SYS == kPotts)
                        potts_sweep_pc<L, 0>(lat, a.pstride, bR, sTH, ring, full, empty, k, bad, (uint32_t)a.q, na);
                    else
                        ising_sweep_pc<SYS, L, 0>(lat, a.pstride, bR, sTH, ring, full, empty, k, bad, a.obs, na);
                } else {
                    if (SYS == kPotts)
                        potts_sweep_pc<L, 1>(lat, a.pstride, bR, sTH, ring, full, empty, k, bad, (uint32_t)a.q, na);
                    else
                        ising_sweep_pc<SYS, L, 1>(lat, a.pstride, bR, sTH, ring, full, empty, k, bad, a.obs, na);
                }
                nacc += na;
                tunnel_step(bR, r_lo, r_hi, tst, ev);
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
    if (!producer && active) {
        a.bin[w] = bR / RS;
        if (a.tun) a.tun[w] = (uint8_t)tst;
    }
    flush_metrics(a.metrics, nacc, ev);
    checks_end(a.state);
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

bool spin_sweep_pc_fits(int system, int L, int B, int walkers_per_block)
{
    return walkers_per_block % 32 == 0 && 2 * walkers_per_block <= kMaxSweepBlock &&
           spin_sweep_pc_smem_bytes(system, L, B, walkers_per_block) <= 227u * 1024u;
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

}  // namespace muca
