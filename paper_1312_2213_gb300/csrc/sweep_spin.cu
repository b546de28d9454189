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
#include "muca_checks.cuh"
#include "sweep_common.cuh"

namespace muca {

template <int SYS, int L, int RECORD>
__device__ __forceinline__ void ising_sweep(uint32_t *__restrict__ lat, int ps, int &bR,
                                            uint32_t *__restrict__ sTH, uint32_t g, uint32_t wid,
                                            const uint32_t (&rk)[20], unsigned long long *obs, unsigned &nacc)
{
    int pc = 0;  // -1 spins of the final rows (observables)
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
        uint32_t T0 = sTH[checked_word(bR + c0)], T1 = 0u;
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
    if (SYS == kIsing && obs) record_observables(obs, bR / RS, L * L, pc);
}

// One sweep of a q-state Potts walker (4-bit spins).  Proposal: a uniform new
// state different from the old one, new = (old + 1 + mulhi(u, q-1)) mod q.
// dE = n_eq(old) - n_eq(new) in [-4, 4]; column dE+4; bin E+2N moves by dE.
// The "left neighbour changed" candidate uses the left site's proposed colour.
// GT (a table too large for shared memory: q-Potts at L = 64, 8193 x 9 words):
// the thresholds are read from the global [B][9] table gT (L2-resident), sTH holds
// only the B histogram counters and bR is the bin itself.
template <int L, int RECORD, bool GT = false>
__device__ __forceinline__ void potts_sweep(uint32_t *__restrict__ lat, int ps, int &bR,
                                            uint32_t *__restrict__ sTH, uint32_t g, uint32_t wid,
                                            const uint32_t (&rk)[20], uint32_t q, unsigned &nacc,
                                            const uint32_t *__restrict__ gT = nullptr, int nbins = 0)
{
    constexpr int WR = potts_words_per_row(L);
    constexpr int RS = GT ? 1 : 10;
    auto tload = [&](int row, int c) -> uint32_t {
        return GT ? __ldg(gT + checked_word(row * 9 + c)) : sTH[checked_word(row + c)];
    };
    auto hist = [&](int row) {
        if (GT)
            atomicAdd(&sTH[checked_index(row, nbins)], 1u);
        else
            atomicAdd(&sTH[checked_word(row + 9)], 1u);
    };
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
        uint32_t T0 = tload(bR, c0), T1 = 0u;
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
                T0 = tload(bR, n0);
                T1 = tload(bR + dR, n1c);
                d0 = e0;
                d1 = e1;
            }
            const bool acc = (T == kAlways) || (u_acc < T);
            if (acc) {
                const int wi = (4 * x) >> 5, sh = (4 * x) & 31;
                cur[wi] = (cur[wi] & ~(15u << sh)) | (nw << sh);
            }
            if (RECORD == 0) hist(acc ? bR + dR : bR);
            accP = acc;
            dRp = dR;
        }
        bR = accP ? bR + dRp : bR;
#pragma unroll
        for (int j = 0; j < WR; ++j) {
            lat[(y * WR + j) * ps] = cur[j];
            nacc += changed_nibbles(old[j], cur[j]);
        }
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
    if (RECORD == 1) hist(bR);
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
    checks_begin(a.B * RS, a.debug_check);
    __syncthreads();

    const int w = w0 + tid;
    const bool active = w < a.p;
    const uint32_t wid = (uint32_t)(w + a.walker_offset);
    const uint32_t g0 = (uint32_t)a.state->sweep_counter;
    uint32_t *lat = a.lattice + (active ? w : 0);
    int bR = (active ? a.bin[w] : 0) * RS;
    unsigned long long *Hb = a.Hpart + (size_t)slot * a.B;
    const int r_lo = a.bin_lo * RS, r_hi = a.bin_hi * RS;
    int tst = (active && a.tun) ? a.tun[w] : 0;
    unsigned ev = 0;
    unsigned long long nacc = 0;

    for (int64_t s0 = 0; s0 < a.sweeps; s0 += a.flush_every) {
        const int64_t s1 = (a.sweeps < s0 + a.flush_every) ? a.sweeps : s0 + a.flush_every;
        if (active) {
            if (a.record == 0) {
#pragma unroll 1
                for (int64_t sw = s0; sw < s1; ++sw) {
                    const uint32_t g = g0 + (uint32_t)sw;
                    unsigned na = 0;
                    if (SYS == kPotts)
                        potts_sweep<L, 0>(lat, a.pstride, bR, sTH, g, wid, a.rk, (uint32_t)a.q, na);
                    else
                        ising_sweep<SYS, L, 0>(lat, a.pstride, bR, sTH, g, wid, a.rk, a.obs, na);
                    nacc += na;
                    tunnel_step(bR, r_lo, r_hi, tst, ev);
                }
            } else {
#pragma unroll 1
                for (int64_t sw = s0; sw < s1; ++sw) {
                    const uint32_t g = g0 + (uint32_t)sw;
                    unsigned na = 0;
                    if (SYS == kPotts)
                        potts_sweep<L, 1>(lat, a.pstride, bR, sTH, g, wid, a.rk, (uint32_t)a.q, na);
                    else
                        ising_sweep<SYS, L, 1>(lat, a.pstride, bR, sTH, g, wid, a.rk, a.obs, na);
                    nacc += na;
                    tunnel_step(bR, r_lo, r_hi, tst, ev);
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
    if (active) {
        a.bin[w] = bR / RS;
        if (a.tun) a.tun[w] = (uint8_t)tst;
    }
    flush_metrics(a.metrics, nacc, ev);
    checks_end(a.state);
}

// q-Potts lattices whose threshold table does not fit in shared memory (L = 64: 8193
// bins x 9 columns, 295 KB): one warp per 32 walkers, the thresholds read from the
// global table (it stays in L2), only the B histogram counters in shared memory.
template <int L>
__device__ __forceinline__ void sweep_block_potts_gt(const SpinSweepArgs &a, int w0, int slot, uint32_t *smem)
{
    uint32_t *sH = smem;
    const int tid = threadIdx.x;
    for (int i = tid; i < a.B; i += blockDim.x) sH[i] = 0u;
    checks_begin(a.B * 9, a.debug_check);
    __syncthreads();

    const int w = w0 + tid;
    const bool active = w < a.p;
    const uint32_t wid = (uint32_t)(w + a.walker_offset);
    const uint32_t g0 = (uint32_t)a.state->sweep_counter;
    uint32_t *lat = a.lattice + (active ? w : 0);
    int bin = active ? a.bin[w] : 0;
    unsigned long long *Hb = a.Hpart + (size_t)slot * a.B;
    int tst = (active && a.tun) ? a.tun[w] : 0;
    unsigned ev = 0;
    unsigned long long nacc = 0;

    for (int64_t s0 = 0; s0 < a.sweeps; s0 += a.flush_every) {
        const int64_t s1 = (a.sweeps < s0 + a.flush_every) ? a.sweeps : s0 + a.flush_every;
        if (active) {
#pragma unroll 1
            for (int64_t sw = s0; sw < s1; ++sw) {
                const uint32_t g = g0 + (uint32_t)sw;
                unsigned na = 0;
                if (a.record == 0)
                    potts_sweep<L, 0, true>(lat, a.pstride, bin, sH, g, wid, a.rk, (uint32_t)a.q, na, a.T, a.B);
                else
                    potts_sweep<L, 1, true>(lat, a.pstride, bin, sH, g, wid, a.rk, (uint32_t)a.q, na, a.T, a.B);
                nacc += na;
                tunnel_step(bin, a.bin_lo, a.bin_hi, tst, ev);
            }
        }
        __syncthreads();
        for (int b = tid; b < a.B; b += blockDim.x) {
            const uint32_t c = sH[b];
            if (c) {
                Hb[b] += c;
                sH[b] = 0u;
            }
        }
        __syncthreads();
    }
    if (active) {
        a.bin[w] = bin;
        if (a.tun) a.tun[w] = (uint8_t)tst;
    }
    flush_metrics(a.metrics, nacc, ev);
    checks_end(a.state);
}

template <int L>
__global__ void __launch_bounds__(kMaxSweepBlock) k_sweep_potts_gt(const SpinSweepArgs a)
{
    extern __shared__ __align__(16) uint32_t smem[];
    sweep_block_potts_gt<L>(a, blockIdx.x * blockDim.x, blockIdx.x, smem);
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

// The global-table Potts form (L = 64).
static bool potts_gt(int system, int L) { return system == kPotts && L == 64; }

bool spin_sweep_supported(int system, int L)
{
    if (system != kIsing && system != kPotts && system != kMuma) return false;
    if (!sweep_L_supported(L)) return false;
    if (potts_gt(system, L)) return true;
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


cudaError_t launch_spin_sweep(int system, int L, const SpinSweepArgs &a, int block, cudaStream_t s)
{
    if (!spin_sweep_supported(system, L)) return cudaErrorInvalidValue;
    if (potts_gt(system, L)) {
        const size_t smem = (size_t)a.B * sizeof(uint32_t);
        cudaError_t e = cudaFuncSetAttribute(k_sweep_potts_gt<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_sweep_potts_gt<64><<<(a.p + block - 1) / block, block, smem, s>>>(a);
        return cudaGetLastError();
    }
    switch (system) {
    case kIsing: return launch_sys<kIsing>(L, a, block, s);
    case kMuma: return launch_sys<kMuma>(L, a, block, s);
    case kPotts: return launch_sys<kPotts>(L, a, block, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace muca
