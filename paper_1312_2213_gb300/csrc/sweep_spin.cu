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
// Lattice rows live in HBM/L2 walker-interleaved (coalesced) and are streamed
// through registers: each thread keeps the row above, the current row and
// the row below, and prefetches the next one while it works on this one.
#include "muca_device.cuh"
#include "muca_internal.h"

namespace muca {

template <int WR>
__device__ __forceinline__ uint32_t bit_at(const uint32_t (&r)[WR], int pos)
{
    return (r[pos >> 5] >> (pos & 31)) & 1u;
}

template <int WR>
__device__ __forceinline__ uint32_t nib_at(const uint32_t (&r)[WR], int x)
{
    return (r[(4 * x) >> 5] >> ((4 * x) & 31)) & 15u;
}

// One sweep of an Ising (MUCA in E) or multimagnetic (weight in M) walker.
// Spin bit 1 means s = -1.  k = 4 - (number of anti-aligned neighbours), so
// dE = 4(k-2); Ising column c = k, bin move k-2; MUMA column c = 5*bit + k,
// bin (M+N)/2 moves by 2*bit-1.
template <int SYS, int L>
__device__ __forceinline__ void ising_sweep(uint32_t *__restrict__ lat, int ps, int &b,
                                            const uint32_t *__restrict__ sT, uint32_t *__restrict__ sH,
                                            uint32_t g, uint32_t wid, uint32_t k0, uint32_t k1, int record)
{
    constexpr int WR = ising_words_per_row(L);
    constexpr int C = (SYS == kMuma) ? 10 : 5;
    uint32_t up[WR], cur[WR], dn[WR], first[WR], nxt[WR];
#pragma unroll
    for (int j = 0; j < WR; ++j) {
        up[j] = lat[((L - 1) * WR + j) * ps];
        cur[j] = lat[j * ps];
        dn[j] = lat[(WR + j) * ps];
        first[j] = 0u;
        nxt[j] = 0u;
    }
    int bC = b * C;
#pragma unroll 1
    for (int y = 0; y < L; ++y) {
        if (y + 2 < L) {
#pragma unroll
            for (int j = 0; j < WR; ++j) nxt[j] = lat[((y + 2) * WR + j) * ps];
        }
#pragma unroll
        for (int gq = 0; gq < L / 4; ++gq) {
            const uint4 u = philox4x32_10(make_uint4((uint32_t)(y * (L / 4) + gq), g, wid, kTagSweep), k0, k1);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int x = 4 * gq + j;
                const uint32_t uw = j == 0 ? u.x : (j == 1 ? u.y : (j == 2 ? u.z : u.w));
                const uint32_t s = bit_at<WR>(cur, x);
                const int n1 = (int)(bit_at<WR>(cur, (x + L - 1) % L) + bit_at<WR>(cur, (x + 1) % L) +
                                     bit_at<WR>(up, x) + bit_at<WR>(dn, x));
                const int k = s ? n1 : 4 - n1;
                int col, db;
                if (SYS == kMuma) {
                    col = 5 * (int)s + k;
                    db = 2 * (int)s - 1;
                } else {
                    col = k;
                    db = k - 2;
                }
                const uint32_t t = sT[bC + col];
                if (t == kAlways || uw < t) {
                    cur[x >> 5] ^= 1u << (x & 31);
                    b += db;
                    bC += db * C;
                }
                if (record == 0) atomicAdd(&sH[b], 1u);
            }
        }
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
    if (record == 1) atomicAdd(&sH[b], 1u);
}

// One sweep of a q-state Potts walker (4-bit spins).  Proposal: a uniform new
// state different from the old one, new = (old + 1 + mulhi(u, q-1)) mod q.
// dE = n_eq(old) - n_eq(new) in [-4, 4]; column dE+4; bin E+2N moves by dE.
template <int L>
__device__ __forceinline__ void potts_sweep(uint32_t *__restrict__ lat, int ps, int &b,
                                            const uint32_t *__restrict__ sT, uint32_t *__restrict__ sH,
                                            uint32_t g, uint32_t wid, uint32_t k0, uint32_t k1, int record,
                                            uint32_t q)
{
    constexpr int WR = potts_words_per_row(L);
    uint32_t up[WR], cur[WR], dn[WR], first[WR], nxt[WR];
#pragma unroll
    for (int j = 0; j < WR; ++j) {
        up[j] = lat[((L - 1) * WR + j) * ps];
        cur[j] = lat[j * ps];
        dn[j] = lat[(WR + j) * ps];
        first[j] = 0u;
        nxt[j] = 0u;
    }
    const uint32_t qm1 = q - 1u;
    int b9 = b * 9;
#pragma unroll 1
    for (int y = 0; y < L; ++y) {
        if (y + 2 < L) {
#pragma unroll
            for (int j = 0; j < WR; ++j) nxt[j] = lat[((y + 2) * WR + j) * ps];
        }
#pragma unroll
        for (int gp = 0; gp < L / 2; ++gp) {
            const uint4 u = philox4x32_10(make_uint4((uint32_t)(y * (L / 2) + gp), g, wid, kTagSweep), k0, k1);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int x = 2 * gp + j;
                const uint32_t u_prop = j ? u.z : u.x;
                const uint32_t u_acc = j ? u.w : u.y;
                const uint32_t old = nib_at<WR>(cur, x);
                const uint32_t nl = nib_at<WR>(cur, (x + L - 1) % L), nr = nib_at<WR>(cur, (x + 1) % L);
                const uint32_t nu = nib_at<WR>(up, x), nd = nib_at<WR>(dn, x);
                uint32_t nw = old + 1u + __umulhi(u_prop, qm1);
                nw = (nw >= q) ? nw - q : nw;
                const int eo = (int)(nl == old) + (int)(nr == old) + (int)(nu == old) + (int)(nd == old);
                const int en = (int)(nl == nw) + (int)(nr == nw) + (int)(nu == nw) + (int)(nd == nw);
                const int dE = eo - en;
                const uint32_t t = sT[b9 + dE + 4];
                if (t == kAlways || u_acc < t) {
                    const int wi = (4 * x) >> 5, sh = (4 * x) & 31;
                    cur[wi] = (cur[wi] & ~(15u << sh)) | (nw << sh);
                    b += dE;
                    b9 += 9 * dE;
                }
                if (record == 0) atomicAdd(&sH[b], 1u);
            }
        }
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
    if (record == 1) atomicAdd(&sH[b], 1u);
}

// The sweep kernel: stage the threshold table in shared memory, run the
// walkers, flush the block histogram to its own uint64 slot every
// `flush_every` sweeps (so no uint32 bin can overflow) and at the end.
template <int SYS, int L>
__global__ void __launch_bounds__(kMaxSweepBlock) k_sweep_spin(const SpinSweepArgs a)
{
    constexpr int C = num_cols(SYS);
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *sT = smem;
    uint32_t *sH = smem + (size_t)a.B * C;
    const int tid = threadIdx.x;
    for (int i = tid; i < a.B * C; i += blockDim.x) sT[i] = a.T[i];
    for (int i = tid; i < a.B; i += blockDim.x) sH[i] = 0u;
    __syncthreads();

    const int w = blockIdx.x * blockDim.x + tid;
    const bool active = w < a.p;
    const uint32_t wid = (uint32_t)(w + a.walker_offset);
    const uint32_t g0 = (uint32_t)a.state->sweep_counter;
    uint32_t *lat = a.lattice + (active ? w : 0);
    int b = active ? a.bin[w] : 0;
    unsigned long long *Hb = a.Hpart + (size_t)blockIdx.x * a.B;

    for (int64_t s0 = 0; s0 < a.sweeps; s0 += a.flush_every) {
        const int64_t s1 = (a.sweeps < s0 + a.flush_every) ? a.sweeps : s0 + a.flush_every;
        if (active) {
#pragma unroll 1
            for (int64_t sw = s0; sw < s1; ++sw) {
                const uint32_t g = g0 + (uint32_t)sw;
                if (SYS == kPotts)
                    potts_sweep<L>(lat, a.pstride, b, sT, sH, g, wid, a.key0, a.key1, a.record, (uint32_t)a.q);
                else
                    ising_sweep<SYS, L>(lat, a.pstride, b, sT, sH, g, wid, a.key0, a.key1, a.record);
            }
        }
        __syncthreads();
        for (int i = tid; i < a.B; i += blockDim.x) {
            const uint32_t c = sH[i];
            if (c) {
                Hb[i] += c;
                sH[i] = 0u;
            }
        }
        __syncthreads();
    }
    if (active) a.bin[w] = b;
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
    switch (system) {
    case kIsing: return launch_sys<kIsing>(L, a, block, s);
    case kMuma: return launch_sys<kMuma>(L, a, block, s);
    case kPotts: return launch_sys<kPotts>(L, a, block, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace muca
