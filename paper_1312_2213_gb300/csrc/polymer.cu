// polymer.cu -- multicanonical sweeps of a single flexible bead-spring polymer
// (paper: polymer paragraph and Eq. 7; the benchmark's parameters: FENE bonds
// K = 40, R = 1.5, Lennard-Jones 12-6 between beads |i-j| >= 2 with eps = sigma
// = 1, cut at 2.5 and shifted; single-bead moves in a cube of side 0.3).
//
// G lanes of a warp per walker (G = 1, 2, 4, 8, 16 or 32; 32/G walkers share a
// warp).
// The beads are visited in order; for bead i every lane of the walker's group
// evaluates the old and the new pair energies with its partner beads
// j = lane, lane + G, ... in FP32 and keeps a compensated (Kahan) sum (the old
// bond energies come from a per-walker cache, updated on acceptance); the lane
// sums are added in FP32 over the group and the total is converted once to 64-bit
// fixed point (2^-32 energy units).  Nothing on the hot path uses FP64, whose
// rate on GB300 is a small fraction of FP32.
//
// Exactness: master coordinates are int64 on a 2^-44 grid and a move adds
// (u - 2^31) * 1229 grid units per axis (a cube of side 1229/4096 = 0.30005), so
// the coordinates of an accepted move are exact and identical to any other
// implementation that draws the same words.  The FP32 pair terms use shadows
// relative to the walker's bead 0 at the start of each sweep, kept as unevaluated
// float pairs (hi + lo): a difference (hi_i - hi_j) + (lo_i - lo_j) keeps the
// separation of two beads to ~1e-7 of itself however far the chain extends, so
// the rounding of FP32 energy changes stays unbiased when walk-in selects moves
// by the sign of their energy change.  The running
// energy is an exact sum of the fixed-point energy changes; it is refreshed from
// scratch after every iterate call, and the largest difference is recorded.
// Acceptance inside the window: d = ln W(b') - ln W(b) from a fixed-point table,
// accept iff d >= 0 or ln(u 2^-32) < d (the FP32 logarithm of each bead's
// acceptance word is taken once a sweep); outside the window a move is accepted
// iff it does not increase the distance to the window (walk-in).  Visits are
// counted in the block's 32-bit shared-memory counters, which the block's last
// warp to finish adds to the 64-bit histogram (an iterate longer than they can
// hold runs as several launches), so that walkers crowding one bin (right after
// they walk in, say) do not queue on one global counter.
#include "muca_device.cuh"
#include "muca_internal.h"

namespace muca {

bool polymer_supported(int N) { return N >= 2 && N <= kPolyMaxN; }

// (sigma/r)^2 from the hardware's approximate reciprocal (PTX rcp.approx.ftz.f32, at most one
// ulp off: the r^-12 term then carries a few ulp, a few 1e-8 of the pair's error scale
// |v| + |r v'|, which is 48 (sigma/r)^12 and more).  A correctly rounded reciprocal took a
// quarter of the sweep's time at N = 128.
__device__ __forceinline__ float lj_energy(float r2, const PolyArgs &a)
{
    float rr;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rr) : "f"(r2));
    const float ir2 = rr * a.lj_sigma2;  // sigma = 1 in model 0
    const float ir6 = ir2 * ir2 * ir2;
    const float v = 4.0f * (ir6 * ir6 - ir6) - a.lj_shift;
    return r2 < a.lj_rc2 ? v : 0.0f;
}

__device__ __forceinline__ float fene_energy(float r2, const PolyArgs &a)
{
    if (a.model == 1) {  // rest length r0: -(K/2) R^2 ln(1 - ((r - r0)/R)^2)
        const float x = (__fsqrt_rn(r2) - a.fene_r0) * a.fene_invR;
        return -a.fene_KR2_half * log1pf(-x * x);
    }
    return -a.fene_KR2_half * log1pf(-r2 * a.fene_invR2);
}

// A bond of squared length r2 is intact: r < R (model 0), |r - r0| < R (model 1).
__device__ __forceinline__ bool fene_intact(float r2, const PolyArgs &a)
{
    if (a.model == 1) return fabsf((__fsqrt_rn(r2) - a.fene_r0) * a.fene_invR) < 1.0f;
    return r2 < 1.0f / a.fene_invR2;
}

// Offset on the 2^-44 grid as an unevaluated pair hi + lo of floats.
__device__ __forceinline__ void grid_to_ff(long long d, float &hi, float &lo)
{
    hi = (float)d;
    lo = (float)(d - (long long)hi);
    hi *= 0x1p-44f;
    lo *= 0x1p-44f;
}

__device__ __forceinline__ long long warp_sum_ll(long long q)
{
#pragma unroll
    for (int off = 16; off; off >>= 1) q += __shfl_xor_sync(0xffffffffu, q, off);
    return q;
}

// llrint(t) for |t| < 2^62 without a 64-bit conversion instruction (those run on
// the FP64 pipe, a small fraction of FP32 on GB300): below 2^31 a 32-bit rounding
// conversion; above, t is an integer m * 2^e with e >= 8, rebuilt from its bits.
__device__ __forceinline__ long long f2ll_exact(float t)
{
    const uint32_t b = __float_as_uint(t);
    const int e = (int)((b >> 23) & 0xffu) - 150;
    const long long m = (long long)((b & 0x7fffffu) | 0x800000u);
    const long long big = (e >= 0 ? (m << (e & 63)) : 0);
    return fabsf(t) < 2147483648.0f ? (long long)__float2int_rn(t) : ((b >> 31) ? -big : big);
}

// A 2^-32 fixed-point value as a float, from its two 32-bit halves (32-bit
// conversions only).
__device__ __forceinline__ float q32_to_float(long long v)
{
    return (float)(int)(v >> 32) + (float)(uint32_t)v * 0x1p-32f;
}

__device__ __forceinline__ int poly_bin(long long E, const PolyArgs &a)
{
    const long long b = ((E - a.elo_q) * a.bin_k) >> 32;
    return b < -1 ? -1 : (b > (long long)a.B ? a.B : (int)b);
}

// n visits of a bin: a shared-memory reduction without a returned value, so nothing
// waits for it.
__device__ __forceinline__ void count_visits(unsigned *h, unsigned n)
{
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(h)), "r"(n) : "memory");
}

// Random-walk initial chain (thread per walker): bead k = bead k-1 + unit vector
// from Marsaglia's method on tag-2 Philox words, rounded to the grid, redrawn (up
// to 64 times) while an earlier bead is closer than 0.9.  Binary64 with explicit
// round-to-nearest operations (run once).
__global__ void k_poly_init(const PolyArgs a)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= a.p) return;
    const int N = a.N;
    const uint32_t wid = (uint32_t)(w + a.walker_offset);
    long long *X = a.X + (size_t)w * 3 * N;
    X[0] = X[N] = X[2 * N] = 0;
    uint32_t draw = 0;
    for (int k = 1; k < N; ++k) {
        long long cand[3] = {0, 0, 0};
        for (int attempt = 0; attempt < 64; ++attempt) {
            double v1 = 0.0, v2 = 0.0, s = 0.5;
            for (int tries = 0; tries < 4096; ++tries) {
                const uint4 u = philox4x32_10(make_uint4(draw++, 0u, wid, kTagPolyInit), a.key0, a.key1);
                v1 = __dsub_rn(__dmul_rn((double)u.x, 0x1p-31), 1.0);
                v2 = __dsub_rn(__dmul_rn((double)u.y, 0x1p-31), 1.0);
                s = __dadd_rn(__dmul_rn(v1, v1), __dmul_rn(v2, v2));
                if (s < 1.0 && s > 0.0) break;
            }
            const double f = __dmul_rn(2.0, __dsqrt_rn(__dsub_rn(1.0, s)));
            const double uh[3] = {__dmul_rn(v1, f), __dmul_rn(v2, f), __dsub_rn(1.0, __dmul_rn(2.0, s))};
            for (int c = 0; c < 3; ++c)
                cand[c] = X[c * N + k - 1] + (long long)rint(__dmul_rn(__dmul_rn(uh[c], a.init_bond), 0x1p44));
            bool ok = true;
            for (int j = 0; j < k - 1 && ok; ++j) {
                const double dx = __dmul_rn((double)(cand[0] - X[j]), 0x1p-44);
                const double dy = __dmul_rn((double)(cand[1] - X[N + j]), 0x1p-44);
                const double dz = __dmul_rn((double)(cand[2] - X[2 * N + j]), 0x1p-44);
                const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                if (d2 < a.init_d2min) ok = false;
            }
            if (ok) break;
        }
        for (int c = 0; c < 3; ++c) X[c * N + k] = cand[c];
    }
}

// Energy from scratch, one warp per walker (FP32 pairs relative to bead 0,
// Kahan per lane, exact fixed-point warp sum).  With track != 0 the largest
// change against the running energy is recorded in state->drift_max_q.
__global__ void k_poly_energy(const PolyArgs a, int track)
{
    extern __shared__ __align__(16) float sh[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, N = a.N;
    const int w = blockIdx.x * (blockDim.x >> 5) + wib;
    if (w >= a.p) return;
    float *xs = sh + (size_t)wib * 6 * N;  // hi[3N], lo[3N]
    float *xl = xs + 3 * N;
    const long long *X = a.X + (size_t)w * 3 * N;
    const long long A0 = X[0], A1 = X[N], A2 = X[2 * N];
    for (int j = lane; j < N; j += 32) {
        grid_to_ff(X[j] - A0, xs[j], xl[j]);
        grid_to_ff(X[N + j] - A1, xs[N + j], xl[N + j]);
        grid_to_ff(X[2 * N + j] - A2, xs[2 * N + j], xl[2 * N + j]);
    }
    __syncwarp();
    float s = 0.0f, c = 0.0f;
    for (int i = 0; i < N; ++i) {
        const float xi = xs[i], yi = xs[N + i], zi = xs[2 * N + i];
        const float li = xl[i], mi = xl[N + i], ni = xl[2 * N + i];
        for (int j = lane; j < N; j += 32) {
            if (j <= i) continue;
            const float dx = (xi - xs[j]) + (li - xl[j]), dy = (yi - xs[N + j]) + (mi - xl[N + j]),
                        dz = (zi - xs[2 * N + j]) + (ni - xl[2 * N + j]);
            const float r2 = dx * dx + dy * dy + dz * dz;
            const float v = (j - i == 1) ? fene_energy(r2, a) : lj_energy(r2, a);
            const float y = v - c;
            const float t = s + y;
            c = (t - s) - y;
            s = t;
        }
    }
    long long q = __float2ll_rn(s * 0x1p32f) - __float2ll_rn(c * 0x1p32f);
    q = warp_sum_ll(q);
    if (lane == 0) {
        if (track) {
            const long long d = q - a.E[w];
            atomicMax(&a.state->drift_max_q, (unsigned long long)(d < 0 ? -d : d));
        }
        a.E[w] = q;
        a.bin[w] = poly_bin(q, a);
    }
}

template <int G>
__device__ __forceinline__ bool group_any(bool p, int gi)
{
    const unsigned bal = __ballot_sync(0xffffffffu, p);
    return G == 32 ? bal != 0u : ((bal >> (gi * G)) & ((1u << (G & 31)) - 1u)) != 0u;
}

// Spherical rotation of bead i (move set 1): the pivot is a bonded neighbour,
// the new position pivot + d n with d = |r_i - r_pivot| and n a unit vector from
// Marsaglia's method on (m.z, m.w) and then on tag-4 blocks (64 i + t), two pairs
// a block, at most 64 pairs.  Every step is a correctly rounded binary64
// operation on exact grid values, so the new grid position is bit-identical to
// any implementation that follows the same steps.  Returns false when no point
// was found (the move is then rejected).
__device__ bool poly_rotation(const long long *Xg, int N, int i, uint32_t g, uint32_t wid, const uint4 m,
                              const uint32_t (&rk)[20], long long out[3])
{
    const int pv = (i == 0) ? 1 : (i == N - 1) ? N - 2 : ((m.y & 1u) ? i + 1 : i - 1);
    double v1 = 0.0, v2 = 0.0, s = 0.0;
    bool found = false;
    uint4 blk = make_uint4(0u, 0u, m.z, m.w);
    for (int t = 0; t < 64 && !found; ++t) {
        if (t & 1) blk = philox4x32_10_rk(make_uint4((uint32_t)(64 * i + (t >> 1)), g, wid, kTagPolySphere), rk);
        const uint32_t aw = (t == 0) ? m.z : ((t & 1) ? blk.x : blk.z);
        const uint32_t bw = (t == 0) ? m.w : ((t & 1) ? blk.y : blk.w);
        v1 = __dsub_rn(__dmul_rn((double)aw, 0x1p-31), 1.0);
        v2 = __dsub_rn(__dmul_rn((double)bw, 0x1p-31), 1.0);
        s = __dadd_rn(__dmul_rn(v1, v1), __dmul_rn(v2, v2));
        found = s < 1.0 && s > 0.0;
    }
    if (!found) return false;
    const double f = __dmul_rn(2.0, __dsqrt_rn(__dsub_rn(1.0, s)));
    const double n[3] = {__dmul_rn(v1, f), __dmul_rn(v2, f), __dsub_rn(1.0, __dmul_rn(2.0, s))};
    double dd[3];
    long long P[3];
    for (int c = 0; c < 3; ++c) {
        P[c] = Xg[c * N + pv];
        dd[c] = __dmul_rn((double)(Xg[c * N + i] - P[c]), 0x1p-44);
    }
    const double d = __dsqrt_rn(
        __dadd_rn(__dadd_rn(__dmul_rn(dd[0], dd[0]), __dmul_rn(dd[1], dd[1])), __dmul_rn(dd[2], dd[2])));
    for (int c = 0; c < 3; ++c) out[c] = P[c] + (long long)rint(__dmul_rn(__dmul_rn(n[c], d), 0x1p44));
    return true;
}

// Shared-memory floats of one walker's slot: the float-pair shadows (6 N) and the
// energies of its N - 1 bonds, rounded up to a multiple of 4 so that the uint4
// Philox blocks behind all slots start 16-byte aligned for any walker count and
// odd N.  (Padding the slots so that the walkers of a warp read disjoint banks was
// measured on GB300 with the 6 N layout: within 1 % at N = 64 and 128, 2-5 %
// slower at N = 32 and 13, so it is not done.)
template <int G>
__host__ __device__ inline int poly_slot_floats(int N)
{
    return (7 * N + 3) & ~3;  // hi[3N], lo[3N], bond energies[N]; a multiple of 4 floats
}

// Sweeps: G lanes per walker, 32/G walkers a warp, all on the same bead i.  A
// walker's float-pair shadows and this sweep's Philox blocks live in shared
// memory (40 N bytes, 56 N with rotations); its int64 master coordinates stay in
// global memory (read at the sweep start and for the moved bead, written on
// acceptance).  The two
// bonds of bead i (FENE) are taken by lanes 0 and 1 of the group, the other
// partners (LJ, |i - j| >= 2) by lanes j mod G, so no lane runs both branches.
template <int G, int RECORD>
__global__ void __launch_bounds__(kMaxSweepBlock) k_sweep_polymer(const PolyArgs a)
{
    constexpr int W = 32 / G;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5, N = a.N;
    const int gi = lane / G, li = lane % G;
    const int spb = wpb * W, slot = wib * W + gi, sst = poly_slot_floats<G>(N);
    float *xs = (float *)smem + (size_t)slot * sst;
    float *xl = xs + 3 * N;
    float *eb = xs + 6 * N;  // eb[j]: FP32 energy of bond (j, j+1) at the current shadows
    uint4 *su = (uint4 *)(smem + (size_t)spb * sst * sizeof(float)) + (size_t)slot * N;
    uint4 *sm = su + (size_t)spb * N;  // moves
    // the block's histogram counters and its count of finished warps, after all slots and
    // Philox blocks
    unsigned *hs = (unsigned *)(smem + (size_t)spb * sst * sizeof(float) +
                                (size_t)spb * N * (a.moves ? 2 : 1) * sizeof(uint4));
    unsigned *done = hs + a.B;
    for (int i = threadIdx.x; i <= a.B; i += blockDim.x) hs[i] = 0u;
    __syncthreads();
    const int w0 = (blockIdx.x * wpb + wib) * W;
    if (w0 >= a.p) return;  // whole warps only; no block-wide barrier follows
    const int w = w0 + gi;
    const bool active = w < a.p;
    const int wr = active ? w : w0;  // a group past the last walker shadows the warp's first one, read-only
    const uint32_t wid = (uint32_t)(wr + a.walker_offset);
    long long *Xg = a.X + (size_t)wr * 3 * N;
    long long E = a.E[wr];
    int b = poly_bin(E, a);
    const uint32_t g0 = (uint32_t)(a.state->sweep_counter + a.sweep_base);
    const int npl = (N + G - 1) / G;
    // metrics: accepted moves and tunnelling between bins 0 and B-1 (group-uniform values)
    unsigned long long nacc = 0;
    unsigned ev = 0;
    int tst = (active && a.tun) ? a.tun[w] : 0;
    const float kStep = (float)a.step_q * 0x1p-44f;
    for (int64_t sw = 0; sw < a.sweeps; ++sw) {
        const uint32_t g = g0 + (uint32_t)sw;
        const long long A0 = Xg[0], A1 = Xg[N], A2 = Xg[2 * N];
        for (int j = li; j < N; j += G) {
            grid_to_ff(Xg[j] - A0, xs[j], xl[j]);
            grid_to_ff(Xg[N + j] - A1, xs[N + j], xl[N + j]);
            grid_to_ff(Xg[2 * N + j] - A2, xs[2 * N + j], xl[2 * N + j]);
            uint4 r = philox4x32_10_rk(make_uint4((uint32_t)j, g, wid, kTagSweep), a.rk);
            // the acceptance test u 2^-32 < exp(d) is taken as ln(u 2^-32) < d: the logarithm
            // (FP32, -inf for u = 0) is taken here, once a bead and sweep, off the serial path
            r.w = __float_as_uint(logf((float)r.w * 0x1p-32f));
            su[j] = r;
            if (a.moves) sm[j] = philox4x32_10_rk(make_uint4((uint32_t)j, g, wid, kTagPolyMove), a.rk);
        }
        __syncwarp();
        for (int j = li; j + 1 < N; j += G) {
            const float dx = (xs[j] - xs[j + 1]) + (xl[j] - xl[j + 1]);
            const float dy = (xs[N + j] - xs[N + j + 1]) + (xl[N + j] - xl[N + j + 1]);
            const float dz = (xs[2 * N + j] - xs[2 * N + j + 1]) + (xl[2 * N + j] - xl[2 * N + j + 1]);
            eb[j] = fene_energy(dx * dx + dy * dy + dz * dz, a);
        }
        __syncwarp();
#pragma unroll 1
        for (int i = 0; i < N; ++i) {
            const uint4 u = su[i];
            // move (u - 2^31) * 1229 grid units per axis: exact on the int64 master
            // coordinates; the float-pair shadow moves by the same amount in FP32
            // (the shadows are rebuilt exactly from the masters every sweep)
            const int sx = (int)(u.x ^ 0x80000000u), sy = (int)(u.y ^ 0x80000000u), sz = (int)(u.z ^ 0x80000000u);
            const long long X0 = Xg[i], X1 = Xg[N + i], X2 = Xg[2 * N + i];
            const float xo = xs[i], yo = xs[N + i], zo = xs[2 * N + i];
            const float lxo = xl[i], lyo = xl[N + i], lzo = xl[2 * N + i];
            const float dx = (float)sx * kStep, dy = (float)sy * kStep, dz = (float)sz * kStep;
            float xn = xo + dx, yn = yo + dy, zn = zo + dz;
            float lxn = lxo + ((xo - xn) + dx), lyn = lyo + ((yo - yn) + dy), lzn = lzo + ((zo - zn) + dz);
            // (32 x 32-bit products: the grid step fits an int)
            long long n0 = X0 + (long long)sx * (long long)a.step_q, n1 = X1 + (long long)sy * (long long)a.step_q,
                      n2 = X2 + (long long)sz * (long long)a.step_q;
            float s = 0.0f, c = 0.0f;
            bool broken = false;
            if (a.moves) {
                const uint4 mv = sm[i];
                if (mv.x >= 0x80000000u) {  // spherical rotation about a bonded neighbour
                    long long nr[3];
                    if (poly_rotation(Xg, N, i, g, wid, mv, a.rk, nr)) {
                        n0 = nr[0];
                        n1 = nr[1];
                        n2 = nr[2];
                        grid_to_ff(n0 - A0, xn, lxn);
                        grid_to_ff(n1 - A1, yn, lyn);
                        grid_to_ff(n2 - A2, zn, lzn);
                    } else {
                        broken = true;  // no point in 64 pairs: rejected
                    }
                }
            }
            // the bonds (i-1, i) and (i, i+1): lanes 0 and 1 of the group, or the walker's only lane
            // for both when G = 1; the old energies come from the bond cache, the new ones are
            // kept to update it if the move is accepted
            float vnb[2] = {0.0f, 0.0f};
#pragma unroll
            for (int t = 0; t < (G == 1 ? 2 : 1); ++t) {
                const int jb = (G == 1 ? t == 0 : li == 0) ? i - 1 : i + 1;
                if ((G == 1 || li < 2) && jb >= 0 && jb < N) {
                    const float xj = xs[jb], yj = xs[N + jb], zj = xs[2 * N + jb];
                    const float ljx = xl[jb], ljy = xl[N + jb], ljz = xl[2 * N + jb];
                    const float bx = (xn - xj) + (lxn - ljx), by = (yn - yj) + (lyn - ljy), bz = (zn - zj) + (lzn - ljz);
                    const float r2n = bx * bx + by * by + bz * bz;
                    const bool brk = !fene_intact(r2n, a);
                    broken = broken || brk;
                    const float vo = eb[jb < i ? jb : i];
                    const float vn = brk ? vo : fene_energy(r2n, a);
                    vnb[t] = vn;
                    const float y = (vn - vo) - c;  // compensated, as the pair terms below
                    const float tt = s + y;
                    c = (tt - s) - y;
                    s = tt;
                }
            }
#pragma unroll 2
            for (int k = 0; k < npl; ++k) {
                const int j = li + G * k, dj = j - i;
                if (j < N && (dj > 1 || dj < -1)) {
                    const float xj = xs[j], yj = xs[N + j], zj = xs[2 * N + j];
                    const float ljx = xl[j], ljy = xl[N + j], ljz = xl[2 * N + j];
                    const float ax = (xo - xj) + (lxo - ljx), ay = (yo - yj) + (lyo - ljy), az = (zo - zj) + (lzo - ljz);
                    const float bx = (xn - xj) + (lxn - ljx), by = (yn - yj) + (lyn - ljy), bz = (zn - zj) + (lzn - ljz);
                    const float r2o = ax * ax + ay * ay + az * az;
                    const float r2n = bx * bx + by * by + bz * bz;
                    const float y = (lj_energy(r2n, a) - lj_energy(r2o, a)) - c;
                    const float t = s + y;
                    c = (t - s) - y;
                    s = t;
                }
            }
            broken = group_any<G>(broken, gi);
            // |lane sum| >= 2^22 only for overlapping beads: such a move is rejected
            const bool huge = group_any<G>(!(fabsf(s) < 4194304.0f), gi);
            // the lanes' compensated sums added in FP32 by a butterfly: every lane adds the same
            // two operands at every step (a + b = b + a exactly), so all lanes of the group end
            // with the same sum, converted once to 2^-32 fixed point
            float lane_sum = s - c;
#pragma unroll
            for (int off = G / 2; off; off >>= 1) lane_sum += __shfl_xor_sync(0xffffffffu, lane_sum, off);
            const long long q = huge ? 0 : f2ll_exact(lane_sum * 0x1p32f);
            const long long En = E + q;
            const int bn = poly_bin(En, a);
            bool acc = false;
            if (!broken && !huge) {
                if (b >= 0 && b < a.B) {
                    if (bn >= 0 && bn < a.B) {
                        const long long dq = __ldg(a.lnWq + bn) - __ldg(a.lnWq + b);
                        // accept iff d >= 0 or ln(u 2^-32) < d (the logarithm is in u.w)
                        acc = dq >= 0 || __uint_as_float(u.w) < q32_to_float(dq);
                    }
                } else {
                    const long long dold = (b < 0) ? a.elo_q - E : E - a.ehi_q;
                    const long long dnew = (bn < 0) ? a.elo_q - En : (bn >= a.B ? En - a.ehi_q : 0);
                    acc = dnew <= dold;
                }
            }
            if (a.trace && li == 0 && active) {  // parity inspection only
                PolyTraceRec r;
                r.dq = q;
                r.E = acc ? En : E;
                r.bn = bn;
                r.b = acc ? bn : b;
                r.flags = (acc ? 1 : 0) | (broken ? 2 : 0) | (huge ? 4 : 0);
                r.pad = 0;
                a.trace[((size_t)w * (size_t)a.trace_sweeps + (size_t)(a.sweep_base + sw)) * (size_t)N + i] = r;
            }
            if (acc) {
                if (G == 1) {
                    if (i > 0) eb[i - 1] = vnb[0];
                    if (i + 1 < N) eb[i] = vnb[1];
                } else if (li < 2) {
                    const int jb = li == 0 ? i - 1 : i + 1;
                    if (jb >= 0 && jb < N) eb[jb < i ? jb : i] = vnb[0];
                }
                if (li == 0) {
                    if (active) {
                        Xg[i] = n0;
                        Xg[N + i] = n1;
                        Xg[2 * N + i] = n2;
                    }
                    xs[i] = xn;
                    xs[N + i] = yn;
                    xs[2 * N + i] = zn;
                    xl[i] = lxn;
                    xl[N + i] = lyn;
                    xl[2 * N + i] = lzn;
                }
                E = En;
                b = bn;
                ++nacc;
            }
            __syncwarp();
            if (RECORD == 0 && li == 0 && active && b >= 0 && b < a.B) count_visits(&hs[b], 1u);
        }
        if (RECORD == 1 && li == 0 && active && b >= 0 && b < a.B) count_visits(&hs[b], 1u);
        tunnel_step(b, 0, a.B - 1, tst, ev);
        __syncwarp();
    }
    // the block's last warp to finish adds the counters to the histogram (the launch's sweeps
    // fit the 32-bit counters: launch_g splits longer iterates)
    __threadfence_block();  // this warp's visits are counted before it reports
    __syncwarp();
    const int nwarps = min(wpb, (a.p - blockIdx.x * spb + W - 1) / W);  // warps of the block with walkers
    unsigned last = 0u;
    if (lane == 0) last = (atomicAdd(done, 1u) == (unsigned)nwarps - 1u);
    if (__shfl_sync(0xffffffffu, last, 0)) {
        __threadfence_block();
        for (int i = lane; i < a.B; i += 32) {
            const unsigned c = hs[i];
            if (c) atomicAdd(a.H + i, (unsigned long long)c);
        }
    }
    const bool lead = li == 0 && active;
    flush_metrics(a.metrics, lead ? nacc : 0ull, lead ? ev : 0u);
    if (lead && a.tun) a.tun[w] = (uint8_t)tst;
    if (!active) return;  // (no warp-wide operation follows)
    // recentre on bead 0 (an exact grid shift) and write back
    const long long A0 = Xg[0], A1 = Xg[N], A2 = Xg[2 * N];
    __syncwarp(__activemask());
    for (int t = li; t < N; t += G) {
        Xg[t] -= A0;
        Xg[N + t] -= A1;
        Xg[2 * N + t] -= A2;
    }
    if (li == 0) {
        a.E[w] = E;
        a.bin[w] = b;
    }
}

__global__ void k_poly_lnwq(const double *lnW, long long *lnWq, int B)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) lnWq[b] = __double2ll_rn(__dmul_rn(lnW[b], 0x1p32));
}

__global__ void k_poly_unpack(const PolyArgs a, double *coords, double *energies)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)a.p * a.N;
    if (t >= n) return;
    const int w = (int)(t / a.N), j = (int)(t - (t / a.N) * a.N);
    const long long *X = a.X + (size_t)w * 3 * a.N;
    for (int c = 0; c < 3; ++c) coords[t * 3 + c] = (double)X[c * a.N + j] * 0x1p-44;
    if (j == 0) energies[w] = (double)a.E[w] * 0x1p-32;
}

cudaError_t launch_poly_init(const PolyArgs &a, cudaStream_t s)
{
    k_poly_init<<<(a.p + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_poly_energy(const PolyArgs &a, int track_drift, cudaStream_t s)
{
    const int wpb = 4;
    const size_t smem = (size_t)wpb * 6 * a.N * sizeof(float);
    k_poly_energy<<<(a.p + wpb - 1) / wpb, wpb * 32, smem, s>>>(a, track_drift);
    return cudaGetLastError();
}

// Shared memory of one warp of the sweep: 32/G walkers' float-pair shadows and Philox blocks.
template <int G>
static size_t poly_warp_smem(const PolyArgs &a)
{
    return (size_t)(32 / G) * ((size_t)poly_slot_floats<G>(a.N) * sizeof(float) +
                               (size_t)a.N * (a.moves ? 2 : 1) * sizeof(uint4));
}

constexpr size_t kPolySmemMax = 227u * 1024u;

// The block's 32-bit histogram counters (one per bin), after the warps' shared memory.
static size_t poly_hist_smem(const PolyArgs &a)
{
    return ((size_t)(a.B + 1) * sizeof(unsigned) + 15) / 16 * 16;
}

template <int G>
static cudaError_t launch_g(const PolyArgs &a, int block, cudaStream_t s)
{
    // as many warps of the requested block as fit the shared memory of one block
    int wpb = block / 32;
    const size_t per_warp = poly_warp_smem<G>(a), hist = poly_hist_smem(a);
    if (hist + (size_t)wpb * per_warp > kPolySmemMax)
        wpb = hist < kPolySmemMax ? (int)((kPolySmemMax - hist) / per_warp) : 0;
    if (wpb < 1) return cudaErrorInvalidValue;
    block = 32 * wpb;
    const int spb = wpb * (32 / G);
    const size_t smem = (size_t)wpb * per_warp + hist;
    const int nblk = (a.p + spb - 1) / spb;
    cudaError_t e = (a.record == 0)
                        ? cudaFuncSetAttribute(k_sweep_polymer<G, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                        : cudaFuncSetAttribute(k_sweep_polymer<G, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // one launch per chunk of sweeps whose visits fit the block's 32-bit counters (spb N a sweep
    // at most), or fewer ("flush_every")
    int64_t fe = (int64_t)(0xFFFFFFFFu / (unsigned)(spb * a.N));
    if (a.flush_every > 0 && a.flush_every < fe) fe = a.flush_every;
    for (int64_t s0 = 0; s0 < a.sweeps; s0 += fe) {
        PolyArgs c = a;
        c.sweep_base = s0;
        c.sweeps = (a.sweeps - s0 < fe) ? a.sweeps - s0 : fe;
        c.trace_sweeps = a.sweeps;
        if (a.record == 0)
            k_sweep_polymer<G, 0><<<nblk, block, smem, s>>>(c);
        else
            k_sweep_polymer<G, 1><<<nblk, block, smem, s>>>(c);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Lanes per walker: the fixed cost of an attempt (group reductions, the bin and
// weight lookups, the decision) is shared by the 32/G walkers of a warp, the pair
// terms are spread over G lanes.  A request for a grouping whose warp does not fit
// the shared memory of a block falls back to the next larger G.  Measured on GB300
// with 4096 walkers (pilot windows), 16 lanes is the fastest at N = 13, 32, 64 and
// 128: fewer lanes share the fixed cost among more walkers but leave 4096 G / 32
// warps to hide latency (G = 4: 2.1e9 against 3.0e9 attempts/s at N = 13; G = 1:
// 1.1e9), so 16 stays the default.
template <int G>
static bool poly_fits(const PolyArgs &a)
{
    return poly_warp_smem<G>(a) + poly_hist_smem(a) <= kPolySmemMax;
}

int poly_lanes(const PolyArgs &a, int requested)
{
    int g = (requested == 1 || requested == 2 || requested == 4 || requested == 8 || requested == 16 ||
             requested == 32) ? requested : 16;
    if (g == 1 && !poly_fits<1>(a)) g = 2;
    if (g == 2 && !poly_fits<2>(a)) g = 4;
    return g;
}

cudaError_t launch_poly_sweep(const PolyArgs &a, int block, cudaStream_t s)
{
    if (!polymer_supported(a.N)) return cudaErrorInvalidValue;
    switch (poly_lanes(a, a.lanes)) {
    case 1: return launch_g<1>(a, block, s);
    case 2: return launch_g<2>(a, block, s);
    case 4: return launch_g<4>(a, block, s);
    case 8: return launch_g<8>(a, block, s);
    case 16: return launch_g<16>(a, block, s);
    default: return launch_g<32>(a, block, s);
    }
}

cudaError_t launch_poly_lnwq(const double *lnW, long long *lnWq, int B, cudaStream_t s)
{
    k_poly_lnwq<<<(B + 255) / 256, 256, 0, s>>>(lnW, lnWq, B);
    return cudaGetLastError();
}

cudaError_t launch_poly_unpack(const PolyArgs &a, double *coords, double *energies, cudaStream_t s)
{
    const long long n = (long long)a.p * a.N;
    k_poly_unpack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, coords, energies);
    return cudaGetLastError();
}

}  // namespace muca
