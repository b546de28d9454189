// update.cu -- everything between two sweeps of the parallel multicanonical
// loop (paper, Fig. 1: "the histograms are merged, the new weights are
// estimated and distributed to all processes again"):
//   k_merge       integer sum of the per-block histograms (exact, so the
//                 result does not depend on how walkers are grouped);
//   k_recursion   accumulated-statistics weight recursion in log form
//                 ("use the full statistics of previous iterations ...
//                 implemented with logarithmic weights"), plus the flatness
//                 statistics of the merged histogram;
//   k_thresholds  the integer acceptance table T[b][c] = floor(2^32 exp(d)),
//                 d = ln W(target) - ln W(b) (- beta dE for the multimagnetic
//                 ensemble, Eq. 3), or "always" for d >= 0;
//   k_reweight    Eq. (2): canonical averages from the merged histogram.
// All binary64 arithmetic of the recursion and the thresholds uses explicit
// round-to-nearest intrinsics (this file is also built with -fmad=false), so
// the results are the same bits on every run and every compiler.
#include <cfloat>

#include "muca_device.cuh"
#include "muca_internal.h"

namespace muca {

#define kNegInf (__longlong_as_double((long long)0xfff0000000000000ULL))

__device__ __forceinline__ void merge_body(const UpdateArgs &a, int b)
{
    if (b >= a.B) return;
    unsigned long long s = 0ull;
    for (int k = 0; k < a.nblocks; ++k) {
        unsigned long long *p = a.Hpart + (size_t)k * a.B + b;
        s += *p;
        *p = 0ull;
    }
    a.H[b] = s;
}

__global__ void k_merge(const UpdateArgs a) { merge_body(a, blockIdx.x * blockDim.x + threadIdx.x); }

__global__ void k_merge_batch(const UpdateArgs *__restrict__ arr)
{
    merge_body(arr[blockIdx.y], blockIdx.x * blockDim.x + threadIdx.x);
}

// Recursion over the ordered reachable bins r_0 < ... < r_{K-1}.  For each
// neighbouring pair with h0 = H(r_k) > 0 and h1 = H(r_{k+1}) > 0:
//   g = h0 h1 / (h0 + h1);  G_k += g;  kappa = g / G_k;
//   lnR_k += kappa (ln h0 - ln h1),
// then ln W(r_0) = 0 and ln W(r_{k+1}) = ln W(r_k) + lnR_k, summed in order by
// one thread.  Pairs are independent, so the first part runs on all threads.
__device__ __forceinline__ void recursion_body(const UpdateArgs &a, double *sm)
{
    double *slog = sm;
    double *slnR = sm + a.nreach;
    __shared__ unsigned long long s_min, s_max, s_sum;
    const int tid = threadIdx.x, bs = blockDim.x;
    if (tid == 0) {
        s_min = ~0ull;
        s_max = 0ull;
        s_sum = 0ull;
    }
    for (int b = tid; b < a.B; b += bs) a.lnW_sampled[b] = a.lnW[b];
    __syncthreads();  // lnW_sampled is the source of the plain update below
    unsigned long long mn = ~0ull, mx = 0ull, sum = 0ull;
    for (int k = tid; k < a.nreach; k += bs) {
        const unsigned long long h = a.H[a.rlist[k]];
        slog[k] = h ? dm_log(__ull2double_rn(h)) : 0.0;
        mn = h < mn ? h : mn;
        mx = h > mx ? h : mx;
        sum += h;
    }
    __syncthreads();
    atomicMin(&s_min, mn);
    atomicMax(&s_max, mx);
    atomicAdd(&s_sum, sum);
    if (a.recursion == 1) {
        // the plain rule W(n+1) = W(n)/H(n) in log form: x_k = ln W(r_k) - ln max(H(r_k), 1),
        // ln W(r_k) = x_k - x_0 (an unvisited bin keeps its weight)
        const double x0 = __dsub_rn(a.lnW_sampled[a.rlist[0]], slog[0]);
        for (int k = tid; k < a.nreach; k += bs)
            a.lnW[a.rlist[k]] = __dsub_rn(__dsub_rn(a.lnW_sampled[a.rlist[k]], slog[k]), x0);
        __syncthreads();
        if (tid == 0) {
            const double mean = __ddiv_rn(__ull2double_rn(s_sum), (double)a.nreach);
            a.state->flat_min = __ull2double_rn(s_min);
            a.state->flat_mean = mean;
            a.state->flat_max = __ull2double_rn(s_max);
            a.state->flat = (s_min > 0ull) && (__ddiv_rn(__ull2double_rn(s_min), mean) >= a.flat_ratio);
            a.state->iteration += 1ull;
        }
        return;
    }
    for (int k = tid; k + 1 < a.nreach; k += bs) {
        const unsigned long long h0 = a.H[a.rlist[k]], h1 = a.H[a.rlist[k + 1]];
        double r = a.lnR[k];
        if (h0 != 0ull && h1 != 0ull) {
            const double x0 = __ull2double_rn(h0), x1 = __ull2double_rn(h1);
            const double g = __ddiv_rn(__dmul_rn(x0, x1), __dadd_rn(x0, x1));
            const double G = __dadd_rn(a.G[k], g);
            a.G[k] = G;
            const double kappa = __ddiv_rn(g, G);
            r = __dadd_rn(r, __dmul_rn(kappa, __dsub_rn(slog[k], slog[k + 1])));
            a.lnR[k] = r;
        }
        slnR[k] = r;
    }
    __syncthreads();
    if (tid == 0) {
        double acc = 0.0;
        a.lnW[a.rlist[0]] = acc;
        for (int k = 0; k + 1 < a.nreach; ++k) {
            acc = __dadd_rn(acc, slnR[k]);
            a.lnW[a.rlist[k + 1]] = acc;
        }
        const double mean = __ddiv_rn(__ull2double_rn(s_sum), (double)a.nreach);
        a.state->flat_min = __ull2double_rn(s_min);
        a.state->flat_mean = mean;
        a.state->flat_max = __ull2double_rn(s_max);
        a.state->flat = (s_min > 0ull) && (__ddiv_rn(__ull2double_rn(s_min), mean) >= a.flat_ratio);
        a.state->iteration += 1ull;
    }
}

// The iteration's metrics become the "last" ones (and are added to the totals);
// the open counters restart.  Runs once per update, after the sweeps' atomics.
__device__ __forceinline__ void close_metrics(const UpdateArgs &a)
{
    unsigned long long *m = a.metrics;
    if (!m || threadIdx.x != 0) return;
    m[2] = m[0];
    m[3] = m[1];
    m[4] += m[0];
    m[5] += m[1];
    const unsigned long long sc = a.state->sweep_counter;
    m[6] = sc - m[7];
    m[7] = sc;
    m[0] = 0ull;
    m[1] = 0ull;
}

__global__ void __launch_bounds__(1024) k_recursion(const UpdateArgs a)
{
    extern __shared__ double sm[];
    recursion_body(a, sm);
    close_metrics(a);
}

__global__ void __launch_bounds__(1024) k_recursion_batch(const UpdateArgs *__restrict__ arr)
{
    extern __shared__ double sm[];
    const UpdateArgs a = arr[blockIdx.y];
    recursion_body(a, sm);
    close_metrics(a);
}

__device__ __forceinline__ void thresholds_body(const UpdateArgs &a, int i)
{
    if (a.system == kPolymer) return;  // its weights go to the fixed-point table instead (k_poly_lnwq)
    const int C = num_cols(a.system);
    if (i >= a.B * C) return;
    const int b = i / C, c = i - (i / C) * C;
    int b2, dE = 0;
    if (a.system == kIsing) {
        b2 = b + c - 2;
    } else if (a.system == kPotts) {
        dE = c - 4;
        b2 = b + dE;
    } else {
        const int sidx = c / 5, k = c - 5 * (c / 5);
        dE = 4 * (k - 2);
        b2 = b - 1 + 2 * sidx;
    }
    uint32_t t = 0u;
    if (a.reach[b] && b2 >= 0 && b2 < a.B && a.reach[b2]) {
        double d = __dsub_rn(a.lnW[b2], a.lnW[b]);
        if (a.system == kMuma) d = __dsub_rn(d, __dmul_rn(a.beta, (double)dE));
        if (d >= 0.0) {
            t = kAlways;
        } else {
            const double scaled = __dmul_rn(dm_exp(d), 4294967296.0);
            t = (scaled >= 4294967296.0) ? kAlways : (uint32_t)floor(scaled);
        }
    }
    a.T[i] = t;
}

__global__ void k_thresholds(const UpdateArgs a) { thresholds_body(a, blockIdx.x * blockDim.x + threadIdx.x); }

__global__ void k_thresholds_batch(const UpdateArgs *__restrict__ arr)
{
    thresholds_body(arr[blockIdx.y], blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_advance(DevState *st, long long sweeps) { st->sweep_counter += (unsigned long long)sweeps; }

__global__ void k_advance_batch(DevState *const *states, const SpinSweepArgs *sys, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) states[i]->sweep_counter += (unsigned long long)sys[i].sweeps;  // each system's own count
}

__global__ void k_init_weights(const UpdateArgs a)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.B) return;
    const double v = a.reach[b] ? 0.0 : kNegInf;  // unreachable bins never carry weight
    a.lnW[b] = v;
    a.lnW_sampled[b] = v;
    a.G[b] = 0.0;
    a.lnR[b] = 0.0;
    a.H[b] = 0ull;
}

// Initial lattices from the INIT stream: word i%4 of Philox((i/4, 0, walker, 0)).
// Ising/MUMA: s = -1 (bit 1) iff the word's top bit is set; Potts: s = mulhi(u, q).
__global__ void k_init_spins(int system, int L, int q, int p, int pstride, uint32_t k0, uint32_t k1,
                             int walker_offset, uint32_t *lat, int32_t *bin)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= p) return;
    const uint32_t wid = (uint32_t)(w + walker_offset);
    const int WR = (system == kPotts) ? potts_words_per_row(L) : ising_words_per_row(L);
    const int bits = (system == kPotts) ? 4 : 1;
    uint32_t *my = lat + w;
    uint4 u = make_uint4(0u, 0u, 0u, 0u);
    for (int y = 0; y < L; ++y) {
        for (int j = 0; j < WR; ++j) {
            uint32_t word = 0u;
            for (int x = j * 32 / bits; x < (j + 1) * 32 / bits && x < L; ++x) {
                const int i = y * L + x;
                if ((i & 3) == 0) u = philox4x32_10(make_uint4((uint32_t)(i / 4), 0u, wid, kTagInit), k0, k1);
                const uint32_t r = (i & 3) == 0 ? u.x : ((i & 3) == 1 ? u.y : ((i & 3) == 2 ? u.z : u.w));
                const uint32_t v = (system == kPotts) ? __umulhi(r, (uint32_t)q) : (r >> 31);
                word |= v << ((x * bits) & 31);
            }
            my[(y * WR + j) * pstride] = word;
        }
    }
    // bin of the initial state, from scratch
    int E = 0, nminus = 0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            const int yd = (y + 1) % L, xr = (x + 1) % L;
            if (system == kPotts) {
                auto nib = [&](int yy, int xx) {
                    return (my[(yy * WR + (4 * xx) / 32) * pstride] >> ((4 * xx) & 31)) & 15u;
                };
                const uint32_t s = nib(y, x);
                E -= (int)(s == nib(y, xr)) + (int)(s == nib(yd, x));
            } else {
                auto bt = [&](int yy, int xx) { return (my[(yy * WR + xx / 32) * pstride] >> (xx & 31)) & 1u; };
                const int s = bt(y, x) ? -1 : 1, sr = bt(y, xr) ? -1 : 1, sd = bt(yd, x) ? -1 : 1;
                E -= s * sr + s * sd;
                nminus += (s < 0);
            }
        }
    const int N = L * L;
    if (system == kIsing) bin[w] = (E + 2 * N) / 4;
    else if (system == kPotts) bin[w] = E + 2 * N;
    else bin[w] = N - nminus;  // (M + N)/2 = number of +1 spins
}

__global__ void k_unpack_spins(int system, int L, int p, int pstride, const uint32_t *lat, int8_t *out)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long N = (long long)L * L;
    if (idx >= (long long)p * N) return;
    const int w = (int)(idx / N), i = (int)(idx - (idx / N) * N);
    const int y = i / L, x = i - (i / L) * L;
    if (system == kPotts) {
        const int WR = potts_words_per_row(L);
        const uint32_t word = lat[(size_t)(y * WR + (4 * x) / 32) * pstride + w];
        out[idx] = (int8_t)((word >> ((4 * x) & 31)) & 15u);
    } else {
        const int WR = ising_words_per_row(L);
        const uint32_t word = lat[(size_t)(y * WR + x / 32) * pstride + w];
        out[idx] = ((word >> (x & 31)) & 1u) ? (int8_t)-1 : (int8_t)1;
    }
}

// Eq. (2) with O a function of the binned variable; ln Omega(b) = ln H(b) -
// ln W(b), W being the weights H was sampled with.  Fixed-order tree
// reductions in one block, so repeated calls give identical results.
__global__ void __launch_bounds__(1024) k_reweight(const UpdateArgs a, double beta, double *out4, double *lnP)
{
    extern __shared__ double sx[];  // B values of x_b
    __shared__ double red[1024];
    const int tid = threadIdx.x, bs = blockDim.x, B = a.B, N = a.N;
    const double NEG_INF = kNegInf;
    double m = NEG_INF;
    for (int b = tid; b < B; b += bs) {
        double x = NEG_INF;
        const unsigned long long h = a.H[b];
        if (a.reach[b] && h) {
            const double lnOmega = log((double)h) - a.lnW_sampled[b];
            if (a.system == kMuma) {
                x = lnOmega;
            } else if (a.system == kPolymer) {
                x = lnOmega - beta * (a.e_lo + a.bin_w * (b + 0.5));
            } else {
                const double E = (a.system == kIsing) ? (double)(4 * b - 2 * N) : (double)(b - 2 * N);
                x = lnOmega - beta * E;
            }
        }
        sx[b] = x;
        m = fmax(m, x);
    }
    red[tid] = m;
    __syncthreads();
    for (int s = bs / 2; s > 0; s >>= 1) {
        if (tid < s) red[tid] = fmax(red[tid], red[tid + s]);
        __syncthreads();
    }
    m = red[0];
    __syncthreads();
    double z = 0.0;
    for (int b = tid; b < B; b += bs)
        if (sx[b] > NEG_INF) z += exp(sx[b] - m);
    red[tid] = z;
    __syncthreads();
    for (int s = bs / 2; s > 0; s >>= 1) {
        if (tid < s) red[tid] += red[tid + s];
        __syncthreads();
    }
    const double lse = m + log(red[0]);
    __syncthreads();
    double a1 = 0.0, a2 = 0.0;
    for (int b = tid; b < B; b += bs) {
        const double x = sx[b];
        const double lp = (x > NEG_INF) ? x - lse : NEG_INF;
        if (lnP) lnP[b] = lp;
        if (x > NEG_INF) {
            const double P = exp(lp);
            double v;
            if (a.system == kMuma) v = fabs((double)(2 * b - N));
            else if (a.system == kPolymer) v = a.e_lo + a.bin_w * (b + 0.5);
            else v = (a.system == kIsing) ? (double)(4 * b - 2 * N) : (double)(b - 2 * N);
            a1 += P * v;
            a2 += P * v * v;
        }
    }
    __shared__ double red2[1024];
    red[tid] = a1;
    red2[tid] = a2;
    __syncthreads();
    for (int s = bs / 2; s > 0; s >>= 1) {
        if (tid < s) {
            red[tid] += red[tid + s];
            red2[tid] += red2[tid + s];
        }
        __syncthreads();
    }
    a1 = red[0];
    a2 = red2[0];
    // polymer: log-sum-exp of ln Omega itself (the normalisation of ln Z)
    double lnNorm = 0.0;
    if (a.system == kPolymer) {
        __syncthreads();
        double m2 = NEG_INF;
        for (int b = tid; b < B; b += bs)
            if (sx[b] > NEG_INF) m2 = fmax(m2, sx[b] + beta * (a.e_lo + a.bin_w * (b + 0.5)));
        red2[tid] = m2;
        __syncthreads();
        for (int st = bs / 2; st > 0; st >>= 1) {
            if (tid < st) red2[tid] = fmax(red2[tid], red2[tid + st]);
            __syncthreads();
        }
        m2 = red2[0];
        __syncthreads();
        double z2 = 0.0;
        for (int b = tid; b < B; b += bs)
            if (sx[b] > NEG_INF) z2 += exp(sx[b] + beta * (a.e_lo + a.bin_w * (b + 0.5)) - m2);
        red2[tid] = z2;
        __syncthreads();
        for (int st = bs / 2; st > 0; st >>= 1) {
            if (tid < st) red2[tid] += red2[tid + st];
            __syncthreads();
        }
        lnNorm = m2 + log(red2[0]);
    }
    if (tid == 0) {
        if (a.system == kPolymer) {
            out4[0] = a1;
            out4[1] = a2;
            out4[2] = beta * beta * (a2 - a1 * a1) / N;
            out4[3] = lse - lnNorm;
        } else if (a.system == kMuma) {
            out4[0] = a1 / N;
            out4[1] = a2 / ((double)N * N);
            out4[2] = a.beta * N * (out4[1] - out4[0] * out4[0]);
            const int b0 = N / 2, bm = N;
            out4[3] = (sx[b0] > NEG_INF && sx[bm] > NEG_INF) ? sx[b0] - sx[bm] : __longlong_as_double(0x7ff8000000000000LL);
        } else {
            out4[0] = a1;
            out4[1] = a2;
            out4[2] = beta * beta * (a2 - a1 * a1) / N;
            const double g0 = (a.system == kIsing) ? 2.0 : (double)a.q;
            if (sx[0] > NEG_INF) out4[3] = lse + log(g0) - (sx[0] - beta * (double)(2 * N));
            else out4[3] = __longlong_as_double(0x7ff8000000000000LL);
        }
    }
}

__global__ void k_det_math(int fn, const double *in, double *out, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = fn == 0 ? dm_exp(in[i]) : dm_log(in[i]);
}

// ---------------------------------------------------------------------------
cudaError_t launch_det_math(int fn, const double *in, double *out, long long n, cudaStream_t s)
{
    k_det_math<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(fn, in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_merge(const UpdateArgs &a, cudaStream_t s)
{
    k_merge<<<(a.B + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_recursion(const UpdateArgs &a, cudaStream_t s)
{
    const size_t smem = (size_t)2 * a.nreach * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_recursion, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_recursion<<<1, 1024, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_thresholds(const UpdateArgs &a, cudaStream_t s)
{
    const int n = a.B * num_cols(a.system);
    k_thresholds<<<(n + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_merge_batch(const UpdateArgs *d_args, int n, int max_bins, cudaStream_t s)
{
    k_merge_batch<<<dim3((max_bins + 255) / 256, n), 256, 0, s>>>(d_args);
    return cudaGetLastError();
}

cudaError_t launch_recursion_batch(const UpdateArgs *d_args, int n, int max_nreach, cudaStream_t s)
{
    const size_t smem = (size_t)2 * max_nreach * sizeof(double);
    k_recursion_batch<<<dim3(1, n), 1024, smem, s>>>(d_args);
    return cudaGetLastError();
}

cudaError_t prepare_recursion_batch(int max_nreach)
{
    return cudaFuncSetAttribute(k_recursion_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)((size_t)2 * max_nreach * sizeof(double)));
}

cudaError_t launch_thresholds_batch(const UpdateArgs *d_args, int n, int max_cells, cudaStream_t s)
{
    k_thresholds_batch<<<dim3((max_cells + 255) / 256, n), 256, 0, s>>>(d_args);
    return cudaGetLastError();
}

cudaError_t launch_advance_batch(DevState *const *d_states, const SpinSweepArgs *d_sys, int n, cudaStream_t s)
{
    k_advance_batch<<<(n + 127) / 128, 128, 0, s>>>(d_states, d_sys, n);
    return cudaGetLastError();
}

cudaError_t launch_advance(DevState *st, int64_t sweeps, cudaStream_t s)
{
    k_advance<<<1, 1, 0, s>>>(st, (long long)sweeps);
    return cudaGetLastError();
}

cudaError_t launch_init_lnW(const UpdateArgs &a, cudaStream_t s)
{
    k_init_weights<<<(a.B + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_init_spins(int system, int L, int q, int p, int pstride, uint32_t key0, uint32_t key1,
                              int walker_offset, uint32_t *lattice, int32_t *bin, cudaStream_t s)
{
    k_init_spins<<<(p + 127) / 128, 128, 0, s>>>(system, L, q, p, pstride, key0, key1, walker_offset, lattice, bin);
    return cudaGetLastError();
}

cudaError_t launch_unpack_spins(int system, int L, int p, int pstride, const uint32_t *lattice, int8_t *out,
                                cudaStream_t s)
{
    const long long n = (long long)p * L * L;
    k_unpack_spins<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(system, L, p, pstride, lattice, out);
    return cudaGetLastError();
}

cudaError_t launch_reweight(const UpdateArgs &a, double beta, double *out4, double *lnP, cudaStream_t s)
{
    const size_t smem = (size_t)a.B * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_reweight, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_reweight<<<1, 1024, smem, s>>>(a, beta, out4, lnP);
    return cudaGetLastError();
}

// Eq. (2) with per-bin sums of an Ising run (samples n, sum |M|, sum M^2 per bin):
// <O>_beta = sum_b S_O(b) e^{x_b} / sum_b n(b) e^{x_b}, x_b = -beta E_b - ln W(b),
// E_b = 4b - 2N, W the weights the sums were sampled with.  One block; out =
// {<|M|>/N, <M^2>/N^2, beta N (<M^2>/N^2 - (<|M|>/N)^2)}, NaN without samples.
__global__ void __launch_bounds__(256) k_reweight_obs(const unsigned long long *__restrict__ sums,
                                                      const double *__restrict__ lnW, int B, int N, double beta,
                                                      double *out)
{
    __shared__ double red[4][256];
    const int t = threadIdx.x;
    double m = -INFINITY;
    for (int b = t; b < B; b += 256)
        if (sums[3 * b] > 0ull) m = fmax(m, -beta * (double)(4 * b - 2 * N) - lnW[b]);
    red[0][t] = m;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (t < o) red[0][t] = fmax(red[0][t], red[0][t + o]);
        __syncthreads();
    }
    const double mx = red[0][0];
    __syncthreads();
    double z = 0.0, a1 = 0.0, a2 = 0.0;
    if (mx > -INFINITY) {
        for (int b = t; b < B; b += 256) {
            if (sums[3 * b] == 0ull) continue;
            const double f = exp(-beta * (double)(4 * b - 2 * N) - lnW[b] - mx);
            z += f * (double)sums[3 * b];
            a1 += f * (double)sums[3 * b + 1];
            a2 += f * (double)sums[3 * b + 2];
        }
    }
    red[1][t] = z;
    red[2][t] = a1;
    red[3][t] = a2;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (t < o) {
            red[1][t] += red[1][t + o];
            red[2][t] += red[2][t + o];
            red[3][t] += red[3][t + o];
        }
        __syncthreads();
    }
    if (t == 0) {
        if (!(mx > -INFINITY)) {
            out[0] = out[1] = out[2] = NAN;
        } else {
            const double m1 = red[2][0] / red[1][0] / N, m2 = red[3][0] / red[1][0] / ((double)N * N);
            out[0] = m1;
            out[1] = m2;
            out[2] = beta * N * (m2 - m1 * m1);
        }
    }
}

cudaError_t launch_reweight_obs(const unsigned long long *sums, const double *lnW_sampled, int B, int N, double beta,
                                double *out3, cudaStream_t s)
{
    k_reweight_obs<<<1, 256, 0, s>>>(sums, lnW_sampled, B, N, beta, out3);
    return cudaGetLastError();
}

}  // namespace muca
