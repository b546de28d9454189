// sweep_common.cuh -- pieces shared by the three forms of the spin sweep
// (one warp per walker group, producer/consumer, producer/consumer with site
// codes): packed-row accessors, the bounded mbarrier hand-over and the
// lattice sizes that have compiled kernels.
#pragma once
#include "muca_device.cuh"
#include "muca_internal.h"

namespace muca {

// Lattice sizes with compiled sweep kernels.
__host__ __device__ constexpr bool sweep_L_supported(int L)
{
    return L == 4 || L == 8 || L == 12 || L == 16 || L == 24 || L == 32 || L == 48 || L == 64;
}

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

// Ring depth (rows) of the producer/consumer forms and the bound on every
// mbarrier wait: a wait that gives up sets the error flag instead of spinning on.
constexpr int kRing = 4;
// 2^17 tries of mbarrier.try_wait (each suspends the warp for a few microseconds
// when the phase is not complete: ~1 s in all on GB300); a healthy hand-over takes
// microseconds.
constexpr int kSpinLimit = 1 << 17;

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

// The block's bound on one wait, in tries: kSpinLimit unless the launch sets its own
// (SpinSweepArgs::spin_limit, from the context's "spin_limit" parameter or the
// MUCA_SPIN_LIMIT environment variable).  Thread 0 sets it before the block's first
// barrier.
__device__ __forceinline__ int &block_spin_limit()
{
    __shared__ int s_limit;
    return s_limit;
}

__device__ __forceinline__ void set_block_spin_limit(int limit)
{
    if (threadIdx.x == 0) block_spin_limit() = limit > 0 ? limit : kSpinLimit;
}

// Bounded wait; returns false (and leaves the barrier alone) after the block's limit.
// The limit is read only when the first try fails, off the hand-over's fast path.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity)
{
    if (mbar_try(bar, parity)) return true;
    const int lim = block_spin_limit();
    for (int i = 1; i < lim; ++i)
        if (mbar_try(bar, parity)) return true;
    return false;
}

// Consumer side of one Ising / MUMA sweep: as ising_sweep, with the random words
// of row y read from ring slot (k % kRing).

// Observables of an Ising walker after a sweep: one sample, |M| and M^2 added to
// the sums of its bin; pc = number of -1 spins (set bits) of its lattice.
__device__ __forceinline__ void record_observables(unsigned long long *obs, int bin, int N, int pc)
{
    const long long M = (long long)N - 2LL * pc;
    unsigned long long *o = obs + 3 * (size_t)bin;
    atomicAdd(o, 1ull);
    atomicAdd(o + 1, (unsigned long long)(M < 0 ? -M : M));
    atomicAdd(o + 2, (unsigned long long)(M * M));
}

}  // namespace muca
