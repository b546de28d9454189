// muca_device.cuh -- device helpers shared by the sm_103a kernels:
//   * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), the counter-based
//     generator every walker draws its random words from;
//   * binary64 exp / log with a fixed operation order (explicit _rn intrinsics,
//     so nothing is contracted into an FMA), used by the weight recursion and
//     the threshold build, whose results must not depend on the compiler.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace muca {

// ---------------------------------------------------------------------------
// Philox4x32-10.  Counter words: (word group, global sweep, walker id, tag).
// The key (seed lo, seed hi) is the same for every thread; the per-round keys
// k + r*W are folded by the compiler into uniform registers.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;
constexpr uint32_t kTagInit = 0u;
constexpr uint32_t kTagSweep = 1u;
constexpr uint32_t kTagPolyInit = 2u;
constexpr uint32_t kTagPolyMove = 3u;    // polymer move set 1: move choice, pivot, first sphere pair
constexpr uint32_t kTagPolySphere = 4u;  // polymer move set 1: further sphere pairs

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
        const uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return c;
}

// Same function as a rolled loop: small code for a rarely taken path.
__device__ __forceinline__ uint4 philox4x32_10_rolled(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll 1
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
        const uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return c;
}

// Same function with the ten round keys precomputed (rk[2r], rk[2r+1] = key of round r);
// when rk lives in the kernel parameters each round reads its key straight from the
// constant bank.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t (&rk)[20])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
        const uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
    }
    return c;
}

// ---------------------------------------------------------------------------
// Deterministic binary64 exp and log.
// exp: Cody-Waite reduction x = k ln2 + r (ln 2 = HI + LO, HI with 32
// significant bits so k*HI is exact), Taylor series of exp(r) through r^13/13!
// in Horner form, then scaling by 2^k.
// log: x = 2^e m, m in [sqrt(1/2), sqrt(2)], s = (m-1)/(m+1),
// ln m = 2 s sum_j s^(2j)/(2j+1) through s^22, ln x = e HI + (e LO + ln m).
// Constants are 1/j! and 1/(2j+1) rounded to nearest and the ln 2 split,
// evaluated once in 300-bit arithmetic and written as hexadecimal literals.
__device__ __forceinline__ double dm_pow2i(int k) // 2^k, -1022 <= k <= 1023
{
    return __longlong_as_double((long long)(k + 1023) << 52);
}

__device__ inline double dm_exp(double x)
{
    const double HI = 0x1.62e42fee00000p-1, LO = 0x1.a39ef35793c76p-33;
    const double INV_LN2 = 0x1.71547652b82fep+0;
    const double C[14] = {0x1.0000000000000p+0,  0x1.0000000000000p+0,  0x1.0000000000000p-1,
                          0x1.5555555555555p-3,  0x1.5555555555555p-5,  0x1.1111111111111p-7,
                          0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13, 0x1.a01a01a01a01ap-16,
                          0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22, 0x1.ae64567f544e4p-26,
                          0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33};
    if (x != x) return x;
    if (x > 709.0) return __longlong_as_double(0x7ff0000000000000LL);
    if (x < -745.0) return 0.0;
    const double kd = floor(__dadd_rn(__dmul_rn(x, INV_LN2), 0.5));
    const int k = (int)kd;
    const double r = __dsub_rn(__dsub_rn(x, __dmul_rn(kd, HI)), __dmul_rn(kd, LO));
    double poly = C[13];
#pragma unroll
    for (int j = 12; j >= 0; --j) poly = __dadd_rn(__dmul_rn(poly, r), C[j]);
    if (k >= -1022) {
        if (k > 1023) return __dmul_rn(__dmul_rn(poly, dm_pow2i(k - 1)), 2.0);
        return __dmul_rn(poly, dm_pow2i(k));
    }
    return __dmul_rn(__dmul_rn(poly, dm_pow2i(k + 64)), dm_pow2i(-64));
}

__device__ inline double dm_log(double x)
{
    const double HI = 0x1.62e42fee00000p-1, LO = 0x1.a39ef35793c76p-33;
    const double SQRT2 = 0x1.6a09e667f3bcdp+0;
    const double D[12] = {0x1.0000000000000p+0, 0x1.5555555555555p-2, 0x1.999999999999ap-3,
                          0x1.2492492492492p-3, 0x1.c71c71c71c71cp-4, 0x1.745d1745d1746p-4,
                          0x1.3b13b13b13b14p-4, 0x1.1111111111111p-4, 0x1.e1e1e1e1e1e1ep-5,
                          0x1.af286bca1af28p-5, 0x1.8618618618618p-5, 0x1.642c8590b2164p-5};
    if (x != x || x < 0.0) return __longlong_as_double(0x7ff8000000000000LL);
    if (x == 0.0) return __longlong_as_double((long long)0xfff0000000000000ULL);
    if (x == __longlong_as_double(0x7ff0000000000000LL)) return x;
    int e_adj = 0;
    if (x < 0x1p-1022) {
        x = __dmul_rn(x, 0x1p54);
        e_adj = -54;
    }
    unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    int e = (int)((bits >> 52) & 0x7ff) - 1023 + e_adj;
    bits = (bits & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL;
    double m = __longlong_as_double((long long)bits);
    if (m > SQRT2) {
        m = __dmul_rn(m, 0.5);
        e = e + 1;
    }
    const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
    const double z = __dmul_rn(s, s);
    double poly = D[11];
#pragma unroll
    for (int j = 10; j >= 0; --j) poly = __dadd_rn(__dmul_rn(poly, z), D[j]);
    const double lnm = __dmul_rn(__dadd_rn(s, s), poly);
    const double ed = (double)e;
    return __dadd_rn(__dmul_rn(ed, HI), __dadd_rn(__dmul_rn(ed, LO), lnm));
}

// Per-iteration metrics.  Accepted moves are counted from the rows themselves (an
// accepted Ising flip changes one bit, an accepted Potts move one nibble, since the
// proposal differs from the old colour) or per decision (polymer).  Tunnelling: a
// walker's bin is sampled at the end of every sweep; an event is an arrival at the
// lowest reachable bin when the highest was the last of the two visited, or the
// reverse.  st: 0 neither visited yet, 1 lowest last, 2 highest last (r, r_lo, r_hi
// in one unit: bins, or row offsets RS bin).
__device__ __forceinline__ void tunnel_step(int r, int r_lo, int r_hi, int &st, unsigned &ev)
{
    if (r == r_lo) {
        ev += (st == 2);
        st = 1;
    } else if (r == r_hi) {
        ev += (st == 1);
        st = 2;
    }
}

// Changed 4-bit fields between two packed Potts words.
__device__ __forceinline__ unsigned changed_nibbles(uint32_t a, uint32_t b)
{
    const uint32_t x = a ^ b;
    return (unsigned)__popc((x | (x >> 1) | (x >> 2) | (x >> 3)) & 0x11111111u);
}

// Add a warp's counts to the context's open counters (accepted, tunnelling
// events); every lane of the warp calls it.
__device__ __forceinline__ void flush_metrics(unsigned long long *m, unsigned long long acc, unsigned ev)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_down_sync(0xffffffffu, acc, o);
        ev += __shfl_down_sync(0xffffffffu, ev, o);
    }
    if ((threadIdx.x & 31) == 0 && m) {
        if (acc) atomicAdd(&m[0], acc);
        if (ev) atomicAdd(&m[1], (unsigned long long)ev);
    }
}

}  // namespace muca
