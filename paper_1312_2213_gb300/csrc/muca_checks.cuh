// muca_checks.cuh -- the checked build's bounds checks on the sweeps' shared-memory
// tables (the library built with -DMUCA_CHECKED, loaded when MUCA_DEBUG=1).  Every
// threshold load and histogram update of a spin sweep goes through checked_word
// (word index into the table) or checked_addr (shared-window byte address).  An
// index outside the table is recorded in a per-block flag and replaced by the
// table's first entry, so the access stays inside the table; the block ORs the
// flag into the device error word (bit 2) at its end and the host reports
// MUCA_ERR_CHECK.  In the regular build both helpers return their argument.
#pragma once
#include "muca_internal.h"

namespace muca {

#ifdef MUCA_CHECKED
__device__ __forceinline__ int &block_check_flag()
{
    __shared__ int s_flag;
    return s_flag;
}

__device__ __forceinline__ int &block_table_words()
{
    __shared__ int s_words;
    return s_words;
}
#endif

// Thread 0, before the block's first barrier: the table's size in words (B RS), or 0
// when the context's "debug_check" hook asks every check to fail.
__device__ __forceinline__ void checks_begin(int table_words, int force_fail)
{
#ifdef MUCA_CHECKED
    if (threadIdx.x == 0) {
        block_check_flag() = 0;
        block_table_words() = force_fail ? 0 : table_words;
    }
#else
    (void)table_words;
    (void)force_fail;
#endif
}

__device__ __forceinline__ int checked_word(int i)
{
#ifdef MUCA_CHECKED
    if ((unsigned)i >= (unsigned)block_table_words()) {
        block_check_flag() = 1;
        return 0;
    }
#endif
    return i;
}

__device__ __forceinline__ int checked_addr(int addr, int base)
{
#ifdef MUCA_CHECKED
    if ((unsigned)(addr - base) >= 4u * (unsigned)block_table_words()) {
        block_check_flag() = 1;
        return base;
    }
#else
    (void)base;
#endif
    return addr;
}

// An index into an array of n entries other than the table (checked build: the
// histogram counters of the global-table Potts form).
__device__ __forceinline__ int checked_index(int i, int n)
{
#ifdef MUCA_CHECKED
    if ((unsigned)i >= (unsigned)n) {
        block_check_flag() = 1;
        return 0;
    }
#else
    (void)n;
#endif
    return i;
}

// After the block's last barrier.
__device__ __forceinline__ void checks_end(const DevState *state)
{
#ifdef MUCA_CHECKED
    if (threadIdx.x == 0 && block_check_flag()) atomicOr(const_cast<int *>(&state->err), 2);
#else
    (void)state;
#endif
}

}  // namespace muca
