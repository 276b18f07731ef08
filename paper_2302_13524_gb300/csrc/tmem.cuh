// tmem.cuh -- tensor memory (TMEM) as a per-CTA scratchpad for FP32 data.
//
// Each SM has 128 lanes x 512 columns of 32-bit tensor-memory cells.  A CTA
// takes a power-of-two number of columns (>= 32) with tcgen05.alloc (one whole
// warp) and returns them with tcgen05.dealloc before it exits.  A warp reaches
// the 32 lanes of its quarter, lanes 32 (warp mod 4) .. + 31; a 32x32b load or
// store moves consecutive columns of each thread's own lane to or from that
// thread's registers.  Loads complete at tcgen05.wait::ld and stores at
// tcgen05.wait::st; a thread that reads back only cells it wrote itself needs
// no other ordering.  The address of a cell is the allocation's base plus
// (lane << 16) plus the column.
#pragma once

#include <stdint.h>

namespace tmr {

// Whole warp: allocate ncols columns; the base address lands in *slot (shared
// memory).  The CTA gives up its right to allocate again, so that other CTAs
// on the SM are not held back.
__device__ __forceinline__ void tmem_alloc_warp(uint32_t *slot, uint32_t ncols)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(slot);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// Whole warp (the one that allocated): return the columns.
__device__ __forceinline__ void tmem_dealloc_warp(uint32_t base, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}

// Ordering of tensor-memory operations across a thread barrier.
__device__ __forceinline__ void tmem_fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Whole warp: two consecutive columns of each thread's lane into r[0..1]
// (valid after tmem_wait_ld and tmem_reg_ready).
__device__ __forceinline__ void tmem_ld2(uint32_t taddr, uint32_t (&r)[2])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(taddr));
}

// Whole warp: four consecutive columns of each thread's lane into r[0..3].
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}

// Whole warp: eight consecutive columns of each thread's lane into r[0..7].
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

// Whole warp: four values into four consecutive columns of each thread's lane.
__device__ __forceinline__ void tmem_st4(uint32_t taddr, float a, float b, float c, float d)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(__float_as_uint(a)),
                 "r"(__float_as_uint(b)), "r"(__float_as_uint(c)), "r"(__float_as_uint(d))
                 : "memory");
}

// Whole warp: two values into two consecutive columns of each thread's lane.
__device__ __forceinline__ void tmem_st2(uint32_t taddr, float a, float b)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(taddr), "r"(__float_as_uint(a)),
                 "r"(__float_as_uint(b))
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// After tmem_wait_ld: ties the loaded registers to the wait, so that no use of
// them is scheduled before it (volatile asm statements keep their order).
__device__ __forceinline__ void tmem_reg_ready(uint32_t (&r)[2]) { asm volatile("" : "+r"(r[0]), "+r"(r[1])); }
__device__ __forceinline__ void tmem_reg_ready(uint32_t (&r)[4])
{
    asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]));
}
__device__ __forceinline__ void tmem_reg_ready(uint32_t (&r)[8])
{
    asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]));
}

}  // namespace tmr
