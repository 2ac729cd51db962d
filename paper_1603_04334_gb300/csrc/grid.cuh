// grid.cuh -- bounded grid-wide barrier for cooperative launches (all CTAs co-resident).
//
// Every wait is bounded: a CTA that has polled `spins` times without the barrier opening
// raises b->err and leaves; CTAs waiting at the same or a later barrier see the
// flag and leave too, so a kernel whose grid can never meet ends within about the spin
// limit and reports through its own status word instead of hanging. Data that other CTAs
// wrote before a barrier is read after it with L1-bypassing loads (__ldcg).
#pragma once
#include "internal.cuh"

namespace sparc {

constexpr unsigned long long kBarrierSpins = 1ull << 25;  // polls (each an L2 round trip + 32 ns)

// The count only grows (the host zeroes the barrier before each launch): a CTA arrives with
// a release add, which returns the arrivals before it, and waits with acquire loads until
// the count reaches the next multiple of nblocks. The last CTA to arrive thus opens the
// barrier with its own add, with no reset on the critical path. Thread 0 arrives and waits
// for its CTA, between two CTA barriers.
__device__ __forceinline__ bool grid_barrier(GridBarrier *b, unsigned nblocks,
                                             unsigned long long spins = kBarrierSpins)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned old;
        asm volatile("atom.add.release.gpu.u32 %0, [%1], 1;"
                     : "=r"(old) : "l"(&b->count) : "memory");
        const unsigned target = (old / nblocks + 1u) * nblocks;
        volatile int *ve = &b->err;
        unsigned long long it = 0;
        for (;;) {
            unsigned c;
            asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(c) : "l"(&b->count) : "memory");
            // leaves when every CTA has arrived, when another CTA has given up, or after
            // `spins` polls (then it raises the flag itself)
            if ((int)(c - target) >= 0 || *ve != 0) break;
            if (++it > spins) {
                atomicExch(&b->err, 1);
                break;
            }
            __nanosleep(32);
        }
    }
    __syncthreads();
    return *((volatile int *)&b->err) == 0;
}

}  // namespace sparc
