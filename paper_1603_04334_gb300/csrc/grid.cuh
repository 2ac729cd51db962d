// grid.cuh -- bounded grid-wide barrier for cooperative launches (all CTAs co-resident).
//
// Every wait is bounded: a CTA that has polled `spins` times without the generation
// moving on raises b->err and leaves; CTAs waiting at the same or a later barrier see the
// flag and leave too, so a kernel whose grid can never meet ends within about the spin
// limit and reports through its own status word instead of hanging. Data that other CTAs
// wrote before a barrier is read after it with L1-bypassing loads (__ldcg).
#pragma once
#include "internal.cuh"

namespace sparc {

constexpr unsigned long long kBarrierSpins = 1ull << 25;  // ~2 s of 64 ns sleeps

__device__ __forceinline__ bool grid_barrier(GridBarrier *b, unsigned nblocks,
                                             unsigned long long spins = kBarrierSpins)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vg = &b->gen;
        volatile int *ve = &b->err;
        const unsigned g = *vg;
        __threadfence();
        if (atomicAdd(&b->count, 1u) == nblocks - 1u) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            unsigned long long it = 0;
            // leaves when the generation moves on, when another CTA has given up, or after
            // `spins` polls (then it raises the flag itself)
            while (*vg == g && *ve == 0) {
                if (++it > spins) {
                    atomicExch(&b->err, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *((volatile int *)&b->err) == 0;
}

}  // namespace sparc
