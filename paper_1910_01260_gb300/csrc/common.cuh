// Device-side helpers: bounded grid barrier, error word, warp reductions.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "st_rom.h"

__device__ __forceinline__ void st_dev_error(int32_t* err, int32_t code) {
    atomicCAS(reinterpret_cast<int*>(err), 0, code);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Counting grid barrier for cooperative launches (all blocks are
// co-resident, so every arrival happens), over the whole grid or over the
// `parties` CTAs of one sub-grid that share the counters.  The wait is bounded: after
// `limit` polls the waiting block records ST_ERR_TIMEOUT in the model error
// word, raises the launch's abort flag and the barrier reports failure, so
// every block returns instead of hanging.  count/gen/abort are zeroed by the
// host before each launch.
struct GridBarrier {
    unsigned int* count;
    unsigned int* gen;
    unsigned int* abort;
    int32_t* err;
    long long limit;
    unsigned int parties;  // CTAs that take part; 0 = the whole grid
};

__device__ __forceinline__ void grid_abort(const GridBarrier& b, int32_t code) {
    st_dev_error(b.err, code);
    atomicExch(b.abort, 1u);
}

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned int atom_add_acq_rel_gpu(unsigned int* p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ void st_relaxed_gpu(unsigned int* p, unsigned int v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void red_release_gpu(unsigned int* p, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_release_gpu(unsigned int* p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier of a cooperative launch (every CTA co-resident).  The
// CTA's writes are ordered before its arrival by the block barrier and the
// release of the arrival atomic; the last CTA to arrive resets the counter
// and releases the generation word, on which the others spin with acquire
// loads.  The spin is bounded: past `limit` polls the kernel records
// ST_ERR_TIMEOUT and raises the abort flag; a CTA that sees the abort flag
// stops waiting.  Returns false after an abort or a timeout (a CTA that
// aborts returns without arriving, so the others never complete the barrier).
__device__ __forceinline__ bool grid_sync(const GridBarrier& b, int* s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int my = ld_acquire_gpu(b.gen);
        const unsigned int arrived = atom_add_acq_rel_gpu(b.count, 1u);
        int ok = 1;
        if (arrived == (b.parties ? b.parties : gridDim.x) - 1) {
            st_relaxed_gpu(b.count, 0u);
            red_release_gpu(b.gen, 1u);
        } else {
            long long it = 0;
            while (ld_acquire_gpu(b.gen) == my) {
                if (++it > b.limit) {
                    grid_abort(b, ST_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                if (*(volatile unsigned int*)b.abort) {
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// Point-to-point wait of a cooperative launch: one thread spins (acquire)
// until the counter *f reaches target, bounded like grid_sync; the caller
// follows with a block barrier.  False after an abort or a timeout.
__device__ __forceinline__ bool wait_ready(const GridBarrier& b, const unsigned int* f, unsigned int target) {
    long long it = 0;
    while (ld_acquire_gpu(f) < target) {
        if (++it > b.limit) {
            grid_abort(b, ST_ERR_TIMEOUT);
            return false;
        }
        if (*(volatile unsigned int*)b.abort) return false;
        __nanosleep(32);
    }
    return true;
}

__device__ __forceinline__ bool st_finite(double x) { return isfinite(x); }
