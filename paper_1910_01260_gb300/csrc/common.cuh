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
// co-resident, so every arrival happens).  The wait is bounded: after
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
};

__device__ __forceinline__ void grid_abort(const GridBarrier& b, int32_t code) {
    st_dev_error(b.err, code);
    atomicExch(b.abort, 1u);
}

__device__ __forceinline__ bool grid_sync(const GridBarrier& b, int* s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* vgen = b.gen;
        unsigned int my = *vgen;
        __threadfence();
        unsigned int arrived = atomicAdd(b.count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(b.count, 0u);
            __threadfence();
            atomicAdd(b.gen, 1u);
        } else {
            long long it = 0;
            while (*vgen == my) {
                if (++it > b.limit || *(volatile unsigned int*)b.abort) {
                    if (it > b.limit) grid_abort(b, ST_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        *s_flag = (*(volatile unsigned int*)b.abort == 0u);
    }
    __syncthreads();
    return *s_flag != 0;
}

__device__ __forceinline__ bool st_finite(double x) { return isfinite(x); }
