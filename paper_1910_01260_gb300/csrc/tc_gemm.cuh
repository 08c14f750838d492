// BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores (tcgen05):
//   C[M x N] = act(A[M x K] * B[N x K]^T + bias),  A and B row major (K-major).
// One CTA (4 warps) computes a 128 x BN tile.  Thread 0 streams K in chunks of
// 64 through an NSTAGE ring of shared-memory stages filled by TMA
// (cp.async.bulk.tensor, 128-byte swizzle) and issues tcgen05.mma (M = 128,
// N = BN, K = 16 per instruction) into an FP32 accumulator in tensor memory;
// tcgen05.commit releases a stage when its MMAs are done.  The four warps
// then read their 32 accumulator lanes with tcgen05.ld and apply the
// epilogue (bias, optional exact GELU, FP32 / BF16 / pre-activation stores).
// Every mbarrier wait is bounded; on a timeout the CTA records ST_ERR_TIMEOUT,
// waits (bounded) for its MMAs, frees its tensor memory and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace tc {

constexpr int kBM = 128;      // rows per CTA tile (UMMA M)
constexpr int kBK = 64;       // K per stage: one 128-byte swizzled row of BF16
constexpr int kStages = 4;
constexpr int kThreads = 128;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor of a K-major operand tile stored with the
// 128-byte swizzle: 8-row atoms of 128-byte rows, atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address (16-byte units)
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= (uint64_t)2 << 61;                     // 128-byte swizzle
    return d;
}

// Instruction descriptor: kind::f16 with BF16 A/B, FP32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float gelu_exact(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

struct GemmArgs {
    int M, N, K;
    const float* bias;       // [N] or null
    int gelu;                // apply GELU in the epilogue
    float* out_f32;          // [M x ldf] or null: activation (or plain result)
    int ldf;
    __nv_bfloat16* out_bf16; // [M x ldb] or null: activation in BF16
    int ldb;
    float* out_pre;          // [M x ldp] or null: pre-activation (z)
    int ldp;
    int32_t* err;
    long long limit;
};

// Dynamic shared memory for a BN-wide tile (1 KB extra for alignment).
__host__ __device__ constexpr size_t smem_bytes(int BN) {
    return (size_t)kStages * (kBM * kBK * 2 + BN * kBK * 2) + 1024 + 256;
}

template <int BN>
__global__ void __launch_bounds__(kThreads) gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                        const __grid_constant__ CUtensorMap tmB, GemmArgs g) {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "UMMA N for M = 128");
    constexpr uint32_t kTmemCols = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
    constexpr uint32_t kStageA = kBM * kBK * 2, kStageB = BN * kBK * 2;
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bars[2 * kStages + 1];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[kStages]), done = smem_u32(&bars[2 * kStages]);
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int kchunks = (g.K + kBK - 1) / kBK;

    if (tid == 0) {
        for (int s = 0; s < 2 * kStages + 1; ++s) mbar_init(smem_u32(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (tid == 0) {
        const uint32_t idesc = idesc_bf16(kBM, BN);
        auto issue = [&](int kc, int s) {
            const uint32_t sa = base + s * (kStageA + kStageB), sb = sa + kStageA;
            mbar_expect_tx(full0 + 8 * s, kStageA + kStageB);
            tma_load_2d(sa, &tmA, kc * kBK, m0, full0 + 8 * s);
            tma_load_2d(sb, &tmB, kc * kBK, n0, full0 + 8 * s);
        };
        int issued = 0, consumed = 0;
        for (int kc = 0; kc < kchunks && kc < kStages; ++kc, ++issued) issue(kc, kc);
        bool ok = true;
        for (int kc = 0; kc < kchunks && ok; ++kc) {
            const int s = kc % kStages;
            const uint32_t phase = (kc / kStages) & 1;
            if (!mbar_wait(full0 + 8 * s, phase, g.limit)) {
                ok = false;
                break;
            }
            ++consumed;
            const uint32_t sa = base + s * (kStageA + kStageB), sb = sa + kStageA;
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk)
                umma_bf16(tmem, sdesc_sw128(sa + kk * 32), sdesc_sw128(sb + kk * 32), idesc,
                          (kc > 0 || kk > 0) ? 1u : 0u);
            umma_commit(empty0 + 8 * s);
            if (kc + kStages < kchunks) {
                if (!mbar_wait(empty0 + 8 * s, phase, g.limit)) {
                    ok = false;
                    break;
                }
                issue(kc + kStages, s);
                ++issued;
            }
        }
        umma_commit(done);
        if (!ok) {
            s_fail = 1;
            // let the loads still in flight land before the CTA's memory is released
            for (int kc = consumed; kc < issued; ++kc)
                mbar_wait(full0 + 8 * (kc % kStages), (kc / kStages) & 1, g.limit);
        }
    }
    __syncthreads();
    // all threads wait for the accumulator (bounded)
    if (!mbar_wait(done, 0, g.limit)) s_fail = 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (!s_fail) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int j0 = 0; j0 < BN; j0 += 16) {
            float v[16];
            tmem_ld16(trow + j0, v);
            if (row < g.M) {
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const int col = n0 + j0 + t;
                    if (col >= g.N) continue;
                    float z = v[t] + (g.bias ? g.bias[col] : 0.0f);
                    if (g.out_pre) g.out_pre[(int64_t)row * g.ldp + col] = z;
                    const float a = g.gelu ? gelu_exact(z) : z;
                    if (g.out_f32) g.out_f32[(int64_t)row * g.ldf + col] = a;
                    if (g.out_bf16) g.out_bf16[(int64_t)row * g.ldb + col] = __float2bfloat16_rn(a);
                }
            }
        }
    } else if (tid == 0) {
        st_dev_error(g.err, ST_ERR_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace tc
