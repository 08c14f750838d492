// Host side of the tcgen05 GEMM: TMA descriptors (cuTensorMapEncodeTiled,
// reached through the runtime's driver entry point) and tile dispatch.
#include <cudaTypedefs.h>

#include <mutex>

#include "tc_host.h"

namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
cudaError_t g_encode_err = cudaSuccess;

st_status encoder(PFN_cuTensorMapEncodeTiled_v12000* out) {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        g_encode_err = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (g_encode_err == cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!g_encode) return st_fail(ST_ERR_CUDA, "cuTensorMapEncodeTiled unavailable (%s)", cudaGetErrorString(g_encode_err));
    *out = g_encode;
    return ST_OK;
}

// 2-D BF16 row-major matrix rows x cols (cols contiguous), tile box_rows x 64.
st_status tmap_bf16(CUtensorMap* map, const void* base, int rows, int cols, int ld, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc;
    ST_TRY(encoder(&enc));
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld * 2) % 16)
        return st_fail(ST_ERR_ARG, "tc_gemm: operands must be 16-byte aligned with row strides multiple of 8");
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)tc::kBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return st_fail(ST_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return ST_OK;
}

}  // namespace

// 3-D BF16 array depth x rows x inner (inner contiguous; row stride ld and
// plane stride `plane` in elements, multiples of 8), tile box_inner x
// box_rows x box_depth with the 128-byte swizzle (box_inner * 2 <= 128).
st_status st_tmap_bf16_3d(CUtensorMap* map, const void* base, int64_t inner, int64_t rows, int64_t depth,
                          int64_t ld, int64_t plane, int box_inner, int box_rows, int box_depth) {
    PFN_cuTensorMapEncodeTiled_v12000 enc;
    ST_TRY(encoder(&enc));
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld * 2) % 16 || (plane * 2) % 16 || box_inner * 2 > 128)
        return st_fail(ST_ERR_ARG, "st_tmap_bf16_3d: misaligned base, strides or box");
    cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)rows, (cuuint64_t)depth};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)plane * 2};
    cuuint32_t box[3] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows, (cuuint32_t)box_depth};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return st_fail(ST_ERR_CUDA, "cuTensorMapEncodeTiled (3-D) failed (%d)", (int)r);
    return ST_OK;
}

namespace {

template <int BN>
st_status launch(st_model* m, int M, int N, const CUtensorMap& ta, const CUtensorMap& tb, const tc::GemmArgs& g) {
    const size_t smem = tc::smem_bytes(BN);
    ST_CUDA_TRY(cudaFuncSetAttribute(tc::gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((M + tc::kBM - 1) / tc::kBM, (N + BN - 1) / BN);
    ST_PROF(m, "tc_gemm_kernel");
    st_prof_flops(m, "tc_gemm_kernel", 2.0 * (double)M * (double)N * (double)g.K);
    tc::gemm_kernel<BN><<<grid, tc::kThreads, smem, m->stream>>>(ta, tb, g);
    return st_check_launch("tc_gemm");
}

}  // namespace

st_status st_tc_gemm(st_model* m, int BN, int M, int N, int K, const __nv_bfloat16* A, int lda,
                     const __nv_bfloat16* B, int ldb, const tc::GemmArgs& epi) {
    if (M <= 0 || N <= 0 || K <= 0) return ST_OK;
    CUtensorMap ta, tb;
    ST_TRY(tmap_bf16(&ta, A, M, K, lda, tc::kBM));
    ST_TRY(tmap_bf16(&tb, B, N, K, ldb, BN));
    tc::GemmArgs g = epi;
    g.M = M;
    g.N = N;
    g.K = K;
    switch (BN) {
        case 64: return launch<64>(m, M, N, ta, tb, g);
        case 128: return launch<128>(m, M, N, ta, tb, g);
        case 240: return launch<240>(m, M, N, ta, tb, g);
        case 256: return launch<256>(m, M, N, ta, tb, g);
        default: return st_fail(ST_ERR_ARG, "tc_gemm: unsupported tile width %d", BN);
    }
}
