// Host side of the tcgen05 GEMM: TMA tensor maps and the launcher.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "tc_gemm.cuh"

// C = act(A[M x K] B[N x K]^T + bias); A, B row major BF16 with row strides
// lda, ldb (elements, multiples of 8).  BN is the tile width (16..256).
st_status st_tc_gemm(st_model* m, int BN, int M, int N, int K, const __nv_bfloat16* A, int lda,
                     const __nv_bfloat16* B, int ldb, const tc::GemmArgs& epilogue);

// Tensor map of a 3-D BF16 array depth x rows x inner (inner contiguous, row
// stride ld and plane stride `plane` in elements, multiples of 8) with a
// box_inner x box_rows x box_depth tile and the 128-byte swizzle.
st_status st_tmap_bf16_3d(CUtensorMap* map, const void* base, int64_t inner, int64_t rows, int64_t depth,
                          int64_t ld, int64_t plane, int box_inner, int box_rows, int box_depth);
