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
