// FP64 SIMT GEMM, column major, batched, with a deterministic split over K.
//
// GB300 issues FP64 at a small fraction of its FP32 rate, so a register tile
// of 2x8 outputs per thread and a 64x64x16 shared-memory tile already keep
// the FP64 pipe busy; the kernel's job is to avoid redundant global traffic,
// to skip the padding of edge tiles, and to expose enough tiles (split-K,
// balanced over the SMs) for the tall-skinny products of the POD, where K is
// the number of spatial unknowns.
#include <algorithm>

#include "internal.h"

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

// 64 x 64 output tile per block, 8 warps: warp w owns the 8 contiguous
// columns 8w..8w+7 and lane l the rows l and l + 32, so a tile that is
// partly outside the matrix drops whole warps (columns) or the second row
// (rows) with warp-uniform branches instead of computing padding.
template <bool TA, bool TB>
__global__ void __launch_bounds__(NT, 3) dgemm_kernel(int64_t M, int64_t Nc, int64_t K, int64_t kchunk,
                                                      double alpha, const double* __restrict__ A,
                                                      int64_t lda, int64_t sA, const double* __restrict__ B,
                                                      int64_t ldb, int64_t sB, double beta, double* C,
                                                      int64_t ldc, int64_t sC, int splits, double* ws) {
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int64_t i0 = (int64_t)blockIdx.x * BM, j0 = (int64_t)blockIdx.y * BN;
    const int bz = blockIdx.z;
    const int batch = bz / splits, split = bz % splits;
    A += batch * sA;
    B += batch * sB;
    C += batch * sC;
    const int64_t kb = (int64_t)split * kchunk;
    const int64_t ke = K < kb + kchunk ? K : kb + kchunk;
    const int64_t rem_rows = M - i0, rem_cols = Nc - j0 - 8 * warp;
    const bool active = rem_cols > 0;     // warp has a valid column
    const bool two_rows = rem_rows > 32;  // rows l + 32 exist in this tile
    double acc[2][8];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc[x][y] = 0.0;

    for (int64_t k0 = kb; k0 < ke; k0 += BK) {
        // A tile: BM x BK
#pragma unroll
        for (int l = 0; l < (BM * BK) / NT; ++l) {
            int idx = tid + l * NT;
            int ii, kk;
            if (!TA) { ii = idx % BM; kk = idx / BM; }
            else     { kk = idx % BK; ii = idx / BK; }
            int64_t gi = i0 + ii, gk = k0 + kk;
            double v = 0.0;
            if (gi < M && gk < ke) v = TA ? A[gk + gi * lda] : A[gi + gk * lda];
            As[kk][ii] = v;
        }
        // B tile: BK x BN
#pragma unroll
        for (int l = 0; l < (BN * BK) / NT; ++l) {
            int idx = tid + l * NT;
            int jj, kk;
            if (!TB) { kk = idx % BK; jj = idx / BK; }
            else     { jj = idx % BN; kk = idx / BN; }
            int64_t gj = j0 + jj, gk = k0 + kk;
            double v = 0.0;
            if (gj < Nc && gk < ke) v = TB ? B[gj + gk * ldb] : B[gk + gj * ldb];
            Bs[kk][jj] = v;
        }
        __syncthreads();
        if (active) {
            if (two_rows) {
#pragma unroll
                for (int kk = 0; kk < BK; ++kk) {
                    const double a0 = As[kk][lane], a1 = As[kk][lane + 32];
#pragma unroll
                    for (int y = 0; y < 8; ++y) {
                        const double bv = Bs[kk][8 * warp + y];
                        acc[0][y] = fma(a0, bv, acc[0][y]);
                        acc[1][y] = fma(a1, bv, acc[1][y]);
                    }
                }
            } else {
#pragma unroll
                for (int kk = 0; kk < BK; ++kk) {
                    const double a0 = As[kk][lane];
#pragma unroll
                    for (int y = 0; y < 8; ++y) acc[0][y] = fma(a0, Bs[kk][8 * warp + y], acc[0][y]);
                }
            }
        }
        __syncthreads();
    }
    if (!active) return;
#pragma unroll
    for (int x = 0; x < 2; ++x) {
        const int64_t gi = i0 + lane + 32 * x;
        if (gi >= M) continue;
#pragma unroll
        for (int y = 0; y < 8; ++y) {
            const int64_t gj = j0 + 8 * warp + y;
            if (gj >= Nc) continue;
            if (splits == 1) {
                double* c = C + gi + gj * ldc;
                *c = beta == 0.0 ? alpha * acc[x][y] : fma(alpha, acc[x][y], beta * *c);
            } else {
                ws[(size_t)split * M * Nc + gi + gj * M] = acc[x][y];
            }
        }
    }
}

__global__ void splitk_reduce(int64_t M, int64_t Nc, int splits, const double* __restrict__ ws,
                              double alpha, double beta, double* C, int64_t ldc) {
    int64_t n = M * Nc;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int p = 0; p < splits; ++p) s += ws[(size_t)p * n + t];
        int64_t i = t % M, j = t / M;
        double* c = C + i + j * ldc;
        *c = beta == 0.0 ? alpha * s : fma(alpha, s, beta * *c);
    }
}

}  // namespace

static bool use_ozaki(const st_model* m, int64_t M, int64_t Nc, int64_t K) {
    return m->opt.fp64_gemm == ST_DGEMM_OZAKI && K >= 8 && 2.0 * (double)M * (double)Nc * (double)K >= 1048576.0;
}

st_status st_dgemm_slot(st_model* m, int slotA, bool reuseA, bool transA, bool transB, int64_t M, int64_t Nc,
                        int64_t K, double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                        double beta, double* C, int64_t ldc) {
    if (M > 0 && Nc > 0 && use_ozaki(m, M, Nc, K))
        return st_ozaki_gemm(m, transA, transB, M, Nc, K, alpha, A, lda, B, ldb, beta, C, ldc, slotA, reuseA);
    return st_dgemm(m, transA, transB, M, Nc, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

st_status st_dgemm(st_model* m, bool transA, bool transB, int64_t M, int64_t Nc, int64_t K,
                   double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                   double beta, double* C, int64_t ldc, int batch, int64_t sA, int64_t sB,
                   int64_t sC) {
    if (M <= 0 || Nc <= 0 || batch <= 0) return ST_OK;
    // large products go to the tensor cores (exact operand splitting)
    if (batch == 1 && use_ozaki(m, M, Nc, K))
        return st_ozaki_gemm(m, transA, transB, M, Nc, K, alpha, A, lda, B, ldb, beta, C, ldc);
    if (K <= 0) {
        // C = beta * C
        if (beta == 1.0) return ST_OK;
        K = 0;
    }
    int64_t tiles = ((M + BM - 1) / BM) * ((Nc + BN - 1) / BN) * batch;
    // split long K so that the blocks fill the resident slots in one wave
    // (never more: a second, nearly empty wave would double the time)
    static int per_sm = 0;
    if (per_sm == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, dgemm_kernel<false, false>, NT, 0) != cudaSuccess) v = 1;
        per_sm = std::max(1, v);
    }
    const int64_t slots = (int64_t)per_sm * m->num_sms;
    int splits = 1;
    if (batch == 1 && K > 2048 && 2 * tiles <= slots) {
        // FP64 issue is the bound, so the time follows the SM with the most
        // blocks: pick the split that balances blocks over the SMs best
        // (at most one resident wave, K chunks of at least 256)
        const int64_t cap = std::min<int64_t>(512, K / 256);
        double best = -1.0;
        for (int64_t sp = 1; sp <= cap && tiles * sp <= slots; ++sp) {
            const int64_t blocks = tiles * sp;
            const int64_t per = (blocks + m->num_sms - 1) / m->num_sms;
            const double eff = (double)blocks / (double)(per * m->num_sms);
            if (eff > best + 1e-9) {
                best = eff;
                splits = (int)sp;
            }
        }
    }
    int64_t kchunk = K > 0 ? ((K + splits - 1) / splits + BK - 1) / BK * BK : 0;
    if (K > 0) splits = (int)((K + kchunk - 1) / kchunk);
    double* ws = nullptr;
    if (splits > 1) {
        ST_TRY(st_grow(m, m->ws_gemm, sizeof(double) * (size_t)splits * M * Nc));
        ws = (double*)m->ws_gemm.p;
    }
    dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((Nc + BN - 1) / BN),
              (unsigned)(batch * std::max(splits, 1)));
    if (grid.y > 65535 || grid.z > 65535) return st_fail(ST_ERR_ARG, "st_dgemm: grid too large");
    int sp = std::max(splits, 1);
    // profile classes: tall-skinny updates (M large), split-K projections,
    // and small products
    const char* pname = splits > 1 ? "dgemm_kernel[split-k]" : (M >= 4096 ? "dgemm_kernel[tall]" : "dgemm_kernel[small]");
    ST_PROF(m, pname);
    st_prof_flops(m, pname, 2.0 * (double)M * (double)Nc * (double)K * (double)batch);
#define ST_LAUNCH(ta, tb)                                                                   \
    dgemm_kernel<ta, tb><<<grid, NT, 0, m->stream>>>(M, Nc, K, kchunk, alpha, A, lda, sA, B, \
                                                     ldb, sB, beta, C, ldc, sC, sp, ws)
    if (!transA && !transB) ST_LAUNCH(false, false);
    else if (transA && !transB) ST_LAUNCH(true, false);
    else if (!transA && transB) ST_LAUNCH(false, true);
    else ST_LAUNCH(true, true);
#undef ST_LAUNCH
    ST_TRY(st_check_launch("dgemm"));
    if (splits > 1) {
        int blocks = (int)std::min<int64_t>((M * Nc + 255) / 256, 4 * m->num_sms);
        splitk_reduce<<<blocks, 256, 0, m->stream>>>(M, Nc, splits, ws, alpha, beta, C, ldc);
        ST_TRY(st_check_launch("splitk_reduce"));
    }
    return ST_OK;
}

extern "C" st_status st_gemm_f64(st_model* m, int32_t trans_a, int32_t trans_b, int64_t M, int64_t N, int64_t K,
                                 double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                                 double beta, double* C, int64_t ldc) {
    if (!m) return st_fail(ST_ERR_ARG, "st_gemm_f64: NULL model");
    if (M < 0 || N < 0 || K < 0) return st_fail(ST_ERR_ARG, "st_gemm_f64: negative size");
    if (M == 0 || N == 0) return ST_OK;
    if (!C || (K > 0 && (!A || !B))) return st_fail(ST_ERR_ARG, "st_gemm_f64: NULL operand");
    const int64_t rowsA = trans_a ? K : M, rowsB = trans_b ? N : K;
    if (lda < std::max<int64_t>(1, rowsA) || ldb < std::max<int64_t>(1, rowsB) || ldc < M)
        return st_fail(ST_ERR_ARG, "st_gemm_f64: leading dimension too small");
    return st_dgemm(m, trans_a != 0, trans_b != 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}
