// Offline assembly of the space-time reduced operators through the block
// structure of Sec. 4.3 (Eqs. blockstructure, ij-block-matrix, j-block-vector,
// block-reduced-initial-vec); the space-time basis Phi_st is never formed.
//
//   Ahat_q = Phi_s^T (A_q Phi_s):  sliced-ELL SpMM (one thread per row and
//            8 basis columns, all samples of the pattern share the column
//            gathers) followed by an FP64 GEMM with the reduction over the N
//            rows split across the GPU.
//   G  = T^T diag(dt) T,  G1 = T^T T,  G2 = T(2:Nt)^T T(1:Nt-1):  FP64 GEMMs;
//        M_i and S_i are the (i, i) diagonal blocks of G1 and G2.
//   fhat^st[i + ns j] = sum_k dt_k T[k, i + ns j] (Phi_s^T B f^k)_i
//   uhat0^st[i + ns j] = T[0, i + ns j] (Phi_s^T u0)_i
// and, for the spatial ROM (Eq. galerkin), Bhat f^k per step and Phi_s^T u0.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int CB = 8;  // basis columns per thread in the SpMM

__global__ void spmm_kernel(int64_t N, const int64_t* __restrict__ slice_ptr,
                            const int32_t* __restrict__ slice_w, const int32_t* __restrict__ col,
                            const double* __restrict__ vals, int64_t ell, int ns,
                            const double* __restrict__ phi, double* Y) {
    const int q = blockIdx.y / ((ns + CB - 1) / CB);
    const int cb = (blockIdx.y % ((ns + CB - 1) / CB)) * CB;
    const double* vq = vals + (int64_t)q * ell;
    double* Yq = Y + (int64_t)q * N * ns;
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < N;
         row += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sl = row / kSlice;
        const int w = slice_w[sl];
        const int64_t base = slice_ptr[sl] + row % kSlice;
        double acc[CB];
#pragma unroll
        for (int u = 0; u < CB; ++u) acc[u] = 0.0;
        for (int k = 0; k < w; ++k) {
            const int64_t e = base + (int64_t)k * kSlice;
            const int c = col[e];
            const double a = vq[e];
#pragma unroll
            for (int u = 0; u < CB; ++u)
                if (cb + u < ns) acc[u] = fma(a, phi[c + (int64_t)(cb + u) * N], acc[u]);
        }
#pragma unroll
        for (int u = 0; u < CB; ++u)
            if (cb + u < ns) Yq[row + (int64_t)(cb + u) * N] = acc[u];
    }
}

// Td[k, c] = dt[k] * T[k, c]
__global__ void scale_rows_kernel(int Nt, int n, const double* __restrict__ dt,
                                  const double* __restrict__ T, double* Td) {
    const int64_t tot = (int64_t)Nt * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
         t += (int64_t)gridDim.x * blockDim.x)
        Td[t] = dt[t % Nt] * T[t];
}

// M_i[j', j] = G1[(i + ns j'), (i + ns j)], S_i likewise from G2.
__global__ void extract_ms_kernel(int ns, int nt, const double* __restrict__ G1,
                                  const double* __restrict__ G2, double* M, double* S) {
    const int n = ns * nt;
    const int tot = ns * nt * nt;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
        const int jp = t % nt, j = (t / nt) % nt, i = t / (nt * nt);
        const int64_t g = (int64_t)(i + ns * jp) + (int64_t)(i + ns * j) * n;
        M[t] = G1[g];
        S[t] = G2[g];
    }
}

// rhs[i + ns j] = sum_k dt_k T[k, i+ns j] sum_s Bhat[i, s] F[k, s] + T[0, i+ns j] u0hat[i]
__global__ void rhs_kernel(int ns, int nt, int Nt, int n_in, const double* __restrict__ dt,
                           const double* __restrict__ T, const double* __restrict__ Bhat,
                           const double* __restrict__ F, const double* __restrict__ u0hat,
                           double* rhs) {
    const int n = ns * nt;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int i = t % ns;
        const double* Tc = T + (int64_t)t * Nt;
        double f = 0.0;
        for (int k = 0; k < Nt; ++k) {
            double g = 0.0;
            for (int s = 0; s < n_in; ++s) g = fma(Bhat[i + (int64_t)s * ns], F[(int64_t)k * n_in + s], g);
            f = fma(dt[k] * Tc[k], g, f);
        }
        if (u0hat) f = fma(Tc[0], u0hat[i], f);
        rhs[t] = f;
    }
}

// bs[i + ns k] = sum_s Bhat[i, s] F[k, s]: the spatial ROM's input term of step k + 1
__global__ void spatial_forcing_kernel(int ns, int Nt, int n_in, const double* __restrict__ Bhat,
                                       const double* __restrict__ F, double* bs) {
    const int tot = ns * Nt;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
        const int i = t % ns, k = t / ns;
        double g = 0.0;
        for (int s = 0; s < n_in; ++s) g = fma(Bhat[i + (int64_t)s * ns], F[(int64_t)k * n_in + s], g);
        bs[t] = g;
    }
}

__global__ void to_f32_kernel(int64_t n, const double* __restrict__ x, float* y) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x)
        y[t] = (float)x[t];
}

int gridn(st_model* m, int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8 * m->num_sms));
}

}  // namespace

extern "C" st_status st_rom_assemble(st_model* m, const double* dt, int32_t n_in, const double* B,
                                     const double* F, const double* u0) {
    if (!m) return st_fail(ST_ERR_ARG, "st_rom_assemble: NULL model");
    if (!m->d_phi) return st_fail(ST_ERR_STATE, "st_rom_assemble: no basis (build or set one first)");
    if (!dt || n_in < 0 || (n_in > 0 && (!B || !F)))
        return st_fail(ST_ERR_ARG, "st_rom_assemble: bad arguments");
    const int ns = m->ns, nt = m->nt, Nt = m->Nt, n = ns * nt, Q = m->Q;
    const int64_t N = m->N;
    for (int k = 0; k < Nt; ++k)
        if (!(dt[k] > 0)) return st_fail(ST_ERR_ARG, "st_rom_assemble: dt must be positive");
    cudaStream_t st = m->stream;
    st_internal_free_reduced(m);
    ST_CUDA_TRY(cudaMalloc(&m->d_Ahat, sizeof(double) * Q * ns * ns));
    ST_CUDA_TRY(cudaMalloc(&m->d_G, sizeof(double) * n * n));
    ST_CUDA_TRY(cudaMalloc(&m->d_G32, sizeof(float) * n * n));
    ST_CUDA_TRY(cudaMalloc(&m->d_M, sizeof(double) * ns * nt * nt));
    ST_CUDA_TRY(cudaMalloc(&m->d_S, sizeof(double) * ns * nt * nt));
    ST_CUDA_TRY(cudaMalloc(&m->d_rhs, sizeof(double) * n));
    ST_CUDA_TRY(cudaMalloc(&m->d_dt, sizeof(double) * Nt));
    ST_CUDA_TRY(cudaMalloc(&m->d_bs, sizeof(double) * ns * Nt));
    ST_CUDA_TRY(cudaMalloc(&m->d_u0s, sizeof(double) * ns));
    // workspace: Y (Q x N x ns) | Td (Nt x n) | G1, G2 (n x n) | Bhat (ns x n_in) | u0hat (ns) | F (Nt x n_in)
    const size_t szY = (size_t)Q * N * ns, szTd = (size_t)Nt * n, szG = (size_t)n * n;
    const size_t szB = (size_t)ns * std::max(n_in, 1), szF = (size_t)Nt * std::max(n_in, 1);
    ST_TRY(st_grow(m, m->ws_pod2, sizeof(double) * (szY + szTd + 2 * szG + szB + ns + szF + 16)));
    double* Y = (double*)m->ws_pod2.p;
    double* Td = Y + szY;
    double* G1 = Td + szTd;
    double* G2 = G1 + szG;
    double* Bhat = G2 + szG;
    double* u0hat = Bhat + szB;
    double* dF = u0hat + ns;
    ST_CUDA_TRY(cudaMemcpyAsync(m->d_dt, dt, sizeof(double) * Nt, cudaMemcpyHostToDevice, st));
    if (n_in > 0)
        ST_CUDA_TRY(cudaMemcpyAsync(dF, F, sizeof(double) * Nt * n_in, cudaMemcpyHostToDevice, st));
    // Ahat_q
    {
        dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((N + 127) / 128, 4 * m->num_sms)),
                  (unsigned)(Q * ((ns + CB - 1) / CB)));
        {
            ST_PROF(m, "spmm_kernel");
            spmm_kernel<<<grid, 128, 0, st>>>(N, m->d_slice_ptr, m->d_slice_w, m->d_col, m->d_vals,
                                              m->ell_size, ns, m->d_phi, Y);
            ST_TRY(st_check_launch("spmm"));
        }
        for (int q = 0; q < Q; ++q)
            ST_TRY(st_dgemm(m, true, false, ns, ns, N, 1.0, m->d_phi, N, Y + (size_t)q * N * ns, N, 0.0,
                            m->d_Ahat + (size_t)q * ns * ns, ns));
    }
    // temporal products
    scale_rows_kernel<<<gridn(m, szTd), 256, 0, st>>>(Nt, n, m->d_dt, m->d_T, Td);
    ST_TRY(st_check_launch("scale_rows"));
    ST_TRY(st_dgemm(m, true, false, n, n, Nt, 1.0, m->d_T, Nt, Td, Nt, 0.0, m->d_G, n));
    ST_TRY(st_dgemm(m, true, false, n, n, Nt, 1.0, m->d_T, Nt, m->d_T, Nt, 0.0, G1, n));
    if (Nt > 1)
        ST_TRY(st_dgemm(m, true, false, n, n, Nt - 1, 1.0, m->d_T + 1, Nt, m->d_T, Nt, 0.0, G2, n));
    else
        ST_CUDA_TRY(cudaMemsetAsync(G2, 0, sizeof(double) * szG, st));
    extract_ms_kernel<<<gridn(m, (int64_t)ns * nt * nt), 256, 0, st>>>(ns, nt, G1, G2, m->d_M, m->d_S);
    ST_TRY(st_check_launch("extract_ms"));
    to_f32_kernel<<<gridn(m, szG), 256, 0, st>>>((int64_t)szG, m->d_G, m->d_G32);
    ST_TRY(st_check_launch("to_f32"));
    // reduced input and initial vectors
    if (n_in > 0) ST_TRY(st_dgemm(m, true, false, ns, n_in, N, 1.0, m->d_phi, N, B, N, 0.0, Bhat, ns));
    if (u0) ST_TRY(st_dgemm(m, true, false, ns, 1, N, 1.0, m->d_phi, N, u0, N, 0.0, u0hat, ns));
    rhs_kernel<<<gridn(m, n), 256, 0, st>>>(ns, nt, Nt, n_in, m->d_dt, m->d_T, Bhat, dF,
                                            u0 ? u0hat : nullptr, m->d_rhs);
    ST_TRY(st_check_launch("rhs"));
    spatial_forcing_kernel<<<gridn(m, (int64_t)ns * Nt), 256, 0, st>>>(ns, Nt, n_in, Bhat, dF, m->d_bs);
    ST_TRY(st_check_launch("spatial forcing"));
    if (u0)
        ST_CUDA_TRY(cudaMemcpyAsync(m->d_u0s, u0hat, sizeof(double) * ns, cudaMemcpyDeviceToDevice, st));
    else
        ST_CUDA_TRY(cudaMemsetAsync(m->d_u0s, 0, sizeof(double) * ns, st));
    m->assembled = true;
    return ST_OK;
}

st_status st_internal_install_reduced(st_model* m, const double* Ahat, const double* G, const double* M,
                                      const double* S, const double* rhs, const double* dt, const double* bs,
                                      const double* u0s) {
    if (!m->d_phi) return st_fail(ST_ERR_STATE, "reduced operators need a basis");
    const size_t ns = m->ns, nt = m->nt, Nt = m->Nt, n = ns * nt, Q = m->Q;
    cudaStream_t st = m->stream;
    st_internal_free_reduced(m);
    double** dst[8] = {&m->d_Ahat, &m->d_G, &m->d_M, &m->d_S, &m->d_rhs, &m->d_dt, &m->d_bs, &m->d_u0s};
    const double* src[8] = {Ahat, G, M, S, rhs, dt, bs, u0s};
    const size_t cnt[8] = {Q * ns * ns, n * n, ns * nt * nt, ns * nt * nt, n, Nt, ns * Nt, ns};
    for (int i = 0; i < 8; ++i) {
        ST_CUDA_TRY(cudaMalloc(dst[i], sizeof(double) * std::max<size_t>(cnt[i], 1)));
        ST_CUDA_TRY(cudaMemcpyAsync(*dst[i], src[i], sizeof(double) * cnt[i], cudaMemcpyHostToDevice, st));
    }
    ST_CUDA_TRY(cudaMalloc(&m->d_G32, sizeof(float) * n * n));
    to_f32_kernel<<<gridn(m, (int64_t)(n * n)), 256, 0, st>>>((int64_t)(n * n), m->d_G, m->d_G32);
    ST_TRY(st_check_launch("to_f32"));
    ST_CUDA_TRY(cudaStreamSynchronize(st));
    m->assembled = true;
    return ST_OK;
}
