// Full-order residual norms of approximate trajectories (Eq. residual):
//     r^k = u^k - u^{k-1} - dt_k A(mu) u^k - dt_k B f^k,   k = 1..Nt,
// the computable factor of the a posteriori error bounds of Theorems 1 and 3
// (the stability constants xi_k = ||(I - dt_k A)^-1||_2 and
// ||(A^st)^-1||_2 multiply it).  Checking a ROM trajectory this way reads the
// trajectory once and applies the operator once per step, instead of solving
// the full-order system.
//
// The values of A(mu) = sum_q theta_q A_q are combined once per sample into
// a sliced-ELL value array (a chunk of samples at a time).  Then one block of
// 256 threads owns 1024 consecutive rows of one step of one sample (grid:
// row blocks x steps x samples, a sample's steps consecutive so that its
// values stay in L2); each thread forms the residual of four rows and the
// block writes the sum of squares of its rows.  A second kernel adds the row
// blocks of each (sample, step) in a fixed order and takes the square root,
// so the norms are deterministic.  Like the full-order march, the pass is
// bound by the FP64 pipe (one fused multiply-add per stored entry and step);
// the trajectory streams from HBM at a small fraction of its bandwidth.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kRowsPerThread = 4;
constexpr int kRowsPerBlock = kThreads * kRowsPerThread;

struct ResArgs {
    int64_t N, ell;
    int Nt, n_in, nbx;
    const int64_t* slice_ptr;
    const int32_t* slice_w;
    const int32_t* col;
    const double* vmu;    // chunk x ell: values of A(mu_p)
    const double* dt;     // Nt
    const double* u0;     // N or null
    const double* B;      // N x n_in
    const double* F;      // Nt x n_in row major
    const double* U;      // n_mu x Nt x N (this chunk)
    double* part;         // n_mu x Nt x nbx
};

__global__ void __launch_bounds__(kThreads) residual_kernel(ResArgs a) {
    const int bx = blockIdx.x, k = blockIdx.y, p = blockIdx.z;
    const double h = a.dt[k];
    const double* vp = a.vmu + (size_t)p * a.ell;
    const double* uk = a.U + ((size_t)p * a.Nt + k) * a.N;
    const double* um = k > 0 ? uk - a.N : a.u0;  // null: u^0 = 0
    double acc = 0.0;
    const int64_t r0 = (int64_t)bx * kRowsPerBlock + threadIdx.x;
#pragma unroll
    for (int t = 0; t < kRowsPerThread; ++t) {
        const int64_t row = r0 + (int64_t)t * kThreads;
        if (row < a.N) {
            const int64_t sl = row / kSlice;
            const int w = a.slice_w[sl];
            const int64_t base = a.slice_ptr[sl] + row % kSlice;
            double au = 0.0;
            for (int j = 0; j < w; ++j) {
                const int64_t e = base + (int64_t)j * kSlice;
                au = fma(vp[e], uk[a.col[e]], au);
            }
            double bf = 0.0;
            for (int s = 0; s < a.n_in; ++s) bf = fma(a.B[row + (size_t)s * a.N], a.F[(size_t)k * a.n_in + s], bf);
            const double r = uk[row] - (um ? um[row] : 0.0) - h * au - h * bf;
            acc = fma(r, r, acc);
        }
    }
    __shared__ double s_w[kThreads / 32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += s_w[w];
        a.part[((size_t)p * a.Nt + k) * a.nbx + bx] = s;
    }
}

// vmu[p ell + e] = sum_q theta[p, q] vals[q ell + e], q ascending
__global__ void combine_kernel(int64_t ell, int Q, int np, const double* __restrict__ theta,
                               const double* __restrict__ vals, double* vmu) {
    const int64_t tot = ell * np;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = t / ell, e = t - p * ell;
        double v = 0.0;
        for (int q = 0; q < Q; ++q) v = fma(theta[p * Q + q], vals[(size_t)q * ell + e], v);
        vmu[t] = v;
    }
}

// rnorm[t] = sqrt(sum over the row blocks of part[t], in order)
__global__ void residual_norm_kernel(int64_t n, int nbx, const double* __restrict__ part, double* rnorm) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nbx; ++b) s += part[t * nbx + b];
        rnorm[t] = sqrt(s);
    }
}

}  // namespace

extern "C" st_status st_rom_residual_norms(st_model* m, int32_t n_mu, const double* theta, int32_t Nt,
                                           const double* dt, const double* u0, int32_t n_in,
                                           const double* B, const double* F, const double* U,
                                           double* rnorm) {
    if (!m) return st_fail(ST_ERR_ARG, "st_rom_residual_norms: NULL model");
    if (n_mu < 0 || Nt < 1 || Nt > 65535 || n_in < 0 || !dt || (n_mu > 0 && (!theta || !U || !rnorm)) ||
        (n_in > 0 && (!B || !F)))
        return st_fail(ST_ERR_ARG, "st_rom_residual_norms: bad arguments");
    for (int k = 0; k < Nt; ++k)
        if (!(dt[k] > 0)) return st_fail(ST_ERR_ARG, "st_rom_residual_norms: dt must be positive");
    if (n_mu == 0) return ST_OK;
    const int64_t N = m->N;
    const int Q = m->Q;
    const int nbx = (int)((N + kRowsPerBlock - 1) / kRowsPerBlock);
    const int64_t ell = m->ell_size;
    // samples per pass: their combined values within 256 MiB, at most 65535 (grid z)
    const int64_t by_mem = std::max<int64_t>(1, ((int64_t)256 << 20) / (8 * std::max<int64_t>(ell, 1)));
    const int chunk = (int)std::min<int64_t>(std::min<int64_t>(n_mu, 65535), by_mem);
    cudaStream_t st = m->stream;
    // workspace: dt [Nt] | F [Nt x n_in] | theta [n_mu x Q] | values [chunk x ell] |
    //            partial sums [chunk x Nt x nbx]
    const size_t szF = (size_t)Nt * std::max(n_in, 1), szT = (size_t)n_mu * Q;
    const size_t szV = (size_t)chunk * ell, szP = (size_t)chunk * Nt * nbx;
    ST_TRY(st_grow(m, m->ws_misc, sizeof(double) * (Nt + szF + szT + szV + szP + 16)));
    double* d_dt = (double*)m->ws_misc.p;
    double* d_F = d_dt + Nt;
    double* d_th = d_F + szF;
    double* vmu = d_th + szT;
    double* part = vmu + szV;
    ST_CUDA_TRY(cudaMemcpyAsync(d_dt, dt, sizeof(double) * Nt, cudaMemcpyHostToDevice, st));
    if (n_in > 0) ST_CUDA_TRY(cudaMemcpyAsync(d_F, F, sizeof(double) * Nt * n_in, cudaMemcpyHostToDevice, st));
    ST_CUDA_TRY(cudaMemcpyAsync(d_th, theta, sizeof(double) * szT, cudaMemcpyHostToDevice, st));
    ST_PROF(m, "residual_kernels");
    for (int p0 = 0; p0 < n_mu; p0 += chunk) {
        const int np = std::min(chunk, n_mu - p0);
        const int gc = (int)std::max<int64_t>(1, std::min<int64_t>((ell * np + 255) / 256, 8 * m->num_sms));
        combine_kernel<<<gc, 256, 0, st>>>(ell, Q, np, d_th + (size_t)p0 * Q, m->d_vals, vmu);
        ST_TRY(st_check_launch("residual combine"));
        ResArgs a{N,  ell, Nt, n_in, nbx, m->d_slice_ptr, m->d_slice_w, m->d_col, vmu,
                  d_dt, u0, B, d_F, U + (size_t)p0 * Nt * N, part};
        residual_kernel<<<dim3((unsigned)nbx, (unsigned)Nt, (unsigned)np), kThreads, 0, st>>>(a);
        ST_TRY(st_check_launch("residual"));
        const int64_t n = (int64_t)np * Nt;
        const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4 * m->num_sms));
        residual_norm_kernel<<<gb, 256, 0, st>>>(n, nbx, part, rnorm + (size_t)p0 * Nt);
        ST_TRY(st_check_launch("residual norm"));
    }
    return ST_OK;
}
