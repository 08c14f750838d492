// Stability constant of the space-time error bound (Theorem 3):
//   ||u^st - u~^st||_2 <= ||(A^st)^{-1}||_2 ||r^st(u~^st)||_2,
// with A^st the block lower bidiagonal space-time matrix of the full-order
// march (Eqs. st-fom, stsystemmat): diagonal blocks K_k = I - dt_k A(mu),
// sub-diagonal blocks -I.
//
// ||(A^st)^{-1}||_2 = 1 / sigma_min(A^st) is estimated by power iteration on
// (A^st)^{-T} (A^st)^{-1}, never forming A^st:
//   y = (A^st)^{-1} v   is the full-order march K_k y_k = y_{k-1} + v_k,
//                        y_0 = 0 (the march with a per-step source);
//   w = (A^st)^{-T} y   is K_k^T w_k = w_{k+1} + y_k backward in time, i.e.
//                        the forward march of the transposed terms A_q^T
//                        over the reversed steps and the reversed source;
//   v <- w / ||w||.
// With ||v|| = 1, ||y||^2 = v^T (A^st)^{-T} (A^st)^{-1} v <= ||w|| <=
// ||(A^st)^{-1}||_2^2, so sqrt(||w||) is a lower estimate that rises to the
// norm; the iteration stops when it changes by less than tol (relative) for
// every sample.  The transposed terms are built once from the model's host
// copy of the operator and kept in a second model.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace {

constexpr int NTC = 256;

__device__ __forceinline__ uint64_t splitmix(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// v[i] uniform in [-1, 1), counter-based in (seed, i)
__global__ void uniform_kernel(int64_t n, uint64_t seed, double* v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = 2.0 * ((double)(splitmix(seed ^ splitmix((uint64_t)i)) >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

// Fixed-order sums of squares of n_mu vectors of length len: block (c, p)
// sums its chunk of vector p; one thread per sample then adds the chunks in
// order.
__global__ void __launch_bounds__(NTC) sumsq_part_kernel(int64_t len, const double* __restrict__ x, int chunks,
                                                         double* part) {
    __shared__ double s[NTC / 32];
    const int p = blockIdx.y, c = blockIdx.x;
    const int64_t per = (len + chunks - 1) / chunks, b = c * per, e = min(len, b + per);
    const double* xp = x + (int64_t)p * len;
    double acc = 0.0;
    for (int64_t i = b + threadIdx.x; i < e; i += NTC) acc = fma(xp[i], xp[i], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < NTC / 32; ++w) t += s[w];
        part[(int64_t)p * chunks + c] = t;
    }
}

__global__ void sumsq_final_kernel(int n_mu, int chunks, const double* __restrict__ part, double* out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_mu) return;
    double t = 0.0;
    for (int c = 0; c < chunks; ++c) t += part[(int64_t)p * chunks + c];
    out[p] = t;
}

// y_p = x_p / sqrt(ss_p) (zero vectors stay zero)
__global__ void normalize_kernel(int64_t len, int n_mu, const double* __restrict__ x, const double* __restrict__ ss,
                                 double* y) {
    const int64_t tot = len * n_mu;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const double s = ss[i / len];
        y[i] = s > 0.0 ? x[i] / sqrt(s) : 0.0;
    }
}

// y[p][Nt-1-k][:] = x[p][k][:]
__global__ void reverse_steps_kernel(int n_mu, int Nt, int64_t N, const double* __restrict__ x, double* y) {
    const int64_t tot = (int64_t)n_mu * Nt * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i % N, pk = i / N;
        const int k = (int)(pk % Nt);
        const int64_t p = pk / Nt;
        y[(p * Nt + (Nt - 1 - k)) * N + row] = x[i];
    }
}

int grid_for(const st_model* m, int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + NTC - 1) / NTC, 8 * (int64_t)m->num_sms));
}

// The model of the transposed terms A_q^T (same options, grid march).
st_status build_adjoint(st_model* m) {
    st_options o = m->opt;
    o.fom_path = ST_FOM_GRID;
    if (m->adj) return st_model_set_options(m->adj, &o);
    const int64_t N = m->N, nnz = m->nnz;
    const int Q = m->Q;
    std::vector<int64_t> rp(N + 1, 0);
    for (int64_t e = 0; e < nnz; ++e) rp[m->h_col[e] + 1] += 1;
    for (int64_t i = 0; i < N; ++i) rp[i + 1] += rp[i];
    std::vector<int64_t> fill(rp.begin(), rp.end() - 1);
    std::vector<int32_t> col(nnz);
    std::vector<double> vals((size_t)Q * nnz);
    for (int64_t r = 0; r < N; ++r)
        for (int64_t e = m->h_rowptr[r]; e < m->h_rowptr[r + 1]; ++e) {
            const int64_t d = fill[m->h_col[e]]++;
            col[d] = (int32_t)r;
            for (int q = 0; q < Q; ++q) vals[(size_t)q * nnz + d] = m->h_vals[(size_t)q * nnz + e];
        }
    std::vector<const double*> vp(Q);
    for (int q = 0; q < Q; ++q) vp[q] = vals.data() + (size_t)q * nnz;
    st_affine_csr csr{N, rp.data(), col.data(), vp.data(), Q};
    return st_model_create(&csr, &o, m->stream, &m->adj);
}

}  // namespace

extern "C" st_status st_fom_st_inverse_norm(st_model* m, int32_t n_mu, const double* theta, int32_t Nt,
                                            const double* dt, int32_t max_iter, double tol, uint64_t seed,
                                            double* norm, int32_t* iters_used) {
    if (!m) return st_fail(ST_ERR_ARG, "st_fom_st_inverse_norm: NULL model");
    if (n_mu < 1 || n_mu > 32 || Nt < 1 || !theta || !dt || max_iter < 1 || !(tol >= 0) || !norm)
        return st_fail(ST_ERR_ARG, "st_fom_st_inverse_norm: bad arguments (1 <= n_mu <= 32)");
    for (int k = 0; k < Nt; ++k)
        if (!(dt[k] > 0) || !std::isfinite(dt[k]))
            return st_fail(ST_ERR_ARG, "st_fom_st_inverse_norm: dt must be positive");
    ST_TRY(build_adjoint(m));
    const int64_t N = m->N, len = (int64_t)Nt * N, tot = len * n_mu;
    const int chunks = (int)std::max<int64_t>(1, std::min<int64_t>(64, len / 4096));
    ST_TRY(st_grow(m, m->ws_cert, sizeof(double) * (3 * (size_t)tot + (size_t)n_mu * (chunks + 2)) + 256));
    double* V = (double*)m->ws_cert.p;
    double* Y = V + tot;
    double* Z = Y + tot;
    double* part = Z + tot;
    double* ss = part + (size_t)n_mu * chunks;
    cudaStream_t st = m->stream;
    std::vector<double> dt_rev(dt, dt + Nt);
    std::reverse(dt_rev.begin(), dt_rev.end());
    std::vector<double> h_ss(n_mu), prev(n_mu, 0.0);
    auto sumsq = [&](const double* x) -> st_status {
        sumsq_part_kernel<<<dim3(chunks, n_mu), NTC, 0, st>>>(len, x, chunks, part);
        ST_TRY(st_check_launch("sumsq_part"));
        sumsq_final_kernel<<<(n_mu + 31) / 32, 32, 0, st>>>(n_mu, chunks, part, ss);
        return st_check_launch("sumsq_final");
    };
    ST_PROF(m, "st_inverse_norm");
    // a seeded start vector of unit norm per sample
    uniform_kernel<<<grid_for(m, tot), NTC, 0, st>>>(tot, seed, Y);
    ST_TRY(st_check_launch("uniform"));
    ST_TRY(sumsq(Y));
    normalize_kernel<<<grid_for(m, tot), NTC, 0, st>>>(len, n_mu, Y, ss, V);
    ST_TRY(st_check_launch("normalize"));
    int it = 0;
    bool done = false;
    while (!done && it < max_iter) {
        ++it;
        // Y = (A^st)^{-1} V
        ST_TRY(st_internal_fom_march(m, n_mu, theta, Nt, dt, nullptr, 0, nullptr, nullptr, V, Y, nullptr,
                                     nullptr));
        // Z = reversed Y; V = reversed (A^st)^{-T} Y; Z = (A^st)^{-T} Y
        reverse_steps_kernel<<<grid_for(m, tot), NTC, 0, st>>>(n_mu, Nt, N, Y, Z);
        ST_TRY(st_check_launch("reverse"));
        ST_TRY(st_internal_fom_march(m->adj, n_mu, theta, Nt, dt_rev.data(), nullptr, 0, nullptr, nullptr, Z, V,
                                     nullptr, nullptr));
        reverse_steps_kernel<<<grid_for(m, tot), NTC, 0, st>>>(n_mu, Nt, N, V, Z);
        ST_TRY(st_check_launch("reverse"));
        ST_TRY(sumsq(Z));
        normalize_kernel<<<grid_for(m, tot), NTC, 0, st>>>(len, n_mu, Z, ss, V);
        ST_TRY(st_check_launch("normalize"));
        ST_CUDA_TRY(cudaMemcpyAsync(h_ss.data(), ss, sizeof(double) * n_mu, cudaMemcpyDeviceToHost, st));
        ST_TRY(st_sync(m));
        ST_TRY(st_sync(m->adj));
        done = true;
        for (int p = 0; p < n_mu; ++p) {
            const double est = std::sqrt(std::sqrt(h_ss[p]));  // sqrt(||w||)
            if (!std::isfinite(est))
                return st_fail(ST_ERR_NONFINITE, "st_fom_st_inverse_norm: non-finite estimate for sample %d", p);
            if (!(std::fabs(est - prev[p]) <= tol * est)) done = false;
            prev[p] = est;
        }
    }
    for (int p = 0; p < n_mu; ++p) norm[p] = prev[p];
    if (iters_used) *iters_used = it;
    return done ? ST_OK : st_fail(ST_ERR_NOT_CONVERGED, "st_fom_st_inverse_norm: %d iterations without reaching "
                                                       "the tolerance (the estimates are returned)", it);
}
