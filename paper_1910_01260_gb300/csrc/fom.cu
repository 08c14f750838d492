// Full-order snapshot march (Eq. fom): backward Euler, one linear solve per
// step, (I - dt_k A(mu)) u^k = u^{k-1} + dt_k B f^k, by BiCGSTAB on the
// sliced-ELL operator, for up to 32 parameter samples at once.
//
// Design (GB300): one cooperative persistent kernel runs the whole march
// (all Nt steps, every BiCGSTAB iteration) with all iteration control on the
// device -- no host round trip per iteration or step.  The samples share
// the sparsity pattern.  The operator is read in its term-split form: an
// entry where only term q of A(mu) = sum_q theta_q A_q is nonzero keeps one
// value for all samples and its row sum is scaled by theta_q once; only the
// entries where several terms overlap (the diagonal, for transport) carry
// per-sample values, interleaved per entry ([entry][sample]).  The operator
// thus stays a few MB and the whole march (operator + 7 Krylov vectors)
// stays resident in L2.  Every vector is [row][sample]: one gathered column
// index serves all samples and each thread moves two samples per 128-bit
// load.  Dot products reduce
// warp -> block -> per-block partials -> fixed-order sums done redundantly
// by every block after a bounded grid barrier, so all blocks take the same
// branch decisions and results are deterministic.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace {

// One CTA of 512 threads per SM: the same warps per SM as two CTAs of 256,
// with half the arrivals at every grid barrier and half the block partials
// in every fixed-order reduction (measured on the c4 march: 127 -> 97 ms).
constexpr int NT = 512;
constexpr int NSLOT = 2;
// Initial iterate of step k: the polynomial of degree kPred through the last
// kPred + 1 levels, evaluated one step ahead,
//   x0 = sum_{i=0}^{o} (-1)^i C(o+1, i+1) u^{k-i},  o = min(k, kPred),
// which only shortens the Krylov iteration (the stopping test is on the true
// system).
#ifndef ST_FOM_PRED_ORDER
#define ST_FOM_PRED_ORDER 4
#endif
constexpr int kPred = ST_FOM_PRED_ORDER;
constexpr int kHist = kPred + 1;  // levels kept
#ifndef ST_FOM_BLOCKS_PER_SM
#define ST_FOM_BLOCKS_PER_SM 1
#endif

// per-sample control states
enum : int { S_ACTIVE = 0, S_CONV = 1, S_FAILED = 2, S_PAD = 3, S_CONV_S = 4, S_ZERO = 5 };

struct FomArgs {
    int64_t N;
    int Q;
    const double* theta;      // [n_mu x Q] affine coefficients of the group
    const int64_t* mx_ptr;    // mixed entries (several nonzero terms)
    const int32_t* mx_w;
    const int32_t* mx_col;
    const double* amu;        // [mx_size * LD] their per-sample values
    const int64_t* tq_ptr;    // entries of a single term q
    const int32_t* tq_w;
    const int32_t* tq_col;
    const double* tq_val;
    int Nt;
    const double* dt;  // [Nt]
    int n_in;
    const double* B;  // [N x n_in]
    const double* F;  // [Nt x n_in]
    double *x, *r, *rh, *p, *v, *s, *t;  // [N * LD]
    double* hist;                        // [kHist x N * LD] solutions of the last kHist levels
    double* partial;                     // [2 x grid * NSLOT * LD]
    double* snap;
    int n_mu;
    int32_t* iters;
    int32_t* status;
    double tol;
    int maxit;
    GridBarrier bar;
};

template <int LD>
struct Cfg {
    static constexpr int VEC = LD >= 2 ? 2 : 1;
    static constexpr int LPR = LD / VEC;  // threads per row
    static constexpr int RPB = NT / LPR;  // rows per block pass
    static constexpr int NW = NT / 32;
};

template <int VEC>
__device__ __forceinline__ void ld_vec(const double* p, double (&o)[VEC]) {
    if constexpr (VEC == 2) {
        double2 t = __ldcg(reinterpret_cast<const double2*>(p));
        o[0] = t.x;
        o[1] = t.y;
    } else {
        o[0] = __ldcg(p);
    }
}
template <int VEC>
__device__ __forceinline__ void ld_vec_ro(const double* p, double (&o)[VEC]) {
    if constexpr (VEC == 2) {
        double2 t = __ldg(reinterpret_cast<const double2*>(p));
        o[0] = t.x;
        o[1] = t.y;
    } else {
        o[0] = __ldg(p);
    }
}
template <int VEC>
__device__ __forceinline__ void st_vec(double* p, const double (&o)[VEC]) {
    if constexpr (VEC == 2) {
        __stcg(reinterpret_cast<double2*>(p), make_double2(o[0], o[1]));
    } else {
        __stcg(p, o[0]);
    }
}

// acc = (A(mu) X)[row] for this thread's samples, A(mu) = sum_q theta_q A_q:
// the mixed entries carry per-sample values; the entries of a single term q
// share one value and their row sum is scaled by theta_q(mu) once, so the
// operator read per product is one value per entry, not one per sample.
template <int LD>
__device__ __forceinline__ void spmv_A(const FomArgs& a, int64_t row, int p0, const double* X,
                                       const double (*s_theta)[LD], double (&acc)[Cfg<LD>::VEC]) {
    constexpr int VEC = Cfg<LD>::VEC;
    const int64_t sl = row / kSlice;
    const int lane = (int)(row % kSlice);
#pragma unroll
    for (int u = 0; u < VEC; ++u) acc[u] = 0.0;
    {
        const int w = __ldg(a.mx_w + sl);
        const int64_t base = __ldg(a.mx_ptr + sl) + lane;
        for (int k = 0; k < w; ++k) {
            const int64_t e = base + (int64_t)k * kSlice;
            const int c = __ldg(a.mx_col + e);
            double av[VEC], xv[VEC];
            ld_vec_ro<VEC>(a.amu + e * LD + p0, av);
            ld_vec<VEC>(X + (int64_t)c * LD + p0, xv);
#pragma unroll
            for (int u = 0; u < VEC; ++u) acc[u] = fma(av[u], xv[u], acc[u]);
        }
    }
    for (int q = 0; q < a.Q; ++q) {
        const int64_t i = sl * a.Q + q;
        const int w = __ldg(a.tq_w + i);
        if (w == 0) continue;
        const int64_t base = __ldg(a.tq_ptr + i) + lane;
        double sq[VEC];
#pragma unroll
        for (int u = 0; u < VEC; ++u) sq[u] = 0.0;
        for (int k = 0; k < w; ++k) {
            const int64_t e = base + (int64_t)k * kSlice;
            const int c = __ldg(a.tq_col + e);
            const double v = __ldg(a.tq_val + e);
            double xv[VEC];
            ld_vec<VEC>(X + (int64_t)c * LD + p0, xv);
#pragma unroll
            for (int u = 0; u < VEC; ++u) sq[u] = fma(v, xv[u], sq[u]);
        }
#pragma unroll
        for (int u = 0; u < VEC; ++u) acc[u] = fma(s_theta[q][p0 + u], sq[u], acc[u]);
    }
}

// Reduce per-thread contributions (NS slots x VEC samples) to this block's
// partial sums.
template <int LD, int NS>
__device__ __forceinline__ void block_partial(double (&c)[NS][Cfg<LD>::VEC], double* partial,
                                              double (*s_warp)[NSLOT][LD]) {
    constexpr int VEC = Cfg<LD>::VEC, LPR = Cfg<LD>::LPR, NW = Cfg<LD>::NW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int sl = 0; sl < NS; ++sl)
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
            double x = c[sl][u];
#pragma unroll
            for (int o = LPR; o < 32; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane < LPR) s_warp[warp][sl][lane * VEC + u] = x;
        }
    __syncthreads();
    if (threadIdx.x < NS * LD) {
        const int sl = threadIdx.x / LD, p = threadIdx.x % LD;
        double acc = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) acc += s_warp[w][sl][p];
        __stcg(partial + ((int64_t)blockIdx.x * NS + sl) * LD + p, acc);
    }
}

// Fixed-order sum of all blocks' partials (run by every block).
template <int LD, int NS>
__device__ __forceinline__ void grid_reduce(const double* partial, double (*s_red)[LD]) {
    constexpr int NW = Cfg<LD>::NW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = warp; q < NS * LD; q += NW) {
        const int sl = q / LD, p = q % LD;
        double acc = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32)
            acc += __ldcg(partial + ((int64_t)b * NS + sl) * LD + p);
        acc = warp_sum(acc);
        if (lane == 0) s_red[sl][p] = acc;
    }
    __syncthreads();
}

template <int LD>
__global__ void __launch_bounds__(NT, ST_FOM_BLOCKS_PER_SM) fom_march_kernel(FomArgs a) {
    using C = Cfg<LD>;
    constexpr int VEC = C::VEC, LPR = C::LPR, RPB = C::RPB, NW = C::NW;
    __shared__ double s_warp[NW][NSLOT][LD];
    __shared__ double s_red[NSLOT][LD];
    __shared__ double s_rho[LD], s_rho_old[LD], s_alpha[LD], s_omega[LD], s_beta[LD], s_bnorm[LD];
    __shared__ int s_state[LD], s_it[LD], s_code[LD];
    __shared__ int s_any, s_flag;
    __shared__ double s_theta[16][LD];

    const int lr = threadIdx.x % LPR;
    const int rb = threadIdx.x / LPR;
    const int p0 = lr * VEC;
    const int64_t N = a.N;
    const int64_t nchunks = (N + RPB - 1) / RPB;

    if (threadIdx.x < LD) {
        s_state[threadIdx.x] = threadIdx.x < a.n_mu ? S_ACTIVE : S_PAD;
        s_code[threadIdx.x] = ST_OK;
    }
    for (int i = threadIdx.x; i < a.Q * LD; i += NT) {
        const int q = i / LD, p = i % LD;
        s_theta[q][p] = p < a.n_mu ? a.theta[(int64_t)p * a.Q + q] : 0.0;
    }
    __syncthreads();
    // The per-block partial sums alternate between two buffers: a block may
    // write the next reduction's partials while a slower block is still
    // summing the previous ones; a buffer is rewritten only two barriers
    // after it was read.
    int red = 0;
    const size_t part_stride = (size_t)gridDim.x * NSLOT * LD;
#define PART (a.partial + (size_t)(red & 1) * part_stride)

#define ROWS_BEGIN                                                                    \
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {                   \
        const int64_t row = ch * RPB + rb;                                            \
        if (row >= N) continue;                                                       \
        const int64_t vi = row * LD + p0;
#define ROWS_END }

    const size_t vecsz = (size_t)N * LD;
    // level 0 (u0) into the history, on this block's rows
    ROWS_BEGIN
        double xv[VEC];
        ld_vec<VEC>(a.x + vi, xv);
        st_vec<VEC>(a.hist + vi, xv);
    ROWS_END
    for (int k = 0; k < a.Nt; ++k) {
        const double h = a.dt[k];
        const double* uk = a.hist + (size_t)(k % kHist) * vecsz;  // the previous level u^k
        // ---- Phase X0: initial iterate by extrapolating the last levels in time
        if (k > 0) {
            const int o = min(k, kPred);
            double coef[kPred + 1];  // (-1)^i C(o+1, i+1)
            {
                double bin = 1.0;  // C(o+1, i) as i grows
#pragma unroll
                for (int i = 0; i <= kPred; ++i) {
                    bin = bin * (double)(o + 1 - i) / (double)(i + 1);  // C(o+1, i+1)
                    coef[i] = i <= o ? ((i & 1) ? -bin : bin) : 0.0;
                }
            }
            ROWS_BEGIN
                double x0[VEC];
#pragma unroll
                for (int u = 0; u < VEC; ++u) x0[u] = 0.0;
#pragma unroll
                for (int i = 0; i <= kPred; ++i) {
                    if (i > o) break;
                    double ui[VEC];
                    ld_vec<VEC>(a.hist + (size_t)((k - i + kHist * kPred) % kHist) * vecsz + vi, ui);
#pragma unroll
                    for (int u = 0; u < VEC; ++u) x0[u] = fma(coef[i], ui[u], x0[u]);
                }
                st_vec<VEC>(a.x + vi, x0);
            ROWS_END
            if (!grid_sync(a.bar, &s_flag)) return;
        }
        // ---- Phase R: b = u^k + h B f^k, r = b - K x0 = b - x0 + h A x0, r^ = r
        {
            double c[NSLOT][VEC];
#pragma unroll
            for (int u = 0; u < VEC; ++u) c[0][u] = c[1][u] = 0.0;
            ROWS_BEGIN
                double bf = 0.0;
                for (int s = 0; s < a.n_in; ++s) bf = fma(__ldg(a.B + row + (int64_t)s * N), __ldg(a.F + (int64_t)k * a.n_in + s), bf);
                double Au[VEC], xv[VEC], ukv[VEC];
                spmv_A<LD>(a, row, p0, a.x, s_theta, Au);
                ld_vec<VEC>(a.x + vi, xv);
                ld_vec<VEC>(uk + vi, ukv);
                double rr[VEC], zero[VEC];
#pragma unroll
                for (int u = 0; u < VEC; ++u) {
                    const bool on = s_state[p0 + u] != S_FAILED && s_state[p0 + u] != S_PAD;
                    const double b = fma(h, bf, ukv[u]);
                    rr[u] = on ? fma(h, Au[u], b - xv[u]) : 0.0;
                    zero[u] = 0.0;
                    if (on) {
                        c[0][u] = fma(b, b, c[0][u]);
                        c[1][u] = fma(rr[u], rr[u], c[1][u]);
                    }
                }
                st_vec<VEC>(a.r + vi, rr);
                st_vec<VEC>(a.rh + vi, rr);
                st_vec<VEC>(a.p + vi, zero);
                st_vec<VEC>(a.v + vi, zero);
            ROWS_END
            block_partial<LD, 2>(c, PART, s_warp);
        }
        if (!grid_sync(a.bar, &s_flag)) return;
        grid_reduce<LD, 2>(PART, s_red);
        ++red;
        if (threadIdx.x < LD) {
            const int p = threadIdx.x;
            s_it[p] = 0;
            if (s_state[p] != S_FAILED && s_state[p] != S_PAD) {
                const double bn = sqrt(s_red[0][p]), rn2 = s_red[1][p];
                s_bnorm[p] = bn;
                s_rho[p] = rn2;
                s_rho_old[p] = s_alpha[p] = s_omega[p] = 1.0;
                if (!isfinite(bn) || !isfinite(rn2)) {
                    s_state[p] = S_FAILED;
                    s_code[p] = ST_ERR_NONFINITE;
                } else if (bn == 0.0) {
                    s_state[p] = S_ZERO;
                } else if (sqrt(rn2) <= a.tol * bn) {
                    s_state[p] = S_CONV;
                } else {
                    s_state[p] = S_ACTIVE;
                }
            }
        }
        __syncthreads();

        for (int it = 0;; ++it) {
            if (threadIdx.x == 0) {
                int any = 0;
                for (int p = 0; p < LD; ++p) any |= (s_state[p] == S_ACTIVE);
                s_any = any;
            }
            __syncthreads();
            if (!s_any) break;
            if (it >= a.maxit) {
                if (threadIdx.x < LD && s_state[threadIdx.x] == S_ACTIVE) {
                    s_state[threadIdx.x] = S_FAILED;
                    s_code[threadIdx.x] = ST_ERR_NOT_CONVERGED;
                }
                __syncthreads();
                break;
            }
            if (threadIdx.x < LD) {
                const int p = threadIdx.x;
                if (s_state[p] == S_ACTIVE) {
                    s_beta[p] = (s_rho[p] / s_rho_old[p]) * (s_alpha[p] / s_omega[p]);
                    s_it[p] += 1;
                }
            }
            __syncthreads();
            // ---- Phase P: p = r + beta (p - omega v)
            ROWS_BEGIN
                double rv[VEC], pv[VEC], vv[VEC];
                ld_vec<VEC>(a.r + vi, rv);
                ld_vec<VEC>(a.p + vi, pv);
                ld_vec<VEC>(a.v + vi, vv);
#pragma unroll
                for (int u = 0; u < VEC; ++u)
                    if (s_state[p0 + u] == S_ACTIVE)
                        pv[u] = fma(s_beta[p0 + u], fma(-s_omega[p0 + u], vv[u], pv[u]), rv[u]);
                st_vec<VEC>(a.p + vi, pv);
            ROWS_END
            if (!grid_sync(a.bar, &s_flag)) return;
            // ---- Phase S1: v = K p, (r^, v)
            {
                double c[1][VEC];
#pragma unroll
                for (int u = 0; u < VEC; ++u) c[0][u] = 0.0;
                ROWS_BEGIN
                    double Ap[VEC], pv[VEC], rhv[VEC], vv[VEC];
                    spmv_A<LD>(a, row, p0, a.p, s_theta, Ap);
                    ld_vec<VEC>(a.p + vi, pv);
                    ld_vec<VEC>(a.rh + vi, rhv);
                    ld_vec<VEC>(a.v + vi, vv);
#pragma unroll
                    for (int u = 0; u < VEC; ++u)
                        if (s_state[p0 + u] == S_ACTIVE) {
                            vv[u] = fma(-h, Ap[u], pv[u]);
                            c[0][u] = fma(rhv[u], vv[u], c[0][u]);
                        }
                    st_vec<VEC>(a.v + vi, vv);
                ROWS_END
                block_partial<LD, 1>(c, PART, s_warp);
            }
            if (!grid_sync(a.bar, &s_flag)) return;
            grid_reduce<LD, 1>(PART, s_red);
            ++red;
            if (threadIdx.x < LD) {
                const int p = threadIdx.x;
                if (s_state[p] == S_ACTIVE) {
                    const double d = s_red[0][p];
                    if (!isfinite(d)) {
                        s_state[p] = S_FAILED;
                        s_code[p] = ST_ERR_NONFINITE;
                    } else if (d == 0.0) {
                        s_state[p] = S_FAILED;
                        s_code[p] = ST_ERR_BREAKDOWN;
                    } else {
                        s_alpha[p] = s_rho[p] / d;
                    }
                }
            }
            __syncthreads();
            // ---- Phase S2: s = r - alpha v, ||s||^2
            {
                double c[1][VEC];
#pragma unroll
                for (int u = 0; u < VEC; ++u) c[0][u] = 0.0;
                ROWS_BEGIN
                    double rv[VEC], vv[VEC], sv[VEC];
                    ld_vec<VEC>(a.r + vi, rv);
                    ld_vec<VEC>(a.v + vi, vv);
                    ld_vec<VEC>(a.s + vi, sv);
#pragma unroll
                    for (int u = 0; u < VEC; ++u)
                        if (s_state[p0 + u] == S_ACTIVE) {
                            sv[u] = fma(-s_alpha[p0 + u], vv[u], rv[u]);
                            c[0][u] = fma(sv[u], sv[u], c[0][u]);
                        }
                    st_vec<VEC>(a.s + vi, sv);
                ROWS_END
                block_partial<LD, 1>(c, PART, s_warp);
            }
            if (!grid_sync(a.bar, &s_flag)) return;
            grid_reduce<LD, 1>(PART, s_red);
            ++red;
            if (threadIdx.x < LD) {
                const int p = threadIdx.x;
                if (s_state[p] == S_ACTIVE) {
                    const double sn = sqrt(s_red[0][p]);
                    if (!isfinite(sn)) {
                        s_state[p] = S_FAILED;
                        s_code[p] = ST_ERR_NONFINITE;
                    } else if (sn <= a.tol * s_bnorm[p]) {
                        s_state[p] = S_CONV_S;
                    }
                }
            }
            __syncthreads();
            // ---- Phase S3: t = K s, (t, s), (t, t); early exit x += alpha p
            {
                double c[NSLOT][VEC];
#pragma unroll
                for (int u = 0; u < VEC; ++u) c[0][u] = c[1][u] = 0.0;
                ROWS_BEGIN
                    double As[VEC], sv[VEC], tv[VEC], xv[VEC], pv[VEC];
                    spmv_A<LD>(a, row, p0, a.s, s_theta, As);
                    ld_vec<VEC>(a.s + vi, sv);
                    ld_vec<VEC>(a.t + vi, tv);
                    ld_vec<VEC>(a.x + vi, xv);
                    ld_vec<VEC>(a.p + vi, pv);
#pragma unroll
                    for (int u = 0; u < VEC; ++u) {
                        const int st = s_state[p0 + u];
                        if (st == S_ACTIVE) {
                            tv[u] = fma(-h, As[u], sv[u]);
                            c[0][u] = fma(tv[u], sv[u], c[0][u]);
                            c[1][u] = fma(tv[u], tv[u], c[1][u]);
                        } else if (st == S_CONV_S) {
                            xv[u] = fma(s_alpha[p0 + u], pv[u], xv[u]);
                        }
                    }
                    st_vec<VEC>(a.t + vi, tv);
                    st_vec<VEC>(a.x + vi, xv);
                ROWS_END
                block_partial<LD, 2>(c, PART, s_warp);
            }
            if (!grid_sync(a.bar, &s_flag)) return;
            grid_reduce<LD, 2>(PART, s_red);
            ++red;
            if (threadIdx.x < LD) {
                const int p = threadIdx.x;
                if (s_state[p] == S_CONV_S) {
                    s_state[p] = S_CONV;
                } else if (s_state[p] == S_ACTIVE) {
                    const double ts = s_red[0][p], tt = s_red[1][p];
                    if (!isfinite(ts) || !isfinite(tt)) {
                        s_state[p] = S_FAILED;
                        s_code[p] = ST_ERR_NONFINITE;
                    } else if (tt == 0.0) {
                        s_state[p] = S_FAILED;
                        s_code[p] = ST_ERR_BREAKDOWN;
                    } else {
                        s_omega[p] = ts / tt;
                    }
                }
            }
            __syncthreads();
            // ---- Phase E: x += alpha p + omega s, r = s - omega t, (r^, r), (r, r)
            {
                double c[NSLOT][VEC];
#pragma unroll
                for (int u = 0; u < VEC; ++u) c[0][u] = c[1][u] = 0.0;
                ROWS_BEGIN
                    double xv[VEC], pv[VEC], sv[VEC], tv[VEC], rv[VEC], rhv[VEC];
                    ld_vec<VEC>(a.x + vi, xv);
                    ld_vec<VEC>(a.p + vi, pv);
                    ld_vec<VEC>(a.s + vi, sv);
                    ld_vec<VEC>(a.t + vi, tv);
                    ld_vec<VEC>(a.r + vi, rv);
                    ld_vec<VEC>(a.rh + vi, rhv);
#pragma unroll
                    for (int u = 0; u < VEC; ++u)
                        if (s_state[p0 + u] == S_ACTIVE) {
                            const double al = s_alpha[p0 + u], om = s_omega[p0 + u];
                            xv[u] = fma(om, sv[u], fma(al, pv[u], xv[u]));
                            rv[u] = fma(-om, tv[u], sv[u]);
                            c[0][u] = fma(rhv[u], rv[u], c[0][u]);
                            c[1][u] = fma(rv[u], rv[u], c[1][u]);
                        }
                    st_vec<VEC>(a.x + vi, xv);
                    st_vec<VEC>(a.r + vi, rv);
                ROWS_END
                block_partial<LD, 2>(c, PART, s_warp);
            }
            if (!grid_sync(a.bar, &s_flag)) return;
            grid_reduce<LD, 2>(PART, s_red);
            ++red;
            if (threadIdx.x < LD) {
                const int p = threadIdx.x;
                if (s_state[p] == S_ACTIVE) {
                    const double rho_new = s_red[0][p], rn = sqrt(s_red[1][p]);
                    s_rho_old[p] = s_rho[p];
                    s_rho[p] = rho_new;
                    if (!isfinite(rho_new) || !isfinite(rn)) {
                        s_state[p] = S_FAILED;
                        s_code[p] = ST_ERR_NONFINITE;
                    } else if (rn <= a.tol * s_bnorm[p]) {
                        s_state[p] = S_CONV;
                    } else if (fabs(s_omega[p]) < 1e-300 || fabs(rho_new) < 1e-300) {
                        s_state[p] = S_FAILED;
                        s_code[p] = ST_ERR_BREAKDOWN;
                    }
                }
            }
            __syncthreads();
        }
        // ---- Phase W: emit snapshot column k, zero solutions, bookkeeping
        ROWS_BEGIN
            double xv[VEC];
            ld_vec<VEC>(a.x + vi, xv);
            bool changed = false;
#pragma unroll
            for (int u = 0; u < VEC; ++u) {
                const int p = p0 + u;
                const int st = s_state[p];
                if (st == S_ZERO || st == S_FAILED) {
                    if (xv[u] != 0.0) changed = true;
                    xv[u] = 0.0;
                }
                if (p < a.n_mu) __stcs(a.snap + ((int64_t)p * a.Nt + k) * N + row, xv[u]);
            }
            if (changed) st_vec<VEC>(a.x + vi, xv);
            st_vec<VEC>(a.hist + (size_t)((k + 1) % kHist) * vecsz + vi, xv);
        ROWS_END
        if (blockIdx.x == 0 && threadIdx.x < a.n_mu) {
            const int p = threadIdx.x;
            if (a.iters) a.iters[(int64_t)k * a.n_mu + p] = s_it[p];
        }
        if (!grid_sync(a.bar, &s_flag)) return;
        if (threadIdx.x < LD && s_state[threadIdx.x] == S_ZERO) s_state[threadIdx.x] = S_CONV;
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x < a.n_mu) {
        const int p = threadIdx.x;
        if (a.status) a.status[p] = s_code[p];
        if (s_code[p] != ST_OK) st_dev_error(a.bar.err, s_code[p]);
    }
#undef ROWS_BEGIN
#undef ROWS_END
#undef PART
}

// amu[e * LD + p] = sum_q theta[p][q] vals[q][src[e]] for the mixed entries
// (zero for padding entries and samples); x = u0 (or 0) for every sample.
template <int LD>
__global__ void fom_setup_kernel(int64_t mx, const int64_t* __restrict__ src, int64_t ell, int Q,
                                 const double* __restrict__ vals, const double* __restrict__ theta,
                                 int n_mu, double* amu, int64_t N, const double* u0, double* x) {
    const int64_t tot = mx * LD;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i / LD;
        const int p = (int)(i % LD);
        const int64_t se = src[e];
        double s = 0.0;
        if (p < n_mu && se >= 0)
            for (int q = 0; q < Q; ++q) s = fma(theta[p * Q + q], vals[(int64_t)q * ell + se], s);
        amu[i] = s;
    }
    const int64_t totx = N * LD;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < totx;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(i % LD);
        x[i] = (u0 && p < n_mu) ? u0[i / LD] : 0.0;
    }
}

template <int LD>
st_status run_group(st_model* m, int n_mu, const double* d_theta, int Nt, const double* d_dt,
                    const double* u0, int n_in, const double* B, const double* d_F, double* snap,
                    int32_t* iters, int32_t* status, int32_t* d_iters_tmp) {
    const int64_t N = m->N, ell = m->ell_size, mx = m->mx_size;
    const size_t vec = (size_t)N * LD;
    int blocks = st_coop_blocks(m, fom_march_kernel<LD>, NT, 0, ST_FOM_BLOCKS_PER_SM);
    if (blocks < 1) return st_fail(ST_ERR_CUDA, "fom: cooperative occupancy query failed");
    const int64_t rpb = Cfg<LD>::RPB;
    const int64_t nchunks = (N + rpb - 1) / rpb;
    if (blocks > nchunks) blocks = (int)std::max<int64_t>(1, nchunks);
    size_t need = sizeof(double) * ((size_t)mx * LD + (7 + kHist) * vec + 2 * (size_t)blocks * NSLOT * LD) + 1024;
    ST_TRY(st_grow(m, m->ws_fom, need));
    double* base = (double*)m->ws_fom.p;
    double* amu = base;
    double* vecs = amu + (size_t)mx * LD;
    double* partial = vecs + (7 + kHist) * vec;
    int sblocks = (int)std::min<int64_t>((std::max(mx, N) * LD + 255) / 256, 8 * m->num_sms);
    {
        ST_PROF(m, "fom_setup_kernel");
        fom_setup_kernel<LD><<<std::max(sblocks, 1), 256, 0, m->stream>>>(
            mx, m->d_mx_src, ell, m->Q, m->d_vals, d_theta, n_mu, amu, N, u0, vecs);
        ST_TRY(st_check_launch("fom_setup"));
    }
    ST_CUDA_TRY(cudaMemsetAsync(m->d_bar, 0, sizeof(unsigned int) * 4, m->stream));
    FomArgs a;
    a.N = N;
    a.Q = m->Q;
    a.theta = d_theta;
    a.mx_ptr = m->d_mx_ptr;
    a.mx_w = m->d_mx_w;
    a.mx_col = m->d_mx_col;
    a.amu = amu;
    a.tq_ptr = m->d_tq_ptr;
    a.tq_w = m->d_tq_w;
    a.tq_col = m->d_tq_col;
    a.tq_val = m->d_tq_val;
    a.Nt = Nt;
    a.dt = d_dt;
    a.n_in = n_in;
    a.B = B;
    a.F = d_F;
    a.x = vecs;
    a.r = vecs + vec;
    a.rh = vecs + 2 * vec;
    a.p = vecs + 3 * vec;
    a.v = vecs + 4 * vec;
    a.s = vecs + 5 * vec;
    a.t = vecs + 6 * vec;
    a.hist = vecs + 7 * vec;
    a.partial = partial;
    a.snap = snap;
    a.n_mu = n_mu;
    a.iters = iters ? d_iters_tmp : nullptr;
    a.status = status;
    a.tol = m->opt.tol;
    a.maxit = m->opt.maxit;
    a.bar = GridBarrier{m->d_bar, m->d_bar + 1, m->d_bar + 2, m->d_err, m->opt.spin_limit};
    void* args[] = {&a};
    ST_PROF(m, "fom_march_kernel");
    ST_CUDA_TRY(cudaLaunchCooperativeKernel((void*)fom_march_kernel<LD>, dim3(blocks), dim3(NT),
                                            args, 0, m->stream));
        st_count_launch();
    return ST_OK;
}

}  // namespace

extern "C" st_status st_fom_march(st_model* m, int32_t n_mu, const double* theta, int32_t Nt,
                                  const double* dt, const double* u0, int32_t n_in,
                                  const double* B, const double* F, double* snapshots,
                                  int32_t* iters, int32_t* status) {
    if (!m) return st_fail(ST_ERR_ARG, "st_fom_march: NULL model");
    if (n_mu < 1 || Nt < 1 || n_in < 0) return st_fail(ST_ERR_ARG, "st_fom_march: bad sizes");
    if (!theta || !dt || !snapshots) return st_fail(ST_ERR_ARG, "st_fom_march: NULL argument");
    if (n_in > 0 && (!B || !F)) return st_fail(ST_ERR_ARG, "st_fom_march: NULL B or F");
    for (int k = 0; k < Nt; ++k)
        if (!(dt[k] > 0) || !std::isfinite(dt[k])) return st_fail(ST_ERR_ARG, "st_fom_march: dt must be positive");
    const int Q = m->Q;
    // small host inputs -> device (theta, dt, F); iteration counts staged per group
    const size_t nF = (size_t)Nt * n_in;
    size_t bytes = sizeof(double) * ((size_t)n_mu * Q + Nt + nF) + sizeof(int32_t) * (size_t)Nt * 32 + 256;
    ST_TRY(st_grow(m, m->ws_misc, bytes));
    double* d_theta = (double*)m->ws_misc.p;
    double* d_dt = d_theta + (size_t)n_mu * Q;
    double* d_F = d_dt + Nt;
    int32_t* d_it = (int32_t*)(d_F + nF);
    ST_CUDA_TRY(cudaMemcpyAsync(d_theta, theta, sizeof(double) * n_mu * Q, cudaMemcpyHostToDevice, m->stream));
    ST_CUDA_TRY(cudaMemcpyAsync(d_dt, dt, sizeof(double) * Nt, cudaMemcpyHostToDevice, m->stream));
    if (nF) ST_CUDA_TRY(cudaMemcpyAsync(d_F, F, sizeof(double) * nF, cudaMemcpyHostToDevice, m->stream));
    for (int g0 = 0; g0 < n_mu; g0 += 32) {
        const int ng = std::min(32, n_mu - g0);
        int ld = 1;
        while (ld < ng) ld <<= 1;
        double* snap = snapshots + (size_t)g0 * Nt * m->N;
        int32_t* st = status ? status + g0 : nullptr;
        const double* th = d_theta + (size_t)g0 * Q;
        st_status rc;
        switch (ld) {
            case 1: rc = run_group<1>(m, ng, th, Nt, d_dt, u0, n_in, B, d_F, snap, iters, st, d_it); break;
            case 2: rc = run_group<2>(m, ng, th, Nt, d_dt, u0, n_in, B, d_F, snap, iters, st, d_it); break;
            case 4: rc = run_group<4>(m, ng, th, Nt, d_dt, u0, n_in, B, d_F, snap, iters, st, d_it); break;
            case 8: rc = run_group<8>(m, ng, th, Nt, d_dt, u0, n_in, B, d_F, snap, iters, st, d_it); break;
            case 16: rc = run_group<16>(m, ng, th, Nt, d_dt, u0, n_in, B, d_F, snap, iters, st, d_it); break;
            default: rc = run_group<32>(m, ng, th, Nt, d_dt, u0, n_in, B, d_F, snap, iters, st, d_it); break;
        }
        if (rc != ST_OK) return rc;
        if (iters) {
            // group counts [Nt x ng] -> caller layout [Nt x n_mu]
            ST_CUDA_TRY(cudaMemcpy2DAsync(iters + g0, sizeof(int32_t) * n_mu, d_it,
                                          sizeof(int32_t) * ng, sizeof(int32_t) * ng, Nt,
                                          cudaMemcpyDeviceToDevice, m->stream));
        }
    }
    return ST_OK;
}
