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
    const double* src;  // [n_mu x Nt x N] extra right-hand side z_k per step, or NULL
    double *x, *r, *rh, *p, *v, *s, *t;  // [N * LD]
    double* hist;                        // [kHist x N * LD] solutions of the last kHist levels
    double* partial;                     // [2 x grid * NSLOT * LD]
    double* snap;
    int n_mu;
    int32_t* iters;
    int32_t* status;
    double tol;
    int maxit;
    GridBarrier bar;  // counters of sub-grid 0; sub-grid s uses count/gen/abort + 4 s
    // sub-grids: CTAs [s * per, (s + 1) * per) march samples [s * per_sub, ...)
    // of the group, with workspace (amu, vectors, partials) at + s * sub_doubles
    int per, per_sub;
    int64_t sub_doubles;
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

// Reduce-scatter of V values per lane over the lanes of a warp that share
// (lane % LPR): at each of the log2(32 / LPR) shuffle levels (offsets 16, 8,
// ...) a lane keeps half of its values and adds its partner's copy of them,
// until one value is left, then plain butterflies follow.  A lane ends with
// the totals of values [base, base + KEEP) in x[0, KEEP); every lane whose
// plain-level bits are zero holds a distinct set.  It takes about V + log2(32
// / LPR) adds per lane instead of V log2(32 / LPR) for separate butterflies
// (an FP64 add costs a warp-instruction slot of the FP64 pipe).
template <int V, int LPR>
struct RsSum {
    static constexpr int LEVELS = LPR >= 32 ? 0 : (LPR >= 16 ? 1 : LPR >= 8 ? 2 : LPR >= 4 ? 3 : LPR >= 2 ? 4 : 5);
    static constexpr int LOGV = V >= 4 ? 2 : (V >= 2 ? 1 : 0);
    static constexpr int H = LOGV < LEVELS ? LOGV : LEVELS;  // halving levels
    static constexpr int KEEP = V >> H;
    static constexpr int PLAIN = LEVELS - H;
    __device__ __forceinline__ static int run(double (&x)[V], int lane) {
        int base = 0;
        int o = 16;
#pragma unroll
        for (int lev = 0; lev < H; ++lev, o >>= 1) {
            const int h = V >> (lev + 1);
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const double send = up ? x[i] : x[i + h];
                const double keep = up ? x[i + h] : x[i];
                x[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
            base += up ? h : 0;
        }
#pragma unroll
        for (int lev = 0; lev < PLAIN; ++lev, o >>= 1)
#pragma unroll
            for (int i = 0; i < KEEP; ++i) x[i] += __shfl_xor_sync(0xffffffffu, x[i], o);
        return base;
    }
    // whether this lane writes its totals (its plain-level bits are zero)
    __device__ __forceinline__ static bool writer(int lane) { return ((lane / LPR) & ((1 << PLAIN) - 1)) == 0; }
};

// Reduce per-thread contributions (NS slots x VEC samples) to this block's
// partial sums: a reduce-scatter in each warp, then a pairwise sum over the
// warps.
template <int LD, int NS>
__device__ __forceinline__ void block_partial(double (&c)[NS][Cfg<LD>::VEC], double* partial,
                                              double (*s_warp)[NSLOT][LD], int bid) {
    constexpr int VEC = Cfg<LD>::VEC, LPR = Cfg<LD>::LPR, NW = Cfg<LD>::NW;
    constexpr int V = NS * VEC;
    using RS = RsSum<V, LPR>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double x[V];
#pragma unroll
    for (int sl = 0; sl < NS; ++sl)
#pragma unroll
        for (int u = 0; u < VEC; ++u) x[sl * VEC + u] = c[sl][u];
    const int base = RS::run(x, lane);
    if (RS::writer(lane)) {
        const int lr = lane % LPR;
#pragma unroll
        for (int i = 0; i < RS::KEEP; ++i) {
            const int v = base + i;
            s_warp[warp][v / VEC][lr * VEC + v % VEC] = x[i];
        }
    }
    __syncthreads();
    if (threadIdx.x < NS * LD) {
        const int sl = threadIdx.x / LD, p = threadIdx.x % LD;
        double t[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) t[w] = s_warp[w][sl][p];
#pragma unroll
        for (int h = NW / 2; h > 0; h >>= 1)
#pragma unroll
            for (int w = 0; w < h; ++w) t[w] += t[w + h];
        __stcg(partial + ((int64_t)bid * NS + sl) * LD + p, t[0]);
    }
}

// Fixed-order sum of all blocks' partials (run by every block).
template <int LD, int NS>
__device__ __forceinline__ void grid_reduce(const double* partial, double (*s_red)[LD], int nblk) {
    constexpr int NW = Cfg<LD>::NW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = warp; q < NS * LD; q += NW) {
        const int sl = q / LD, p = q % LD;
        double acc = 0.0;
        for (int b = lane; b < nblk; b += 32)
            acc += __ldcg(partial + ((int64_t)b * NS + sl) * LD + p);
        acc = warp_sum(acc);
        if (lane == 0) s_red[sl][p] = acc;
    }
    __syncthreads();
}

// SRC: the right-hand side of step k also carries a per-sample vector z_k
// (a general source, as in the space-time system A^st u = z).
// One cooperative launch holds several independent sub-grids of `per` CTAs:
// sub-grid s marches its own samples with its own barrier counters and
// partials (fewer arrivals per barrier, fewer partials per reduction, and no
// lock step between the sub-grids' samples).  The sub-grid's view of the
// arguments is made once at entry.
constexpr int kMaxSub = 8;

template <int LD, bool SRC>
__global__ void __launch_bounds__(NT, ST_FOM_BLOCKS_PER_SM) fom_march_kernel(FomArgs A) {
    const int sub = blockIdx.x / A.per;
    const int bid = blockIdx.x - sub * A.per, nblk = A.per;
    FomArgs a = A;
    {
        const int p0 = sub * A.per_sub;
        const size_t off = (size_t)sub * A.sub_doubles;
        a.n_mu = min(A.per_sub, A.n_mu - p0);
        a.theta = A.theta + (size_t)p0 * A.Q;
        a.amu = A.amu + off;
        a.x = A.x + off;
        a.r = A.r + off;
        a.rh = A.rh + off;
        a.p = A.p + off;
        a.v = A.v + off;
        a.s = A.s + off;
        a.t = A.t + off;
        a.hist = A.hist + off;
        a.partial = A.partial + off;
        a.snap = A.snap + (size_t)p0 * A.Nt * A.N;
        a.src = A.src ? A.src + (size_t)p0 * A.Nt * A.N : nullptr;
        a.iters = A.iters ? A.iters + (size_t)A.Nt * p0 : nullptr;
        a.status = A.status ? A.status + p0 : nullptr;
        a.bar.count = A.bar.count + 4 * sub;
        a.bar.gen = A.bar.gen + 4 * sub;
        a.bar.abort = A.bar.abort + 4 * sub;
        a.bar.parties = (unsigned int)A.per;
    }
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
    // this CTA's rows: a contiguous, balanced share of the kSlice-row slices
    // (so a warp's rows stay in one slice), swept in passes of RPB rows.  A
    // round-robin deal of RPB-row chunks would give some CTAs a whole pass
    // more than others (96 chunks over 19 CTAs at N = 49152), and every
    // phase waits for the slowest CTA at its barrier.
    const int64_t nsl = (N + kSlice - 1) / kSlice;
    const int64_t row_lo = (nsl * bid / nblk) * kSlice;
    const int64_t row_hi = min(N, (nsl * (bid + 1) / nblk) * kSlice);

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
    const size_t part_stride = (size_t)nblk * NSLOT * LD;
#define PART (a.partial + (size_t)(red & 1) * part_stride)

#define ROWS_BEGIN                                                                    \
    for (int64_t row = row_lo + rb; row < row_hi; row += RPB) {                       \
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
        // (the initial iterate x0 of this step was formed by the previous
        // step's phase W from the levels it had just completed)
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
                    double b = fma(h, bf, ukv[u]);
                    if constexpr (SRC) {
                        if (p0 + u < a.n_mu) b += __ldg(a.src + ((int64_t)(p0 + u) * a.Nt + k) * N + row);
                    }
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
            block_partial<LD, 2>(c, PART, s_warp, bid);
        }
        if (!grid_sync(a.bar, &s_flag)) return;
        grid_reduce<LD, 2>(PART, s_red, nblk);
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
                block_partial<LD, 1>(c, PART, s_warp, bid);
            }
            if (!grid_sync(a.bar, &s_flag)) return;
            grid_reduce<LD, 1>(PART, s_red, nblk);
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
                block_partial<LD, 1>(c, PART, s_warp, bid);
            }
            if (!grid_sync(a.bar, &s_flag)) return;
            grid_reduce<LD, 1>(PART, s_red, nblk);
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
                block_partial<LD, 2>(c, PART, s_warp, bid);
            }
            if (!grid_sync(a.bar, &s_flag)) return;
            grid_reduce<LD, 2>(PART, s_red, nblk);
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
                block_partial<LD, 2>(c, PART, s_warp, bid);
            }
            if (!grid_sync(a.bar, &s_flag)) return;
            grid_reduce<LD, 2>(PART, s_red, nblk);
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
        // ---- Phase W: emit snapshot column k, zero solutions, bookkeeping,
        // and the next step's initial iterate by extrapolating the last
        // levels in time (a thread's own rows only: the barrier below orders
        // it before the next step's products)
        //   x0 = sum_{i=0}^{o} (-1)^i C(o+1, i+1) u^{k+1-i},  o = min(k+1, kPred)
        const bool extrap = k + 1 < a.Nt;
        const int o = min(k + 1, kPred);
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
            st_vec<VEC>(a.hist + (size_t)((k + 1) % kHist) * vecsz + vi, xv);
            if (extrap) {
                double x0[VEC];
#pragma unroll
                for (int u = 0; u < VEC; ++u) x0[u] = fma(coef[0], xv[u], 0.0);
#pragma unroll
                for (int i = 1; i <= kPred; ++i) {
                    if (i > o) break;
                    double ui[VEC];
                    ld_vec<VEC>(a.hist + (size_t)((k + 1 - i + kHist * kPred) % kHist) * vecsz + vi, ui);
#pragma unroll
                    for (int u = 0; u < VEC; ++u) x0[u] = fma(coef[i], ui[u], x0[u]);
                }
                st_vec<VEC>(a.x + vi, x0);
            } else if (changed) {
                st_vec<VEC>(a.x + vi, xv);
            }
        ROWS_END
        if (bid == 0 && threadIdx.x < a.n_mu) {
            const int p = threadIdx.x;
            if (a.iters) a.iters[(int64_t)k * a.n_mu + p] = s_it[p];
        }
        if (!grid_sync(a.bar, &s_flag)) return;
        if (threadIdx.x < LD && s_state[threadIdx.x] == S_ZERO) s_state[threadIdx.x] = S_CONV;
        __syncthreads();
    }
    if (bid == 0 && threadIdx.x < a.n_mu) {
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

// ---------------------------------------------------------------------------
// One thread-block cluster per parameter sample.
//
// The grid-wide march above keeps all samples in lock step and pays five
// grid barriers (atomics and L2 round trips over every SM) per BiCGSTAB
// iteration.  Here each sample gets its own cluster of CL CTAs (one 512-
// thread CTA per SM, co-scheduled by the hardware): CTA c owns a contiguous
// 1/CL of the sliced-ELL slices (one warp per slice, one row per lane).  The
// vectors only its own rows read -- r, r^, v, t -- live in its shared memory;
// p, s and x, which the products gather from every CTA, and the history
// levels live in global memory (L2).  Each synchronisation is a hardware
// cluster barrier with release/acquire semantics; a dot product is a CTA
// partial in shared memory that warp 0 of every CTA reads from all CL CTAs
// through distributed shared memory, in rank order, so every CTA forms the
// same sums and takes the same branches (no device-side wait can hang: the
// cluster's CTAs are resident together).  Samples march independently, each
// at its own iteration count.  The scalar recurrences run in one thread and
// are broadcast through shared memory.
constexpr int CT = 512;             // threads per CTA
constexpr int CW = CT / 32;         // warps per CTA
constexpr int kClVecs = 4;          // r, r^, v, t in shared memory
#ifndef ST_FOM_CLUSTER_CTAS
#define ST_FOM_CLUSTER_CTAS 8
#endif
constexpr int CL = ST_FOM_CLUSTER_CTAS;  // CTAs per cluster (one sample per cluster)
static_assert(CL >= 2 && CL <= 8, "portable cluster sizes only");

struct FomClArgs {
    int64_t N;
    int Q;
    const double* theta;  // [n_mu x Q]
    const int64_t* mx_ptr;
    const int32_t* mx_w;
    const int32_t* mx_col;
    const double* amu;  // [n_mu x mx_size] per-sample values of the mixed entries
    int64_t mx_size;
    const int64_t* tq_ptr;
    const int32_t* tq_w;
    const int32_t* tq_col;
    const double* tq_val;
    int64_t n_slices;
    int Nt;
    const double* dt;
    int n_in;
    const double* B;
    const double* F;
    double* vecs;  // per sample [x | p | s | hist_0 .. hist_{kHist-1}], N each
    double* snap;
    int n_mu;
    int32_t* iters;  // [Nt x n_mu] or NULL
    int32_t* status;
    int32_t* err;
    double tol;
    int maxit;
    int max_slices;  // most slices a CTA owns (shared-memory vector length / 32)
};

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

__device__ __forceinline__ unsigned int cluster_rank() {
    unsigned int r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// value of the shared-memory double at `p` (this CTA's address) in CTA `rank`
__device__ __forceinline__ double ld_dsmem(const double* p, unsigned int rank) {
    const unsigned int a = (unsigned int)__cvta_generic_to_shared(p);
    unsigned int ra;
    double v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(ra) : "memory");
    return v;
}

// (A(mu) X)[row] for the sample of this cluster: per-sample values on the
// mixed entries, shared values (scaled by theta_q per row) on single-term
// entries.  X is gathered from L2 (written by any CTA of the cluster).
__device__ __forceinline__ double spmv_row_cl(const FomClArgs& a, const double* amu_p, int64_t sl, int lane,
                                              const double* X, const double* s_theta) {
    double acc = 0.0;
    {
        const int w = __ldg(a.mx_w + sl);
        const int64_t base = __ldg(a.mx_ptr + sl) + lane;
        for (int k = 0; k < w; ++k) {
            const int64_t e = base + (int64_t)k * kSlice;
            acc = fma(__ldg(amu_p + e), __ldcg(X + __ldg(a.mx_col + e)), acc);
        }
    }
    for (int q = 0; q < a.Q; ++q) {
        const int64_t i = sl * a.Q + q;
        const int w = __ldg(a.tq_w + i);
        if (w == 0) continue;
        const int64_t base = __ldg(a.tq_ptr + i) + lane;
        double sq = 0.0;
#pragma unroll 4
        for (int k = 0; k < w; ++k) {
            const int64_t e = base + (int64_t)k * kSlice;
            sq = fma(__ldg(a.tq_val + e), __ldcg(X + __ldg(a.tq_col + e)), sq);
        }
        acc = fma(s_theta[q], sq, acc);
    }
    return acc;
}

// Cluster-wide fixed-order sums of NV per-thread values.  The CTA partial of
// value v goes to s_part[buf][v]; after the cluster barrier warp 0 reads the
// CL partials (lane = rank) and sums them in butterfly order; lane 0 leaves
// the sums in s_red and, if `then` is given, runs it (the scalar
// recurrences) before the CTA barrier that publishes both.
template <int NV, typename Then>
__device__ __forceinline__ void cl_reduce(double (&c)[NV], double (*s_warp)[2], double (*s_part)[2], int buf,
                                          double* s_red, Then then) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const double x = warp_sum(c[v]);
        if (lane == 0) s_warp[warp][v] = x;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double acc = 0.0;
#pragma unroll
        for (int w = 0; w < CW; ++w) acc += s_warp[w][threadIdx.x];
        s_part[buf][threadIdx.x] = acc;
    }
    cluster_sync_all();
    if (warp == 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const double x = warp_sum(lane < CL ? ld_dsmem(&s_part[buf][v], (unsigned int)lane) : 0.0);
            if (lane == 0) s_red[v] = x;
        }
        if (lane == 0) then();
    }
    __syncthreads();
}

__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(CT, 1) fom_cluster_kernel(FomClArgs a) {
    extern __shared__ double cl_smem[];
    __shared__ double s_warp[CW][2];
    __shared__ double s_part[2][2];
    __shared__ double s_red[2];
    __shared__ double s_theta[16];
    __shared__ double s_rho, s_rho_old, s_alpha, s_omega, s_beta, s_bnorm;
    __shared__ int s_state, s_code, s_it;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned int crank = cluster_rank();
    const int sample = (int)(blockIdx.x / CL);
    const int64_t N = a.N;
    const int64_t s_begin = (int64_t)crank * a.n_slices / CL;
    const int64_t s_end = (int64_t)(crank + 1) * a.n_slices / CL;
    const int vlen = a.max_slices * kSlice;
    double* sr = cl_smem;             // r
    double* srh = cl_smem + vlen;     // r^
    double* sv = cl_smem + 2 * vlen;  // v
    double* st = cl_smem + 3 * vlen;  // t
    double* gx = a.vecs + (size_t)sample * (3 + kHist) * N;
    double* gp = gx + N;
    double* gs = gp + N;
    double* gh = gs + N;  // kHist levels
    const double* amu_p = a.amu + (size_t)sample * a.mx_size;
    if (threadIdx.x < a.Q) s_theta[threadIdx.x] = a.theta[(int64_t)sample * a.Q + threadIdx.x];
    if (threadIdx.x == 0) {
        s_state = S_ACTIVE;
        s_code = ST_OK;
    }
    __syncthreads();
    int buf = 0;

#define CL_ROWS_BEGIN                                                     \
    for (int64_t sl = s_begin + warp; sl < s_end; sl += CW) {             \
        const int64_t row = sl * kSlice + lane;                           \
        const int li = (int)(sl - s_begin) * kSlice + lane;               \
        const bool valid = row < N;                                       \
        (void)li;
#define CL_ROWS_END }

    // level 0 (u0, or 0) into the history
    CL_ROWS_BEGIN
        if (valid) gh[row] = __ldcg(gx + row);
    CL_ROWS_END
    for (int k = 0; k < a.Nt; ++k) {
        const double h = a.dt[k];
        const double* uk = gh + (size_t)(k % kHist) * N;
        // ---- X0: initial iterate by extrapolating the last levels
        if (k > 0) {
            const int o = min(k, kPred);
            double coef[kPred + 1];
            {
                double bin = 1.0;
#pragma unroll
                for (int i = 0; i <= kPred; ++i) {
                    bin = bin * (double)(o + 1 - i) / (double)(i + 1);
                    coef[i] = i <= o ? ((i & 1) ? -bin : bin) : 0.0;
                }
            }
            CL_ROWS_BEGIN
                if (valid) {
                    double x0 = 0.0;
#pragma unroll
                    for (int i = 0; i <= kPred; ++i) {
                        if (i > o) break;
                        x0 = fma(coef[i], __ldcg(gh + (size_t)((k - i + kHist * kPred) % kHist) * N + row), x0);
                    }
                    __stcg(gx + row, x0);
                }
            CL_ROWS_END
            cluster_sync_all();
        }
        // ---- R: b = u^k + h B f^k, r = b - x0 + h A x0, r^ = r, p = v = 0
        {
            double c[2] = {0.0, 0.0};
            const bool on = s_state != S_FAILED;
            CL_ROWS_BEGIN
                double rr = 0.0;
                if (valid) {
                    double bf = 0.0;
                    for (int q = 0; q < a.n_in; ++q)
                        bf = fma(__ldg(a.B + row + (int64_t)q * N), __ldg(a.F + (int64_t)k * a.n_in + q), bf);
                    const double Ax = spmv_row_cl(a, amu_p, sl, lane, gx, s_theta);
                    const double b = fma(h, bf, __ldcg(uk + row));
                    rr = on ? fma(h, Ax, b - __ldcg(gx + row)) : 0.0;
                    if (on) {
                        c[0] = fma(b, b, c[0]);
                        c[1] = fma(rr, rr, c[1]);
                    }
                    __stcg(gp + row, 0.0);
                }
                sr[li] = rr;
                srh[li] = rr;
                sv[li] = 0.0;
            CL_ROWS_END
            cl_reduce<2>(c, s_warp, s_part, buf, s_red, [&]() {
                s_it = 0;
                if (s_state == S_FAILED) return;
                const double bn = sqrt(s_red[0]), rn2 = s_red[1];
                s_bnorm = bn;
                s_rho = rn2;
                s_rho_old = s_alpha = s_omega = 1.0;
                if (!isfinite(bn) || !isfinite(rn2)) {
                    s_state = S_FAILED;
                    s_code = ST_ERR_NONFINITE;
                } else if (bn == 0.0) {
                    s_state = S_ZERO;
                } else if (sqrt(rn2) <= a.tol * bn) {
                    s_state = S_CONV;
                } else {
                    s_state = S_ACTIVE;
                }
                s_beta = 1.0;
            });
            buf ^= 1;
        }
        for (int it = 0; s_state == S_ACTIVE; ++it) {
            if (it >= a.maxit) {
                __syncthreads();
                if (threadIdx.x == 0) {
                    s_state = S_FAILED;
                    s_code = ST_ERR_NOT_CONVERGED;
                }
                __syncthreads();
                break;
            }
            // ---- P: p = r + beta (p - omega v)
            {
                const double be = s_beta, om = s_omega;
                CL_ROWS_BEGIN
                    if (valid) __stcg(gp + row, fma(be, fma(-om, sv[li], __ldcg(gp + row)), sr[li]));
                CL_ROWS_END
            }
            cluster_sync_all();
            if (threadIdx.x == 0) s_it += 1;
            // ---- S1: v = p - h A p, (r^, v)
            {
                double c[1] = {0.0};
                CL_ROWS_BEGIN
                    if (valid) {
                        const double Ap = spmv_row_cl(a, amu_p, sl, lane, gp, s_theta);
                        const double vv = fma(-h, Ap, __ldcg(gp + row));
                        sv[li] = vv;
                        c[0] = fma(srh[li], vv, c[0]);
                    }
                CL_ROWS_END
                cl_reduce<1>(c, s_warp, s_part, buf, s_red, [&]() {
                    const double d = s_red[0];
                    if (!isfinite(d)) {
                        s_state = S_FAILED;
                        s_code = ST_ERR_NONFINITE;
                    } else if (d == 0.0) {
                        s_state = S_FAILED;
                        s_code = ST_ERR_BREAKDOWN;
                    } else {
                        s_alpha = s_rho / d;
                    }
                });
                buf ^= 1;
            }
            if (s_state != S_ACTIVE) break;
            // ---- S2: s = r - alpha v, ||s||^2
            {
                const double al = s_alpha;
                double c[1] = {0.0};
                CL_ROWS_BEGIN
                    if (valid) {
                        const double sv_ = fma(-al, sv[li], sr[li]);
                        __stcg(gs + row, sv_);
                        c[0] = fma(sv_, sv_, c[0]);
                    }
                CL_ROWS_END
                cl_reduce<1>(c, s_warp, s_part, buf, s_red, [&]() {
                    const double sn = sqrt(s_red[0]);
                    if (!isfinite(sn)) {
                        s_state = S_FAILED;
                        s_code = ST_ERR_NONFINITE;
                    } else if (sn <= a.tol * s_bnorm) {
                        s_state = S_CONV_S;
                    }
                });
                buf ^= 1;
            }
            if (s_state == S_CONV_S) {
                // half-step exit: x += alpha p
                const double al = s_alpha;
                CL_ROWS_BEGIN
                    if (valid) __stcg(gx + row, fma(al, __ldcg(gp + row), __ldcg(gx + row)));
                CL_ROWS_END
                __syncthreads();
                if (threadIdx.x == 0) s_state = S_CONV;
                __syncthreads();
                break;
            }
            if (s_state != S_ACTIVE) break;
            // ---- S3: t = s - h A s, (t, s), (t, t)
            {
                double c[2] = {0.0, 0.0};
                CL_ROWS_BEGIN
                    if (valid) {
                        const double As = spmv_row_cl(a, amu_p, sl, lane, gs, s_theta);
                        const double sv_ = __ldcg(gs + row);
                        const double tv = fma(-h, As, sv_);
                        st[li] = tv;
                        c[0] = fma(tv, sv_, c[0]);
                        c[1] = fma(tv, tv, c[1]);
                    }
                CL_ROWS_END
                cl_reduce<2>(c, s_warp, s_part, buf, s_red, [&]() {
                    const double ts = s_red[0], tt = s_red[1];
                    if (!isfinite(ts) || !isfinite(tt)) {
                        s_state = S_FAILED;
                        s_code = ST_ERR_NONFINITE;
                    } else if (tt == 0.0) {
                        s_state = S_FAILED;
                        s_code = ST_ERR_BREAKDOWN;
                    } else {
                        s_omega = ts / tt;
                    }
                });
                buf ^= 1;
            }
            if (s_state != S_ACTIVE) break;
            // ---- E: x += alpha p + omega s, r = s - omega t, (r^, r), (r, r)
            {
                const double al = s_alpha, om = s_omega;
                double c[2] = {0.0, 0.0};
                CL_ROWS_BEGIN
                    if (valid) {
                        const double sv_ = __ldcg(gs + row);
                        __stcg(gx + row, fma(om, sv_, fma(al, __ldcg(gp + row), __ldcg(gx + row))));
                        const double rv = fma(-om, st[li], sv_);
                        sr[li] = rv;
                        c[0] = fma(srh[li], rv, c[0]);
                        c[1] = fma(rv, rv, c[1]);
                    }
                CL_ROWS_END
                cl_reduce<2>(c, s_warp, s_part, buf, s_red, [&]() {
                    const double rho_new = s_red[0], rn = sqrt(s_red[1]);
                    s_rho_old = s_rho;
                    s_rho = rho_new;
                    if (!isfinite(rho_new) || !isfinite(rn)) {
                        s_state = S_FAILED;
                        s_code = ST_ERR_NONFINITE;
                    } else if (rn <= a.tol * s_bnorm) {
                        s_state = S_CONV;
                    } else if (fabs(s_omega) < 1e-300 || fabs(rho_new) < 1e-300) {
                        s_state = S_FAILED;
                        s_code = ST_ERR_BREAKDOWN;
                    } else {
                        s_beta = (s_rho / s_rho_old) * (s_alpha / s_omega);
                    }
                });
                buf ^= 1;
            }
        }
        // ---- W: snapshot column k and the next history level
        {
            const bool zero = s_state == S_ZERO || s_state == S_FAILED;
            CL_ROWS_BEGIN
                if (valid) {
                    double xv = __ldcg(gx + row);
                    if (zero) {
                        xv = 0.0;
                        __stcg(gx + row, 0.0);
                    }
                    if (sample < a.n_mu) __stcs(a.snap + ((int64_t)sample * a.Nt + k) * N + row, xv);
                    __stcg(gh + (size_t)((k + 1) % kHist) * N + row, xv);
                }
            CL_ROWS_END
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (crank == 0 && a.iters) a.iters[(int64_t)k * a.n_mu + sample] = s_it;
            if (s_state == S_ZERO) s_state = S_CONV;
        }
        __syncthreads();
    }
    if (crank == 0 && threadIdx.x == 0) {
        if (a.status) a.status[sample] = s_code;
        if (s_code != ST_OK) st_dev_error(a.err, s_code);
    }
    // no CTA leaves while a peer may still read its shared memory
    cluster_sync_all();
#undef CL_ROWS_BEGIN
#undef CL_ROWS_END
}

// amu[p * mx + e] = sum_q theta[p][q] vals[q][src[e]]; x of sample p = u0 or 0.
__global__ void fom_cluster_setup_kernel(int64_t mx, const int64_t* __restrict__ src, int64_t ell, int Q,
                                         const double* __restrict__ vals, const double* __restrict__ theta,
                                         int n_mu, double* amu, int64_t N, const double* u0, double* vecs,
                                         int64_t vec_stride) {
    const int64_t tot = mx * n_mu;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(i / mx);
        const int64_t se = src[i % mx];
        double s = 0.0;
        if (se >= 0)
            for (int q = 0; q < Q; ++q) s = fma(theta[p * Q + q], vals[(int64_t)q * ell + se], s);
        amu[i] = s;
    }
    const int64_t totx = N * n_mu;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < totx;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(i / N);
        const int64_t row = i % N;
        vecs[p * vec_stride + row] = u0 ? u0[row] : 0.0;
    }
}

// Shared memory of the cluster march for the model's operator (0 if the
// vectors of one CTA's rows do not fit).
size_t cluster_smem(const st_model* m) {
    const int64_t max_slices = (m->n_slices + CL - 1) / CL;
    const size_t bytes = sizeof(double) * kClVecs * (size_t)max_slices * kSlice;
    return bytes <= 200 * 1024 ? bytes : 0;
}

st_status run_cluster(st_model* m, int n_mu, const double* d_theta, int Nt, const double* d_dt, const double* u0,
                      int n_in, const double* B, const double* d_F, double* snap, int32_t* iters, int32_t* status) {
    const int64_t N = m->N, ell = m->ell_size, mx = m->mx_size;
    const size_t smem = cluster_smem(m);
    const int64_t vstride = (3 + kHist) * N;
    const size_t need = sizeof(double) * ((size_t)mx * n_mu + (size_t)vstride * n_mu) + 1024;
    ST_TRY(st_grow(m, m->ws_fom, need));
    double* amu = (double*)m->ws_fom.p;
    double* vecs = amu + (size_t)mx * n_mu;
    {
        const int sblocks = (int)std::max<int64_t>(1, std::min<int64_t>((std::max(mx, N) * n_mu + 255) / 256,
                                                                          8 * m->num_sms));
        ST_PROF(m, "fom_setup_kernel");
        fom_cluster_setup_kernel<<<sblocks, 256, 0, m->stream>>>(mx, m->d_mx_src, ell, m->Q, m->d_vals, d_theta,
                                                                  n_mu, amu, N, u0, vecs, vstride);
        ST_TRY(st_check_launch("fom_cluster_setup"));
    }
    ST_CUDA_TRY(cudaFuncSetAttribute(fom_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FomClArgs a;
    a.N = N;
    a.Q = m->Q;
    a.theta = d_theta;
    a.mx_ptr = m->d_mx_ptr;
    a.mx_w = m->d_mx_w;
    a.mx_col = m->d_mx_col;
    a.amu = amu;
    a.mx_size = mx;
    a.tq_ptr = m->d_tq_ptr;
    a.tq_w = m->d_tq_w;
    a.tq_col = m->d_tq_col;
    a.tq_val = m->d_tq_val;
    a.n_slices = m->n_slices;
    a.Nt = Nt;
    a.dt = d_dt;
    a.n_in = n_in;
    a.B = B;
    a.F = d_F;
    a.vecs = vecs;
    a.snap = snap;
    a.n_mu = n_mu;
    a.iters = iters;
    a.status = status;
    a.err = m->d_err;
    a.tol = m->opt.tol;
    a.maxit = m->opt.maxit;
    a.max_slices = (int)((m->n_slices + CL - 1) / CL);
    ST_PROF(m, "fom_march_kernel");
    fom_cluster_kernel<<<dim3((unsigned)(n_mu * CL)), dim3(CT), smem, m->stream>>>(a);
    return st_check_launch("fom_cluster");
}

// Sub-grids per launch for a group of n_mu samples: two samples per
// sub-grid, at most kMaxSub (ST_FOM_SUBGRIDS fixes the count).  Measured on
// the c4 march of 16 samples (200 steps): 1, 2, 4, 8, 16 sub-grids take
// 97.5, 86.5, 82.5, 80.0, 92.5 ms -- with one sample per sub-grid the shared
// operator is read once per sample and the loads are 8 bytes.
#ifndef ST_FOM_SUBGRIDS
#define ST_FOM_SUBGRIDS 0
#endif
int fom_subgrids(int n_mu) {
    if (ST_FOM_SUBGRIDS > 0) return std::min(ST_FOM_SUBGRIDS, std::min(kMaxSub, n_mu));
    return std::max(1, std::min(kMaxSub, n_mu / 2));
}

// March n_mu samples (at most n_sub * LD) in one cooperative launch of n_sub
// sub-grids; sub-grid s takes samples [s * per_sub, ...).
template <int LD>
st_status run_group(st_model* m, int n_mu, int n_sub, const double* d_theta, int Nt, const double* d_dt,
                    const double* u0, int n_in, const double* B, const double* d_F, const double* src,
                    double* snap, int32_t* iters, int32_t* status, int32_t* d_iters_tmp) {
    const int64_t N = m->N, ell = m->ell_size, mx = m->mx_size;
    const size_t vec = (size_t)N * LD;
    const void* kern = src ? (const void*)fom_march_kernel<LD, true> : (const void*)fom_march_kernel<LD, false>;
    int blocks = st_coop_blocks(m, fom_march_kernel<LD, false>, NT, 0, ST_FOM_BLOCKS_PER_SM);
    if (src) blocks = std::min(blocks, st_coop_blocks(m, fom_march_kernel<LD, true>, NT, 0, ST_FOM_BLOCKS_PER_SM));
    if (blocks < n_sub) return st_fail(ST_ERR_CUDA, "fom: cooperative occupancy query failed");
    const int64_t rpb = Cfg<LD>::RPB;
    const int64_t nchunks = (N + rpb - 1) / rpb;
    int per = blocks / n_sub;
    if (per > nchunks) per = (int)std::max<int64_t>(1, nchunks);
    const int per_sub = (n_mu + n_sub - 1) / n_sub;
    const size_t sub_doubles = (size_t)mx * LD + (7 + kHist) * vec + 2 * (size_t)per * NSLOT * LD;
    const size_t need = sizeof(double) * (sub_doubles * n_sub) + sizeof(unsigned int) * 4 * kMaxSub + 1024;
    ST_TRY(st_grow(m, m->ws_fom, need));
    unsigned int* bars = (unsigned int*)((double*)m->ws_fom.p + sub_doubles * n_sub);
    ST_CUDA_TRY(cudaMemsetAsync(bars, 0, sizeof(unsigned int) * 4 * kMaxSub, m->stream));
    FomArgs a;
    double* base = (double*)m->ws_fom.p;
    for (int sb = 0; sb < n_sub; ++sb) {
        const int p0 = sb * per_sub, ng = std::max(0, std::min(per_sub, n_mu - p0));
        double* amu = base + sub_doubles * sb;
        if (ng > 0) {
            int sblocks = (int)std::min<int64_t>((std::max(mx, N) * LD + 255) / 256, 8 * m->num_sms);
            ST_PROF(m, "fom_setup_kernel");
            fom_setup_kernel<LD><<<std::max(sblocks, 1), 256, 0, m->stream>>>(
                mx, m->d_mx_src, ell, m->Q, m->d_vals, d_theta + (size_t)p0 * m->Q, ng, amu, N, u0,
                amu + (size_t)mx * LD);
            ST_TRY(st_check_launch("fom_setup"));
        }
    }
    double* amu = base;
    double* vecs = amu + (size_t)mx * LD;
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
    a.src = src;
    a.x = vecs;
    a.r = vecs + vec;
    a.rh = vecs + 2 * vec;
    a.p = vecs + 3 * vec;
    a.v = vecs + 4 * vec;
    a.s = vecs + 5 * vec;
    a.t = vecs + 6 * vec;
    a.hist = vecs + 7 * vec;
    a.partial = vecs + (7 + kHist) * vec;
    a.snap = snap;
    a.n_mu = n_mu;
    a.iters = iters ? d_iters_tmp : nullptr;
    a.status = status;
    a.tol = m->opt.tol;
    a.maxit = m->opt.maxit;
    a.bar = GridBarrier{bars, bars + 1, bars + 2, m->d_err, m->opt.spin_limit, (unsigned int)per};
    a.per = per;
    a.per_sub = per_sub;
    a.sub_doubles = (int64_t)sub_doubles;
    void* args[] = {&a};
    ST_PROF(m, "fom_march_kernel");
    ST_CUDA_TRY(cudaLaunchCooperativeKernel(kern, dim3(per * n_sub), dim3(NT), args, 0, m->stream));
    st_count_launch();
    return ST_OK;
}

}  // namespace

// The march of st_fom_march with an optional per-step source src (dev
// [n_mu x Nt x N], added to the right-hand side of every step; grid march).
st_status st_internal_fom_march(st_model* m, int32_t n_mu, const double* theta, int32_t Nt, const double* dt,
                                const double* u0, int32_t n_in, const double* B, const double* F,
                                const double* src, double* snapshots, int32_t* iters, int32_t* status) {
    if (!m) return st_fail(ST_ERR_ARG, "st_fom_march: NULL model");
    if (n_mu < 1 || Nt < 1 || n_in < 0) return st_fail(ST_ERR_ARG, "st_fom_march: bad sizes");
    if (!theta || !dt || !snapshots) return st_fail(ST_ERR_ARG, "st_fom_march: NULL argument");
    if (n_in > 0 && (!B || !F)) return st_fail(ST_ERR_ARG, "st_fom_march: NULL B or F");
    for (int k = 0; k < Nt; ++k)
        if (!(dt[k] > 0) || !std::isfinite(dt[k])) return st_fail(ST_ERR_ARG, "st_fom_march: dt must be positive");
    const int Q = m->Q;
    // small host inputs -> device (theta, dt, F); iteration counts staged per group
    const size_t nF = (size_t)Nt * n_in;
    size_t bytes = sizeof(double) * ((size_t)n_mu * Q + Nt + nF) + sizeof(int32_t) * (size_t)Nt * 64 + 256;
    ST_TRY(st_grow(m, m->ws_misc, bytes));
    double* d_theta = (double*)m->ws_misc.p;
    double* d_dt = d_theta + (size_t)n_mu * Q;
    double* d_F = d_dt + Nt;
    int32_t* d_it = (int32_t*)(d_F + nF);
    ST_CUDA_TRY(cudaMemcpyAsync(d_theta, theta, sizeof(double) * n_mu * Q, cudaMemcpyHostToDevice, m->stream));
    ST_CUDA_TRY(cudaMemcpyAsync(d_dt, dt, sizeof(double) * Nt, cudaMemcpyHostToDevice, m->stream));
    if (nF) ST_CUDA_TRY(cudaMemcpyAsync(d_F, F, sizeof(double) * nF, cudaMemcpyHostToDevice, m->stream));
    // the grid-wide march unless the cluster march is asked for (measured on
    // the 2-D S4 operator of N = 49,152 with 16 samples: 95 ms grid, 167 ms
    // cluster -- 15 clusters of 8 CTAs are resident at once, so 16 samples
    // take two waves, and one sample on 8 SMs takes 85 ms)
    const bool use_cluster = !src && m->opt.fom_path == ST_FOM_CLUSTER && cluster_smem(m) > 0;
    if (!src && m->opt.fom_path == ST_FOM_CLUSTER && !use_cluster)
        return st_fail(ST_ERR_ARG, "st_fom_march: the cluster march does not fit N = %lld", (long long)m->N);
    if (use_cluster) {
        // samples in groups of at most 64 clusters (the iteration counts are
        // written per group in the caller's layout directly)
        for (int g0 = 0; g0 < n_mu; g0 += 64) {
            const int ng = std::min(64, n_mu - g0);
            double* snap = snapshots + (size_t)g0 * Nt * m->N;
            int32_t* st = status ? status + g0 : nullptr;
            ST_TRY(run_cluster(m, ng, d_theta + (size_t)g0 * Q, Nt, d_dt, u0, n_in, B, d_F, snap,
                               iters ? d_it : nullptr, st));
            if (iters)
                ST_CUDA_TRY(cudaMemcpy2DAsync(iters + g0, sizeof(int32_t) * n_mu, d_it, sizeof(int32_t) * ng,
                                              sizeof(int32_t) * ng, Nt, cudaMemcpyDeviceToDevice, m->stream));
        }
        return ST_OK;
    }
    for (int g0 = 0; g0 < n_mu; g0 += 32) {
        const int ng = std::min(32, n_mu - g0);
        const int per_sub = (ng + fom_subgrids(ng) - 1) / fom_subgrids(ng);
        const int n_sub = (ng + per_sub - 1) / per_sub;  // no empty sub-grid
        int ld = 1;
        while (ld < per_sub) ld <<= 1;
        double* snap = snapshots + (size_t)g0 * Nt * m->N;
        int32_t* st = status ? status + g0 : nullptr;
        const double* th = d_theta + (size_t)g0 * Q;
        const double* sg = src ? src + (size_t)g0 * Nt * m->N : nullptr;
        st_status rc;
        switch (ld) {
            case 1: rc = run_group<1>(m, ng, n_sub, th, Nt, d_dt, u0, n_in, B, d_F, sg, snap, iters, st, d_it); break;
            case 2: rc = run_group<2>(m, ng, n_sub, th, Nt, d_dt, u0, n_in, B, d_F, sg, snap, iters, st, d_it); break;
            case 4: rc = run_group<4>(m, ng, n_sub, th, Nt, d_dt, u0, n_in, B, d_F, sg, snap, iters, st, d_it); break;
            case 8: rc = run_group<8>(m, ng, n_sub, th, Nt, d_dt, u0, n_in, B, d_F, sg, snap, iters, st, d_it); break;
            case 16: rc = run_group<16>(m, ng, n_sub, th, Nt, d_dt, u0, n_in, B, d_F, sg, snap, iters, st, d_it); break;
            default: rc = run_group<32>(m, ng, n_sub, th, Nt, d_dt, u0, n_in, B, d_F, sg, snap, iters, st, d_it); break;
        }
        if (rc != ST_OK) return rc;
        if (iters) {
            // each sub-grid's counts [Nt x its samples] -> caller layout [Nt x n_mu]
            for (int p0 = 0; p0 < ng; p0 += per_sub) {
                const int c = std::min(per_sub, ng - p0);
                ST_CUDA_TRY(cudaMemcpy2DAsync(iters + g0 + p0, sizeof(int32_t) * n_mu, d_it + (size_t)Nt * p0,
                                              sizeof(int32_t) * c, sizeof(int32_t) * c, Nt,
                                              cudaMemcpyDeviceToDevice, m->stream));
            }
        }
    }
    return ST_OK;
}

extern "C" st_status st_fom_march(st_model* m, int32_t n_mu, const double* theta, int32_t Nt,
                                  const double* dt, const double* u0, int32_t n_in,
                                  const double* B, const double* F, double* snapshots,
                                  int32_t* iters, int32_t* status) {
    return st_internal_fom_march(m, n_mu, theta, Nt, dt, u0, n_in, B, F, nullptr, snapshots, iters, status);
}

extern "C" st_status st_fom_cluster_occupancy(st_model* m, int32_t* cluster_ctas, int32_t* max_active_clusters,
                                              int64_t* smem_bytes) {
    if (!m) return st_fail(ST_ERR_ARG, "st_fom_cluster_occupancy: NULL model");
    const size_t smem = cluster_smem(m);
    if (cluster_ctas) *cluster_ctas = CL;
    if (smem_bytes) *smem_bytes = (int64_t)smem;
    if (max_active_clusters) {
        *max_active_clusters = 0;
        if (smem > 0) {
            ST_CUDA_TRY(cudaFuncSetAttribute(fom_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(CL * 64);
            cfg.blockDim = dim3(CT);
            cfg.dynamicSmemBytes = smem;
            cfg.stream = m->stream;
            int n = 0;
            ST_CUDA_TRY(cudaOccupancyMaxActiveClusters(&n, (void*)fom_cluster_kernel, &cfg));
            *max_active_clusters = n;
        }
    }
    return ST_OK;
}
