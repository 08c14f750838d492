// Basis generation (Secs. 4.1-4.2): block-incremental SVD of the snapshot
// matrix U = [U_1 ... U_nmu], one parameter block U_p (N x Nt) per update,
// then per-mode temporal bases.
//
// Per block (the rank-one update of Eqs. factorization1-rankOneUpdateSVD2
// applied to Nt columns at once):
//   1. L1 = W^T U_p, E1 = U_p - W L1 (FP64 GEMMs, split over the N rows);
//   2. column-wise Gram-Schmidt with re-orthogonalisation of E1 inside one
//      cooperative kernel: E1 = J1 P1, a column adds a direction only if its
//      remainder norm exceeds eps_svd * (largest column norm of U_p);
//   2b. second block pass: L2 = W^T J1, J1 - W L2 = J P2 (same kernel), so
//      that directions normalised from small remainders lose the rounding
//      they carried along W; L = L1 + L2 P1, P = P2 P1;
//   3. bordered middle matrix Q = [[diag(sigma), L], [0, P]] (Eq. middleMat),
//      thin SVD in FP64, preconditioned one-sided Jacobi: pivoted Householder
//      QR Q^T Pi = Q1 R, one-sided (Hestenes) Jacobi on R^T with the
//      rotations accumulated in Y, so Q = (Pi U_z) Sigma (Q1 Y)^T with U_z
//      the normalised Jacobi columns (the QR cuts the sweeps about 2.5x);
//   4. W <- [W J] Ubar, V <- blkdiag(V, I) Vbar, sigma <- Sigma_bar, dropping
//      sigma < eps_sv * sigma_max and keeping at most r_max;
//   5. orthogonality check |w_1^T w_r| > min(eps_svd, eps N) and, if it fires,
//      re-orthogonalisation of W by Gram-Schmidt QR (positive R diagonal).
// Finally Phi_s = W(:, 1:ns) and, for each i < ns, the temporal snapshot
// matrix Upsilon_i[k, p] = V[p Nt + k, i] is factorised by one-sided Jacobi in
// shared memory: Phi_t^i = its leading nt left singular vectors.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int NT = 256;
constexpr int NWARP = NT / 32;
constexpr int kGsPanel = 128;  // columns per Gram-Schmidt panel

// ---------------------------------------------------------------------------
// tau = eps * max_j ||U[:, j]||: block (j, c) sums column j over row chunk c
// into part[j * chunks + c]; one block then finishes the norms and the max.
__global__ void colnorm_part_kernel(int64_t N, const double* __restrict__ U, int chunks,
                                    double* part) {
    __shared__ double s_part[NWARP];
    const int j = blockIdx.x, c = blockIdx.y;
    const int64_t len = (N + chunks - 1) / chunks;
    const int64_t r0 = (int64_t)c * len, r1 = min(N, r0 + len);
    double acc = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += NT) {
        const double v = U[i + (int64_t)j * N];
        acc = fma(v, v, acc);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < NWARP; ++w) s += s_part[w];
        part[(int64_t)j * chunks + c] = s;
    }
}

__global__ void colnorm_max_kernel(int m, int chunks, const double* __restrict__ part, double eps,
                                   double* tau) {
    __shared__ double s_max[NT];
    double mx = 0.0;
    for (int j = threadIdx.x; j < m; j += NT) {
        double s = 0.0;
        for (int c = 0; c < chunks; ++c) s += part[(int64_t)j * chunks + c];
        mx = fmax(mx, sqrt(s));
    }
    s_max[threadIdx.x] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int t = 0; t < NT; ++t) v = fmax(v, s_max[t]);
        *tau = eps * v;
    }
}

// ---------------------------------------------------------------------------
// Column-wise classical Gram-Schmidt with re-orthogonalisation, E = J P.
struct Gs2Args {
    int64_t N;
    int m;          // columns of E
    double* E;      // N x m (ld N), scratch: its contents are undefined on return
    double* J;      // N x m (ld N) output directions
    double* P;      // coefficients, column j at P + j * ldp, zeroed by the host
    int ldp;
    int* k_out;
    const double* tau;  // NULL: every column adds a direction
    double* partial;    // [2 x grid x (m + 2)]
    unsigned long long* work;  // accumulated: multiply-adds per row (the flop count is 2 N times it)
    GridBarrier bar;
    int64_t rs;  // rows per block (the last block may own fewer)
    int ks;      // directions whose rows of the block are kept in shared memory
};

// Shared memory of gs2_kernel: the four coefficient vectors, with E_SMEM a
// ring of three columns of E, then the first ks directions (block rows).
inline size_t gs2_smem(int m, int64_t rs, bool e_smem, int ks) {
    return sizeof(double) * (4 * (size_t)m + (e_smem ? 3 * (size_t)rs : 0) + (size_t)ks * (size_t)rs);
}

__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
    const unsigned int d = (unsigned int)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_but_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Every block owns rows [r0, r0 + R) of E and J.  The block's rows of the
// three columns in flight (with E_SMEM) and of the first ks directions stay
// in shared memory; the column after them is fetched by asynchronous copies
// one column ahead.  Updates are row-local; dot products are a warp per
// value over the block's rows, then across blocks: a reduction writes
// per-block partials (slots 0..m-1 dots, m the squared norm, m+1 the cross
// term) to one of two buffers, alternating, and every block sums all
// blocks' partials in a fixed order, so a buffer is rewritten only two
// barriers after it was read.  The norm of column j, its product with
// column j+1 and the first-pass projections of column j+1 share one
// reduction (the coefficient on a direction accepted from column j is
// e_j^T e_{j+1} / ||e_j||): two grid barriers per column.  The work of a
// column is small, so the code a column runs through is kept small too
// (loops whose bodies every warp reuses, one body for both passes): its
// instructions are fetched from the SM's caches, not from L2.
template <bool E_SMEM>
__global__ void __launch_bounds__(NT, 1) gs2_kernel(Gs2Args a) {
    extern __shared__ double sm[];
    // pass-1 / pass-2 coefficients of the column being finished (hc, h2c)
    // and of the column being projected (hn, h2n); swapped every column
    double* hc = sm;
    double* h2c = sm + a.m;
    double* hn = sm + 2 * (size_t)a.m;
    double* h2n = sm + 3 * (size_t)a.m;
    double* s_e = sm + 4 * (size_t)a.m;                    // [3][rs] with E_SMEM
    double* s_j = s_e + (E_SMEM ? 3 * (size_t)a.rs : 0);  // [ks][rs]
    __shared__ double s_nu, s_inv, s_cross;
    __shared__ int s_flag;
    const int G = gridDim.x, b = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t r0 = (int64_t)b * a.rs;
    const int R = (int)max((int64_t)0, min(a.N, r0 + a.rs) - r0);
    const int64_t rs = a.rs;
    const int ks = a.ks;
    const int m = a.m;
    // this block's rows of column c of E and of direction c of J
    auto e_col = [&](int c) -> double* {
        if (E_SMEM) return s_e + (size_t)(c % 3) * rs;
        return a.E + (int64_t)c * a.N + r0;
    };
    auto j_col = [&](int c) -> double* {
        return c < ks ? s_j + (size_t)c * rs : a.J + (int64_t)c * a.N + r0;
    };
    // a thread leaves only after its asynchronous copies have landed
    auto leave = [&]() {
        if (E_SMEM) cp_async_wait_all();
    };
    // this thread's share of column c into its ring slot (one copy group,
    // committed even when empty so that the group count stays aligned)
    auto prefetch = [&](int c) {
        if (!E_SMEM) return;
        if (c < m) {
            double* dst = e_col(c);
            const double* src = a.E + (int64_t)c * a.N + r0;
#pragma unroll 1
            for (int r = tid; r < R; r += NT) cp_async8(dst + r, src + r);
        }
        cp_async_commit();
    };
    const double tau = a.tau ? *a.tau : -1.0;
    const int S = m + 2;
    int red = 0;
    auto part_of = [&](int bb, int slot) { return a.partial + ((size_t)(red & 1) * G + bb) * S + slot; };
    // Block partials of nv values, a warp per value: value q < nj is
    // J(:, q)^T y, value nj is v^T v and nj+1 is v^T y (v, y columns of E, y
    // < 0 a zero column); the partial of value q goes to slot q (q < nj) or
    // m + q - nj.  Lane-strided rows, two accumulators, then the warp.
    auto block_dots = [&](int nj, int nv, int vc, int yc) {
        const double* v = e_col(vc);
        const double* y = yc >= 0 ? e_col(yc) : nullptr;
#pragma unroll 1
        for (int q = warp; q < nv; q += NWARP) {
            const double* x = q < nj ? j_col(q) : v;
            const double* z = q == nj ? v : y;
            double s0 = 0.0, s1 = 0.0;
            if (z) {
                int r = lane;
#pragma unroll 1
                for (; r + 32 < R; r += 64) {
                    s0 = fma(x[r], z[r], s0);
                    s1 = fma(x[r + 32], z[r + 32], s1);
                }
                if (r < R) s0 = fma(x[r], z[r], s0);
            }
            const double t = warp_sum(s0 + s1);
            if (lane == 0) __stcg(part_of(b, q < nj ? q : m + (q - nj)), t);
        }
    };
    // Fixed-order sums over the blocks of ns slots (slot q for q < nq, m +
    // q - nq after), a warp per slot, the loads of eight blocks per lane in
    // flight together: h[q] for q < nq, then ||e||, 1/||e|| and the cross
    // term.
    auto sum_slots = [&](int nq, int ns, double* h) {
#pragma unroll 1
        for (int q = warp; q < ns; q += NWARP) {
            const int sl = q < nq ? q : m + (q - nq);
            double acc = 0.0;
#pragma unroll 1
            for (int b0 = lane; b0 < G; b0 += 8 * 32) {
                double v[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int bb = b0 + 32 * i;
                    v[i] = bb < G ? __ldcg(part_of(bb, sl)) : 0.0;
                }
                acc += ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
            }
            const double t = warp_sum(acc);
            if (lane == 0) {
                if (q < nq) h[q] = t;
                else if (q == nq) {
                    // ||e_j|| and its inverse from one reciprocal square root
                    // (a zero column: both zero; Inf or NaN: a non-finite norm)
                    const double iv = t > 0.0 ? rsqrt(t) : 0.0;
                    s_inv = iv;
                    s_nu = t > 0.0 ? t * iv : (t == 0.0 ? 0.0 : t);
                } else s_cross = t;
            }
        }
    };
    int k = 0;   // directions found so far
    int kc = 0;  // directions the finishing column was projected on
    unsigned long long work = 2;  // multiply-adds per row: ||e_0||^2 and e_0^T e_1
    prefetch(0);
    prefetch(1);
    prefetch(2);
    leave();
    __syncthreads();
    // column 0 has nothing to project: ||e_0||^2 and e_0^T e_1
    block_dots(0, 2, 0, m > 1 ? 1 : -1);
#pragma unroll 1
    for (int j = 0; j < m; ++j) {
        // reduction A: ||e_j||^2, e_j^T e_{j+1}, J(:, 0:k)^T e_{j+1}
        if (!grid_sync(a.bar, &s_flag)) {
            leave();
            return;
        }
        sum_slots(k, k + 2, hn);
        ++red;
        __syncthreads();
        const double nu = s_nu;
        if (!isfinite(nu)) {
            if (tid == 0) grid_abort(a.bar, ST_ERR_NONFINITE);
            leave();
            return;
        }
        // finish column j: its coefficients, and a new direction if the
        // remainder is above the threshold
        if (b == 0)
#pragma unroll 1
            for (int c = tid; c < kc; c += NT) a.P[c + (int64_t)j * a.ldp] = hc[c] + h2c[c];
        if (nu > tau && nu > 0.0) {
            const double inv = s_inv;
            const double* ej = e_col(j);
            double* jk = a.J + (int64_t)k * a.N + r0;
            double* sk = k < ks ? s_j + (size_t)k * rs : jk;
#pragma unroll 1
            for (int r = tid; r < R; r += NT) {
                const double v = ej[r] * inv;
                sk[r] = v;
                __stcg(jk + r, v);
            }
            if (b == 0 && tid == 0) a.P[k + (int64_t)j * a.ldp] = nu;
            if (tid == 0) hn[k] = s_cross * inv;
            ++k;
        }
        __syncthreads();
        if (j + 1 == m) break;
        // column j's ring slot is free (its last reads precede the barrier)
        prefetch(j + 3);
        // both passes' updates and dot products, the next column's first-pass
        // dot products, the squared norm and the cross term
        work += 3 * (unsigned long long)k + (j + 2 < m ? k : 0) + 2;
        // pass 0 (with directions): e_{j+1} -= J hn, then J^T e_{j+1}, reduced
        // into h2n; pass 1: e_{j+1} -= J h2n, then the first-pass products of
        // e_{j+2}, ||e_{j+1}||^2 and e_{j+1}^T e_{j+2}
        double* e1 = e_col(j + 1);
#pragma unroll 1
        for (int pass = k > 0 ? 0 : 1; pass < 2; ++pass) {
            const double* h = pass ? h2n : hn;
            if (k > 0)
#pragma unroll 1
                for (int r = tid; r < R; r += NT) {
                    double v = e1[r], w = 0.0;
                    int c = 0;
#pragma unroll 1
                    for (; c + 1 < k; c += 2) {
                        v = fma(-j_col(c)[r], h[c], v);
                        w = fma(-j_col(c + 1)[r], h[c + 1], w);
                    }
                    if (c < k) v = fma(-j_col(c)[r], h[c], v);
                    e1[r] = v + w;
                }
            if (E_SMEM && pass == 1) cp_async_wait_all_but_one();  // column j+2 has landed
            __syncthreads();
            if (pass == 0) {
                block_dots(k, k, j + 1, j + 1);
                // reduction B: J(:, 0:k)^T e_{j+1} (second pass)
                if (!grid_sync(a.bar, &s_flag)) {
                    leave();
                    return;
                }
                sum_slots(k, k, h2n);
                ++red;
                __syncthreads();
            } else {
                block_dots(k, k + 2, j + 1, j + 2 < m ? j + 2 : -1);
            }
        }
        kc = k;
        double* t = hc;
        hc = hn;
        hn = t;
        t = h2c;
        h2c = h2n;
        h2n = t;
    }
    leave();
    if (b == 0 && tid == 0) {
        *a.k_out = k;
        if (a.work) atomicAdd(a.work, work);
    }
}

// D(0:rows, 0:cols) += S(0:rows, 0:cols) (column major).
__global__ void add_block_kernel(int rows, int cols, const double* __restrict__ S, int lds, double* D, int ldd) {
    const int64_t tot = (int64_t)rows * cols;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t % rows), j = (int)(t / rows);
        D[i + (int64_t)j * ldd] += S[i + (int64_t)j * lds];
    }
}

// ---------------------------------------------------------------------------
// Cholesky QR step for a well-conditioned block (the second block pass):
// G = R^T R (upper R, written with leading dimension ldr) and Rinv = R^{-1}
// (ld k).  A pivot below 1e-8 of its diagonal entry of G sets *fail so the
// host can fall back to column-wise Gram-Schmidt.
__global__ void __launch_bounds__(NT) chol_inv_kernel(int k, const double* __restrict__ G, double* R,
                                                      int ldr, double* Rinv, int* fail) {
    __shared__ double s_d;
    for (int t = threadIdx.x; t < k * k; t += NT) {
        const int i = t % k, j = t / k;
        R[i + (int64_t)j * ldr] = 0.0;
        Rinv[t] = 0.0;
    }
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        if (threadIdx.x == 0) {
            double d = G[j + (int64_t)j * k];
            for (int i = 0; i < j; ++i) d -= R[i + (int64_t)j * ldr] * R[i + (int64_t)j * ldr];
            if (!(d > 1e-16 * G[j + (int64_t)j * k])) {
                *fail = 1;
                d = 1.0;
            }
            s_d = sqrt(d);
            R[j + (int64_t)j * ldr] = s_d;
        }
        __syncthreads();
        const double rjj = s_d;
        for (int c = j + 1 + threadIdx.x; c < k; c += NT) {
            double v = G[j + (int64_t)c * k];
            for (int i = 0; i < j; ++i) v -= R[i + (int64_t)j * ldr] * R[i + (int64_t)c * ldr];
            R[j + (int64_t)c * ldr] = v / rjj;
        }
        __syncthreads();
    }
    // Rinv column c solves R x = e_c (upper triangular back substitution)
    for (int c = threadIdx.x; c < k; c += NT) {
        double* x = Rinv + (int64_t)c * k;
        for (int i = c; i >= 0; --i) {
            double v = (i == c) ? 1.0 : 0.0;
            for (int l = i + 1; l <= c; ++l) v -= R[i + (int64_t)l * ldr] * x[l];
            x[i] = v / R[i + (int64_t)i * ldr];
        }
    }
}

// ---------------------------------------------------------------------------
// X = Q^T for Q = [[diag(sigma), L], [0, P(0:k, :)]]:  X is (r + m) x (r + k).
__global__ void build_qt_kernel(int r, int k, int m, const double* __restrict__ sigma,
                                const double* __restrict__ L, int ldl, const double* __restrict__ P,
                                int ldp, double* X, int ldx) {
    const int rows = r + m, cols = r + k;
    const int64_t tot = (int64_t)rows * cols;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(t % rows), c = (int)(t / rows);
        double v = 0.0;
        if (c < r) v = a < r ? (a == c ? sigma[c] : 0.0) : L[c + (int64_t)(a - r) * ldl];
        else v = a < r ? 0.0 : P[(c - r) + (int64_t)(a - r) * ldp];
        X[a + (int64_t)c * ldx] = v;
    }
}

// ---------------------------------------------------------------------------
// Householder QR with column pivoting of X (m x n, m >= n), in place and
// without moving columns: logical column k of X Pi is physical column
// piv[k].  Step k picks the unused column with the largest trailing norm
// (smallest index on ties), builds the reflector H_k = I - tau_k v v^T that
// maps its rows k..m-1 to beta_k e_k (v_k = 1, v_i = x_i / (x_k - beta_k)),
// and applies H_k to every other unused column.  The pivot column keeps its
// pre-reflection rows k..m-1 (from which v is rebuilt) and rows 0..k-1 hold
// R(0:k, k); R(k, k) = beta_k.  Columns are owned by CTAs (j mod grid), so a
// step needs one grid barrier; the trailing norms are recomputed exactly and
// double buffered, -1 marking pivoted columns.  Used as the preconditioner of
// the one-sided Jacobi SVD: Jacobi on R^T needs far fewer sweeps than on X.
struct QrpArgs {
    int m, n;
    double* X;
    int ldx;
    double* beta;   // [n]
    double* tau;    // [n]
    double* scale;  // [n] 1 / (x_k - beta_k), 0 for a zero column
    int* piv;       // [n]
    double* nrm;    // [2 n]
    GridBarrier bar;
};

constexpr int QT = 256;
constexpr int QW = QT / 32;

__global__ void __launch_bounds__(QT) qrp_kernel(QrpArgs a) {
    extern __shared__ double qv[];  // [m] pivot column, then the reflector
    __shared__ double s_val[QW];
    __shared__ int s_idx[QW];
    __shared__ int s_p, s_flag;
    __shared__ double s_tau, s_scale;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, b = blockIdx.x;
    // squared norms of the owned columns (warp per column)
    {
        int cnt = 0;
        for (int j = b; j < a.n; j += G, ++cnt) {
            if (cnt % QW != warp) continue;
            const double* x = a.X + (int64_t)j * a.ldx;
            double s = 0.0;
            for (int i = lane; i < a.m; i += 32) {
                const double v = __ldcg(x + i);
                s = fma(v, v, s);
            }
            s = warp_sum(s);
            if (lane == 0) __stcg(a.nrm + j, s);
        }
    }
    if (!grid_sync(a.bar, &s_flag)) return;
    for (int k = 0; k < a.n; ++k) {
        const double* nin = a.nrm + (size_t)(k & 1) * a.n;
        double* nout = a.nrm + (size_t)((k + 1) & 1) * a.n;
        // pivot: largest trailing norm, smallest index on ties
        double bv = -1.0;
        int bi = a.n;
        for (int j = tid; j < a.n; j += QT) {
            const double v = __ldcg(nin + j);
            if (v > bv) {
                bv = v;
                bi = j;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, bv, off);
            const int oi = __shfl_down_sync(0xffffffffu, bi, off);
            if (ov > bv || (ov == bv && oi < bi)) {
                bv = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            s_val[warp] = bv;
            s_idx[warp] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            double v = s_val[0];
            int p = s_idx[0];
            for (int w = 1; w < QW; ++w)
                if (s_val[w] > v || (s_val[w] == v && s_idx[w] < p)) {
                    v = s_val[w];
                    p = s_idx[w];
                }
            s_p = p;
        }
        __syncthreads();
        const int p = s_p;
        // pivot column rows k..m-1 and its norm
        const double* xp = a.X + (int64_t)p * a.ldx;
        double s = 0.0;
        for (int i = k + tid; i < a.m; i += QT) {
            const double v = __ldcg(xp + i);
            qv[i] = v;
            s = fma(v, v, s);
        }
        s = warp_sum(s);
        if (lane == 0) s_val[warp] = s;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < QW; ++w) t += s_val[w];
            const double alpha = qv[k], nx = sqrt(t);
            double beta = 0.0, tau = 0.0, sc = 0.0;
            if (nx > 0.0) {
                beta = -copysign(nx, alpha);
                tau = (beta - alpha) / beta;
                sc = 1.0 / (alpha - beta);
            }
            s_tau = tau;
            s_scale = sc;
            if (b == 0) {
                a.beta[k] = beta;
                a.tau[k] = tau;
                a.scale[k] = sc;
                a.piv[k] = p;
            }
        }
        __syncthreads();
        const double sc = s_scale, tau = s_tau;
        for (int i = k + 1 + tid; i < a.m; i += QT) qv[i] *= sc;
        if (tid == 0) qv[k] = 1.0;
        __syncthreads();
        // apply H_k to the owned unused columns, new trailing norms
        int cnt = 0;
        for (int j = b; j < a.n; j += G, ++cnt) {
            if (cnt % QW != warp) continue;
            const double nj = __ldcg(nin + j);
            if (j == p || nj < 0.0) {
                if (lane == 0) __stcg(nout + j, -1.0);
                continue;
            }
            double* x = a.X + (int64_t)j * a.ldx;
            double w = 0.0;
            for (int i = k + lane; i < a.m; i += 32) w = fma(qv[i], __ldcg(x + i), w);
            w = warp_sum(w) * tau;
            double s2 = 0.0;
            for (int i = k + lane; i < a.m; i += 32) {
                const double v = fma(-w, qv[i], __ldcg(x + i));
                __stcg(x + i, v);
                if (i > k) s2 = fma(v, v, s2);
            }
            s2 = warp_sum(s2);
            if (lane == 0) __stcg(nout + j, s2);
        }
        if (!grid_sync(a.bar, &s_flag)) return;
    }
}

// Z = R^T (n x n, lower triangular) from the in-place pivoted QR, and Y = I.
__global__ void build_rt_kernel(int n, const double* __restrict__ X, int ldx, const int* __restrict__ piv,
                                const double* __restrict__ beta, double* Z, int ldz, double* Y, int ldy) {
    const int64_t tot = (int64_t)n * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t % n), i = (int)(t / n);  // Z[c, i] = R[i, c]
        double v = 0.0;
        if (i < c) v = X[i + (int64_t)piv[c] * ldx];
        else if (i == c) v = beta[c];
        Z[c + (int64_t)i * ldz] = v;
        Y[c + (int64_t)i * ldy] = c == i ? 1.0 : 0.0;
    }
}

// The reflectors of qrp_kernel as the columns of Y (m x n, ld ldy): column k
// is v_k = e_k + (x_k scaled) below row k, zero above; zero for a skipped
// reflector (tau_k = 0), so H_k = I - tau_k v_k v_k^T.
__global__ void build_wy_kernel(int m, int n, const double* __restrict__ X, int ldx, const int* __restrict__ piv,
                                const double* __restrict__ tau, const double* __restrict__ scale, double* Y,
                                int ldy) {
    const int64_t tot = (int64_t)m * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t % m), k = (int)(t / m);
        double v = 0.0;
        if (tau[k] != 0.0 && i >= k) v = i == k ? 1.0 : X[i + (int64_t)piv[k] * ldx] * scale[k];
        Y[i + (int64_t)k * ldy] = v;
    }
}

// Triangular factor of a block of b reflectors (LAPACK's forward, columnwise
// larft): H_0 H_1 ... H_{b-1} = I - Y T Y^T with T upper triangular,
// T(j, j) = tau_j, T(0:j, j) = -tau_j T(0:j, 0:j) (Y(:, 0:j)^T v_j), from the
// Gram matrix G = Y^T Y (b x b, ld ldg).  One CTA, b <= 64.
__global__ void __launch_bounds__(64) larft_kernel(int b, const double* __restrict__ G, int ldg,
                                                   const double* __restrict__ tau, double* T, int ldt) {
    __shared__ double z[64];
    const int tid = threadIdx.x;
    for (int t = tid; t < b * b; t += blockDim.x) T[t % b + (int64_t)(t / b) * ldt] = 0.0;
    __syncthreads();
    for (int j = 0; j < b; ++j) {
        const double tj = tau[j];
        if (tid < j) z[tid] = -tj * G[tid + (int64_t)j * ldg];
        __syncthreads();
        if (tid < j) {
            double acc = 0.0;
            for (int i = tid; i < j; ++i) acc = fma(T[tid + (int64_t)i * ldt], z[i], acc);
            T[tid + (int64_t)j * ldt] = acc;
        }
        if (tid == 0) T[j + (int64_t)j * ldt] = tj;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// One-sided (Hestenes) Jacobi on the columns of X (m x n), rotations
// accumulated into Y (n x n), cyclic by blocks.  The columns, visited in
// decreasing-norm order each sweep, are grouped into blocks of KB; a
// round-robin tournament over the blocks gives each CTA a pair of blocks per
// round.  The CTA stages those 2 KB columns of X and Y in shared memory and
// rotates every cross pair (block I column against block J column) in KB
// inner rounds of KB disjoint pairs, one pair per JW / KB warps; in a sweep's
// first round the pairs inside each block are rotated as well.  Every pair of
// columns is thus met once per sweep, as in the classical cyclic ordering.
// A block pair waits only for its own two blocks: a counter per block holds
// the round it is ready for, released by the CTA that last rotated it, and
// grid barriers remain only around the norms and ordering at the start of a
// sweep and its convergence test at the end.  Squared column norms are
// carried with the rotations and recomputed at the start of every sweep.
// The sweep loop stops after a sweep without rotation, or after a sweep whose
// rotations all had |cos| = |gamma| / sqrt(alpha beta) below sqrt(tol) / 10:
// cyclic Jacobi converges quadratically near the end, so the next sweep
// would find nothing above tol to rotate (it only confirmed convergence).
struct JacArgs {
    int m, n;
    double* X;
    int ldx;
    double* Y;
    int ldy;
    int max_sweeps;
    double tol;
    int* flags;    // [3] a rotation in the sweep
    int* big;      // [3] a rotation with |cos| >= sqrt(tol) / 10 in the sweep
    int* sweeps;   // out
    double* nrm2;  // [n + 1]: squared column norms, then the largest
    double* nsort; // [n] the norms at the start of the sweep, for the ordering
    double cut;    // relative singular-value cut below which columns are dropped
    unsigned long long* rotations;  // out: rotations applied (accumulated)
    unsigned int* ready;  // [ceil(n / KB)] zeroed: the round each column block is ready for
    GridBarrier bar;
};

// The Jacobi rotation of a column pair with squared norms alpha, beta and
// product gamma (gamma != 0): the angle with tan 2theta = 2 gamma / (beta -
// alpha), |theta| <= pi/4.  With d = beta - alpha, h = 2 gamma and r =
// sqrt(d^2 + h^2), cos 2theta = |d| / r; with w = r + |d| and q = 1 / sqrt(2 r w)
// this gives c = w q and s = sign(d) h q, and c^2 + s^2 = (w^2 + h^2) q^2 = 1
// (w^2 + h^2 = 2 r w).  d and h are first scaled by a power of two (exactly)
// so that the larger lies in [1, 4): no overflow or underflow in d^2 + h^2.
// One square root and one reciprocal square root: on this GPU's FP64 pipe a
// dependent square root or division costs about as much as ten FMAs.
__device__ __forceinline__ void jacobi_pair_rot(double alpha, double beta, double gamma, double& c,
                                                double& s) {
    double d = beta - alpha, h = 2.0 * gamma;
    const long long ex = (__double_as_longlong(fmax(fabs(d), fabs(h))) >> 52) & 0x7ff;
    const long long ec = ex < 1 ? 1 : (ex > 2045 ? 2045 : ex);
    const double sc = __longlong_as_double((2046 - ec) << 52);  // 2^(1023 - ec)
    d *= sc;
    h *= sc;
    const double r = sqrt(fma(d, d, h * h));
    const double w = r + fabs(d);
    const double q = rsqrt(2.0 * r * w);
    c = w * q;
    s = (d < 0.0 ? -h : h) * q;
}

// Whether a pair is rotated: |gamma| > tol sqrt(alpha beta), squared where
// alpha beta is finite (no square roots).
__device__ __forceinline__ bool jacobi_rotates(double alpha, double beta, double gamma, double tol) {
    const double p = alpha * beta;
    if (p <= 1.0e308) return gamma * gamma > (tol * tol) * p;
    return fabs(gamma) > tol * sqrt(alpha) * sqrt(beta);
}

constexpr int JW = 8;  // warps per Jacobi CTA
#ifndef ST_JACOBI_KB
#define ST_JACOBI_KB 2
#endif
constexpr size_t kJacobiSmemMax = 200 * 1024;

// Round-robin tournament of np (even) players: round t, table q -> (i, j).
__device__ __forceinline__ void rr_pair(int np, int t, int q, int& i, int& j) {
    if (q == 0) {
        i = t;
        j = np - 1;
    } else {
        i = (t + q) % (np - 1);
        j = (t - q + np - 1) % (np - 1);
    }
}

template <int KB>
__global__ void __launch_bounds__(32 * JW) jacobi_kernel(JacArgs a) {
    constexpr int NC = 2 * KB;     // columns staged per block pair
    constexpr int WPP = JW / KB;   // warps per column pair
    extern __shared__ double jsm[];
    double* sX = jsm;                           // NC x m
    double* sY = sX + (size_t)NC * a.m;         // NC x n
    double* snrm = sY + (size_t)NC * a.n;       // [n] norms, for the ordering
    int* sperm = reinterpret_cast<int*>(snrm + a.n);  // [n] positions -> columns
    __shared__ double s_dot[32 * JW];  // per-thread partial dot products
    __shared__ double s_nrm[NC];
    __shared__ int s_dirty[NC];
    __shared__ int s_col[NC];
    __shared__ int s_rot[KB];
    __shared__ double s_cs[2 * KB];  // (c, s) of each pair slot
    __shared__ int s_flag;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = 32 * JW;
    const int pr = warp / WPP, sub = warp % WPP;  // pair slot of this warp, part of the rows
    const int nb = (a.n + KB - 1) / KB, nbp = nb + (nb & 1);
    const int npairs = nbp / 2;
    unsigned long long rot_count = 0;
    int sweep = 0;
    bool converged = false;
    for (; sweep < a.max_sweeps; ++sweep) {
        if (blockIdx.x == 0 && tid == 0) {
            a.flags[(sweep + 1) % 3] = 0;
            a.big[(sweep + 1) % 3] = 0;
        }
        // squared column norms, one warp per column
        for (int c = blockIdx.x * JW + warp; c < a.n; c += gridDim.x * JW) {
            const double* xc = a.X + (int64_t)c * a.ldx;
            double acc = 0.0;
            for (int r = lane; r < a.m; r += 32) {
                const double u = __ldcg(xc + r);
                acc = fma(u, u, acc);
            }
            acc = warp_sum(acc);
            if (lane == 0) {
                __stcg(a.nrm2 + c, acc);
                __stcg(a.nsort + c, acc);
                // largest squared norm (positive doubles order like their bit patterns)
                if (sweep == 0)
                    atomicMax(reinterpret_cast<unsigned long long*>(a.nrm2 + a.n),
                              (unsigned long long)__double_as_longlong(acc));
            }
        }
        if (!grid_sync(a.bar, &s_flag)) return;
        // visiting order of this sweep: decreasing norm, ties by index; every
        // CTA ranks the norms itself into shared memory (from a copy that the
        // rounds of this sweep do not update)
        for (int c = tid; c < a.n; c += nthr) snrm[c] = __ldcg(a.nsort + c);
        __syncthreads();
        for (int c = tid; c < a.n; c += nthr) {
            const double v = snrm[c];
            int rank = 0;
            for (int d = 0; d < a.n; ++d) {
                const double w = snrm[d];
                rank += (w > v) || (w == v && d < c);
            }
            sperm[rank] = c;
        }
        __syncthreads();
        // pairs of columns that both lie below the truncation cut are dropped
        // after the SVD whatever their rotation, so they are not rotated
        const double cut2 = a.cut * a.cut * __ldcg(a.nrm2 + a.n);
        for (int t = 0; t < nbp - 1; ++t) {
            // round index over the whole launch: block b is ready for this
            // round once ready[b] reaches it (every block plays every round)
            const unsigned int R = (unsigned int)(sweep * (nbp - 1) + t);
            for (int q = blockIdx.x; q < npairs; q += gridDim.x) {
                int I, J;
                rr_pair(nbp, t, q, I, J);
                if (tid == 0) {
                    int ok = 1;
                    if (I < nb) ok = wait_ready(a.bar, a.ready + I, R);
                    if (ok && J < nb) ok = wait_ready(a.bar, a.ready + J, R);
                    s_flag = ok;
                }
                __syncthreads();
                if (!s_flag) return;
                int cols[NC];
                unsigned int vmask = 0;  // bit c: staged column c exists
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int pos = c < KB ? I * KB + c : J * KB + c - KB;
                    cols[c] = pos < a.n ? sperm[pos] : -1;
                    vmask |= (cols[c] >= 0 ? 1u : 0u) << c;
                }
                // stage the columns and their norms: independent loads in flight
                if (tid < NC) {
                    const int pos = tid < KB ? I * KB + tid : J * KB + tid - KB;
                    const int col = pos < a.n ? sperm[pos] : -1;
                    s_col[tid] = col;
                    s_nrm[tid] = col >= 0 ? __ldcg(a.nrm2 + col) : 0.0;
                    s_dirty[tid] = 0;
                }
                for (int r = tid; r < a.m; r += nthr) {
                    double v[NC];
#pragma unroll
                    for (int c = 0; c < NC; ++c) v[c] = cols[c] >= 0 ? __ldcg(a.X + (int64_t)cols[c] * a.ldx + r) : 0.0;
#pragma unroll
                    for (int c = 0; c < NC; ++c) sX[c * a.m + r] = v[c];
                }
                for (int r = tid; r < a.n; r += nthr) {
                    double v[NC];
#pragma unroll
                    for (int c = 0; c < NC; ++c) v[c] = cols[c] >= 0 ? __ldcg(a.Y + (int64_t)cols[c] * a.ldy + r) : 0.0;
#pragma unroll
                    for (int c = 0; c < NC; ++c) sY[c * a.n + r] = v[c];
                }
                __syncthreads();
                const bool full = (t == 0);
                const int inner = full ? NC - 1 : KB;
                for (int s = 0; s < inner; ++s) {
                    int i, j;
                    if (full) rr_pair(NC, s, pr, i, j);
                    else {
                        i = pr;
                        j = KB + (pr + s) % KB;
                    }
                    const bool valid = ((vmask >> i) & (vmask >> j) & 1u) != 0;
                    double* xi = sX + (size_t)i * a.m;
                    double* xj = sX + (size_t)j * a.m;
                    double g = 0.0, g2 = 0.0;
                    if (valid) {
                        int r = sub * 32 + lane;
                        for (; r + 32 * WPP < a.m; r += 64 * WPP) {
                            g = fma(xi[r], xj[r], g);
                            g2 = fma(xi[r + 32 * WPP], xj[r + 32 * WPP], g2);
                        }
                        if (r < a.m) g = fma(xi[r], xj[r], g);
                    }
                    s_dot[tid] = g + g2;
                    __syncthreads();
                    // the first warp of each pair sums the pair's partials and
                    // one of its threads computes the rotation (the square
                    // roots cost as much per warp instruction as the pair's
                    // whole dot product and update)
                    if (sub == 0) {
                        double ga = s_dot[pr * WPP * 32 + lane];
#pragma unroll
                        for (int w = 1; w < WPP; ++w) ga += s_dot[(pr * WPP + w) * 32 + lane];
                        ga = warp_sum(ga);
                        if (lane == 0) {
                            const double al = s_nrm[i], be = s_nrm[j];
                            const bool rot = valid && ga != 0.0 && (al > cut2 || be > cut2) &&
                                             jacobi_rotates(al, be, ga, a.tol);
                            double c = 1.0, sn = 0.0;
                            if (rot) {
                                jacobi_pair_rot(al, be, ga, c, sn);
                                // new squared norms: c^2 al - 2cs ga + s^2 be and s^2 al + 2cs ga + c^2 be
                                // (the pairs of a round are disjoint: no other thread reads them now)
                                const double cs2 = 2.0 * c * sn * ga;
                                s_nrm[i] = fmax(c * c * al - cs2 + sn * sn * be, 0.0);
                                s_nrm[j] = fmax(sn * sn * al + cs2 + c * c * be, 0.0);
                                s_dirty[i] = 1;
                                s_dirty[j] = 1;
                                ++rot_count;
                                const double ab = al * be;
                                if (!(ab <= 1.0e308) || ga * ga > 0.01 * a.tol * ab)
                                    *(volatile int*)(a.big + sweep % 3) = 1;
                            }
                            s_rot[pr] = rot ? 1 : 0;
                            s_cs[2 * pr] = c;
                            s_cs[2 * pr + 1] = sn;
                        }
                    }
                    __syncthreads();
                    if (s_rot[pr]) {
                        const double c = s_cs[2 * pr], sn = s_cs[2 * pr + 1];
                        for (int r = sub * 32 + lane; r < a.m; r += 32 * WPP) {
                            const double u = xi[r], v = xj[r];
                            xi[r] = c * u - sn * v;
                            xj[r] = sn * u + c * v;
                        }
                        double* yi = sY + (size_t)i * a.n;
                        double* yj = sY + (size_t)j * a.n;
                        for (int r = sub * 32 + lane; r < a.n; r += 32 * WPP) {
                            const double u = yi[r], v = yj[r];
                            yi[r] = c * u - sn * v;
                            yj[r] = sn * u + c * v;
                        }
                    }
                    // the next inner round reads columns that other warps rotated
                    __syncthreads();
                }
                bool dirty[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) dirty[c] = s_dirty[c] != 0;
                for (int r = tid; r < a.m; r += nthr) {
#pragma unroll
                    for (int c = 0; c < NC; ++c)
                        if (dirty[c]) __stcg(a.X + (int64_t)cols[c] * a.ldx + r, sX[c * a.m + r]);
                }
                for (int r = tid; r < a.n; r += nthr) {
#pragma unroll
                    for (int c = 0; c < NC; ++c)
                        if (dirty[c]) __stcg(a.Y + (int64_t)cols[c] * a.ldy + r, sY[c * a.n + r]);
                }
                if (tid < NC && s_dirty[tid]) {
                    __stcg(a.nrm2 + s_col[tid], s_nrm[tid]);
                    *(volatile int*)(a.flags + sweep % 3) = 1;
                }
                // every store of this pair is made before the blocks are
                // released to the next round; shared memory is then restaged
                __syncthreads();
                if (tid == 0) {
                    __threadfence();
                    if (I < nb) st_release_gpu(a.ready + I, R + 1);
                    if (J < nb) st_release_gpu(a.ready + J, R + 1);
                }
            }
        }
        // the convergence flag of the sweep and the columns of its last round
        if (!grid_sync(a.bar, &s_flag)) return;
        if (*(volatile int*)(a.flags + sweep % 3) == 0 || *(volatile int*)(a.big + sweep % 3) == 0) {
            converged = true;
            ++sweep;
            break;
        }
    }
    if (rot_count) atomicAdd(a.rotations, rot_count);
    if (blockIdx.x == 0 && tid == 0) {
        *a.sweeps = sweep;
        if (!converged) st_dev_error(a.bar.err, ST_ERR_NOT_CONVERGED);
    }
}

// Shared memory of the block Jacobi kernel for KB columns per block.
inline size_t jacobi_smem(int kb, int m, int n) {
    return sizeof(double) * (2 * (size_t)kb * (m + n) + n) + sizeof(int) * (size_t)n;
}

// ---------------------------------------------------------------------------
// Column norms of X, descending order, truncation count.
__global__ void __launch_bounds__(1024) sort_kernel(int m, int n, const double* __restrict__ X,
                                                    int ldx, double eps_sv, int r_max,
                                                    double* sig_sorted, int* perm, int* r_new,
                                                    double* sig_tmp, int32_t* err) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = warp; c < n; c += nw) {
        double acc = 0.0;
        for (int r = lane; r < m; r += 32) {
            const double v = X[r + (int64_t)c * ldx];
            acc = fma(v, v, acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) sig_tmp[c] = sqrt(acc);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const double sc = sig_tmp[c];
        if (!isfinite(sc)) st_dev_error(err, ST_ERR_NONFINITE);
        int rank = 0;
        for (int d = 0; d < n; ++d) {
            const double sd = sig_tmp[d];
            rank += (sd > sc) || (sd == sc && d < c);
        }
        perm[rank] = c;
        sig_sorted[rank] = sc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double smax = n > 0 ? sig_sorted[0] : 0.0;
        int keep = 0;
        while (keep < n && keep < r_max && sig_sorted[keep] > eps_sv * smax && sig_sorted[keep] > 0.0)
            ++keep;
        *r_new = keep;
    }
}

// Kept singular vectors of the middle matrix Q = (Pi U_z) Sigma (Q1 Y)^T:
//   Ysel[piv[j], q] = Z[j, perm[q]] / sigma_q        (left, n x rk)
//   Vsel[:, q] = [Y[:, perm[q]]; 0]                  (right before Q1, m x rk)
__global__ void gather_kernel(int n, int m, int rk, const int* __restrict__ perm,
                              const int* __restrict__ piv, const double* __restrict__ sig,
                              const double* __restrict__ Y, int ldy, const double* __restrict__ Z,
                              int ldz, double* Ysel, int ldys, double* Vsel, int ldvs) {
    const int64_t t1 = (int64_t)n * rk, t2 = (int64_t)m * rk;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < t1 + t2;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < t1) {
            const int j = (int)(t % n), q = (int)(t / n);
            Ysel[piv[j] + (int64_t)q * ldys] = Z[j + (int64_t)perm[q] * ldz] / sig[q];
        } else {
            const int64_t u = t - t1;
            const int i = (int)(u % m), q = (int)(u / m);
            Vsel[i + (int64_t)q * ldvs] = i < n ? Y[i + (int64_t)perm[q] * ldy] : 0.0;
        }
    }
}

__global__ void dot_kernel(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                           double* out) {
    __shared__ double s_part[NWARP];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += NT) acc = fma(x[i], y[i], acc);
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < NWARP; ++w) s += s_part[w];
        *out = s;
    }
}

// ---------------------------------------------------------------------------
// Temporal bases: block i factorises Upsilon_i (Nt x nmu) in shared memory.
__global__ void __launch_bounds__(512) temporal_kernel(int Nt, int nmu, int ns, int nt,
                                                       const double* __restrict__ V, int64_t ldv,
                                                       double* T, int max_sweeps, double tol,
                                                       int32_t* err) {
    extern __shared__ double sm[];
    double* X = sm;                       // Nt x nmu
    double* nrm = sm + (size_t)Nt * nmu;  // nmu
    __shared__ int s_rot;
    __shared__ int s_perm[64];
    const int i = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int t = threadIdx.x; t < Nt * nmu; t += blockDim.x) {
        const int k = t % Nt, p = t / Nt;
        X[t] = V[(int64_t)p * Nt + k + (int64_t)i * ldv];
    }
    __syncthreads();
    const int np = nmu + (nmu & 1), npairs = np / 2;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) s_rot = 0;
        __syncthreads();
        for (int t = 0; t < np - 1; ++t) {
            for (int q = warp; q < npairs; q += nw) {
                int a, b;
                if (q == 0) { a = t; b = np - 1; }
                else { a = (t + q) % (np - 1); b = (t - q + np - 1) % (np - 1); }
                if (a >= nmu || b >= nmu) continue;
                double* xa = X + (size_t)a * Nt;
                double* xb = X + (size_t)b * Nt;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int r = lane; r < Nt; r += 32) {
                    al = fma(xa[r], xa[r], al);
                    be = fma(xb[r], xb[r], be);
                    ga = fma(xa[r], xb[r], ga);
                }
                al = warp_sum(al);
                be = warp_sum(be);
                ga = warp_sum(ga);
                if (ga != 0.0 && jacobi_rotates(al, be, ga, tol)) {
                    double c, s;
                    jacobi_pair_rot(al, be, ga, c, s);
                    for (int r = lane; r < Nt; r += 32) {
                        const double u = xa[r], v = xb[r];
                        xa[r] = c * u - s * v;
                        xb[r] = s * u + c * v;
                    }
                    if (lane == 0) s_rot = 1;
                }
            }
            __syncthreads();
        }
        if (!s_rot) break;
        __syncthreads();
    }
    if (sweep >= max_sweeps && threadIdx.x == 0) st_dev_error(err, ST_ERR_NOT_CONVERGED);
    for (int c = warp; c < nmu; c += nw) {
        double acc = 0.0;
        for (int r = lane; r < Nt; r += 32) acc = fma(X[c * Nt + r], X[c * Nt + r], acc);
        acc = warp_sum(acc);
        if (lane == 0) nrm[c] = sqrt(acc);
    }
    __syncthreads();
    if (threadIdx.x < nmu) {
        const int c = threadIdx.x;
        int rank = 0;
        for (int d = 0; d < nmu; ++d) rank += (nrm[d] > nrm[c]) || (nrm[d] == nrm[c] && d < c);
        s_perm[rank] = c;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < Nt * nt; t += blockDim.x) {
        const int k = t % Nt, j = t / Nt;
        const int c = s_perm[j];
        const double sv = nrm[c];
        T[k + (int64_t)(i + ns * j) * Nt] = sv > 0.0 ? X[c * Nt + k] / sv : 0.0;
    }
}

int grid_for(st_model* m, int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8 * m->num_sms));
}

}  // namespace

namespace {

// Grow buf to at least `bytes`, keeping its first keep_bytes (st_grow drops
// the contents).
st_status grow_keep(st_model* m, DevBuf& buf, size_t bytes, size_t keep_bytes) {
    if (bytes <= buf.bytes) return ST_OK;
    void* p = nullptr;
    const size_t want = bytes + bytes / 8 + 256;
    ST_CUDA_TRY(cudaMalloc(&p, want));
    if (buf.p && keep_bytes)
        ST_CUDA_TRY(cudaMemcpyAsync(p, buf.p, std::min(keep_bytes, buf.bytes), cudaMemcpyDeviceToDevice, m->stream));
    if (buf.p) {
        ST_CUDA_TRY(cudaStreamSynchronize(m->stream));
        ST_CUDA_TRY(cudaFree(buf.p));
    }
    buf.p = p;
    buf.bytes = want;
    return ST_OK;
}

// Make room for the state: W (N x wcols) keeping its r columns, and V with
// a leading dimension of at least ldv_min rows and vcols columns, keeping its
// pod_rows x r block.
st_status pod_reserve(st_model* m, int wcols, int64_t ldv_min, int vcols) {
    const int64_t N = m->N;
    const int r = m->pod_r;
    ST_TRY(grow_keep(m, m->W, sizeof(double) * N * wcols, sizeof(double) * N * r));
    if (m->pod_ldv >= ldv_min && m->V.bytes >= sizeof(double) * (size_t)m->pod_ldv * vcols) return ST_OK;
    const int64_t ld = std::max(ldv_min, m->pod_ldv);
    void* p = nullptr;
    const size_t want = sizeof(double) * (size_t)ld * std::max(vcols, 1) + 256;
    ST_CUDA_TRY(cudaMalloc(&p, want));
    if (m->V.p && r > 0 && m->pod_rows > 0)
        ST_CUDA_TRY(cudaMemcpy2DAsync(p, sizeof(double) * ld, m->V.p, sizeof(double) * m->pod_ldv,
                                      sizeof(double) * m->pod_rows, r, cudaMemcpyDeviceToDevice, m->stream));
    if (m->V.p) {
        ST_CUDA_TRY(cudaStreamSynchronize(m->stream));
        ST_CUDA_TRY(cudaFree(m->V.p));
    }
    m->V.p = p;
    m->V.bytes = want;
    m->pod_ldv = ld;
    return ST_OK;
}

void pod_clear(st_model* m) {
    m->pod_r = 0;
    m->pod_rows = 0;
    m->sigma.clear();
    m->pod_sweeps.clear();
    m->pod_reorth = 0;
}

// Updates of the incremental SVD held by the model (W, sigma, V, r, rows)
// with the ncols_all columns at `snapshots` (N x ncols_all, column major),
// bcols columns per update (the last one may be narrower).
st_status pod_update_impl(st_model* m, int64_t ncols_all, const double* snapshots, int bcols) {
    const int64_t N = m->N;
    int r = m->pod_r;
    int64_t rows = m->pod_rows;
    // rank cap; a state installed with more columns keeps them until the
    // next truncation
    const int rmax = (int)std::min<int64_t>(m->opt.r_max, N);
    const int rcap = std::max(rmax, r);
    bcols = (int)std::min<int64_t>(bcols, ncols_all);
    const int bmax = bcols;  // widest block
    const int cap = rcap + bmax;
    ST_TRY(pod_reserve(m, cap, rows + ncols_all, rcap));
    const int64_t ldv = m->pod_ldv;
    const int pdim = std::max(bmax, rcap);
    cudaStream_t st = m->stream;
    st_oz_invalidate(m);

    // buffers
    const size_t szW2 = (size_t)N * cap, szV2 = (size_t)ldv * rcap, szE = (size_t)N * bmax,
                 szL = (size_t)rcap * bmax, szP = (size_t)pdim * pdim, szX = (size_t)cap * cap;
    // Gram-Schmidt kernel: one block per SM, gs_rs rows each
    const int gs_blocks = (int)std::min<int64_t>(m->num_sms, std::max<int64_t>(1, N / 64));
    const int64_t gs_rs = (N + gs_blocks - 1) / gs_blocks;
    int gs_smem_max = 0;
    {
        int dev = 0;
        ST_CUDA_TRY(cudaGetDevice(&dev));
        ST_CUDA_TRY(cudaDeviceGetAttribute(&gs_smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    }
    // launch of gs2_kernel on g.m columns: the block's rows of three columns
    // of E in shared memory when they fit, and as many directions as fit.
    // The function attributes are set (and the fit checked) once per shared
    // memory size: the launches follow host synchronisations, so host calls
    // here delay the GPU.
    size_t gs_smem_set[2] = {0, 0};  // dynamic shared memory set for gs2_kernel<false>, <true>
    int64_t gs_static = 0;
    {
        cudaFuncAttributes fa{};
        ST_CUDA_TRY(cudaFuncGetAttributes(&fa, gs2_kernel<true>));
        gs_static = (int64_t)fa.sharedSizeBytes;
    }
    auto launch_gs2 = [&](Gs2Args g) -> st_status {
        const int64_t budget = (int64_t)gs_smem_max - gs_static;
        const int64_t col = (int64_t)sizeof(double) * gs_rs;
        const int64_t base = (int64_t)sizeof(double) * 4 * g.m;
        const bool e_smem = base + 3 * col <= budget;
        const int64_t room = budget - base - (e_smem ? 3 * col : 0);
        g.rs = gs_rs;
        g.ks = (int)std::max<int64_t>(0, std::min<int64_t>(g.m, room / col));
        const size_t smem = gs2_smem(g.m, gs_rs, e_smem, g.ks);
        const void* fn = e_smem ? (const void*)gs2_kernel<true> : (const void*)gs2_kernel<false>;
        if (gs_smem_set[e_smem] < smem) {
            ST_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            int per_sm = 0;
            ST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, smem));
            if (per_sm < 1)
                return st_fail(ST_ERR_CUDA, "st_rom_build_basis: Gram-Schmidt kernel does not fit an SM");
            gs_smem_set[e_smem] = smem;
        }
        void* args[] = {&g};
        ST_PROF(m, "gs2_kernel");
        ST_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(gs_blocks), dim3(NT), args, smem, st));
        st_count_launch();
        return ST_OK;
    };
    const size_t szPart = std::max((size_t)2 * std::max(gs_blocks, 1) * (pdim + 2), (size_t)64 * bmax);
    const size_t szPan = (size_t)pdim * kGsPanel + 4 * (size_t)kGsPanel * kGsPanel;
    const size_t doubles = szW2 + szV2 + szE + 2 * szL + 3 * szP + 3 * szX + (size_t)cap * rcap * 2 +
                           szPart + pdim + 9 * cap + szPan + 32;
    ST_TRY(st_grow(m, m->ws_pod, sizeof(double) * doubles + sizeof(int) * (2 * cap + 16)));
    double* W2 = (double*)m->ws_pod.p;
    double* V2 = W2 + szW2;
    double* E = V2 + szV2;
    double* L = E + szE;
    double* L2 = L + szL;
    double* P = L2 + szL;
    double* P1 = P + szP;
    double* P2 = P1 + szP;
    double* X = P2 + szP;
    double* Y = X + szX;
    double* Z = Y + szX;
    double* Ysel = Z + szX;
    double* Vsel = Ysel + (size_t)cap * rcap;
    double* partial = Vsel + (size_t)cap * rcap;
    // Gram-Schmidt panel workspace: H [pdim x panel] projections of a panel
    // on the earlier directions, G, R, Rinv, Pt [panel x panel]
    double* gsH = partial + szPart;
    double* gsG = gsH + (size_t)pdim * kGsPanel;
    double* gsR = gsG + (size_t)kGsPanel * kGsPanel;
    double* gsRi = gsR + (size_t)kGsPanel * kGsPanel;
    double* gsPt = gsRi + (size_t)kGsPanel * kGsPanel;
    double* q_beta = partial + szPart + szPan;  // [cap] R diagonal of the pivoted QR
    double* q_tau = q_beta + cap;        // [cap] Householder coefficients
    double* q_scale = q_tau + cap;       // [cap] 1 / (x_k - beta_k)
    double* q_nrm = q_scale + cap;       // [2 cap] QR trailing norms (double buffered), then the Jacobi sweep-start norms and block counters
    double* d_sig = q_nrm + 2 * cap;     // [cap] current sigma (device copy)
    double* d_sig_sorted = d_sig + cap;  // [cap]
    double* d_sig_tmp = d_sig_sorted + cap;
    double* d_scalar = d_sig_tmp + cap + 8;  // [16]: tau, dot (d_sig_tmp[cap] is the Jacobi norm max)
    int* d_int = (int*)(d_scalar + 16);  // [16]: k, r_new, sweeps, flags[3], -, panel Cholesky failure, big[3]
    int* d_perm = d_int + 16;            // [cap]
    int* d_piv = d_perm + cap;           // [cap] column pivots of the QR
    unsigned long long* d_rot = reinterpret_cast<unsigned long long*>(d_scalar + 4);
    // Gram-Schmidt multiply-adds per row, accumulated over the update (profiling)
    unsigned long long* d_gs_work = reinterpret_cast<unsigned long long*>(d_scalar + 5);
    ST_CUDA_TRY(cudaMemsetAsync(d_gs_work, 0, sizeof(unsigned long long), st));
    double* W = (double*)m->W.p;
    double* V = (double*)m->V.p;

    const GridBarrier bar{m->d_bar, m->d_bar + 1, m->d_bar + 2, m->d_err, m->opt.spin_limit};
    // pivoted Householder QR of the transposed middle matrix
    auto run_qrp = [&](int mrows, int ncols) -> st_status {
        const size_t smem = sizeof(double) * mrows;
        if (smem > 48 * 1024)
            ST_CUDA_TRY(cudaFuncSetAttribute(qrp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        ST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qrp_kernel, QT, smem));
        if (per_sm < 1) return st_fail(ST_ERR_CUDA, "st_rom_build_basis: QR kernel does not fit on an SM");
        const int qb = std::max(1, std::min({per_sm * m->num_sms, m->num_sms, (ncols + 1) / 2}));
        ST_CUDA_TRY(cudaMemsetAsync(m->d_bar, 0, sizeof(unsigned int) * 4, st));
        QrpArgs qa{mrows, ncols, X, cap, q_beta, q_tau, q_scale, d_piv, q_nrm, bar};
        void* args[] = {&qa};
        ST_PROF(m, "qrp_kernel");
        ST_CUDA_TRY(cudaLaunchCooperativeKernel((void*)qrp_kernel, dim3(qb), dim3(QT), args, smem, st));
        st_count_launch();
        double fl = 0.0;
        for (int kk = 0; kk < ncols; ++kk) fl += 2.0 * (mrows - kk) + 6.0 * (ncols - kk - 1) * (mrows - kk);
        st_prof_flops(m, "qrp_kernel", fl + 2.0 * mrows * ncols);
        return ST_OK;
    };
    // middle-matrix SVD: KB columns per Jacobi block, fewer where the staged
    // columns would not fit in shared memory
    auto run_jacobi = [&](int mrows, int ncols) -> st_status {
        int kb = ST_JACOBI_KB;
        while (kb > 1 && jacobi_smem(kb, mrows, ncols) > kJacobiSmemMax) kb /= 2;
        const size_t smem = jacobi_smem(kb, mrows, ncols);
        if (smem > kJacobiSmemMax)
            return st_fail(ST_ERR_ARG, "st_rom_build_basis: r_max + Nt too large for the middle-matrix SVD");
        const void* fn = kb == 4 ? (const void*)jacobi_kernel<4>
                       : kb == 2 ? (const void*)jacobi_kernel<2> : (const void*)jacobi_kernel<1>;
        ST_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        ST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * JW, smem));
        if (per_sm < 1) return st_fail(ST_ERR_CUDA, "st_rom_build_basis: Jacobi kernel does not fit on an SM");
        const int nb = (ncols + kb - 1) / kb;
        const int npairs = (nb + (nb & 1)) / 2;
        const int jb = std::max(1, std::min(per_sm * m->num_sms, npairs));
        ST_CUDA_TRY(cudaMemsetAsync(d_int + 3, 0, sizeof(int) * 3, st));
        ST_CUDA_TRY(cudaMemsetAsync(d_int + 8, 0, sizeof(int) * 3, st));
        ST_CUDA_TRY(cudaMemsetAsync(m->d_bar, 0, sizeof(unsigned int) * 4, st));
        // the largest squared column norm is accumulated with atomicMax from zero
        ST_CUDA_TRY(cudaMemsetAsync(d_sig_tmp + ncols, 0, sizeof(double), st));
        ST_CUDA_TRY(cudaMemsetAsync(d_rot, 0, sizeof(unsigned long long), st));
        // the block readiness counters live in the second half of the QR norms
        unsigned int* d_ready = reinterpret_cast<unsigned int*>(q_nrm + cap);
        ST_CUDA_TRY(cudaMemsetAsync(d_ready, 0, sizeof(unsigned int) * nb, st));
        // Z = R^T: stop when every pair of columns is orthogonal to
        // sqrt(m) * eps relative (the left singular vectors of the middle
        // matrix are these columns, normalised)
        JacArgs ja{mrows, ncols, Z, cap, Y, cap, m->opt.jacobi_sweeps,
                   std::sqrt((double)mrows) * 2.220446049250313e-16, d_int + 3, d_int + 8, d_int + 2, d_sig_tmp,
                   q_nrm, 0.1 * m->opt.eps_sv, d_rot, d_ready, bar};
        void* args[] = {&ja};
        ST_PROF(m, "jacobi_kernel");
        ST_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(jb), dim3(32 * JW), args, smem, st));
        st_count_launch();
        return ST_OK;
    };
    std::vector<double> h_sig;
    // the singular values of the state on the device
    if (r > 0)
        ST_CUDA_TRY(cudaMemcpyAsync(d_sig, m->sigma.data(), sizeof(double) * r, cudaMemcpyHostToDevice, st));
    auto read_k = [&](int* out) -> st_status {
        ST_CUDA_TRY(cudaMemcpyAsync(out, d_int, sizeof(int), cudaMemcpyDeviceToHost, st));
        ST_CUDA_TRY(cudaStreamSynchronize(st));
        int32_t herr = 0;
        ST_CUDA_TRY(cudaMemcpy(&herr, m->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (herr) return st_fail(herr, "st_rom_build_basis: Gram-Schmidt failed (%s)", st_status_string(herr));
        return ST_OK;
    };
    // E (N x mcols) = J P with the column-wise CGS2 semantics (a column adds
    // a direction when its remainder exceeds tau), by panels of kGsPanel
    // columns.  A panel is projected twice on the directions J0 found before
    // it with GEMMs, then the cooperative kernel orthogonalises its columns
    // among themselves.  A direction normalised from a small remainder
    // carries rounding along J0 amplified by the normalisation, so the
    // panel's new directions Jn are projected on J0 once more (H3 = J0^T Jn,
    // Jn -= J0 H3) and re-orthonormalised by Cholesky QR (Jn = Jn' R):
    // E_panel = J0 (P0 + H3 Pn) + Jn' (R Pn).  P: column j at Pout + j * ldp;
    // *k_total receives the number of directions.
    auto gs_block = [&](double* Ein, int mcols, double* Jout, double* Pout, int ldp, const double* tau,
                        int* k_total) -> st_status {
        ST_CUDA_TRY(cudaMemsetAsync(Pout, 0, sizeof(double) * (size_t)ldp * mcols, st));
        ST_CUDA_TRY(cudaMemsetAsync(d_int + 7, 0, sizeof(int), st));
        int k = 0;
        for (int c0 = 0; c0 < mcols; c0 += kGsPanel) {
            const int pw = std::min(kGsPanel, mcols - c0);
            double* Ep = Ein + (size_t)c0 * N;
            double* Pp = Pout + (size_t)c0 * ldp;
            if (k > 0) {
                // J0 is the same matrix in all four products: its digit
                // planes (tensor-core path) are made once per layout
                ST_TRY(st_dgemm_slot(m, 0, false, true, false, k, pw, N, 1.0, Jout, N, Ep, N, 0.0, Pp, ldp));
                ST_TRY(st_dgemm_slot(m, 1, false, false, false, N, pw, k, -1.0, Jout, N, Pp, ldp, 1.0, Ep, N));
                ST_TRY(st_dgemm_slot(m, 0, true, true, false, k, pw, N, 1.0, Jout, N, Ep, N, 0.0, gsH, k));
                ST_TRY(st_dgemm_slot(m, 1, true, false, false, N, pw, k, -1.0, Jout, N, gsH, k, 1.0, Ep, N));
                add_block_kernel<<<grid_for(m, (int64_t)k * pw), 256, 0, st>>>(k, pw, gsH, k, Pp, ldp);
                ST_TRY(st_check_launch("add_block"));
            }
            ST_CUDA_TRY(cudaMemsetAsync(m->d_bar, 0, sizeof(unsigned int) * 4, st));
            double* Jn = Jout + (size_t)k * N;
            ST_TRY(launch_gs2(Gs2Args{N, pw, Ep, Jn, Pp + k, ldp, d_int, tau, partial, d_gs_work, bar, 0, 0}));
            int kp = 0;
            ST_TRY(read_k(&kp));
            if (k > 0 && kp > 0) {
                // Jn -= J0 (J0^T Jn); Jn = Jn' R; P0 += H3 Pn; Pn = R Pn
                ST_TRY(st_dgemm_slot(m, 0, true, true, false, k, kp, N, 1.0, Jout, N, Jn, N, 0.0, gsH, k));
                ST_TRY(st_dgemm_slot(m, 1, true, false, false, N, kp, k, -1.0, Jout, N, gsH, k, 1.0, Jn, N));
                ST_TRY(st_dgemm(m, true, false, kp, kp, N, 1.0, Jn, N, Jn, N, 0.0, gsG, kp));
                {
                    ST_PROF(m, "chol_inv_kernel");
                    chol_inv_kernel<<<1, NT, 0, st>>>(kp, gsG, gsR, kGsPanel, gsRi, d_int + 7);
                    ST_TRY(st_check_launch("chol_inv panel"));
                }
                ST_TRY(st_dgemm(m, false, false, N, kp, kp, 1.0, Jn, N, gsRi, kp, 0.0, Ep, N));
                ST_CUDA_TRY(cudaMemcpyAsync(Jn, Ep, sizeof(double) * (size_t)N * kp, cudaMemcpyDeviceToDevice, st));
                ST_TRY(st_dgemm(m, false, false, k, pw, kp, 1.0, gsH, k, Pp + k, ldp, 1.0, Pp, ldp));
                ST_TRY(st_dgemm(m, false, false, kp, pw, kp, 1.0, gsR, kGsPanel, Pp + k, ldp, 0.0, gsPt, kGsPanel));
                ST_CUDA_TRY(cudaMemcpy2DAsync(Pp + k, sizeof(double) * ldp, gsPt, sizeof(double) * kGsPanel,
                                              sizeof(double) * kp, pw, cudaMemcpyDeviceToDevice, st));
            }
            k += kp;
        }
        if (k > 0) {
            int fail = 0;
            ST_CUDA_TRY(cudaMemcpyAsync(&fail, d_int + 7, sizeof(int), cudaMemcpyDeviceToHost, st));
            ST_CUDA_TRY(cudaStreamSynchronize(st));
            if (fail)
                return st_fail(ST_ERR_BREAKDOWN, "st_rom_build_basis: panel re-orthonormalisation failed");
        }
        *k_total = k;
        return ST_OK;
    };
    for (int64_t c0 = 0; c0 < ncols_all; c0 += bcols) {
        const int bw = (int)std::min<int64_t>(bcols, ncols_all - c0);  // columns of this block
        const double* Up = snapshots + (size_t)c0 * N;
        {
            const int chunks = (int)std::max<int64_t>(1, std::min<int64_t>(64, N / 2048));
            ST_PROF(m, "colnorm_kernels");
            colnorm_part_kernel<<<dim3(bw, chunks), NT, 0, st>>>(N, Up, chunks, partial);
            ST_TRY(st_check_launch("colnorm_part"));
            colnorm_max_kernel<<<1, NT, 0, st>>>(bw, chunks, partial, m->opt.eps_svd, d_scalar);
            ST_TRY(st_check_launch("colnorm_max"));
        }
        ST_CUDA_TRY(cudaMemcpyAsync(E, Up, sizeof(double) * (size_t)N * bw, cudaMemcpyDeviceToDevice, st));
        double* J = W + (size_t)r * N;
        int k = 0;
        if (r > 0) {
            // first block pass: L = W^T U_p, E1 = U_p - W L, E1 = J1 P1
            ST_TRY(st_dgemm_slot(m, 2, false, true, false, r, bw, N, 1.0, W, N, Up, N, 0.0, L, rcap));
            ST_TRY(st_dgemm_slot(m, 3, false, false, false, N, bw, r, -1.0, W, N, L, rcap, 1.0, E, N));
            int k1 = 0;
            ST_TRY(gs_block(E, bw, J, P1, bw, d_scalar, &k1));
            if (k1 > 0) {
                // second block pass: L2 = W^T J1, E2 = J1 - W L2 = J P2 by Cholesky QR
                // (E2 is orthonormal up to the rounding carried along W, so its
                // Gram matrix is well conditioned); L += L2 P1, P = P2 P1
                ST_TRY(st_dgemm_slot(m, 2, true, true, false, r, k1, N, 1.0, W, N, J, N, 0.0, L2, rcap));
                ST_CUDA_TRY(cudaMemcpyAsync(E, J, sizeof(double) * N * k1, cudaMemcpyDeviceToDevice, st));
                ST_TRY(st_dgemm_slot(m, 3, true, false, false, N, k1, r, -1.0, W, N, L2, rcap, 1.0, E, N));
                ST_TRY(st_dgemm(m, true, false, k1, k1, N, 1.0, E, N, E, N, 0.0, Y, k1));
                ST_CUDA_TRY(cudaMemsetAsync(d_int + 6, 0, sizeof(int), st));
                {
                    ST_PROF(m, "chol_inv_kernel");
                    chol_inv_kernel<<<1, NT, 0, st>>>(k1, Y, P2, k1, X, d_int + 6);
                    ST_TRY(st_check_launch("chol_inv"));
                }
                int chol_fail = 0;
                ST_CUDA_TRY(cudaMemcpyAsync(&chol_fail, d_int + 6, sizeof(int), cudaMemcpyDeviceToHost, st));
                ST_CUDA_TRY(cudaStreamSynchronize(st));
                if (!chol_fail) {
                    ST_TRY(st_dgemm(m, false, false, N, k1, k1, 1.0, E, N, X, k1, 0.0, J, N));
                    k = k1;
                } else {
                    ST_TRY(gs_block(E, k1, J, P2, k1, nullptr, &k));
                }
                ST_TRY(st_dgemm(m, false, false, r, bw, k1, 1.0, L2, rcap, P1, bw, 1.0, L, rcap));
                if (k > 0) ST_TRY(st_dgemm(m, false, false, k, bw, k1, 1.0, P2, k1, P1, bw, 0.0, P, bw));
            }
        } else {
            ST_TRY(gs_block(E, bw, J, P, bw, d_scalar, &k));
        }
        const int mrows = r + bw, ncols = r + k;
        if (ncols == 0) {  // nothing to add: the block is zero and W is empty
            rows += bw;
            continue;
        }
        // middle matrix, transposed: X = Q^T (mrows x ncols); pivoted QR
        // X Pi = Q1 R, then one-sided Jacobi on Z = R^T with rotations
        // accumulated in Y:  Q = (Pi U_z) Sigma (Q1 Y)^T
        build_qt_kernel<<<grid_for(m, (int64_t)mrows * ncols), 256, 0, st>>>(r, k, bw, d_sig, L, rcap, P, bw, X, cap);
        ST_TRY(st_check_launch("build_qt"));
        ST_TRY(run_qrp(mrows, ncols));
        build_rt_kernel<<<grid_for(m, (int64_t)ncols * ncols), 256, 0, st>>>(ncols, X, cap, d_piv, q_beta, Z, cap, Y, cap);
        ST_TRY(st_check_launch("build_rt"));
        ST_TRY(run_jacobi(ncols, ncols));
        {
            ST_PROF(m, "sort_kernel");
            sort_kernel<<<1, 1024, 0, st>>>(ncols, ncols, Z, cap, m->opt.eps_sv, rmax, d_sig_sorted,
                                            d_perm, d_int + 1, d_sig_tmp, m->d_err);
            ST_TRY(st_check_launch("sort"));
        }
        int rs[2] = {0, 0};  // r_new, sweeps
        unsigned long long nrot = 0;
        ST_CUDA_TRY(cudaMemcpyAsync(rs, d_int + 1, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
        ST_CUDA_TRY(cudaMemcpyAsync(&nrot, d_rot, sizeof(nrot), cudaMemcpyDeviceToHost, st));
        ST_CUDA_TRY(cudaStreamSynchronize(st));
        const int rnew = rs[0];
        m->pod_sweeps.push_back(rs[1]);
        // algorithmic work: per sweep the column norms (2 m n) and a dot
        // product per pair (2 m); per rotation 6 (m + n)
        st_prof_flops(m, "jacobi_kernel",
                      rs[1] * (2.0 * ncols * ncols + (double)ncols * (ncols - 1) * ncols) +
                          12.0 * (double)nrot * ncols);
        {
            int32_t herr = 0;
            ST_CUDA_TRY(cudaMemcpy(&herr, m->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
            if (herr) return st_fail(herr, "st_rom_build_basis: middle-matrix SVD failed (%s)", st_status_string(herr));
        }
        if (rnew == 0) {
            rows += bw;
            r = 0;
            continue;
        }
        gather_kernel<<<grid_for(m, (int64_t)(ncols + mrows) * rnew), 256, 0, st>>>(
            ncols, mrows, rnew, d_perm, d_piv, d_sig_sorted, Y, cap, Z, cap, Ysel, cap, Vsel, cap);
        ST_TRY(st_check_launch("gather"));
        {
            // Vsel <- Q1 Vsel = H_0 ... H_{n-1} Vsel in blocks of kWy
            // reflectors in the compact WY form Q_b = I - Y_b T_b Y_b^T, last
            // block first: Vsel -= Y_b (T_b (Y_b^T Vsel)), the products on the
            // FP64 GEMM path.  Z (free after the gather) holds the
            // reflectors; the block temporaries live in ws_pod2 (used
            // otherwise only by the assembly).
            constexpr int kWy = 64;
            double* Yall = Z;  // [mrows x ncols], ld cap
            ST_TRY(st_grow(m, m->ws_pod2, sizeof(double) * (2 * (size_t)kWy * rnew + 2 * (size_t)kWy * kWy)));
            double* Wt = (double*)m->ws_pod2.p;           // [kWy x rnew]
            double* Wt2 = Wt + (size_t)kWy * rnew;        // [kWy x rnew]
            double* Gb = Wt2 + (size_t)kWy * rnew;        // [kWy x kWy]
            double* Tb = Gb + (size_t)kWy * kWy;          // [kWy x kWy]
            {
                ST_PROF(m, "apply_q_wy_kernels");
                build_wy_kernel<<<grid_for(m, (int64_t)mrows * ncols), 256, 0, st>>>(mrows, ncols, X, cap, d_piv,
                                                                                   q_tau, q_scale, Yall, cap);
                ST_TRY(st_check_launch("build_wy"));
            }
            for (int k0 = ((ncols - 1) / kWy) * kWy; k0 >= 0; k0 -= kWy) {
                const int b = std::min(kWy, ncols - k0), rows_b = mrows - k0;
                const double* Yb = Yall + k0 + (size_t)k0 * cap;  // rows k0.. (zero above)
                ST_TRY(st_dgemm(m, true, false, b, b, rows_b, 1.0, Yb, cap, Yb, cap, 0.0, Gb, kWy));
                {
                    ST_PROF(m, "apply_q_wy_kernels");
                    larft_kernel<<<1, 64, 0, st>>>(b, Gb, kWy, q_tau + k0, Tb, kWy);
                    ST_TRY(st_check_launch("larft"));
                }
                ST_TRY(st_dgemm(m, true, false, b, rnew, rows_b, 1.0, Yb, cap, Vsel + k0, cap, 0.0, Wt, kWy));
                ST_TRY(st_dgemm(m, false, false, b, rnew, b, 1.0, Tb, kWy, Wt, kWy, 0.0, Wt2, kWy));
                ST_TRY(st_dgemm(m, false, false, rows_b, rnew, b, -1.0, Yb, cap, Wt2, kWy, 1.0, Vsel + k0, cap));
            }
        }
        // W2 = [W J] Ysel
        ST_TRY(st_dgemm(m, false, false, N, rnew, ncols, 1.0, W, N, Ysel, cap, 0.0, W2, N));
        // V2 = blkdiag(V, I) Vsel
        if (r > 0 && rows > 0)
            ST_TRY(st_dgemm(m, false, false, rows, rnew, r, 1.0, V, ldv, Vsel, cap, 0.0, V2, ldv));
        else if (rows > 0)  // earlier columns added no direction: their rows of V are zero
            ST_CUDA_TRY(cudaMemset2DAsync(V2, sizeof(double) * ldv, 0, sizeof(double) * rows, rnew, st));
        ST_CUDA_TRY(cudaMemcpy2DAsync(V2 + rows, sizeof(double) * ldv, Vsel + r, sizeof(double) * cap,
                                      sizeof(double) * bw, rnew, cudaMemcpyDeviceToDevice, st));
        ST_CUDA_TRY(cudaMemcpyAsync(W, W2, sizeof(double) * N * rnew, cudaMemcpyDeviceToDevice, st));
        ST_CUDA_TRY(cudaMemcpy2DAsync(V, sizeof(double) * ldv, V2, sizeof(double) * ldv,
                                      sizeof(double) * (rows + bw), rnew, cudaMemcpyDeviceToDevice, st));
        ST_CUDA_TRY(cudaMemcpyAsync(d_sig, d_sig_sorted, sizeof(double) * rnew, cudaMemcpyDeviceToDevice, st));
        r = rnew;
        rows += bw;
        // orthogonality check of Algorithm 2 and QR re-orthogonalisation
        if (r > 1) {
            dot_kernel<<<1, NT, 0, st>>>(N, W, W + (size_t)(r - 1) * N, d_scalar + 1);
            ST_TRY(st_check_launch("dot"));
            double dotv = 0.0;
            ST_CUDA_TRY(cudaMemcpyAsync(&dotv, d_scalar + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
            ST_CUDA_TRY(cudaStreamSynchronize(st));
            if (std::fabs(dotv) > std::min(m->opt.eps_svd, 2.220446049250313e-16 * (double)N)) {
                ++m->pod_reorth;
                ST_CUDA_TRY(cudaMemsetAsync(P, 0, sizeof(double) * (size_t)r * r, st));
                ST_CUDA_TRY(cudaMemsetAsync(m->d_bar, 0, sizeof(unsigned int) * 4, st));
                ST_TRY(launch_gs2(Gs2Args{N, r, W, W2, P, r, d_int, nullptr, partial, d_gs_work, bar, 0, 0}));
                ST_CUDA_TRY(cudaMemcpyAsync(W, W2, sizeof(double) * N * r, cudaMemcpyDeviceToDevice, st));
            }
        }
    }
    h_sig.resize(std::max(r, 1));
    unsigned long long gs_work = 0;
    ST_CUDA_TRY(cudaMemcpyAsync(&gs_work, d_gs_work, sizeof(gs_work), cudaMemcpyDeviceToHost, st));
    if (r > 0) ST_CUDA_TRY(cudaMemcpyAsync(h_sig.data(), d_sig, sizeof(double) * r, cudaMemcpyDeviceToHost, st));
    ST_CUDA_TRY(cudaStreamSynchronize(st));
    st_prof_flops(m, "gs2_kernel", 2.0 * (double)N * (double)gs_work);
    m->pod_r = r;
    m->pod_rows = rows;
    m->sigma.assign(h_sig.begin(), h_sig.begin() + r);
    return ST_OK;
}

// Phi_s = W(:, 1:ns) and the temporal bases of the state's V read as n_mu
// blocks of Nt rows (Eqs. spatialincrementalbasis, incrementaltemporalsnapshotmat,
// temporalincrementalbasis).
st_status pod_finish_impl(st_model* m, int n_mu, int Nt, int ns, int nt) {
    const int64_t N = m->N;
    const int r = m->pod_r;
    cudaStream_t st = m->stream;
    if (ns > r) return st_fail(ST_ERR_ARG, "st_rom_build_basis: ns = %d exceeds the rank %d", ns, r);
    if ((int64_t)n_mu * Nt != m->pod_rows)
        return st_fail(ST_ERR_ARG, "st_pod_finish: n_mu * Nt = %lld differs from the %lld snapshot columns consumed",
                       (long long)n_mu * Nt, (long long)m->pod_rows);
    const size_t smem = sizeof(double) * ((size_t)Nt * n_mu + n_mu);
    if (smem > 220 * 1024) return st_fail(ST_ERR_ARG, "st_rom_build_basis: Nt * n_mu too large for the temporal SVD");
    st_internal_free_basis(m);
    ST_CUDA_TRY(cudaMalloc(&m->d_phi, sizeof(double) * N * ns));
    ST_CUDA_TRY(cudaMalloc(&m->d_T, sizeof(double) * (size_t)Nt * ns * nt));
    ST_CUDA_TRY(cudaMemcpyAsync(m->d_phi, m->W.p, sizeof(double) * N * ns, cudaMemcpyDeviceToDevice, st));
    {
        if (smem > 48 * 1024)
            ST_CUDA_TRY(cudaFuncSetAttribute(temporal_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ST_PROF(m, "temporal_kernel");
        temporal_kernel<<<ns, 512, smem, st>>>(Nt, n_mu, ns, nt, (const double*)m->V.p, m->pod_ldv, m->d_T,
                                               m->opt.jacobi_sweeps, std::sqrt((double)Nt) * 2.220446049250313e-16,
                                               m->d_err);
        ST_TRY(st_check_launch("temporal"));
    }
    m->ns = ns;
    m->nt = nt;
    m->Nt = Nt;
    return ST_OK;
}

}  // namespace

extern "C" st_status st_pod_reset(st_model* m) {
    if (!m) return st_fail(ST_ERR_ARG, "st_pod_reset: NULL model");
    pod_clear(m);
    return ST_OK;
}

extern "C" st_status st_pod_update(st_model* m, int64_t n_cols, const double* snapshots, int32_t cols_per_update) {
    if (!m) return st_fail(ST_ERR_ARG, "st_pod_update: NULL model");
    if (n_cols < 0 || (n_cols > 0 && !snapshots) || cols_per_update < 1)
        return st_fail(ST_ERR_ARG, "st_pod_update: bad arguments");
    if (n_cols == 0) return ST_OK;
    return pod_update_impl(m, n_cols, snapshots, cols_per_update);
}

extern "C" st_status st_pod_finish(st_model* m, int32_t n_mu, int32_t Nt, int32_t ns, int32_t nt) {
    if (!m) return st_fail(ST_ERR_ARG, "st_pod_finish: NULL model");
    if (n_mu < 1 || Nt < 1 || ns < 1 || nt < 1 || nt > Nt || nt > n_mu)
        return st_fail(ST_ERR_ARG, "st_pod_finish: bad sizes");
    return pod_finish_impl(m, n_mu, Nt, ns, nt);
}

extern "C" st_status st_pod_set_state(st_model* m, int32_t r, int64_t rows, const double* W, const double* sigma,
                                      const double* V) {
    if (!m) return st_fail(ST_ERR_ARG, "st_pod_set_state: NULL model");
    if (r < 0 || r > m->N || rows < 0 || (r > 0 && (!W || !sigma || (rows > 0 && !V))))
        return st_fail(ST_ERR_ARG, "st_pod_set_state: bad arguments");
    for (int i = 0; i < r; ++i)
        if (!(sigma[i] >= 0.0) || !std::isfinite(sigma[i]) || (i > 0 && sigma[i] > sigma[i - 1]))
            return st_fail(ST_ERR_ARG, "st_pod_set_state: sigma must be finite, non-negative and non-increasing");
    pod_clear(m);
    ST_TRY(pod_reserve(m, std::max(r, 1), std::max<int64_t>(rows, 1), std::max(r, 1)));
    if (r > 0) {
        ST_CUDA_TRY(cudaMemcpyAsync(m->W.p, W, sizeof(double) * m->N * r, cudaMemcpyDeviceToDevice, m->stream));
        if (rows > 0)
            ST_CUDA_TRY(cudaMemcpy2DAsync(m->V.p, sizeof(double) * m->pod_ldv, V, sizeof(double) * rows,
                                          sizeof(double) * rows, r, cudaMemcpyDeviceToDevice, m->stream));
        ST_CUDA_TRY(cudaStreamSynchronize(m->stream));
    }
    m->pod_r = r;
    m->pod_rows = rows;
    m->sigma.assign(sigma, sigma + r);
    st_oz_invalidate(m);
    return ST_OK;
}

extern "C" st_status st_rom_build_basis(st_model* m, int32_t n_mu, int32_t Nt, const double* snapshots,
                                        int32_t ns, int32_t nt, double* sigma_out, int32_t* rank_out) {
    if (!m) return st_fail(ST_ERR_ARG, "st_rom_build_basis: NULL model");
    if (!snapshots || n_mu < 1 || Nt < 1 || ns < 1 || nt < 1)
        return st_fail(ST_ERR_ARG, "st_rom_build_basis: bad arguments");
    if (nt > Nt || nt > n_mu) return st_fail(ST_ERR_ARG, "st_rom_build_basis: nt > min(Nt, n_mu)");
    if (n_mu > 64) return st_fail(ST_ERR_ARG, "st_rom_build_basis: at most 64 parameter samples");
    // one update takes the snapshots of pod_block parameter samples, or
    // pod_cols consecutive snapshot columns (1: the rank-one stream of
    // Algorithm 2)
    const int64_t ncols_all = (int64_t)n_mu * Nt;
    const int pb = std::min<int>(m->opt.pod_block, n_mu);
    const int bcols = m->opt.pod_cols > 0 ? (int)std::min<int64_t>(m->opt.pod_cols, ncols_all) : Nt * pb;
    st_internal_free_basis(m);
    pod_clear(m);
    // V's rows for the whole snapshot set at once
    ST_TRY(pod_reserve(m, 1, ncols_all, (int)std::min<int64_t>(m->opt.r_max, m->N)));
    ST_TRY(pod_update_impl(m, ncols_all, snapshots, bcols));
    const int r = m->pod_r;
    if (rank_out) *rank_out = r;
    if (sigma_out) for (int i = 0; i < r; ++i) sigma_out[i] = m->sigma[i];
    return pod_finish_impl(m, n_mu, Nt, ns, nt);
}
