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
//      thin SVD by one-sided (Hestenes) Jacobi in FP64 on Q^T, with rotations
//      accumulated to give the left singular vectors of Q;
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
    double* E;      // N x m (ld N), overwritten
    double* J;      // N x m (ld N) output directions
    double* P;      // m x m (ld m), zeroed by the host
    int* k_out;
    const double* tau;  // NULL: every column adds a direction
    double* partial;    // [grid x m]
    double* hbuf;       // [m]
    GridBarrier bar;
};

__global__ void __launch_bounds__(NT) gs2_kernel(Gs2Args a) {
    extern __shared__ double sm[];
    double* h = sm;          // [m]
    double* h2 = sm + a.m;   // [m]
    __shared__ double s_part[NWARP];
    __shared__ double s_nu;
    __shared__ int s_flag;
    const int G = gridDim.x, b = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t R = (a.N + G - 1) / G;
    const int64_t r0 = (int64_t)b * R, r1 = min(a.N, r0 + R);
    const double tau = a.tau ? *a.tau : -1.0;
    int k = 0;
    for (int j = 0; j < a.m; ++j) {
        double* e = a.E + (int64_t)j * a.N;
        for (int pass = 0; pass < 2; ++pass) {
            double* hh = pass == 0 ? h : h2;
            if (k > 0) {
                // partial projections J(:, c)^T e over this block's rows
                for (int c = warp; c < k; c += NWARP) {
                    const double* jc = a.J + (int64_t)c * a.N;
                    double acc = 0.0;
                    for (int64_t i = r0 + lane; i < r1; i += 32) acc = fma(__ldcg(jc + i), __ldcg(e + i), acc);
                    acc = warp_sum(acc);
                    if (lane == 0) __stcg(a.partial + (int64_t)b * a.m + c, acc);
                }
                if (!grid_sync(a.bar, &s_flag)) return;
                // level-2: block b sums entries c = b, b + G, ...
                for (int c = b + warp * G; c < k; c += NWARP * G) {
                    double acc = 0.0;
                    for (int bb = lane; bb < G; bb += 32) acc += __ldcg(a.partial + (int64_t)bb * a.m + c);
                    acc = warp_sum(acc);
                    if (lane == 0) __stcg(a.hbuf + c, acc);
                }
                if (!grid_sync(a.bar, &s_flag)) return;
                for (int c = threadIdx.x; c < k; c += NT) hh[c] = __ldcg(a.hbuf + c);
                __syncthreads();
                // e -= J h
                for (int64_t i = r0 + threadIdx.x; i < r1; i += NT) {
                    double v = __ldcg(e + i);
                    for (int c = 0; c < k; ++c) v = fma(-__ldcg(a.J + (int64_t)c * a.N + i), hh[c], v);
                    __stcg(e + i, v);
                }
                // the next pass reads e with a lane-per-row mapping
                __syncthreads();
            } else {
                for (int c = threadIdx.x; c < a.m; c += NT) hh[c] = 0.0;
            }
        }
        // ||e||^2
        double acc = 0.0;
        for (int64_t i = r0 + threadIdx.x; i < r1; i += NT) {
            const double v = __ldcg(e + i);
            acc = fma(v, v, acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) s_part[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < NWARP; ++w) s += s_part[w];
            __stcg(a.partial + (int64_t)b * a.m, s);
        }
        if (!grid_sync(a.bar, &s_flag)) return;
        if (warp == 0) {
            double s = 0.0;
            for (int bb = lane; bb < G; bb += 32) s += __ldcg(a.partial + (int64_t)bb * a.m);
            s = warp_sum(s);
            if (lane == 0) s_nu = sqrt(s);
        }
        __syncthreads();
        const double nu = s_nu;
        if (!isfinite(nu)) {
            if (threadIdx.x == 0) grid_abort(a.bar, ST_ERR_NONFINITE);
            return;
        }
        if (b == 0)
            for (int c = threadIdx.x; c < k; c += NT) a.P[c + (int64_t)j * a.m] = h[c] + h2[c];
        if (nu > tau && nu > 0.0) {
            const double inv = 1.0 / nu;
            double* jk = a.J + (int64_t)k * a.N;
            for (int64_t i = r0 + threadIdx.x; i < r1; i += NT) __stcg(jk + i, __ldcg(e + i) * inv);
            if (b == 0 && threadIdx.x == 0) a.P[k + (int64_t)j * a.m] = nu;
            ++k;
        }
        // the partial buffer is reused next column: all blocks must have read it
        if (!grid_sync(a.bar, &s_flag)) return;
    }
    if (b == 0 && threadIdx.x == 0) *a.k_out = k;
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

__global__ void eye_kernel(int n, double* Y, int ldy) {
    const int64_t tot = (int64_t)n * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t % n), j = (int)(t / n);
        Y[i + (int64_t)j * ldy] = i == j ? 1.0 : 0.0;
    }
}

// ---------------------------------------------------------------------------
// One-sided Jacobi on the columns of X (m x n), rotations accumulated into Y
// (n x n).  Round-robin ordering: every round pairs each column once, a
// sweep of n_p - 1 rounds meets every pair.  One warp per pair and one warp
// per block, so the pairs of a round spread over all SMs (the rotations are
// FP64-throughput bound).  Squared column norms are kept in nrm2 and updated
// with each rotation; they are recomputed at the start of every sweep.
struct JacArgs {
    int m, n;
    double* X;
    int ldx;
    double* Y;
    int ldy;
    int max_sweeps;
    double tol;
    int* flags;    // [3]
    int* sweeps;   // out
    double* nrm2;  // [n + 1]: squared column norms, then the largest
    double cut;    // relative singular-value cut below which columns are dropped
    int* perm;     // [n] visiting order of the current sweep
    GridBarrier bar;
};

__device__ __forceinline__ void jacobi_pair_rot(double alpha, double beta, double gamma, double& c,
                                                double& s) {
    const double zeta = (beta - alpha) / (2.0 * gamma);
    double t;
    if (fabs(zeta) > 1e150) t = 0.5 / zeta;
    else t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    c = 1.0 / sqrt(1.0 + t * t);
    s = c * t;
}

constexpr int JW = 4;  // warps per Jacobi pair (one pair per block)

__device__ __forceinline__ double jac_block_sum(double v, double* s_red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < JW; ++w) t += s_red[w];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(32 * JW) jacobi_kernel(JacArgs a) {
    __shared__ int s_flag;
    __shared__ double s_red[JW];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int gw = blockIdx.x, nw = gridDim.x;
    const int np = a.n + (a.n & 1);
    const int npairs = np / 2;
    int sweep = 0;
    bool converged = false;
    for (; sweep < a.max_sweeps; ++sweep) {
        if (blockIdx.x == 0 && tid == 0) a.flags[(sweep + 1) % 3] = 0;
        for (int c = gw; c < a.n; c += nw) {
            const double* xc = a.X + (int64_t)c * a.ldx;
            double acc = 0.0;
            for (int r = tid; r < a.m; r += nthr) {
                const double u = __ldcg(xc + r);
                acc = fma(u, u, acc);
            }
            acc = jac_block_sum(acc, s_red);
            if (tid == 0) {
                __stcg(a.nrm2 + c, acc);
                // largest squared norm (positive doubles order like their bit patterns)
                if (sweep == 0)
                    atomicMax(reinterpret_cast<unsigned long long*>(a.nrm2 + a.n),
                              (unsigned long long)__double_as_longlong(acc));
            }
        }
        if (!grid_sync(a.bar, &s_flag)) return;
        // visit columns in decreasing-norm order this sweep (the tournament
        // pairs positions; perm maps positions to columns)
        if (blockIdx.x == 0) {
            for (int c = tid; c < a.n; c += nthr) {
                const double v = __ldcg(a.nrm2 + c);
                int rank = 0;
                for (int d = 0; d < a.n; ++d) {
                    const double w = __ldcg(a.nrm2 + d);
                    rank += (w > v) || (w == v && d < c);
                }
                __stcg(a.perm + rank, c);
            }
        }
        if (!grid_sync(a.bar, &s_flag)) return;
        // pairs of columns that both lie below the truncation cut are dropped
        // after the SVD whatever their rotation, so they are not rotated
        const double cut2 = a.cut * a.cut * __ldcg(a.nrm2 + a.n);
        for (int t = 0; t < np - 1; ++t) {
            for (int q = gw; q < npairs; q += nw) {
                int i, j;
                if (q == 0) { i = t; j = np - 1; }
                else { i = (t + q) % (np - 1); j = (t - q + np - 1) % (np - 1); }
                if (i >= a.n || j >= a.n) continue;
                i = __ldcg(a.perm + i);
                j = __ldcg(a.perm + j);
                double* xi = a.X + (int64_t)i * a.ldx;
                double* xj = a.X + (int64_t)j * a.ldx;
                const double al = __ldcg(a.nrm2 + i), be = __ldcg(a.nrm2 + j);
                double ga = 0.0;
                for (int r = tid; r < a.m; r += nthr) ga = fma(__ldcg(xi + r), __ldcg(xj + r), ga);
                ga = jac_block_sum(ga, s_red);
                if ((al > cut2 || be > cut2) && fabs(ga) > a.tol * sqrt(al) * sqrt(be)) {
                    double c, s;
                    jacobi_pair_rot(al, be, ga, c, s);
                    for (int r = tid; r < a.m; r += nthr) {
                        const double u = __ldcg(xi + r), v = __ldcg(xj + r);
                        __stcg(xi + r, c * u - s * v);
                        __stcg(xj + r, s * u + c * v);
                    }
                    double* yi = a.Y + (int64_t)i * a.ldy;
                    double* yj = a.Y + (int64_t)j * a.ldy;
                    for (int r = tid; r < a.n; r += nthr) {
                        const double u = __ldcg(yi + r), v = __ldcg(yj + r);
                        __stcg(yi + r, c * u - s * v);
                        __stcg(yj + r, s * u + c * v);
                    }
                    if (tid == 0) {
                        // new squared norms: c^2 al - 2cs ga + s^2 be and s^2 al + 2cs ga + c^2 be
                        const double cs2 = 2.0 * c * s * ga;
                        __stcg(a.nrm2 + i, fmax(c * c * al - cs2 + s * s * be, 0.0));
                        __stcg(a.nrm2 + j, fmax(s * s * al + cs2 + c * c * be, 0.0));
                        atomicExch(a.flags + sweep % 3, 1);
                    }
                }
            }
            if (!grid_sync(a.bar, &s_flag)) return;
        }
        if (*(volatile int*)(a.flags + sweep % 3) == 0) {
            converged = true;
            ++sweep;
            break;
        }
    }
    if (blockIdx.x == 0 && tid == 0) {
        *a.sweeps = sweep;
        if (!converged) st_dev_error(a.bar.err, ST_ERR_NOT_CONVERGED);
    }
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

// Ysel[:, q] = Y[:, perm[q]];  Vsel[:, q] = X[:, perm[q]] / sigma_q.
__global__ void gather_kernel(int n, int m, int rk, const int* __restrict__ perm,
                              const double* __restrict__ sig, const double* __restrict__ Y, int ldy,
                              const double* __restrict__ X, int ldx, double* Ysel, int ldys,
                              double* Vsel, int ldvs) {
    const int64_t t1 = (int64_t)n * rk, t2 = (int64_t)m * rk;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < t1 + t2;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < t1) {
            const int i = (int)(t % n), q = (int)(t / n);
            Ysel[i + (int64_t)q * ldys] = Y[i + (int64_t)perm[q] * ldy];
        } else {
            const int64_t u = t - t1;
            const int i = (int)(u % m), q = (int)(u / m);
            Vsel[i + (int64_t)q * ldvs] = X[i + (int64_t)perm[q] * ldx] / sig[q];
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
                if (ga != 0.0 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
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

extern "C" st_status st_rom_build_basis(st_model* m, int32_t n_mu, int32_t Nt,
                                        const double* snapshots, int32_t ns, int32_t nt,
                                        double* sigma_out, int32_t* rank_out) {
    if (!m) return st_fail(ST_ERR_ARG, "st_rom_build_basis: NULL model");
    if (!snapshots || n_mu < 1 || Nt < 1 || ns < 1 || nt < 1)
        return st_fail(ST_ERR_ARG, "st_rom_build_basis: bad arguments");
    if (nt > Nt || nt > n_mu) return st_fail(ST_ERR_ARG, "st_rom_build_basis: nt > min(Nt, n_mu)");
    if (n_mu > 64) return st_fail(ST_ERR_ARG, "st_rom_build_basis: at most 64 parameter samples");
    const int64_t N = m->N;
    const int rmax = (int)std::min<int64_t>(m->opt.r_max, N);
    const int cap = rmax + Nt;
    const int64_t ldv = (int64_t)n_mu * Nt;
    const int pdim = std::max(Nt, rmax);
    cudaStream_t st = m->stream;
    st_internal_free_basis(m);
    m->pod_r = 0;
    m->pod_rows = 0;
    m->sigma.clear();

    // buffers
    ST_TRY(st_grow(m, m->W, sizeof(double) * N * cap));
    ST_TRY(st_grow(m, m->V, sizeof(double) * ldv * rmax));
    const size_t szW2 = (size_t)N * cap, szV2 = (size_t)ldv * rmax, szE = (size_t)N * Nt,
                 szL = (size_t)rmax * Nt, szP = (size_t)pdim * pdim, szX = (size_t)cap * cap;
    int gs_blocks = 0;
    {
        int per_sm = 0;
        size_t smem = sizeof(double) * 2 * pdim;
        if (smem > 48 * 1024)
            ST_CUDA_TRY(cudaFuncSetAttribute(gs2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gs2_kernel, NT, smem));
        gs_blocks = std::max(1, std::min(per_sm, 1)) * m->num_sms;
        gs_blocks = (int)std::min<int64_t>(gs_blocks, std::max<int64_t>(1, N / 64));
    }
    const size_t szPart = std::max((size_t)std::max(gs_blocks, 1) * pdim, (size_t)64 * Nt);
    const size_t doubles = szW2 + szV2 + szE + 2 * szL + 3 * szP + 2 * szX + (size_t)cap * rmax * 2 +
                           szPart + pdim + 4 * cap + 32;
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
    double* Ysel = Y + szX;
    double* Vsel = Ysel + (size_t)cap * rmax;
    double* partial = Vsel + (size_t)cap * rmax;
    double* hbuf = partial + szPart;
    double* d_sig = hbuf + pdim;         // [cap] current sigma (device copy)
    double* d_sig_sorted = d_sig + cap;  // [cap]
    double* d_sig_tmp = d_sig_sorted + cap;
    double* d_scalar = d_sig_tmp + cap + 8;  // [16]: tau, dot (d_sig_tmp[cap] is the Jacobi norm max)
    int* d_int = (int*)(d_scalar + 16);  // [16]: k, r_new, sweeps, flags[3]
    int* d_perm = d_int + 16;            // [cap]
    double* W = (double*)m->W.p;
    double* V = (double*)m->V.p;

    int jac_blocks_max = 0;
    {
        int per_sm = 0;
        ST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel, 32 * JW, 0));
        jac_blocks_max = std::max(1, std::min(per_sm, 2)) * m->num_sms;
    }
    const GridBarrier bar{m->d_bar, m->d_bar + 1, m->d_bar + 2, m->d_err, m->opt.spin_limit};
    int r = 0;
    int64_t rows = 0;
    std::vector<double> h_sig;
    auto run_gs = [&](double* Ein, int mcols, double* Jout, double* Pout, const double* tau) -> st_status {
        ST_CUDA_TRY(cudaMemsetAsync(Pout, 0, sizeof(double) * (size_t)mcols * mcols, st));
        ST_CUDA_TRY(cudaMemsetAsync(m->d_bar, 0, sizeof(unsigned int) * 4, st));
        Gs2Args g{N, mcols, Ein, Jout, Pout, d_int, tau, partial, hbuf, bar};
        void* args[] = {&g};
        ST_CUDA_TRY(cudaLaunchCooperativeKernel((void*)gs2_kernel, dim3(gs_blocks), dim3(NT), args,
                                                sizeof(double) * 2 * pdim, st));
        st_count_launch();
        return ST_OK;
    };
    auto read_k = [&](int* out) -> st_status {
        ST_CUDA_TRY(cudaMemcpyAsync(out, d_int, sizeof(int), cudaMemcpyDeviceToHost, st));
        ST_CUDA_TRY(cudaStreamSynchronize(st));
        int32_t herr = 0;
        ST_CUDA_TRY(cudaMemcpy(&herr, m->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (herr) return st_fail(herr, "st_rom_build_basis: Gram-Schmidt failed (%s)", st_status_string(herr));
        return ST_OK;
    };
    for (int p = 0; p < n_mu; ++p) {
        const double* Up = snapshots + (size_t)p * Nt * N;
        {
            const int chunks = (int)std::max<int64_t>(1, std::min<int64_t>(64, N / 2048));
            colnorm_part_kernel<<<dim3(Nt, chunks), NT, 0, st>>>(N, Up, chunks, partial);
            ST_TRY(st_check_launch("colnorm_part"));
            colnorm_max_kernel<<<1, NT, 0, st>>>(Nt, chunks, partial, m->opt.eps_svd, d_scalar);
            ST_TRY(st_check_launch("colnorm_max"));
        }
        ST_CUDA_TRY(cudaMemcpyAsync(E, Up, sizeof(double) * szE, cudaMemcpyDeviceToDevice, st));
        double* J = W + (size_t)r * N;
        int k = 0;
        if (r > 0) {
            // first block pass: L = W^T U_p, E1 = U_p - W L, E1 = J1 P1
            ST_TRY(st_dgemm(m, true, false, r, Nt, N, 1.0, W, N, Up, N, 0.0, L, rmax));
            ST_TRY(st_dgemm(m, false, false, N, Nt, r, -1.0, W, N, L, rmax, 1.0, E, N));
            ST_TRY(run_gs(E, Nt, J, P1, d_scalar));
            int k1 = 0;
            ST_TRY(read_k(&k1));
            if (k1 > 0) {
                // second block pass: L2 = W^T J1, E2 = J1 - W L2 = J P2 by Cholesky QR
                // (E2 is orthonormal up to the rounding carried along W, so its
                // Gram matrix is well conditioned); L += L2 P1, P = P2 P1
                ST_TRY(st_dgemm(m, true, false, r, k1, N, 1.0, W, N, J, N, 0.0, L2, rmax));
                ST_CUDA_TRY(cudaMemcpyAsync(E, J, sizeof(double) * N * k1, cudaMemcpyDeviceToDevice, st));
                ST_TRY(st_dgemm(m, false, false, N, k1, r, -1.0, W, N, L2, rmax, 1.0, E, N));
                ST_TRY(st_dgemm(m, true, false, k1, k1, N, 1.0, E, N, E, N, 0.0, Y, k1));
                ST_CUDA_TRY(cudaMemsetAsync(d_int + 6, 0, sizeof(int), st));
                chol_inv_kernel<<<1, NT, 0, st>>>(k1, Y, P2, k1, X, d_int + 6);
                ST_TRY(st_check_launch("chol_inv"));
                int chol_fail = 0;
                ST_CUDA_TRY(cudaMemcpyAsync(&chol_fail, d_int + 6, sizeof(int), cudaMemcpyDeviceToHost, st));
                ST_CUDA_TRY(cudaStreamSynchronize(st));
                if (!chol_fail) {
                    ST_TRY(st_dgemm(m, false, false, N, k1, k1, 1.0, E, N, X, k1, 0.0, J, N));
                    k = k1;
                } else {
                    ST_TRY(run_gs(E, k1, J, P2, nullptr));
                    ST_TRY(read_k(&k));
                }
                ST_TRY(st_dgemm(m, false, false, r, Nt, k1, 1.0, L2, rmax, P1, Nt, 1.0, L, rmax));
                if (k > 0) ST_TRY(st_dgemm(m, false, false, k, Nt, k1, 1.0, P2, k1, P1, Nt, 0.0, P, Nt));
            }
        } else {
            ST_TRY(run_gs(E, Nt, J, P, d_scalar));
            ST_TRY(read_k(&k));
        }
        const int mrows = r + Nt, ncols = r + k;
        if (ncols == 0) {  // nothing to add: the block is zero and W is empty
            rows += Nt;
            continue;
        }
        build_qt_kernel<<<grid_for(m, (int64_t)mrows * ncols), 256, 0, st>>>(r, k, Nt, d_sig, L, rmax, P, Nt, X, cap);
        ST_TRY(st_check_launch("build_qt"));
        eye_kernel<<<grid_for(m, (int64_t)ncols * ncols), 256, 0, st>>>(ncols, Y, cap);
        ST_TRY(st_check_launch("eye"));
        ST_CUDA_TRY(cudaMemsetAsync(d_int + 3, 0, sizeof(int) * 3, st));
        ST_CUDA_TRY(cudaMemsetAsync(m->d_bar, 0, sizeof(unsigned int) * 4, st));
        // the largest squared column norm is accumulated with atomicMax from zero
        ST_CUDA_TRY(cudaMemsetAsync(d_sig_tmp + ncols, 0, sizeof(double), st));
        {
            const int npairs = (ncols + 1) / 2;
            int jb = std::max(1, std::min(jac_blocks_max, npairs));
            // stop when every pair is orthogonal to m * eps relative
            JacArgs ja{mrows, ncols, X, cap, Y, cap, m->opt.jacobi_sweeps,
                       (double)mrows * 2.220446049250313e-16, d_int + 3, d_int + 2, d_sig_tmp,
                       0.1 * m->opt.eps_sv, d_perm, bar};
            void* args[] = {&ja};
            ST_CUDA_TRY(cudaLaunchCooperativeKernel((void*)jacobi_kernel, dim3(jb), dim3(32 * JW), args, 0, st));
        st_count_launch();
        }
        sort_kernel<<<1, 1024, 0, st>>>(mrows, ncols, X, cap, m->opt.eps_sv, rmax, d_sig_sorted,
                                        d_perm, d_int + 1, d_sig_tmp, m->d_err);
        ST_TRY(st_check_launch("sort"));
        int rnew = 0;
        ST_CUDA_TRY(cudaMemcpyAsync(&rnew, d_int + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        ST_CUDA_TRY(cudaStreamSynchronize(st));
        {
            int32_t herr = 0;
            ST_CUDA_TRY(cudaMemcpy(&herr, m->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
            if (herr) return st_fail(herr, "st_rom_build_basis: middle-matrix SVD failed (%s)", st_status_string(herr));
        }
        if (rnew == 0) {
            rows += Nt;
            r = 0;
            continue;
        }
        gather_kernel<<<grid_for(m, (int64_t)(ncols + mrows) * rnew), 256, 0, st>>>(
            ncols, mrows, rnew, d_perm, d_sig_sorted, Y, cap, X, cap, Ysel, cap, Vsel, cap);
        ST_TRY(st_check_launch("gather"));
        // W2 = [W J] Ysel
        ST_TRY(st_dgemm(m, false, false, N, rnew, ncols, 1.0, W, N, Ysel, cap, 0.0, W2, N));
        // V2 = blkdiag(V, I) Vsel
        if (r > 0 && rows > 0)
            ST_TRY(st_dgemm(m, false, false, rows, rnew, r, 1.0, V, ldv, Vsel, cap, 0.0, V2, ldv));
        ST_CUDA_TRY(cudaMemcpy2DAsync(V2 + rows, sizeof(double) * ldv, Vsel + r, sizeof(double) * cap,
                                      sizeof(double) * Nt, rnew, cudaMemcpyDeviceToDevice, st));
        ST_CUDA_TRY(cudaMemcpyAsync(W, W2, sizeof(double) * N * rnew, cudaMemcpyDeviceToDevice, st));
        ST_CUDA_TRY(cudaMemcpy2DAsync(V, sizeof(double) * ldv, V2, sizeof(double) * ldv,
                                      sizeof(double) * (rows + Nt), rnew, cudaMemcpyDeviceToDevice, st));
        ST_CUDA_TRY(cudaMemcpyAsync(d_sig, d_sig_sorted, sizeof(double) * rnew, cudaMemcpyDeviceToDevice, st));
        r = rnew;
        rows += Nt;
        // orthogonality check of Algorithm 2 and QR re-orthogonalisation
        if (r > 1) {
            dot_kernel<<<1, NT, 0, st>>>(N, W, W + (size_t)(r - 1) * N, d_scalar + 1);
            ST_TRY(st_check_launch("dot"));
            double dotv = 0.0;
            ST_CUDA_TRY(cudaMemcpyAsync(&dotv, d_scalar + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
            ST_CUDA_TRY(cudaStreamSynchronize(st));
            if (std::fabs(dotv) > std::min(m->opt.eps_svd, 2.220446049250313e-16 * (double)N)) {
                ST_CUDA_TRY(cudaMemsetAsync(P, 0, sizeof(double) * (size_t)r * r, st));
                ST_CUDA_TRY(cudaMemsetAsync(m->d_bar, 0, sizeof(unsigned int) * 4, st));
                Gs2Args g{N, r, W, W2, P, d_int, nullptr, partial, hbuf, bar};
                void* args[] = {&g};
                ST_CUDA_TRY(cudaLaunchCooperativeKernel((void*)gs2_kernel, dim3(gs_blocks), dim3(NT),
                                                        args, sizeof(double) * 2 * pdim, st));
        st_count_launch();
                ST_CUDA_TRY(cudaMemcpyAsync(W, W2, sizeof(double) * N * r, cudaMemcpyDeviceToDevice, st));
            }
        }
    }
    h_sig.resize(std::max(r, 1));
    if (r > 0) {
        ST_CUDA_TRY(cudaMemcpyAsync(h_sig.data(), d_sig, sizeof(double) * r, cudaMemcpyDeviceToHost, st));
        ST_CUDA_TRY(cudaStreamSynchronize(st));
    }
    m->pod_r = r;
    m->pod_rows = ldv;
    m->sigma.assign(h_sig.begin(), h_sig.begin() + r);
    if (rank_out) *rank_out = r;
    if (sigma_out) for (int i = 0; i < r; ++i) sigma_out[i] = h_sig[i];
    if (ns > r) return st_fail(ST_ERR_ARG, "st_rom_build_basis: ns = %d exceeds the rank %d", ns, r);
    // bases
    ST_CUDA_TRY(cudaMalloc(&m->d_phi, sizeof(double) * N * ns));
    ST_CUDA_TRY(cudaMalloc(&m->d_T, sizeof(double) * (size_t)Nt * ns * nt));
    ST_CUDA_TRY(cudaMemcpyAsync(m->d_phi, W, sizeof(double) * N * ns, cudaMemcpyDeviceToDevice, st));
    {
        size_t smem = sizeof(double) * ((size_t)Nt * n_mu + n_mu);
        if (smem > 220 * 1024) return st_fail(ST_ERR_ARG, "st_rom_build_basis: Nt * n_mu too large for the temporal SVD");
        if (smem > 48 * 1024)
            ST_CUDA_TRY(cudaFuncSetAttribute(temporal_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        temporal_kernel<<<ns, 512, smem, st>>>(Nt, n_mu, ns, nt, V, ldv, m->d_T, m->opt.jacobi_sweeps,
                                               std::sqrt((double)Nt) * 2.220446049250313e-16, m->d_err);
        ST_TRY(st_check_launch("temporal"));
    }
    m->ns = ns;
    m->nt = nt;
    m->Nt = Nt;
    return ST_OK;
}
