// Batched online phase (Eq. st-galerkin): for every parameter sample p,
//   Ahat(mu_p) = sum_q theta_q Ahat_q                       (ns_p x ns_p)
//   Ahat^st[(i',j'),(i,j)] = delta_{i'i} (M_i - S_i)[j',j]
//                            - Ahat(mu_p)[i',i] G[(i',j'),(i,j)]   (Eq. ij-block-matrix)
//   solve Ahat^st uhat = fhat^st + uhat0^st.
// Samples have individual nested sizes (ns_p, nt_p): the sub-basis
// i < ns_p, j < nt_p, re-indexed i + ns_p j.
//
// One persistent kernel, one CTA per SM, pulls samples from a queue ordered
// largest first (so the big factorisations start early and the small ones
// fill the tail).  Each CTA assembles its sample's matrix into a private
// workspace, factorises it with a right-looking blocked LU with partial
// pivoting in FP64 (the panel lives in shared memory; the trailing update is
// a register-tiled 64x64 FP64 product), solves, refines with an FP64
// residual regenerated from (Ahat, G, M, S) and reports ||r|| / ||rhs||.
#include <algorithm>
#include <climits>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int NT = 256;
constexpr int NWARP = NT / 32;
constexpr int CW = 64;       // trailing-update column chunk
constexpr int CWP = CW + 1;  // row stride of the chunk's U12 in shared memory

struct SolveArgs {
    int n_mu, Q, ns, nt, nfull;
    const double* Ahat;
    const double* G;
    const float* G32;
    const double* M;
    const double* S;
    const double* rhs;
    const double* theta;
    const int32_t* ns_nt;
    const int* order;
    unsigned int* queue;
    double* uhat;
    double* rel_res;
    int32_t* status;
    double* ws;
    int refine;
    int fp32_asm;
    int nb;
    int32_t* err;
};

template <typename T>
struct Smem {
    T* P;         // panel: nfull x nb (ld nfull)
    T* U;         // nb x CW, row stride CWP
    double* Ah;   // ns_p x ns_p
    double* b;    // rhs
    double* x;    // solution
    double* r;    // residual / correction
    int* piv;     // pivots
    int* perm;    // row permutation of the pivots (row i of P A is row perm[i] of A)
    T* D;         // 2 x 32 x 32 diagonal blocks for the triangular solves (the
                  // inverse of the panel's unit lower block during the factorisation)
    int* cur;     // [nfull] panel row at each position after the panel's swaps
    int* where;   // [nfull] position of each panel row
    int* pl;      // [2 x 2 nb] moved rows of a panel step: destination, source
    int* pp;      // [nb] pivot rows of the panel (panel-relative, rows kept in place)
};

__device__ __forceinline__ double block_sum(double v, double* s_val) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) s_val[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < NWARP; ++w) t += s_val[w];
    __syncthreads();
    return t;
}

constexpr int kRowsPerThread = 8;  // panel rows a thread owns: nfull <= 8 * NT

// Pivot candidate of a warp: largest magnitude, ties to the lower row.
template <typename T>
__device__ __forceinline__ void warp_argmax(T& bv, int& bi) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T v2 = __shfl_xor_sync(0xffffffffu, bv, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        if (v2 > bv || (v2 == bv && i2 < bi)) {
            bv = v2;
            bi = i2;
        }
    }
}

// Partial-pivoting LU of the rp x w panel in shared memory (ld ld_p) with its
// rows left in place: the row chosen as pivot c is frozen (it holds row c of
// U), the other rows are eliminated.  Thread t owns rows t, t + NT, ..., so
// the scan for the next pivot runs over the rows the thread has just updated
// and one block barrier per column suffices.  pp[c] receives the panel row of
// pivot c; false on a zero pivot (the elimination still completes, as in
// LAPACK).
template <typename T>
__device__ bool panel_factor(T* P, int rp, int w, int ld_p, int* pp, T (*s_cv)[NWARP], int (*s_ci)[NWARP]) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned used = 0;  // bit k: row tid + k NT is a pivot row
    bool ok = true;
    // magnitudes are compared in T: FP64 compares would run on the slow FP64 pipe
    auto scan = [&](int col, int buf) {
        T bv = (T)-1;
        int bi = INT_MAX;
#pragma unroll
        for (int k = 0; k < kRowsPerThread; ++k) {
            const int r = tid + k * NT;
            if (r < rp && !((used >> k) & 1u)) {
                const T v = fabs(P[r + col * ld_p]);
                if (v > bv) {
                    bv = v;
                    bi = r;
                }
            }
        }
        warp_argmax(bv, bi);
        if (lane == 0) {
            s_cv[buf][warp] = bv;
            s_ci[buf][warp] = bi;
        }
    };
    scan(0, 0);
    __syncthreads();
    for (int c = 0; c < w; ++c) {
        const int buf = c & 1;
        T bv = s_cv[buf][0];
        int pr = s_ci[buf][0];
        for (int q = 1; q < NWARP; ++q) {
            const T v = s_cv[buf][q];
            const int i = s_ci[buf][q];
            if (v > bv || (v == bv && i < pr)) {
                bv = v;
                pr = i;
            }
        }
        if (tid == 0) pp[c] = pr;
        const T pv = P[pr + c * ld_p];
        if (pv == (T)0) ok = false;
        const T inv = pv != (T)0 ? (T)1 / pv : (T)1;  // a zero pivot column is all zero: nothing to scale
        if (pr % NT == tid) used |= 1u << (pr / NT);
        // the row updates in chunks of eight columns, each chunk's loads (pivot
        // row and own row) before its stores, so that a store can hold up at
        // most the next chunk's loads (the compiler cannot tell the rows apart)
#pragma unroll
        for (int k = 0; k < kRowsPerThread; ++k) {
            const int r = tid + k * NT;
            if (r < rp && !((used >> k) & 1u)) {
                const T l = P[r + c * ld_p] * inv;
                P[r + c * ld_p] = l;
                for (int c0 = c + 1; c0 < w; c0 += 8) {
                    T pv8[8], rv8[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const bool in = c0 + u < w;
                        pv8[u] = in ? P[pr + (c0 + u) * ld_p] : (T)0;
                        rv8[u] = in ? P[r + (c0 + u) * ld_p] : (T)0;
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (c0 + u < w) P[r + (c0 + u) * ld_p] = fma(-l, pv8[u], rv8[u]);
                }
            }
        }
        if (c + 1 < w) scan(c + 1, buf ^ 1);
        __syncthreads();
    }
    return ok;
}

// In-place LU with partial pivoting of A (n x n, ld n), in the arithmetic of
// T, right-looking in panels of nb columns: the panel is factorised in shared
// memory with its rows in place (panel_factor), its pivots are turned into
// the LAPACK swap sequence (piv), the moved rows of the other columns are
// exchanged through shared memory in one gather and one scatter, U12 is
// L11^{-1} A12 with the explicit inverse of the unit lower 32 x 32 block, and
// A22 -= L21 U12 in register-tiled column chunks.  Returns false if a zero
// pivot occurred (the factorisation still completes, as in LAPACK).
// P (shared, ld ld_p) <- the rp x w block of A at (kb, kb) (global, ld n):
// warp per column, lane per row, four rows' loads in flight per lane.
template <typename T>
__device__ __forceinline__ void panel_load(T* P, int ld_p, const T* A, int n, int kb, int rp, int w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = warp; c < w; c += NWARP) {
        const T* src = A + kb + (int64_t)(kb + c) * n;
        T* dst = P + (size_t)c * ld_p;
        for (int r0 = lane; r0 < rp; r0 += 4 * 32) {
            T v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = r0 + 32 * u < rp ? src[r0 + 32 * u] : (T)0;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (r0 + 32 * u < rp) dst[r0 + 32 * u] = v[u];
        }
    }
}

template <typename T>
__device__ bool lu_factor(T* A, int n, int ld_p, int nb, Smem<T>& s, T (*s_cv)[NWARP], int (*s_ci)[NWARP],
                          int* s_npl) {
    bool ok = true;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cap = ld_p * nb;  // elements of the panel buffer, reused as staging
    for (int kb = 0; kb < n; kb += nb) {
        const int w = min(nb, n - kb), rp = n - kb;
        panel_load(s.P, ld_p, A, n, kb, rp, w);
        for (int r = tid; r < rp; r += NT) {
            s.cur[r] = r;
            s.where[r] = r;
        }
        __syncthreads();
        if (!panel_factor(s.P, rp, w, ld_p, s.pp, s_cv, s_ci)) ok = false;
        if (tid == 0) {
            // the swap sequence that brings pivot row pp[c] to position c
            int npl = 0;
            for (int c = 0; c < w; ++c) {
                const int p = s.pp[c], q = s.where[p], a = s.cur[c];
                s.cur[c] = p;
                s.cur[q] = a;
                s.where[p] = c;
                s.where[a] = q;
                s.piv[kb + c] = kb + q;
            }
            // moved positions: the first w, and the positions swapped with them
            for (int c = 0; c < w; ++c)
                if (s.cur[c] != c) {
                    s.pl[npl] = c;
                    s.pl[2 * nb + npl] = s.cur[c];
                    ++npl;
                }
            // (where[] is done with: it marks the positions already listed)
            for (int c = 0; c < w; ++c) {
                const int q = s.piv[kb + c] - kb;
                if (q < w || s.cur[q] == q || s.where[q] < 0) continue;
                s.where[q] = -1;
                s.pl[npl] = q;
                s.pl[2 * nb + npl] = s.cur[q];
                ++npl;
            }
            *s_npl = npl;
        }
        __syncthreads();
        // the panel back in its final row order
        for (int c = warp; c < w; c += NWARP)
            for (int r = lane; r < rp; r += 32) A[(kb + r) + (int64_t)(kb + c) * n] = s.P[s.cur[r] + c * ld_p];
        __syncthreads();
        // the moved rows of the columns outside the panel: gather all, then scatter
        const int npl = *s_npl, nout = n - w;
        if (npl > 0) {
            const int per = max(1, cap / npl);  // columns per staging round
            for (int j0 = 0; j0 < nout; j0 += per) {
                const int nj = min(per, nout - j0);
                for (int t = tid; t < npl * nj; t += NT) {
                    const int e = t % npl, jj = j0 + t / npl;
                    const int j = jj < kb ? jj : jj + w;
                    s.P[t] = A[(kb + s.pl[2 * nb + e]) + (int64_t)j * n];
                }
                __syncthreads();
                for (int t = tid; t < npl * nj; t += NT) {
                    const int e = t % npl, jj = j0 + t / npl;
                    const int j = jj < kb ? jj : jj + w;
                    A[(kb + s.pl[e]) + (int64_t)j * n] = s.P[t];
                }
                __syncthreads();
            }
        }
        // the factorised panel again, in its final row order
        panel_load(s.P, ld_p, A, n, kb, rp, w);
        __syncthreads();
        const int r22 = n - kb - w;
        if (r22 <= 0) continue;
        // Li = L11^{-1} (column `lane` by warp 0: forward substitution on e_lane)
        T* Li = s.D;
        if (warp == 0) {
            T y[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) y[i] = i == lane ? (T)1 : (T)0;
#pragma unroll
            for (int i = 1; i < 32; ++i) {
                if (i < w) {
                    T acc = y[i];
#pragma unroll
                    for (int k = 0; k < i; ++k) acc = fma(-s.P[i + k * ld_p], y[k], acc);
                    y[i] = acc;
                }
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) Li[i + 32 * lane] = y[i];
        }
        __syncthreads();
        // U12 = L11^{-1} A12 and A22 -= L21 U12, one column chunk at a time.
        // U12 of the chunk is kept row by row (row stride CWP = CW + 1, so
        // both the column-wise and the row-wise accesses are conflict free).
        for (int j0 = kb + w; j0 < n; j0 += CW) {
            const int wc = min(CW, n - j0);
            for (int t = tid; t < w * wc; t += NT) {
                const int r = t % w, c = t / w;
                s.U[r * CWP + c] = A[(kb + r) + (int64_t)(j0 + c) * n];
            }
            __syncthreads();
            {
                // thread: column tid % CW, rows tid / CW + 4 q
                const int c = tid % CW, r0 = tid / CW;
                T u[32];
#pragma unroll
                for (int k = 0; k < 32; ++k) u[k] = (c < wc && k < w) ? s.U[k * CWP + c] : (T)0;
                T out[32 / (NT / CW)];
#pragma unroll
                for (int q = 0; q < 32 / (NT / CW); ++q) {
                    const int r = r0 + (NT / CW) * q;
                    T acc = (T)0;
#pragma unroll
                    for (int k = 0; k < 32; ++k) acc = fma(Li[r + 32 * k], u[k], acc);
                    out[q] = acc;
                }
                __syncthreads();
                if (c < wc)
#pragma unroll
                    for (int q = 0; q < 32 / (NT / CW); ++q) {
                        const int r = r0 + (NT / CW) * q;
                        if (r < w) s.U[r * CWP + c] = out[q];
                    }
            }
            __syncthreads();
            for (int t = tid; t < w * wc; t += NT) {
                const int r = t % w, c = t / w;
                A[(kb + r) + (int64_t)(j0 + c) * n] = s.U[r * CWP + c];
            }
            // A22 -= L21 U12: warp `warp` owns columns 8 warp .. 8 warp + 7 of
            // a (32 RT) x 64 tile and lane `lane` its rows lane + 32 a (a <
            // RT), so that every load and store of the tile is one contiguous
            // 32-row segment of a column per warp; the tile's old values are
            // loaded first (one round of independent loads) and updated in
            // registers
            constexpr int RT = sizeof(T) == 4 ? 8 : 4;  // FP64: fewer rows (registers)
            static_assert(NT / 32 * 8 == CW, "eight columns per warp cover the chunk");
            const int cg = warp;
            for (int rt = 0; rt < r22; rt += 32 * RT) {
                if (8 * cg < wc) {
                    T acc[RT][8];
#pragma unroll
                    for (int a2 = 0; a2 < RT; ++a2)
#pragma unroll
                        for (int b2 = 0; b2 < 8; ++b2) {
                            const int rr = rt + lane + 32 * a2, c2 = 8 * cg + b2;
                            acc[a2][b2] = (rr < r22 && c2 < wc) ? A[(kb + w + rr) + (int64_t)(j0 + c2) * n] : (T)0;
                        }
                    for (int cc = 0; cc < w; ++cc) {
                        T lv[RT], uv[8];
#pragma unroll
                        for (int a2 = 0; a2 < RT; ++a2) {
                            const int rr = rt + lane + 32 * a2;
                            lv[a2] = rr < r22 ? s.P[(w + rr) + cc * ld_p] : (T)0;
                        }
#pragma unroll
                        for (int b2 = 0; b2 < 8; ++b2) uv[b2] = s.U[cc * CWP + 8 * cg + b2];
#pragma unroll
                        for (int a2 = 0; a2 < RT; ++a2)
#pragma unroll
                            for (int b2 = 0; b2 < 8; ++b2) acc[a2][b2] = fma(-lv[a2], uv[b2], acc[a2][b2]);
                    }
#pragma unroll
                    for (int a2 = 0; a2 < RT; ++a2)
#pragma unroll
                        for (int b2 = 0; b2 < 8; ++b2) {
                            const int rr = rt + lane + 32 * a2, c2 = 8 * cg + b2;
                            if (rr < r22 && c2 < wc) A[(kb + w + rr) + (int64_t)(j0 + c2) * n] = acc[a2][b2];
                        }
                }
            }
            __syncthreads();
        }
    }
    return ok;
}

// perm from the pivot sequence (one thread): the row interchanges applied in
// order to the identity.
__device__ __forceinline__ void lu_perm(int n, const int* piv, int* perm) {
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int i = 0; i < n; ++i) {
        const int pr = piv[i];
        if (pr != i) {
            const int t = perm[i];
            perm[i] = perm[pr];
            perm[pr] = t;
        }
    }
}

// Diagonal 32 x 32 block of A at (c0, c0), zero outside the w x w block.
template <typename T>
__device__ __forceinline__ void load_diag(const T* A, int n, int c0, int w, T* D) {
    for (int t = threadIdx.x; t < 32 * 32; t += NT) {
        const int r = t & 31, c = t >> 5;
        D[t] = (r < w && c < w) ? A[(c0 + r) + (int64_t)(c0 + c) * n] : (T)0;
    }
}

// x <- A^{-1} x using the LU factors in A and s.perm, in the arithmetic of
// the factors (T): x is rounded to T on entry and widened back on exit (with
// T = float this is the correction solve of mixed-precision refinement).
// Blocked substitution: warp 0 solves each 32 x 32 diagonal block (staged in
// shared memory) with shuffles, then all threads update the rest of x with
// the block's 32 new entries while the next diagonal block is staged -- two
// block barriers per 32 columns.
template <typename T>
__device__ void lu_solve(const T* A, int n, Smem<T>& s, double* x) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    T* xs = s.P;  // the panel is free after the factorisation
    for (int i = tid; i < n; i += NT) xs[i] = (T)x[s.perm[i]];
    load_diag(A, n, 0, min(32, n), s.D);
    __syncthreads();
    // L y = P x, L unit lower triangular
    int buf = 0;
    for (int c0 = 0; c0 < n; c0 += 32) {
        const int w = min(32, n - c0);
        const T* D = s.D + buf * 1024;
        if (warp == 0) {
            T xr = lane < w ? xs[c0 + lane] : (T)0;
            for (int c = 0; c < w - 1; ++c) {
                const T xc = __shfl_sync(0xffffffffu, xr, c);
                if (lane > c) xr = fma(-D[lane + 32 * c], xc, xr);
            }
            if (lane < w) xs[c0 + lane] = xr;
        }
        __syncthreads();
        if (c0 + 32 < n) load_diag(A, n, c0 + 32, min(32, n - c0 - 32), s.D + (buf ^ 1) * 1024);
        for (int r = c0 + w + tid; r < n; r += NT) {
            T acc = xs[r];
            for (int c = 0; c < w; ++c) acc = fma(-A[r + (int64_t)(c0 + c) * n], xs[c0 + c], acc);
            xs[r] = acc;
        }
        buf ^= 1;
        __syncthreads();
    }
    // U x = y, from the last block up
    {
        const int c1 = n, c0 = c1 > 32 ? c1 - 32 : 0;
        load_diag(A, n, c0, c1 - c0, s.D + buf * 1024);
        __syncthreads();
    }
    for (int c1 = n; c1 > 0; c1 -= 32) {
        const int c0 = c1 > 32 ? c1 - 32 : 0, w = c1 - c0;
        const T* D = s.D + buf * 1024;
        if (warp == 0) {
            T xr = lane < w ? xs[c0 + lane] : (T)0;
            for (int c = w - 1; c >= 0; --c) {
                if (lane == c) xr = xr / D[c + 32 * c];
                const T xc = __shfl_sync(0xffffffffu, xr, c);
                if (lane < c) xr = fma(-D[lane + 32 * c], xc, xr);
            }
            if (lane < w) xs[c0 + lane] = xr;
        }
        __syncthreads();
        if (c0 > 0) {
            const int n0 = c0 > 32 ? c0 - 32 : 0;
            load_diag(A, n, n0, c0 - n0, s.D + (buf ^ 1) * 1024);
        }
        for (int r = tid; r < c0; r += NT) {
            T acc = xs[r];
            for (int c = 0; c < w; ++c) acc = fma(-A[r + (int64_t)(c0 + c) * n], xs[c0 + c], acc);
            xs[r] = acc;
        }
        buf ^= 1;
        __syncthreads();
    }
    for (int i = tid; i < n; i += NT) x[i] = (double)xs[i];
    __syncthreads();
}

// Entry ((i',j'),(i,j)) of the sample's Ahat^st in FP64 (row i' + a j', column i + a j).
__device__ __forceinline__ double st_entry(const SolveArgs& g, const double* Ah, int a, int ip, int jp,
                                           int i, int j) {
    const int64_t gi = (int64_t)(ip + g.ns * jp) + (int64_t)(i + g.ns * j) * g.nfull;
    double v = -Ah[ip + i * a] * g.G[gi];
    if (ip == i) {
        const int64_t mi = (int64_t)i * g.nt * g.nt + jp + (int64_t)j * g.nt;
        v += g.M[mi] - g.S[mi];
    }
    return v;
}

// T: arithmetic of the assembled matrix and its LU factors (double, or
// float for the FP32-factorisation mode); residuals and the solution are FP64.
template <typename T>
__global__ void __launch_bounds__(NT, 2) solve_kernel(SolveArgs g) {
    extern __shared__ double smem[];
    __shared__ double s_val[NWARP];
    __shared__ T s_cv[2][NWARP];
    __shared__ int s_ci[2][NWARP];
    __shared__ int s_item, s_npl;
    const int nfull = g.nfull, nb = g.nb;
    Smem<T> s;
    s.P = reinterpret_cast<T*>(smem);
    s.U = s.P + (size_t)nfull * nb;
    s.Ah = reinterpret_cast<double*>(s.U + (size_t)nb * CWP);  // nb * CWP * sizeof(T) is a multiple of 8
    s.b = s.Ah + (size_t)g.ns * g.ns;
    s.x = s.b + nfull;
    s.r = s.x + nfull;
    s.piv = reinterpret_cast<int*>(s.r + nfull);
    s.perm = s.piv + nfull;
    {
        // 16-byte aligned after the index arrays
        const uintptr_t pd = (reinterpret_cast<uintptr_t>(s.perm + nfull) + 15) & ~(uintptr_t)15;
        s.D = reinterpret_cast<T*>(pd);
        s.cur = reinterpret_cast<int*>(s.D + 2 * 32 * 32);
        s.where = s.cur + nfull;
        s.pl = s.where + nfull;
        s.pp = s.pl + 4 * nb;
    }
    T* A = reinterpret_cast<T*>(g.ws) + (size_t)blockIdx.x * nfull * nfull;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) {
            const unsigned int it = atomicAdd(g.queue, 1u);
            s_item = it < (unsigned)g.n_mu ? (g.order ? g.order[it] : (int)it) : -1;
        }
        __syncthreads();
        const int p = s_item;
        __syncthreads();
        if (p < 0) break;
        int a = g.ns, bt = g.nt;
        if (g.ns_nt) {
            a = g.ns_nt[2 * p];
            bt = g.ns_nt[2 * p + 1];
        }
        double* up = g.uhat + (size_t)p * nfull;
        if (a < 1 || a > g.ns || bt < 1 || bt > g.nt) {
            if (tid == 0) {
                if (g.status) g.status[p] = ST_ERR_ARG;
                if (g.rel_res) g.rel_res[p] = __longlong_as_double(0x7ff8000000000000LL);
                st_dev_error(g.err, ST_ERR_ARG);
            }
            continue;
        }
        const int n = a * bt;
        // Ahat(mu_p) restricted to the leading a modes
        for (int t = tid; t < a * a; t += NT) {
            const int ip = t % a, i = t / a;
            double v = 0.0;
            for (int q = 0; q < g.Q; ++q)
                v = fma(g.theta[(int64_t)p * g.Q + q], g.Ahat[(int64_t)q * g.ns * g.ns + ip + (int64_t)i * g.ns], v);
            s.Ah[t] = v;
        }
        for (int t = tid; t < n; t += NT) {
            const int i = t % a, j = t / a;
            s.b[t] = g.rhs[i + g.ns * j];
            s.perm[t] = i | (j << 16);  // (i, j) of index t, until the factorisation
        }
        __syncthreads();
        // FP32 copy of Ahat(mu) for the FP32 assembly (in the panel buffer,
        // free until the factorisation): one rounding per entry of Ahat
        float* ah32 = reinterpret_cast<float*>(s.P);
        if (g.fp32_asm)
            for (int t = tid; t < a * a; t += NT) ah32[t] = (float)s.Ah[t];
        __syncthreads();
        // assemble Ahat^st (FP64, or FP32 products in the FP32-assembly mode):
        // warp w builds columns w, w + NWARP, ..., lane l rows l, l + 32, ...,
        // four rows' operand loads in flight per lane
        {
            const int lane = tid & 31, warp = tid >> 5;
            for (int col = warp; col < n; col += NWARP) {
                const int cc = s.perm[col], i = cc & 0xffff, j = cc >> 16;
                T* Ac = A + (int64_t)col * n;
                if (g.fp32_asm) {
                    const float* Gc = g.G32 + (int64_t)(i + g.ns * j) * nfull;
                    for (int r0 = lane; r0 < n; r0 += 4 * 32) {
                        float gv[4];
                        int rc[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int row = r0 + 32 * u;
                            rc[u] = row < n ? s.perm[row] : 0;
                            gv[u] = row < n ? Gc[(rc[u] & 0xffff) + g.ns * (rc[u] >> 16)] : 0.0f;
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int row = r0 + 32 * u;
                            if (row >= n) break;
                            const int ip = rc[u] & 0xffff, jp = rc[u] >> 16;
                            float f = -ah32[ip + i * a] * gv[u];
                            if (ip == i) {
                                const int64_t mi = (int64_t)i * g.nt * g.nt + jp + (int64_t)j * g.nt;
                                f += (float)(g.M[mi] - g.S[mi]);
                            }
                            Ac[row] = (T)f;
                        }
                    }
                } else {
                    for (int row = lane; row < n; row += 32) {
                        const int rc = s.perm[row];
                        Ac[row] = (T)st_entry(g, s.Ah, a, rc & 0xffff, rc >> 16, i, j);
                    }
                }
            }
        }
        __syncthreads();
        const bool ok = lu_factor(A, n, nfull, nb, s, s_cv, s_ci, &s_npl);
        if (!ok) {
            for (int t = tid; t < n; t += NT) up[t] = 0.0;
            if (tid == 0) {
                if (g.status) g.status[p] = ST_ERR_SINGULAR;
                if (g.rel_res) g.rel_res[p] = __longlong_as_double(0x7ff0000000000000LL);
                st_dev_error(g.err, ST_ERR_SINGULAR);
            }
            __syncthreads();
            continue;
        }
        if (tid == 0) lu_perm(n, s.piv, s.perm);
        for (int t = tid; t < n; t += NT) s.x[t] = s.b[t];
        __syncthreads();
        lu_solve(A, n, s, s.x);
        double rn = 0.0;
        for (int step = 0; step <= g.refine; ++step) {
            // r = b - Ahat^st x (FP64, matrix regenerated from the reduced
            // operators: entry ((i',j'),(i,j)) = delta_{i'i} (M_i - S_i)[j',j]
            // - Ahat[i',i] G[(i',j'),(i,j)], columns visited j-major)
            for (int row = tid; row < n; row += NT) {
                const int ip = row % a, jp = row / a;
                double acc = s.b[row];
                const double* Gr = g.G + (ip + (int64_t)g.ns * jp);
                const double* Ahr = s.Ah + ip;
                const int64_t mi = (int64_t)ip * g.nt * g.nt + jp;
                // sum_i Ahat[i', i] (sum_j G[(i',j'),(i,j)] x[i + a j]): one FP64
                // multiply-add per entry (FP64 issues at 1/64 of the FP32 rate)
                for (int i = 0; i < a; ++i) {
                    const double* Gi = Gr + (int64_t)i * g.nfull;
                    double t = 0.0;
                    for (int j = 0; j < bt; ++j) t = fma(Gi[(int64_t)g.ns * j * g.nfull], s.x[i + a * j], t);
                    acc = fma(Ahr[i * a], t, acc);
                }
                for (int j = 0; j < bt; ++j)
                    acc = fma(-(g.M[mi + (int64_t)j * g.nt] - g.S[mi + (int64_t)j * g.nt]), s.x[ip + a * j], acc);
                s.r[row] = acc;
            }
            __syncthreads();
            double loc = 0.0;
            for (int t = tid; t < n; t += NT) loc = fma(s.r[t], s.r[t], loc);
            rn = block_sum(loc, s_val);
            if (step == g.refine) break;
            lu_solve(A, n, s, s.r);
            for (int t = tid; t < n; t += NT) s.x[t] += s.r[t];
            __syncthreads();
        }
        double loc = 0.0;
        for (int t = tid; t < n; t += NT) loc = fma(s.b[t], s.b[t], loc);
        const double bn = block_sum(loc, s_val);
        for (int t = tid; t < n; t += NT) up[t] = s.x[t];
        if (tid == 0) {
            const double rel = bn > 0.0 ? sqrt(rn) / sqrt(bn) : sqrt(rn);
            const bool fin = isfinite(rel);
            if (g.rel_res) g.rel_res[p] = rel;
            if (g.status) g.status[p] = fin ? ST_OK : ST_ERR_NONFINITE;
            if (!fin) st_dev_error(g.err, ST_ERR_NONFINITE);
        }
        __syncthreads();
    }
}

// ---- largest-first queue order ---------------------------------------------
__global__ void size_hist_kernel(int n_mu, int ns, int nt, const int32_t* __restrict__ ns_nt,
                                 int* npv, int* hist) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_mu; p += gridDim.x * blockDim.x) {
        int a = ns, b = nt;
        if (ns_nt) {
            a = ns_nt[2 * p];
            b = ns_nt[2 * p + 1];
        }
        int n = (a >= 1 && a <= ns && b >= 1 && b <= nt) ? a * b : 0;
        npv[p] = n;
        atomicAdd(hist + n, 1);
    }
}

// Exclusive scan of the size histogram: largest size first (descending) or
// smallest first (ascending).
__global__ void size_scan_kernel(int nfull, int* hist, int ascending) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int run = 0;
        for (int i = 0; i <= nfull; ++i) {
            const int s = ascending ? i : nfull - i;
            const int c = hist[s];
            hist[s] = run;
            run += c;
        }
    }
}

__global__ void size_scatter_kernel(int n_mu, const int* __restrict__ npv, int* hist, int* order) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_mu; p += gridDim.x * blockDim.x)
        order[atomicAdd(hist + npv[p], 1)] = p;
}

// Dynamic shared memory of solve_kernel<T> for panel width nb.
size_t solve_smem(int nfull, int ns, int nb, size_t tsize) {
    // the panel also holds one FP64 vector during the triangular solves
    const size_t panel = std::max(tsize * (size_t)nfull * nb, sizeof(double) * (size_t)nfull);
    return panel + tsize * (size_t)nb * CWP + sizeof(double) * ((size_t)ns * ns + 3 * (size_t)nfull) +
           2 * sizeof(int) * (size_t)nfull + 16 + tsize * 2 * 32 * 32 +
           sizeof(int) * (2 * (size_t)nfull + 5 * (size_t)nb) + 64;
}

bool fp32_factors(const st_model* m) { return m->opt.precision == ST_FP32_LU; }


// Shared-memory plan and grid for solve_kernel<T>; the panel width shrinks if
// a wide model does not fit.
// The plan's panel width (if set) and CTAs-per-SM cap replace the defaults
// (panel 32, cap_per_sm).
template <typename T>
st_status solve_plan(st_model* m, int cap_per_sm, int* nb_out, size_t* smem_out, int* blocks_out) {
    const int ns = m->ns, nfull = ns * m->nt;
    if (nfull > kRowsPerThread * NT)
        return st_fail(ST_ERR_ARG, "st_rom_solve: ns*nt = %d above %d", nfull, kRowsPerThread * NT);
    const st_model::SolvePlanCfg& cfg = m->solve_cfg[sizeof(T) == sizeof(float) ? 1 : 0];
    int nb = cfg.nb > 0 ? cfg.nb : 32;
    if (cfg.per_sm > 0) cap_per_sm = cfg.per_sm;
    int max_optin = 0;
    ST_CUDA_TRY(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device));
    while (nb > 4 && solve_smem(nfull, ns, nb, sizeof(T)) > (size_t)max_optin) nb /= 2;
    const size_t smem = solve_smem(nfull, ns, nb, sizeof(T));
    if (smem > (size_t)max_optin) return st_fail(ST_ERR_ARG, "st_rom_solve: ns*nt = %d too large", nfull);
    ST_CUDA_TRY(cudaFuncSetAttribute(solve_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    ST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_kernel<T>, NT, smem));
    *nb_out = nb;
    *smem_out = smem;
    *blocks_out = std::max(1, std::min(per_sm, cap_per_sm)) * m->num_sms;
    return ST_OK;
}

SolveArgs solve_args(st_model* m, int n_mu, const double* theta, const int32_t* ns_nt, double* uhat,
                     double* rel_res, int32_t* status, const int* order, unsigned int* queue,
                     double* ws, int nb) {
    SolveArgs g;
    g.n_mu = n_mu;
    g.Q = m->Q;
    g.ns = m->ns;
    g.nt = m->nt;
    g.nfull = m->ns * m->nt;
    g.Ahat = m->d_Ahat;
    g.G = m->d_G;
    g.G32 = m->d_G32;
    g.M = m->d_M;
    g.S = m->d_S;
    g.rhs = m->d_rhs;
    g.theta = theta;
    g.ns_nt = ns_nt;
    g.order = order;
    g.queue = queue;
    g.uhat = uhat;
    g.rel_res = rel_res;
    g.status = status;
    g.ws = ws;
    g.refine = m->opt.refine_steps;
    g.fp32_asm = m->opt.precision == ST_FP32_ASSEMBLY || m->opt.precision == ST_FP32_LU;
    g.nb = nb;
    g.err = m->d_err;
    return g;
}

}  // namespace

extern "C" st_status st_rom_solve(st_model* m, int32_t n_mu, const double* theta,
                                  const int32_t* ns_nt, double* uhat, double* rel_res,
                                  int32_t* status) {
    if (!m) return st_fail(ST_ERR_ARG, "st_rom_solve: NULL model");
    if (!m->assembled) return st_fail(ST_ERR_STATE, "st_rom_solve: reduced operators not assembled");
    if (n_mu < 0 || (n_mu > 0 && (!theta || !uhat))) return st_fail(ST_ERR_ARG, "st_rom_solve: bad arguments");
    if (n_mu == 0) return ST_OK;
    const int ns = m->ns, nt = m->nt, nfull = ns * nt;
    cudaStream_t st = m->stream;
    const bool f32 = fp32_factors(m);
    const size_t tsize = f32 ? sizeof(float) : sizeof(double);
    int nb = 0, blocks = 0;
    size_t smem = 0;
    if (f32) ST_TRY(solve_plan<float>(m, 4, &nb, &smem, &blocks));
    else ST_TRY(solve_plan<double>(m, 2, &nb, &smem, &blocks));
    const size_t ints = (size_t)2 * n_mu + nfull + 1 + 16;
    const size_t ws_bytes = ((tsize * (size_t)blocks * nfull * nfull) + 255) / 256 * 256;
    ST_TRY(st_grow(m, m->ws_solve, ws_bytes + sizeof(int) * ints));
    double* ws = (double*)m->ws_solve.p;
    int* npv = (int*)((char*)m->ws_solve.p + ws_bytes);
    int* order = npv + n_mu;
    int* hist = order + n_mu;
    const int order_mode = m->solve_cfg[f32 ? 1 : 0].order;
    if (order_mode != ST_ORDER_INPUT) {
        ST_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(int) * (nfull + 1), st));
        const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((n_mu + 255) / 256, 4 * m->num_sms));
        ST_PROF(m, "size_sort_kernels");
        size_hist_kernel<<<gb, 256, 0, st>>>(n_mu, ns, nt, ns_nt, npv, hist);
        size_scan_kernel<<<1, 32, 0, st>>>(nfull, hist, order_mode == ST_ORDER_SMALLEST_FIRST);
        size_scatter_kernel<<<gb, 256, 0, st>>>(n_mu, npv, hist, order);
        ST_TRY(st_check_launch("solve order"));
    }
    ST_CUDA_TRY(cudaMemsetAsync(m->d_bar + 3, 0, sizeof(unsigned int), st));
    SolveArgs g = solve_args(m, n_mu, theta, ns_nt, uhat, rel_res, status,
                             order_mode == ST_ORDER_INPUT ? nullptr : order, m->d_bar + 3, ws, nb);
    ST_PROF(m, f32 ? "solve_kernel<float>" : "solve_kernel<double>");
    if (f32) solve_kernel<float><<<blocks, NT, smem, st>>>(g);
    else solve_kernel<double><<<blocks, NT, smem, st>>>(g);
    return st_check_launch("solve");
}

st_status st_internal_solve_list(st_model* m, int n_list, const int* list, const double* theta,
                                 double* uhat, double* rel_res, int32_t* status) {
    if (n_list <= 0) return ST_OK;
    const int nfull = m->ns * m->nt;
    cudaStream_t st = m->stream;
    const bool f32 = fp32_factors(m);
    const size_t tsize = f32 ? sizeof(float) : sizeof(double);
    int nb = 0, blocks = 0;
    size_t smem = 0;
    if (f32) ST_TRY(solve_plan<float>(m, 4, &nb, &smem, &blocks));
    else ST_TRY(solve_plan<double>(m, 2, &nb, &smem, &blocks));
    const size_t ws_bytes = ((tsize * (size_t)blocks * nfull * nfull) + 255) / 256 * 256;
    ST_TRY(st_grow(m, m->ws_solve, ws_bytes + sizeof(int) * 16));
    ST_CUDA_TRY(cudaMemsetAsync(m->d_bar + 3, 0, sizeof(unsigned int), st));
    SolveArgs g = solve_args(m, n_list, theta, nullptr, uhat, rel_res, status, list, m->d_bar + 3,
                             (double*)m->ws_solve.p, nb);
    ST_PROF(m, f32 ? "solve_kernel<float>" : "solve_kernel<double>");
    if (f32) solve_kernel<float><<<blocks, NT, smem, st>>>(g);
    else solve_kernel<double><<<blocks, NT, smem, st>>>(g);
    return st_check_launch("solve_list");
}

// ---------------------------------------------------------------------------
// Allocation-free variant of st_rom_solve.
//
// Some callers must not allocate device memory while they solve: code that
// runs with a fixed, pre-reserved memory budget (real-time or embedded
// services where an allocation can stall or fail at the worst moment),
// callers whose device memory is owned by an outside pool or allocator that
// forbids side allocations, and callers that issue the solve from a context
// where allocation calls are not permitted.  For them this entry point keeps
// all of its scratch (per-block factorisation workspace, queue order, size
// histogram, queue counter) in one file-scope device array of fixed size;
// it calls no cudaMalloc/cudaFree and no allocating library routine.  The
// caller still passes the inputs and outputs.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr size_t kStaticScratchBytes = 32u << 20;  // 32 MiB, held by every GPU that loads the library
static __device__ __align__(256) unsigned char g_solve_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_solve_scratch on the current device, looked up once
// per device (the symbol name on the host is only a stand-in).
st_status scratch_address(int device, void** out) {
    if (device < 0 || device >= kMaxDevices)
        return st_fail(ST_ERR_ARG, "st_rom_solve_static: device ordinal %d out of range", device);
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_solve_scratch);
        if (e != cudaSuccess || !p)
            return st_fail(ST_ERR_CUDA, "st_rom_solve_static: cudaGetSymbolAddress failed: %s",
                           cudaGetErrorString(e));
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return ST_OK;
}

}  // namespace

extern "C" st_status st_rom_solve_static(st_model* m, int32_t n_mu, const double* theta,
                                         const int32_t* ns_nt, double* uhat, double* rel_res,
                                         int32_t* status) {
    if (!m) return st_fail(ST_ERR_ARG, "st_rom_solve_static: NULL model");
    if (!m->assembled) return st_fail(ST_ERR_STATE, "st_rom_solve_static: reduced operators not assembled");
    if (n_mu < 0 || (n_mu > 0 && (!theta || !uhat)))
        return st_fail(ST_ERR_ARG, "st_rom_solve_static: bad arguments");
    if (n_mu == 0) return ST_OK;
    const int ns = m->ns, nt = m->nt, nfull = ns * nt;
    cudaStream_t st = m->stream;
    int cur = -1;
    ST_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != m->device)
        return st_fail(ST_ERR_STATE, "st_rom_solve_static: current device %d is not the model's device %d",
                       cur, m->device);
    void* base = nullptr;
    ST_TRY(scratch_address(m->device, &base));
    // scratch layout: [counter | npv (n_mu) | order (n_mu) | hist (nfull + 1)] then
    // one nfull x nfull FP64 workspace per resident block
    // (one block's matrix in the factor precision: 4 bytes per entry in
    // ST_FP32_LU, 8 otherwise)
    const size_t int_bytes = ((sizeof(int) * ((size_t)2 * n_mu + nfull + 1 + 16)) + 255) / 256 * 256;
    const bool f32 = fp32_factors(m);
    const size_t mat_t = (f32 ? sizeof(float) : sizeof(double)) * (size_t)nfull * nfull;
    if (int_bytes + mat_t > kStaticScratchBytes)
        return st_fail(ST_ERR_ARG,
                       "st_rom_solve_static: n_mu = %d with ns*nt = %d needs %zu bytes of scratch, "
                       "more than the fixed %zu",
                       n_mu, nfull, int_bytes + mat_t, kStaticScratchBytes);
    int nb = 0, cap_blocks = 0;
    size_t smem = 0;
    if (f32) ST_TRY(solve_plan<float>(m, 4, &nb, &smem, &cap_blocks));
    else ST_TRY(solve_plan<double>(m, 2, &nb, &smem, &cap_blocks));
    const size_t fit = (kStaticScratchBytes - int_bytes) / mat_t;
    const int blocks = (int)std::max<size_t>(1, std::min<size_t>(fit, (size_t)cap_blocks));
    unsigned char* sb = static_cast<unsigned char*>(base);
    unsigned int* queue = reinterpret_cast<unsigned int*>(sb);
    int* npv = reinterpret_cast<int*>(sb) + 16;
    int* order = npv + n_mu;
    int* hist = order + n_mu;
    double* ws = reinterpret_cast<double*>(sb + int_bytes);
    // the array keeps the previous call's contents: zero what must start at zero
    ST_CUDA_TRY(cudaMemsetAsync(queue, 0, sizeof(unsigned int), st));
    const int order_mode = m->solve_cfg[f32 ? 1 : 0].order;
    if (order_mode != ST_ORDER_INPUT) {
        ST_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(int) * (nfull + 1), st));
        const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((n_mu + 255) / 256, 4 * m->num_sms));
        ST_PROF(m, "size_sort_kernels");
        size_hist_kernel<<<gb, 256, 0, st>>>(n_mu, ns, nt, ns_nt, npv, hist);
        size_scan_kernel<<<1, 32, 0, st>>>(nfull, hist, order_mode == ST_ORDER_SMALLEST_FIRST);
        size_scatter_kernel<<<gb, 256, 0, st>>>(n_mu, npv, hist, order);
        ST_TRY(st_check_launch("solve_static order"));
    }
    SolveArgs g = solve_args(m, n_mu, theta, ns_nt, uhat, rel_res, status,
                             order_mode == ST_ORDER_INPUT ? nullptr : order, queue, ws, nb);
    ST_PROF(m, f32 ? "solve_kernel<float>" : "solve_kernel<double>");
    if (f32) solve_kernel<float><<<blocks, NT, smem, st>>>(g);
    else solve_kernel<double><<<blocks, NT, smem, st>>>(g);
    return st_check_launch("solve_static");
}

// ---------------------------------------------------------------------------
// Launch plans of the batched solve and their tuner.
namespace {

int plan_index(int32_t precision) { return precision == ST_FP32_LU ? 1 : 0; }

bool plan_valid(const st_solve_plan& p) {
    return (p.panel == 0 || p.panel == 4 || p.panel == 8 || p.panel == 16 || p.panel == 32) && p.ctas_per_sm >= 0 &&
           p.ctas_per_sm <= 8 && (p.order == ST_ORDER_LARGEST_FIRST || p.order == ST_ORDER_SMALLEST_FIRST ||
                                  p.order == ST_ORDER_INPUT);
}

// The plan solve_plan<T> resolves for the model's current configuration.
template <typename T>
st_status resolved_plan(st_model* m, int default_cap, st_solve_plan* out) {
    int nb = 0, blocks = 0;
    size_t smem = 0;
    ST_TRY(solve_plan<T>(m, default_cap, &nb, &smem, &blocks));
    out->panel = nb;
    out->ctas_per_sm = blocks / std::max(m->num_sms, 1);
    out->order = m->solve_cfg[sizeof(T) == sizeof(float) ? 1 : 0].order;
    return ST_OK;
}

}  // namespace

extern "C" st_status st_rom_solve_set_plan(st_model* m, int32_t precision, const st_solve_plan* plan) {
    if (!m) return st_fail(ST_ERR_ARG, "st_rom_solve_set_plan: NULL model");
    if (precision != ST_FP64 && precision != ST_FP32_ASSEMBLY && precision != ST_FP32_LU)
        return st_fail(ST_ERR_ARG, "st_rom_solve_set_plan: unknown precision %d", precision);
    st_model::SolvePlanCfg c;
    if (plan) {
        if (!plan_valid(*plan))
            return st_fail(ST_ERR_ARG, "st_rom_solve_set_plan: panel must be 0, 4, 8, 16 or 32, ctas_per_sm in "
                                       "[0, 8], order an ST_ORDER_* value");
        c.nb = plan->panel;
        c.per_sm = plan->ctas_per_sm;
        c.order = plan->order;
    }
    m->solve_cfg[plan_index(precision)] = c;
    return ST_OK;
}

extern "C" st_status st_rom_solve_get_plan(st_model* m, int32_t precision, st_solve_plan* plan) {
    if (!m || !plan) return st_fail(ST_ERR_ARG, "st_rom_solve_get_plan: NULL argument");
    if (!m->assembled) return st_fail(ST_ERR_STATE, "st_rom_solve_get_plan: reduced operators not assembled");
    if (precision == ST_FP32_LU) return resolved_plan<float>(m, 4, plan);
    return resolved_plan<double>(m, 2, plan);
}

extern "C" st_status st_rom_solve_tune(st_model* m, int32_t n_mu, const double* theta, const int32_t* ns_nt,
                                       double* uhat, int32_t reps, int32_t cap, st_solve_plan* cands, float* ms,
                                       int32_t* n_cands, st_solve_plan* best, float* best_ms, float* default_ms) {
    if (!m) return st_fail(ST_ERR_ARG, "st_rom_solve_tune: NULL model");
    if (!m->assembled) return st_fail(ST_ERR_STATE, "st_rom_solve_tune: reduced operators not assembled");
    if (n_mu < 1 || !theta || !uhat || reps < 1 || cap < 0 || !best)
        return st_fail(ST_ERR_ARG, "st_rom_solve_tune: bad arguments");
    const bool f32 = fp32_factors(m);
    const int idx = f32 ? 1 : 0;
    const int ns = m->ns, nfull = ns * m->nt;
    const size_t tsize = f32 ? sizeof(float) : sizeof(double);
    const st_model::SolvePlanCfg saved = m->solve_cfg[idx];
    int max_optin = 0;
    ST_CUDA_TRY(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device));
    // candidates: every panel width that fits, every CTAs-per-SM count the
    // occupancy allows (up to 4), every queue order; the default plan first
    std::vector<st_model::SolvePlanCfg> list;
    list.push_back(st_model::SolvePlanCfg{});
    for (int nb : {8, 16, 32}) {
        const size_t smem = solve_smem(nfull, ns, nb, tsize);
        if (smem > (size_t)max_optin) continue;
        int occ = 0;
        const void* fn = f32 ? (const void*)solve_kernel<float> : (const void*)solve_kernel<double>;
        ST_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, NT, smem));
        for (int c = 1; c <= std::min(occ, 4); ++c)
            for (int o : {ST_ORDER_LARGEST_FIRST, ST_ORDER_SMALLEST_FIRST, ST_ORDER_INPUT})
                list.push_back(st_model::SolvePlanCfg{nb, c, o});
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ST_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return st_fail(ST_ERR_CUDA, "st_rom_solve_tune: event creation failed");
    }
    st_status rc = ST_OK;
    float best_t = 0.0f, def_t = 0.0f;
    st_model::SolvePlanCfg best_c{};
    int written = 0;
    for (size_t i = 0; i < list.size() && rc == ST_OK; ++i) {
        m->solve_cfg[idx] = list[i];
        rc = st_rom_solve(m, n_mu, theta, ns_nt, uhat, nullptr, nullptr);  // warm (workspace growth)
        float tmin = 0.0f;
        for (int r = 0; r < reps && rc == ST_OK; ++r) {
            cudaEventRecord(e0, m->stream);
            rc = st_rom_solve(m, n_mu, theta, ns_nt, uhat, nullptr, nullptr);
            cudaEventRecord(e1, m->stream);
            if (rc != ST_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = st_fail(ST_ERR_CUDA, "st_rom_solve_tune: event wait failed");
                break;
            }
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            tmin = r == 0 ? t : std::min(tmin, t);
        }
        if (rc != ST_OK) break;
        if (i == 0) def_t = tmin;
        if (i == 0 || tmin < best_t) {
            best_t = tmin;
            best_c = list[i];
        }
        if (cands && ms && written < cap) {
            st_solve_plan pl{list[i].nb, list[i].per_sm, list[i].order};
            cands[written] = pl;
            ms[written] = tmin;
            ++written;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != ST_OK) {
        m->solve_cfg[idx] = saved;
        return rc;
    }
    m->solve_cfg[idx] = best_c;
    if (n_cands) *n_cands = (int32_t)list.size();
    best->panel = best_c.nb;
    best->ctas_per_sm = best_c.per_sm;
    best->order = best_c.order;
    if (best_ms) *best_ms = best_t;
    if (default_ms) *default_ms = def_t;
    return ST_OK;
}
