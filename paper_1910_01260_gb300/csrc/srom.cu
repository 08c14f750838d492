// Spatial Galerkin ROM of Sec. 3.1 (Eq. galerkin, reference state 0) marched
// by backward Euler (Eq. space_reduced_discretized_ODE) for a batch of
// parameters:
//     (I - dt_k Ahat(mu)) uhat^k = uhat^{k-1} + dt_k Bhat f^k,
//     uhat^0 = Phi_s^T u0,   Ahat(mu) = sum_q theta_q Ahat_q.
// This is the comparison model of the space-time ROM: Nt small dependent
// solves per parameter instead of one larger one.
//
// One block of 128 threads marches one parameter at a time, with the system
// matrix in shared memory.  The matrix I - dt Ahat(mu) changes only with the
// step size, so it is inverted once per run of equal steps (once for uniform
// steps) by Gauss-Jordan elimination with partial pivoting, and every step is
// then a gather by the pivot interchanges and one matrix-vector product.  The
// march is bound by the FP64 pipe (a warp-wide FP64 instruction occupies it
// for many cycles on this GPU), so the product spends no FP64 work on
// shuffles: each row is split into P = 128/n contiguous parts, one thread
// each, and the P partial sums are added in a fixed order by the thread that
// next reads that entry, while it forms the following step's right-hand
// side; P minimises the warp-wide FP64 instructions of one product.  The
// blocks are persistent and take the samples from a queue ordered by
// decreasing ns_p (a counting sort), so the costliest marches start first.
// The vectors Bhat f^k (ns x Nt) and Phi_s^T u0 come from the assembly and
// are shared by all parameters.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int kThreads = 128;
constexpr int kWarps = kThreads / 32;

struct SromArgs {
    int ns, Nt, Q, n_mu;
    const double* Ahat;     // Q x ns x ns, term q column major at Ahat + q ns^2
    const double* theta;    // n_mu x Q row major
    const int32_t* ns_mu;   // n_mu or null (all ns)
    const double* bs;       // ns x Nt: Bhat f^k in column k-1
    const double* u0s;      // ns: Phi_s^T u0
    const double* dt;       // Nt
    double* uhat;           // n_mu x Nt x ns
    int32_t* status;        // n_mu or null
    int32_t* err;
    const int* order;       // samples by decreasing ns_p, bad sizes last
    unsigned int* queue;    // next position in order (zero at launch)
};

// Counting sort of the samples by decreasing ns_p; bin 0 holds bad sizes.
__global__ void srom_hist_kernel(int n_mu, int ns, const int32_t* __restrict__ ns_mu, int* bin,
                                 int* hist) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_mu; p += gridDim.x * blockDim.x) {
        const int b = ns_mu ? ns_mu[p] : ns;
        const int c = (b >= 1 && b <= ns) ? b : 0;
        bin[p] = c;
        atomicAdd(hist + c, 1);
    }
}

__global__ void srom_scan_kernel(int ns, int* hist) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int run = 0;
        for (int c = ns; c >= 0; --c) {
            const int k = hist[c];
            hist[c] = run;
            run += k;
        }
    }
}

__global__ void srom_scatter_kernel(int n_mu, const int* __restrict__ bin, int* hist, int* order) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_mu; p += gridDim.x * blockDim.x)
        order[atomicAdd(hist + bin[p], 1)] = p;
}

// Parts per row of the n x n product: the P in [1, min(kThreads / n, n)]
// with the fewest warp-wide FP64 instructions, ceil(n P / 32) ceil(n / P)
// fused multiply-adds plus ceil(n / 32) (P - 1) additions (the smallest P
// among equals).
__host__ __device__ inline int srom_split(int n) {
    const int pmax = n >= kThreads ? 1 : min(kThreads / n, n);
    int best = 0x7fffffff, P = 1;
    for (int c = 1; c <= pmax; ++c) {
        const int cost = (n * c + 31) / 32 * ((n + c - 1) / c) + (n + 31) / 32 * (c - 1);
        if (cost < best) {
            best = cost;
            P = c;
        }
    }
    return P;
}

// Shared memory: the n x n working matrix (odd row stride, so that threads
// reading consecutive rows hit distinct banks), three vectors of ns, the
// partial sums of one product (n P <= max(kThreads, ns) of them), theta, and
// the gather index of the interchanges.
__host__ __device__ inline int srom_ld(int ns) { return (ns & 1) ? ns + 2 : ns + 1; }
__host__ __device__ inline int srom_parts(int ns) { return ns > kThreads ? ns : kThreads; }

size_t srom_smem(int ns, int Q) {
    return sizeof(double) * ((size_t)ns * srom_ld(ns) + 3 * (size_t)ns + srom_parts(ns) + Q) +
           sizeof(int) * (size_t)ns;
}

__device__ __forceinline__ bool finite_bits(double v) {
    return ((__double_as_longlong(v) >> 52) & 0x7ff) != 0x7ff;
}

// 12 blocks per SM: what the shared memory of ns = 40 admits (40 registers)
__global__ void __launch_bounds__(kThreads, 12) spatial_march_kernel(SromArgs a) {
    extern __shared__ double sm[];
    const int ns = a.ns, ld = srom_ld(ns);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double* X = sm;                   // row r at X + r ld
    double* x = X + (size_t)ns * ld;  // uhat^0
    double* y = x + ns;               // interchanged right-hand side
    double* f = y + ns;               // elimination multipliers of one column
    double* part = f + ns;            // part[s n + i]: part s of row i of X y
    double* th = part + srom_parts(ns);  // theta of the sample
    int* q = (int*)(th + a.Q);        // (P v)[r] = v[q[r]]
    __shared__ int s_piv, s_bad, s_nf, s_item;
    __shared__ double s_pv, s_cc;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);

    for (;;) {
        if (tid == 0) {
            const unsigned int i = atomicAdd(a.queue, 1u);
            s_item = i < (unsigned int)a.n_mu ? a.order[i] : -1;
        }
        __syncthreads();
        const int p = s_item;
        __syncthreads();
        if (p < 0) break;
        const int n = a.ns_mu ? a.ns_mu[p] : ns;
        double* up = a.uhat + (size_t)p * a.Nt * ns;
        if (n < 1 || n > ns) {
            if (tid == 0) {
                if (a.status) a.status[p] = ST_ERR_ARG;
                st_dev_error(a.err, ST_ERR_ARG);
            }
            continue;
        }
        const int P = srom_split(n);    // parts per row of a product
        const int L = (n + P - 1) / P;  // columns per part
        for (int i = tid; i < a.Q; i += kThreads) th[i] = a.theta[(size_t)p * a.Q + i];
        for (int i = tid; i < n; i += kThreads) x[i] = a.u0s[i];
        if (tid == 0) {
            s_bad = 0;
            s_nf = 0;
        }
        __syncthreads();
        double h_inv = 0.0;  // step size of the inverse held in X (steps are > 0)
        int k = 0;
        for (; k < a.Nt; ++k) {
            const double h = a.dt[k];
            if (h != h_inv) {
                // X = I - h Ahat(mu) on the leading n modes
                for (int r = warp; r < n; r += kWarps)
                    for (int j = lane; j < n; j += 32) {
                        double s = 0.0;
                        for (int t = 0; t < a.Q; ++t)
                            s = fma(th[t], a.Ahat[(size_t)t * ns * ns + r + (size_t)ns * j], s);
                        X[r * ld + j] = (r == j ? 1.0 : 0.0) - h * s;
                    }
                for (int i = tid; i < n; i += kThreads) q[i] = i;
                __syncthreads();
                // in-place Gauss-Jordan: X <- (P X)^-1, P the row interchanges
                for (int c = 0; c < n; ++c) {
                    if (warp == 0) {
                        double best = -1.0;
                        int bi = c;
                        for (int r = c + lane; r < n; r += 32) {
                            const double v = fabs(X[r * ld + c]);
                            if (v > best) {
                                best = v;
                                bi = r;
                            }
                        }
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                            if (ob > best || (ob == best && oi < bi)) {
                                best = ob;
                                bi = oi;
                            }
                        }
                        if (lane == 0) {
                            s_piv = bi;
                            s_pv = X[bi * ld + c];
                            s_cc = X[c * ld + c];
                            if (!(best > 0.0) || !isfinite(best)) s_bad = 1;
                        }
                    }
                    __syncthreads();
                    if (s_bad) break;
                    const int pr = s_piv;
                    const double inv = 1.0 / s_pv;
                    // swap rows c and pr and scale the pivot row; the pivot
                    // entry becomes 1/pivot.  Only rows c and pr are written.
                    for (int j = tid; j < n; j += kThreads) {
                        const double rc = X[c * ld + j], rp = X[pr * ld + j];
                        X[pr * ld + j] = rc;
                        X[c * ld + j] = j == c ? inv : rp * inv;
                    }
                    // multipliers: column c after the swap (row pr holds the
                    // old row c), read from rows other than c and pr
                    for (int r = tid; r < n; r += kThreads)
                        f[r] = r == c ? 0.0 : (r == pr ? s_cc : X[r * ld + c]);
                    if (tid == 0 && pr != c) {
                        const int t = q[c];
                        q[c] = q[pr];
                        q[pr] = t;
                    }
                    __syncthreads();
                    for (int r = warp; r < n; r += kWarps) {
                        if (r == c) continue;
                        const double fr = f[r];
                        for (int j = lane; j < n; j += 32)
                            X[r * ld + j] = (j == c ? 0.0 : X[r * ld + j]) - fr * X[c * ld + j];
                    }
                    __syncthreads();
                }
                if (s_bad) break;
                h_inv = h;
            }
            // y = P (uhat^{k-1} + h Bhat f^k); uhat^{k-1} (k > 0) is the sum
            // of the previous product's parts, written out here
            for (int r = tid; r < n; r += kThreads) {
                const int g = q[r];
                double xg;
                if (k == 0) {
                    xg = x[g];
                } else {
                    xg = part[g];
                    for (int s = 1; s < P; ++s) xg += part[s * n + g];
                    up[(size_t)(k - 1) * ns + g] = xg;
                    if (!finite_bits(xg)) s_nf = 1;
                }
                y[r] = fma(h, a.bs[g + (size_t)ns * k], xg);
            }
            __syncthreads();
            // parts of uhat^k = X y: thread t sums row t mod n over the
            // columns of part t / n
            for (int t = tid; t < n * P; t += kThreads) {
                const int i = t % n, s = t / n;
                const int r0 = s * L, r1 = min(n, r0 + L);
                const double* Xi = X + i * ld;
                double acc = 0.0;
                for (int r = r0; r < r1; ++r) acc = fma(Xi[r], y[r], acc);
                part[s * n + i] = acc;
            }
            __syncthreads();
        }
        // the last marched step
        if (k > 0)
            for (int i = tid; i < n; i += kThreads) {
                double xi = part[i];
                for (int s = 1; s < P; ++s) xi += part[s * n + i];
                up[(size_t)(k - 1) * ns + i] = xi;
                if (!finite_bits(xi)) s_nf = 1;
            }
        __syncthreads();
        // steps after a singular matrix are not marched
        for (int kk = k; kk < a.Nt; ++kk)
            for (int i = tid; i < n; i += kThreads) up[(size_t)kk * ns + i] = nan;
        if (tid == 0) {
            const int32_t code = s_bad ? ST_ERR_SINGULAR : (s_nf ? ST_ERR_NONFINITE : ST_OK);
            if (a.status) a.status[p] = code;
            if (code != ST_OK) st_dev_error(a.err, code);
        }
        __syncthreads();
    }
}

}  // namespace

extern "C" st_status st_rom_spatial_march(st_model* m, int32_t n_mu, const double* theta,
                                          const int32_t* ns_mu, double* uhat, int32_t* status) {
    if (!m) return st_fail(ST_ERR_ARG, "st_rom_spatial_march: NULL model");
    if (!m->assembled) return st_fail(ST_ERR_STATE, "st_rom_spatial_march: reduced operators not assembled");
    if (n_mu < 0 || (n_mu > 0 && (!theta || !uhat)))
        return st_fail(ST_ERR_ARG, "st_rom_spatial_march: bad arguments");
    if (n_mu == 0) return ST_OK;
    const size_t smem = srom_smem(m->ns, m->Q);
    int max_optin = 0;
    ST_CUDA_TRY(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device));
    if (smem > (size_t)max_optin) return st_fail(ST_ERR_ARG, "st_rom_spatial_march: ns = %d too large", m->ns);
    ST_CUDA_TRY(cudaFuncSetAttribute(spatial_march_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    ST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spatial_march_kernel, kThreads, smem));
    const int blocks = (int)std::min<int64_t>(n_mu, (int64_t)std::max(per_sm, 1) * m->num_sms);
    // queue order: hist [ns + 1] | bin [n_mu] | order [n_mu]
    const int ns = m->ns;
    cudaStream_t st = m->stream;
    ST_TRY(st_grow(m, m->ws_srom, sizeof(int) * ((size_t)ns + 1 + 2 * (size_t)n_mu)));
    int* hist = (int*)m->ws_srom.p;
    int* bin = hist + ns + 1;
    int* order = bin + n_mu;
    ST_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(int) * (ns + 1), st));
    const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((n_mu + 255) / 256, 4 * m->num_sms));
    {
        ST_PROF(m, "spatial_order_kernels");
        srom_hist_kernel<<<gb, 256, 0, st>>>(n_mu, ns, ns_mu, bin, hist);
        srom_scan_kernel<<<1, 32, 0, st>>>(ns, hist);
        srom_scatter_kernel<<<gb, 256, 0, st>>>(n_mu, bin, hist, order);
        ST_TRY(st_check_launch("spatial march order"));
    }
    ST_CUDA_TRY(cudaMemsetAsync(m->d_bar + 3, 0, sizeof(unsigned int), st));
    SromArgs a{m->ns, m->Nt,  m->Q,    n_mu,   m->d_Ahat, theta, ns_mu, m->d_bs,
               m->d_u0s, m->d_dt, uhat, status, m->d_err,  order, m->d_bar + 3};
    ST_PROF(m, "spatial_march_kernel");
    spatial_march_kernel<<<blocks, kThreads, smem, st>>>(a);
    return st_check_launch("spatial march");
}
