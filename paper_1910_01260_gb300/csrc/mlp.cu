// Learned surrogate mu -> uhat with a residual gate, for many-query use of
// the reduced model (the paper has no counterpart).
//
// Network: x = affine map of mu onto [-1,1]^2 -> Z1 = x W1^T + b1 ->
// H1 = gelu(Z1) -> Z2 = H1 W2^T + b2 -> H2 = gelu(Z2) -> Y = H2 W3^T + b3,
// Y = (uhat - mean) / std per component.  FP32 master weights, BF16 copies
// feed the tensor cores; accumulation and outputs are FP32.
//   * the two wide layers (and the two matching backward products dH = dZ W)
//     run on tcgen05 tensor cores (tc_gemm.cuh): BF16 operands via TMA,
//     FP32 accumulators in tensor memory, bias/GELU fused in the epilogue;
//   * the K = 2 input layer, the loss, GELU derivatives, weight gradients
//     (reductions over the batch) and Adam are FP32 SIMT kernels;
//   * inference checks every prediction with the reduced space-time residual
//     ||Ahat^st(mu) uhat - rhs|| / ||rhs||, computed in FP32 from
//     Ahat^st = K_MS - sum_q theta_q K_q (K_MS = blockdiag(M_i - S_i), K_q =
//     Ahat_q o G), and sends the samples above the gate to the batched LU.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "tc_host.h"

namespace {

constexpr int NT = 256;

struct Offsets {
    int64_t W1, b1, W2, b2, W3, b3, total;
};

Offsets offsets(int n_in, int H, int n_out) {
    Offsets o;
    o.W1 = 0;
    o.b1 = o.W1 + (int64_t)H * n_in;
    o.W2 = o.b1 + H;
    o.b2 = o.W2 + (int64_t)H * H;
    o.W3 = o.b2 + H;
    o.b3 = o.W3 + (int64_t)n_out * H;
    o.total = o.b3 + n_out;
    return o;
}

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.3989422804014327f;
}

int grid1d(st_model* m, int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + NT - 1) / NT, 16 * m->num_sms));
}

// Inputs x (and normalised targets) of the samples idx = (a*i + c) mod n for
// i in [i0, i0 + B); a = 1, c = 0 keeps the natural order.
__global__ void gather_kernel(int B, int i0, int n, int64_t a, int64_t c, const double* __restrict__ mu,
                              double lo0, double lo1, double hi0, double hi1, float* X,
                              const double* __restrict__ uhat, int ldu, int n_out,
                              const double* __restrict__ mean, const double* __restrict__ stdv, float* T) {
    const int64_t tot = (int64_t)B * (T ? n_out : 0) + (int64_t)B;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        if (t < B) {
            const int b = (int)t;
            const int64_t idx = ((a * (int64_t)(i0 + b)) + c) % n;
            X[2 * b] = (float)(2.0 * (mu[2 * idx] - lo0) / (hi0 - lo0) - 1.0);
            X[2 * b + 1] = (float)(2.0 * (mu[2 * idx + 1] - lo1) / (hi1 - lo1) - 1.0);
        } else {
            const int64_t u = t - B;
            const int b = (int)(u / n_out), j = (int)(u % n_out);
            const int64_t idx = ((a * (int64_t)(i0 + b)) + c) % n;
            T[(int64_t)b * n_out + j] = (float)((uhat[idx * ldu + j] - mean[j]) / stdv[j]);
        }
    }
}

// Z1 = X W1^T + b1, H1 = gelu(Z1) (K = 2)
__global__ void layer1_kernel(int B, int H, const float* __restrict__ X, const float* __restrict__ W1,
                              const float* __restrict__ b1, float* Z1, __nv_bfloat16* H1) {
    const int64_t tot = (int64_t)B * H;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / H), o = (int)(t % H);
        const float z = fmaf(X[2 * b], W1[2 * o], fmaf(X[2 * b + 1], W1[2 * o + 1], b1[o]));
        if (Z1) Z1[t] = z;
        H1[t] = __float2bfloat16_rn(gelu_f(z));
    }
}

// dY = 2 (Y - T) / (B n_out); per-block partial sums of (Y - T)^2
__global__ void loss_kernel(int B, int n_out, const float* __restrict__ Y, const float* __restrict__ T, float* dY,
                            __nv_bfloat16* dYb, float* partial) {
    __shared__ float s[NT / 32];
    const int64_t tot = (int64_t)B * n_out;
    const float scale = 2.0f / (float)tot;
    float acc = 0.0f;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const float r = Y[t] - T[t];
        acc = fmaf(r, r, acc);
        const float d = scale * r;
        dY[t] = d;
        dYb[t] = __float2bfloat16_rn(d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = 0.0f;
        for (int w = 0; w < NT / 32; ++w) v += s[w];
        partial[blockIdx.x] = v;
    }
}

__global__ void sum_kernel(int n, const float* __restrict__ part, float scale, float* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += part[i];
        *out = (float)(s * scale);
    }
}

// dZ = dH * gelu'(Z) (FP32 and BF16 copies)
__global__ void gelu_back_kernel(int64_t n, const float* __restrict__ dH, const float* __restrict__ Z, float* dZ,
                                 __nv_bfloat16* dZb) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const float d = dH[t] * gelu_grad_f(Z[t]);
        dZ[t] = d;
        if (dZb) dZb[t] = __float2bfloat16_rn(d);
    }
}

template <typename TH>
__device__ __forceinline__ float to_f(TH v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// dW[o][i] = sum_b dZ[b][o] H[b][i] (O x I, batch reduction in a fixed order);
// db[o] = sum_b dZ[b][o] when db is not null.  32 x 32 output tiles.
template <typename TH>
__global__ void wgrad_kernel(int B, int O, int I, const float* __restrict__ dZ, const TH* __restrict__ Hm, float* dW,
                             float* db) {
    __shared__ float sz[32][33];
    __shared__ float sh[32][33];
    const int o0 = blockIdx.y * 32, i0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    float bacc = 0.f;
    for (int b0 = 0; b0 < B; b0 += 32) {
        for (int r = ty; r < 32; r += 8) {
            const int b = b0 + r;
            sz[r][tx] = (b < B && o0 + tx < O) ? dZ[(int64_t)b * O + o0 + tx] : 0.f;
            sh[r][tx] = (b < B && i0 + tx < I) ? to_f<TH>(Hm[(int64_t)b * I + i0 + tx]) : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int r = 0; r < 32; ++r) {
            const float h = sh[r][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fmaf(sz[r][ty + 8 * q], h, acc[q]);
        }
        if (db && blockIdx.x == 0 && ty == 0)
            for (int r = 0; r < 32; ++r) bacc += sz[r][tx];
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int o = o0 + ty + 8 * q, i = i0 + tx;
        if (o < O && i < I) dW[(int64_t)o * I + i] = acc[q];
    }
    if (db && blockIdx.x == 0 && ty == 0 && o0 + tx < O) db[o0 + tx] = bacc;
}

// Adam with bias correction on the FP32 masters
__global__ void adam_kernel(int64_t n, float* P, const float* __restrict__ G, float* Mv, float* Vv, float lr,
                            float bc1, float bc2) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const float g = G[t];
        const float m = 0.9f * Mv[t] + 0.1f * g;
        const float v = 0.999f * Vv[t] + 0.001f * g * g;
        Mv[t] = m;
        Vv[t] = v;
        P[t] -= lr * (m / bc1) / (sqrtf(v / bc2) + 1e-8f);
    }
}

// BF16 copies of W2, W3 and of their transposes (for dH = dZ W)
__global__ void refresh_kernel(int H, int n_out, const float* __restrict__ W2, const float* __restrict__ W3,
                               __nv_bfloat16* W2b, __nv_bfloat16* W3b, __nv_bfloat16* W2t, __nv_bfloat16* W3t) {
    const int64_t n2 = (int64_t)H * H, n3 = (int64_t)n_out * H;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n2 + n3; t += (int64_t)gridDim.x * blockDim.x) {
        if (t < n2) {
            const int o = (int)(t / H), i = (int)(t % H);
            const __nv_bfloat16 v = __float2bfloat16_rn(W2[t]);
            W2b[t] = v;
            W2t[(int64_t)i * H + o] = v;
        } else {
            const int64_t u = t - n2;
            const int o = (int)(u / H), i = (int)(u % H);
            const __nv_bfloat16 v = __float2bfloat16_rn(W3[u]);
            W3b[u] = v;
            W3t[(int64_t)i * n_out + o] = v;
        }
    }
}

// per-component mean and standard deviation of the training targets (FP64)
__global__ void stats_kernel(int n, int n_out, const double* __restrict__ uhat, int ldu, double* mean, double* stdv) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_out; j += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += uhat[(int64_t)i * ldu + j];
        const double mu = s / n;
        double v = 0.0;
        for (int i = 0; i < n; ++i) {
            const double d = uhat[(int64_t)i * ldu + j] - mu;
            v += d * d;
        }
        mean[j] = mu;
        stdv[j] = sqrt(fmax(v / n, 1e-30));
    }
}

// uhat = Y * std + mean (FP64 output)
__global__ void denorm_kernel(int64_t n, int n_out, const float* __restrict__ Y, const double* __restrict__ mean,
                              const double* __restrict__ stdv, double* uhat, int ldu) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * n_out; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / n_out;
        const int j = (int)(t % n_out);
        uhat[b * ldu + j] = (double)Y[t] * stdv[j] + mean[j];
    }
}

// K_all (4n x n, row major, FP32): rows [0,n) K_MS, rows [(q+1) n, (q+2) n) K_q
__global__ void kall_kernel(int ns, int nt, int Q, const double* __restrict__ Ahat, const double* __restrict__ G,
                            const double* __restrict__ M, const double* __restrict__ S, float* K) {
    const int n = ns * nt;
    const int64_t tot = (int64_t)(Q + 1) * n * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(t / ((int64_t)n * n));
        const int64_t rc = t % ((int64_t)n * n);
        const int row = (int)(rc / n), col = (int)(rc % n);
        const int ip = row % ns, jp = row / ns, i = col % ns, j = col / ns;
        double v;
        if (q == 0) {
            v = (ip == i) ? M[(int64_t)i * nt * nt + jp + (int64_t)j * nt] - S[(int64_t)i * nt * nt + jp + (int64_t)j * nt] : 0.0;
        } else {
            v = Ahat[(int64_t)(q - 1) * ns * ns + ip + (int64_t)i * ns] * G[(int64_t)row + (int64_t)col * n];
        }
        K[t] = (float)v;
    }
}

// C[b][r] = sum_j U[b][j] K[r][j] (FP32 SIMT, 64 x 64 tiles, 4 x 4 per thread);
// U is the FP64 prediction read as FP32.
__global__ void __launch_bounds__(256) gate_gemm_kernel(int Bn, int R, int n, const double* __restrict__ U, int ldu,
                                                        const float* __restrict__ K, float* C) {
    __shared__ float su[16][65];
    __shared__ float sk[16][65];
    const int b0 = blockIdx.y * 64, r0 = blockIdx.x * 64;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < n; k0 += 16) {
        for (int l = threadIdx.x; l < 64 * 16; l += 256) {
            const int rr = l / 16, kk = l % 16;
            su[kk][rr] = (b0 + rr < Bn && k0 + kk < n) ? (float)U[(int64_t)(b0 + rr) * ldu + k0 + kk] : 0.f;
            sk[kk][rr] = (r0 + rr < R && k0 + kk < n) ? K[(int64_t)(r0 + rr) * n + k0 + kk] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], c[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = su[kk][ty + 16 * q];
                c[q] = sk[kk][tx + 16 * q];
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], c[y], acc[x][y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int b = b0 + ty + 16 * x, r = r0 + tx + 16 * y;
            if (b < Bn && r < R) C[(int64_t)b * R + r] = acc[x][y];
        }
}

// per sample: r = K_MS u - sum_q theta_q K_q u - rhs; flag samples above the gate
__global__ void gate_kernel(int Bn, int b0, int n, int Q, const float* __restrict__ C,
                            const double* __restrict__ theta, const double* __restrict__ rhs, double gate,
                            double* rel_res, int32_t* used, int* list, unsigned int* count) {
    const int b = blockIdx.x;
    if (b >= Bn) return;
    __shared__ double s_r[8], s_f[8];
    double rr = 0.0, ff = 0.0;
    const float* c = C + (int64_t)b * (Q + 1) * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double v = (double)c[j];
        for (int q = 0; q < Q; ++q) v -= theta[(int64_t)b * Q + q] * (double)c[(int64_t)(q + 1) * n + j];
        v -= rhs[j];
        rr += v * v;
        ff += rhs[j] * rhs[j];
    }
    rr = warp_sum(rr);
    ff = warp_sum(ff);
    if ((threadIdx.x & 31) == 0) {
        s_r[threadIdx.x >> 5] = rr;
        s_f[threadIdx.x >> 5] = ff;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, f = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += s_r[w];
            f += s_f[w];
        }
        const double rel = f > 0.0 ? sqrt(a / f) : sqrt(a);
        const bool ok = isfinite(rel) && rel <= gate;
        rel_res[b] = rel;
        used[b] = ok ? 0 : 1;
        if (!ok) list[atomicAdd(count, 1u)] = b0 + b;
    }
}

uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// epoch permutation i -> (a i + c) mod n with gcd(a, n) = 1
void epoch_perm(int64_t n, uint64_t seed, int epoch, int64_t* a, int64_t* c) {
    int64_t aa = (int64_t)(splitmix64(seed + 2ull * (uint64_t)epoch) % (uint64_t)n);
    *c = (int64_t)(splitmix64(seed + 2ull * (uint64_t)epoch + 1ull) % (uint64_t)n);
    aa = std::max<int64_t>(aa, 1);
    while (std::gcd(aa, n) != 1) aa = aa + 1 < n ? aa + 1 : 1;
    *a = aa;
}

// device views of the surrogate buffers
struct Views {
    Offsets o;
    float *P, *Gd, *Mv, *Vv;
    __nv_bfloat16 *W2b, *W3b, *W2t, *W3t;
    double *mean, *stdv;
};

Views views(st_model* m) {
    auto& s = m->mlp;
    Views v;
    v.o = offsets(s.n_in, s.hidden, s.n_out);
    v.P = (float*)s.params.p;
    v.Gd = (float*)s.grad.p;
    v.Mv = (float*)s.adam_m.p;
    v.Vv = (float*)s.adam_v.p;
    const int64_t H = s.hidden, n_out = s.n_out;
    v.W2b = (__nv_bfloat16*)s.wbf.p;
    v.W3b = v.W2b + H * H;
    v.W2t = v.W3b + n_out * H;
    v.W3t = v.W2t + H * H;
    v.mean = (double*)s.stats.p;
    v.stdv = v.mean + n_out;
    return v;
}

// activation buffers for a batch of B rows (rows padded to the 128-row tile)
struct Acts {
    float *X, *T, *Z1, *Z2, *Y, *dY, *dH, *dZ, *part;
    __nv_bfloat16 *H1, *H2, *dYb, *dZb;
};

st_status acts(st_model* m, int B, Acts* a) {
    const int64_t H = m->mlp.hidden, n_out = m->mlp.n_out;
    const int64_t Bp = (B + 127) / 128 * 128;
    const int64_t f32 = Bp * (2 + n_out + H + H + n_out + n_out + H + H) + 4096;
    const int64_t b16 = Bp * (H + H + n_out + H);
    ST_TRY(st_grow(m, m->mlp.act, sizeof(float) * f32 + sizeof(__nv_bfloat16) * b16 + 1024));
    float* f = (float*)m->mlp.act.p;
    a->X = f;
    a->T = a->X + Bp * 2;
    a->Z1 = a->T + Bp * n_out;
    a->Z2 = a->Z1 + Bp * H;
    a->Y = a->Z2 + Bp * H;
    a->dY = a->Y + Bp * n_out;
    a->dH = a->dY + Bp * n_out;
    a->dZ = a->dH + Bp * H;
    a->part = a->dZ + Bp * H;
    __nv_bfloat16* h = (__nv_bfloat16*)(a->part + 4096);
    a->H1 = h;
    a->H2 = a->H1 + Bp * H;
    a->dYb = a->H2 + Bp * H;
    a->dZb = a->dYb + Bp * n_out;
    return ST_OK;
}

tc::GemmArgs epi(st_model* m) {
    tc::GemmArgs g{};
    g.err = m->d_err;
    g.limit = m->opt.spin_limit;
    return g;
}

int bn_for(int N) { return N <= 256 ? (N <= 64 ? 64 : (N <= 128 ? 128 : 256)) : (N % 240 == 0 ? 240 : 256); }

// forward for B rows already gathered in a.X; Y (FP32) in a.Y
st_status forward(st_model* m, const Views& v, const Acts& a, int B, bool keep_pre) {
    const int H = m->mlp.hidden, n_out = m->mlp.n_out;
    cudaStream_t st = m->stream;
    layer1_kernel<<<grid1d(m, (int64_t)B * H), NT, 0, st>>>(B, H, a.X, v.P + v.o.W1, v.P + v.o.b1,
                                                               keep_pre ? a.Z1 : nullptr, a.H1);
    ST_TRY(st_check_launch("mlp layer1"));
    tc::GemmArgs g2 = epi(m);
    g2.bias = v.P + v.o.b2;
    g2.gelu = 1;
    g2.out_bf16 = a.H2;
    g2.ldb = H;
    g2.out_pre = keep_pre ? a.Z2 : nullptr;
    g2.ldp = H;
    ST_TRY(st_tc_gemm(m, bn_for(H), B, H, H, a.H1, H, v.W2b, H, g2));
    tc::GemmArgs g3 = epi(m);
    g3.bias = v.P + v.o.b3;
    g3.out_f32 = a.Y;
    g3.ldf = n_out;
    ST_TRY(st_tc_gemm(m, bn_for(n_out), B, n_out, H, a.H2, H, v.W3b, H, g3));
    return ST_OK;
}

// loss (into loss_slot) and all gradients into v.Gd for B gathered rows
st_status backward(st_model* m, const Views& v, const Acts& a, int B, float* loss_slot) {
    const int H = m->mlp.hidden, n_out = m->mlp.n_out;
    cudaStream_t st = m->stream;
    const int lb = std::min(grid1d(m, (int64_t)B * n_out), 4096);
    loss_kernel<<<lb, NT, 0, st>>>(B, n_out, a.Y, a.T, a.dY, a.dYb, a.part);
    ST_TRY(st_check_launch("mlp loss"));
    sum_kernel<<<1, 32, 0, st>>>(lb, a.part, 1.0f / (float)((int64_t)B * n_out), loss_slot);
    ST_TRY(st_check_launch("mlp loss sum"));
    // layer 3
    wgrad_kernel<__nv_bfloat16><<<dim3((H + 31) / 32, (n_out + 31) / 32), 256, 0, st>>>(
        B, n_out, H, a.dY, a.H2, v.Gd + v.o.W3, v.Gd + v.o.b3);
    ST_TRY(st_check_launch("mlp wgrad3"));
    tc::GemmArgs gh = epi(m);
    gh.out_f32 = a.dH;
    gh.ldf = H;
    ST_TRY(st_tc_gemm(m, bn_for(H), B, H, n_out, a.dYb, n_out, v.W3t, n_out, gh));
    gelu_back_kernel<<<grid1d(m, (int64_t)B * H), NT, 0, st>>>((int64_t)B * H, a.dH, a.Z2, a.dZ, a.dZb);
    ST_TRY(st_check_launch("mlp gelu back 2"));
    // layer 2
    wgrad_kernel<__nv_bfloat16><<<dim3((H + 31) / 32, (H + 31) / 32), 256, 0, st>>>(B, H, H, a.dZ, a.H1,
                                                                                   v.Gd + v.o.W2, v.Gd + v.o.b2);
    ST_TRY(st_check_launch("mlp wgrad2"));
    tc::GemmArgs gh1 = epi(m);
    gh1.out_f32 = a.dH;
    gh1.ldf = H;
    ST_TRY(st_tc_gemm(m, bn_for(H), B, H, H, a.dZb, H, v.W2t, H, gh1));
    gelu_back_kernel<<<grid1d(m, (int64_t)B * H), NT, 0, st>>>((int64_t)B * H, a.dH, a.Z1, a.dZ, nullptr);
    ST_TRY(st_check_launch("mlp gelu back 1"));
    // layer 1
    wgrad_kernel<float><<<dim3(1, (H + 31) / 32), 256, 0, st>>>(B, H, 2, a.dZ, a.X, v.Gd + v.o.W1, v.Gd + v.o.b1);
    return st_check_launch("mlp wgrad1");
}

st_status refresh(st_model* m, const Views& v) {
    const int H = m->mlp.hidden, n_out = m->mlp.n_out;
    refresh_kernel<<<grid1d(m, (int64_t)H * H + (int64_t)n_out * H), NT, 0, m->stream>>>(
        H, n_out, v.P + v.o.W2, v.P + v.o.W3, v.W2b, v.W3b, v.W2t, v.W3t);
    return st_check_launch("mlp refresh");
}

st_status setup(st_model* m, const float* init_host, uint64_t seed) {
    auto& s = m->mlp;
    s.n_out = m->ns * m->nt;
    const Offsets o = offsets(s.n_in, s.hidden, s.n_out);
    s.n_params = o.total;
    ST_TRY(st_grow(m, s.params, sizeof(float) * o.total));
    ST_TRY(st_grow(m, s.grad, sizeof(float) * o.total));
    ST_TRY(st_grow(m, s.adam_m, sizeof(float) * o.total));
    ST_TRY(st_grow(m, s.adam_v, sizeof(float) * o.total));
    ST_TRY(st_grow(m, s.wbf, sizeof(__nv_bfloat16) * ((int64_t)2 * s.hidden * s.hidden + 2 * (int64_t)s.n_out * s.hidden)));
    ST_TRY(st_grow(m, s.stats, sizeof(double) * 2 * s.n_out));
    std::vector<float> h(o.total, 0.0f);
    if (init_host) {
        std::copy(init_host, init_host + o.total, h.begin());
    } else {
        // Kaiming-uniform (bound sqrt(6 / fan_in)) from SplitMix64, zero biases
        uint64_t ctr = seed;
        auto fill = [&](int64_t off, int64_t count, int fan_in) {
            const double bound = std::sqrt(6.0 / fan_in);
            for (int64_t i = 0; i < count; ++i) {
                const double u = (double)(splitmix64(ctr++) >> 11) * (1.0 / 9007199254740992.0);
                h[off + i] = (float)((2.0 * u - 1.0) * bound);
            }
        };
        fill(o.W1, o.b1 - o.W1, s.n_in);
        fill(o.W2, o.b2 - o.W2, s.hidden);
        fill(o.W3, o.b3 - o.W3, s.hidden);
    }
    ST_CUDA_TRY(cudaMemcpyAsync(s.params.p, h.data(), sizeof(float) * o.total, cudaMemcpyHostToDevice, m->stream));
    ST_CUDA_TRY(cudaMemsetAsync(s.adam_m.p, 0, sizeof(float) * o.total, m->stream));
    ST_CUDA_TRY(cudaMemsetAsync(s.adam_v.p, 0, sizeof(float) * o.total, m->stream));
    ST_CUDA_TRY(cudaStreamSynchronize(m->stream));
    s.adam_t = 0;
    return refresh(m, views(m));
}

}  // namespace

extern "C" st_status st_rom_surrogate_train(st_model* m, int32_t n, const double* mu, const double* mu_lo,
                                            const double* mu_hi, const double* uhat, const float* init,
                                            int32_t epochs, int32_t batch, float lr, uint64_t seed,
                                            float* epoch_loss) {
    if (!m) return st_fail(ST_ERR_ARG, "st_rom_surrogate_train: NULL model");
    if (!m->d_phi) return st_fail(ST_ERR_STATE, "st_rom_surrogate_train: the model has no basis");
    if (n < 2 || !mu || !uhat || !mu_lo || !mu_hi || epochs < 0 || batch < 1 || !(lr > 0))
        return st_fail(ST_ERR_ARG, "st_rom_surrogate_train: bad arguments");
    if (!(mu_hi[0] > mu_lo[0]) || !(mu_hi[1] > mu_lo[1]))
        return st_fail(ST_ERR_ARG, "st_rom_surrogate_train: empty parameter box");
    if ((m->ns * m->nt) % 8 != 0) return st_fail(ST_ERR_ARG, "st_rom_surrogate_train: ns*nt must be a multiple of 8");
    auto& s = m->mlp;
    ST_TRY(setup(m, init, seed));
    s.lo[0] = mu_lo[0];
    s.lo[1] = mu_lo[1];
    s.hi[0] = mu_hi[0];
    s.hi[1] = mu_hi[1];
    const int n_out = s.n_out;
    const int ldu = n_out;
    Views v = views(m);
    stats_kernel<<<(n_out + 127) / 128, 128, 0, m->stream>>>(n, n_out, uhat, ldu, v.mean, v.stdv);
    ST_TRY(st_check_launch("mlp stats"));
    const int B = std::min(batch, (int)n);
    const int steps_per_epoch = (n + B - 1) / B;
    const int64_t total = (int64_t)epochs * steps_per_epoch;
    Acts a;
    ST_TRY(acts(m, B, &a));
    float* d_loss = nullptr;
    ST_TRY(st_grow(m, m->ws_misc, sizeof(float) * (size_t)std::max<int64_t>(total, 1) + 256));
    d_loss = (float*)m->ws_misc.p;
    int64_t step = 0;
    for (int e = 0; e < epochs; ++e) {
        int64_t pa, pc;
        epoch_perm(n, seed, e, &pa, &pc);
        for (int j = 0; j < steps_per_epoch; ++j, ++step) {
            const int i0 = j * B, bb = std::min(B, (int)n - i0);
            gather_kernel<<<grid1d(m, (int64_t)bb * (n_out + 1)), NT, 0, m->stream>>>(
                bb, i0, n, pa, pc, mu, s.lo[0], s.lo[1], s.hi[0], s.hi[1], a.X, uhat, ldu, n_out, v.mean, v.stdv, a.T);
            ST_TRY(st_check_launch("mlp gather"));
            ST_TRY(forward(m, v, a, bb, true));
            ST_TRY(backward(m, v, a, bb, d_loss + step));
            s.adam_t += 1;
            const double lr_t = 0.5 * lr * (1.0 + std::cos(M_PI * (double)step / (double)std::max<int64_t>(total, 1)));
            const float bc1 = (float)(1.0 - std::pow(0.9, (double)s.adam_t));
            const float bc2 = (float)(1.0 - std::pow(0.999, (double)s.adam_t));
            adam_kernel<<<grid1d(m, s.n_params), NT, 0, m->stream>>>(s.n_params, v.P, v.Gd, v.Mv, v.Vv, (float)lr_t, bc1, bc2);
            ST_TRY(st_check_launch("mlp adam"));
            ST_TRY(refresh(m, v));
        }
    }
    if (epoch_loss && total > 0) {
        std::vector<float> h(total);
        ST_CUDA_TRY(cudaMemcpyAsync(h.data(), d_loss, sizeof(float) * total, cudaMemcpyDeviceToHost, m->stream));
        ST_CUDA_TRY(cudaStreamSynchronize(m->stream));
        for (int e = 0; e < epochs; ++e) {
            double acc = 0.0;
            for (int j = 0; j < steps_per_epoch; ++j) {
                const int bb = std::min(B, (int)n - j * B);
                acc += (double)h[(int64_t)e * steps_per_epoch + j] * bb;
            }
            epoch_loss[e] = (float)(acc / n);
        }
    }
    s.trained = true;
    return ST_OK;
}

namespace {
// the tensor-core residual products (defined with the refinement below)
bool tc_residual_ok(const st_model* m);
st_status residual_prepare(st_model* m);
st_status residual_products(st_model* m, int rows, const double* X, int ldx, float* C);
}  // namespace

extern "C" st_status st_rom_surrogate_infer(st_model* m, int32_t n, const double* mu, const double* theta, double gate,
                                            double* uhat, double* rel_res, int32_t* used_fallback, int32_t* n_fallback) {
    if (!m) return st_fail(ST_ERR_ARG, "st_rom_surrogate_infer: NULL model");
    if (!m->mlp.trained) return st_fail(ST_ERR_STATE, "st_rom_surrogate_infer: the surrogate is not trained");
    if (!m->assembled) return st_fail(ST_ERR_STATE, "st_rom_surrogate_infer: reduced operators not assembled");
    if (m->ns * m->nt != m->mlp.n_out) return st_fail(ST_ERR_STATE, "st_rom_surrogate_infer: basis changed since training");
    if (n < 0 || (n > 0 && (!mu || !theta || !uhat || !rel_res || !used_fallback)) || !(gate >= 0))
        return st_fail(ST_ERR_ARG, "st_rom_surrogate_infer: bad arguments");
    if (n == 0) {
        if (n_fallback) *n_fallback = 0;
        return ST_OK;
    }
    auto& s = m->mlp;
    const int n_out = s.n_out, Q = m->Q;
    const int R = (Q + 1) * n_out;
    cudaStream_t st = m->stream;
    Views v = views(m);
    // gate operator: the affine pieces of Ahat^st (three-part BF16 splits for
    // the tensor-core products, or FP32 for the SIMT ones)
    const bool tc = tc_residual_ok(m);
    if (tc) {
        ST_TRY(residual_prepare(m));
    } else {
        ST_TRY(st_grow(m, s.kall, sizeof(float) * (size_t)R * n_out));
        kall_kernel<<<grid1d(m, (int64_t)R * n_out), NT, 0, st>>>(m->ns, m->nt, Q, m->d_Ahat, m->d_G, m->d_M,
                                                                 m->d_S, (float*)s.kall.p);
        ST_TRY(st_check_launch("mlp kall"));
    }
    const int chunk = 65536;
    ST_TRY(st_grow(m, s.list, sizeof(int) * (size_t)n + 64));
    int* list = (int*)s.list.p;
    unsigned int* count = (unsigned int*)(list + n);
    ST_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(unsigned int), st));
    Acts a;
    ST_TRY(acts(m, std::min(n, chunk), &a));
    ST_TRY(st_grow(m, m->ws_misc, sizeof(float) * (size_t)std::min(n, chunk) * R + 256));
    float* C = (float*)m->ws_misc.p;
    for (int b0 = 0; b0 < n; b0 += chunk) {
        const int bb = std::min(chunk, n - b0);
        gather_kernel<<<grid1d(m, bb), NT, 0, st>>>(bb, 0, bb, 1, 0, mu + 2 * (int64_t)b0, s.lo[0], s.lo[1], s.hi[0],
                                                    s.hi[1], a.X, nullptr, 0, n_out, nullptr, nullptr, nullptr);
        ST_TRY(st_check_launch("mlp gather"));
        ST_TRY(forward(m, v, a, bb, false));
        denorm_kernel<<<grid1d(m, (int64_t)bb * n_out), NT, 0, st>>>(bb, n_out, a.Y, v.mean, v.stdv,
                                                                     uhat + (int64_t)b0 * n_out, n_out);
        ST_TRY(st_check_launch("mlp denorm"));
        if (tc) {
            ST_TRY(residual_products(m, bb, uhat + (int64_t)b0 * n_out, n_out, C));
        } else {
            ST_PROF(m, "gate_gemm_kernel");
            gate_gemm_kernel<<<dim3((R + 63) / 64, (bb + 63) / 64), 256, 0, st>>>(
                bb, R, n_out, uhat + (int64_t)b0 * n_out, n_out, (float*)s.kall.p, C);
            ST_TRY(st_check_launch("mlp gate gemm"));
        }
        {
            ST_PROF(m, "gate_kernel");
            gate_kernel<<<bb, 128, 0, st>>>(bb, b0, n_out, Q, C, theta + (int64_t)b0 * Q, m->d_rhs, gate,
                                           rel_res + b0, used_fallback + b0, list, count);
            ST_TRY(st_check_launch("mlp gate"));
        }
    }
    unsigned int hc = 0;
    ST_CUDA_TRY(cudaMemcpyAsync(&hc, count, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    ST_CUDA_TRY(cudaStreamSynchronize(st));
    if (n_fallback) *n_fallback = (int32_t)hc;
    // fallback: batched LU for the samples above the gate
    ST_TRY(st_internal_solve_list(m, (int)hc, list, theta, uhat, rel_res, nullptr));
    return ST_OK;
}

extern "C" st_status st_rom_surrogate_params(st_model* m, float* params, int64_t* count) {
    if (!m) return st_fail(ST_ERR_ARG, "st_rom_surrogate_params: NULL model");
    if (!m->mlp.params.p || m->mlp.n_params == 0) return st_fail(ST_ERR_STATE, "st_rom_surrogate_params: no surrogate");
    if (count) *count = m->mlp.n_params;
    if (params) {
        ST_CUDA_TRY(cudaStreamSynchronize(m->stream));
        ST_CUDA_TRY(cudaMemcpy(params, m->mlp.params.p, sizeof(float) * m->mlp.n_params, cudaMemcpyDeviceToHost));
    }
    return ST_OK;
}

extern "C" st_status st_rom_surrogate_loss_grad(st_model* m, int32_t n, const double* mu, const double* mu_lo,
                                                const double* mu_hi, const double* uhat, const float* params,
                                                float* grad, float* loss) {
    if (!m) return st_fail(ST_ERR_ARG, "st_rom_surrogate_loss_grad: NULL model");
    if (!m->d_phi) return st_fail(ST_ERR_STATE, "st_rom_surrogate_loss_grad: the model has no basis");
    if (n < 1 || !mu || !uhat || !params || !mu_lo || !mu_hi)
        return st_fail(ST_ERR_ARG, "st_rom_surrogate_loss_grad: bad arguments");
    if ((m->ns * m->nt) % 8 != 0) return st_fail(ST_ERR_ARG, "st_rom_surrogate_loss_grad: ns*nt must be a multiple of 8");
    auto& s = m->mlp;
    ST_TRY(setup(m, params, 0));
    s.lo[0] = mu_lo[0];
    s.lo[1] = mu_lo[1];
    s.hi[0] = mu_hi[0];
    s.hi[1] = mu_hi[1];
    const int n_out = s.n_out;
    Views v = views(m);
    stats_kernel<<<(n_out + 127) / 128, 128, 0, m->stream>>>(n, n_out, uhat, n_out, v.mean, v.stdv);
    ST_TRY(st_check_launch("mlp stats"));
    Acts a;
    ST_TRY(acts(m, n, &a));
    ST_TRY(st_grow(m, m->ws_misc, 256));
    float* d_loss = (float*)m->ws_misc.p;
    gather_kernel<<<grid1d(m, (int64_t)n * (n_out + 1)), NT, 0, m->stream>>>(
        n, 0, n, 1, 0, mu, s.lo[0], s.lo[1], s.hi[0], s.hi[1], a.X, uhat, n_out, n_out, v.mean, v.stdv, a.T);
    ST_TRY(st_check_launch("mlp gather"));
    ST_TRY(forward(m, v, a, n, true));
    ST_TRY(backward(m, v, a, n, d_loss));
    ST_CUDA_TRY(cudaStreamSynchronize(m->stream));
    if (grad) ST_CUDA_TRY(cudaMemcpy(grad, v.Gd, sizeof(float) * s.n_params, cudaMemcpyDeviceToHost));
    if (loss) ST_CUDA_TRY(cudaMemcpy(loss, d_loss, sizeof(float), cudaMemcpyDeviceToHost));
    s.trained = false;
    return ST_OK;
}

st_status st_internal_mlp_install(st_model* m, int hidden, const float* params, const float* adam_m,
                                  const float* adam_v, const double* mean, const double* stdv, const double* lo,
                                  const double* hi, int64_t adam_t) {
    auto& s = m->mlp;
    if (hidden != s.hidden) return st_fail(ST_ERR_ARG, "saved surrogate: hidden width %d is not %d", hidden, s.hidden);
    ST_TRY(setup(m, params, 0));
    const size_t np = (size_t)s.n_params, no = (size_t)s.n_out;
    ST_CUDA_TRY(cudaMemcpyAsync(s.adam_m.p, adam_m, sizeof(float) * np, cudaMemcpyHostToDevice, m->stream));
    ST_CUDA_TRY(cudaMemcpyAsync(s.adam_v.p, adam_v, sizeof(float) * np, cudaMemcpyHostToDevice, m->stream));
    ST_CUDA_TRY(cudaMemcpyAsync(s.stats.p, mean, sizeof(double) * no, cudaMemcpyHostToDevice, m->stream));
    ST_CUDA_TRY(cudaMemcpyAsync((double*)s.stats.p + no, stdv, sizeof(double) * no, cudaMemcpyHostToDevice,
                                m->stream));
    ST_CUDA_TRY(cudaStreamSynchronize(m->stream));
    s.lo[0] = lo[0];
    s.lo[1] = lo[1];
    s.hi[0] = hi[0];
    s.hi[1] = hi[1];
    s.adam_t = adam_t;
    s.trained = true;
    return ST_OK;
}

// ---------------------------------------------------------------------------
// Preconditioned refinement of the reduced space-time solves.
//
// Ahat^st(mu) is affine in theta(mu), and the systems at nearby parameters
// are close: with P_g = Ahat^st(mu_g)^{-1} at the reference parameter mu_g
// nearest to mu, the Richardson iteration
//     x <- x + P_g (fhat^st - Ahat^st(mu) x)
// contracts fast (||I - P_g Ahat^st(mu)|| small).  Each step is two batched
// products over the batch: the residual through the affine pieces K_q of
// Ahat^st (the gate's operator) and the correction through P_g, with the
// samples sorted by reference so that every 64-row tile of the correction
// product uses one P_g.  The start is the surrogate's prediction (or zero),
// so the network's accuracy buys iterations; answers still above the gate
// after the iterations fall back to the batched LU.
namespace {

constexpr int kTile = 64;  // rows per tile of the batched products

// [A | I] of Ahat^st(theta_g) in FP32 (row major, ld 2n), one reference per
// blockIdx.y
__global__ void ref_assemble_kernel(int ns, int nt, int Q, const double* __restrict__ Ahat,
                                    const double* __restrict__ G, const double* __restrict__ M,
                                    const double* __restrict__ S, const double* __restrict__ theta, float* aug) {
    const int n = ns * nt, g = blockIdx.y;
    const double* th = theta + (int64_t)g * Q;
    float* A = aug + (int64_t)g * n * 2 * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)n * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int row = (int)(t / n), col = (int)(t % n);
        const int ip = row % ns, jp = row / ns, i = col % ns, j = col / ns;
        double ah = 0.0;
        for (int q = 0; q < Q; ++q) ah = fma(th[q], Ahat[(int64_t)q * ns * ns + ip + (int64_t)i * ns], ah);
        double v = -ah * G[(int64_t)row + (int64_t)col * n];
        if (ip == i) v += M[(int64_t)i * nt * nt + jp + (int64_t)j * nt] - S[(int64_t)i * nt * nt + jp + (int64_t)j * nt];
        A[(int64_t)row * 2 * n + col] = (float)v;
        A[(int64_t)row * 2 * n + n + col] = row == col ? 1.f : 0.f;
    }
}

// Gauss-Jordan elimination with partial pivoting of [A | I] (one CTA per
// reference): leaves A^{-1} in the right half.  A zero pivot sets *err.
__global__ void __launch_bounds__(1024) gauss_jordan_kernel(int n, float* aug, int32_t* err) {
    __shared__ float s_mult[4096];
    __shared__ float s_v[32];
    __shared__ int s_i[32];
    __shared__ int s_piv;
    float* A = aug + (int64_t)blockIdx.x * n * 2 * n;
    const int ld = 2 * n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int k = 0; k < n; ++k) {
        // pivot: largest |A[i][k]|, i >= k (smallest index on ties)
        float best = -1.f;
        int bi = n;
        for (int i = k + tid; i < n; i += blockDim.x) {
            const float v = fabsf(A[(int64_t)i * ld + k]);
            if (v > best) {
                best = v;
                bi = i;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            s_v[warp] = best;
            s_i[warp] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            float b = -1.f;
            int p = n;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                if (s_v[w] > b || (s_v[w] == b && s_i[w] < p)) {
                    b = s_v[w];
                    p = s_i[w];
                }
            if (!(b > 0.f)) {
                atomicCAS(reinterpret_cast<int*>(err), 0, ST_ERR_SINGULAR);
                p = k;
            }
            s_piv = p;
        }
        __syncthreads();
        const int p = s_piv;
        // swap rows k and p, then scale row k by 1 / pivot
        if (p != k)
            for (int c = tid; c < ld; c += blockDim.x) {
                const float a = A[(int64_t)k * ld + c];
                A[(int64_t)k * ld + c] = A[(int64_t)p * ld + c];
                A[(int64_t)p * ld + c] = a;
            }
        __syncthreads();
        const float piv = A[(int64_t)k * ld + k];
        const float inv = piv != 0.f ? 1.f / piv : 0.f;
        __syncthreads();
        for (int c = tid; c < ld; c += blockDim.x) A[(int64_t)k * ld + c] *= inv;
        for (int i = tid; i < n; i += blockDim.x) s_mult[i] = i == k ? 0.f : A[(int64_t)i * ld + k];
        __syncthreads();
        // eliminate column k from every other row: columns k .. 2n - 1 (the
        // A part left of k is already zero there; with row exchanges the
        // right half's nonzeros can sit in any column)
        const int w = ld - k;
        for (int64_t t = tid; t < (int64_t)n * w; t += blockDim.x) {
            const int i = (int)(t / w), c = k + (int)(t % w);
            const float mlt = s_mult[i];
            if (mlt != 0.f) A[(int64_t)i * ld + c] = fmaf(-mlt, A[(int64_t)k * ld + c], A[(int64_t)i * ld + c]);
        }
        __syncthreads();
    }
}

// P[g] (n x n, row major) = right half of aug[g]
__global__ void ref_extract_kernel(int n, int n_ref, const float* __restrict__ aug, float* P) {
    const int64_t tot = (int64_t)n_ref * n * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = t / ((int64_t)n * n), rc = t % ((int64_t)n * n);
        const int64_t r = rc / n, c = rc % n;
        P[t] = aug[g * n * 2 * n + r * 2 * n + n + c];
    }
}

// nearest reference of every sample (coordinates scaled by the references'
// spread), and the per-reference counts
__global__ void ref_assign_kernel(int n, const double* __restrict__ mu, int n_ref, const double* __restrict__ mu_ref,
                                  double s0, double s1, int* grp, int* hist) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        double best = 1e300;
        int bg = 0;
        for (int g = 0; g < n_ref; ++g) {
            const double d0 = (mu[2 * p] - mu_ref[2 * g]) * s0, d1 = (mu[2 * p + 1] - mu_ref[2 * g + 1]) * s1;
            const double d = d0 * d0 + d1 * d1;
            if (d < best) {
                best = d;
                bg = g;
            }
        }
        grp[p] = bg;
        atomicAdd(hist + bg, 1);
    }
}

// sorted position of every sample: its reference's (tile-aligned) offset
// plus a slot; perm maps sorted rows back to samples (-1 for padding)
__global__ void ref_place_kernel(int n, const int* __restrict__ grp, const int* __restrict__ off, int* fill,
                                 int* perm, int* pos) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int g = grp[p];
        const int s = off[g] + atomicAdd(fill + g, 1);
        perm[s] = p;
        pos[p] = s;
    }
}

// dst[pos[p]] = src[p] (rows of nf doubles), or the reverse
__global__ void rows_move_kernel(int n, int nf, const int* __restrict__ pos, const double* __restrict__ src,
                                 double* dst, int to_sorted) {
    const int64_t tot = (int64_t)n * nf;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = t / nf, j = t % nf;
        if (to_sorted) dst[(int64_t)pos[p] * nf + j] = src[t];
        else dst[t] = src[(int64_t)pos[p] * nf + j];
    }
}

// sorted row b: r = rhs - (K_0 x - sum_q theta_q K_q x) from the products C
// (FP32 products combined in FP64), rel = ||r|| / ||rhs||; rows above the
// gate are counted.  Padding rows give r = 0.
__global__ void refine_residual_kernel(int rows, int n, int Q, const float* __restrict__ C, const int* __restrict__ perm,
                                       const double* __restrict__ theta, const double* __restrict__ rhs, double gate,
                                       double* Rs, double* rel, unsigned int* n_above) {
    const int b = blockIdx.x;
    if (b >= rows) return;
    __shared__ double s_r[8], s_f[8];
    const int p = perm[b];
    double rr = 0.0, ff = 0.0;
    const float* c = C + (int64_t)b * (Q + 1) * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double v = 0.0;
        if (p >= 0) {
            v = (double)c[j];
            for (int q = 0; q < Q; ++q) v -= theta[(int64_t)p * Q + q] * (double)c[(int64_t)(q + 1) * n + j];
            v = rhs[j] - v;
        }
        Rs[(int64_t)b * n + j] = v;
        rr += v * v;
        ff += rhs[j] * rhs[j];
    }
    rr = warp_sum(rr);
    ff = warp_sum(ff);
    if ((threadIdx.x & 31) == 0) {
        s_r[threadIdx.x >> 5] = rr;
        s_f[threadIdx.x >> 5] = ff;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, f = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += s_r[w];
            f += s_f[w];
        }
        const double r = p < 0 ? 0.0 : (f > 0.0 ? sqrt(a / f) : sqrt(a));
        rel[b] = r;
        if (p >= 0 && !(r <= gate)) atomicAdd(n_above, 1u);
    }
}

// X[b] += P_g R[b] for the sorted rows, g = the reference of the row's tile
// (64 x 64 output tiles, FP32 products, FP64 accumulation into X)
__global__ void __launch_bounds__(256) ref_correct_kernel(int rows, int n, const double* __restrict__ Rm,
                                                          const float* __restrict__ P, const int* __restrict__ tile_ref,
                                                          double* X) {
    __shared__ float su[16][65];
    __shared__ float sk[16][65];
    const int b0 = blockIdx.y * kTile, r0 = blockIdx.x * kTile;
    const float* K = P + (int64_t)tile_ref[blockIdx.y] * n * n;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < n; k0 += 16) {
        for (int l = threadIdx.x; l < 64 * 16; l += 256) {
            const int rr = l / 16, kk = l % 16;
            su[kk][rr] = (b0 + rr < rows && k0 + kk < n) ? (float)Rm[(int64_t)(b0 + rr) * n + k0 + kk] : 0.f;
            sk[kk][rr] = (r0 + rr < n && k0 + kk < n) ? K[(int64_t)(r0 + rr) * n + k0 + kk] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], c[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = su[kk][ty + 16 * q];
                c[q] = sk[kk][tx + 16 * q];
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], c[y], acc[x][y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int b = b0 + ty + 16 * x, r = r0 + tx + 16 * y;
            if (b < rows && r < n) X[(int64_t)b * n + r] += (double)acc[x][y];
        }
}

// ---- the residual products on the tensor cores ------------------------------
// C = X K_all^T with both operands split into three BF16 parts, x = x1 + x2 +
// x3 (8 significant bits each, x2 and x3 the rounded remainders), and the six
// cross products with i + j <= 4 accumulated in FP32 by one BF16 GEMM over
// the concatenated K: A' = [x1 x1 x1 x2 x2 x3], B' = [k1 k2 k3 k1 k2 k1].  The
// products are as accurate as FP32 ones (the dropped terms are 2^-24 of the
// product); the GEMM is the tcgen05 kernel of the surrogate.

__device__ __forceinline__ void split3(double x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
    a = __double2bfloat16(x);
    const double r1 = x - (double)__bfloat162float(a);
    b = __double2bfloat16(r1);
    const double r2 = r1 - (double)__bfloat162float(b);
    c = __double2bfloat16(r2);
}

// A'[b] = [x1 x1 x1 x2 x2 x3] for the rows of X (rows x n, ld ldx)
__global__ void split_rows_kernel(int rows, int n, const double* __restrict__ X, int ldx, __nv_bfloat16* A) {
    const int64_t tot = (int64_t)rows * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / n, k = t % n;
        __nv_bfloat16 x1, x2, x3;
        split3(X[b * ldx + k], x1, x2, x3);
        __nv_bfloat16* a = A + b * 6 * n + k;
        a[0] = x1;
        a[n] = x1;
        a[2 * n] = x1;
        a[3 * n] = x2;
        a[4 * n] = x2;
        a[5 * n] = x3;
    }
}

// B'[r] = [k1 k2 k3 k1 k2 k1] for the rows r of K_all (the affine pieces of
// Ahat^st, formed in FP64 as in kall_kernel)
__global__ void kall_split_kernel(int ns, int nt, int Q, const double* __restrict__ Ahat, const double* __restrict__ G,
                                  const double* __restrict__ M, const double* __restrict__ S, __nv_bfloat16* Bp) {
    const int n = ns * nt;
    const int64_t tot = (int64_t)(Q + 1) * n * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(t / ((int64_t)n * n));
        const int64_t rc = t % ((int64_t)n * n);
        const int row = (int)(rc / n), col = (int)(rc % n);
        const int ip = row % ns, jp = row / ns, i = col % ns, j = col / ns;
        double v;
        if (q == 0) {
            v = (ip == i) ? M[(int64_t)i * nt * nt + jp + (int64_t)j * nt] - S[(int64_t)i * nt * nt + jp + (int64_t)j * nt] : 0.0;
        } else {
            v = Ahat[(int64_t)(q - 1) * ns * ns + ip + (int64_t)i * ns] * G[(int64_t)row + (int64_t)col * n];
        }
        __nv_bfloat16 k1, k2, k3;
        split3(v, k1, k2, k3);
        __nv_bfloat16* b = Bp + ((int64_t)q * n + row) * 6 * n + col;
        b[0] = k1;
        b[n] = k2;
        b[2 * n] = k3;
        b[3 * n] = k1;
        b[4 * n] = k2;
        b[5 * n] = k1;
    }
}

bool tc_residual_ok(const st_model* m) { return (m->ns * m->nt) % 4 == 0; }

// B' for the model's reduced operators (rebuilt on every call that uses it)
st_status residual_prepare(st_model* m) {
    const int n = m->ns * m->nt, R = (m->Q + 1) * n;
    ST_TRY(st_grow(m, m->mlp.kall16, sizeof(__nv_bfloat16) * (size_t)R * 6 * n + 256));
    kall_split_kernel<<<grid1d(m, (int64_t)R * n), NT, 0, m->stream>>>(m->ns, m->nt, m->Q, m->d_Ahat, m->d_G, m->d_M,
                                                                      m->d_S, (__nv_bfloat16*)m->mlp.kall16.p);
    return st_check_launch("kall split");
}

// C (rows x R, FP32) = X (rows x n, FP64, ld ldx) K_all^T on the tensor cores
st_status residual_products(st_model* m, int rows, const double* X, int ldx, float* C) {
    const int n = m->ns * m->nt, R = (m->Q + 1) * n;
    ST_TRY(st_grow(m, m->mlp.xsplit, sizeof(__nv_bfloat16) * (size_t)rows * 6 * n + 256));
    __nv_bfloat16* A = (__nv_bfloat16*)m->mlp.xsplit.p;
    {
        ST_PROF(m, "residual_split_kernel");
        split_rows_kernel<<<grid1d(m, (int64_t)rows * n), NT, 0, m->stream>>>(rows, n, X, ldx, A);
        ST_TRY(st_check_launch("residual split"));
    }
    tc::GemmArgs g = epi(m);
    g.out_f32 = C;
    g.ldf = R;
    return st_tc_gemm(m, bn_for(R), rows, R, 6 * n, A, 6 * n, (const __nv_bfloat16*)m->mlp.kall16.p, 6 * n, g);
}

// per sample: the final residual of its sorted row; 1 and a slot in the
// fallback list when it is above the gate (or not finite)
__global__ void refine_verdict_kernel(int n, const int* __restrict__ pos, const double* __restrict__ rel, double gate,
                                      double* rel_res, int32_t* used, int* list, unsigned int* count) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const double r = rel[pos[p]];
        const bool ok = isfinite(r) && r <= gate;
        rel_res[p] = r;
        used[p] = ok ? 0 : 1;
        if (!ok) list[atomicAdd(count, 1u)] = p;
    }
}

}  // namespace

extern "C" st_status st_rom_precond_build(st_model* m, int32_t n_ref, const double* mu_ref, const double* theta_ref) {
    if (!m) return st_fail(ST_ERR_ARG, "st_rom_precond_build: NULL model");
    if (!m->assembled) return st_fail(ST_ERR_STATE, "st_rom_precond_build: reduced operators not assembled");
    if (n_ref < 1 || n_ref > 1024 || !mu_ref || !theta_ref) return st_fail(ST_ERR_ARG, "st_rom_precond_build: bad arguments");
    const int n = m->ns * m->nt, Q = m->Q;
    if (n > 4096) return st_fail(ST_ERR_ARG, "st_rom_precond_build: ns*nt = %d above 4096", n);
    auto& P = m->prec;
    P.n_ref = 0;
    const size_t aug = (size_t)n_ref * n * 2 * n, inv = (size_t)n_ref * n * n;
    ST_TRY(st_grow(m, P.work, sizeof(float) * aug + sizeof(double) * (size_t)n_ref * (Q + 2) + 256));
    ST_TRY(st_grow(m, P.inv, sizeof(float) * inv));
    float* d_aug = (float*)P.work.p;
    double* d_theta = (double*)(d_aug + aug + (aug & 1));
    cudaStream_t st = m->stream;
    ST_CUDA_TRY(cudaMemcpyAsync(d_theta, theta_ref, sizeof(double) * n_ref * Q, cudaMemcpyHostToDevice, st));
    {
        ST_PROF(m, "precond_build_kernels");
        const int gx = (int)std::min<int64_t>(((int64_t)n * n + 255) / 256, 1024);
        ref_assemble_kernel<<<dim3(gx, n_ref), 256, 0, st>>>(m->ns, m->nt, Q, m->d_Ahat, m->d_G, m->d_M, m->d_S,
                                                             d_theta, d_aug);
        ST_TRY(st_check_launch("precond assemble"));
        gauss_jordan_kernel<<<n_ref, 1024, 0, st>>>(n, d_aug, m->d_err);
        ST_TRY(st_check_launch("precond inverse"));
        ref_extract_kernel<<<grid1d(m, (int64_t)inv), NT, 0, st>>>(n, n_ref, d_aug, (float*)P.inv.p);
        ST_TRY(st_check_launch("precond extract"));
    }
    ST_TRY(st_sync(m));
    P.mu.assign(mu_ref, mu_ref + 2 * (size_t)n_ref);
    P.n_ref = n_ref;
    P.n = n;
    return ST_OK;
}

extern "C" st_status st_rom_refine(st_model* m, int32_t n, const double* mu, const double* theta, int32_t guess,
                                   double gate, int32_t max_iter, double* uhat, double* rel_res,
                                   int32_t* used_fallback, int32_t* iters_run, int32_t* n_fallback) {
    if (!m) return st_fail(ST_ERR_ARG, "st_rom_refine: NULL model");
    if (!m->assembled) return st_fail(ST_ERR_STATE, "st_rom_refine: reduced operators not assembled");
    const int nf = m->ns * m->nt, Q = m->Q, R = (Q + 1) * nf;
    auto& P = m->prec;
    auto& s = m->mlp;
    if (P.n_ref < 1 || P.n != nf) return st_fail(ST_ERR_STATE, "st_rom_refine: no preconditioner for this basis");
    if (guess != ST_GUESS_SURROGATE && guess != ST_GUESS_ZERO) return st_fail(ST_ERR_ARG, "st_rom_refine: bad guess");
    if (guess == ST_GUESS_SURROGATE && (!s.trained || s.n_out != nf))
        return st_fail(ST_ERR_STATE, "st_rom_refine: no trained surrogate for this basis");
    if (n < 0 || (n > 0 && (!mu || !theta || !uhat || !rel_res || !used_fallback)) || !(gate >= 0) || max_iter < 0)
        return st_fail(ST_ERR_ARG, "st_rom_refine: bad arguments");
    if (n == 0) {
        if (n_fallback) *n_fallback = 0;
        if (iters_run) *iters_run = 0;
        return ST_OK;
    }
    cudaStream_t st = m->stream;
    // 1. start: the surrogate's prediction, or zero
    if (guess == ST_GUESS_SURROGATE) {
        Views v = views(m);
        const int chunk = 65536;
        Acts a;
        ST_TRY(acts(m, std::min(n, chunk), &a));
        for (int b0 = 0; b0 < n; b0 += chunk) {
            const int bb = std::min(chunk, n - b0);
            gather_kernel<<<grid1d(m, bb), NT, 0, st>>>(bb, 0, bb, 1, 0, mu + 2 * (int64_t)b0, s.lo[0], s.lo[1],
                                                        s.hi[0], s.hi[1], a.X, nullptr, 0, nf, nullptr, nullptr,
                                                        nullptr);
            ST_TRY(st_check_launch("refine gather"));
            ST_TRY(forward(m, v, a, bb, false));
            denorm_kernel<<<grid1d(m, (int64_t)bb * nf), NT, 0, st>>>(bb, nf, a.Y, v.mean, v.stdv,
                                                                      uhat + (int64_t)b0 * nf, nf);
            ST_TRY(st_check_launch("refine denorm"));
        }
    } else {
        ST_CUDA_TRY(cudaMemsetAsync(uhat, 0, sizeof(double) * (size_t)n * nf, st));
    }
    // 2. the affine pieces of Ahat^st (three-part BF16 splits for the
    //    tensor-core products, or FP32 for the SIMT ones)
    const bool tc = tc_residual_ok(m);
    if (tc) {
        ST_TRY(residual_prepare(m));
    } else {
        ST_TRY(st_grow(m, s.kall, sizeof(float) * (size_t)R * nf));
        kall_kernel<<<grid1d(m, (int64_t)R * nf), NT, 0, st>>>(m->ns, m->nt, Q, m->d_Ahat, m->d_G, m->d_M, m->d_S,
                                                               (float*)s.kall.p);
        ST_TRY(st_check_launch("refine kall"));
    }
    // 3. samples sorted by nearest reference, each reference's rows padded to
    //    whole tiles
    const int nr = P.n_ref;
    double lo[2] = {1e300, 1e300}, hi[2] = {-1e300, -1e300};
    for (int g = 0; g < nr; ++g)
        for (int c = 0; c < 2; ++c) {
            lo[c] = std::min(lo[c], P.mu[2 * g + c]);
            hi[c] = std::max(hi[c], P.mu[2 * g + c]);
        }
    const double sc0 = hi[0] > lo[0] ? 1.0 / (hi[0] - lo[0]) : 1.0, sc1 = hi[1] > lo[1] ? 1.0 / (hi[1] - lo[1]) : 1.0;
    const int64_t rows_max = (int64_t)n + (int64_t)nr * kTile;
    const size_t ints = (size_t)2 * n + rows_max + 3 * (size_t)nr + (size_t)rows_max / kTile + 64;
    const size_t dbl = (size_t)rows_max * nf * 2 + rows_max + 2 * (size_t)nr;
    const size_t flt = (size_t)rows_max * R;
    ST_TRY(st_grow(m, m->ws_misc, sizeof(double) * dbl + sizeof(float) * flt + sizeof(int) * ints + 1024));
    double* Xs = (double*)m->ws_misc.p;
    double* Rs = Xs + (size_t)rows_max * nf;
    double* rel = Rs + (size_t)rows_max * nf;
    double* d_mur = rel + rows_max;
    float* C = (float*)(d_mur + 2 * (size_t)nr);
    int* grp = (int*)(C + flt);
    int* pos = grp + n;
    int* perm = pos + n;
    int* hist = perm + rows_max;
    int* off = hist + nr;
    int* fill = off + nr;
    int* tile_ref = fill + nr;
    unsigned int* cnt = (unsigned int*)(tile_ref + rows_max / kTile + 8);
    ST_CUDA_TRY(cudaMemcpyAsync(d_mur, P.mu.data(), sizeof(double) * 2 * nr, cudaMemcpyHostToDevice, st));
    ST_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(int) * 2 * nr + sizeof(int) * nr, st));
    ref_assign_kernel<<<grid1d(m, n), NT, 0, st>>>(n, mu, nr, d_mur, sc0, sc1, grp, hist);
    ST_TRY(st_check_launch("refine assign"));
    std::vector<int> h_hist(nr), h_off(nr), h_tiles;
    ST_CUDA_TRY(cudaMemcpyAsync(h_hist.data(), hist, sizeof(int) * nr, cudaMemcpyDeviceToHost, st));
    ST_CUDA_TRY(cudaStreamSynchronize(st));
    int rows = 0;
    for (int g = 0; g < nr; ++g) {
        h_off[g] = rows;
        const int t = (h_hist[g] + kTile - 1) / kTile;
        for (int i = 0; i < t; ++i) h_tiles.push_back(g);
        rows += t * kTile;
    }
    ST_CUDA_TRY(cudaMemcpyAsync(off, h_off.data(), sizeof(int) * nr, cudaMemcpyHostToDevice, st));
    ST_CUDA_TRY(cudaMemcpyAsync(tile_ref, h_tiles.data(), sizeof(int) * h_tiles.size(), cudaMemcpyHostToDevice, st));
    ST_CUDA_TRY(cudaMemsetAsync(fill, 0, sizeof(int) * nr, st));
    ST_CUDA_TRY(cudaMemsetAsync(perm, 0xff, sizeof(int) * rows, st));
    ref_place_kernel<<<grid1d(m, n), NT, 0, st>>>(n, grp, off, fill, perm, pos);
    ST_TRY(st_check_launch("refine place"));
    ST_CUDA_TRY(cudaMemsetAsync(Xs, 0, sizeof(double) * (size_t)rows * nf, st));
    rows_move_kernel<<<grid1d(m, (int64_t)n * nf), NT, 0, st>>>(n, nf, pos, uhat, Xs, 1);
    ST_TRY(st_check_launch("refine to sorted"));
    // 4. residual, then correction, until every row meets the gate
    int it = 0;
    for (;; ++it) {
        if (tc) {
            ST_TRY(residual_products(m, rows, Xs, nf, C));
        } else {
            ST_PROF(m, "gate_gemm_kernel");
            gate_gemm_kernel<<<dim3((R + 63) / 64, (rows + 63) / 64), 256, 0, st>>>(rows, R, nf, Xs, nf,
                                                                                   (float*)s.kall.p, C);
            ST_TRY(st_check_launch("refine residual products"));
        }
        ST_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned int), st));
        refine_residual_kernel<<<rows, 128, 0, st>>>(rows, nf, Q, C, perm, theta, m->d_rhs, gate, Rs, rel, cnt);
        ST_TRY(st_check_launch("refine residual"));
        unsigned int above = 0;
        ST_CUDA_TRY(cudaMemcpyAsync(&above, cnt, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
        ST_CUDA_TRY(cudaStreamSynchronize(st));
        if (above == 0 || it >= max_iter) break;
        ST_PROF(m, "precond_correct_kernel");
        ref_correct_kernel<<<dim3((nf + kTile - 1) / kTile, rows / kTile), 256, 0, st>>>(rows, nf, Rs,
                                                                                      (const float*)P.inv.p,
                                                                                      tile_ref, Xs);
        ST_TRY(st_check_launch("refine correction"));
    }
    if (iters_run) *iters_run = it;
    // 5. back to the samples' order; the gate's verdict; LU for the rest
    rows_move_kernel<<<grid1d(m, (int64_t)n * nf), NT, 0, st>>>(n, nf, pos, Xs, uhat, 0);
    ST_TRY(st_check_launch("refine from sorted"));
    ST_TRY(st_grow(m, s.list, sizeof(int) * (size_t)n + 64));
    int* list = (int*)s.list.p;
    unsigned int* lcount = (unsigned int*)(list + n);
    ST_CUDA_TRY(cudaMemsetAsync(lcount, 0, sizeof(unsigned int), st));
    refine_verdict_kernel<<<grid1d(m, n), NT, 0, st>>>(n, pos, rel, gate, rel_res, used_fallback, list, lcount);
    ST_TRY(st_check_launch("refine verdict"));
    unsigned int hc = 0;
    ST_CUDA_TRY(cudaMemcpyAsync(&hc, lcount, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    ST_CUDA_TRY(cudaStreamSynchronize(st));
    if (n_fallback) *n_fallback = (int32_t)hc;
    return st_internal_solve_list(m, (int)hc, list, theta, uhat, rel_res, nullptr);
}
