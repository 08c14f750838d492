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
    // gate operator
    ST_TRY(st_grow(m, s.kall, sizeof(float) * (size_t)R * n_out));
    kall_kernel<<<grid1d(m, (int64_t)R * n_out), NT, 0, st>>>(m->ns, m->nt, Q, m->d_Ahat, m->d_G, m->d_M, m->d_S,
                                                             (float*)s.kall.p);
    ST_TRY(st_check_launch("mlp kall"));
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
        {
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
