// FP64 GEMM on the BF16 tensor cores by exact splitting of the operands (the
// error-free transformation of matrix products of Ozaki, Ogita, Oishi and
// Rump, Numer. Algorithms 59, 2012), for the products of the incremental SVD.
//
// The dot-product vectors are the rows of op(A) and the columns of op(B).
// Each is scaled by a power of two 2^e with all its entries in (-1, 1), and
// every scaled entry is written with eight balanced base-128 digits,
//     x 2^-e = sum_t d_t 2^(-7(t+1)),   |d_t| <= 64,
// exact to 2^-55 of the vector's scale (the scale is one power of two above
// the largest entry, so the leading digit stays within 64 too).  The digits
// are small integers, exact in BF16.  A product of two entries is the sum of
// the digit products d_s d_t 2^(-7(s+t+2)); the pairs with s + t <= 7 are
// kept (the dropped ones weigh below 2^-55 of the scales' product).  All
// pairs of one diagonal D = s + t share a power of two, so one FP32
// accumulator in tensor memory per diagonal sums them over a K chunk of at
// most 448: every term is an integer of magnitude <= 2^12, a diagonal has at
// most 8 pairs, and 8 * 2^12 * 448 < 2^24, so every partial sum is an integer below
// 2^24 in magnitude that FP32 holds exactly, in whatever order the tensor
// core adds.  The epilogue turns the eight exact sums into two 64-bit integers and
// scales them into FP64; the chunks of a long K are added in FP64 in a fixed
// order.  The result is deterministic and as accurate as an FP64 GEMM.
//
// GB300 issues FP64 at 1/64 of its FP32 rate while its BF16 tensor cores run
// near 2 PFLOP/s, so the 36 digit-pair products per output cost less than
// the FP64 multiply-adds they replace; what remains in FP64 is a handful of
// operations per output and K chunk.
#include <cuda.h>

#include <algorithm>
#include <climits>

#include "internal.h"
#include "tc_host.h"

namespace {

constexpr int kSlices = 8;  // digits per entry
constexpr int kDiags = 8;   // kept diagonals D = 0..7
constexpr int kBM = 128, kBN = 64, kBK = 64;
constexpr int kChunk = 448;  // longest K of one exact accumulation (7 stages)
constexpr int kARing = 6;    // A digit-plane tiles in flight
constexpr int kThreads = 256;  // 8 warps: two per 32-lane quarter of the accumulators
constexpr uint32_t kTileA = kBM * kBK * 2;      // one digit plane of the A tile (16 KB)
constexpr uint32_t kPlaneB = kBN * kBK * 2;     // one digit plane of the B tile (8 KB)
constexpr uint32_t kTileB = kSlices * kPlaneB;  // all planes of the B tile (64 KB)
constexpr size_t kSmem = 2 * (size_t)kTileB + kARing * (size_t)kTileA + 1024;
constexpr uint32_t kTmemCols = kDiags * kBN;  // 512: the whole tensor memory
constexpr int kTile = 64;                     // split kernels: 64 x 64 element tiles
static_assert(kChunk % kBK == 0, "chunk of whole K stages");
static_assert(8LL * 4096 * kChunk < (1LL << 24), "exact FP32 sums of one diagonal over a chunk");
static_assert(kTmemCols <= 512, "accumulators fit the tensor memory");

// ---- splitting ---------------------------------------------------------------

// Element (i, k) of an operand whose rows are the dot-product vectors.
template <bool kRowContig>
__device__ __forceinline__ double elem(const double* p, int64_t ld, int64_t i, int64_t k) {
    return kRowContig ? p[i * ld + k] : p[i + k * ld];
}

// Largest biased exponent field of each row (integer max, independent of
// order).  A row's scale is 2^(emax - 1021): every |x| < 2^(E - 1022).
template <bool kRowContig>
__global__ void __launch_bounds__(256) exp_kernel(int64_t R, int64_t K, const double* __restrict__ p, int64_t ld,
                                                  int32_t* emax, int32_t* err) {
    __shared__ int s_max[kTile];
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * kTile, k0 = (int64_t)blockIdx.y * kTile;
    if (tid < kTile) s_max[tid] = 0;
    __syncthreads();
    int local = 0;
    bool bad = false;
#pragma unroll 4
    for (int it = 0; it < kTile * kTile / 256; ++it) {
        const int idx = tid + 256 * it;
        const int r = kRowContig ? idx / kTile : idx % kTile;
        const int kk = kRowContig ? idx % kTile : idx / kTile;
        const int64_t i = r0 + r, k = k0 + kk;
        int e = 0;
        if (i < R && k < K) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(elem<kRowContig>(p, ld, i, k));
            e = (int)((b >> 52) & 0x7FF);
            if (e == 0x7FF) {
                bad = true;
                e = 0;
            }
        }
        if (kRowContig) {
            // the 32 lanes of a warp read one row
            e = __reduce_max_sync(0xffffffffu, e);
            if ((tid & 31) == 0 && e > 0) atomicMax(&s_max[r], e);
        } else {
            local = max(local, e);  // a thread reads one row
        }
    }
    if (!kRowContig && local > 0) atomicMax(&s_max[tid % kTile], local);
    if (bad) st_dev_error(err, ST_ERR_NONFINITE);
    __syncthreads();
    if (tid < kTile && r0 + tid < R && s_max[tid] > 0) atomicMax(&emax[r0 + tid], s_max[tid]);
}

// Balanced base-128 digits of |x| 2^(56 - e) (e = emax - 1021: the row
// scale), sign on every digit, packed as BF16 into plane t of `packed` at
// half-word h.
//
// The scaled magnitude X < 2^55 is cut into three 21-bit chunks (bits 0-20,
// 21-41, 42-54), each an exact FP32 value (2^23 + c - 2^23), so that the
// digits come from FP32 operations, all exact: q = rint(f / 128) (by the
// rounding constant 1.5 * 2^23; |f| / 128 < 2^15), r = f - 128 q with
// |r| <= 64, and the quotient carried into the next chunk.  A chunk holds
// three digits; the last quotient is the leading digit (X < 2^55: |d_0| <=
// 64).  A digit is an integer of at most seven bits, so its BF16 pattern is
// the upper half of its FP32 pattern.  (The integer pipe, which bit-by-bit
// digit and BF16 arithmetic would load, is half as wide as the FP32 one.)
__device__ __forceinline__ void put_digits(double x, int emax, uint32_t (&packed)[kSlices][4], int h) {
    static_assert(kSlices == 8, "three 21-bit chunks of three, three and two digits");
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    unsigned long long X = 0;
    if (E != 0 && E != 0x7FF) {
        const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int s = E - emax + 2;  // <= 2: X < 2^55
        X = s >= 0 ? mant << s : (s > -64 ? mant >> (-s) : 0ull);
    }
    const uint32_t lo = (uint32_t)X, hi = (uint32_t)(X >> 32);
    const float sg = (b >> 63) ? -1.0f : 1.0f;
    constexpr float kTwo23 = 8388608.0f, kRound = 12582912.0f;
    float f0 = sg * (__uint_as_float(0x4B000000u | (lo & 0x1FFFFFu)) - kTwo23);
    float f1 = sg * (__uint_as_float(0x4B000000u | (((lo >> 21) | (hi << 11)) & 0x1FFFFFu)) - kTwo23);
    float f2 = sg * (__uint_as_float(0x4B000000u | (hi >> 10)) - kTwo23);
    float d[kSlices];
    auto step = [&](float& f) -> float {
        const float q = __fadd_rn(__fmul_rn(f, 0.0078125f), kRound) - kRound;
        const float r = __fmaf_rn(-128.0f, q, f);
        f = q;
        return r;
    };
    d[7] = step(f0);
    d[6] = step(f0);
    d[5] = step(f0);
    f1 += f0;
    d[4] = step(f1);
    d[3] = step(f1);
    d[2] = step(f1);
    f2 += f1;
    d[1] = step(f2);
    d[0] = f2;
#pragma unroll
    for (int t = 0; t < kSlices; ++t) {
        const uint32_t bits = __float_as_uint(d[t]);
        packed[t][h >> 1] |= (h & 1) ? (bits & 0xFFFF0000u) : (bits >> 16);
    }
}

// Digit planes: plane t holds digit t of every element, row-major R x Kp
// (K contiguous), zero in the K padding.  The grid covers R x Kp (its last
// row tile may stick out of R: those rows are skipped).
template <bool kRowContig>
__global__ void __launch_bounds__(256) split_kernel(int64_t R, int64_t K, int64_t Kp, const double* __restrict__ p,
                                                    int64_t ld, const int32_t* __restrict__ emax,
                                                    uint16_t* __restrict__ planes, int64_t plane) {
    __shared__ double tile[kTile][kTile + 1];
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * kTile, k0 = (int64_t)blockIdx.y * kTile;
#pragma unroll 4
    for (int it = 0; it < kTile * kTile / 256; ++it) {
        const int idx = tid + 256 * it;
        const int r = kRowContig ? idx / kTile : idx % kTile;
        const int kk = kRowContig ? idx % kTile : idx / kTile;
        const int64_t i = r0 + r, k = k0 + kk;
        tile[r][kk] = (i < R && k < K) ? elem<kRowContig>(p, ld, i, k) : 0.0;
    }
    __syncthreads();
#pragma unroll 1
    for (int q = 0; q < 2; ++q) {
        // eight lanes cover the 64 K of a row: 128-byte stores per plane
        const int task = tid + 256 * q;
        const int r = task / 8, g = task % 8;
        const int64_t i = r0 + r, k = k0 + 8 * g;
        if (i >= R) continue;
        const int em = emax[i];
        uint32_t packed[kSlices][4];
#pragma unroll
        for (int t = 0; t < kSlices; ++t)
#pragma unroll
            for (int w = 0; w < 4; ++w) packed[t][w] = 0u;
#pragma unroll
        for (int e = 0; e < 8; ++e) put_digits(tile[r][8 * g + e], em, packed, e);
        uint16_t* dst = planes + i * Kp + k;
#pragma unroll
        for (int t = 0; t < kSlices; ++t)
            *reinterpret_cast<uint4*>(dst + (int64_t)t * plane) =
                make_uint4(packed[t][0], packed[t][1], packed[t][2], packed[t][3]);
    }
}

// ---- tensor-core product ---------------------------------------------------

struct OzArgs {
    int M, N, K;
    int chunk;          // K per CTA: a multiple of kBK, at most kChunk
    const int32_t* ea;  // [M] exponent fields of the rows of op(A)
    const int32_t* eb;  // [N] exponent fields of the columns of op(B)
    double alpha, beta;
    double* C;
    int64_t ldc;
    double* part;  // [chunks][M x N] partial products, or null (single chunk)
    int32_t* err;
    long long limit;
    int n_fast;  // grid x runs over the N tiles (y over the M tiles), else the reverse
};

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

// Eight FP32 accumulator columns of this thread's lane; the registers pass
// through the wait so no use can be scheduled before the load completes.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
                 :
                 : "memory");
}

// 2^p as a double (0 below the normal range, +inf above it).
__device__ __forceinline__ double pow2(int p) {
    if (p < -1022) return 0.0;
    if (p > 1023) return __longlong_as_double(0x7FF0000000000000ll);
    return __longlong_as_double((long long)(p + 1023) << 52);
}

// One CTA: a 128 x 64 tile of C over one K chunk.  Warp 0 (one thread)
// streams the K stages of the chunk: the eight B digit planes of a stage (one
// 3-D TMA box, double buffered) and, one plane at a time, the A digit planes
// through a ring of six stages.  Warp 1 (one thread) issues, for A plane s,
// the products with B planes t = 0..7-s into accumulator D = s + t (M = 128,
// N = 64, K = 16 each) and releases each stage with tcgen05.commit, so the
// products run back to back while the copies of the next planes land.  Each
// of the eight warps then reads 32 rows x 32 columns of the eight
// accumulators (warps w and w + 4 share a 32-lane quarter) and combines them;
// the old values of C it updates are loaded before the wait for the products,
// so their latency hides behind the main loop.  Every wait is bounded; on a timeout the CTA records ST_ERR_TIMEOUT,
// lets its copies and products land, frees its tensor memory and returns.
__global__ void __launch_bounds__(kThreads, 1) oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                              const __grid_constant__ CUtensorMap tmB, OzArgs g) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bars[2 * kARing + 5];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail;
    __shared__ double s_cs[kBN];  // column scales (alpha folded in unless partial)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t base = (tc::smem_u32(smem_raw) + 1023u) & ~1023u;
    const uint32_t sB0 = base, sA0 = base + 2 * kTileB;
    const uint32_t a_full = tc::smem_u32(&bars[0]), a_empty = tc::smem_u32(&bars[kARing]);
    const uint32_t b_full = tc::smem_u32(&bars[2 * kARing]), b_empty = tc::smem_u32(&bars[2 * kARing + 2]);
    const uint32_t done = tc::smem_u32(&bars[2 * kARing + 4]);
    const int m0 = (g.n_fast ? blockIdx.y : blockIdx.x) * kBM, n0 = (g.n_fast ? blockIdx.x : blockIdx.y) * kBN;
    const int chunk = blockIdx.z;
    const int kbeg = chunk * g.chunk;
    const int klen = min(g.chunk, g.K - kbeg);
    const int nks = (klen + kBK - 1) / kBK;
    const int nA = nks * kSlices;

    if (tid == 0) {
        for (int s = 0; s < 2 * kARing + 5; ++s) tc::mbar_init(tc::smem_u32(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (tid < kBN) {
        const int col = n0 + tid;
        const double sc = col < g.N ? pow2(g.eb[col] - 1021) : 0.0;
        s_cs[tid] = g.part ? sc : g.alpha * sc;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc::smem_u32(&tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (tid == 0) {
        // producer: B planes of stage ks, then its eight A planes
        int a_issued = 0, b_issued = 0;
        bool ok = true;
        for (int ks = 0; ks < nks && ok; ++ks) {
            const int b = ks & 1;
            if (ks >= 2 && !tc::mbar_wait(b_empty + 8 * b, ((ks >> 1) - 1) & 1, g.limit)) {
                ok = false;
                break;
            }
            tc::mbar_expect_tx(b_full + 8 * b, kTileB);
            tma_load_3d(sB0 + b * kTileB, &tmB, kbeg + ks * kBK, n0, 0, b_full + 8 * b);
            ++b_issued;
            for (int sa = 0; sa < kSlices; ++sa) {
                const int n = ks * kSlices + sa, slot = n % kARing;
                if (n >= kARing && !tc::mbar_wait(a_empty + 8 * slot, ((n / kARing) - 1) & 1, g.limit)) {
                    ok = false;
                    break;
                }
                tc::mbar_expect_tx(a_full + 8 * slot, kTileA);
                tma_load_3d(sA0 + slot * kTileA, &tmA, kbeg + ks * kBK, m0, sa, a_full + 8 * slot);
                ++a_issued;
            }
        }
        if (!ok) {
            s_fail = 1;
            // let the copies still in flight land before the CTA exits
            for (int n = max(0, a_issued - kARing); n < a_issued; ++n)
                tc::mbar_wait(a_full + 8 * (n % kARing), (n / kARing) & 1, g.limit);
            for (int ks = max(0, b_issued - 2); ks < b_issued; ++ks)
                tc::mbar_wait(b_full + 8 * (ks & 1), (ks >> 1) & 1, g.limit);
        }
    } else if (tid == 32) {
        // MMA issuer
        const uint32_t idesc = tc::idesc_bf16(kBM, kBN);
        for (int n = 0; n < nA; ++n) {
            const int ks = n / kSlices, sa = n % kSlices, slot = n % kARing;
            if (sa == 0 && !tc::mbar_wait(b_full + 8 * (ks & 1), (ks >> 1) & 1, g.limit)) {
                s_fail = 1;
                break;
            }
            if (!tc::mbar_wait(a_full + 8 * slot, (n / kARing) & 1, g.limit)) {
                s_fail = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa_addr = sA0 + slot * kTileA, sb_addr = sB0 + (ks & 1) * kTileB;
            for (int sb = 0; sb < kSlices - sa; ++sb) {
                const uint32_t acc = tmem + (uint32_t)((sa + sb) * kBN);
#pragma unroll
                for (int kk = 0; kk < kBK / 16; ++kk)
                    tc::umma_bf16(acc, tc::sdesc_sw128(sa_addr + kk * 32),
                                  tc::sdesc_sw128(sb_addr + sb * kPlaneB + kk * 32), idesc,
                                  (ks > 0 || sa > 0 || kk > 0) ? 1u : 0u);
            }
            tc::umma_commit(a_empty + 8 * slot);
            if (sa == kSlices - 1) tc::umma_commit(b_empty + 8 * (ks & 1));
        }
        tc::umma_commit(done);
    }
    // epilogue mapping: lane quarter q = warp % 4 (rows), column half h
    const int q = warp & 3, h = warp >> 2;
    const int row = m0 + q * 32 + lane;
    const bool has_row = row < g.M;
    double* part = g.part ? g.part + (size_t)chunk * g.M * g.N : nullptr;
    const int mode = part ? 0 : (g.beta == 0.0 ? 1 : (g.beta == 1.0 ? 2 : 3));
    constexpr int kCols = kBN / 2;
    double cold[kCols];
    if (mode >= 2) {
        // old values of C, loaded while the products run
#pragma unroll
        for (int c = 0; c < kCols; ++c) {
            const int col = n0 + h * kCols + c;
            cold[c] = (has_row && col < g.N) ? g.C[row + (size_t)col * g.ldc] : 0.0;
        }
    }
    __syncthreads();
    if (!tc::mbar_wait(done, 0, g.limit)) s_fail = 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (!s_fail) {
        const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * kCols);
        // value = (S_hi 2^-35 + S_lo 2^-63) 2^(ea - 1021) 2^(eb - 1021)
        const int ea = has_row ? g.ea[row] : 0;
        const double p_hi = pow2(ea - 1021 - 35), p_lo = pow2(ea - 1021 - 63);
#pragma unroll
        for (int j0 = 0; j0 < kCols; j0 += 8) {
            if (n0 + h * kCols + j0 >= g.N) break;  // warp-uniform
            uint32_t v[kDiags][8];
#pragma unroll
            for (int d = 0; d < kDiags; ++d) tmem_ld8(trow + (uint32_t)(d * kBN + j0), v[d]);
            if (!has_row) continue;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int jc = h * kCols + j0 + c, col = n0 + jc;
                if (col >= g.N) break;
                long long hi = 0, lo = 0;
#pragma unroll
                for (int d = 0; d < 4; ++d) hi = hi * 128 + (long long)__float2int_rn(__uint_as_float(v[d][c]));
#pragma unroll
                for (int d = 4; d < 8; ++d) lo = lo * 128 + (long long)__float2int_rn(__uint_as_float(v[d][c]));
                const double val = fma((double)hi, p_hi, (double)lo * p_lo);
                const double cs = s_cs[jc];
                if (mode == 0) {
                    part[row + (size_t)col * g.M] = val * cs;
                } else {
                    double* cp = g.C + row + (size_t)col * g.ldc;
                    if (mode == 1) *cp = val * cs;
                    else if (mode == 2) *cp = fma(val, cs, cold[j0 + c]);
                    else *cp = fma(val, cs, g.beta * cold[j0 + c]);
                }
            }
        }
    } else if (tid == 0) {
        st_dev_error(g.err, ST_ERR_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// C = alpha * sum_c part[c] + beta * C, chunks added in order.
__global__ void oz_reduce_kernel(int64_t M, int64_t N, int chunks, const double* __restrict__ part, double alpha,
                                 double beta, double* C, int64_t ldc) {
    const int64_t n = M * N;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < chunks; ++c) s += part[(size_t)c * n + t];
        const int64_t i = t % M, j = t / M;
        double* cp = C + i + j * ldc;
        *cp = beta == 0.0 ? alpha * s : fma(alpha, s, beta * *cp);
    }
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

void st_oz_invalidate(st_model* m) {
    for (OzSlot& sl : m->oz_slot) sl.valid = false;
}

st_status st_ozaki_gemm(st_model* m, bool transA, bool transB, int64_t M, int64_t Nc, int64_t K, double alpha,
                        const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                        int64_t ldc, int slotA, bool reuseA) {
    if (M <= 0 || Nc <= 0) return ST_OK;
    if (K <= 0) return st_dgemm(m, transA, transB, M, Nc, K, alpha, A, lda, B, ldb, beta, C, ldc);
    if (M > INT_MAX / 2 || Nc > INT_MAX / 2 || K > INT_MAX / 2)
        return st_fail(ST_ERR_ARG, "st_ozaki_gemm: dimensions too large");
    // K padded to whole stages with zero digits; the rows of the planes are
    // not padded: the TMA boxes past the last row read zeros
    const int64_t Kp = (K + kBK - 1) / kBK * kBK;
    // K per CTA: the whole stages (up to kChunk) that minimise the waves of
    // CTAs over the SMs times the work of one CTA (its stages plus ~2 stages
    // of epilogue); a long-K product with few output tiles gets shorter
    // chunks so that its CTAs fill the SMs
    int64_t chunk = kChunk;
    {
        const int64_t tiles = ((M + kBM - 1) / kBM) * ((Nc + kBN - 1) / kBN);
        double best = 1e300;
        for (int s = kChunk / kBK; s >= 1; --s) {
            const int64_t c = (int64_t)s * kBK, nch = (K + c - 1) / c;
            const int64_t waves = (tiles * nch + m->num_sms - 1) / m->num_sms;
            const double cost = (double)waves * (std::min<int64_t>(s, (K + kBK - 1) / kBK) + 2);
            if (cost < best - 1e-9) {
                best = cost;
                chunk = c;
            }
        }
    }
    const int64_t chunks = (K + chunk - 1) / chunk;
    if (Kp / kTile > 65535 || (Nc + kBN - 1) / kBN > 65535 || chunks > 65535)
        return st_fail(ST_ERR_ARG, "st_ozaki_gemm: grid too large");
    if (slotA >= kOzSlots) return st_fail(ST_ERR_ARG, "st_ozaki_gemm: bad operand slot");
    // workspace: A planes (unless cached), B planes, exponents, chunk partials
    const size_t bytesA = align256(sizeof(uint16_t) * kSlices * (size_t)M * Kp);
    const size_t bytesB = align256(sizeof(uint16_t) * kSlices * (size_t)Nc * Kp);
    const size_t bytesE = align256(sizeof(int32_t) * (size_t)(M + Nc));
    const size_t bytesP = chunks > 1 ? sizeof(double) * (size_t)chunks * M * Nc : 0;
    const size_t ownA = slotA >= 0 ? 0 : bytesA;
    ST_TRY(st_grow(m, m->ws_oz, ownA + bytesB + bytesE + bytesP));
    uint8_t* ws = (uint8_t*)m->ws_oz.p;
    uint16_t* planesA = (uint16_t*)ws;
    uint16_t* planesB = (uint16_t*)(ws + ownA);
    int32_t* ea = (int32_t*)(ws + ownA + bytesB);
    int32_t* eb = ea + M;
    double* part = chunks > 1 ? (double*)(ws + ownA + bytesB + bytesE) : nullptr;
    bool sliceA = true;
    if (slotA >= 0) {
        OzSlot& sl = m->oz_slot[slotA];
        const bool same = sl.valid && sl.src == A && sl.ld == lda && sl.rows == M && sl.K == K &&
                          sl.transposed == transA;
        sliceA = !(reuseA && same);
        if (sliceA) {
            sl.valid = false;
            ST_TRY(st_grow(m, sl.planes, bytesA));
            ST_TRY(st_grow(m, sl.exps, sizeof(int32_t) * (size_t)M));
        }
        planesA = (uint16_t*)sl.planes.p;
        ea = (int32_t*)sl.exps.p;
    }
    cudaStream_t st = m->stream;
    {
        ST_PROF(m, "ozaki_split_kernels");
        const dim3 ga((unsigned)((M + kTile - 1) / kTile), (unsigned)((K + kTile - 1) / kTile));
        const dim3 gb((unsigned)((Nc + kTile - 1) / kTile), (unsigned)((K + kTile - 1) / kTile));
        const dim3 sa(ga.x, (unsigned)(Kp / kTile)), sb(gb.x, (unsigned)(Kp / kTile));
        if (sliceA) {
            // rows of op(A): A^T's rows are A's columns (contiguous)
            ST_CUDA_TRY(cudaMemsetAsync(ea, 0, sizeof(int32_t) * (size_t)M, st));
            if (transA) exp_kernel<true><<<ga, 256, 0, st>>>(M, K, A, lda, ea, m->d_err);
            else exp_kernel<false><<<ga, 256, 0, st>>>(M, K, A, lda, ea, m->d_err);
            ST_TRY(st_check_launch("ozaki exp A"));
            if (transA) split_kernel<true><<<sa, 256, 0, st>>>(M, K, Kp, A, lda, ea, planesA, M * Kp);
            else split_kernel<false><<<sa, 256, 0, st>>>(M, K, Kp, A, lda, ea, planesA, M * Kp);
            ST_TRY(st_check_launch("ozaki split A"));
            if (slotA >= 0) {
                OzSlot& sl = m->oz_slot[slotA];
                sl.src = A;
                sl.ld = lda;
                sl.rows = M;
                sl.K = K;
                sl.transposed = transA;
                sl.valid = true;
            }
        }
        // columns of op(B): B's columns (contiguous) unless transposed
        ST_CUDA_TRY(cudaMemsetAsync(eb, 0, sizeof(int32_t) * (size_t)Nc, st));
        if (!transB) exp_kernel<true><<<gb, 256, 0, st>>>(Nc, K, B, ldb, eb, m->d_err);
        else exp_kernel<false><<<gb, 256, 0, st>>>(Nc, K, B, ldb, eb, m->d_err);
        ST_TRY(st_check_launch("ozaki exp B"));
        if (!transB) split_kernel<true><<<sb, 256, 0, st>>>(Nc, K, Kp, B, ldb, eb, planesB, Nc * Kp);
        else split_kernel<false><<<sb, 256, 0, st>>>(Nc, K, Kp, B, ldb, eb, planesB, Nc * Kp);
        ST_TRY(st_check_launch("ozaki split B"));
    }
    CUtensorMap ta, tb;
    ST_TRY(st_tmap_bf16_3d(&ta, planesA, Kp, M, kSlices, Kp, M * Kp, kBK, kBM, 1));
    ST_TRY(st_tmap_bf16_3d(&tb, planesB, Kp, Nc, kSlices, Kp, Nc * Kp, kBK, kBN, kSlices));
    // tile order: with more M tiles than N tiles the N tiles run fastest, so
    // that the CTAs of a wave share the digit planes of a few M tiles (a tall
    // product would otherwise stream all of op(A)'s planes once per N tile)
    const int64_t mt = (M + kBM - 1) / kBM, nt = (Nc + kBN - 1) / kBN;
    const int n_fast = mt > nt ? 1 : 0;
    OzArgs g{(int)M, (int)Nc, (int)K, (int)chunk, ea, eb, alpha, beta, C, ldc, part, m->d_err, m->opt.spin_limit,
             n_fast};
    {
        ST_PROF(m, "ozaki_gemm_kernel");
        st_prof_flops(m, "ozaki_gemm_kernel", 2.0 * (double)M * (double)Nc * (double)K);
        static bool attr = false;
        if (!attr) {
            ST_CUDA_TRY(cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
            attr = true;
        }
        const dim3 grid((unsigned)(n_fast ? nt : mt), (unsigned)(n_fast ? mt : nt), (unsigned)chunks);
        oz_gemm_kernel<<<grid, kThreads, kSmem, st>>>(ta, tb, g);
        ST_TRY(st_check_launch("ozaki gemm"));
    }
    if (chunks > 1) {
        ST_PROF(m, "ozaki_reduce_kernel");
        const int blocks = (int)std::min<int64_t>((M * Nc + 255) / 256, 8 * (int64_t)m->num_sms);
        oz_reduce_kernel<<<blocks, 256, 0, st>>>(M, Nc, (int)chunks, part, alpha, beta, C, ldc);
        ST_TRY(st_check_launch("ozaki reduce"));
    }
    return ST_OK;
}
