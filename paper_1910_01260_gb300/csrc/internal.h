// Internal declarations shared by the translation units of libst_rom.so.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "st_rom.h"

// Slice height of the sliced-ELL layout (one warp-row group per slice).
constexpr int kSlice = 32;

// Growable device buffer owned by a model.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Per-kernel timing (st_profile_enable): CUDA events recorded around each
// launch on the model's stream, read back by st_profile_read.
struct ProfState {
    bool on = false;
    struct Rec {
        const char* name;
        cudaEvent_t a, b;
    };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    std::vector<std::string> names;
    std::vector<double> ms;
    std::vector<int64_t> launches;
    std::vector<double> flops;
};

// Digit planes of one operand of the tensor-core FP64 GEMM kept across calls
// (the basis W and the block's directions J of the incremental SVD), with the
// key of the matrix they were made from.
struct OzSlot {
    DevBuf planes, exps;
    const double* src = nullptr;
    int64_t ld = 0, rows = 0, K = 0;
    bool transposed = false, valid = false;
};
constexpr int kOzSlots = 4;

struct st_model {
    int device = 0;
    cudaStream_t stream = nullptr;
    st_options opt{};
    int num_sms = 0;

    // affine operator terms as given (host CSR, kept for st_model_save)
    std::vector<int64_t> h_rowptr;
    std::vector<int32_t> h_col;
    std::vector<double> h_vals;  // Q x nnz
    // affine operator terms in sliced-ELL form
    int64_t N = 0, nnz = 0;
    int Q = 0;
    int64_t n_slices = 0, ell_size = 0;
    int max_width = 0;
    int64_t* d_slice_ptr = nullptr;  // [n_slices + 1] entry offsets
    int32_t* d_slice_w = nullptr;    // [n_slices] widths
    int32_t* d_col = nullptr;        // [ell_size]
    double* d_vals = nullptr;        // [Q * ell_size]
    // the same operator split by affine term for the full-order march:
    // entries with several nonzero terms ("mixed", per-sample values built
    // at march time from d_vals via d_mx_src), and per term q the entries
    // where only term q is nonzero (one shared value, scaled by theta_q once
    // per row).  Each group is sliced-ELL with its own widths.
    int64_t mx_size = 0, tq_size = 0;
    int64_t* d_mx_ptr = nullptr;  // [n_slices + 1]
    int32_t* d_mx_w = nullptr;    // [n_slices]
    int32_t* d_mx_col = nullptr;  // [mx_size]
    int64_t* d_mx_src = nullptr;  // [mx_size] entry of d_vals, -1 for padding
    int64_t* d_tq_ptr = nullptr;  // [n_slices * Q + 1]
    int32_t* d_tq_w = nullptr;    // [n_slices * Q]
    int32_t* d_tq_col = nullptr;  // [tq_size]
    double* d_tq_val = nullptr;   // [tq_size]

    // bases
    int ns = 0, nt = 0, Nt = 0;
    double* d_phi = nullptr;  // N x ns
    double* d_T = nullptr;    // Nt x ns*nt

    // incremental SVD state
    int pod_r = 0;
    int64_t pod_rows = 0;  // snapshot columns consumed (rows of V)
    int64_t pod_ldv = 0;   // leading dimension of V
    DevBuf W, V;
    std::vector<double> sigma;
    // per block update of the last basis build: middle-matrix Jacobi sweeps,
    // and the number of Gram-Schmidt re-orthogonalisations of W
    std::vector<int> pod_sweeps;
    int pod_reorth = 0;
    ProfState prof;

    // reduced operators
    bool assembled = false;
    double* d_Ahat = nullptr;  // Q x ns x ns
    double* d_G = nullptr;     // n x n
    float* d_G32 = nullptr;    // n x n (FP32 copy for the FP32 assembly mode)
    double* d_M = nullptr;     // ns x nt x nt
    double* d_S = nullptr;     // ns x nt x nt
    double* d_rhs = nullptr;   // n: fhat^st + uhat0^st
    double* d_dt = nullptr;    // Nt
    double* d_bs = nullptr;    // ns x Nt: Bhat f^k of the spatial ROM in column k-1
    double* d_u0s = nullptr;   // ns: Phi_s^T u0 (zero without u0)

    // device error word and barrier counters
    int32_t* d_err = nullptr;
    unsigned int* d_bar = nullptr;  // [4]: arrival count, generation, abort flag, queue head

    // scratch buffers (grown on demand, reused across calls)
    DevBuf ws_fom, ws_pod, ws_pod2, ws_gemm, ws_oz, ws_solve, ws_misc, ws_srom, ws_cert;
    // reference preconditioner of the reduced space-time systems: FP32
    // inverses of Ahat^st at n_ref reference parameters (n x n each, row
    // major) and those parameters
    struct Precond {
        int n_ref = 0, n = 0;
        std::vector<double> mu;  // [n_ref x 2]
        DevBuf inv, work;
    } prec;
    // the transposed terms A_q^T (built on first use by the Theorem 3
    // stability-constant estimate)
    st_model* adj = nullptr;
    OzSlot oz_slot[kOzSlots];

    // launch plan of the batched reduced solve per factor precision ([0] FP64
    // factors, [1] FP32 factors): panel width, CTAs per SM, queue order (0 =
    // library default), set by st_rom_solve_set_plan or st_rom_solve_tune
    struct SolvePlanCfg {
        int nb = 0, per_sm = 0, order = 0;
    } solve_cfg[2];

    // learned surrogate mu -> uhat (3-layer MLP, FP32 masters, BF16 copies)
    struct Mlp {
        int n_in = 2, hidden = 256, n_out = 0;
        int64_t n_params = 0;
        bool trained = false;
        int64_t adam_t = 0;
        double lo[2] = {0, 0}, hi[2] = {1, 1};
        DevBuf params, grad, adam_m, adam_v, wbf, stats, act, kall, list;
        DevBuf kall16, xsplit;  // BF16 three-part splits for the tensor-core residual product
    } mlp;
};

// ---- error handling -------------------------------------------------------
void st_set_error(const char* fmt, ...);
st_status st_fail(st_status code, const char* fmt, ...);

#define ST_CUDA_TRY(call)                                                              \
    do {                                                                               \
        cudaError_t e__ = (call);                                                      \
        if (e__ != cudaSuccess)                                                        \
            return st_fail(e__ == cudaErrorMemoryAllocation ? ST_ERR_OOM : ST_ERR_CUDA, \
                           "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e__),      \
                           __FILE__, __LINE__);                                        \
    } while (0)

#define ST_TRY(expr)                  \
    do {                              \
        st_status s__ = (expr);       \
        if (s__ != ST_OK) return s__; \
    } while (0)

// Make sure buf holds at least `bytes`; synchronises the model stream before
// releasing a smaller buffer that queued work may still use.
st_status st_grow(st_model* m, DevBuf& buf, size_t bytes);
st_status st_check_launch(const char* what);
// Scope timer: while profiling is on, records an event pair around the
// launches made inside the scope, attributed to `name` (a string literal).
struct ProfScope {
    st_model* m;
    const char* name;
    cudaEvent_t a = nullptr;
    ProfScope(st_model* model, const char* kernel);
    ~ProfScope();
};
#define ST_PROF_CAT2(a, b) a##b
#define ST_PROF_CAT(a, b) ST_PROF_CAT2(a, b)
// Add algorithmic flops to a kernel's profile entry (no-op unless profiling).
void st_prof_flops(st_model* m, const char* name, double flops);
#define ST_PROF(m, name) ProfScope ST_PROF_CAT(st_prof_scope_, __LINE__)((m), (name))
// Count one kernel launch (st_check_launch counts the launch it checks).
void st_count_launch();

// Number of co-resident blocks for a cooperative launch of `kernel`.
template <typename K>
int st_coop_blocks(st_model* m, K kernel, int threads, size_t smem, int per_sm_cap) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess)
        return 0;
    if (per_sm > per_sm_cap) per_sm = per_sm_cap;
    return per_sm * m->num_sms;
}

// ---- FP64 GEMM (column major): C = alpha * op(A) * op(B) + beta * C -------
// Batched with element strides sA, sB, sC.  For long K the product is split
// over K into a workspace and reduced in a fixed order (deterministic).
st_status st_dgemm(st_model* m, bool transA, bool transB, int64_t M, int64_t Ncols, int64_t K,
                   double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                   double beta, double* C, int64_t ldc, int batch = 1, int64_t sA = 0,
                   int64_t sB = 0, int64_t sC = 0);

// The same product on the BF16 tensor cores by exact operand splitting (batch
// 1; FP64-accurate, deterministic).  st_dgemm routes its large products here
// when options.fp64_gemm is ST_DGEMM_OZAKI.  With slotA >= 0 the digit planes
// of op(A) are kept in m->oz_slot[slotA]; reuseA = true asserts that A has not
// changed since that slot was filled from the same matrix (same pointer,
// leading dimension, shape and transposition), so its planes are used as
// they are.
st_status st_ozaki_gemm(st_model* m, bool transA, bool transB, int64_t M, int64_t Ncols, int64_t K, double alpha,
                        const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                        int64_t ldc, int slotA = -1, bool reuseA = false);
// st_dgemm with the operand-plane cache of the tensor-core path (ignored on
// the SIMT path).
st_status st_dgemm_slot(st_model* m, int slotA, bool reuseA, bool transA, bool transB, int64_t M, int64_t Ncols,
                        int64_t K, double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                        double beta, double* C, int64_t ldc);
// Forget every cached operand (the matrices they came from may change).
void st_oz_invalidate(st_model* m);

// Release basis (and reduced operators) / reduced operators only.
void st_internal_free_basis(st_model* m);
void st_internal_free_reduced(st_model* m);

// Solve the reduced systems of the samples listed in list[0..n_list) (full
// (ns, nt) of the model) with the batched LU kernel; same outputs as
// st_rom_solve for those samples.
st_status st_internal_solve_list(st_model* m, int n_list, const int* list, const double* theta,
                                 double* uhat, double* rel_res, int32_t* status);

// Install reduced operators from host arrays (layouts of the "REDU" section
// of a saved model; the FP32 copy of G is made on the device).
st_status st_internal_install_reduced(st_model* m, const double* Ahat, const double* G, const double* M,
                                      const double* S, const double* rhs, const double* dt, const double* bs,
                                      const double* u0s);
// Install a trained surrogate from host arrays (FP32 parameters and Adam
// moments, FP64 output statistics, the parameter box, the Adam step count).
st_status st_internal_mlp_install(st_model* m, int hidden, const float* params, const float* adam_m,
                                  const float* adam_v, const double* mean, const double* stdv, const double* lo,
                                  const double* hi, int64_t adam_t);

// The full-order march of st_fom_march with an optional per-step source
// src (dev [n_mu x Nt x N]) added to the right-hand side of step k.
st_status st_internal_fom_march(st_model* m, int32_t n_mu, const double* theta, int32_t Nt, const double* dt,
                                const double* u0, int32_t n_in, const double* B, const double* F,
                                const double* src, double* snapshots, int32_t* iters, int32_t* status);
