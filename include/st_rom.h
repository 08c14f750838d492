/*
 * st_rom.h -- C ABI of the GB300-native space-time reduced-order model for
 * parametric linear dynamical systems (Choi, Brown, Arrighi, Anderson,
 * "Space-time reduced order model for large-scale linear dynamical systems
 * with application to Boltzmann transport problems").
 *
 * Problem (Sec. 2, Eq. Dynamicalstate):  du/dt = A(mu) u + B f(t), u(0) = u0,
 * stepped by backward Euler (Eq. fom).  A(mu) is given in affine form
 * A(mu) = sum_q theta_q A_q over Q sparse terms that share one pattern; the
 * caller maps mu -> theta.
 *
 * Conventions used by every entry point:
 *  - Dense matrices are column major (Fortran order).  "dev" pointers are
 *    CUDA device pointers on the model's device; "host" pointers are ordinary
 *    host memory.  The caller owns every pointer it passes; the library owns
 *    the model handle and everything allocated inside it.
 *  - Calls are enqueued on the model's stream and return before the GPU work
 *    finishes, unless a call's comment says "synchronous".  Argument errors
 *    are returned immediately (ST_ERR_ARG / ST_ERR_STATE) and nothing is
 *    enqueued.  Errors detected on the device (non-convergence, breakdown,
 *    zero pivot, non-finite values, a device wait that hit its limit) are
 *    written to per-sample status arrays when the call takes one and to the
 *    model's error word, which st_sync() returns and clears.
 *  - Reduced unknowns are ordered i + ns*j (spatial mode i < ns fastest,
 *    temporal mode j < nt), as in Eq. spacetimebasis.
 *  - A model and its stream are used by one host thread at a time.
 *  - st_last_error() returns a thread-local message for the last failure.
 */
#ifndef ST_ROM_H
#define ST_ROM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t st_status;
#define ST_OK                0
#define ST_ERR_ARG           1  /* invalid argument (checked on the host)           */
#define ST_ERR_CUDA          2  /* a CUDA runtime call failed                       */
#define ST_ERR_OOM           3  /* device allocation failed                         */
#define ST_ERR_NOT_CONVERGED 4  /* iteration limit reached (BiCGSTAB, Jacobi SVD)   */
#define ST_ERR_BREAKDOWN     5  /* BiCGSTAB breakdown (rho or omega vanished)       */
#define ST_ERR_SINGULAR      6  /* zero pivot in the reduced LU factorisation       */
#define ST_ERR_NONFINITE     7  /* NaN or Inf met in device arithmetic              */
#define ST_ERR_TIMEOUT       8  /* a device-side wait exceeded options.spin_limit   */
#define ST_ERR_STATE         9  /* call out of order (e.g. solve before assemble)   */

/* Arithmetic of the reduced solve (st_options.precision). */
#define ST_FP64          0  /* FP64 assembly, FP64 LU, FP64 refinement                 */
#define ST_FP32_ASSEMBLY 1  /* FP32 assembly of Ahat^st, FP64 LU + FP64 refinement     */
#define ST_FP32_LU       2  /* FP32 assembly and LU factors, FP64 residual refinement   */

/* Arithmetic of the FP64 products of the basis construction and assembly
 * (st_options.fp64_gemm). */
#define ST_DGEMM_SIMT   0  /* FP64 multiply-adds on the SIMT cores                   */
#define ST_DGEMM_OZAKI  1  /* BF16 tensor cores on exact 8-digit operand splits
                              (Ozaki et al., Numer. Algorithms 59, 2012): FP64-
                              accurate, deterministic; used for products of at
                              least 2^20 flops with K >= 8                       */

/* Opaque model handle: operator terms, bases, reduced operators, workspace. */
typedef struct st_model st_model;

/* Affine sparse operator, host CSR (Sec. 2; the transport operator of
 * Sec. 6 is split into terms A_q).  All n_terms share rowptr/col. */
typedef struct {
    int64_t        n_rows;   /* N: spatial unknowns (square operator)            */
    const int64_t* rowptr;   /* host [N + 1], rowptr[0] = 0, non-decreasing       */
    const int32_t* col;      /* host [nnz], 0 <= col < N, unique within a row     */
    const double* const* vals; /* host [n_terms] pointers to nnz values of A_q    */
    int32_t        n_terms;  /* Q >= 1                                            */
} st_affine_csr;

typedef struct {
    double  tol;          /* BiCGSTAB: stop at ||r|| <= tol * ||rhs||        (1e-13)  */
    int32_t maxit;        /* BiCGSTAB iterations per time step               (1000)   */
    double  eps_svd;      /* incremental SVD dependence test, relative to the
                             largest column norm of the incoming block       (1e-12)  */
    double  eps_sv;       /* drop singular values < eps_sv * sigma_max       (1e-14)  */
    int32_t r_max;        /* rank cap of the incremental SVD                 (256)    */
    int32_t precision;    /* ST_FP64, ST_FP32_ASSEMBLY or ST_FP32_LU         (FP64)   */
    int64_t spin_limit;   /* polls of any device-side wait before it gives up
                             with ST_ERR_TIMEOUT (one poll ~ 0.1 us)         (2e7)    */
    int32_t refine_steps; /* iterative-refinement steps of the reduced solve (1)      */
    int32_t jacobi_sweeps;/* sweep cap of the one-sided Jacobi SVD           (40)     */
    int32_t pod_block;    /* parameter samples whose snapshots form one update
                             of the incremental SVD (block of pod_block * Nt
                             columns; the paper streams one sample's
                             snapshots, 1)                                   (1)      */
    int32_t fp64_gemm;    /* ST_DGEMM_SIMT or ST_DGEMM_OZAKI            (ST_DGEMM_OZAKI)  */
    int32_t pod_cols;     /* when > 0: consecutive snapshot columns per update
                             instead of whole samples; 1 streams one snapshot
                             per update, the rank-one update of Algorithm 2  (0)      */
    int32_t fom_path;     /* kernel of st_fom_march: ST_FOM_AUTO, ST_FOM_GRID or
                             ST_FOM_CLUSTER                                 (AUTO)    */
} st_options;

/* Kernel of the full-order march (st_options.fom_path). */
#define ST_FOM_AUTO     0  /* the faster kernel as measured on this library's
                              workloads: the grid march                              */
#define ST_FOM_GRID     1  /* one cooperative grid marching up to 32 samples in step  */
#define ST_FOM_CLUSTER  2  /* one 8-CTA thread-block cluster per sample; needs one
                              CTA's share of 4 vectors (4 * 8 * ceil(N/256) * 32
                              bytes) to fit 200 KB of shared memory (N <= ~51,000),
                              ST_ERR_ARG otherwise                                   */

/* Fill *opt with the defaults shown above. */
void st_options_default(st_options* opt);

/* Thread-local description of the last error returned on this thread. */
const char* st_last_error(void);

/* Static name of a status code. */
const char* st_status_string(st_status s);

/* Number of CUDA kernels this library has launched in this process (all
 * models, all devices); a diagnostic counter, never reset. */
int64_t st_kernel_launches(void);

/* Measured FP64 fused multiply-add throughput of the current device
 * (synchronous): blocks_per_sm x (SM count) blocks of 256 threads each run 16
 * independent FMA chains of `iters` steps, timed with CUDA events after one
 * shorter untimed launch.  *tflops = 2 * 16 * iters * threads / seconds / 1e12;
 * ms (may be NULL) receives the timed launch's milliseconds.  The roofline
 * denominator of the library's FP64-bound kernels.  ST_ERR_ARG for
 * blocks_per_sm outside [1, 32], iters < 1 or a NULL tflops. */
st_status st_probe_fp64_fma(int32_t blocks_per_sm, int64_t iters, double* tflops, double* ms);

/* Create a model on the current CUDA device.  Converts the host CSR terms to
 * the library's sliced-ELL layout and uploads them (synchronous).
 * stream: a cudaStream_t (NULL = the legacy default stream); the model keeps
 * it for every later call.  opt may be NULL (defaults).  On success *out
 * receives a handle that st_model_destroy releases.
 * Errors: ST_ERR_ARG (bad CSR), ST_ERR_OOM, ST_ERR_CUDA. */
st_status st_model_create(const st_affine_csr* A, const st_options* opt, void* stream,
                          st_model** out);

/* Replace the model's options (validated as in st_model_create); later calls
 * use them, e.g. a different precision or refinement count for st_rom_solve.
 * r_max changes take effect at the next st_rom_build_basis.  ST_ERR_ARG if
 * invalid (the old options stay). */
st_status st_model_set_options(st_model* m, const st_options* opt);

/* Copy the model's current options to *opt. */
st_status st_model_get_options(st_model* m, st_options* opt);

/* Release every resource of the model (synchronises its stream first). */
void st_model_destroy(st_model* m);

/* Wait for the model's stream, then return and clear the first device-side
 * error recorded since the previous st_sync (ST_OK if none). */
st_status st_sync(st_model* m);

/* Full-order snapshot march (Eq. fom):
 *   (I - dt_k A(mu_p)) u^k = u^{k-1} + dt_k B f^k,  k = 1..Nt, t_k = sum dt_j,
 * for n_mu parameter samples marched together; each step is solved by
 * BiCGSTAB on the sliced-ELL operator, with all iteration control on the
 * device, from the initial iterate x0 = sum_{i=0}^{o} (-1)^i C(o+1, i+1)
 * u^{k-1-i}, o = min(k-1, 4) (the degree-o extrapolation of the previous
 * levels, u^0 = u0; x0 = u0 at the first step); the stopping test
 * ||r|| <= tol ||rhs|| is on the true system.
 *   theta     host [n_mu x Q] row major: theta_q(mu_p) at theta[p*Q + q]
 *   dt        host [Nt] time steps
 *   u0        dev  [N] initial state shared by all samples, or NULL for 0
 *   B         dev  [N x n_in] input matrix; F host [Nt x n_in] row major, f^k
 *             at F[(k-1)*n_in + s]  (n_in may be 0: no input)
 *   snapshots dev  [N x (Nt*n_mu)]: column p*Nt + (k-1) receives u^k(mu_p),
 *             i.e. U = [U_1 ... U_nmu] of Eq. snapshotmat
 *   iters     dev  [Nt x n_mu] (or NULL): iterations of step k for sample p
 *             at iters[(k-1)*n_mu + p]
 *   status    dev  [n_mu] (or NULL): ST_OK, ST_ERR_NOT_CONVERGED,
 *             ST_ERR_BREAKDOWN, ST_ERR_NONFINITE or ST_ERR_TIMEOUT per sample;
 *             a failed sample stops marching, its later columns are zero.
 * 1 <= n_mu (processed in groups of at most 32), 1 <= Nt. */
st_status st_fom_march(st_model* m, int32_t n_mu, const double* theta, int32_t Nt,
                       const double* dt, const double* u0, int32_t n_in, const double* B,
                       const double* F, double* snapshots, int32_t* iters, int32_t* status);

/* Capacity of the cluster march on the current device for this model's
 * operator: CTAs per cluster (one cluster per parameter sample), the number
 * of such clusters the device runs at once (more samples run in waves), and
 * the dynamic shared memory per CTA (0: the operator is too large for the
 * cluster march).  Any pointer may be NULL. */
st_status st_fom_cluster_occupancy(st_model* m, int32_t* cluster_ctas, int32_t* max_active_clusters,
                                   int64_t* smem_bytes);

/* Spatial and temporal bases by the incremental POD of Secs. 4.1-4.2
 * (synchronous).  The snapshot matrix U = [U_1 ... U_nmu] (N x Nt*n_mu,
 * dev, column major, as written by st_fom_march) is consumed one parameter
 * block U_p at a time: projection on the current left singular vectors W,
 * column-wise Gram-Schmidt (two passes) of the remainder with the eps_svd
 * dependence test, a second block pass (the new directions are projected on W
 * again and re-orthogonalised), FP64 one-sided Jacobi SVD of the bordered
 * middle matrix (Eq. middleMat), update of W, sigma, V (Eqs.
 * rankOneUpdateSVD1-2), truncation by eps_sv and r_max.  Then
 * Phi_s = W(:, 1:ns) (Eq. spatialincrementalbasis) and, for each i < ns, the
 * temporal snapshot matrix Upsilon_i (Nt x n_mu) from the unscaled right
 * singular vector v_i (Eq. incrementaltemporalsnapshotmat) and its SVD give
 * Phi_t^i = Lambda_i(:, 1:nt) (Eq. temporalincrementalbasis).
 *   sigma  host [r_max] or NULL: singular values, descending, rank entries set
 *   rank   host or NULL: number of singular triplets kept (r)
 * Requires ns <= r and nt <= min(Nt, n_mu); ST_ERR_ARG otherwise.
 * Replaces any basis or reduced operators held by the model. */
st_status st_rom_build_basis(st_model* m, int32_t n_mu, int32_t Nt, const double* snapshots,
                             int32_t ns, int32_t nt, double* sigma, int32_t* rank);

/* Install caller-provided bases (e.g. to assemble from another POD).
 * phi_s dev [N x ns]; T dev [Nt x ns*nt] with column i + ns*j = phi_t^{i,j}
 * (Eq. spacetimebasisvec).  Copies them (asynchronous).  Clears reduced ops. */
st_status st_model_set_basis(st_model* m, int32_t ns, int32_t nt, int32_t Nt,
                             const double* phi_s, const double* T);

/* Copy the bases out.  phi_s dev [N x ns] or NULL, T dev [Nt x ns*nt] or
 * NULL; dims host [3] or NULL receives (ns, nt, Nt). */
st_status st_model_get_basis(st_model* m, double* phi_s, double* T, int32_t* dims);

/* Incremental-SVD state after st_rom_build_basis (synchronous copy):
 * W dev [N x r] or NULL, V dev [(Nt*n_mu) x r] or NULL, sigma host [r] or
 * NULL, r host or NULL. */
st_status st_pod_get_state(st_model* m, double* W, double* V, double* sigma, int32_t* r);

/* Per-kernel timing.  st_profile_enable(m, 1) makes every later call on the
 * model record a pair of CUDA events on the model's stream around each of
 * its kernel launches (a few microseconds of overhead per launch);
 * st_profile_enable(m, 0) stops it.  Either call synchronises the stream
 * and clears the totals.  st_profile_read synchronises and returns, for each
 * kernel name seen since the last enable, sorted by total time (largest
 * first): names [cap x ST_PROFILE_NAME_LEN] NUL-terminated, ms [cap] total
 * milliseconds, launches [cap], flops [cap] the algorithmic floating-point
 * operations the library can count on the host (2MNK per GEMM; norms, dot
 * products and 6(m + n) per applied rotation in the middle-matrix Jacobi
 * SVD; 0 where the count depends on device-side data); any of the four may
 * be NULL.  *n_kernels receives the number of names (which may exceed cap).
 * A name covers one kernel, or a kernel with its small helper (the split-K
 * reduction of a GEMM, the size sort of a batched solve). */
#define ST_PROFILE_NAME_LEN 64
st_status st_profile_enable(st_model* m, int32_t on);
st_status st_profile_read(st_model* m, int32_t cap, char* names, double* ms, int64_t* launches,
                          double* flops, int32_t* n_kernels);

/* Diagnostics of the last st_rom_build_basis (host, synchronous): the number
 * of block updates in *n_updates; the one-sided Jacobi sweeps of each
 * update's middle-matrix SVD in sweeps[0 .. min(n_updates, cap) - 1] (sweeps
 * may be NULL); the number of updates whose orthogonality check fired and
 * re-orthogonalised W in *n_reorth (may be NULL). */
st_status st_pod_get_stats(st_model* m, int32_t* n_updates, int32_t* sweeps, int32_t cap,
                           int32_t* n_reorth);

/* Resumable incremental SVD (Sec. 4.2, Algorithms 1-2).  The paper's
 * incremental SVD exists to fold snapshots in as they are produced, without
 * holding the whole snapshot matrix; these calls expose its state so a build
 * can be continued later (with st_model_save/st_model_load in between) or fed
 * group by group while the full-order march produces the next group.
 * st_rom_build_basis is st_pod_reset + st_pod_update (all columns, updates of
 * options.pod_block samples or options.pod_cols columns) + st_pod_finish.
 *
 * st_pod_reset: forget the state (r = 0, no columns consumed).
 * st_pod_update (synchronous): fold the n_cols columns at snapshots (dev,
 *   N x n_cols, column major) into the state, cols_per_update columns per
 *   update (the last update may be narrower; 1 = the rank-one update of
 *   Algorithm 2), with the truncation of options.eps_sv and options.r_max and
 *   the dependence test of options.eps_svd (relative to each update's largest
 *   column norm).  V gains n_cols rows.  ST_ERR_ARG for n_cols < 0 or
 *   cols_per_update < 1; device errors of the update as for st_rom_build_basis.
 * st_pod_finish (asynchronous after its checks): bases from the state,
 *   Phi_s = W(:, 1:ns) (Eq. spatialincrementalbasis) and Phi_t^i from V read as
 *   n_mu consecutive blocks of Nt rows (Eqs. incrementaltemporalsnapshotmat,
 *   temporalincrementalbasis), replacing any basis and reduced operators.
 *   Requires n_mu * Nt = columns consumed, ns <= r, nt <= min(Nt, n_mu);
 *   ST_ERR_ARG otherwise.
 * st_pod_set_state (synchronous): install a state: W dev [N x r], sigma host
 *   [r] (finite, >= 0, non-increasing), V dev [rows x r] (rows = snapshot
 *   columns the state stands for), all copied.  r = 0 clears W and sigma.
 *   W need not be exactly orthonormal: the next update's orthogonality check
 *   (end of Algorithm 2) re-orthogonalises it when |w_1^T w_r| exceeds
 *   min(eps_svd, eps N).
 * st_pod_get_dims: rank r and rows (columns consumed) of the state; either
 *   pointer may be NULL. */
st_status st_pod_reset(st_model* m);
st_status st_pod_update(st_model* m, int64_t n_cols, const double* snapshots, int32_t cols_per_update);
st_status st_pod_finish(st_model* m, int32_t n_mu, int32_t Nt, int32_t ns, int32_t nt);
st_status st_pod_set_state(st_model* m, int32_t r, int64_t rows, const double* W, const double* sigma,
                           const double* V);
st_status st_pod_get_dims(st_model* m, int32_t* r, int64_t* rows);

/* Persistence of a model (the offline stage's results, Secs. 4.2-4.3, for a
 * later online stage or a resumed basis build).
 * st_model_save (synchronous): writes the options, the affine operator, the
 *   incremental-SVD state (W, sigma, V, per-update sweep counts and
 *   re-orthogonalisations), the bases, the reduced operators and a trained
 *   surrogate (parameters, Adam moments and step, output statistics,
 *   parameter box) -- each part that exists -- to `path`, through a temporary
 *   file renamed at the end.  ST_ERR_ARG if the file cannot be written.
 * st_model_load (synchronous): creates a model on the current device with
 *   `stream` (as st_model_create) from such a file and restores every saved
 *   part; solves, reconstructions and surrogate inference then give the
 *   saved model's results bit for bit, and st_pod_update continues the build.
 *   ST_ERR_ARG for a missing, truncated or corrupt file (every section carries
 *   a checksum), ST_ERR_OOM / ST_ERR_CUDA as st_model_create.
 * st_model_file_info (host only, no GPU needed): validates a file as
 *   st_model_load does and reports what it holds.
 * File layout (little endian): "STROMMDL", u32 version 1, u32 section count,
 * then per section char tag[4], u32 0, u64 payload bytes, payload, u64
 * FNV-1a-64 of the payload; sections OPTS and OPER first, then any of PODS,
 * BASE, REDU, SURR (payload layouts are listed in the library's io.cu). */
typedef struct {
    int32_t version;    /* file format version                                  */
    int32_t n_terms;    /* Q                                                    */
    int64_t n_rows;     /* N                                                    */
    int64_t nnz;        /* stored entries of the operator pattern               */
    int64_t pod_rows;   /* snapshot columns the incremental SVD has consumed    */
    int32_t pod_rank;   /* r (0: no incremental-SVD state)                      */
    int32_t ns, nt, Nt; /* basis sizes (0: no basis)                            */
    int32_t assembled;  /* 1: reduced operators stored                          */
    int32_t surrogate;  /* 1: trained surrogate stored                          */
    int64_t n_params;   /* surrogate parameter count (0 without one)            */
} st_model_info;
st_status st_model_save(st_model* m, const char* path);
st_status st_model_load(const char* path, void* stream, st_model** out);
st_status st_model_file_info(const char* path, st_model_info* info);

/* The FP64 matrix product of the incremental SVD and of the assembly
 * (Sec. 4.2: projections of snapshot blocks on the basis, W^T U and
 * U - W (W^T U), and the basis rotation), on the model's stream with the
 * model's options.fp64_gemm:
 *     C = alpha op(A) op(B) + beta C,  op(A) M x K, op(B) K x N, C M x N,
 * column major; op(X) = X^T when trans_X is nonzero.  A, B, C are DEVICE
 * pointers with leading dimensions lda >= rows of A as stored, etc.; C must
 * not overlap A or B.  K = 0 scales C by beta.  Asynchronous: ST_ERR_ARG for
 * a NULL model or negative sizes; device-side NaN/Inf in an operand of the
 * tensor-core path is reported as ST_ERR_NONFINITE by a later
 * synchronising call. */
st_status st_gemm_f64(st_model* m, int32_t trans_a, int32_t trans_b, int64_t M, int64_t N, int64_t K,
                      double alpha, const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                      double* C, int64_t ldc);

/* Offline assembly of the space-time reduced operators through the block
 * structure of Sec. 4.3, never forming Phi_st:
 *   Ahat_q = Phi_s^T A_q Phi_s           (reduced system matrix, Eq. galerkin)
 *   G[(i',j'),(i,j)] = sum_k dt_k phi_{i'j'}[k] phi_{ij}[k]
 *   M_i[j',j] = sum_k phi_{ij'}[k] phi_{ij}[k]
 *   S_i[j',j] = sum_{k<Nt} phi_{ij'}[k+1] phi_{ij}[k]    (Eq. ij-block-matrix)
 *   fhat^st block j = sum_k dt_k D_k^j Phi_s^T B f^k     (Eq. j-block-vector)
 *   uhat0^st block j = D_1^j Phi_s^T u0  (Phi_st^T u0^st from Eq. ststate)
 * dt host [Nt]; B dev [N x n_in]; F host [Nt x n_in] row major; u0 dev [N]
 * or NULL.  Requires a basis.  Asynchronous. */
st_status st_rom_assemble(st_model* m, const double* dt, int32_t n_in, const double* B,
                          const double* F, const double* u0);

/* Copy the assembled reduced operators to host memory (synchronous); any
 * pointer may be NULL.  Ahat [Q x ns x ns] (term q at Ahat + q*ns*ns, column
 * major), G [n x n], M and S [ns x nt x nt] (mode i at + i*nt*nt, column
 * major), rhs [n] = fhat^st + uhat0^st, with n = ns*nt. */
st_status st_model_get_reduced(st_model* m, double* Ahat, double* G, double* M, double* S,
                               double* rhs);

/* Batched online solve of the space-time Galerkin system (Eq. st-galerkin)
 *   Ahat^st(mu) uhat = fhat^st + uhat0^st
 * with Ahat^st[(i',j'),(i,j)] = delta_{i'i} (M_i - S_i)[j',j]
 *                              - Ahat(mu)[i',i] G[(i',j'),(i,j)],
 * Ahat(mu) = sum_q theta_q Ahat_q, for n_mu samples with individual nested
 * sizes (ns_p <= ns, nt_p <= nt; the sub-basis i < ns_p, j < nt_p).  One
 * persistent kernel assembles, LU-factorises with partial pivoting (FP64),
 * solves and refines each sample, largest first.
 *   theta   dev [n_mu x Q] row major
 *   ns_nt   dev [n_mu x 2] (ns_p, nt_p) or NULL for the model's (ns, nt)
 *   uhat    dev [n_mu x ns*nt]: sample p writes its ns_p*nt_p coefficients,
 *           ordered i + ns_p*j, at uhat + p*ns*nt
 *   rel_res dev [n_mu] or NULL: ||rhs - Ahat^st uhat|| / ||rhs|| after refinement
 *   status  dev [n_mu] or NULL: ST_OK, ST_ERR_SINGULAR, ST_ERR_NONFINITE
 * Asynchronous; repeated calls reuse the model's workspace. */
st_status st_rom_solve(st_model* m, int32_t n_mu, const double* theta, const int32_t* ns_nt,
                       double* uhat, double* rel_res, int32_t* status);

/* st_rom_solve without any device allocation.  This entry point has no
 * counterpart in the paper; it exists for callers that cannot allocate device
 * memory during a solve -- services running under a fixed, pre-reserved memory
 * budget (an allocation there may stall or fail), programs whose device memory
 * belongs to an outside pool that forbids side allocations, and code issuing
 * the solve where allocation calls are not allowed.
 * Same arguments, results and status codes as st_rom_solve.  All scratch lives
 * in one fixed 32 MiB device array inside the library (every GPU that loads
 * the library holds it until the process exits); the caller still passes the
 * inputs and outputs, and the call makes no cudaMalloc/cudaFree or other
 * allocating call.  Limit: 4*(2*n_mu + ns*nt + 17) bytes (rounded up to 256)
 * plus one factor matrix of (ns*nt)^2 entries (8 bytes each in the ST_FP64
 * and ST_FP32_ASSEMBLY modes, 4 in ST_FP32_LU) must fit in 32 MiB, else
 * ST_ERR_ARG with a message; the batch runs on as many blocks as matrices
 * fit (at most the allocating path's count), so at large ns*nt fewer blocks
 * run (slower, same results).  The first call on a device looks up that
 * array's device address (once per device, with the model's device current)
 * and keeps it for the life of the process; make that first call before any
 * stream capture, and do not keep using the library across a
 * cudaDeviceReset of that device (the kept address would be stale).  Every call uses the same array and zeroes what
 * must start at zero: calls that overlap on the GPU (other streams, other
 * models on the same device) race and must be serialised by the caller. */
st_status st_rom_solve_static(st_model* m, int32_t n_mu, const double* theta,
                              const int32_t* ns_nt, double* uhat, double* rel_res,
                              int32_t* status);

/* Launch plan of the batched solve (st_rom_solve, st_rom_solve_static and the
 * surrogate's fallback), one per factor precision (ST_FP32_LU, or the FP64
 * factors of ST_FP64 / ST_FP32_ASSEMBLY).  No counterpart in the paper: these
 * are tile and scheduling choices of this library's kernel.
 *   panel        LU panel width: 4, 8, 16 or 32 (0 = the widest that fits
 *                shared memory, at most 32)
 *   ctas_per_sm  resident CTAs per SM, capped by occupancy (0 = the default:
 *                4 with FP32 factors, 2 with FP64 factors)
 *   order        queue order of the samples (ST_ORDER_*)
 * Plans with the same panel width give the same results bit for bit (a
 * sample is solved by one CTA in a fixed order whichever CTA takes it); the
 * panel width sets the blocking of the LU and so its rounding (results agree
 * to the solve's accuracy). */
typedef struct {
    int32_t panel;
    int32_t ctas_per_sm;
    int32_t order;
} st_solve_plan;
#define ST_ORDER_LARGEST_FIRST  0  /* largest ns_p * nt_p first (default)  */
#define ST_ORDER_SMALLEST_FIRST 1  /* smallest first                       */
#define ST_ORDER_INPUT          2  /* the samples' own order, no size sort  */

/* Install a plan for `precision`'s factor arithmetic; NULL restores the
 * defaults.  ST_ERR_ARG for invalid fields.  Host-only bookkeeping. */
st_status st_rom_solve_set_plan(st_model* m, int32_t precision, const st_solve_plan* plan);

/* The plan the solve would use now for `precision`, with the defaults and
 * limits resolved (panel width after shrinking to fit, CTAs per SM after the
 * occupancy cap).  Requires the reduced operators (ST_ERR_STATE otherwise). */
st_status st_rom_solve_get_plan(st_model* m, int32_t precision, st_solve_plan* plan);

/* Autotuner (synchronous): times st_rom_solve on the caller's batch (theta,
 * ns_nt, uhat as for st_rom_solve; uhat is overwritten) under the model's
 * current precision for every candidate plan -- the default plan first, then
 * each panel width in {8, 16, 32} that fits shared memory x each CTAs-per-SM
 * count from 1 to min(occupancy, 4) x each queue order -- one untimed run and
 * `reps` runs timed with CUDA events on the model's stream each (best kept),
 * then installs the fastest for that precision.  Optional outputs: the first
 * `cap` candidates and their best times in cands/ms, the number of
 * candidates in *n_cands, the best time in *best_ms, the default plan's time
 * in *default_ms; *best receives the installed plan (fields 0 where the
 * default is kept).  ST_ERR_STATE before assembly, ST_ERR_ARG for bad
 * arguments; a failing solve aborts the tuning and keeps the previous plan. */
st_status st_rom_solve_tune(st_model* m, int32_t n_mu, const double* theta, const int32_t* ns_nt,
                            double* uhat, int32_t reps, int32_t cap, st_solve_plan* cands, float* ms,
                            int32_t* n_cands, st_solve_plan* best, float* best_ms, float* default_ms);

/* Reconstruction u^st ~= Phi_st uhat (Eq. ststateapproximation) by blocks:
 *   C[i,k] = sum_j uhat[i + ns_p j] phi_t^{i,j}[k],  u^k = Phi_s C[:,k].
 *   uhat  dev [n_mu x ns*nt] as written by st_rom_solve; ns_nt as there
 *   u     dev [N x Nt x n_mu] or NULL: full fields, u^k(mu_p) in column
 *         p*Nt + (k-1)
 *   Cout  dev [N x n_out] or NULL; y dev [n_out x Nt x n_mu] or NULL: outputs
 *         y^k = Cout^T u^k (Eq. Dynamicaloutput) computed through
 *         Chat = Phi_s^T Cout without forming u (Eq. outputFromReducedsol).
 * Asynchronous. */
st_status st_rom_reconstruct(st_model* m, int32_t n_mu, const double* uhat,
                             const int32_t* ns_nt, double* u, int32_t n_out, const double* Cout,
                             double* y);

/* Batched spatial Galerkin ROM (Sec. 3.1, Eq. galerkin with reference state
 * 0), the model the space-time ROM is compared with, marched by backward
 * Euler (Eq. space_reduced_discretized_ODE) over the assembled steps:
 *   (I - dt_k Ahat(mu)) uhat^k = uhat^{k-1} + dt_k Bhat f^k,  k = 1..Nt,
 *   uhat^0 = Phi_s^T u0 (0 without u0),  Ahat(mu) = sum_q theta_q Ahat_q,
 * with Bhat = Phi_s^T B and f^k the rows of F given to st_rom_assemble.
 * Sample p uses the leading ns_p spatial modes.  The matrix of each run of
 * equal steps is inverted once, by Gauss-Jordan elimination with partial
 * pivoting in FP64; every step is then one matrix-vector product.
 *   theta  dev [n_mu x Q] row major
 *   ns_mu  dev [n_mu] (ns_p, 1 <= ns_p <= ns) or NULL for the model's ns
 *   uhat   dev [n_mu x Nt x ns]: sample p writes uhat^k_i (i < ns_p) at
 *          uhat[(p Nt + k - 1) ns + i]; entries i >= ns_p are left as they
 *          are; after a singular matrix the remaining steps are NaN
 *   status dev [n_mu] or NULL: ST_OK, ST_ERR_ARG (bad ns_p, nothing
 *          written), ST_ERR_SINGULAR (a zero or non-finite pivot column),
 *          ST_ERR_NONFINITE; any of these is also reported by st_sync
 * Requires st_rom_assemble (ST_ERR_STATE otherwise); ST_ERR_ARG when the
 * ns x ns matrix does not fit one block's shared memory (ns above ~160).
 * Samples run largest ns_p first.  Asynchronous and deterministic (a
 * sample's result does not depend on the batch); a workspace of
 * 4 (ns + 1 + 2 n_mu) bytes grows on demand. */
st_status st_rom_spatial_march(st_model* m, int32_t n_mu, const double* theta,
                               const int32_t* ns_mu, double* uhat, int32_t* status);

/* Full-order residual norms of approximate trajectories (Eq. residual):
 *   r^k = u^k - u^{k-1} - dt_k A(mu) u^k - dt_k B f^k,  k = 1..Nt,  u^0 = u0,
 * the factor of the a posteriori error bounds that a trajectory determines:
 *   ||u^k - u~^k|| <= sum_{i<=k} (prod_{j=i..k} xi_j) ||r^i||   (Theorem 1,
 *                     xi_j = ||(I - dt_j A)^-1||_2, u~^0 = u^0),
 *   max_k ||u^k - u~^k|| <= sqrt(Nt) ||(A^st)^-1||_2 max_k ||r^k||  (Theorem 3),
 * for a ROM trajectory u~ (the fields of st_rom_reconstruct, or Phi_s uhat^k
 * of st_rom_spatial_march) at the cost of one operator application per step.
 * Needs only the operator (no basis).
 *   theta host [n_mu x Q] row major; dt host [Nt], all > 0
 *   u0    dev [N] or NULL for 0
 *   B     dev [N x n_in] column major; F host [Nt x n_in] row major (n_in may be 0)
 *   U     dev [n_mu x Nt x N]: u^k(mu_p) at U + (p Nt + k - 1) N, the
 *         layout of st_fom_march's snapshots and st_rom_reconstruct's fields
 *   rnorm dev [n_mu x Nt]: ||r^k(mu_p)||_2 at rnorm[p Nt + k - 1]
 * Deterministic (fixed-order sums).  1 <= Nt <= 65535.  Asynchronous. */
st_status st_rom_residual_norms(st_model* m, int32_t n_mu, const double* theta, int32_t Nt,
                                const double* dt, const double* u0, int32_t n_in,
                                const double* B, const double* F, const double* U,
                                double* rnorm);

/* Stability constant of the space-time error bound (Theorem 3),
 *   ||u^st - u~^st||_2 <= ||(A^st)^{-1}||_2 ||r^st||_2,
 * for n_mu parameter samples (1..32): A^st is the block lower bidiagonal
 * matrix of the backward-Euler march (diagonal blocks I - dt_k A(mu), sub-
 * diagonal blocks -I; Eqs. st-fom, stsystemmat).  Estimated by power iteration
 * on (A^st)^{-T} (A^st)^{-1} from a seeded start vector: each iteration is one
 * full-order march with a per-step source (applying (A^st)^{-1}) and one march
 * of the transposed terms A_q^T over the reversed steps (applying
 * (A^st)^{-T}); the transposed terms are built on the first call from the
 * model's copy of the operator and kept.  The estimate sqrt(||w||) (w the
 * power iterate before normalisation) rises monotonically to the norm from
 * below; iteration stops once every sample's estimate changed by at most
 * tol (relative) in one iteration.  Synchronous.
 *   theta host [n_mu x Q]; dt host [Nt] (> 0); seed of the start vector
 *   norm  host [n_mu]: the estimates; iters_used host or NULL
 * A march that fails is reported with its status; ST_ERR_NOT_CONVERGED when
 * max_iter iterations did not reach tol (norm still holds the estimates).
 * Workspace: 3 n_mu Nt N doubles. */
st_status st_fom_st_inverse_norm(st_model* m, int32_t n_mu, const double* theta, int32_t Nt, const double* dt,
                                 int32_t max_iter, double tol, uint64_t seed, double* norm, int32_t* iters_used);

/* Learned surrogate mu -> uhat (no counterpart in the paper; it serves the
 * many-query use the paper motivates): a 3-layer MLP 2 -> 256 -> 256 -> ns*nt
 * with exact-erf GELU, FP32 master weights, BF16 copies on the tensor cores,
 * FP32 accumulation and outputs.  The input is mu mapped affinely from the box
 * [mu_lo, mu_hi] onto [-1, 1]^2; the targets are the FP64 reduced solutions
 * uhat normalised per component by their mean and standard deviation.
 * Training: Adam (0.9, 0.999, eps 1e-8, bias correction) with cosine decay of
 * lr over all steps; each epoch visits the samples in the order
 * i -> (a i + c) mod n, with a, c from SplitMix64 keyed by (seed, epoch), in
 * minibatches of `batch`.  Synchronous.
 *   mu     dev [n x 2] parameters, uhat dev [n x ns*nt] targets (full basis)
 *   mu_lo, mu_hi host [2] parameter box
 *   init   host [count] initial FP32 parameters (W1, b1, W2, b2, W3, b3, row
 *          major [out x in]) or NULL for Kaiming-uniform from seed
 *   epoch_loss host [epochs] or NULL: mean training loss of each epoch
 * Requires a basis; ns*nt must be a multiple of 8. */
st_status st_rom_surrogate_train(st_model* m, int32_t n, const double* mu, const double* mu_lo,
                                 const double* mu_hi, const double* uhat, const float* init,
                                 int32_t epochs, int32_t batch, float lr, uint64_t seed,
                                 float* epoch_loss);

/* Surrogate inference gated by the reduced space-time residual: every
 * prediction is accepted if ||Ahat^st(mu) uhat - rhs|| / ||rhs|| <= gate
 * (evaluated in FP32 from the affine pieces of Ahat^st, Eq. ij-block-matrix),
 * otherwise the sample is solved by the batched FP64 LU of st_rom_solve.
 * The residual's products run on the tensor cores when ns*nt is a multiple of
 * 4: both operands split into three BF16 parts (8 bits each), the six cross
 * products of order <= 4 summed in FP32 by one BF16 GEMM (FP32-accurate);
 * otherwise in FP32 on the SIMT cores.
 *   mu dev [n x 2], theta dev [n x Q] (same samples), uhat dev [n x ns*nt]
 *   rel_res dev [n]: gate residual, or the LU residual for fallback samples
 *   used_fallback dev [n]: 1 where the LU was used
 *   n_fallback host or NULL: number of fallback samples (synchronises). */
st_status st_rom_surrogate_infer(st_model* m, int32_t n, const double* mu, const double* theta,
                                 double gate, double* uhat, double* rel_res, int32_t* used_fallback,
                                 int32_t* n_fallback);

/* Reference preconditioner for the reduced space-time systems (no counterpart
 * in the paper): Ahat^st at n_ref reference parameters (e.g. the training
 * grid) is assembled and inverted in FP32 (Gauss-Jordan with partial
 * pivoting, one CTA per reference) and kept by the model.  Requires the
 * reduced operators; replaced by the next call.
 *   mu_ref host [n_ref x 2] (the parameters, for nearest-reference lookup),
 *   theta_ref host [n_ref x Q]; 1 <= n_ref <= 1024, ns*nt <= 4096.
 * Synchronous; ST_ERR_SINGULAR if a reference matrix has a zero pivot. */
st_status st_rom_precond_build(st_model* m, int32_t n_ref, const double* mu_ref, const double* theta_ref);

/* Reduced solves by preconditioned Richardson refinement, started from the
 * surrogate's prediction (ST_GUESS_SURROGATE) or from zero (ST_GUESS_ZERO):
 *   x <- x + P_g (fhat^st - Ahat^st(mu) x),  P_g = Ahat^st(mu_g)^{-1},
 * with mu_g the reference nearest to mu (coordinates scaled by the
 * references' spread).  Every step evaluates the residual of the whole batch
 * through the affine pieces of Ahat^st (FP32-accurate products -- on the
 * tensor cores as for the surrogate's gate -- combined in FP64) and stops as soon as every sample satisfies
 * ||rhs - Ahat^st x|| / ||rhs|| <= gate, or after max_iter corrections;
 * samples still above the gate are then solved by the batched LU of
 * st_rom_solve (their rel_res is the LU's).  Full (ns, nt) only.  The
 * residual's FP32 products limit the reachable gate to about 1e-6.
 *   mu dev [n x 2], theta dev [n x Q], uhat dev [n x ns*nt] (output),
 *   rel_res dev [n], used_fallback dev [n]; iters_run host or NULL:
 *   corrections applied; n_fallback host or NULL.
 * Requires st_rom_precond_build (ST_ERR_STATE otherwise) and, with
 * ST_GUESS_SURROGATE, a trained surrogate.  Synchronous. */
#define ST_GUESS_SURROGATE 0
#define ST_GUESS_ZERO      1
st_status st_rom_refine(st_model* m, int32_t n, const double* mu, const double* theta, int32_t guess, double gate,
                        int32_t max_iter, double* uhat, double* rel_res, int32_t* used_fallback,
                        int32_t* iters_run, int32_t* n_fallback);

/* Current FP32 surrogate parameters (host [count], layout as for init);
 * params may be NULL to query count.  Synchronous. */
st_status st_rom_surrogate_params(st_model* m, float* params, int64_t* count);

/* Loss and gradients of the surrogate loss at the given parameters on one
 * batch (targets normalised with the batch's own statistics), for checking the
 * backward kernels.  grad host [count] or NULL, loss host or NULL.
 * Synchronous; leaves the surrogate untrained. */
st_status st_rom_surrogate_loss_grad(st_model* m, int32_t n, const double* mu, const double* mu_lo,
                                     const double* mu_hi, const double* uhat, const float* params,
                                     float* grad, float* loss);

#ifdef __cplusplus
}
#endif

#endif /* ST_ROM_H */
