// Model lifecycle, options, errors, sliced-ELL conversion and accessors.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"

#include <atomic>

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

void st_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void st_set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

st_status st_fail(st_status code, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

st_status st_grow(st_model* m, DevBuf& buf, size_t bytes) {
    if (bytes <= buf.bytes) return ST_OK;
    if (buf.p) {
        ST_CUDA_TRY(cudaStreamSynchronize(m->stream));
        ST_CUDA_TRY(cudaFree(buf.p));
        buf.p = nullptr;
        buf.bytes = 0;
    }
    size_t want = bytes + bytes / 8 + 256;
    ST_CUDA_TRY(cudaMalloc(&buf.p, want));
    buf.bytes = want;
    return ST_OK;
}

st_status st_check_launch(const char* what) {
    st_count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return st_fail(ST_ERR_CUDA, "%s launch failed: %s", what, cudaGetErrorString(e));
    return ST_OK;
}

// ---------------------------------------------------------------------------
// Per-kernel timing
static cudaEvent_t prof_event(st_model* m) {
    cudaEvent_t e = nullptr;
    if (!m->prof.pool.empty()) {
        e = m->prof.pool.back();
        m->prof.pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        e = nullptr;
    }
    return e;
}

ProfScope::ProfScope(st_model* model, const char* kernel) : m(model), name(kernel) {
    if (!m || !m->prof.on) {
        m = nullptr;
        return;
    }
    a = prof_event(m);
    if (a) cudaEventRecord(a, m->stream);
}

ProfScope::~ProfScope() {
    if (!m || !a) return;
    cudaEvent_t b = prof_event(m);
    if (!b) {
        m->prof.pool.push_back(a);
        return;
    }
    cudaEventRecord(b, m->stream);
    m->prof.pending.push_back({name, a, b});
}

static size_t prof_slot(ProfState& p, const char* name) {
    size_t i = 0;
    while (i < p.names.size() && p.names[i] != name) ++i;
    if (i == p.names.size()) {
        p.names.emplace_back(name);
        p.ms.push_back(0.0);
        p.launches.push_back(0);
        p.flops.push_back(0.0);
    }
    return i;
}

void st_prof_flops(st_model* m, const char* name, double flops) {
    if (!m || !m->prof.on) return;
    m->prof.flops[prof_slot(m->prof, name)] += flops;
}

static void prof_collect(st_model* m) {
    ProfState& p = m->prof;
    for (const ProfState::Rec& r : p.pending) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            const size_t i = prof_slot(p, r.name);
            p.ms[i] += ms;
            p.launches[i] += 1;
        }
        p.pool.push_back(r.a);
        p.pool.push_back(r.b);
    }
    p.pending.clear();
}

extern "C" {

void st_options_default(st_options* o) {
    if (!o) return;
    o->tol = 1e-13;
    o->maxit = 1000;
    o->eps_svd = 1e-12;
    o->eps_sv = 1e-14;
    o->r_max = 256;
    o->precision = ST_FP64;
    o->spin_limit = 20000000LL;
    o->refine_steps = 1;
    o->jacobi_sweeps = 40;
    o->pod_block = 1;
    o->fp64_gemm = ST_DGEMM_OZAKI;
    o->pod_cols = 0;
    o->fom_path = ST_FOM_AUTO;
}

const char* st_last_error(void) { return g_last_error.c_str(); }

int64_t st_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

const char* st_status_string(st_status s) {
    switch (s) {
        case ST_OK: return "ST_OK";
        case ST_ERR_ARG: return "ST_ERR_ARG";
        case ST_ERR_CUDA: return "ST_ERR_CUDA";
        case ST_ERR_OOM: return "ST_ERR_OOM";
        case ST_ERR_NOT_CONVERGED: return "ST_ERR_NOT_CONVERGED";
        case ST_ERR_BREAKDOWN: return "ST_ERR_BREAKDOWN";
        case ST_ERR_SINGULAR: return "ST_ERR_SINGULAR";
        case ST_ERR_NONFINITE: return "ST_ERR_NONFINITE";
        case ST_ERR_TIMEOUT: return "ST_ERR_TIMEOUT";
        case ST_ERR_STATE: return "ST_ERR_STATE";
        default: return "ST_ERR_UNKNOWN";
    }
}

static bool options_valid(const st_options& o) {
    return (o.tol > 0) && o.maxit >= 1 && o.r_max >= 1 && (o.eps_svd >= 0) && (o.eps_sv >= 0) &&
           o.spin_limit >= 1 && o.refine_steps >= 0 && o.refine_steps <= 16 && o.jacobi_sweeps >= 1 &&
           o.pod_block >= 1 && o.pod_block <= 64 && o.pod_cols >= 0 &&
           (o.fp64_gemm == ST_DGEMM_SIMT || o.fp64_gemm == ST_DGEMM_OZAKI) &&
           (o.fom_path == ST_FOM_AUTO || o.fom_path == ST_FOM_GRID || o.fom_path == ST_FOM_CLUSTER) &&
           (o.precision == ST_FP64 || o.precision == ST_FP32_ASSEMBLY || o.precision == ST_FP32_LU);
}

st_status st_model_set_options(st_model* m, const st_options* opt) {
    if (!m || !opt) return st_fail(ST_ERR_ARG, "st_model_set_options: NULL argument");
    if (!options_valid(*opt)) return st_fail(ST_ERR_ARG, "st_model_set_options: invalid st_options");
    m->opt = *opt;
    return ST_OK;
}

st_status st_model_get_options(st_model* m, st_options* opt) {
    if (!m || !opt) return st_fail(ST_ERR_ARG, "st_model_get_options: NULL argument");
    *opt = m->opt;
    return ST_OK;
}

static void free_basis(st_model* m) {
    cudaFree(m->d_phi);
    cudaFree(m->d_T);
    m->d_phi = m->d_T = nullptr;
    m->ns = m->nt = m->Nt = 0;
}

static void free_reduced(st_model* m) {
    cudaFree(m->d_Ahat);
    cudaFree(m->d_G);
    cudaFree(m->d_G32);
    cudaFree(m->d_M);
    cudaFree(m->d_S);
    cudaFree(m->d_rhs);
    cudaFree(m->d_dt);
    cudaFree(m->d_bs);
    cudaFree(m->d_u0s);
    m->d_Ahat = m->d_G = m->d_M = m->d_S = m->d_rhs = m->d_dt = nullptr;
    m->d_bs = m->d_u0s = nullptr;
    m->d_G32 = nullptr;
    m->assembled = false;
}

st_status st_profile_enable(st_model* m, int32_t on) {
    if (!m) return st_fail(ST_ERR_ARG, "st_profile_enable: NULL model");
    ST_CUDA_TRY(cudaStreamSynchronize(m->stream));
    prof_collect(m);
    m->prof.names.clear();
    m->prof.ms.clear();
    m->prof.launches.clear();
    m->prof.flops.clear();
    m->prof.on = on != 0;
    return ST_OK;
}

st_status st_profile_read(st_model* m, int32_t cap, char* names, double* ms, int64_t* launches,
                          double* flops, int32_t* n_kernels) {
    if (!m || !n_kernels || cap < 0) return st_fail(ST_ERR_ARG, "st_profile_read: bad arguments");
    ST_CUDA_TRY(cudaStreamSynchronize(m->stream));
    prof_collect(m);
    const ProfState& p = m->prof;
    std::vector<int> order(p.names.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return p.ms[x] > p.ms[y]; });
    *n_kernels = (int32_t)order.size();
    for (int i = 0; i < (int)order.size() && i < cap; ++i) {
        const int k = order[i];
        if (names) {
            std::strncpy(names + (size_t)i * ST_PROFILE_NAME_LEN, p.names[k].c_str(), ST_PROFILE_NAME_LEN - 1);
            names[(size_t)i * ST_PROFILE_NAME_LEN + ST_PROFILE_NAME_LEN - 1] = '\0';
        }
        if (ms) ms[i] = p.ms[k];
        if (launches) launches[i] = p.launches[k];
        if (flops) flops[i] = p.flops[k];
    }
    return ST_OK;
}

void st_model_destroy(st_model* m) {
    if (!m) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(m->device);
    cudaStreamSynchronize(m->stream);
    for (const ProfState::Rec& r : m->prof.pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : m->prof.pool) cudaEventDestroy(e);
    free_basis(m);
    free_reduced(m);
    cudaFree(m->d_slice_ptr);
    cudaFree(m->d_slice_w);
    cudaFree(m->d_col);
    cudaFree(m->d_vals);
    cudaFree(m->d_mx_ptr);
    cudaFree(m->d_mx_w);
    cudaFree(m->d_mx_col);
    cudaFree(m->d_mx_src);
    cudaFree(m->d_tq_ptr);
    cudaFree(m->d_tq_w);
    cudaFree(m->d_tq_col);
    cudaFree(m->d_tq_val);
    cudaFree(m->d_err);
    cudaFree(m->d_bar);
    if (m->adj) st_model_destroy(m->adj);
    for (DevBuf* b : {&m->W, &m->V, &m->ws_fom, &m->ws_pod, &m->ws_pod2, &m->ws_gemm, &m->ws_oz,
                      &m->ws_solve, &m->ws_misc, &m->ws_srom, &m->ws_cert, &m->prec.inv, &m->prec.work, &m->mlp.params, &m->mlp.grad, &m->mlp.adam_m,
                      &m->mlp.adam_v, &m->mlp.wbf, &m->mlp.stats, &m->mlp.act, &m->mlp.kall,
                      &m->mlp.list, &m->mlp.kall16, &m->mlp.xsplit})
        cudaFree(b->p);
    for (OzSlot& sl : m->oz_slot) {
        cudaFree(sl.planes.p);
        cudaFree(sl.exps.p);
    }
    cudaSetDevice(cur);
    delete m;
}

st_status st_model_create(const st_affine_csr* A, const st_options* opt, void* stream,
                          st_model** out) {
    if (!A || !out) return st_fail(ST_ERR_ARG, "st_model_create: NULL argument");
    *out = nullptr;
    const int64_t N = A->n_rows;
    if (N <= 0 || N > (int64_t)INT32_MAX) return st_fail(ST_ERR_ARG, "n_rows out of range");
    if (A->n_terms < 1 || A->n_terms > 16) return st_fail(ST_ERR_ARG, "n_terms must be in [1,16]");
    if (!A->rowptr || !A->col || !A->vals) return st_fail(ST_ERR_ARG, "NULL CSR array");
    if (A->rowptr[0] != 0) return st_fail(ST_ERR_ARG, "rowptr[0] must be 0");
    for (int q = 0; q < A->n_terms; ++q)
        if (!A->vals[q]) return st_fail(ST_ERR_ARG, "NULL value array for term %d", q);
    const int64_t nnz = A->rowptr[N];
    int max_w = 0;
    for (int64_t r = 0; r < N; ++r) {
        int64_t len = A->rowptr[r + 1] - A->rowptr[r];
        if (len < 0) return st_fail(ST_ERR_ARG, "rowptr decreases at row %lld", (long long)r);
        if (len > 4096) return st_fail(ST_ERR_ARG, "row %lld has more than 4096 entries", (long long)r);
        max_w = std::max(max_w, (int)len);
    }
    for (int64_t e = 0; e < nnz; ++e)
        if (A->col[e] < 0 || A->col[e] >= N)
            return st_fail(ST_ERR_ARG, "column index out of range at entry %lld", (long long)e);
    st_options o;
    st_options_default(&o);
    if (opt) o = *opt;
    if (!options_valid(o)) return st_fail(ST_ERR_ARG, "invalid st_options");

    st_model* m = new st_model();
    m->opt = o;
    try {
        m->h_rowptr.assign(A->rowptr, A->rowptr + N + 1);
        m->h_col.assign(A->col, A->col + nnz);
        m->h_vals.resize((size_t)A->n_terms * nnz);
    } catch (...) {
        delete m;
        return st_fail(ST_ERR_OOM, "st_model_create: no host memory for the operator copy");
    }
    for (int q = 0; q < A->n_terms; ++q)
        std::copy(A->vals[q], A->vals[q] + nnz, m->h_vals.begin() + (size_t)q * nnz);
    m->stream = (cudaStream_t)stream;
    m->N = N;
    m->nnz = nnz;
    m->Q = A->n_terms;
    if (cudaGetDevice(&m->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device) != cudaSuccess) {
        delete m;
        return st_fail(ST_ERR_CUDA, "no CUDA device available");
    }
    // sliced-ELL: slices of kSlice consecutive rows; entry (k, lane) of
    // slice s at slice_ptr[s] + k * kSlice + lane; padding has value 0 and
    // points at the row itself.
    const int64_t ns_ = (N + kSlice - 1) / kSlice;
    std::vector<int64_t> sptr(ns_ + 1, 0);
    std::vector<int32_t> sw(ns_, 0);
    for (int64_t s = 0; s < ns_; ++s) {
        int w = 0;
        for (int64_t r = s * kSlice; r < std::min<int64_t>(N, (s + 1) * kSlice); ++r)
            w = std::max<int>(w, (int)(A->rowptr[r + 1] - A->rowptr[r]));
        sw[s] = w;
        sptr[s + 1] = sptr[s] + (int64_t)w * kSlice;
    }
    const int64_t ell = sptr[ns_];
    std::vector<int32_t> col(ell);
    std::vector<double> vals((size_t)m->Q * ell, 0.0);
    for (int64_t s = 0; s < ns_; ++s) {
        for (int lane = 0; lane < kSlice; ++lane) {
            int64_t r = s * kSlice + lane;
            int64_t b = r < N ? A->rowptr[r] : 0, len = r < N ? A->rowptr[r + 1] - b : 0;
            for (int k = 0; k < sw[s]; ++k) {
                int64_t e = sptr[s] + (int64_t)k * kSlice + lane;
                if (k < len) {
                    col[e] = A->col[b + k];
                    for (int q = 0; q < m->Q; ++q) vals[(size_t)q * ell + e] = A->vals[q][b + k];
                } else {
                    col[e] = r < N ? (int32_t)r : 0;
                }
            }
        }
    }
    m->n_slices = ns_;
    m->ell_size = ell;
    m->max_width = max_w;
    // term split: group g = 0 mixed entries, g = 1 + q entries of term q only
    // (entries with no nonzero term are dropped)
    const int Qn = m->Q;
    auto group_of = [&](int64_t csr_e) -> int {
        int cnt = 0, last = 0;
        for (int q = 0; q < Qn; ++q)
            if (A->vals[q][csr_e] != 0.0) {
                ++cnt;
                last = q;
            }
        return cnt == 0 ? -1 : (cnt == 1 ? 1 + last : 0);
    };
    std::vector<int32_t> gw((size_t)ns_ * (Qn + 1), 0);
    for (int64_t s = 0; s < ns_; ++s)
        for (int64_t r = s * kSlice; r < std::min<int64_t>(N, (s + 1) * kSlice); ++r) {
            std::vector<int> cnt(Qn + 1, 0);
            for (int64_t e = A->rowptr[r]; e < A->rowptr[r + 1]; ++e) {
                const int g = group_of(e);
                if (g >= 0) ++cnt[g];
            }
            for (int g = 0; g <= Qn; ++g)
                gw[(size_t)s * (Qn + 1) + g] = std::max(gw[(size_t)s * (Qn + 1) + g], cnt[g]);
        }
    std::vector<int64_t> mx_ptr(ns_ + 1, 0), tq_ptr((size_t)ns_ * Qn + 1, 0);
    std::vector<int32_t> mx_w(ns_), tq_w((size_t)ns_ * Qn);
    for (int64_t s = 0; s < ns_; ++s) {
        mx_w[s] = gw[(size_t)s * (Qn + 1)];
        mx_ptr[s + 1] = mx_ptr[s] + (int64_t)mx_w[s] * kSlice;
        for (int q = 0; q < Qn; ++q) {
            const size_t i = (size_t)s * Qn + q;
            tq_w[i] = gw[(size_t)s * (Qn + 1) + 1 + q];
            tq_ptr[i + 1] = tq_ptr[i] + (int64_t)tq_w[i] * kSlice;
        }
    }
    const int64_t mx_n = mx_ptr[ns_], tq_n = tq_ptr[(size_t)ns_ * Qn];
    std::vector<int32_t> mx_col(mx_n), tq_col(tq_n);
    std::vector<int64_t> mx_src(mx_n, -1);
    std::vector<double> tq_val(tq_n, 0.0);
    for (int64_t s = 0; s < ns_; ++s)
        for (int lane = 0; lane < kSlice; ++lane) {
            const int64_t r = s * kSlice + lane;
            const int32_t self = r < N ? (int32_t)r : 0;
            std::vector<int> fill(Qn + 1, 0);
            if (r < N)
                for (int64_t k = 0; k < A->rowptr[r + 1] - A->rowptr[r]; ++k) {
                    const int64_t ce = A->rowptr[r] + k;
                    const int g = group_of(ce);
                    if (g < 0) continue;
                    const int slot = fill[g]++;
                    if (g == 0) {
                        const int64_t e = mx_ptr[s] + (int64_t)slot * kSlice + lane;
                        mx_col[e] = A->col[ce];
                        mx_src[e] = sptr[s] + k * kSlice + lane;  // same entry in the sliced-ELL
                    } else {
                        const int64_t e = tq_ptr[(size_t)s * Qn + g - 1] + (int64_t)slot * kSlice + lane;
                        tq_col[e] = A->col[ce];
                        tq_val[e] = A->vals[g - 1][ce];
                    }
                }
            for (int g = 0; g <= Qn; ++g) {
                const int w = g == 0 ? mx_w[s] : tq_w[(size_t)s * Qn + g - 1];
                for (int slot = fill[g]; slot < w; ++slot) {
                    if (g == 0) mx_col[mx_ptr[s] + (int64_t)slot * kSlice + lane] = self;
                    else tq_col[tq_ptr[(size_t)s * Qn + g - 1] + (int64_t)slot * kSlice + lane] = self;
                }
            }
        }
    m->mx_size = mx_n;
    m->tq_size = tq_n;
    auto fail = [&](cudaError_t e) {
        st_model_destroy(m);
        return st_fail(e == cudaErrorMemoryAllocation ? ST_ERR_OOM : ST_ERR_CUDA,
                       "st_model_create: %s", cudaGetErrorString(e));
    };
    cudaError_t e;
    if ((e = cudaMalloc(&m->d_slice_ptr, sizeof(int64_t) * (ns_ + 1))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&m->d_slice_w, sizeof(int32_t) * ns_)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&m->d_col, sizeof(int32_t) * std::max<int64_t>(ell, 1))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&m->d_vals, sizeof(double) * m->Q * std::max<int64_t>(ell, 1))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&m->d_err, sizeof(int32_t))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&m->d_bar, sizeof(unsigned int) * 4)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(m->d_slice_ptr, sptr.data(), sizeof(int64_t) * (ns_ + 1), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(m->d_slice_w, sw.data(), sizeof(int32_t) * ns_, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
    if (ell > 0) {
        if ((e = cudaMemcpy(m->d_col, col.data(), sizeof(int32_t) * ell, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
        if ((e = cudaMemcpy(m->d_vals, vals.data(), sizeof(double) * m->Q * ell, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
    }
    {
        auto up = [&](void** dst, const void* src, size_t bytes) -> cudaError_t {
            cudaError_t ee = cudaMalloc(dst, std::max<size_t>(bytes, 16));
            if (ee != cudaSuccess || bytes == 0) return ee;
            return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
        };
        if ((e = up((void**)&m->d_mx_ptr, mx_ptr.data(), sizeof(int64_t) * mx_ptr.size())) != cudaSuccess) return fail(e);
        if ((e = up((void**)&m->d_mx_w, mx_w.data(), sizeof(int32_t) * mx_w.size())) != cudaSuccess) return fail(e);
        if ((e = up((void**)&m->d_mx_col, mx_col.data(), sizeof(int32_t) * mx_col.size())) != cudaSuccess) return fail(e);
        if ((e = up((void**)&m->d_mx_src, mx_src.data(), sizeof(int64_t) * mx_src.size())) != cudaSuccess) return fail(e);
        if ((e = up((void**)&m->d_tq_ptr, tq_ptr.data(), sizeof(int64_t) * tq_ptr.size())) != cudaSuccess) return fail(e);
        if ((e = up((void**)&m->d_tq_w, tq_w.data(), sizeof(int32_t) * tq_w.size())) != cudaSuccess) return fail(e);
        if ((e = up((void**)&m->d_tq_col, tq_col.data(), sizeof(int32_t) * tq_col.size())) != cudaSuccess) return fail(e);
        if ((e = up((void**)&m->d_tq_val, tq_val.data(), sizeof(double) * tq_val.size())) != cudaSuccess) return fail(e);
    }
    if ((e = cudaMemset(m->d_err, 0, sizeof(int32_t))) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(m->d_bar, 0, sizeof(unsigned int) * 4)) != cudaSuccess) return fail(e);
    *out = m;
    return ST_OK;
}

st_status st_sync(st_model* m) {
    if (!m) return st_fail(ST_ERR_ARG, "st_sync: NULL model");
    ST_CUDA_TRY(cudaStreamSynchronize(m->stream));
    int32_t h = 0;
    ST_CUDA_TRY(cudaMemcpy(&h, m->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (h != 0) {
        ST_CUDA_TRY(cudaMemset(m->d_err, 0, sizeof(int32_t)));
        return st_fail(h, "device reported %s", st_status_string(h));
    }
    return ST_OK;
}

st_status st_model_set_basis(st_model* m, int32_t ns, int32_t nt, int32_t Nt, const double* phi_s,
                             const double* T) {
    if (!m || !phi_s || !T) return st_fail(ST_ERR_ARG, "st_model_set_basis: NULL argument");
    if (ns < 1 || nt < 1 || Nt < 1 || ns > m->N || nt > Nt)
        return st_fail(ST_ERR_ARG, "st_model_set_basis: bad sizes");
    free_reduced(m);
    free_basis(m);
    ST_CUDA_TRY(cudaMalloc(&m->d_phi, sizeof(double) * m->N * ns));
    ST_CUDA_TRY(cudaMalloc(&m->d_T, sizeof(double) * (size_t)Nt * ns * nt));
    ST_CUDA_TRY(cudaMemcpyAsync(m->d_phi, phi_s, sizeof(double) * m->N * ns,
                                cudaMemcpyDeviceToDevice, m->stream));
    ST_CUDA_TRY(cudaMemcpyAsync(m->d_T, T, sizeof(double) * (size_t)Nt * ns * nt,
                                cudaMemcpyDeviceToDevice, m->stream));
    m->ns = ns;
    m->nt = nt;
    m->Nt = Nt;
    return ST_OK;
}

st_status st_model_get_basis(st_model* m, double* phi_s, double* T, int32_t* dims) {
    if (!m) return st_fail(ST_ERR_ARG, "st_model_get_basis: NULL model");
    if (!m->d_phi) return st_fail(ST_ERR_STATE, "st_model_get_basis: no basis");
    if (dims) {
        dims[0] = m->ns;
        dims[1] = m->nt;
        dims[2] = m->Nt;
    }
    if (phi_s)
        ST_CUDA_TRY(cudaMemcpyAsync(phi_s, m->d_phi, sizeof(double) * m->N * m->ns,
                                    cudaMemcpyDeviceToDevice, m->stream));
    if (T)
        ST_CUDA_TRY(cudaMemcpyAsync(T, m->d_T, sizeof(double) * (size_t)m->Nt * m->ns * m->nt,
                                    cudaMemcpyDeviceToDevice, m->stream));
    return ST_OK;
}

st_status st_pod_get_state(st_model* m, double* W, double* V, double* sigma, int32_t* r) {
    if (!m) return st_fail(ST_ERR_ARG, "st_pod_get_state: NULL model");
    if (r) *r = m->pod_r;
    if (m->pod_r == 0) return ST_OK;
    if (W)
        ST_CUDA_TRY(cudaMemcpyAsync(W, m->W.p, sizeof(double) * m->N * m->pod_r,
                                    cudaMemcpyDeviceToDevice, m->stream));
    if (V && m->pod_rows > 0)
        ST_CUDA_TRY(cudaMemcpy2DAsync(V, sizeof(double) * m->pod_rows, m->V.p, sizeof(double) * m->pod_ldv,
                                      sizeof(double) * m->pod_rows, m->pod_r, cudaMemcpyDeviceToDevice,
                                      m->stream));
    if (sigma) std::memcpy(sigma, m->sigma.data(), sizeof(double) * m->pod_r);
    ST_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return ST_OK;
}

st_status st_pod_get_dims(st_model* m, int32_t* r, int64_t* rows) {
    if (!m) return st_fail(ST_ERR_ARG, "st_pod_get_dims: NULL model");
    if (r) *r = m->pod_r;
    if (rows) *rows = m->pod_rows;
    return ST_OK;
}

st_status st_pod_get_stats(st_model* m, int32_t* n_updates, int32_t* sweeps, int32_t cap,
                           int32_t* n_reorth) {
    if (!m || !n_updates || cap < 0) return st_fail(ST_ERR_ARG, "st_pod_get_stats: bad arguments");
    *n_updates = (int32_t)m->pod_sweeps.size();
    if (sweeps)
        for (int i = 0; i < (int)m->pod_sweeps.size() && i < cap; ++i) sweeps[i] = m->pod_sweeps[i];
    if (n_reorth) *n_reorth = m->pod_reorth;
    return ST_OK;
}

st_status st_model_get_reduced(st_model* m, double* Ahat, double* G, double* M, double* S,
                               double* rhs) {
    if (!m) return st_fail(ST_ERR_ARG, "st_model_get_reduced: NULL model");
    if (!m->assembled) return st_fail(ST_ERR_STATE, "st_model_get_reduced: not assembled");
    const size_t ns = m->ns, nt = m->nt, n = ns * nt;
    ST_CUDA_TRY(cudaStreamSynchronize(m->stream));
    if (Ahat) ST_CUDA_TRY(cudaMemcpy(Ahat, m->d_Ahat, sizeof(double) * m->Q * ns * ns, cudaMemcpyDeviceToHost));
    if (G) ST_CUDA_TRY(cudaMemcpy(G, m->d_G, sizeof(double) * n * n, cudaMemcpyDeviceToHost));
    if (M) ST_CUDA_TRY(cudaMemcpy(M, m->d_M, sizeof(double) * ns * nt * nt, cudaMemcpyDeviceToHost));
    if (S) ST_CUDA_TRY(cudaMemcpy(S, m->d_S, sizeof(double) * ns * nt * nt, cudaMemcpyDeviceToHost));
    if (rhs) ST_CUDA_TRY(cudaMemcpy(rhs, m->d_rhs, sizeof(double) * n, cudaMemcpyDeviceToHost));
    return ST_OK;
}

}  // extern "C"

// Used by st_rom_build_basis to replace the basis it produced.
void st_internal_free_basis(st_model* m) {
    free_reduced(m);
    free_basis(m);
}
void st_internal_free_reduced(st_model* m) { free_reduced(m); }
