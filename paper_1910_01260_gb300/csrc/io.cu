// Model persistence: st_model_save, st_model_load, st_model_file_info.
//
// The paper's method splits into an offline stage (snapshots, bases, reduced
// operators; Secs. 4.2-4.3) and an online stage that only needs the reduced
// operators.  A saved model carries everything a later process needs to
// continue either stage: the affine operator, the options, the state of the
// incremental SVD (so a basis build can resume with more snapshots), the
// bases, the reduced operators and a trained surrogate.
//
// File layout (little endian):
//   magic "STROMMDL" (8 bytes), u32 version (1), u32 section count, then per
//   section: char tag[4], u32 zero, u64 payload bytes, payload, u64 FNV-1a
//   (64-bit) of the payload.  Sections, in this order, the first two always:
//   "OPTS" f64 tol, i32 maxit, f64 eps_svd, f64 eps_sv, i32 r_max,
//          i32 precision, i64 spin_limit, i32 refine_steps, i32 jacobi_sweeps,
//          i32 pod_block, i32 fp64_gemm, i32 pod_cols, i32 fom_path
//          (packed, 68 bytes)
//   "OPER" i64 N, i64 nnz, i32 Q, i32 0, i64 rowptr[N+1], i32 col[nnz]
//          (padded to 8 bytes), f64 vals[Q][nnz]
//   "PODS" i32 r, i32 n_updates, i64 rows, i32 n_reorth, i32 0, f64 sigma[r],
//          i32 sweeps[n_updates] (padded to 8 bytes), f64 W[r][N],
//          f64 V[r][rows]   (column major, i.e. column by column)
//   "BASE" i32 ns, i32 nt, i32 Nt, i32 0, f64 phi_s[ns][N], f64 T[ns*nt][Nt]
//   "REDU" i32 ns, i32 nt, i32 Nt, i32 Q, f64 Ahat[Q][ns][ns], G[n][n],
//          M[ns][nt][nt], S[ns][nt][nt], rhs[n], dt[Nt], bs[Nt][ns], u0s[ns]
//          (n = ns*nt, every matrix column major)
//   "SURR" i32 n_in, i32 hidden, i32 n_out, i32 trained, i64 n_params,
//          i64 adam_steps, f64 lo[2], f64 hi[2], f32 params[n_params],
//          f32 adam_m[n_params], f32 adam_v[n_params] (padded to 8 bytes),
//          f64 mean[n_out], f64 std[n_out]
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "internal.h"

namespace {

constexpr char kMagic[8] = {'S', 'T', 'R', 'O', 'M', 'M', 'D', 'L'};
constexpr uint32_t kVersion = 1;

uint64_t fnv1a(const uint8_t* p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

struct Out {
    std::vector<uint8_t> b;
    void raw(const void* p, size_t n) {
        const uint8_t* c = static_cast<const uint8_t*>(p);
        b.insert(b.end(), c, c + n);
    }
    template <typename T>
    void put(T v) {
        raw(&v, sizeof(T));
    }
    void pad8() {
        while (b.size() % 8) b.push_back(0);
    }
};

// Bounds-checked cursor over one section's payload.
struct In {
    const uint8_t* p;
    size_t n, at = 0;
    bool ok = true;
    bool raw(void* dst, size_t bytes) {
        if (!ok || bytes > n - at) {
            ok = false;
            return false;
        }
        if (bytes) std::memcpy(dst, p + at, bytes);
        at += bytes;
        return true;
    }
    template <typename T>
    T get() {
        T v{};
        raw(&v, sizeof(T));
        return v;
    }
    void pad8() {
        const size_t to = (at + 7) / 8 * 8;
        if (to > n) ok = false;
        else at = to;
    }
    // byte count of `count` elements of `size`, or fail if it cannot fit
    bool fits(uint64_t count, size_t size) {
        if (!ok || (size && count > (n - at) / size)) ok = false;
        return ok;
    }
};

struct Section {
    char tag[4];
    std::vector<uint8_t> data;
};

// Everything a file holds, on the host.
struct Image {
    st_options opt{};
    int64_t N = 0, nnz = 0;
    int32_t Q = 0;
    std::vector<int64_t> rowptr;
    std::vector<int32_t> col;
    std::vector<double> vals;  // Q x nnz
    bool has_pod = false;
    int32_t r = 0, n_reorth = 0;
    int64_t rows = 0;
    std::vector<double> sigma, W, V;
    std::vector<int32_t> sweeps;
    bool has_basis = false;
    int32_t ns = 0, nt = 0, Nt = 0;
    std::vector<double> phi, T;
    bool has_reduced = false;
    std::vector<double> Ahat, G, M, S, rhs, dt, bs, u0s;
    bool has_surrogate = false;
    int32_t n_in = 0, hidden = 0, n_out = 0, trained = 0;
    int64_t n_params = 0, adam_t = 0;
    double lo[2] = {0, 0}, hi[2] = {0, 0};
    std::vector<float> params, adam_m, adam_v;
    std::vector<double> mean, stdv;
};

template <typename T>
bool get_vec(In& in, std::vector<T>& v, uint64_t count) {
    if (!in.fits(count, sizeof(T))) return false;
    v.resize(count);
    return in.raw(v.data(), sizeof(T) * count);
}

st_status read_file(const char* path, std::vector<Section>& secs) {
    std::unique_ptr<FILE, int (*)(FILE*)> f(std::fopen(path, "rb"), &std::fclose);
    if (!f) return st_fail(ST_ERR_ARG, "cannot open %s for reading", path);
    char magic[8];
    uint32_t ver = 0, count = 0;
    if (std::fread(magic, 1, 8, f.get()) != 8 || std::memcmp(magic, kMagic, 8) != 0)
        return st_fail(ST_ERR_ARG, "%s is not a saved st_rom model (bad magic)", path);
    if (std::fread(&ver, 4, 1, f.get()) != 1 || std::fread(&count, 4, 1, f.get()) != 1)
        return st_fail(ST_ERR_ARG, "%s: truncated header", path);
    if (ver != kVersion) return st_fail(ST_ERR_ARG, "%s: unsupported version %u", path, ver);
    if (count < 2 || count > 16) return st_fail(ST_ERR_ARG, "%s: bad section count %u", path, count);
    for (uint32_t s = 0; s < count; ++s) {
        Section sec;
        uint32_t zero = 0;
        uint64_t len = 0, sum = 0;
        if (std::fread(sec.tag, 1, 4, f.get()) != 4 || std::fread(&zero, 4, 1, f.get()) != 1 ||
            std::fread(&len, 8, 1, f.get()) != 1)
            return st_fail(ST_ERR_ARG, "%s: truncated section header %u", path, s);
        if (zero != 0 || len > (uint64_t)1 << 40) return st_fail(ST_ERR_ARG, "%s: corrupt section header %u", path, s);
        try {
            sec.data.resize(len);
        } catch (...) {
            return st_fail(ST_ERR_OOM, "%s: no host memory for a section of %llu bytes", path,
                           (unsigned long long)len);
        }
        if ((len && std::fread(sec.data.data(), 1, len, f.get()) != len) || std::fread(&sum, 8, 1, f.get()) != 1)
            return st_fail(ST_ERR_ARG, "%s: truncated section %.4s", path, sec.tag);
        if (sum != fnv1a(sec.data.data(), len))
            return st_fail(ST_ERR_ARG, "%s: checksum mismatch in section %.4s", path, sec.tag);
        secs.push_back(std::move(sec));
    }
    if (std::fgetc(f.get()) != EOF) return st_fail(ST_ERR_ARG, "%s: trailing bytes after the last section", path);
    return ST_OK;
}

bool tag_is(const Section& s, const char* t) { return std::memcmp(s.tag, t, 4) == 0; }

// Parse the sections into an Image.  With `headers_only` the large arrays
// are skipped (their sizes are still checked against the payload).
st_status parse(const std::vector<Section>& secs, Image& im, bool headers_only) {
    auto bad = [](const char* t) { return st_fail(ST_ERR_ARG, "saved model: malformed section %s", t); };
    if (!tag_is(secs[0], "OPTS") || !tag_is(secs[1], "OPER"))
        return st_fail(ST_ERR_ARG, "saved model: the first sections must be OPTS and OPER");
    {
        In in{secs[0].data.data(), secs[0].data.size()};
        st_options& o = im.opt;
        o.tol = in.get<double>();
        o.maxit = in.get<int32_t>();
        o.eps_svd = in.get<double>();
        o.eps_sv = in.get<double>();
        o.r_max = in.get<int32_t>();
        o.precision = in.get<int32_t>();
        o.spin_limit = in.get<int64_t>();
        o.refine_steps = in.get<int32_t>();
        o.jacobi_sweeps = in.get<int32_t>();
        o.pod_block = in.get<int32_t>();
        o.fp64_gemm = in.get<int32_t>();
        o.pod_cols = in.get<int32_t>();
        o.fom_path = in.get<int32_t>();
        if (!in.ok || in.at != in.n) return bad("OPTS");
    }
    auto skip = [&](In& in, uint64_t count, size_t size) {
        if (!in.fits(count, size)) return false;
        in.at += count * size;
        return true;
    };
    {
        In in{secs[1].data.data(), secs[1].data.size()};
        im.N = in.get<int64_t>();
        im.nnz = in.get<int64_t>();
        im.Q = in.get<int32_t>();
        in.get<int32_t>();
        if (!in.ok || im.N < 1 || im.nnz < 0 || im.Q < 1 || im.Q > 16) return bad("OPER");
        if (headers_only) {
            if (!skip(in, im.N + 1, 8) || !skip(in, im.nnz, 4)) return bad("OPER");
            in.pad8();
            if (!skip(in, (uint64_t)im.Q * im.nnz, 8)) return bad("OPER");
        } else {
            if (!get_vec(in, im.rowptr, im.N + 1) || !get_vec(in, im.col, im.nnz)) return bad("OPER");
            in.pad8();
            if (!get_vec(in, im.vals, (uint64_t)im.Q * im.nnz)) return bad("OPER");
            if (im.rowptr[0] != 0 || im.rowptr[im.N] != im.nnz) return bad("OPER");
        }
        if (!in.ok || in.at != in.n) return bad("OPER");
    }
    for (size_t s = 2; s < secs.size(); ++s) {
        In in{secs[s].data.data(), secs[s].data.size()};
        if (tag_is(secs[s], "PODS")) {
            im.has_pod = true;
            im.r = in.get<int32_t>();
            const int32_t nup = in.get<int32_t>();
            im.rows = in.get<int64_t>();
            im.n_reorth = in.get<int32_t>();
            in.get<int32_t>();
            if (!in.ok || im.r < 0 || im.r > im.N || nup < 0 || im.rows < 0) return bad("PODS");
            if (!get_vec(in, im.sigma, im.r) || !get_vec(in, im.sweeps, nup)) return bad("PODS");
            in.pad8();
            if (headers_only) {
                if (!skip(in, (uint64_t)im.r * im.N, 8) || !skip(in, (uint64_t)im.r * im.rows, 8)) return bad("PODS");
            } else if (!get_vec(in, im.W, (uint64_t)im.r * im.N) || !get_vec(in, im.V, (uint64_t)im.r * im.rows)) {
                return bad("PODS");
            }
        } else if (tag_is(secs[s], "BASE")) {
            im.has_basis = true;
            im.ns = in.get<int32_t>();
            im.nt = in.get<int32_t>();
            im.Nt = in.get<int32_t>();
            in.get<int32_t>();
            if (!in.ok || im.ns < 1 || im.nt < 1 || im.Nt < 1 || im.ns > im.N || im.nt > im.Nt) return bad("BASE");
            const uint64_t nphi = (uint64_t)im.ns * im.N, nT = (uint64_t)im.Nt * im.ns * im.nt;
            if (headers_only) {
                if (!skip(in, nphi, 8) || !skip(in, nT, 8)) return bad("BASE");
            } else if (!get_vec(in, im.phi, nphi) || !get_vec(in, im.T, nT)) {
                return bad("BASE");
            }
        } else if (tag_is(secs[s], "REDU")) {
            im.has_reduced = true;
            const int32_t ns = in.get<int32_t>(), nt = in.get<int32_t>(), Nt = in.get<int32_t>(),
                          Q = in.get<int32_t>();
            if (!in.ok || !im.has_basis || ns != im.ns || nt != im.nt || Nt != im.Nt || Q != im.Q)
                return bad("REDU");
            const uint64_t n = (uint64_t)ns * nt;
            const uint64_t cnt[8] = {(uint64_t)Q * ns * ns, n * n, (uint64_t)ns * nt * nt, (uint64_t)ns * nt * nt,
                                     n, (uint64_t)Nt, (uint64_t)ns * Nt, (uint64_t)ns};
            std::vector<double>* dst[8] = {&im.Ahat, &im.G, &im.M, &im.S, &im.rhs, &im.dt, &im.bs, &im.u0s};
            for (int i = 0; i < 8; ++i) {
                if (headers_only ? !skip(in, cnt[i], 8) : !get_vec(in, *dst[i], cnt[i])) return bad("REDU");
            }
        } else if (tag_is(secs[s], "SURR")) {
            im.has_surrogate = true;
            im.n_in = in.get<int32_t>();
            im.hidden = in.get<int32_t>();
            im.n_out = in.get<int32_t>();
            im.trained = in.get<int32_t>();
            im.n_params = in.get<int64_t>();
            im.adam_t = in.get<int64_t>();
            im.lo[0] = in.get<double>();
            im.lo[1] = in.get<double>();
            im.hi[0] = in.get<double>();
            im.hi[1] = in.get<double>();
            const int64_t want = (int64_t)im.hidden * im.n_in + im.hidden + (int64_t)im.hidden * im.hidden +
                                 im.hidden + (int64_t)im.n_out * im.hidden + im.n_out;
            if (!in.ok || im.n_in != 2 || im.hidden < 1 || im.n_out < 1 || im.n_params != want) return bad("SURR");
            if (headers_only) {
                if (!skip(in, 3 * (uint64_t)im.n_params, 4)) return bad("SURR");
                in.pad8();
                if (!skip(in, 2 * (uint64_t)im.n_out, 8)) return bad("SURR");
            } else {
                if (!get_vec(in, im.params, im.n_params) || !get_vec(in, im.adam_m, im.n_params) ||
                    !get_vec(in, im.adam_v, im.n_params))
                    return bad("SURR");
                in.pad8();
                if (!get_vec(in, im.mean, im.n_out) || !get_vec(in, im.stdv, im.n_out)) return bad("SURR");
            }
        } else {
            return st_fail(ST_ERR_ARG, "saved model: unknown section %.4s", secs[s].tag);
        }
        if (!in.ok || in.at != in.n) return st_fail(ST_ERR_ARG, "saved model: malformed section %.4s", secs[s].tag);
    }
    return ST_OK;
}

// device -> host copy of `count` doubles (synchronous on the model's stream)
template <typename T>
st_status download(st_model* m, std::vector<T>& h, const void* d, size_t count) {
    h.resize(count);
    if (count == 0) return ST_OK;
    ST_CUDA_TRY(cudaMemcpyAsync(h.data(), d, sizeof(T) * count, cudaMemcpyDeviceToHost, m->stream));
    ST_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return ST_OK;
}

// host array -> fresh device buffer, released by the returned holder
struct DevTmp {
    void* p = nullptr;
    ~DevTmp() {
        if (p) cudaFree(p);
    }
};

st_status upload(DevTmp& t, const void* h, size_t bytes) {
    ST_CUDA_TRY(cudaMalloc(&t.p, std::max<size_t>(bytes, 16)));
    if (bytes) ST_CUDA_TRY(cudaMemcpy(t.p, h, bytes, cudaMemcpyHostToDevice));
    return ST_OK;
}

}  // namespace

extern "C" st_status st_model_file_info(const char* path, st_model_info* info) {
    if (!path || !info) return st_fail(ST_ERR_ARG, "st_model_file_info: NULL argument");
    std::vector<Section> secs;
    ST_TRY(read_file(path, secs));
    Image im;
    ST_TRY(parse(secs, im, true));
    std::memset(info, 0, sizeof(*info));
    info->version = (int32_t)kVersion;
    info->n_rows = im.N;
    info->nnz = im.nnz;
    info->n_terms = im.Q;
    info->pod_rank = im.r;
    info->pod_rows = im.rows;
    info->ns = im.ns;
    info->nt = im.nt;
    info->Nt = im.Nt;
    info->assembled = im.has_reduced ? 1 : 0;
    info->surrogate = im.has_surrogate && im.trained ? 1 : 0;
    info->n_params = im.has_surrogate ? im.n_params : 0;
    return ST_OK;
}

extern "C" st_status st_model_save(st_model* m, const char* path) {
    if (!m || !path) return st_fail(ST_ERR_ARG, "st_model_save: NULL argument");
    ST_CUDA_TRY(cudaStreamSynchronize(m->stream));
    std::vector<Section> secs;
    auto add = [&](const char* tag, Out& o) {
        Section s;
        std::memcpy(s.tag, tag, 4);
        s.data.swap(o.b);
        secs.push_back(std::move(s));
    };
    {
        Out o;
        const st_options& p = m->opt;
        o.put(p.tol);
        o.put(p.maxit);
        o.put(p.eps_svd);
        o.put(p.eps_sv);
        o.put(p.r_max);
        o.put(p.precision);
        o.put(p.spin_limit);
        o.put(p.refine_steps);
        o.put(p.jacobi_sweeps);
        o.put(p.pod_block);
        o.put(p.fp64_gemm);
        o.put(p.pod_cols);
        o.put(p.fom_path);
        add("OPTS", o);
    }
    {
        Out o;
        o.put<int64_t>(m->N);
        o.put<int64_t>(m->nnz);
        o.put<int32_t>(m->Q);
        o.put<int32_t>(0);
        o.raw(m->h_rowptr.data(), sizeof(int64_t) * m->h_rowptr.size());
        o.raw(m->h_col.data(), sizeof(int32_t) * m->h_col.size());
        o.pad8();
        o.raw(m->h_vals.data(), sizeof(double) * m->h_vals.size());
        add("OPER", o);
    }
    if (m->pod_r > 0 || m->pod_rows > 0) {
        Out o;
        const int r = m->pod_r;
        o.put<int32_t>(r);
        o.put<int32_t>((int32_t)m->pod_sweeps.size());
        o.put<int64_t>(m->pod_rows);
        o.put<int32_t>(m->pod_reorth);
        o.put<int32_t>(0);
        o.raw(m->sigma.data(), sizeof(double) * r);
        for (int s : m->pod_sweeps) o.put<int32_t>(s);
        o.pad8();
        std::vector<double> h;
        ST_TRY(download(m, h, m->W.p, (size_t)m->N * r));
        o.raw(h.data(), sizeof(double) * h.size());
        h.assign((size_t)m->pod_rows * r, 0.0);
        if (r > 0 && m->pod_rows > 0) {
            ST_CUDA_TRY(cudaMemcpy2DAsync(h.data(), sizeof(double) * m->pod_rows, m->V.p, sizeof(double) * m->pod_ldv,
                                          sizeof(double) * m->pod_rows, r, cudaMemcpyDeviceToHost, m->stream));
            ST_CUDA_TRY(cudaStreamSynchronize(m->stream));
        }
        o.raw(h.data(), sizeof(double) * h.size());
        add("PODS", o);
    }
    if (m->d_phi) {
        Out o;
        o.put<int32_t>(m->ns);
        o.put<int32_t>(m->nt);
        o.put<int32_t>(m->Nt);
        o.put<int32_t>(0);
        std::vector<double> h;
        ST_TRY(download(m, h, m->d_phi, (size_t)m->N * m->ns));
        o.raw(h.data(), sizeof(double) * h.size());
        ST_TRY(download(m, h, m->d_T, (size_t)m->Nt * m->ns * m->nt));
        o.raw(h.data(), sizeof(double) * h.size());
        add("BASE", o);
    }
    if (m->assembled) {
        Out o;
        const size_t ns = m->ns, nt = m->nt, Nt = m->Nt, n = ns * nt;
        o.put<int32_t>(m->ns);
        o.put<int32_t>(m->nt);
        o.put<int32_t>(m->Nt);
        o.put<int32_t>(m->Q);
        const double* src[8] = {m->d_Ahat, m->d_G, m->d_M, m->d_S, m->d_rhs, m->d_dt, m->d_bs, m->d_u0s};
        const size_t cnt[8] = {(size_t)m->Q * ns * ns, n * n, ns * nt * nt, ns * nt * nt, n, Nt, ns * Nt, ns};
        std::vector<double> h;
        for (int i = 0; i < 8; ++i) {
            ST_TRY(download(m, h, src[i], cnt[i]));
            o.raw(h.data(), sizeof(double) * h.size());
        }
        add("REDU", o);
    }
    if (m->mlp.trained) {
        Out o;
        const auto& s = m->mlp;
        o.put<int32_t>(s.n_in);
        o.put<int32_t>(s.hidden);
        o.put<int32_t>(s.n_out);
        o.put<int32_t>(1);
        o.put<int64_t>(s.n_params);
        o.put<int64_t>(s.adam_t);
        o.put(s.lo[0]);
        o.put(s.lo[1]);
        o.put(s.hi[0]);
        o.put(s.hi[1]);
        std::vector<float> hf;
        for (const DevBuf* b : {&s.params, &s.adam_m, &s.adam_v}) {
            ST_TRY(download(m, hf, b->p, (size_t)s.n_params));
            o.raw(hf.data(), sizeof(float) * hf.size());
        }
        o.pad8();
        std::vector<double> hd;
        ST_TRY(download(m, hd, s.stats.p, 2 * (size_t)s.n_out));
        o.raw(hd.data(), sizeof(double) * hd.size());
        add("SURR", o);
    }
    // write to a temporary name, then rename: a reader never sees a partial file
    const std::string tmp = std::string(path) + ".tmp";
    {
        std::unique_ptr<FILE, int (*)(FILE*)> f(std::fopen(tmp.c_str(), "wb"), &std::fclose);
        if (!f) return st_fail(ST_ERR_ARG, "st_model_save: cannot open %s for writing", tmp.c_str());
        const uint32_t ver = kVersion, count = (uint32_t)secs.size();
        bool ok = std::fwrite(kMagic, 1, 8, f.get()) == 8 && std::fwrite(&ver, 4, 1, f.get()) == 1 &&
                  std::fwrite(&count, 4, 1, f.get()) == 1;
        for (const Section& s : secs) {
            const uint32_t zero = 0;
            const uint64_t len = s.data.size(), sum = fnv1a(s.data.data(), s.data.size());
            ok = ok && std::fwrite(s.tag, 1, 4, f.get()) == 4 && std::fwrite(&zero, 4, 1, f.get()) == 1 &&
                 std::fwrite(&len, 8, 1, f.get()) == 1 &&
                 (len == 0 || std::fwrite(s.data.data(), 1, len, f.get()) == len) &&
                 std::fwrite(&sum, 8, 1, f.get()) == 1;
        }
        ok = ok && std::fflush(f.get()) == 0;
        if (!ok) {
            f.reset();
            std::remove(tmp.c_str());
            return st_fail(ST_ERR_ARG, "st_model_save: write to %s failed", tmp.c_str());
        }
    }
    if (std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return st_fail(ST_ERR_ARG, "st_model_save: cannot rename %s to %s", tmp.c_str(), path);
    }
    return ST_OK;
}

extern "C" st_status st_model_load(const char* path, void* stream, st_model** out) {
    if (!path || !out) return st_fail(ST_ERR_ARG, "st_model_load: NULL argument");
    *out = nullptr;
    std::vector<Section> secs;
    ST_TRY(read_file(path, secs));
    Image im;
    ST_TRY(parse(secs, im, false));
    secs.clear();
    std::vector<const double*> vp(im.Q);
    for (int q = 0; q < im.Q; ++q) vp[q] = im.vals.data() + (size_t)q * im.nnz;
    st_affine_csr csr{im.N, im.rowptr.data(), im.col.data(), vp.data(), im.Q};
    st_model* m = nullptr;
    ST_TRY(st_model_create(&csr, &im.opt, stream, &m));
    std::unique_ptr<st_model, void (*)(st_model*)> hold(m, &st_model_destroy);
    if (im.has_pod) {
        DevTmp dW, dV;
        ST_TRY(upload(dW, im.W.data(), sizeof(double) * im.W.size()));
        ST_TRY(upload(dV, im.V.data(), sizeof(double) * im.V.size()));
        ST_TRY(st_pod_set_state(m, im.r, im.rows, (const double*)dW.p, im.sigma.data(), (const double*)dV.p));
        m->pod_sweeps.assign(im.sweeps.begin(), im.sweeps.end());
        m->pod_reorth = im.n_reorth;
    }
    if (im.has_basis) {
        DevTmp dphi, dT;
        ST_TRY(upload(dphi, im.phi.data(), sizeof(double) * im.phi.size()));
        ST_TRY(upload(dT, im.T.data(), sizeof(double) * im.T.size()));
        ST_TRY(st_model_set_basis(m, im.ns, im.nt, im.Nt, (const double*)dphi.p, (const double*)dT.p));
        ST_CUDA_TRY(cudaStreamSynchronize(m->stream));
    }
    if (im.has_reduced)
        ST_TRY(st_internal_install_reduced(m, im.Ahat.data(), im.G.data(), im.M.data(), im.S.data(), im.rhs.data(),
                                           im.dt.data(), im.bs.data(), im.u0s.data()));
    if (im.has_surrogate && im.trained) {
        if (!im.has_basis || im.n_out != im.ns * im.nt)
            return st_fail(ST_ERR_ARG, "st_model_load: the surrogate does not match the basis");
        ST_TRY(st_internal_mlp_install(m, im.hidden, im.params.data(), im.adam_m.data(), im.adam_v.data(),
                                       im.mean.data(), im.stdv.data(), im.lo, im.hi, im.adam_t));
    }
    ST_CUDA_TRY(cudaStreamSynchronize(m->stream));
    *out = hold.release();
    return ST_OK;
}
