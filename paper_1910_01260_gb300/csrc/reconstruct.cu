// Reconstruction u^st ~= Phi_st uhat by blocks (Eqs. blockstructure,
// ststateapproximation): each spatial mode i has its own temporal basis, so
//   C_p[i, k] = sum_{j < nt_p} uhat_p[i + ns_p j] phi_t^{i,j}[k]   (i < ns_p, else 0)
//   u_p^k     = Phi_s C_p[:, k]             (one FP64 GEMM for all samples:
//               the C_p lie side by side, and so do the u_p)
//   y_p^k     = Chat^T C_p[:, k], Chat = Phi_s^T Cout   (outputs, Eq.
//               outputFromReducedsol, without forming u)
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace {

__global__ void temporal_contract_kernel(int n_mu, int ns, int nt, int Nt,
                                         const double* __restrict__ uhat,
                                         const int32_t* __restrict__ ns_nt,
                                         const double* __restrict__ T, double* C) {
    const int64_t per = (int64_t)ns * Nt;
    const int64_t tot = per * n_mu;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(t / per);
        const int64_t rem = t % per;
        const int i = (int)(rem % ns), k = (int)(rem / ns);
        int a = ns, b = nt;
        if (ns_nt) {
            a = ns_nt[2 * p];
            b = ns_nt[2 * p + 1];
        }
        double v = 0.0;
        if (a >= 1 && a <= ns && b >= 1 && b <= nt && i < a) {
            const double* up = uhat + (int64_t)p * ns * nt;
            for (int j = 0; j < b; ++j) v = fma(up[i + a * j], T[k + (int64_t)(i + ns * j) * Nt], v);
        }
        C[t] = v;  // C_p is ns x Nt, column major
    }
}

// y[o, c] = sum_i Chat[i, o] C[i, c] for the ncols columns of all samples'
// C side by side (ns x ncols, ld ns): one output per thread, the ns products
// in order.  n_out is a handful of functionals, far too few rows for a GEMM
// tile.
__global__ void outputs_kernel(int ns, int n_out, int64_t ncols, const double* __restrict__ Chat,
                               const double* __restrict__ C, double* y) {
    const int64_t tot = ncols * n_out;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(t % n_out);
        const int64_t c = t / n_out;
        const double* cc = C + c * ns;
        const double* ch = Chat + (int64_t)o * ns;
        double v = 0.0;
        for (int i = 0; i < ns; ++i) v = fma(ch[i], cc[i], v);
        y[t] = v;  // y_p is n_out x Nt: column c of all samples at o + n_out c
    }
}

}  // namespace

extern "C" st_status st_rom_reconstruct(st_model* m, int32_t n_mu, const double* uhat,
                                        const int32_t* ns_nt, double* u, int32_t n_out,
                                        const double* Cout, double* y) {
    if (!m) return st_fail(ST_ERR_ARG, "st_rom_reconstruct: NULL model");
    if (!m->d_phi) return st_fail(ST_ERR_STATE, "st_rom_reconstruct: no basis");
    if (n_mu < 0 || (n_mu > 0 && !uhat)) return st_fail(ST_ERR_ARG, "st_rom_reconstruct: bad arguments");
    if ((y || Cout) && (n_out < 1 || !y || !Cout))
        return st_fail(ST_ERR_ARG, "st_rom_reconstruct: outputs need Cout, y and n_out >= 1");
    if (n_mu == 0 || (!u && !y)) return ST_OK;
    const int ns = m->ns, nt = m->nt, Nt = m->Nt;
    const int64_t N = m->N;
    cudaStream_t st = m->stream;
    const size_t szC = (size_t)ns * Nt * n_mu;
    const size_t szCh = y ? (size_t)ns * n_out : 0;
    ST_TRY(st_grow(m, m->ws_misc, sizeof(double) * (szC + szCh + 16)));
    double* C = (double*)m->ws_misc.p;
    double* Chat = C + szC;
    const int gb = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)szC + 255) / 256, 8 * m->num_sms));
    {
        ST_PROF(m, "temporal_contract_kernel");
        temporal_contract_kernel<<<gb, 256, 0, st>>>(n_mu, ns, nt, Nt, uhat, ns_nt, m->d_T, C);
        ST_TRY(st_check_launch("temporal_contract"));
    }
    // u = Phi_s [C_0 ... C_{n_mu-1}]: N x (Nt n_mu), sample p's field at
    // column p Nt (one product, on the tensor cores when it is large)
    if (u)
        ST_TRY(st_dgemm(m, false, false, N, (int64_t)Nt * n_mu, ns, 1.0, m->d_phi, N, C, ns, 0.0, u, N));
    if (y) {
        ST_TRY(st_dgemm(m, true, false, ns, n_out, N, 1.0, m->d_phi, N, Cout, N, 0.0, Chat, ns));
        const int64_t ncols = (int64_t)Nt * n_mu;
        const int gy = (int)std::max<int64_t>(1, std::min<int64_t>((ncols * n_out + 255) / 256, 8 * m->num_sms));
        ST_PROF(m, "outputs_kernel");
        outputs_kernel<<<gy, 256, 0, st>>>(ns, n_out, ncols, Chat, C, y);
        ST_TRY(st_check_launch("outputs"));
    }
    return ST_OK;
}
