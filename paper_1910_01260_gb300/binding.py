"""ctypes binding of libst_rom.so (the C ABI declared in include/st_rom.h).

Argument marshalling only: every step of the method runs inside the CUDA
library.  Device buffers are passed as anything with ``data_ptr()`` (torch
tensors) or as raw integer addresses; host arrays are numpy arrays.  Every
function has the C name; a non-zero status raises ``StError`` carrying the
library's message.  If the library has not been built the import fails: there
is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libst_rom.so")

ST_OK = 0
ST_ERR_ARG = 1
ST_ERR_CUDA = 2
ST_ERR_OOM = 3
ST_ERR_NOT_CONVERGED = 4
ST_ERR_BREAKDOWN = 5
ST_ERR_SINGULAR = 6
ST_ERR_NONFINITE = 7
ST_ERR_TIMEOUT = 8
ST_ERR_STATE = 9
ST_FP64 = 0
ST_FP32_ASSEMBLY = 1
ST_FP32_LU = 2
ST_DGEMM_SIMT = 0
ST_DGEMM_OZAKI = 1
ST_FOM_AUTO = 0
ST_FOM_GRID = 1
ST_FOM_CLUSTER = 2
ST_ORDER_LARGEST_FIRST = 0
ST_ORDER_SMALLEST_FIRST = 1
ST_ORDER_INPUT = 2
ST_GUESS_SURROGATE = 0
ST_GUESS_ZERO = 1
PROFILE_NAME_LEN = 64


class StError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{code}: {msg}")
        self.code = code


class st_options(ctypes.Structure):
    _fields_ = [("tol", c_double), ("maxit", c_int32), ("eps_svd", c_double),
                ("eps_sv", c_double), ("r_max", c_int32), ("precision", c_int32),
                ("spin_limit", c_int64), ("refine_steps", c_int32), ("jacobi_sweeps", c_int32),
                ("pod_block", c_int32), ("fp64_gemm", c_int32), ("pod_cols", c_int32),
                ("fom_path", c_int32)]


class st_model_info(ctypes.Structure):
    _fields_ = [("version", c_int32), ("n_terms", c_int32), ("n_rows", c_int64), ("nnz", c_int64),
                ("pod_rows", c_int64), ("pod_rank", c_int32), ("ns", c_int32), ("nt", c_int32),
                ("Nt", c_int32), ("assembled", c_int32), ("surrogate", c_int32), ("n_params", c_int64)]


class st_solve_plan(ctypes.Structure):
    _fields_ = [("panel", c_int32), ("ctas_per_sm", c_int32), ("order", c_int32)]


class st_affine_csr(ctypes.Structure):
    _fields_ = [("n_rows", c_int64), ("rowptr", POINTER(c_int64)), ("col", POINTER(c_int32)),
                ("vals", POINTER(POINTER(c_double))), ("n_terms", c_int32)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -c 'import __graft_entry__ as g; g.build()'`")
lib = ctypes.CDLL(LIB_PATH)

_P = c_void_p
_SIGS = {
    "st_options_default": (None, [POINTER(st_options)]),
    "st_last_error": (c_char_p, []),
    "st_status_string": (c_char_p, [c_int32]),
    "st_kernel_launches": (c_int64, []),
    "st_model_create": (c_int32, [POINTER(st_affine_csr), POINTER(st_options), _P, POINTER(_P)]),
    "st_model_destroy": (None, [_P]),
    "st_model_set_options": (c_int32, [_P, POINTER(st_options)]),
    "st_sync": (c_int32, [_P]),
    "st_fom_march": (c_int32, [_P, c_int32, _P, c_int32, _P, _P, c_int32, _P, _P, _P, _P, _P]),
    "st_rom_build_basis": (c_int32, [_P, c_int32, c_int32, _P, c_int32, c_int32, _P, _P]),
    "st_model_set_basis": (c_int32, [_P, c_int32, c_int32, c_int32, _P, _P]),
    "st_model_get_basis": (c_int32, [_P, _P, _P, _P]),
    "st_pod_get_state": (c_int32, [_P, _P, _P, _P, _P]),
    "st_pod_get_stats": (c_int32, [_P, _P, _P, c_int32, _P]),
    "st_pod_reset": (c_int32, [_P]),
    "st_pod_update": (c_int32, [_P, c_int64, _P, c_int32]),
    "st_pod_finish": (c_int32, [_P, c_int32, c_int32, c_int32, c_int32]),
    "st_pod_set_state": (c_int32, [_P, c_int32, c_int64, _P, _P, _P]),
    "st_pod_get_dims": (c_int32, [_P, _P, _P]),
    "st_model_get_options": (c_int32, [_P, POINTER(st_options)]),
    "st_model_save": (c_int32, [_P, c_char_p]),
    "st_model_load": (c_int32, [c_char_p, _P, POINTER(_P)]),
    "st_model_file_info": (c_int32, [c_char_p, POINTER(st_model_info)]),
    "st_probe_fp64_fma": (c_int32, [c_int32, c_int64, _P, _P]),
    "st_fom_cluster_occupancy": (c_int32, [_P, _P, _P, _P]),
    "st_fom_st_inverse_norm": (c_int32, [_P, c_int32, _P, c_int32, _P, c_int32, c_double, ctypes.c_uint64, _P, _P]),
    "st_rom_solve_set_plan": (c_int32, [_P, c_int32, POINTER(st_solve_plan)]),
    "st_rom_solve_get_plan": (c_int32, [_P, c_int32, POINTER(st_solve_plan)]),
    "st_rom_solve_tune": (c_int32, [_P, c_int32, _P, _P, _P, c_int32, c_int32, _P, _P, _P,
                                    POINTER(st_solve_plan), _P, _P]),
    "st_profile_enable": (c_int32, [_P, c_int32]),
    "st_profile_read": (c_int32, [_P, c_int32, _P, _P, _P, _P, _P]),
    "st_gemm_f64": (c_int32, [_P, c_int32, c_int32, c_int64, c_int64, c_int64, c_double, _P, c_int64, _P,
                              c_int64, c_double, _P, c_int64]),
    "st_rom_assemble": (c_int32, [_P, _P, c_int32, _P, _P, _P]),
    "st_model_get_reduced": (c_int32, [_P, _P, _P, _P, _P, _P]),
    "st_rom_solve": (c_int32, [_P, c_int32, _P, _P, _P, _P, _P]),
    "st_rom_solve_static": (c_int32, [_P, c_int32, _P, _P, _P, _P, _P]),
    "st_rom_reconstruct": (c_int32, [_P, c_int32, _P, _P, _P, c_int32, _P, _P]),
    "st_rom_spatial_march": (c_int32, [_P, c_int32, _P, _P, _P, _P]),
    "st_rom_residual_norms": (c_int32, [_P, c_int32, _P, c_int32, _P, _P, c_int32, _P, _P, _P, _P]),
    "st_rom_surrogate_train": (c_int32, [_P, c_int32, _P, _P, _P, _P, _P, c_int32, c_int32, ctypes.c_float,
                                         ctypes.c_uint64, _P]),
    "st_rom_surrogate_infer": (c_int32, [_P, c_int32, _P, _P, c_double, _P, _P, _P, _P]),
    "st_rom_surrogate_params": (c_int32, [_P, _P, _P]),
    "st_rom_precond_build": (c_int32, [_P, c_int32, _P, _P]),
    "st_rom_refine": (c_int32, [_P, c_int32, _P, _P, c_int32, c_double, c_int32, _P, _P, _P, _P, _P]),
    "st_rom_surrogate_loss_grad": (c_int32, [_P, c_int32, _P, _P, _P, _P, _P, _P, _P]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def ptr(x) -> int | None:
    """Address of a device tensor, host numpy array or raw integer (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _host(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def last_error() -> str:
    return lib.st_last_error().decode()


def check(code: int) -> None:
    if code != ST_OK:
        raise StError(code, last_error())


def options(**kw) -> st_options:
    o = st_options()
    lib.st_options_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def st_model_file_info(path) -> dict:
    """Validate a saved model file on the host (no GPU) and report its contents."""
    info = st_model_info()
    check(lib.st_model_file_info(os.fsencode(path), ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in st_model_info._fields_}


def st_probe_fp64_fma(blocks_per_sm=4, iters=20000):
    """(TFLOP/s, ms) of the library's FP64 FMA throughput probe on the current device."""
    tf = np.zeros(1, dtype=np.float64)
    ms = np.zeros(1, dtype=np.float64)
    check(lib.st_probe_fp64_fma(int(blocks_per_sm), int(iters), ptr(tf), ptr(ms)))
    return float(tf[0]), float(ms[0])


class Model:
    """Owner of one st_model handle; methods are the C entry points with the
    model argument bound.  Host inputs are converted to contiguous arrays."""

    @classmethod
    def st_model_load(cls, path, stream=None) -> "Model":
        """A model restored from a file written by st_model_save."""
        h = c_void_p()
        st = stream if stream is None or isinstance(stream, int) else getattr(stream, "cuda_stream", stream)
        check(lib.st_model_load(os.fsencode(path), st, ctypes.byref(h)))
        self = cls.__new__(cls)
        self.handle = h
        info = st_model_file_info(path)
        self.N, self.Q = int(info["n_rows"]), int(info["n_terms"])
        self.opts = st_options()
        check(lib.st_model_get_options(h, ctypes.byref(self.opts)))
        self._keep = []
        return self

    def __init__(self, rowptr, col, vals, opts: st_options | None = None, stream=None):
        self._rowptr = _host(rowptr, np.int64)
        self._col = _host(col, np.int32)
        vals = np.asarray(vals, dtype=np.float64)
        if vals.ndim == 1:
            vals = vals[None]
        self._vals = [np.ascontiguousarray(v) for v in vals]
        arr = (POINTER(c_double) * len(self._vals))(
            *[v.ctypes.data_as(POINTER(c_double)) for v in self._vals])
        self._csr = st_affine_csr(self._rowptr.shape[0] - 1,
                                  self._rowptr.ctypes.data_as(POINTER(c_int64)),
                                  self._col.ctypes.data_as(POINTER(c_int32)),
                                  ctypes.cast(arr, POINTER(POINTER(c_double))), len(self._vals))
        self._arr = arr
        self.opts = opts if opts is not None else options()
        h = c_void_p()
        st = stream if stream is None or isinstance(stream, int) else getattr(stream, "cuda_stream", stream)
        check(lib.st_model_create(ctypes.byref(self._csr), ctypes.byref(self.opts), st,
                                  ctypes.byref(h)))
        self.handle = h
        self.N = int(self._rowptr.shape[0] - 1)
        self.Q = len(self._vals)
        self._keep = []

    def close(self) -> None:
        if getattr(self, "handle", None):
            lib.st_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C entry points ---------------------------------------------------
    def st_model_set_options(self, **kw) -> None:
        o = st_options()
        ctypes.memmove(ctypes.byref(o), ctypes.byref(self.opts), ctypes.sizeof(o))
        for k, v in kw.items():
            setattr(o, k, v)
        check(lib.st_model_set_options(self.handle, ctypes.byref(o)))
        self.opts = o

    def st_sync(self) -> None:
        check(lib.st_sync(self.handle))

    def st_fom_march(self, theta, dt, u0, B, F, snapshots, iters=None, status=None) -> None:
        th = _host(theta, np.float64)
        dth = _host(dt, np.float64)
        Fh = _host(F, np.float64) if F is not None else None
        n_in = 0 if Fh is None else (Fh.shape[1] if Fh.ndim == 2 else 1)
        self._keep = [th, dth, Fh]
        check(lib.st_fom_march(self.handle, th.shape[0], ptr(th), dth.shape[0], ptr(dth), ptr(u0),
                               n_in, ptr(B), ptr(Fh), ptr(snapshots), ptr(iters), ptr(status)))

    def st_rom_build_basis(self, n_mu, Nt, snapshots, ns, nt):
        sig = np.zeros(max(int(self.opts.r_max), 1), dtype=np.float64)
        rank = np.zeros(1, dtype=np.int32)
        check(lib.st_rom_build_basis(self.handle, n_mu, Nt, ptr(snapshots), ns, nt, ptr(sig),
                                     ptr(rank)))
        return sig[:rank[0]].copy(), int(rank[0])

    def st_model_set_basis(self, ns, nt, Nt, phi_s, T) -> None:
        check(lib.st_model_set_basis(self.handle, ns, nt, Nt, ptr(phi_s), ptr(T)))

    def st_model_get_basis(self, phi_s=None, T=None):
        dims = np.zeros(3, dtype=np.int32)
        check(lib.st_model_get_basis(self.handle, ptr(phi_s), ptr(T), ptr(dims)))
        return tuple(int(d) for d in dims)

    def st_pod_get_state(self, W=None, V=None):
        r = np.zeros(1, dtype=np.int32)
        check(lib.st_pod_get_state(self.handle, None, None, None, ptr(r)))
        sig = np.zeros(max(int(r[0]), 1), dtype=np.float64)
        check(lib.st_pod_get_state(self.handle, ptr(W), ptr(V), ptr(sig), ptr(r)))
        return sig[:r[0]].copy(), int(r[0])

    def st_pod_get_stats(self):
        """(Jacobi sweeps per block update, number of W re-orthogonalisations)."""
        n = np.zeros(1, dtype=np.int32)
        check(lib.st_pod_get_stats(self.handle, ptr(n), None, 0, None))
        sw = np.zeros(max(int(n[0]), 1), dtype=np.int32)
        ro = np.zeros(1, dtype=np.int32)
        check(lib.st_pod_get_stats(self.handle, ptr(n), ptr(sw), int(n[0]), ptr(ro)))
        return sw[:n[0]].tolist(), int(ro[0])

    def st_fom_cluster_occupancy(self):
        """(CTAs per cluster, clusters resident at once, shared memory per CTA)."""
        c = np.zeros(1, dtype=np.int32)
        n = np.zeros(1, dtype=np.int32)
        b = np.zeros(1, dtype=np.int64)
        check(lib.st_fom_cluster_occupancy(self.handle, ptr(c), ptr(n), ptr(b)))
        return int(c[0]), int(n[0]), int(b[0])

    def st_fom_st_inverse_norm(self, theta, dt, max_iter=200, tol=1e-8, seed=7):
        """(||(A^st)^-1||_2 estimates per sample, iterations used)."""
        th = _host(theta, np.float64)
        if th.ndim == 1:
            th = th[None]
        dth = _host(dt, np.float64)
        out = np.zeros(th.shape[0], dtype=np.float64)
        it = np.zeros(1, dtype=np.int32)
        self._keep = [th, dth]
        check(lib.st_fom_st_inverse_norm(self.handle, th.shape[0], ptr(th), dth.shape[0], ptr(dth), int(max_iter),
                                         float(tol), ctypes.c_uint64(seed), ptr(out), ptr(it)))
        return out, int(it[0])

    def st_pod_reset(self) -> None:
        check(lib.st_pod_reset(self.handle))

    def st_pod_update(self, n_cols, snapshots, cols_per_update) -> None:
        check(lib.st_pod_update(self.handle, int(n_cols), ptr(snapshots), int(cols_per_update)))

    def st_pod_finish(self, n_mu, Nt, ns, nt) -> None:
        check(lib.st_pod_finish(self.handle, n_mu, Nt, ns, nt))

    def st_pod_set_state(self, r, rows, W, sigma, V) -> None:
        sig = _host(sigma, np.float64)
        check(lib.st_pod_set_state(self.handle, int(r), int(rows), ptr(W), ptr(sig), ptr(V)))

    def st_pod_get_dims(self):
        r = np.zeros(1, dtype=np.int32)
        rows = np.zeros(1, dtype=np.int64)
        check(lib.st_pod_get_dims(self.handle, ptr(r), ptr(rows)))
        return int(r[0]), int(rows[0])

    def st_model_save(self, path) -> None:
        check(lib.st_model_save(self.handle, os.fsencode(path)))

    def st_profile_enable(self, on: bool = True) -> None:
        check(lib.st_profile_enable(self.handle, 1 if on else 0))

    def st_profile_read(self):
        """{kernel name: (total ms, launches, algorithmic flops or 0)} since the
        last st_profile_enable, largest total time first."""
        n = np.zeros(1, dtype=np.int32)
        check(lib.st_profile_read(self.handle, 0, None, None, None, None, ptr(n)))
        k = int(n[0])
        names = np.zeros((max(k, 1), PROFILE_NAME_LEN), dtype=np.uint8)
        ms = np.zeros(max(k, 1), dtype=np.float64)
        cnt = np.zeros(max(k, 1), dtype=np.int64)
        fl = np.zeros(max(k, 1), dtype=np.float64)
        check(lib.st_profile_read(self.handle, k, ptr(names), ptr(ms), ptr(cnt), ptr(fl), ptr(n)))
        out = {}
        for i in range(min(k, int(n[0]))):
            name = bytes(names[i]).split(b"\0", 1)[0].decode()
            out[name] = (float(ms[i]), int(cnt[i]), float(fl[i]))
        return out

    def st_gemm_f64(self, trans_a, trans_b, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc) -> None:
        check(lib.st_gemm_f64(self.handle, int(trans_a), int(trans_b), M, N, K, alpha, ptr(A), lda, ptr(B), ldb,
                              beta, ptr(C), ldc))

    def st_rom_assemble(self, dt, B, F, u0=None) -> None:
        dth = _host(dt, np.float64)
        Fh = _host(F, np.float64) if F is not None else None
        n_in = 0 if Fh is None else (Fh.shape[1] if Fh.ndim == 2 else 1)
        self._keep = [dth, Fh]
        check(lib.st_rom_assemble(self.handle, ptr(dth), n_in, ptr(B), ptr(Fh), ptr(u0)))

    def st_model_get_reduced(self, ns, nt):
        n = ns * nt
        Ahat = np.zeros((self.Q, ns, ns))
        G = np.zeros((n, n))
        M = np.zeros((ns, nt, nt))
        S = np.zeros((ns, nt, nt))
        rhs = np.zeros(n)
        check(lib.st_model_get_reduced(self.handle, ptr(Ahat), ptr(G), ptr(M), ptr(S), ptr(rhs)))
        # library layout is column major per matrix
        return (Ahat.transpose(0, 2, 1).copy(), G.T.copy(), M.transpose(0, 2, 1).copy(),
                S.transpose(0, 2, 1).copy(), rhs)

    def st_rom_solve(self, n_mu, theta, ns_nt, uhat, rel_res=None, status=None) -> None:
        check(lib.st_rom_solve(self.handle, n_mu, ptr(theta), ptr(ns_nt), ptr(uhat), ptr(rel_res),
                               ptr(status)))

    def st_rom_solve_static(self, n_mu, theta, ns_nt, uhat, rel_res=None, status=None) -> None:
        check(lib.st_rom_solve_static(self.handle, n_mu, ptr(theta), ptr(ns_nt), ptr(uhat),
                                      ptr(rel_res), ptr(status)))

    def st_rom_solve_set_plan(self, precision, plan=None) -> None:
        """plan: dict(panel, ctas_per_sm, order) or None for the defaults."""
        if plan is None:
            check(lib.st_rom_solve_set_plan(self.handle, int(precision), None))
            return
        p = st_solve_plan(int(plan["panel"]), int(plan["ctas_per_sm"]), int(plan["order"]))
        check(lib.st_rom_solve_set_plan(self.handle, int(precision), ctypes.byref(p)))

    def st_rom_solve_get_plan(self, precision) -> dict:
        p = st_solve_plan()
        check(lib.st_rom_solve_get_plan(self.handle, int(precision), ctypes.byref(p)))
        return {"panel": p.panel, "ctas_per_sm": p.ctas_per_sm, "order": p.order}

    def st_rom_solve_tune(self, n_mu, theta, ns_nt, uhat, reps=2, cap=64) -> dict:
        """Time every candidate plan on this batch and install the fastest."""
        cands = (st_solve_plan * cap)()
        ms = np.zeros(cap, dtype=np.float32)
        n = np.zeros(1, dtype=np.int32)
        best = st_solve_plan()
        bms = np.zeros(1, dtype=np.float32)
        dms = np.zeros(1, dtype=np.float32)
        check(lib.st_rom_solve_tune(self.handle, n_mu, ptr(theta), ptr(ns_nt), ptr(uhat), int(reps), cap,
                                    ctypes.addressof(cands), ptr(ms), ptr(n), ctypes.byref(best), ptr(bms),
                                    ptr(dms)))
        k = min(int(n[0]), cap)
        return {"best": {"panel": best.panel, "ctas_per_sm": best.ctas_per_sm, "order": best.order},
                "best_ms": float(bms[0]), "default_ms": float(dms[0]), "n_candidates": int(n[0]),
                "candidates": [{"panel": cands[i].panel, "ctas_per_sm": cands[i].ctas_per_sm,
                                "order": cands[i].order, "ms": float(ms[i])} for i in range(k)]}

    def st_rom_reconstruct(self, n_mu, uhat, ns_nt, u=None, n_out=0, Cout=None, y=None) -> None:
        check(lib.st_rom_reconstruct(self.handle, n_mu, ptr(uhat), ptr(ns_nt), ptr(u), n_out,
                                     ptr(Cout), ptr(y)))

    def st_rom_residual_norms(self, theta, dt, u0, B, F, U, rnorm) -> None:
        th = _host(theta, np.float64)
        dth = _host(dt, np.float64)
        Fh = _host(F, np.float64) if F is not None else None
        n_in = 0 if Fh is None else (Fh.shape[1] if Fh.ndim == 2 else 1)
        self._keep = [th, dth, Fh]
        check(lib.st_rom_residual_norms(self.handle, th.shape[0], ptr(th), dth.shape[0], ptr(dth),
                                        ptr(u0), n_in, ptr(B), ptr(Fh), ptr(U), ptr(rnorm)))

    def st_rom_spatial_march(self, n_mu, theta, ns_mu, uhat, status=None) -> None:
        check(lib.st_rom_spatial_march(self.handle, n_mu, ptr(theta), ptr(ns_mu), ptr(uhat),
                                       ptr(status)))


def _surrogate_methods():
    def st_rom_surrogate_train(self, n, mu, mu_lo, mu_hi, uhat, init=None, epochs=100, batch=1024,
                               lr=1e-3, seed=5):
        lo = _host(mu_lo, np.float64)
        hi = _host(mu_hi, np.float64)
        ini = None if init is None else _host(init, np.float32)
        losses = np.zeros(max(int(epochs), 1), dtype=np.float32)
        self._keep = [lo, hi, ini, losses]
        check(lib.st_rom_surrogate_train(self.handle, n, ptr(mu), ptr(lo), ptr(hi), ptr(uhat), ptr(ini),
                                         epochs, batch, ctypes.c_float(lr), ctypes.c_uint64(seed),
                                         ptr(losses)))
        return losses[:epochs].copy()

    def st_rom_surrogate_infer(self, n, mu, theta, gate, uhat, rel_res, used_fallback):
        nf = np.zeros(1, dtype=np.int32)
        check(lib.st_rom_surrogate_infer(self.handle, n, ptr(mu), ptr(theta), gate, ptr(uhat), ptr(rel_res),
                                         ptr(used_fallback), ptr(nf)))
        return int(nf[0])

    def st_rom_surrogate_params(self):
        cnt = np.zeros(1, dtype=np.int64)
        check(lib.st_rom_surrogate_params(self.handle, None, ptr(cnt)))
        out = np.zeros(int(cnt[0]), dtype=np.float32)
        check(lib.st_rom_surrogate_params(self.handle, ptr(out), ptr(cnt)))
        return out

    def st_rom_surrogate_loss_grad(self, n, mu, mu_lo, mu_hi, uhat, params):
        lo = _host(mu_lo, np.float64)
        hi = _host(mu_hi, np.float64)
        pr = _host(params, np.float32)
        grad = np.zeros_like(pr)
        loss = np.zeros(1, dtype=np.float32)
        check(lib.st_rom_surrogate_loss_grad(self.handle, n, ptr(mu), ptr(lo), ptr(hi), ptr(uhat), ptr(pr),
                                             ptr(grad), ptr(loss)))
        return float(loss[0]), grad

    def st_rom_precond_build(self, mu_ref, theta_ref):
        mr = _host(mu_ref, np.float64)
        tr = _host(theta_ref, np.float64)
        check(lib.st_rom_precond_build(self.handle, mr.shape[0], ptr(mr), ptr(tr)))

    def st_rom_refine(self, n, mu, theta, guess, gate, max_iter, uhat, rel_res, used_fallback):
        """(corrections applied, fallback count)."""
        it = np.zeros(1, dtype=np.int32)
        nf = np.zeros(1, dtype=np.int32)
        check(lib.st_rom_refine(self.handle, n, ptr(mu), ptr(theta), int(guess), float(gate), int(max_iter),
                                ptr(uhat), ptr(rel_res), ptr(used_fallback), ptr(it), ptr(nf)))
        return int(it[0]), int(nf[0])

    for f in (st_rom_surrogate_train, st_rom_surrogate_infer, st_rom_surrogate_params,
              st_rom_surrogate_loss_grad, st_rom_precond_build, st_rom_refine):
        setattr(Model, f.__name__, f)


_surrogate_methods()
