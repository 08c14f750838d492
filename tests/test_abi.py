"""The C-ABI library: loads, exports every declared entry point, matches the
binding's struct layouts, and validates host-side arguments (no GPU needed)."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "st_rom.h")


@pytest.fixture(scope="module")
def st():
    import __graft_entry__
    __graft_entry__._builder().build()
    import paper_1910_01260_gb300 as st
    return st


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:st_status|void|const char\s*\*)\s*(st_\w+)\s*\(", txt, re.M)))


def test_exports_every_declared_symbol(st):
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", st.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(\w+)$", out, re.M))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(st.lib, n)


def test_struct_layout_matches_c(st):
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "st_rom.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(st_options), offsetof(st_options, maxit),
         offsetof(st_options, eps_svd), offsetof(st_options, r_max), offsetof(st_options, spin_limit),
         offsetof(st_options, jacobi_sweeps), offsetof(st_options, pod_block), offsetof(st_options, fp64_gemm),
         offsetof(st_options, pod_cols),
         sizeof(st_affine_csr), offsetof(st_affine_csr, col),
         offsetof(st_affine_csr, vals), offsetof(st_affine_csr, n_terms));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = list(map(int, subprocess.run([exe], capture_output=True, text=True).stdout.split()))
    o, a = st.binding.st_options, st.binding.st_affine_csr
    mine = [ctypes.sizeof(o), o.maxit.offset, o.eps_svd.offset, o.r_max.offset, o.spin_limit.offset,
            o.jacobi_sweeps.offset, o.pod_block.offset, o.fp64_gemm.offset, o.pod_cols.offset, ctypes.sizeof(a),
            a.col.offset, a.vals.offset,
            a.n_terms.offset]
    assert vals == mine


def test_defaults_and_names(st):
    o = st.options()
    assert o.tol == 1e-13 and o.maxit == 1000 and o.r_max == 256 and o.refine_steps == 1 and o.pod_block == 1
    assert o.fp64_gemm == st.ST_DGEMM_OZAKI and o.pod_cols == 0
    assert st.lib.st_status_string(st.ST_ERR_SINGULAR) == b"ST_ERR_SINGULAR"
    assert st.lib.st_status_string(99) == b"ST_ERR_UNKNOWN"


def _csr(rowptr, col, vals, n_terms=1):
    st = __import__("paper_1910_01260_gb300")
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    vv = [np.ascontiguousarray(vals, dtype=np.float64) for _ in range(n_terms)]
    arr = (ctypes.POINTER(ctypes.c_double) * n_terms)(*[v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for v in vv])
    s = st.binding.st_affine_csr(len(rp) - 1, rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 cl.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 ctypes.cast(arr, ctypes.POINTER(ctypes.POINTER(ctypes.c_double))), n_terms)
    return s, (rp, cl, vv, arr)


@pytest.mark.parametrize("case", ["rowptr0", "col_range", "decreasing", "no_terms"])
def test_create_rejects_bad_csr_before_touching_the_gpu(st, case):
    rowptr, col, vals, nt = [0, 1, 2], [0, 1], [1.0, 1.0], 1
    if case == "rowptr0":
        rowptr = [1, 1, 2]
    elif case == "col_range":
        col = [0, 5]
    elif case == "decreasing":
        rowptr, col, vals = [0, 2, 1], [0, 1], [1.0, 1.0]
    elif case == "no_terms":
        nt = 0
    s, keep = _csr(rowptr, col, vals, max(nt, 1))
    s.n_terms = nt
    h = ctypes.c_void_p()
    rc = st.lib.st_model_create(ctypes.byref(s), None, None, ctypes.byref(h))
    assert rc == st.ST_ERR_ARG
    assert len(st.last_error()) > 0
    assert not h.value


def test_null_handle_arguments(st):
    assert st.lib.st_sync(None) == st.ST_ERR_ARG
    assert st.lib.st_rom_solve(None, 1, None, None, None, None, None) == st.ST_ERR_ARG
    assert st.lib.st_rom_assemble(None, None, 0, None, None, None) == st.ST_ERR_ARG
    assert st.lib.st_profile_enable(None, 1) == st.ST_ERR_ARG
    assert st.lib.st_profile_read(None, 0, None, None, None, None, None) == st.ST_ERR_ARG
    assert st.lib.st_pod_get_stats(None, None, None, 0, None) == st.ST_ERR_ARG
    assert st.lib.st_gemm_f64(None, 0, 0, 1, 1, 1, 1.0, None, 1, None, 1, 0.0, None, 1) == st.ST_ERR_ARG
    assert st.lib.st_rom_spatial_march(None, 1, None, None, None, None) == st.ST_ERR_ARG
    assert st.lib.st_rom_residual_norms(None, 1, None, 1, None, None, 0, None, None, None, None) == st.ST_ERR_ARG
    st.lib.st_model_destroy(None)
