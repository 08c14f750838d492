"""The saved-model file format (st_model_save / st_model_load /
st_model_file_info), checked on the host: a file written here from the
documented layout is read back by the library's validator, and damaged files
are rejected.  The GPU round trip (save, load, identical solves, resumed
basis build) is in tests/test_gpu_persist.py."""
import os
import struct

import numpy as np
import pytest


@pytest.fixture(scope="module")
def st():
    import __graft_entry__
    __graft_entry__._builder().build()
    import paper_1910_01260_gb300 as st
    return st


def fnv1a(b: bytes) -> int:
    h = 1469598103934665603
    for x in b:
        h ^= x
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def pad8(b: bytes) -> bytes:
    return b + b"\0" * (-len(b) % 8)


def section(tag: bytes, payload: bytes) -> bytes:
    return tag + struct.pack("<IQ", 0, len(payload)) + payload + struct.pack("<Q", fnv1a(payload))


def model_bytes(N=6, Q=2, r=3, rows=8, ns=2, nt=2, Nt=4, reduced=True, surrogate=True, seed=0):
    rng = np.random.default_rng(seed)
    rowptr = np.arange(0, 2 * N + 1, 2, dtype=np.int64)
    nnz = int(rowptr[-1])
    col = np.array([[i, (i + 1) % N] for i in range(N)], dtype=np.int32).ravel()
    vals = rng.standard_normal((Q, nnz))
    opts = struct.pack("<diddiiqiiiiii", 1e-13, 1000, 1e-12, 1e-14, 256, 0, 20000000, 1, 40, 1, 1, 0, 0)
    assert len(opts) == 68
    secs = [section(b"OPTS", opts),
            section(b"OPER", pad8(struct.pack("<qqii", N, nnz, Q, 0) + rowptr.tobytes() + col.tobytes())
                    + vals.tobytes())]
    sweeps = np.array([5, 7], dtype=np.int32)
    pods = (struct.pack("<iiqii", r, len(sweeps), rows, 1, 0) + np.sort(rng.random(r))[::-1].tobytes()
            + sweeps.tobytes())
    pods = pad8(pods) + rng.standard_normal(N * r).tobytes() + rng.standard_normal(rows * r).tobytes()
    secs.append(section(b"PODS", pods))
    secs.append(section(b"BASE", struct.pack("<iiii", ns, nt, Nt, 0) + rng.standard_normal(N * ns).tobytes()
                        + rng.standard_normal(Nt * ns * nt).tobytes()))
    n = ns * nt
    if reduced:
        arrs = [Q * ns * ns, n * n, ns * nt * nt, ns * nt * nt, n, Nt, ns * Nt, ns]
        secs.append(section(b"REDU", struct.pack("<iiii", ns, nt, Nt, Q)
                            + b"".join(rng.standard_normal(c).tobytes() for c in arrs)))
    if surrogate:
        H = 8
        n_params = H * 2 + H + H * H + H + n * H + n
        body = struct.pack("<iiiiqqdddd", 2, H, n, 1, n_params, 17, 0.5, 0.1, 1.5, 0.95)
        body += b"".join(rng.standard_normal(n_params).astype(np.float32).tobytes() for _ in range(3))
        body = pad8(body) + rng.standard_normal(2 * n).tobytes()
        secs.append(section(b"SURR", body))
    head = b"STROMMDL" + struct.pack("<II", 1, len(secs))
    return head + b"".join(secs), dict(N=N, nnz=nnz, Q=Q, r=r, rows=rows, ns=ns, nt=nt, Nt=Nt)


def test_file_info_reads_the_documented_layout(st, tmp_path):
    data, d = model_bytes()
    p = tmp_path / "m.strom"
    p.write_bytes(data)
    info = st.st_model_file_info(str(p))
    assert info["version"] == 1
    assert (info["n_rows"], info["nnz"], info["n_terms"]) == (d["N"], d["nnz"], d["Q"])
    assert (info["pod_rank"], info["pod_rows"]) == (d["r"], d["rows"])
    assert (info["ns"], info["nt"], info["Nt"]) == (d["ns"], d["nt"], d["Nt"])
    assert info["assembled"] == 1 and info["surrogate"] == 1 and info["n_params"] > 0


def test_file_info_optional_sections(st, tmp_path):
    data, _ = model_bytes(reduced=False, surrogate=False)
    p = tmp_path / "m.strom"
    p.write_bytes(data)
    info = st.st_model_file_info(str(p))
    assert info["assembled"] == 0 and info["surrogate"] == 0 and info["n_params"] == 0


@pytest.mark.parametrize("damage", ["magic", "version", "checksum", "truncated", "trailing", "length",
                                    "section_order", "unknown_section"])
def test_damaged_files_are_rejected(st, tmp_path, damage):
    data, _ = model_bytes()
    b = bytearray(data)
    if damage == "magic":
        b[0:8] = b"STROMXXX"
    elif damage == "version":
        b[8:12] = struct.pack("<I", 2)
    elif damage == "checksum":
        b[16 + 16 + 3] ^= 0x01          # a byte of the OPTS payload
    elif damage == "truncated":
        b = b[:-9]
    elif damage == "trailing":
        b += b"\0"
    elif damage == "length":
        b[16 + 8:16 + 16] = struct.pack("<Q", 60)  # OPTS claims 60 bytes
    elif damage == "section_order":
        # swap the OPTS and OPER section tags (checksums cover payloads only)
        off2 = 16 + 16 + 68 + 8
        b[16:20], b[off2:off2 + 4] = b"OPER", b"OPTS"
    elif damage == "unknown_section":
        b[12:16] = struct.pack("<I", 7)
        b += section(b"ZZZZ", b"12345678")
    p = tmp_path / "m.strom"
    p.write_bytes(bytes(b))
    with pytest.raises(st.StError) as e:
        st.st_model_file_info(str(p))
    assert e.value.code == st.ST_ERR_ARG


def test_missing_file(st, tmp_path):
    with pytest.raises(st.StError) as e:
        st.st_model_file_info(str(tmp_path / "absent.strom"))
    assert e.value.code == st.ST_ERR_ARG
