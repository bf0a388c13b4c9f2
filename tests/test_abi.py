"""The C-ABI library builds, loads and exports every symbol include/rs.h declares;
struct layouts agree between C and the ctypes binding.  No compute calls."""
import ctypes as C
import os
import subprocess

import pytest

from paper_2510_26611_gb300 import lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_header_symbol():
    syms = lib.header_symbols()
    assert len(syms) >= 11
    so = C.CDLL(lib.LIBRARY_PATH)
    missing = [s for s in syms if not hasattr(so, s)]
    assert not missing, missing


def test_params_default():
    p = lib.rs_params_default()
    assert (p.n, p.b, p.sigma, p.R_l, p.tucker_cap) == (257, 32.0, 3.0, 20, 0)
    assert p.r_min == 0.5 and p.tau == 4.0 and p.short_tol == 1e-9 and p.eps_r == 1e-7
    assert "sm_103a" in lib.rs_version()


def test_struct_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "rs.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(rs_params), offsetof(rs_params, b),
         offsetof(rs_params, tucker_cap), offsetof(rs_params, eps_r), sizeof(rs_protein_info));
  printf("%zu %zu %zu\n", offsetof(rs_protein_info, rank), offsetof(rs_protein_info, sv_tail),
         offsetof(rs_protein_info, device_bytes));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = list(map(int, out))
    P, I = lib.rs_params, lib.rs_protein_info
    want = [C.sizeof(P), P.b.offset, P.tucker_cap.offset, P.eps_r.offset, C.sizeof(I),
            I.rank.offset, I.sv_tail.offset, I.device_bytes.offset]
    assert got == want


def test_invalid_arguments_return_status_not_crash():
    # NULL context / protein are rejected before any device work
    st = lib._lib.rs_energy_poses(None, None, 1, None, None, 1, None, None, None, None, 0, None)
    assert st == lib.RS_ERR_INVALID
    assert "NULL" in lib.rs_last_error()
    out = C.c_void_p()
    st = lib._lib.rs_build_protein(None, 1, None, None, None, 0, None, C.byref(out))
    assert st == lib.RS_ERR_INVALID
    # add-and-compress: NULL context or part list, before any device work
    out = C.c_void_p(1)
    parts = (C.c_void_p * 1)(None)
    assert lib._lib.rs_protein_add_compress(None, parts, 1, 8, 1e-7, None, C.byref(out)) == lib.RS_ERR_INVALID
    assert lib._lib.rs_protein_add_compress(None, None, 0, 8, 1e-7, None, C.byref(out)) == lib.RS_ERR_INVALID
    assert lib._lib.rs_protein_add_compress(None, parts, 1, 8, 1e-7, None, None) == lib.RS_ERR_INVALID
    assert "NULL" in lib.rs_last_error()
    # batches and local boxes: NULL context
    assert lib._lib.rs_batch_create(None, 1, None, 1, C.byref(out)) == lib.RS_ERR_INVALID
    assert lib._lib.rs_protein_local_box(None, None, None, None, 1e-7, C.byref(out)) == lib.RS_ERR_INVALID


def test_ctx_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lib.RSError) as ei:
        lib.rs_ctx_create(0)
    assert ei.value.status == lib.RS_ERR_CUDA


def test_serving_struct_layout_matches_c(tmp_path):
    src = tmp_path / "serve_layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "rs.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(rs_request), offsetof(rs_request, params),
         offsetof(rs_request, L), offsetof(rs_request, P), offsetof(rs_request, trans),
         sizeof(rs_result));
  printf("%zu %zu %zu %zu %zu %zu\n", offsetof(rs_result, message), sizeof(rs_serve_params),
         offsetof(rs_serve_params, inject_alloc_failures), offsetof(rs_serve_params, hold_builds),
         sizeof(rs_serve_stats), offsetof(rs_serve_stats, mean_requests_per_launch));
  printf("%zu %zu %zu %zu\n", sizeof(rs_batch_info), offsetof(rs_batch_info, chunk_atoms),
         offsetof(rs_batch_info, nchunks), offsetof(rs_batch_info, streams));
  return 0;
}
''')
    exe = tmp_path / "serve_layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                       check=True).stdout.split()))
    R, Z, S, T = lib.rs_request, lib.rs_result, lib.rs_serve_params, lib.rs_serve_stats
    B = lib.rs_batch_info
    want = [C.sizeof(R), R.params.offset, R.L.offset, R.P.offset, R.trans.offset, C.sizeof(Z),
            Z.message.offset, C.sizeof(S), S.inject_alloc_failures.offset, S.hold_builds.offset, C.sizeof(T),
            T.mean_requests_per_launch.offset, C.sizeof(B), B.chunk_atoms.offset, B.nchunks.offset, B.streams.offset]
    assert got == want


def _request(**kw):
    import numpy as np
    rng = np.random.default_rng(5)
    arrays = dict(prot_xyz=rng.normal(size=(10, 3)), prot_q=rng.normal(size=10),
                  lig_xyz=rng.normal(size=(4, 3)), lig_q=rng.normal(size=4),
                  quat=rng.normal(size=(3, 4)), trans=rng.normal(size=(3, 3)))
    req, keep = lib.make_request(7, params=lib.rs_params_default(), **arrays)
    for k, v in kw.items():
        setattr(req, k, v)
    return req, keep


def test_request_validation_without_gpu():
    req, keep = _request()
    assert lib.rs_request_validate(req) == lib.RS_OK
    for field, bad in [("L", 0), ("L", 5000), ("P", -1), ("N", 0), ("lig_xyz", None),
                       ("quat", None), ("prot_q", None)]:
        r, k = _request(**{field: bad})
        assert lib.rs_request_validate(r) == lib.RS_ERR_INVALID, field
        assert lib.rs_last_error()
    r, k = _request()
    r.params.n = 20000
    assert lib.rs_request_validate(r) == lib.RS_ERR_INVALID
    r, k = _request()
    r.params.tucker_cap = 33
    assert lib.rs_request_validate(r) == lib.RS_ERR_INVALID
    # no poses: pose pointers may be NULL
    r, k = _request(P=0, quat=None, trans=None)
    assert lib.rs_request_validate(r) == lib.RS_OK
    assert lib.rs_request_validate(None) == lib.RS_ERR_INVALID


def test_serve_params_default_and_argument_checks():
    p = lib.rs_serve_params_default()
    assert p.mem_budget_bytes == 0 and p.max_inflight_launches == 2 and p.max_queue == 65536
    assert p.inject_alloc_failures == 0
    out = C.c_void_p()
    bad = lib.rs_serve_params_default(max_inflight_launches=0)
    assert lib._lib.rs_serve_create(0, C.byref(bad), C.byref(out)) == lib.RS_ERR_INVALID
    bad = lib.rs_serve_params_default(inject_alloc_failures=-1)
    assert lib._lib.rs_serve_create(0, C.byref(bad), C.byref(out)) == lib.RS_ERR_INVALID
    rid = C.c_uint64()
    req, keep = _request()
    assert lib._lib.rs_serve_submit(None, C.byref(req), None, None, C.byref(rid)) == lib.RS_ERR_INVALID
    assert lib._lib.rs_serve_poll(None, 1, None) == lib.RS_ERR_INVALID
    assert lib._lib.rs_serve_cancel(None, 1) == lib.RS_ERR_INVALID
    lib._lib.rs_serve_destroy(None)  # no-op


def test_serve_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lib.RSError) as ei:
        lib.rs_serve_create(0)
    assert ei.value.status == lib.RS_ERR_CUDA
