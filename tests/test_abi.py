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


def test_ctx_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lib.RSError) as ei:
        lib.rs_ctx_create(0)
    assert ei.value.status == lib.RS_ERR_CUDA
