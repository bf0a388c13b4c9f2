"""The no-allocation variant of the pose-energy call.

rs_energy_poses_noalloc exists for callers that may not cause device memory
allocation while they run, such as a service thread that must never hit
cudaMalloc/cudaFree (both can synchronise the device) or a plug-in whose host
application owns all GPU memory.  It must give the same energies and flags as
rs_energy_poses.  This file is collected last, and each test builds its own
context and protein, so it passes alone in a fresh process as well as after the
other tests.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cap", [0, 8])
def test_noalloc_matches_rs_energy_poses_on_two_calls(cap):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_26611_gb300 import lib
    ctx = lib.Context(0)
    w = W.plain_small(P=500)
    params = lib.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=cap)
    prot = lib.Protein(ctx, w.prot_xyz, w.prot_q, params)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    # two calls in a row with different ligands and pose counts: the shared scratch
    # keeps the previous call's contents and must be rewritten correctly
    lig2 = w.lig_xyz[:7] * 0.8
    calls = [(w.lig_xyz, w.lig_q, w.quat, w.trans),
             (lig2, w.lig_q[:7], w.quat[:333], w.trans[:333] * 1.1)]
    for lx, lq, qu, tr in calls:
        E_ref, f_ref = prot.energies(T(lx), T(lq), T(qu), T(tr))
        free0 = torch.cuda.mem_get_info()[0]
        E, f = lib.rs_energy_poses_noalloc(prot.handle, T(lx), T(lq), T(qu), T(tr))
        torch.cuda.synchronize()
        E, f, E_ref, f_ref = E.cpu().numpy(), f.cpu().numpy(), E_ref.cpu().numpy(), f_ref.cpu().numpy()
        # same per-block kernel and summation order as rs_energy_poses at this size
        assert np.array_equal(E, E_ref)
        assert np.array_equal(f, f_ref)
    # after the first call on the device, a call leaves free device memory unchanged
    free1 = torch.cuda.mem_get_info()[0]
    E, f = lib.rs_energy_poses_noalloc(prot.handle, T(w.lig_xyz), T(w.lig_q), T(w.quat), T(w.trans))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free1
    prot.close()
    ctx.close()


def test_noalloc_rejects_ligands_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_26611_gb300 import lib
    ctx = lib.Context(0)
    w = W.plain_small(P=4)
    prot = lib.Protein(ctx, w.prot_xyz, w.prot_q,
                       lib.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l))
    big = torch.zeros((4097, 3), dtype=torch.float64, device="cuda")
    q = torch.zeros(4097, dtype=torch.float64, device="cuda")
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    with pytest.raises(lib.RSError) as ei:
        lib.rs_energy_poses_noalloc(prot.handle, big, q, T(w.quat), T(w.trans))
    assert ei.value.status == lib.RS_ERR_UNSUPPORTED
    assert "4096" in lib.rs_last_error()
    prot.close()
    ctx.close()


def test_noalloc_refuses_host_buffers_before_launching():
    """A host array passed straight through the C ABI is refused with
    RS_ERR_INVALID: the check runs on the host, so no kernel ever sees the pointer."""
    import ctypes
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_26611_gb300 import lib
    ctx = lib.Context(0)
    w = W.plain_small(P=8)
    prot = lib.Protein(ctx, w.prot_xyz, w.prot_q,
                       lib.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l))
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    lx, lq, qu, tr = T(w.lig_xyz), T(w.lig_q), T(w.quat), T(w.trans)
    E = torch.empty(w.P, dtype=torch.float64, device="cuda")
    f = torch.empty(w.P, dtype=torch.uint8, device="cuda")
    host_xyz = np.ascontiguousarray(w.lig_xyz)
    host_E = np.zeros(w.P)
    launches0 = lib.rs_stats_kernel_launches()
    for args in ((host_xyz.ctypes.data, lq.data_ptr(), E.data_ptr()),
                 (lx.data_ptr(), lq.data_ptr(), host_E.ctypes.data)):
        st = lib._lib.rs_energy_poses_noalloc(prot.handle, w.L, args[0], args[1], w.P,
                                              qu.data_ptr(), tr.data_ptr(), args[2],
                                              f.data_ptr(), ctypes.c_void_p(0))
        assert st == lib.RS_ERR_INVALID
        assert "device memory" in lib.rs_last_error()
    assert lib.rs_stats_kernel_launches() == launches0
    # the context is still usable afterwards
    E2, f2 = lib.rs_energy_poses_noalloc(prot.handle, lx, lq, qu, tr)
    E1, f1 = prot.energies(lx, lq, qu, tr)
    torch.cuda.synchronize()
    assert np.array_equal(E2.cpu().numpy(), E1.cpu().numpy())
    prot.close()
    ctx.close()
