"""The paper's finite-difference force (Eq. differ_ligand) and rigid-cluster
resultants (Eq. Field_Xcenter, Eq. Field_phi) on the GPU against the FP64 oracle,
host and device buffers, several chunks, and argument checks."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.parity import E_TOL, G_TOL, assert_energies, assert_flags

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_26611_gb300 import lib
    return lib


@pytest.fixture(scope="module")
def ctx(L):
    c = L.Context(0)
    yield c
    c.close()


def assert_fd(out, ref, tol=G_TOL):
    """Every resultant per pose within tol of max(|ref|, 1e-2 x the per-atom scale)."""
    assert_energies(np.asarray(out["E"]), ref)
    assert_flags(np.asarray(out["flags"]), ref)
    worst = {}
    for k, rk, sk in (("F", "Fsum", "T_ref"), ("F0", "F0", "T_ref"), ("Fphi", "Fphi", "T_ref"),
                      ("M", "M", "W_ref")):
        a = np.asarray(out[k])
        sc = np.maximum(np.maximum(np.linalg.norm(ref[rk], axis=1), 1e-2 * ref[sk]), 1e-300)
        e = np.abs(a - ref[rk]).max(axis=1) / sc
        worst[k] = float(e.max())
        assert e.max() <= tol, (k, float(e.max()), int(np.argmax(e)))
    return worst


@pytest.fixture(scope="module")
def small(L, ctx):
    w = W.plain_small(P=256)
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l, tucker_cap=12)
    prot = L.Protein(ctx, w.prot_xyz, w.prot_q,
                     L.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=12))
    rv = W.random_rotvecs(np.random.default_rng(41), w.P)
    yield w, m, prot, rv
    prot.close()


def test_fd_small_matches_oracle(L, small):
    w, m, prot, rv = small
    out = prot.fd_forces(w.lig_xyz, w.lig_q, rv, w.trans)
    ref = O.fd_forces(m, w.lig_xyz, w.lig_q, rv, w.trans)
    print("fd small worst:", assert_fd(out, ref))


def test_fd_step_and_radius_arguments(L, small):
    w, m, prot, rv = small
    h, r0 = 0.05, 2.5
    out = prot.fd_forces(w.lig_xyz, w.lig_q, rv[:64], w.trans[:64], h=h, r0=r0)
    ref = O.fd_forces(m, w.lig_xyz, w.lig_q, rv[:64], w.trans[:64], h=h, r0=r0)
    assert_fd(out, ref)


def test_fd_device_buffers_equal_host(L, ctx, small):
    import torch
    w, m, prot, rv = small
    a = prot.fd_forces(w.lig_xyz, w.lig_q, rv, w.trans)
    T = lambda x: torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    b = prot.fd_forces(T(w.lig_xyz), T(w.lig_q), T(rv), T(w.trans))
    torch.cuda.synchronize()
    for k in ("E", "F", "F0", "Fphi", "M", "flags"):
        assert np.array_equal(np.asarray(a[k]), b[k].cpu().numpy()), k


def test_fd_single_atom_ligand(L, small):
    # one atom: it sits at the centre, so F0 = F, Fphi = 0 and M = 0
    w, m, prot, rv = small
    lig, q = w.lig_xyz[:1], w.lig_q[:1]
    out = prot.fd_forces(lig, q, rv[:32], w.trans[:32])
    ref = O.fd_forces(m, lig, q, rv[:32], w.trans[:32])
    assert_fd(out, ref)
    assert np.array_equal(out["F0"], out["F"])
    assert np.all(out["Fphi"] == 0.0) and np.all(out["M"] == 0.0)


def test_fd_empty_and_argument_errors(L, ctx, small):
    w, m, prot, rv = small
    out = prot.fd_forces(w.lig_xyz, w.lig_q, rv[:0], w.trans[:0])
    assert out["E"].shape == (0,)
    for kw in ({"h": -1.0}, {"r0": -0.5}, {"h": float("nan")}):
        with pytest.raises(L.RSError) as e:
            prot.fd_forces(w.lig_xyz, w.lig_q, rv[:4], w.trans[:4], **kw)
        assert e.value.status == L.RS_ERR_INVALID


def test_fd_needs_tucker_protein(L, ctx):
    w = W.plain_small(P=4)
    prot = L.Protein(ctx, w.prot_xyz, w.prot_q,
                     L.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=0))
    try:
        with pytest.raises(L.RSError) as e:
            prot.fd_forces(w.lig_xyz, w.lig_q, np.zeros((4, 3)), w.trans)
        assert e.value.status == L.RS_ERR_UNSUPPORTED
    finally:
        prot.close()


@pytest.fixture(scope="module")
def protein(L, ctx):
    w = W.plain_protein(P=50_000)
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l, tucker_cap=20)
    prot = L.Protein(ctx, w.prot_xyz, w.prot_q,
                     L.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=w.tucker_cap))
    rv = W.random_rotvecs(np.random.default_rng(43), w.P)
    yield w, m, prot, rv
    prot.close()


@pytest.mark.parametrize("mode", [1, 0], ids=["tensor-core", "float-pair"])
def test_fd_protein_matches_oracle(L, protein, mode):
    # 3000 poses x 4 evaluation poses x 50 atoms: the dense (tensor-core) W form when on
    w, m, prot, rv = protein
    P = 3000
    prev = L.rs_set_wform_kernel(mode)
    try:
        out = prot.fd_forces(w.lig_xyz, w.lig_q, rv[:P], w.trans[:P])
    finally:
        L.rs_set_wform_kernel(prev)
    ref = O.fd_forces(m, w.lig_xyz, w.lig_q, rv[:P], w.trans[:P])
    print("fd protein worst:", assert_fd(out, ref))
    assert L.rs_tc_error_count(0) == 0


def test_fd_several_chunks_sampled(L, protein):
    # 50 000 poses x 4 x 50 atoms = 1e7 evaluation atoms: two chunks of the
    # cell-grouped path; poses sampled across both and at the boundary
    w, m, prot, rv = protein
    out = prot.fd_forces(w.lig_xyz, w.lig_q, rv, w.trans)
    idx = np.unique(np.concatenate([np.arange(0, w.P, 197), np.arange(41_900, 42_100), [w.P - 1]]))
    ref = O.fd_forces(m, w.lig_xyz, w.lig_q, rv[idx], w.trans[idx])
    assert_fd({k: np.asarray(v)[idx] for k, v in out.items()}, ref)
