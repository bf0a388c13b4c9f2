"""The Tucker build's block products G Q on the tensor cores (six exact BF16 slices,
exact FP32 sums per K chunk) against the float-pair GEMM on the FP32 pipes: same
ranks, the same singular-value gaps and tails, and energies that agree far inside
the parity tolerance; and the tensor-core build against the oracle's RHOSVD."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.parity import assert_energies, assert_flags, path_errors

pytestmark = pytest.mark.gpu


def _build_both(lib, ctx, w, cap):
    prm = lib.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=cap)
    out = {}
    for mode in (1, 0):
        old = lib.rs_set_build_gemm_kernel(mode)
        try:
            pr = lib.Protein(ctx, w.prot_xyz, w.prot_q, prm)
        finally:
            lib.rs_set_build_gemm_kernel(old)
        E, f = pr.energies(w.lig_xyz, w.lig_q, w.quat, w.trans)
        out[mode] = (pr.info, np.asarray(E), np.asarray(f))
        pr.close()
    return out


# block sizes of the subspace iteration: cap 4 -> 16, cap 12 and 20 -> 32, cap 32 -> 48
@pytest.mark.parametrize("kind,cap", [("small", 4), ("small", 12), ("small", 32), ("protein", 20)])
def test_tensor_core_gram_products_match_float_pairs(kind, cap):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_26611_gb300 import lib
    ctx = lib.Context(0)
    try:
        w = W.plain_small(P=2000) if kind == "small" else W.plain_protein(P=3000)
        out = _build_both(lib, ctx, w, cap)
    finally:
        ctx.close()
    (i1, E1, f1), (i0, E0, f0) = out[1], out[0]
    assert list(i1["rank"]) == list(i0["rank"])
    for a in range(3):
        assert abs(i1["sv_gap"][a] - i0["sv_gap"][a]) <= 1e-8 * abs(i0["sv_gap"][a])
        assert abs(i1["sv_tail"][a] - i0["sv_tail"][a]) <= 1e-8 * abs(i0["sv_tail"][a]) + 1e-300
    assert np.array_equal(f1, f0)
    err = path_errors(E1, E0)
    assert err.max() <= 1e-9, f"tensor-core vs float-pair build: {err.max():.3e}"


def test_tensor_core_build_matches_oracle_at_grid_4097():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_26611_gb300 import lib
    rng = np.random.default_rng(4097)
    prot, r_p = W.sphere_lattice(rng, 400)
    zq = W.mixed_charges(rng, 400, 0.3, 0.08)
    L, r_l = 30, 5.0 * (30 / 20.0) ** (1.0 / 3.0)
    lig = W.ball_uniform(rng, L, r_l)
    lq = rng.normal(0.0, 0.3, L)
    P = 600
    quat = W.shoemake_quaternions(rng, P)
    trans = W.shell_translations(rng, P, r_p, r_p + 2 * r_l + 3)
    b = r_p + 2 * r_l + 8
    ctx = lib.Context(0)
    try:
        pr = lib.Protein(ctx, prot, zq, lib.rs_params_default(n=4097, b=b, sigma=3.0, R_l=20, tucker_cap=20))
        E, f = pr.energies(lig, lq, quat, trans)
        info = pr.info
        pr.close()
    finally:
        ctx.close()
    m = O.build_model(prot, zq, 4097, b, 3.0, 20, tucker_cap=20)
    assert [v.shape[1] for v in m.V] == list(info["rank"])
    ref = O.pose_energies(m, lig, lq, quat, trans)
    assert_energies(np.asarray(E), ref)
    assert_flags(np.asarray(f), ref)


def test_rank_deficient_gram_builds_in_both_modes():
    """One protein charge: each axis Gram has rank R_l = 8 below the block size 16, so
    the block's Gram matrices are singular; the shifted Cholesky still orthonormalises
    and both GEMMs give the oracle's energies."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_26611_gb300 import lib
    xyz, q = np.zeros((1, 3)), np.array([1.0])
    prm = lib.rs_params_default(n=33, b=8.0, sigma=1.0, R_l=8, tucker_cap=4)
    m = O.build_model(xyz, q, 33, 8.0, 1.0, 8, tucker_cap=4)
    lig = np.array([[0.5, 0.0, 0.0], [-0.5, 0.2, 0.0]])
    lq = np.array([0.3, -0.3])
    rng = np.random.default_rng(3)
    quat = W.shoemake_quaternions(rng, 64)
    trans = W.shell_translations(rng, 64, 2.0, 6.0)
    ref = O.pose_energies(m, lig, lq, quat, trans)
    ctx = lib.Context(0)
    try:
        for mode in (1, 0):
            old = lib.rs_set_build_gemm_kernel(mode)
            try:
                pr = lib.Protein(ctx, xyz, q, prm)
            finally:
                lib.rs_set_build_gemm_kernel(old)
            E, f = pr.energies(lig, lq, quat, trans)
            assert list(pr.info["rank"]) == [v.shape[1] for v in m.V]
            pr.close()
            assert_energies(np.asarray(E), ref)
            assert_flags(np.asarray(f), ref)
    finally:
        ctx.close()


def test_narrow_gaussians_take_direct_values_in_the_projection():
    """A coarse grid (h = 0.5 A) and a small sigma (0.4 A): the two narrowest long-range
    terms have t^2 h^2 > 8, where the projection evaluates every Gaussian value by the
    pair exponential instead of the ratio recurrence.  Both build GEMMs against the
    oracle's RHOSVD."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_26611_gb300 import lib
    rng = np.random.default_rng(65)
    prot, r_p = W.sphere_lattice(rng, 60)
    zq = W.mixed_charges(rng, 60, 0.3, 0.08)
    lig = W.ball_uniform(rng, 12, 2.0)
    lq = rng.normal(0.0, 0.3, 12)
    P = 400
    quat = W.shoemake_quaternions(rng, P)
    trans = W.shell_translations(rng, P, r_p, r_p + 4.0)
    n, b, sigma, Rl, cap = 65, 16.0, 0.4, 14, 8
    tab = O.sinc_table(b, sigma, Rl)
    t_long = np.asarray(tab.t)[np.asarray(tab.is_long)]
    assert (t_long ** 2 * (2 * b / (n - 1)) ** 2 > 8.0).sum() >= 2
    m = O.build_model(prot, zq, n, b, sigma, Rl, tucker_cap=cap)
    ref = O.pose_energies(m, lig, lq, quat, trans)
    prm = lib.rs_params_default(n=n, b=b, sigma=sigma, R_l=Rl, tucker_cap=cap)
    ctx = lib.Context(0)
    try:
        for mode in (1, 0):
            old = lib.rs_set_build_gemm_kernel(mode)
            try:
                pr = lib.Protein(ctx, prot, zq, prm)
            finally:
                lib.rs_set_build_gemm_kernel(old)
            E, f = pr.energies(lig, lq, quat, trans)
            assert list(pr.info["rank"]) == [v.shape[1] for v in m.V]
            pr.close()
            assert_energies(np.asarray(E), ref)
            assert_flags(np.asarray(f), ref)
    finally:
        ctx.close()
