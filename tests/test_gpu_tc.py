"""Tensor-core W form: the BF16-sliced contraction of one tile against FP64 (exact for
8-bit inputs, within the slicing bound for random ones), and the cell-grouped pose
paths in tensor-core mode against float-pair mode and the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.parity import (assert_energies, assert_flags, assert_gradients, assert_paths_agree,
                          away_from_planes, path_errors)

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


@pytest.mark.parametrize("RP", [4, 12, 20, 32])
def test_contract_exact_for_8bit_integers(L, RP):
    # integers below 2^7 in magnitude take two slices exactly (top slice <= 32, then a
    # multiple of 2^-8); every product and partial sum is representable, so the
    # tensor-core result is exact
    rng = np.random.default_rng(RP)
    rows = 128
    v = rng.integers(-100, 101, size=(rows, RP)).astype(np.float64)
    v[:, 0] = 101.0  # every row's maximum in [64, 128): scale 1
    Wm = rng.integers(-100, 101, size=(RP, RP)).astype(np.float64)
    Dm = rng.integers(-100, 101, size=(RP, RP)).astype(np.float64)
    Wm[:, 0] = 127.0
    Dm[:, 0] = -90.0
    X, Xd = L.rs_diag_tc_contract(RP, v, Wm, Dm)
    assert np.array_equal(X, v @ Wm.T)
    assert np.array_equal(Xd, v @ Dm.T)


@pytest.mark.parametrize("RP,rows", [(4, 128), (20, 128), (20, 77), (20, 1), (32, 100)])
def test_contract_random_within_slicing_bound(L, RP, rows):
    rng = np.random.default_rng(1000 * RP + rows)
    v = rng.normal(size=(rows, RP)) * 10.0 ** rng.integers(-6, 7, size=(rows, 1))
    Wm = rng.normal(size=(RP, RP)) * 10.0 ** rng.integers(-4, 5, size=(RP, 1))
    Dm = rng.normal(size=(RP, RP)) * 1e-3
    if rows > 2:
        v[1] = 0.0
    X, Xd = L.rs_diag_tc_contract(RP, v, Wm, Dm)
    for out, B in ((X, Wm), (Xd, Dm)):
        ref = v @ B.T
        # the second accumulator's FP32 rounding and the dropped slice products
        # (i + j >= 5) leave ~2^-33 of K max max; an FP32-accumulated CPU emulation of
        # the scheme stays below 0.32 of this bound on these cases
        bound = 2.0 ** -31 * RP * np.abs(v).max(axis=1, keepdims=True) * np.abs(B).max(axis=1)[None, :]
        err = np.abs(out - ref)
        assert np.all(err <= bound), float((err / np.maximum(bound, 1e-300)).max())
        if rows > 2:
            assert np.all(out[1] == 0.0)
        # far better than FP32 in practice (the emulation: median 6e-4 .. 3e-3 of it)
        fp32 = (v.astype(np.float32) @ B.T.astype(np.float32)).astype(np.float64)
        assert np.median(err) < 2e-2 * max(np.median(np.abs(fp32 - ref)), 1e-300) or np.median(err) == 0.0


@pytest.fixture(scope="module")
def protein(L, ctx):
    w = W.plain_protein(P=20_000)
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l, tucker_cap=20)
    prm = L.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=w.tucker_cap)
    prot = L.Protein(ctx, w.prot_xyz, w.prot_q, prm)
    ref = O.pose_energies(m, w.lig_xyz, w.lig_q, w.quat, w.trans)
    yield w, m, prot, ref
    prot.close()


def _both_modes(L, fn):
    prev = L.rs_set_wform_kernel(1)
    try:
        a = fn()
        L.rs_set_wform_kernel(0)
        b = fn()
    finally:
        L.rs_set_wform_kernel(prev)
    return a, b


def test_sorted_energies_tc_vs_pairs_and_oracle(L, protein):
    w, m, prot, ref = protein
    assert w.P * w.L >= 1 << 17  # the cell-grouped path
    (E1, f1), (E0, f0) = _both_modes(L, lambda: prot.energies(w.lig_xyz, w.lig_q, w.quat, w.trans))
    assert_energies(E1, ref)
    assert_flags(f1, ref)
    err = assert_paths_agree(E1, E0, f1, f0)
    print(f"tensor-core vs float-pair energies: max {err.max():.2e}, median {np.median(err):.2e}")
    assert L.rs_tc_error_count(0) == 0


def test_sorted_tc_launch_fills_tmem(L, protein):
    # rank 20: two accumulators of 48 columns -> 128 TMEM columns per CTA, so four
    # CTAs per SM and a grid of four CTAs per SM for a large energy call
    import torch
    w, m, prot, _ = protein
    prot.energies(w.lig_xyz, w.lig_q, w.quat, w.trans)
    info = L.rs_diag_tc_launch()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    print("tensor-core launch:", info)
    assert info["per_sm"] == 4
    assert info["grid"] == 4 * sms


def test_sorted_gradients_tc_vs_pairs_and_oracle(L, protein):
    w, m, prot, _ = protein
    P = 4000
    rv = W.random_rotvecs(np.random.default_rng(31), P)
    tr = w.trans[:P]
    assert P * w.L >= 1 << 17
    (E1, gt1, gw1, f1), (E0, gt0, gw0, f0) = _both_modes(
        L, lambda: prot.energies_grad(w.lig_xyz, w.lig_q, rv, tr))
    ref = O.pose_gradients(m, w.lig_xyz, w.lig_q, rv, tr)
    keep = away_from_planes(m, w.lig_xyz, O.rotvec_to_rot(rv), tr)
    assert_energies(E1, ref)
    assert_flags(f1, ref)
    assert_gradients(gt1, gw1, ref, keep)
    assert_paths_agree(E1, E0, f1, f0)
    for a, b in ((gt1, gt0), (gw1, gw0)):
        a, b = np.asarray(a), np.asarray(b)
        scale = np.maximum(np.linalg.norm(b, axis=1), np.median(np.linalg.norm(b, axis=1)))
        e = np.abs(a - b).max(axis=1) / scale
        print(f"tensor-core vs float-pair gradients: max {e.max():.2e}")
        assert e.max() <= 1e-7
    assert L.rs_tc_error_count(0) == 0


def test_sorted_tc_deterministic_and_order_independent(L, protein):
    # a row's MMA result does not depend on the other rows of its tile
    w, m, prot, _ = protein
    E1, f1 = prot.energies(w.lig_xyz, w.lig_q, w.quat, w.trans)
    perm = np.random.default_rng(3).permutation(w.P)
    E2, f2 = prot.energies(w.lig_xyz, w.lig_q, w.quat[perm], w.trans[perm])
    assert np.array_equal(E2, E1[perm]) and np.array_equal(f2, f1[perm])


def test_grouped_batch_tc_vs_pairs(L, ctx, protein):
    import torch
    w, m, prot, ref = protein
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    cuts = [0, 3000, 3001, 11000, 20000]
    pairs = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        pairs.append(dict(prot=prot.handle, lig_xyz=T(w.lig_xyz), lig_q=T(w.lig_q), quat=T(w.quat[a:b]),
                          trans=T(w.trans[a:b]),
                          E_out=torch.empty(b - a, dtype=torch.float64, device="cuda"),
                          flags_out=torch.empty(b - a, dtype=torch.uint8, device="cuda")))

    def run():
        bt, keep = L.rs_batch_create(ctx.handle, pairs, autotune=0)
        try:
            assert L.rs_batch_get_info(bt)["mode"] == 1
            L.rs_batch_run(bt)
            torch.cuda.synchronize()
        finally:
            L.rs_batch_free(bt)
        return (np.concatenate([p["E_out"].cpu().numpy() for p in pairs]),
                np.concatenate([p["flags_out"].cpu().numpy() for p in pairs]))

    (E1, f1), (E0, f0) = _both_modes(L, run)
    assert_energies(E1, ref)
    assert_flags(f1, ref)
    assert_paths_agree(E1, E0, f1, f0)
    # the grouped and the single-pair tensor-core kernels give the same bits
    Ep, fp = prot.energies(w.lig_xyz, w.lig_q, w.quat, w.trans)
    assert np.array_equal(E1, Ep) and np.array_equal(f1, fp)
    assert L.rs_tc_error_count(0) == 0


def test_path_errors_helper_scale():
    # the path tolerance is taken against max(|E|, median |E|): a pose near zero energy
    # is judged on the batch's typical magnitude
    e = path_errors(np.array([1.0, 1e-12, -3.0]), np.array([1.0, 0.0, -3.0]))
    assert e[1] == pytest.approx(1e-12, rel=1e-9)


def test_pair_exponential_against_fp64(L):
    # the build's Gaussian seeds: exp of a float pair, ~2^-46 relative over the range
    # they use (exponents >= -50; below about -70 the low word of the result is an FP32
    # subnormal and the pair loses precision)
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.uniform(-60.0, 60.0, 20000), rng.uniform(-1e-3, 1e-3, 2000),
                        np.array([0.0, -50.0, 50.0, np.log(2.0), -np.log(2.0) / 512])])
    y = L.rs_diag_pair_exp(x)
    h = x.astype(np.float32).astype(np.float64)
    xp = h + (x - h).astype(np.float32).astype(np.float64)  # the float pair the kernel reads
    rel = np.abs(y - np.exp(xp)) / np.exp(xp)
    assert rel.max() < 2.0 ** -44, rel.max()
