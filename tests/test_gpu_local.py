"""Local-box handles (scheme C of Sec. 3.2) on the GPU: energies and gradients against
the oracle's local model, against the global handle within the truncation bound, the
box flags, ranks, and the handle family's lifetime."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.parity import E_TOL, assert_energies, assert_flags, assert_gradients, away_from_planes

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


def _box_poses(w, c, spread, P, seed):
    rng = np.random.default_rng(seed)
    quat = W.shoemake_quaternions(rng, P)
    trans = c + rng.uniform(-spread, spread, size=(P, 3))
    return quat, trans


@pytest.fixture(scope="module", params=["small", "protein"])
def case(request, L, ctx):
    if request.param == "small":
        w = W.plain_small(P=1)
        cap, c, half = 12, np.array([22.0, 3.0, -2.0]), 9.0
    else:
        w = W.plain_protein(P=1)
        cap, c, half = 20, np.array([4.0, -3.0, 21.0]), 13.0
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l, tucker_cap=cap)
    prot = L.Protein(ctx, w.prot_xyz, w.prot_q,
                     L.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=cap))
    # translations keep every ligand atom inside the box
    spread = half - np.linalg.norm(w.lig_xyz - w.lig_xyz.mean(axis=0), axis=1).max() - 0.5
    yield w, m, prot, c, half, spread
    prot.close()


def test_local_box_energies(L, case):
    w, m, prot, c, half, spread = case
    lo, hi = c - half, c + half
    loc = prot.local_box(lo, hi, eps=1e-7)
    lm = O.local_box_model(m, lo, hi, eps=1e-7)
    try:
        print("local ranks gpu", loc.info["rank"], "oracle", lm.ranks, "global", prot.info["rank"])
        assert max(loc.info["rank"][:2]) <= 32
        # poses inside the box (ligand radius < spread margin) and a few outside it
        quat, trans = _box_poses(w, c, spread, 3000, 7)
        trans[:50] += np.array([half + 2.0, 0.0, 0.0])
        E, f = loc.energies(w.lig_xyz, w.lig_q, quat, trans)
        ref = O.pose_energies(lm, w.lig_xyz, w.lig_q, quat, trans)
        assert_flags(f, ref)
        assert np.all(np.asarray(f)[:50] & O.FLAG_OUT_OF_GRID)
        inside = (np.asarray(f) & O.FLAG_OUT_OF_GRID) == 0
        assert inside.sum() == 2950
        err = np.abs(np.asarray(E) - ref["E"])[inside] / O.tolerance_scale(ref["E"], ref["S_ref"])[inside]
        assert err.max() <= E_TOL, err.max()
        # against the global handle: within the truncation bound sum_j |q_j| x bound
        Eg, fg = prot.energies(w.lig_xyz, w.lig_q, quat, trans)
        bound = np.abs(w.lig_q).sum() * lm.trunc_bound
        d = np.abs(np.asarray(E) - np.asarray(Eg))[inside]
        scale = O.tolerance_scale(ref["E"], ref["S_ref"])[inside]
        assert np.all(d <= 4 * bound + E_TOL * scale), (d.max(), bound)
        print("local vs global: max |dE|", float(d.max()), "bound", bound)
    finally:
        loc.close()


def test_local_box_gradients(L, case):
    w, m, prot, c, half, spread = case
    lo, hi = c - half, c + half
    loc = prot.local_box(lo, hi, eps=1e-7)
    lm = O.local_box_model(m, lo, hi, eps=1e-7)
    try:
        rng = np.random.default_rng(9)
        rv = W.random_rotvecs(rng, 600)
        tr = c + rng.uniform(-spread, spread, size=(600, 3))
        E, gt, gw, f = loc.energies_grad(w.lig_xyz, w.lig_q, rv, tr)
        ref = O.pose_gradients(lm, w.lig_xyz, w.lig_q, rv, tr)
        keep = away_from_planes(lm, w.lig_xyz, O.rotvec_to_rot(rv), tr)
        assert_energies(E, ref)
        assert_flags(f, ref)
        assert_gradients(gt, gw, ref, keep)
    finally:
        loc.close()


def test_local_box_lifetime_and_errors(L, ctx, case):
    w, m, prot, c, half, spread = case
    # the parent may be freed first: the local handle keeps its short-range data
    parent = L.Protein(ctx, w.prot_xyz, w.prot_q, L.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l,
                                                                        tucker_cap=12))
    loc = parent.local_box(c - half, c + half)
    quat, trans = _box_poses(w, c, spread, 200, 3)
    E0, _ = loc.energies(w.lig_xyz, w.lig_q, quat, trans)
    parent.close()
    E1, _ = loc.energies(w.lig_xyz, w.lig_q, quat, trans)
    assert np.array_equal(np.asarray(E0), np.asarray(E1))
    with pytest.raises(L.RSError) as e:
        loc.local_box(c - 1.0, c + 1.0)
    assert e.value.status == L.RS_ERR_INVALID
    loc.close()
    for lo, hi, eps in ((c + 1.0, c - 1.0, 1e-7), (c - 1.0, c + 1.0, 1.5)):
        with pytest.raises(L.RSError) as e:
            prot.local_box(lo, hi, eps=eps)
        assert e.value.status == L.RS_ERR_INVALID
    canon = L.Protein(ctx, w.prot_xyz[:50], w.prot_q[:50],
                      L.rs_params_default(n=129, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=0))
    try:
        with pytest.raises(L.RSError) as e:
            canon.local_box(c - 2.0, c + 2.0)
        assert e.value.status == L.RS_ERR_INVALID
    finally:
        canon.close()
