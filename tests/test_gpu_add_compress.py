"""Add-and-compress on the GPU (Algorithm TEP step 4, Sec. 3.4; the complex of Eq.
EnergySum_Mcomplex as one Tucker tensor) against the oracle's add_and_compress: the
same ranks, energies and flags within the parity tolerance, the sum of the parts'
potentials within the truncation, and the argument checks."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.parity import assert_energies, assert_flags, assert_gradients, away_from_planes, path_errors

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


def _halves(w):
    """Two molecules: the protein's atoms split at the median x coordinate."""
    order = np.argsort(w.prot_xyz[:, 0], kind="stable")
    h = order.size // 2
    return [(w.prot_xyz[i], w.prot_q[i]) for i in (order[:h], order[h:])]


def _parts(L, ctx, w, cap):
    prm = L.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=cap)
    prots, models = [], []
    for xyz, q in _halves(w):
        prots.append(L.Protein(ctx, xyz, q, prm))
        models.append(O.build_model(xyz, q, w.n, w.b, w.sigma, w.R_l, tucker_cap=cap))
    return prots, models


@pytest.mark.parametrize("kind,cap_parts,cap", [("small", 12, 12), ("small", 8, 20), ("protein", 20, 20)])
def test_two_molecules_match_the_oracle(L, ctx, kind, cap_parts, cap):
    w = W.plain_small(P=2000) if kind == "small" else W.plain_protein(P=2000)
    prots, models = _parts(L, ctx, w, cap_parts)
    try:
        ac = L.Protein.add_compress(ctx, prots, cap)
        try:
            ref_m = O.add_and_compress(models, cap)
            assert list(ac.info["rank"]) == list(ref_m.ranks)
            assert ac.info["N"] == w.prot_xyz.shape[0] and ac.info["kind"] == 1
            E, f = ac.energies(w.lig_xyz, w.lig_q, w.quat, w.trans)
            ref = O.pose_energies(ref_m, w.lig_xyz, w.lig_q, w.quat, w.trans)
            assert_energies(np.asarray(E), ref)
            assert_flags(np.asarray(f), ref)
            # the complex computed molecule by molecule (the parts' sum, before truncation)
            Ec, fc = L.rs_energy_poses_complex(ctx.handle, [p.handle for p in prots], w.lig_xyz, w.lig_q, w.quat,
                                               w.trans)
            assert np.array_equal(np.asarray(f), np.asarray(fc))
            if ref_m.trunc_bound == 0.0:
                # nothing truncated: the same potential up to rounding
                err = path_errors(E, Ec).max()
                assert err <= 1e-8, f"compressed sum vs complex: {err:.3e}"
            else:
                # trilinear values are convex combinations of grid values, each within
                # the HOSVD bound on the Frobenius norm of the truncation
                dE = np.abs(np.asarray(E) - np.asarray(Ec))
                assert dE.max() <= np.abs(w.lig_q).sum() * ref_m.trunc_bound * (1 + 1e-6) + 1e-9 * np.abs(Ec).max()
        finally:
            ac.close()
    finally:
        for p in prots:
            p.close()


def test_three_molecules_one_given_twice(L, ctx):
    """Three parts, the first repeated (its columns add no direction to the stacked
    factors, so the QR meets exactly dependent columns), against the oracle."""
    w = W.plain_small(P=1500)
    order = np.argsort(w.prot_xyz[:, 1], kind="stable")
    thirds = np.array_split(order, 3)
    prm = L.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=8)
    prots, models = [], []
    try:
        for idx in (thirds[0], thirds[1], thirds[0]):
            prots.append(L.Protein(ctx, w.prot_xyz[idx], w.prot_q[idx], prm))
            models.append(O.build_model(w.prot_xyz[idx], w.prot_q[idx], w.n, w.b, w.sigma, w.R_l, tucker_cap=8))
        ac = L.Protein.add_compress(ctx, prots, 16)
        try:
            ref_m = O.add_and_compress(models, 16)
            assert list(ac.info["rank"]) == list(ref_m.ranks)
            assert ac.info["N"] == 2 * thirds[0].size + thirds[1].size
            E, f = ac.energies(w.lig_xyz, w.lig_q, w.quat, w.trans)
            ref = O.pose_energies(ref_m, w.lig_xyz, w.lig_q, w.quat, w.trans)
            assert_energies(np.asarray(E), ref)
            assert_flags(np.asarray(f), ref)
        finally:
            ac.close()
    finally:
        for p in prots:
            p.close()


def test_one_molecule_recompressed_to_a_lower_rank(L, ctx):
    w = W.plain_small(P=2000)
    prm = L.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=16)
    prot = L.Protein(ctx, w.prot_xyz, w.prot_q, prm)
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l, tucker_cap=16)
    try:
        for cap in (16, 6):
            ac = L.Protein.add_compress(ctx, [prot], cap)
            try:
                ref_m = O.add_and_compress([m], cap)
                assert list(ac.info["rank"]) == list(ref_m.ranks)
                E, f = ac.energies(w.lig_xyz, w.lig_q, w.quat, w.trans)
                ref = O.pose_energies(ref_m, w.lig_xyz, w.lig_q, w.quat, w.trans)
                assert_energies(np.asarray(E), ref)
                assert_flags(np.asarray(f), ref)
                if cap == 16:
                    # nothing to truncate: the parent's energies again
                    E0, f0 = prot.energies(w.lig_xyz, w.lig_q, w.quat, w.trans)
                    assert path_errors(E, E0).max() <= 1e-9
                    assert np.array_equal(np.asarray(f), np.asarray(f0))
            finally:
                ac.close()
    finally:
        prot.close()


def test_compressed_handle_serves_the_other_entry_points(L, ctx):
    """The handle is an ordinary Tucker protein: exact gradients against the oracle,
    and repeated calls give the same bits."""
    w = W.plain_small(P=1000)
    prots, models = _parts(L, ctx, w, 12)
    try:
        ac = L.Protein.add_compress(ctx, prots, 12)
        ref_m = O.add_and_compress(models, 12)
        try:
            rng = np.random.default_rng(9)
            rv = W.random_rotvecs(rng, 300)
            tr = w.trans[:300]
            E, gt, gw, f = ac.energies_grad(w.lig_xyz, w.lig_q, rv, tr)
            ref = O.pose_gradients(ref_m, w.lig_xyz, w.lig_q, rv, tr)
            keep = away_from_planes(ref_m, w.lig_xyz, O.rotvec_to_rot(rv), tr)
            assert_energies(E, ref)
            assert_flags(f, ref)
            assert_gradients(gt, gw, ref, keep)
            E, f = ac.energies(w.lig_xyz, w.lig_q, w.quat, w.trans)
            E2, f2 = ac.energies(w.lig_xyz, w.lig_q, w.quat, w.trans)
            assert np.array_equal(np.asarray(E), np.asarray(E2)) and np.array_equal(np.asarray(f), np.asarray(f2))
        finally:
            ac.close()
    finally:
        for p in prots:
            p.close()


def test_argument_checks(L, ctx):
    w = W.plain_small(P=10)
    (xa, qa), (xb, qb) = _halves(w)
    prm = L.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=8)
    a = L.Protein(ctx, xa, qa, prm)
    others = [L.Protein(ctx, xb, qb, L.rs_params_default(n=129, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=8)),
              L.Protein(ctx, xb, qb, L.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=0))]
    try:
        others.append(a.local_box(xa.mean(axis=0) - 2.0, xa.mean(axis=0) + 2.0))
        for o in others:
            with pytest.raises(L.RSError) as e:
                L.Protein.add_compress(ctx, [a, o], 8)
            assert e.value.status == L.RS_ERR_INVALID
        for cap, eps in ((0, 1e-7), (33, 1e-7), (8, 1.0), (8, -1e-3)):
            with pytest.raises(L.RSError) as e:
                L.Protein.add_compress(ctx, [a], cap, eps)
            assert e.value.status == L.RS_ERR_INVALID
        with pytest.raises(L.RSError) as e:
            L.rs_protein_add_compress(ctx.handle, [], 8)
        assert e.value.status == L.RS_ERR_INVALID
    finally:
        for o in reversed(others):
            o.close()
        a.close()
