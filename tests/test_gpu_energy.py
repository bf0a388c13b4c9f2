"""GPU parity: librs pose energies, flags and gradients against the FP64 oracle,
called through the C ABI (ctypes binding)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.parity import (assert_energies, assert_flags, assert_gradients, assert_topk,
                          away_from_planes)

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


def _params(L, w, cap=None, n=None):
    return L.rs_params_default(n=n or w.n, b=w.b, sigma=w.sigma, R_l=w.R_l,
                               tucker_cap=w.tucker_cap if cap is None else cap)


@pytest.fixture(scope="module")
def small(L, ctx):
    w = W.plain_small()
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l)
    prot = L.Protein(ctx, w.prot_xyz, w.prot_q, _params(L, w))
    ref = O.pose_energies(m, w.lig_xyz, w.lig_q, w.quat, w.trans)
    yield w, m, prot, ref
    prot.close()


@pytest.fixture(scope="module")
def small_tucker(L, ctx):
    w = W.plain_small()
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l, tucker_cap=12)
    prot = L.Protein(ctx, w.prot_xyz, w.prot_q, _params(L, w, cap=12))
    ref = O.pose_energies(m, w.lig_xyz, w.lig_q, w.quat, w.trans)
    yield w, m, prot, ref
    prot.close()


@pytest.fixture(scope="module")
def protein(L, ctx):
    w = W.plain_protein(P=100_000).subset(np.arange(3000))
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l, tucker_cap=20)
    prot = L.Protein(ctx, w.prot_xyz, w.prot_q, _params(L, w))
    ref = O.pose_energies(m, w.lig_xyz, w.lig_q, w.quat, w.trans)
    yield w, m, prot, ref
    prot.close()


# ------------------------------------------------------------------ canonical
def test_sinc_table_matches_oracle(L, small):
    w, m, prot, _ = small
    t, a, il = L.rs_protein_get_table(prot.handle)
    assert np.allclose(t, m.table.t, rtol=1e-14, atol=0)
    assert np.allclose(a, m.table.a, rtol=1e-14, atol=0)
    assert np.array_equal(il, m.table.is_long)
    assert abs(prot.info["r_c"] - m.table.r_c) < 1e-9
    assert prot.info["kind"] == 0 and prot.info["rank"][0] == w.N * w.R_l


def test_canonical_energies_flags_topk(L, small):
    w, m, prot, ref = small
    E, f = prot.energies(w.lig_xyz, w.lig_q, w.quat, w.trans)
    assert_energies(E, ref)
    assert_flags(f, ref)
    assert_topk(E, f, ref)
    assert 0 < (f == 0).sum() < w.P


def test_canonical_gradients(L, small):
    w, m, prot, _ = small
    rv = W.random_rotvecs(np.random.default_rng(11), 300)
    tr = w.trans[:300]
    ref = O.pose_gradients(m, w.lig_xyz, w.lig_q, rv, tr)
    E, gt, gw, f = prot.energies_grad(w.lig_xyz, w.lig_q, rv, tr)
    keep = away_from_planes(m, w.lig_xyz, O.rotvec_to_rot(rv), tr)
    assert keep.sum() > 250
    assert_energies(E, ref)
    assert_flags(f, ref)
    assert_gradients(gt, gw, ref, keep)


# ------------------------------------------------------------------ Tucker
def test_tucker_small_energies(L, small_tucker):
    w, m, prot, ref = small_tucker
    assert prot.info["kind"] == 1 and prot.info["rank"] == list(m.ranks)
    E, f = prot.energies(w.lig_xyz, w.lig_q, w.quat, w.trans)
    assert_energies(E, ref)
    assert_flags(f, ref)
    assert_topk(E, f, ref)


def test_tucker_small_gradients(L, small_tucker):
    w, m, prot, _ = small_tucker
    rv = W.random_rotvecs(np.random.default_rng(12), 300)
    tr = w.trans[300:600]
    ref = O.pose_gradients(m, w.lig_xyz, w.lig_q, rv, tr)
    E, gt, gw, f = prot.energies_grad(w.lig_xyz, w.lig_q, rv, tr)
    keep = away_from_planes(m, w.lig_xyz, O.rotvec_to_rot(rv), tr)
    assert_energies(E, ref)
    assert_gradients(gt, gw, ref, keep)


def test_tucker_protein_energies(L, protein):
    w, m, prot, ref = protein
    info = prot.info
    assert info["rank"] == [20, 20, 20]
    # singular-value diagnostics agree with the oracle's SVD
    for ax in range(3):
        s = m.svals[ax]
        assert abs(info["sv_gap"][ax] - s[19] / s[20]) < 1e-6 * s[19] / s[20]
        assert abs(info["sv_tail"][ax] - np.sqrt((s[20:] ** 2).sum()) / s[0]) < 1e-6
    E, f = prot.energies(w.lig_xyz, w.lig_q, w.quat, w.trans)
    assert_energies(E, ref)
    assert_flags(f, ref)
    assert_topk(E, f, ref)


def test_tucker_protein_gradients(L, protein):
    w, m, prot, _ = protein
    rv = W.random_rotvecs(np.random.default_rng(13), 500)
    tr = w.trans[:500]
    ref = O.pose_gradients(m, w.lig_xyz, w.lig_q, rv, tr)
    E, gt, gw, f = prot.energies_grad(w.lig_xyz, w.lig_q, rv, tr)
    keep = away_from_planes(m, w.lig_xyz, O.rotvec_to_rot(rv), tr)
    assert_energies(E, ref)
    assert_flags(f, ref)
    assert_gradients(gt, gw, ref, keep)


# ------------------------------------------------------------------ invariances
def test_host_and_device_modes_bitwise_equal(L, small):
    import torch
    w, m, prot, _ = small
    E_h, f_h = prot.energies(w.lig_xyz, w.lig_q, w.quat, w.trans)
    t = lambda a: torch.as_tensor(a, device="cuda")
    # results read right after the call: the call must be ordered on torch's stream
    E_d, f_d = prot.energies(t(w.lig_xyz), t(w.lig_q), t(w.quat), t(w.trans))
    assert np.array_equal(E_h, E_d.cpu().numpy())
    assert np.array_equal(f_h, f_d.cpu().numpy())


def test_device_call_on_a_side_stream(L, small):
    import torch
    w, m, prot, _ = small
    E_h, f_h = prot.energies(w.lig_xyz, w.lig_q, w.quat, w.trans)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        t = lambda a: torch.as_tensor(a, device="cuda")
        E_d, f_d = prot.energies(t(w.lig_xyz), t(w.lig_q), t(w.quat), t(w.trans))
        out = E_d.cpu().numpy(), f_d.cpu().numpy()
    assert np.array_equal(E_h, out[0]) and np.array_equal(f_h, out[1])


def test_deterministic_and_order_independent(L, protein):
    w, m, prot, _ = protein
    E1, f1 = prot.energies(w.lig_xyz, w.lig_q, w.quat, w.trans)
    E2, f2 = prot.energies(w.lig_xyz, w.lig_q, w.quat, w.trans)
    assert np.array_equal(E1, E2) and np.array_equal(f1, f2)
    perm = np.random.default_rng(0).permutation(w.P)
    E3, f3 = prot.energies(w.lig_xyz, w.lig_q, w.quat[perm], w.trans[perm])
    assert np.array_equal(E3, E1[perm]) and np.array_equal(f3, f1[perm])


def test_rebuild_is_bitwise_reproducible(L, ctx, small_tucker):
    w, m, prot, _ = small_tucker
    prot2 = L.Protein(ctx, w.prot_xyz, w.prot_q, _params(L, w, cap=12))
    a, _ = prot.energies(w.lig_xyz, w.lig_q, w.quat[:200], w.trans[:200])
    b, _ = prot2.energies(w.lig_xyz, w.lig_q, w.quat[:200], w.trans[:200])
    prot2.close()
    assert np.array_equal(a, b)


# ------------------------------------------------------------------ edge cases
def test_empty_single_and_ragged_batches(L, small):
    w, m, prot, ref = small
    E0, f0 = prot.energies(w.lig_xyz, w.lig_q, w.quat[:0], w.trans[:0])
    assert E0.shape == (0,)
    for P in (1, 7, 26, 999):
        E, f = prot.energies(w.lig_xyz, w.lig_q, w.quat[:P], w.trans[:P])
        sub = {k: v[:P] for k, v in ref.items()}
        assert_energies(E, sub)
        assert_flags(f, sub)


def test_single_atom_ligand_and_out_of_grid(L, small):
    w, m, prot, _ = small
    lig = np.array([[0.3, -0.2, 0.1]])
    q = np.array([0.7])
    trans = np.array([[25.0, 0, 0], [0, 0, 40.0], [31.999, 0.5, 0.5], [-32.0, 0, 0], [1e6, 0, 0]])
    quat = np.tile([1.0, 0, 0, 0], (5, 1))
    ref = O.pose_energies(m, lig, q, quat, trans)
    E, f = prot.energies(lig, q, quat, trans)
    assert_energies(E, ref)
    assert_flags(f, ref)
    assert f[1] & L.RS_FLAG_OUT_OF_GRID and f[4] & L.RS_FLAG_OUT_OF_GRID
    assert not (f[2] & L.RS_FLAG_OUT_OF_GRID)


def test_clash_boundary_decided_in_fp64(L, small):
    """Ligand atom placed at distance sigma*(1 +- 1e-9) from a protein atom: the
    vdW decision matches the FP64 oracle exactly."""
    w, m, prot, _ = small
    a = w.prot_xyz[np.argmax(np.linalg.norm(w.prot_xyz, axis=1))]
    d = a / np.linalg.norm(a)
    lig = np.array([[0.0, 0.0, 0.0]])
    q = np.array([1.0])
    trans = np.stack([a + d * w.sigma * (1 + e) for e in (-1e-9, 1e-9, -1e-6, 1e-6, 0.0)])
    quat = np.tile([1.0, 0, 0, 0], (len(trans), 1))
    ref = O.pose_energies(m, lig, q, quat, trans)
    E, f = prot.energies(lig, q, quat, trans)
    assert_flags(f, ref)
    assert f[0] & 1 and not (f[1] & 1)


def test_edge_cases_through_the_cell_grouped_path(L, small_tucker):
    """A single-atom ligand in 2^17 + 10 poses, so the call takes the cell-grouped path
    with the tensor-core W form (sort keys, records at their sorted positions): random
    placements plus atoms outside the grid beyond each kind of face, far away, just
    inside a face, on a face, and at sigma (1 +- 1e-9) and (1 +- 1e-6) from the outermost
    protein atom; every flag and energy against the oracle."""
    w, m, prot, _ = small_tucker
    rng = np.random.default_rng(17)
    P0 = (1 << 17) + 10
    trans = rng.uniform(-0.9 * w.b, 0.9 * w.b, (P0, 3))
    a = w.prot_xyz[np.argmax(np.linalg.norm(w.prot_xyz, axis=1))]
    d = a / np.linalg.norm(a)
    edge = [[w.b + 8.0, 0.0, 0.0], [0.0, -(w.b + 8.0), 0.0], [0.0, 0.0, w.b + 1e-3], [1e6, 0.0, 0.0],
            [w.b - 1e-3, 0.5, 0.5], [-w.b, 0.0, 0.0]]
    edge += [a + d * w.sigma * (1 + e) for e in (-1e-9, 1e-9, -1e-6, 1e-6)]
    idx = rng.choice(P0, len(edge), replace=False)
    trans[idx] = np.asarray(edge)
    quat = W.shoemake_quaternions(rng, P0)
    lig, q = np.zeros((1, 3)), np.array([0.8])
    ref = O.pose_energies(m, lig, q, quat, trans)
    E, f = prot.energies(lig, q, quat, trans)
    assert_flags(f, ref)
    assert_energies(E, ref)
    for i in idx[:4]:
        assert f[i] & L.RS_FLAG_OUT_OF_GRID
    assert not (f[idx[4]] & L.RS_FLAG_OUT_OF_GRID)
    assert f[idx[6]] & 1 and not (f[idx[7]] & 1)


def test_invalid_arguments(L, ctx, small):
    w, m, prot, _ = small
    with pytest.raises(L.RSError) as ei:
        L.rs_energy_poses(ctx.handle, prot.handle, np.zeros((0, 3)), np.zeros(0), w.quat[:2], w.trans[:2])
    assert ei.value.status == L.RS_ERR_INVALID
    with pytest.raises(L.RSError):
        L.rs_build_protein(ctx.handle, w.prot_xyz, w.prot_q, L.rs_params_default(n=2))
    with pytest.raises(L.RSError) as ei:
        L.rs_build_protein(ctx.handle, w.prot_xyz, w.prot_q, L.rs_params_default(tucker_cap=40))
    assert ei.value.status in (L.RS_ERR_INVALID, L.RS_ERR_UNSUPPORTED)
