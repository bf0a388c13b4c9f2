"""Parity at the benchmark's full size (protein-scale workload, P = 1e5 poses,
device-resident buffers, the launch configuration bench.py times): every flag and
the top-10 feasible ranking against the oracle over all poses, energies over all
poses, gradients on a sample."""
import numpy as np
import pytest

import oracle as O
from tests.parity import (assert_energies, assert_flags, assert_gradients, assert_topk,
                          away_from_planes)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from bench import workload
    from paper_2510_26611_gb300 import lib
    w, rv = workload(100_000)
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l, tucker_cap=w.tucker_cap)
    ref = O.pose_energies(m, w.lig_xyz, w.lig_q, w.quat, w.trans)
    ctx = lib.Context(0)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    params = lib.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=w.tucker_cap)
    h = lib.rs_build_protein(ctx.handle, T(w.prot_xyz), T(w.prot_q), params)
    yield lib, ctx, h, w, rv, m, ref, T
    lib.rs_protein_free(h)
    ctx.close()


def test_fullsize_energies_flags_topk(full):
    lib, ctx, h, w, rv, m, ref, T = full
    E, f = lib.rs_energy_poses(ctx.handle, h, T(w.lig_xyz), T(w.lig_q), T(w.quat), T(w.trans))
    E, f = E.cpu().numpy(), f.cpu().numpy()
    assert_flags(f, ref)
    err = assert_energies(E, ref)
    assert_topk(E, f, ref)
    print(f"full-size energies: max rel err {err.max():.3e}, feasible {np.mean(f == 0):.3f}")


def test_fullsize_gradients_sample(full):
    lib, ctx, h, w, rv, m, ref_e, T = full
    idx = np.random.default_rng(5).choice(w.P, 1500, replace=False)
    Eg, gt, gw, fg = lib.rs_energy_grad_poses(ctx.handle, h, T(w.lig_xyz), T(w.lig_q), T(rv),
                                              T(w.trans))
    ref = O.pose_gradients(m, w.lig_xyz, w.lig_q, rv[idx], w.trans[idx])
    keep = away_from_planes(m, w.lig_xyz, O.rotvec_to_rot(rv[idx]), w.trans[idx])
    assert_energies(Eg.cpu().numpy()[idx], ref)
    assert_gradients(gt.cpu().numpy()[idx], gw.cpu().numpy()[idx], ref, keep)
    # the gradient call's energies equal the energy call's for the same rotations
    assert np.allclose(Eg.cpu().numpy()[idx], ref_e["E"][idx],
                       rtol=0, atol=1e-5 * np.abs(ref_e["E"][idx]).max())


def test_two_chunk_call_is_order_independent(full):
    """A call larger than one chunk (2^23 pose-atoms): 167 772 + 1000 poses, the second
    chunk far below the tensor-core form's fill threshold on its own.  Every chunk of a
    call takes the same W-form kernel, so permuting the poses permutes the energies bit
    for bit; the small chunk's poses also match the oracle."""
    lib, ctx, h, w, rv, m, ref, T = full
    from bench import workload
    P = (1 << 23) // w.L + 1000
    w2, _ = workload(P)
    E1, f1 = lib.rs_energy_poses(ctx.handle, h, T(w2.lig_xyz), T(w2.lig_q), T(w2.quat), T(w2.trans))
    perm = np.random.default_rng(11).permutation(P)
    E2, f2 = lib.rs_energy_poses(ctx.handle, h, T(w2.lig_xyz), T(w2.lig_q), T(w2.quat[perm]), T(w2.trans[perm]))
    E1, f1, E2, f2 = (x.cpu().numpy() for x in (E1, f1, E2, f2))
    assert np.array_equal(E2, E1[perm]) and np.array_equal(f2, f1[perm])
    idx = np.arange(P - 300, P)  # poses of the second chunk of the first call
    sub = O.pose_energies(m, w2.lig_xyz, w2.lig_q, w2.quat[idx], w2.trans[idx])
    assert_energies(E1[idx], sub)
    assert_flags(f1[idx], sub)
