"""Molecular complexes (Eq. EnergySum_Mcomplex) and Galerkin factors (Eq. galten) on
the GPU against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.parity import assert_energies, assert_flags

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


def test_complex_of_two_molecules(L, ctx):
    # two molecules on different grids and forms: the sum of their potentials
    w = W.plain_small(P=2000)
    half = w.prot_xyz.shape[0] // 2
    specs = [(w.prot_xyz[:half], w.prot_q[:half], 257, 12), (w.prot_xyz[half:], w.prot_q[half:], 129, 0)]
    prots, models = [], []
    for xyz, q, n, cap in specs:
        prots.append(L.Protein(ctx, xyz, q, L.rs_params_default(n=n, b=w.b, sigma=w.sigma, R_l=w.R_l,
                                                                tucker_cap=cap)))
        models.append(O.build_model(xyz, q, n, w.b, w.sigma, w.R_l, tucker_cap=cap))
    try:
        E, f = L.rs_energy_poses_complex(ctx.handle, [p.handle for p in prots], w.lig_xyz, w.lig_q, w.quat, w.trans)
        ref = O.complex_energies(models, w.lig_xyz, w.lig_q, w.quat, w.trans)
        assert_energies(E, ref)
        assert_flags(f, ref)
        # the sum of the single-molecule calls, in molecule order
        parts = [p.energies(w.lig_xyz, w.lig_q, w.quat, w.trans) for p in prots]
        assert np.array_equal(np.asarray(E), np.asarray(parts[0][0]) + np.asarray(parts[1][0]))
        assert np.array_equal(np.asarray(f), np.asarray(parts[0][1]) | np.asarray(parts[1][1]))
        # device buffers give the same bits
        import torch
        T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
        Ed, fd = L.rs_energy_poses_complex(ctx.handle, [p.handle for p in prots], T(w.lig_xyz), T(w.lig_q),
                                           T(w.quat), T(w.trans))
        assert np.array_equal(Ed.cpu().numpy(), np.asarray(E)) and np.array_equal(fd.cpu().numpy(), np.asarray(f))
    finally:
        for p in prots:
            p.close()


def test_galerkin_canonical_energies(L, ctx):
    # poses among the protein's atoms, where the narrow long-range Gaussians matter
    # and cell averages differ from node values by far more than the tolerance
    w = W.plain_small(P=600)
    trans = W.ball_uniform(np.random.default_rng(4), w.P, 12.0)
    prot = L.Protein(ctx, w.prot_xyz, w.prot_q,
                     L.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=0, galerkin=1))
    try:
        m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l, galerkin=True)
        E, f = prot.energies(w.lig_xyz, w.lig_q, w.quat, trans)
        ref = O.pose_energies(m, w.lig_xyz, w.lig_q, w.quat, trans)
        err = assert_energies(E, ref)
        assert_flags(f, ref)
        mc = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l)
        refc = O.pose_energies(mc, w.lig_xyz, w.lig_q, w.quat, trans)
        sep = np.abs(ref["E"] - refc["E"]) / O.tolerance_scale(ref["E"], ref["S_ref"])
        assert (sep > 10 * err.max()).mean() > 0.2
    finally:
        prot.close()


def test_galerkin_needs_canonical(L, ctx):
    w = W.plain_small(P=1)
    with pytest.raises(L.RSError) as e:
        L.Protein(ctx, w.prot_xyz, w.prot_q,
                  L.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=12, galerkin=1))
    assert e.value.status == L.RS_ERR_UNSUPPORTED
