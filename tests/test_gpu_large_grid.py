"""Fine grids (n = 8193, 16385): the Tucker build and the pose kernel against the
oracle's reduced model at the same n, on a small protein so the oracle's SVD of the
n x (N R_l) factor matrices stays in seconds."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.parity import assert_energies, assert_flags

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [8193, 16385])
def test_fine_grid_tucker_matches_oracle(n):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_26611_gb300 import lib
    rng = np.random.default_rng(n)
    prot, r_p = W.sphere_lattice(rng, 150)
    zq = W.mixed_charges(rng, 150, 0.3, 0.08)
    L = 20
    r_l = 5.0
    lig = W.ball_uniform(rng, L, r_l)
    lq = rng.normal(0.0, 0.3, L)
    P = 400
    quat = W.shoemake_quaternions(rng, P)
    trans = W.shell_translations(rng, P, r_p, r_p + 2 * r_l + 3)
    b = r_p + 2 * r_l + 8
    ctx = lib.Context(0)
    try:
        pr = lib.Protein(ctx, prot, zq, lib.rs_params_default(n=n, b=b, sigma=3.0, R_l=20,
                                                              tucker_cap=20))
        E, f = pr.energies(lig, lq, quat, trans)
        info = pr.info
        pr.close()
    finally:
        ctx.close()
    assert info["kind"] == 1 and info["n"] == n
    m = O.build_model(prot, zq, n, b, 3.0, 20, tucker_cap=20)
    assert [v.shape[1] for v in m.V] == list(info["rank"])
    ref = O.pose_energies(m, lig, lq, quat, trans)
    assert_energies(np.asarray(E), ref)
    assert_flags(np.asarray(f), ref)
