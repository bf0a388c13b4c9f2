"""Pins of the oracle's add-and-compress (Sec. 3.4, Algorithm TEP step 4; Sec. 5.1,
Eq. EnergySum_Mcomplex): the recompressed sum of two molecules' Tucker tensors
against the plain sum of their full grid tensors, the HOSVD truncation bound, and the
energies of the complex computed molecule by molecule."""
import numpy as np

import oracle as O
import workloads as W


def _models(cap=6):
    rng = np.random.default_rng(23)
    xa = rng.normal(0.0, 1.2, (6, 3)) + np.array([-1.5, 0.3, 0.0])
    xb = rng.normal(0.0, 1.2, (5, 3)) + np.array([1.8, -0.4, 0.5])
    qa, qb = rng.normal(0.0, 0.6, 6), rng.normal(0.0, 0.6, 5)
    kw = dict(n=33, b=8.0, sigma=1.0, R_l=8, tucker_cap=cap)
    return O.build_model(xa, qa, **kw), O.build_model(xb, qb, **kw)


def _full(m):
    return np.einsum("abc,ia,jb,kc->ijk", m.beta, m.V[0], m.V[1], m.V[2], optimize=True)


def test_sum_without_truncation_is_exact():
    m1, m2 = _models()
    ac = O.add_and_compress([m1, m2], cap=1000, eps_r=0.0)
    T = _full(m1) + _full(m2)
    assert np.linalg.norm(_full(ac) - T) <= 1e-12 * np.linalg.norm(T)
    assert ac.trunc_bound <= 1e-12 * np.linalg.norm(T)
    assert np.array_equal(ac.prot_q, np.concatenate([m1.prot_q, m2.prot_q]))


def test_single_molecule_is_reproduced():
    m1, _ = _models()
    ac = O.add_and_compress([m1], cap=1000, eps_r=0.0)
    T = _full(m1)
    assert ac.ranks == m1.ranks
    assert np.linalg.norm(_full(ac) - T) <= 1e-13 * np.linalg.norm(T)


def test_equal_molecules_double_the_tensor():
    m1, _ = _models()
    ac = O.add_and_compress([m1, m1], cap=1000, eps_r=1e-12)
    T = _full(m1)
    assert ac.ranks == m1.ranks  # the repeated columns add no direction
    assert np.linalg.norm(_full(ac) - 2.0 * T) <= 1e-12 * np.linalg.norm(T)


def test_truncation_within_the_hosvd_bound():
    m1, m2 = _models()
    ac = O.add_and_compress([m1, m2], cap=4, eps_r=0.0)
    T = _full(m1) + _full(m2)
    err = np.linalg.norm(_full(ac) - T)
    assert max(ac.ranks) == 4 and ac.trunc_bound > 1e-8 * np.linalg.norm(T)
    assert err <= ac.trunc_bound * (1.0 + 1e-9)
    # the leading singular values of the summed tensor's unfoldings, from the full tensor
    for ax in range(3):
        M = np.moveaxis(T, ax, 0).reshape(T.shape[ax], -1)
        s = np.linalg.svd(M, compute_uv=False)
        k = len(ac.svals[ax])
        assert np.allclose(ac.svals[ax], s[:k], rtol=1e-10, atol=1e-12 * s[0])


def test_energies_equal_the_complex_computed_molecule_by_molecule():
    m1, m2 = _models()
    ac = O.add_and_compress([m1, m2], cap=1000, eps_r=0.0)
    rng = np.random.default_rng(5)
    lig = W.ball_uniform(rng, 4, 1.0)
    lq = rng.normal(0.0, 0.4, 4)
    quat = W.shoemake_quaternions(rng, 200)
    trans = rng.uniform(-5.0, 5.0, (200, 3))
    e_ac = O.pose_energies(ac, lig, lq, quat, trans)
    e_cx = O.complex_energies([m1, m2], lig, lq, quat, trans)
    assert np.array_equal(e_ac["flags"], e_cx["flags"])
    assert np.max(np.abs(e_ac["E"] - e_cx["E"]) / np.maximum(e_cx["S_ref"], 1e-300)) <= 1e-11
