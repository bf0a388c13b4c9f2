"""Pins of the oracle's local-box model (scheme C of Sec. 3.2, Table 1): exact
restriction without truncation, the HOSVD truncation bound, the box flags, and ranks
in a solvent box below the global ones.  CPU only."""
import numpy as np
import pytest

import oracle as O
import workloads as W


@pytest.fixture(scope="module")
def model():
    w = W.plain_small(P=1)
    return O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l, tucker_cap=20)


def _points(rng, lo, hi, k=400):
    return lo + (hi - lo) * rng.uniform(0.02, 0.98, size=(k, 3))


def test_local_box_without_truncation_is_the_restriction(model):
    c = np.array([24.0, 3.0, -2.0])
    lo, hi = c - 5.0, c + 5.0
    lm = O.local_box_model(model, lo, hi, eps=0.0)
    x = _points(np.random.default_rng(1), lo, hi)
    g, _, _, _ = O.potential(model, x)
    l, _, _, _ = O.potential(lm, x)
    assert np.abs(l - g).max() <= 1e-12 * np.abs(g).max()


@pytest.mark.parametrize("eps", [1e-3, 1e-5])
def test_local_box_truncation_bound(model, eps):
    # trilinear weights are >= 0 and sum to 1, so the error at any point of the box is
    # at most the largest node error, which is at most the HOSVD bound (Frobenius)
    c = np.array([-6.0, 25.0, 4.0])
    lo, hi = c - 6.0, c + 6.0
    lm = O.local_box_model(model, lo, hi, eps=eps)
    x = _points(np.random.default_rng(2), lo, hi)
    g, _, _, _ = O.potential(model, x)
    l, _, _, _ = O.potential(lm, x)
    err = np.abs(l - g).max()
    assert err <= lm.trunc_bound * (1 + 1e-9) + 1e-15
    assert lm.trunc_bound <= 3 ** 0.5 * eps * max(sv[0] for sv in lm.svals) * 30
    # a coarser eps gives no larger ranks
    lm2 = O.local_box_model(model, lo, hi, eps=eps * 100)
    assert all(a <= b for a, b in zip(lm2.ranks, lm.ranks))


def test_local_box_flags_outside(model):
    c = np.array([24.0, 3.0, -2.0])
    lm = O.local_box_model(model, c - 4.0, c + 4.0)
    lig = np.zeros((1, 3))
    quat = np.array([[1.0, 0, 0, 0]] * 3)
    trans = np.array([c, c + np.array([5.0, 0, 0]), c - np.array([0, 0, 4.6])])
    r = O.pose_energies(lm, lig, np.array([1.0]), quat, trans)
    assert list(r["flags"] & O.FLAG_OUT_OF_GRID) == [0, O.FLAG_OUT_OF_GRID, O.FLAG_OUT_OF_GRID]


def test_solvent_box_ranks_below_global(model):
    # Table 1: the potential restricted to a small box outside the cluster has small
    # ranks, nearly independent of the cluster (here 20 -> about 10 at eps = 1e-7)
    c = np.array([0.0, 0.0, 27.0])
    lm = O.local_box_model(model, c - 4.0, c + 4.0, eps=1e-7)
    assert max(lm.ranks) <= 14 and max(lm.ranks) < max(model.ranks)
