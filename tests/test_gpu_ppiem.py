"""Pose scan of Algorithm PPIEM on the GPU against the FP64 oracle: contact offsets,
contact-pose energies and flags, best rotation per direction, local minima; host and
device buffers; a protein-scale scan checked on a sample and by its own invariants."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.parity import E_TOL

pytestmark = pytest.mark.gpu

S_TOL = 1e-9    # contact offsets (A): the same FP64 expression on both sides


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


def _scale(E, S):
    return np.maximum(np.abs(E), 1e-2 * S)


def assert_scan(out, ref):
    s, E, F = (np.asarray(out[k]) for k in ("s", "E", "flags"))
    fin = np.isfinite(ref["s"])
    assert np.array_equal(np.isfinite(s), fin)
    assert np.abs(s[fin] - ref["s"][fin]).max() <= S_TOL
    assert np.array_equal(F, ref["flags"])
    assert np.all(np.isinf(E[~fin]))
    sc = _scale(ref["E"][fin], ref["S_ref"][fin])
    err = np.abs(E[fin] - ref["E"][fin]) / sc
    assert err.max() <= E_TOL, err.max()
    # per direction: the best rotation, or a near-tie of it
    Eb, rb = np.asarray(out["E_best"]), np.asarray(out["rot_best"])
    has = rb >= 0
    assert np.array_equal(has, ref["rot_best"] >= 0)
    d = np.nonzero(has)[0]
    same = rb[d] == ref["rot_best"][d]
    for k in d[~same]:
        a, b = rb[k], ref["rot_best"][k]
        assert abs(ref["E"][k, a] - ref["E"][k, b]) <= 2e-5 * max(_scale(ref["E"][k, a], ref["S_ref"][k, a]),
                                                               _scale(ref["E"][k, b], ref["S_ref"][k, b]))
    assert np.all(Eb[d] == E[d, rb[d]])
    # local minima: equal, except where a neighbour pair is a near-tie
    im = np.asarray(out["is_min"]).astype(bool)
    for k in np.nonzero(im != ref["is_min"])[0]:
        assert np.isfinite(ref["E_best"][k])
        gap = np.abs(ref["E_best"] - ref["E_best"][k])
        assert np.min(gap[np.arange(gap.size) != k]) <= 2e-5 * abs(ref["E_best"][k]) + 1e-12
    return same.mean()


@pytest.fixture(scope="module", params=[12, 0], ids=["tucker", "canonical"])
def small(request, L, ctx):
    cap = request.param
    w = W.plain_small(P=1)
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l, tucker_cap=cap)
    prot = L.Protein(ctx, w.prot_xyz, w.prot_q,
                     L.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=cap))
    yield w, m, prot
    prot.close()


def test_scan_small_matches_oracle(L, small):
    w, m, prot = small
    quats = W.euler_grid_quaternions(4)
    out = prot.ppiem_scan(w.lig_xyz, w.lig_q, quats, 6, 12)
    ref = O.ppiem_scan(m, w.lig_xyz, w.lig_q, quats, 6, 12)
    print("same best rotation:", assert_scan(out, ref))
    # the best translation is its contact pose's
    d = np.nonzero(np.asarray(out["rot_best"]) >= 0)[0]
    r = np.asarray(out["rot_best"])[d]
    t = ref["x_P"] + (np.asarray(out["s"])[d, r] + 1e-6 * w.sigma)[:, None] * ref["dirs"][d]
    assert np.allclose(np.asarray(out["t_best"])[d], t, rtol=0, atol=1e-12)


def test_scan_given_centre_and_margin(L, small):
    w, m, prot = small
    quats = W.euler_grid_quaternions(2)
    xP = np.array([1.5, -2.0, 0.75])
    out = prot.ppiem_scan(w.lig_xyz, w.lig_q, quats, 4, 8, x_P=xP, margin=0.05)
    ref = O.ppiem_scan(m, w.lig_xyz, w.lig_q, quats, 4, 8, x_P=xP, margin=0.05)
    assert_scan(out, ref)


def test_scan_device_buffers_equal_host(L, small):
    import torch
    w, m, prot = small
    quats = W.euler_grid_quaternions(2)
    a = prot.ppiem_scan(w.lig_xyz, w.lig_q, quats, 4, 8)
    T = lambda x: torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    b = prot.ppiem_scan(T(w.lig_xyz), T(w.lig_q), T(quats), 4, 8)
    torch.cuda.synchronize()
    for k in a:
        assert np.array_equal(np.asarray(a[k]), b[k].cpu().numpy(), equal_nan=True), k


def test_scan_without_contact(L, ctx):
    # one protein atom: directions whose ligand lines all miss it have no contact
    prot = L.Protein(ctx, np.zeros((1, 3)), np.array([1.0]),
                     L.rs_params_default(n=33, b=8.0, sigma=1.0, R_l=8, tucker_cap=4))
    m = O.build_model(np.zeros((1, 3)), np.array([1.0]), 33, 8.0, 1.0, 8, tucker_cap=4)
    try:
        lig = np.array([[2.0, 0, 0], [-2.0, 0, 0]])
        quats = np.array([[1.0, 0, 0, 0]])
        out = prot.ppiem_scan(lig, np.array([0.3, -0.3]), quats, 4, 8)
        ref = O.ppiem_scan(m, lig, np.array([0.3, -0.3]), quats, 4, 8)
        none = ~np.isfinite(ref["s"][:, 0])
        assert none.any()
        assert np.all(np.asarray(out["flags"])[none, 0] == 4) and np.all(np.asarray(out["rot_best"])[none] == -1)
        assert np.all(np.isinf(np.asarray(out["E_best"])[none]))
        assert_scan(out, ref)
    finally:
        prot.close()


def test_scan_argument_errors(L, small):
    w, m, prot = small
    q = W.euler_grid_quaternions(2)
    for kw in (dict(n_theta=0, n_phi=4), dict(n_theta=300, n_phi=300)):
        with pytest.raises(L.RSError) as e:
            prot.ppiem_scan(w.lig_xyz, w.lig_q, q, **kw)
        assert e.value.status == L.RS_ERR_INVALID
    with pytest.raises(L.RSError):
        prot.ppiem_scan(w.lig_xyz, w.lig_q, q, 4, 4, margin=-1.0)
    with pytest.raises(L.RSError):
        prot.ppiem_scan(w.lig_xyz, w.lig_q, q[:0], 4, 4)


def test_scan_protein_scale_sampled(L, ctx):
    # 128 directions x 108 rotations x 50 atoms on the N=3000 protein (cell-grouped pose
    # path): a sample of (direction, rotation) pairs against the oracle, and the
    # scan's own invariants everywhere
    w = W.plain_protein(P=1)
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l, tucker_cap=20)
    prot = L.Protein(ctx, w.prot_xyz, w.prot_q,
                     L.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=w.tucker_cap))
    try:
        quats = W.euler_grid_quaternions(6)
        out = prot.ppiem_scan(w.lig_xyz, w.lig_q, quats, 8, 16)
        s, E, F = (np.asarray(out[k]) for k in ("s", "E", "flags"))
        D, R = s.shape
        rng = np.random.default_rng(5)
        pick = rng.choice(D * R, 300, replace=False)
        d, r = pick // R, pick % R
        U = O.ppiem_directions(8, 16)
        x_P = w.prot_xyz.mean(axis=0)
        s_ref = O.contact_offsets(w.prot_xyz, w.sigma, w.lig_xyz, quats[r], x_P, U[d])
        assert np.abs(s[d, r] - s_ref).max() <= S_TOL
        t = x_P + (s_ref + 1e-6 * w.sigma)[:, None] * U[d]
        ev = O.pose_energies(m, w.lig_xyz, w.lig_q, quats[r], t)
        err = np.abs(E[d, r] - ev["E"]) / O.tolerance_scale(ev["E"], ev["S_ref"])
        assert err.max() <= E_TOL
        assert np.array_equal(F[d, r], ev["flags"])
        # invariants: best = lowest feasible energy of its direction; minima consistent
        Ef = np.where(F == 0, E, np.inf)
        assert np.array_equal(np.asarray(out["E_best"]), Ef.min(axis=1))
        assert np.array_equal(np.asarray(out["rot_best"]), np.where(np.isfinite(Ef.min(axis=1)), Ef.argmin(axis=1), -1))
        ref_min = np.zeros(D, dtype=bool)
        Eb = np.asarray(out["E_best"])
        for k in range(D):
            a, b = divmod(k, 16)
            nb = [x * 16 + b for x in (a - 1, a + 1) if 0 <= x < 8] + [a * 16 + (b - 1) % 16, a * 16 + (b + 1) % 16]
            ref_min[k] = np.isfinite(Eb[k]) and all(Eb[k] < Eb[e] or (Eb[k] == Eb[e] and k < e) for e in nb)
        assert np.array_equal(np.asarray(out["is_min"]).astype(bool), ref_min)
        print("feasible contact poses:", float((F == 0).mean()), "minima:", int(ref_min.sum()))
    finally:
        prot.close()
