"""Differentiation: the projected-gradient step of Eq. Energy_Min against the oracle's
step at identical input poses, monotone energy over many steps, and the autograd
binding against the adjoint and against central differences of the energy."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.rs_oracle import _rotvec_to_quat
from tests.parity import E_TOL, away_from_planes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[0, 12], ids=["canonical", "tucker"])
def setup(request):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_26611_gb300 import lib
    cap = request.param
    ctx = lib.Context(0)
    w = W.plain_small(P=256)
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l, tucker_cap=cap)
    prot = lib.Protein(ctx, w.prot_xyz, w.prot_q,
                       lib.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=cap))
    rv = W.random_rotvecs(np.random.default_rng(31), w.P)
    yield lib, ctx, prot, m, w, rv
    prot.close()
    ctx.close()


def _T(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda").clone()


def test_one_step_matches_oracle(setup):
    lib, ctx, prot, m, w, rv0 = setup
    rv, tr = _T(rv0), _T(w.trans)
    E, f, acc = lib.rs_pgd_run(ctx.handle, prot.handle, _T(w.lig_xyz), _T(w.lig_q), rv, tr, 1)
    ref = O.pgd_step(m, w.lig_xyz, w.lig_q, rv0, w.trans)
    acc, rv, tr, E, f = acc.cpu().numpy(), rv.cpu().numpy(), tr.cpu().numpy(), E.cpu().numpy(), f.cpu().numpy()
    same = acc == ref["accepted"]
    assert same.mean() > 0.97
    # where the accepted level agrees, the new pose is the same step; the step
    # direction carries the gradient's tolerance (1e-4), so poses agree to eta * 1e-4
    assert np.allclose(tr[same], ref["trans"][same], rtol=0, atol=1e-5)
    assert np.allclose(rv[same], ref["rotvec"][same], rtol=0, atol=1e-5)
    # energies reported for the GPU's new poses equal the oracle's at those poses
    chk = O.pose_energies(m, w.lig_xyz, w.lig_q, _rotvec_to_quat(rv), tr)
    ok = chk["flags"] == 0
    scale = O.tolerance_scale(chk["E"], chk["S_ref"])
    assert np.all((np.abs(E - chk["E"]) <= E_TOL * scale)[ok])
    # a differing decision must be a near-tie of E_trial and E_start
    for p in np.nonzero(~same)[0]:
        lv = acc[p] if acc[p] >= 0 else ref["accepted"][p]
        sc = 0.5 ** lv
        gt, gw = ref["dE_dt"][p], ref["dE_dw"][p]
        t1 = w.trans[p] - sc * 0.1 * gt / np.linalg.norm(gt)
        w1 = rv0[p] - sc * 0.02 * gw / np.linalg.norm(gw)
        e1 = O.pose_gradients(m, w.lig_xyz, w.lig_q, w1[None], t1[None])["E"][0]
        assert abs(e1 - ref["E_start"][p]) <= 1e-6 * max(abs(ref["E_start"][p]), 1e-3)


def test_many_steps_monotone_and_feasible(setup):
    import torch
    lib, ctx, prot, m, w, rv0 = setup
    rv, tr = _T(rv0), _T(w.trans)
    lx, lq = _T(w.lig_xyz), _T(w.lig_q)
    E0, f0, _ = lib.rs_pgd_run(ctx.handle, prot.handle, lx, lq, rv, tr, 1)
    prev, prev_f = E0.cpu().numpy(), f0.cpu().numpy()
    for _ in range(3):
        E, f, acc = lib.rs_pgd_run(ctx.handle, prot.handle, lx, lq, rv, tr, 5)
        E, f = E.cpu().numpy(), f.cpu().numpy()
        feas = prev_f == 0
        assert np.all(E[feas] <= prev[feas] + 1e-12 * np.abs(prev[feas]))
        assert np.all(f[feas] == 0)
        prev, prev_f = E, f
    # final energies are those of the final poses
    q = _rotvec_to_quat(rv.cpu().numpy())
    ref = O.pose_energies(m, w.lig_xyz, w.lig_q, q, tr.cpu().numpy())
    keep = ref["flags"] == 0
    assert np.all(np.abs(prev[keep] - ref["E"][keep]) <= E_TOL * np.maximum(np.abs(ref["E"][keep]),
                                                                             1e-2 * ref["S_ref"][keep]))


def test_autograd_matches_adjoint_and_fd(setup):
    import torch
    from paper_2510_26611_gb300.autograd import rs_energy
    lib, ctx, prot, m, w, rv0 = setup
    n = 64
    rv = _T(rv0[:n]).requires_grad_(True)
    tr = _T(w.trans[:n]).requires_grad_(True)
    lx, lq = _T(w.lig_xyz), _T(w.lig_q)
    E, f = rs_energy(prot, lx, lq, rv, tr)
    weights = torch.linspace(0.5, 1.5, n, dtype=torch.float64, device="cuda")
    (weights * E).sum().backward()
    Eg, gt, gw, _ = lib.rs_energy_grad_poses(ctx.handle, prot.handle, lx, lq, rv.detach(), tr.detach())
    assert torch.equal(E.detach(), Eg)
    assert torch.allclose(tr.grad, weights[:, None] * gt, rtol=0, atol=0)
    assert torch.allclose(rv.grad, weights[:, None] * gw, rtol=0, atol=0)
    # central differences of the FP64 oracle energy (both kinds), and of the GPU
    # energy itself where its evaluation is smooth to ~1e-12 relative (the Tucker
    # W-form path in pair arithmetic; the canonical path sums FP32 blocks, whose
    # rounding a 1e-4 step amplifies beyond the tolerance)
    keep = away_from_planes(m, w.lig_xyz, O.rotvec_to_rot(rv0[:n]), w.trans[:n], eps=2e-3)
    h = 1e-4
    rvn, trn = rv0[:n], w.trans[:n]
    fd_t, fd_w = np.zeros((n, 3)), np.zeros((n, 3))
    ofd_t, ofd_w = np.zeros((n, 3)), np.zeros((n, 3))
    oE = lambda r, t: O.pose_gradients(m, w.lig_xyz, w.lig_q, r, t)["E"]
    for a in range(3):
        d = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        d[:, a] = h
        dn = d.cpu().numpy()
        Ep = lib.rs_energy_grad_poses(ctx.handle, prot.handle, lx, lq, rv.detach(), tr.detach() + d)[0]
        Em = lib.rs_energy_grad_poses(ctx.handle, prot.handle, lx, lq, rv.detach(), tr.detach() - d)[0]
        fd_t[:, a] = ((Ep - Em) / (2 * h)).cpu().numpy()
        Ep = lib.rs_energy_grad_poses(ctx.handle, prot.handle, lx, lq, rv.detach() + d, tr.detach())[0]
        Em = lib.rs_energy_grad_poses(ctx.handle, prot.handle, lx, lq, rv.detach() - d, tr.detach())[0]
        fd_w[:, a] = ((Ep - Em) / (2 * h)).cpu().numpy()
        ofd_t[:, a] = (oE(rvn, trn + dn) - oE(rvn, trn - dn)) / (2 * h)
        ofd_w[:, a] = (oE(rvn + dn, trn) - oE(rvn - dn, trn)) / (2 * h)
    gt, gw = gt.cpu().numpy(), gw.cpu().numpy()
    sc = np.maximum(np.abs(gt).max(axis=1), np.abs(gw).max(axis=1))[:, None] + 1e-12
    assert np.all((np.abs(gt - ofd_t) / sc)[keep] <= 1e-4)
    assert np.all((np.abs(gw - ofd_w) / sc)[keep] <= 1e-4)
    if prot.info["kind"] == 1:
        assert np.all((np.abs(gt - fd_t) / sc)[keep] <= 1e-4)
        assert np.all((np.abs(gw - fd_w) / sc)[keep] <= 1e-4)
