"""Oracle parity at the sizes of the three system patterns.

* Differentiation: protein N=10000, ligand L=100, n=2049 (the projected-gradient
  workload); 256 of its 4096 feasible starting poses: one step against the oracle's
  step, the autograd gradients against the oracle's exact gradient, and the energies
  after 50 steps against the oracle's energies of the final poses.
* Batching: a persistent batched launch over pairs of the uneven-pairs workload with
  grids n = 513, 1025, 2049 and 4097 (1e4 poses each); every pair's energies and flags
  on a pose sample against the oracle.
* Serving: Tucker requests on n = 16385 and n = 8193 grids (2048 poses each, ligands
  of the serving stream) mixed with a pool protein's requests in one server; every
  request against the oracle on all of its poses.  The fine-grid proteins keep N = 200
  so that the oracle's SVD of the n x (N R_l) factor matrices stays within seconds.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O
import workloads as W
from tests.parity import (E_TOL, assert_energies, assert_flags, assert_gradients,
                          assert_paths_agree, away_from_planes)

pytestmark = pytest.mark.gpu


def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_26611_gb300 import lib
    return torch, lib


def _T(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda").clone()


def _rotvec(quat):
    """Unit quaternions (w, x, y, z) -> rotation vectors, through scipy (scalar last)."""
    q = np.asarray(quat)
    return Rotation.from_quat(np.concatenate([q[:, 1:], q[:, :1]], axis=1)).as_rotvec()


def _quat(rv):
    x = Rotation.from_rotvec(np.asarray(rv)).as_quat()
    return np.concatenate([x[:, 3:], x[:, :3]], axis=1)


# ------------------------------------------------------------ differentiation
@pytest.fixture(scope="module")
def pgd():
    torch, lib = _cuda()
    ctx = lib.Context(0)
    w0 = W.pgd_start(P=1)
    prm = lib.rs_params_default(n=w0.n, b=w0.b, sigma=w0.sigma, R_l=w0.R_l, tucker_cap=w0.tucker_cap)
    prot = lib.Protein(ctx, w0.prot_xyz, w0.prot_q, prm)
    lx, lq = _T(w0.lig_xyz), _T(w0.lig_q)

    def feasible(qq, tt):
        E, f = prot.energies(lx, lq, _T(qq), _T(tt))
        return f.cpu().numpy() == 0

    w = W.pgd_start(P=4096, feasible=feasible)
    pick = np.sort(np.random.default_rng(41).choice(w.P, 256, replace=False))
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l, tucker_cap=w.tucker_cap)
    assert [v.shape[1] for v in m.V] == list(prot.info["rank"])
    rv0, tr0 = _rotvec(w.quat[pick]), w.trans[pick]
    yield lib, ctx, prot, m, w, rv0, tr0
    prot.close()
    ctx.close()


def test_pgd_workload_one_step_against_oracle(pgd):
    lib, ctx, prot, m, w, rv0, tr0 = pgd
    rv, tr = _T(rv0), _T(tr0)
    E, f, acc = lib.rs_pgd_run(ctx.handle, prot.handle, _T(w.lig_xyz), _T(w.lig_q), rv, tr, 1)
    ref = O.pgd_step(m, w.lig_xyz, w.lig_q, rv0, tr0)
    acc, rv, tr = acc.cpu().numpy(), rv.cpu().numpy(), tr.cpu().numpy()
    E, f = E.cpu().numpy(), f.cpu().numpy()
    assert np.all(ref["E"] <= ref["E_start"])
    same = acc == ref["accepted"]
    assert same.mean() > 0.97
    # the step direction carries the gradient tolerance (1e-4): new poses within eta * 1e-4
    assert np.abs(tr[same] - ref["trans"][same]).max() <= 1e-5
    assert np.abs(rv[same] - ref["rotvec"][same]).max() <= 1e-5
    chk = O.pose_energies(m, w.lig_xyz, w.lig_q, _quat(rv), tr)
    assert np.array_equal(chk["flags"], f)
    assert_energies(E[f == 0], {k: v[f == 0] for k, v in chk.items()})
    # a differing decision is a near-tie between the trial and the starting energy
    for p in np.nonzero(~same)[0]:
        lv = acc[p] if acc[p] >= 0 else ref["accepted"][p]
        sc = 0.5 ** lv
        gt, gw = ref["dE_dt"][p], ref["dE_dw"][p]
        t1 = tr0[p] - sc * 0.1 * gt / np.linalg.norm(gt)
        w1 = rv0[p] - sc * 0.02 * gw / np.linalg.norm(gw)
        e1 = O.pose_energies(m, w.lig_xyz, w.lig_q, _quat(w1[None]), t1[None])["E"][0]
        assert abs(e1 - ref["E_start"][p]) <= 1e-6 * max(abs(ref["E_start"][p]), 1e-3)


def test_pgd_workload_autograd_against_oracle_gradient(pgd):
    import torch
    from paper_2510_26611_gb300.autograd import rs_energy
    lib, ctx, prot, m, w, rv0, tr0 = pgd
    rv = _T(rv0).requires_grad_(True)
    tr = _T(tr0).requires_grad_(True)
    E, f = rs_energy(prot, _T(w.lig_xyz), _T(w.lig_q), rv, tr)
    E.sum().backward()
    ref = O.pose_gradients(m, w.lig_xyz, w.lig_q, rv0, tr0)
    keep = away_from_planes(m, w.lig_xyz, O.rotvec_to_rot(rv0), tr0)
    assert keep.mean() > 0.5
    assert_energies(E.detach().cpu().numpy(), ref)
    assert_flags(f.cpu().numpy(), ref)
    assert_gradients(tr.grad.cpu().numpy(), rv.grad.cpu().numpy(), ref, keep=keep)


def test_pgd_workload_fifty_steps_against_oracle(pgd):
    lib, ctx, prot, m, w, rv0, tr0 = pgd
    rv, tr = _T(rv0), _T(tr0)
    E0 = O.pose_energies(m, w.lig_xyz, w.lig_q, _quat(rv0), tr0)["E"]
    E, f, acc = lib.rs_pgd_run(ctx.handle, prot.handle, _T(w.lig_xyz), _T(w.lig_q), rv, tr, 50)
    E, f = E.cpu().numpy(), f.cpu().numpy()
    rv, tr = rv.cpu().numpy(), tr.cpu().numpy()
    assert np.all(f == 0)
    ref = O.pose_energies(m, w.lig_xyz, w.lig_q, _quat(rv), tr)
    assert_flags(f, ref)
    assert_energies(E, ref)
    # every accepted step lowered (or kept) the energy: the end is below the start
    scale = O.tolerance_scale(E0, ref["S_ref"])
    assert np.all(ref["E"] <= E0 + E_TOL * scale)
    assert (ref["E"] < E0 - 1e-3 * scale).mean() > 0.5


# ------------------------------------------------------------------- batching
@pytest.fixture(scope="module")
def batch():
    torch, lib = _cuda()
    ws = W.batch_pairs(seed=2, pairs=64, P=10_000)
    by_n = {}
    for w in sorted(ws, key=lambda w: w.N):
        by_n.setdefault(w.n, []).append(w)
    sel = [by_n[513][0], by_n[1025][0], by_n[2049][0], by_n[2049][1], by_n[4097][0]]
    ctx = lib.Context(0)
    prots, pairs = [], []
    for w in sel:
        prm = lib.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=w.tucker_cap)
        pr = lib.Protein(ctx, w.prot_xyz, w.prot_q, prm)
        prots.append(pr)
        pairs.append(dict(prot=pr.handle, lig_xyz=_T(w.lig_xyz), lig_q=_T(w.lig_q), quat=_T(w.quat),
                          trans=_T(w.trans),
                          E_out=torch.full((w.P,), float("nan"), dtype=torch.float64, device="cuda"),
                          flags_out=torch.full((w.P,), 255, dtype=torch.uint8, device="cuda")))
    b, keep = lib.rs_batch_create(ctx.handle, pairs, autotune=True)
    lib.rs_batch_run(b)
    torch.cuda.synchronize()
    yield lib, sel, prots, pairs, b
    lib.rs_batch_free(b)
    for p in prots:
        p.close()
    ctx.close()


@pytest.mark.parametrize("k", range(5), ids=["n513", "n1025", "n2049a", "n2049b", "n4097"])
def test_batch_workload_pair_against_oracle(batch, k):
    lib, sel, prots, pairs, b = batch
    w = sel[k]
    pick = np.sort(np.random.default_rng(100 + k).choice(w.P, 1500, replace=False))
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l, tucker_cap=w.tucker_cap)
    assert [v.shape[1] for v in m.V] == list(prots[k].info["rank"])
    ref = O.pose_energies(m, w.lig_xyz, w.lig_q, w.quat[pick], w.trans[pick])
    E = pairs[k]["E_out"].cpu().numpy()
    f = pairs[k]["flags_out"].cpu().numpy()
    assert_energies(E[pick], ref)
    assert_flags(f[pick], ref)
    # every pose of the pair: the batched launch equals the plain call
    Ep, fp = prots[k].energies(pairs[k]["lig_xyz"], pairs[k]["lig_q"], pairs[k]["quat"], pairs[k]["trans"])
    assert_paths_agree(E, Ep.cpu().numpy(), f, fp.cpu().numpy())


# -------------------------------------------------------------------- serving
def _fine_grid_protein(rng, n, pid, N=200):
    prot, r_p = W.sphere_lattice(rng, N)
    r_l_max = 5.0 * (200 / 20.0) ** (1.0 / 3.0)
    return {"id": pid, "xyz": prot, "q": W.mixed_charges(rng, N, 0.3, 0.08), "r_p": r_p,
            "b": r_p + 2.0 * r_l_max + 8.0, "sigma": 3.0, "R_l": 20, "tucker_cap": 20, "n": n}


def test_served_fine_grid_requests_against_oracle():
    torch, lib = _cuda()
    rng = np.random.default_rng(77)
    pool = W.serve_pool(n_max=16385)
    small = min((e for e in pool if e["n"] == 1025), key=lambda e: e["xyz"].shape[0])
    prots = [_fine_grid_protein(rng, 16385, 1001), _fine_grid_protein(rng, 8193, 1002), small]
    gen = np.random.default_rng(78)
    reqs = [(e, W.serve_request(gen, e)) for e in prots for _ in range(2)]
    srv = lib.Server(0)
    try:
        ids = []
        for e, r in reqs:
            prm = lib.rs_params_default(n=e["n"], b=e["b"], sigma=e["sigma"], R_l=e["R_l"],
                                        tucker_cap=e["tucker_cap"])
            ids.append(srv.submit(e["id"], e["xyz"], e["q"], prm, r["lig_xyz"], r["lig_q"],
                                  r["quat"], r["trans"]))
        res = [srv.wait(rid, 600_000) for rid in ids]
    finally:
        srv.close()
    models = {}
    for (e, r), out in zip(reqs, res):
        assert out["status"] == 0
        if e["id"] not in models:
            models[e["id"]] = O.build_model(e["xyz"], e["q"], e["n"], e["b"], e["sigma"], e["R_l"],
                                            tucker_cap=e["tucker_cap"])
        ref = O.pose_energies(models[e["id"]], r["lig_xyz"], r["lig_q"], r["quat"], r["trans"])
        assert out["E"].shape == (2048,)
        assert_energies(out["E"], ref)
        assert_flags(out["flags"], ref)
        assert (ref["flags"] == 0).any() and (ref["flags"] != 0).any()
