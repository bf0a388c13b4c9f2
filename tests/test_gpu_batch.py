"""Batched persistent launch: pairs of uneven size in one graph-captured launch give
the same energies and flags as one plain call per pair (bit for bit where both take
the same W-form kernel, as the pair-by-pair modes do on one stream or on concurrent
streams, else within the path tolerance), before and after the poses are rewritten in
place; one pair is checked against the oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.parity import assert_energies, assert_flags, assert_paths_agree

pytestmark = pytest.mark.gpu


def _pairs(rng):
    specs = [(400, 10, 257, 700), (1200, 35, 257, 1), (2500, 120, 513, 333), (800, 57, 513, 1000),
             (3000, 200, 257, 129), (600, 23, 513, 0)]
    out = []
    for N, L, n, P in specs:
        prot, r_p = W.sphere_lattice(rng, N)
        zq = W.mixed_charges(rng, N, 0.3, 0.08)
        r_l = 5.0 * (L / 20.0) ** (1.0 / 3.0)
        lig = W.ball_uniform(rng, L, r_l)
        lq = rng.normal(0.0, 0.3, L)
        quat = W.shoemake_quaternions(rng, P)
        trans = W.shell_translations(rng, P, r_p, r_p + 2 * r_l + 3)
        b = r_p + 2 * r_l + 8
        out.append(W.Workload(f"b{N}", prot, zq, lig, lq, quat, trans, n=n, b=b, sigma=3.0,
                              R_l=20, tucker_cap=16))
    return out


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_26611_gb300 import lib
    ctx = lib.Context(0)
    ws = _pairs(np.random.default_rng(21))
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    prots, pairs = [], []
    for w in ws:
        prm = lib.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=w.tucker_cap)
        pr = lib.Protein(ctx, w.prot_xyz, w.prot_q, prm)
        prots.append(pr)
        pairs.append(dict(prot=pr.handle, lig_xyz=T(w.lig_xyz), lig_q=T(w.lig_q), quat=T(w.quat),
                          trans=T(w.trans),
                          E_out=torch.empty(w.P, dtype=torch.float64, device="cuda"),
                          flags_out=torch.empty(w.P, dtype=torch.uint8, device="cuda")))
    b, keep = lib.rs_batch_create(ctx.handle, pairs, autotune=True)
    yield lib, ctx, ws, prots, pairs, b
    lib.rs_batch_free(b)
    for p in prots:
        p.close()
    ctx.close()


def _plain(lib, prots, pairs):
    out = []
    for pr, p in zip(prots, pairs):
        E, f = pr.energies(p["lig_xyz"], p["lig_q"], p["quat"], p["trans"])
        out.append((E.cpu().numpy(), f.cpu().numpy()))
    return out


def test_batch_equals_plain_calls(setup):
    import torch
    lib, ctx, ws, prots, pairs, b = setup
    info = lib.rs_batch_get_info(b)
    assert info["npairs"] == len(ws)
    if info["mode"] == 0:
        assert info["nitems"] > 0 and info["threads"] in (128, 256)
    elif info["mode"] == 1:
        assert info["nchunks"] > 0 and info["warps_per_cta"] in (4, 8)
    else:
        assert info["mode"] in (2, 3) and info["streams"] in ((1,) if info["mode"] == 2 else (2, 4))
    lib.rs_batch_run(b)
    torch.cuda.synchronize()
    ref = _plain(lib, prots, pairs)
    for p, (E, f) in zip(pairs, ref):
        assert_paths_agree(p["E_out"].cpu().numpy(), E, p["flags_out"].cpu().numpy(), f)


@pytest.mark.parametrize("mode", [0, 2, 3, 4], ids=["cell-grouped", "per-block", "pair-by-pair", "streams"])
def test_both_batch_paths_equal_plain_calls(setup, mode):
    import torch
    lib, ctx, ws, prots, pairs, b = setup
    outs = [dict(p, E_out=torch.full_like(p["E_out"], float("nan")),
                 flags_out=torch.full_like(p["flags_out"], 255)) for p in pairs]
    b2, keep = lib.rs_batch_create(ctx.handle, outs, autotune=mode)
    try:
        info = lib.rs_batch_get_info(b2)
        assert info["mode"] == {0: 1, 2: 0, 3: 2, 4: 3}[mode]
        assert info["streams"] == (4 if mode == 4 else 1)
        lib.rs_batch_run(b2)
        torch.cuda.synchronize()
    finally:
        lib.rs_batch_free(b2)
    ref = _plain(lib, prots, pairs)
    for p, (E, f) in zip(outs, ref):
        assert_paths_agree(p["E_out"].cpu().numpy(), E, p["flags_out"].cpu().numpy(), f)
        if mode in (3, 4):
            # the pair-by-pair modes run each pair through the plain call's own dispatch
            assert np.array_equal(p["E_out"].cpu().numpy(), E)
            assert np.array_equal(p["flags_out"].cpu().numpy(), f)


def test_batch_replay_after_rewriting_poses(setup):
    import torch
    lib, ctx, ws, prots, pairs, b = setup
    rng = np.random.default_rng(5)
    for p in pairs:
        P = p["quat"].shape[0]
        if P:
            p["quat"].copy_(torch.as_tensor(W.shoemake_quaternions(rng, P), device="cuda"))
            p["trans"].mul_(1.02)
    lib.rs_batch_run(b)
    torch.cuda.synchronize()
    ref = _plain(lib, prots, pairs)
    for p, (E, f) in zip(pairs, ref):
        assert_paths_agree(p["E_out"].cpu().numpy(), E, p["flags_out"].cpu().numpy(), f)


def test_batch_pair_against_oracle(setup):
    import torch
    lib, ctx, ws, prots, pairs, b = setup
    k = 3
    w = ws[k]
    lib.rs_batch_run(b)
    torch.cuda.synchronize()
    quat, trans = pairs[k]["quat"].cpu().numpy(), pairs[k]["trans"].cpu().numpy()
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l, tucker_cap=w.tucker_cap)
    ref = O.pose_energies(m, w.lig_xyz, w.lig_q, quat, trans)
    assert_energies(pairs[k]["E_out"].cpu().numpy(), ref)
    assert_flags(pairs[k]["flags_out"].cpu().numpy(), ref)


def test_batch_rejects_unreduced_proteins(setup):
    import torch
    lib, ctx, ws, prots, pairs, b = setup
    w = ws[0]
    pr = lib.Protein(ctx, w.prot_xyz, w.prot_q,
                     lib.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=0))
    bad = dict(pairs[0])
    bad["prot"] = pr.handle
    with pytest.raises(lib.RSError) as ei:
        lib.rs_batch_create(ctx.handle, [bad], autotune=False)
    assert ei.value.status == lib.RS_ERR_UNSUPPORTED
    pr.close()
