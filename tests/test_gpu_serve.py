"""Serving: requests of different proteins, ligands and grid sizes through the request
loop give the same energies and flags alone and in any mix, bit for bit, and the same
as one plain rs_energy_poses call each (within the path tolerance where the two take
different W-form kernels); the small canonical case is checked against
the oracle.  Resident factors, eviction under a memory budget, injected allocation
failures, cancellation and bounded waits are exercised on the host side."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.parity import assert_energies, assert_flags, assert_paths_agree

pytestmark = pytest.mark.gpu


def _proteins(rng):
    # (N, n, tucker_cap): three Tucker ranks and grids, one unreduced canonical protein
    specs = [(900, 257, 8), (2200, 513, 16), (1500, 513, 20), (200, 257, 0)]
    out = []
    for N, n, cap in specs:
        prot, r_p = W.sphere_lattice(rng, N)
        zq = W.mixed_charges(rng, N, 0.3, 0.08)
        out.append(dict(xyz=prot, q=zq, r_p=r_p, n=n, cap=cap))
    return out


def _ligands(rng):
    ligs = []
    for L in (12, 47, 130):
        r_l = 5.0 * (L / 20.0) ** (1.0 / 3.0)
        ligs.append(dict(xyz=W.ball_uniform(rng, L, r_l), q=rng.normal(0.0, 0.3, L), r_l=r_l))
    return ligs


def _params(lib, pr, r_l_max):
    b = pr["r_p"] + 2 * r_l_max + 8
    return lib.rs_params_default(n=pr["n"], b=b, sigma=3.0, R_l=20, tucker_cap=pr["cap"])


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_26611_gb300 import lib
    rng = np.random.default_rng(41)
    prots, ligs = _proteins(rng), _ligands(rng)
    r_l_max = max(l["r_l"] for l in ligs)
    params = [_params(lib, p, r_l_max) for p in prots]
    # requests: (protein index, ligand index, poses)
    reqs = []
    for i in range(24):
        pi, li = int(rng.integers(0, 4)), int(rng.integers(0, 3))
        P = int(rng.integers(0, 900)) if i % 7 else 1
        pr, lg = prots[pi], ligs[li]
        quat = W.shoemake_quaternions(rng, P)
        trans = W.shell_translations(rng, P, pr["r_p"], pr["r_p"] + 2 * lg["r_l"] + 3)
        reqs.append(dict(pi=pi, li=li, quat=quat, trans=trans))
    # plain path: one rs_energy_poses call per request on separately built proteins
    ctx = lib.Context(0)
    plain_prots = [lib.Protein(ctx, p["xyz"], p["q"], prm) for p, prm in zip(prots, params)]
    plain = []
    for r in reqs:
        lg = ligs[r["li"]]
        E, f = lib.rs_energy_poses(ctx.handle, plain_prots[r["pi"]].handle, lg["xyz"], lg["q"],
                                   r["quat"], r["trans"])
        plain.append((np.asarray(E), np.asarray(f)))
    yield lib, prots, ligs, params, reqs, plain, plain_prots
    for p in plain_prots:
        p.close()
    ctx.close()


def _submit(lib, srv, prots, ligs, params, r, pid=None):
    pr, lg = prots[r["pi"]], ligs[r["li"]]
    return srv.submit(r["pi"] + 1 if pid is None else pid, pr["xyz"], pr["q"], params[r["pi"]],
                      lg["xyz"], lg["q"], r["quat"], r["trans"])


def test_same_alone_and_in_the_mix(setup):
    lib, prots, ligs, params, reqs, plain, _ = setup
    srv = lib.Server(0)
    try:
        x = 5
        alone = srv.wait(_submit(lib, srv, prots, ligs, params, reqs[x]))
        assert alone["status"] == lib.RS_OK, alone["message"]
        ids = [_submit(lib, srv, prots, ligs, params, r) for r in reqs]
        res = [srv.wait(i) for i in ids]
        st = srv.stats()
    finally:
        srv.close()
    for r, (E, f) in zip(res, plain):
        assert r["status"] == lib.RS_OK, r["message"]
        assert_paths_agree(r["E"], E, r["flags"], f)
        assert r["t_submit_ns"] <= r["t_admit_ns"] <= r["t_start_ns"] <= r["t_end_ns"]
    assert np.array_equal(res[x]["E"], alone["E"]) and np.array_equal(res[x]["flags"], alone["flags"])
    assert st["done"] == len(reqs) + 1 and st["failed"] == 0
    # one build per protein id; every other request found its protein resident
    assert st["builds"] == len({r["pi"] for r in reqs} | {reqs[x]["pi"]})
    assert st["cache_hits"] == len(reqs) + 1 - st["builds"]
    assert st["mean_requests_per_launch"] > 1.0  # requests were batched together


def test_canonical_request_matches_oracle(setup):
    lib, prots, ligs, params, reqs, plain, _ = setup
    pr, lg, prm = prots[3], ligs[0], params[3]
    rng = np.random.default_rng(3)
    quat = W.shoemake_quaternions(rng, 300)
    trans = W.shell_translations(rng, 300, pr["r_p"], pr["r_p"] + 2 * lg["r_l"] + 3)
    srv = lib.Server(0)
    try:
        res = srv.wait(srv.submit(0, pr["xyz"], pr["q"], prm, lg["xyz"], lg["q"], quat, trans))
        assert srv.stats()["cached_proteins"] == 0  # an anonymous protein is freed after use
    finally:
        srv.close()
    assert res["status"] == lib.RS_OK
    m = O.build_model(pr["xyz"], pr["q"], prm.n, prm.b, prm.sigma, prm.R_l, tucker_cap=0)
    ref = O.pose_energies(m, lg["xyz"], lg["q"], quat, trans)
    assert_energies(res["E"], ref)
    assert_flags(res["flags"], ref)


def test_eviction_under_a_memory_budget(setup):
    lib, prots, ligs, params, reqs, plain, plain_prots = setup
    big = max(p.info["device_bytes"] for p in plain_prots[:3])
    # room for about one protein: every switch of protein must evict the idle one
    srv = lib.Server(0, mem_budget_bytes=int(1.3 * big) + (4 << 20))
    try:
        order = [0, 1, 2, 0, 1, 2, 1]
        out = []
        for k in order:  # one at a time, so idle proteins must make room for the next
            i = next(i for i, r in enumerate(reqs) if r["pi"] == k and r["quat"].shape[0] > 1)
            out.append((i, srv.wait(_submit(lib, srv, prots, ligs, params, reqs[i]))))
        st = srv.stats()
    finally:
        srv.close()
    for i, res in out:
        assert res["status"] == lib.RS_OK, res["message"]
        assert_paths_agree(res["E"], plain[i][0], res["flags"], plain[i][1])
    assert st["evictions"] >= 1 and st["builds"] > 3
    assert st["used_bytes"] <= st["budget_bytes"] + big


def test_over_budget_and_injected_failures_fail_only_that_request(setup):
    lib, prots, ligs, params, reqs, plain, _ = setup
    i = next(i for i, r in enumerate(reqs) if r["pi"] == 1 and r["quat"].shape[0] > 1)
    r = reqs[i]
    srv = lib.Server(0, mem_budget_bytes=1 << 20)
    try:
        res = srv.wait(_submit(lib, srv, prots, ligs, params, r))
        assert res["status"] == lib.RS_ERR_OOM and "budget" in res["message"]
        assert srv.stats()["failed"] == 1
    finally:
        srv.close()
    srv = lib.Server(0, inject_alloc_failures=1)
    try:
        first = srv.wait(_submit(lib, srv, prots, ligs, params, r))
        second = srv.wait(_submit(lib, srv, prots, ligs, params, r))
        st = srv.stats()
    finally:
        srv.close()
    assert first["status"] == lib.RS_ERR_OOM and "allocation" in first["message"]
    assert second["status"] == lib.RS_OK
    assert_paths_agree(second["E"], plain[i][0], second["flags"], plain[i][1])
    assert st["failed"] == 1 and st["done"] == 1


def test_cancel_wait_timeout_and_empty_request(setup):
    lib, prots, ligs, params, reqs, plain, _ = setup
    srv = lib.Server(0, hold_builds=1)
    try:
        r = next(r for r in reqs if r["pi"] == 2 and r["quat"].shape[0] > 1)
        a = _submit(lib, srv, prots, ligs, params, r)
        b = _submit(lib, srv, prots, ligs, params, r)
        # the protein's build is held, so both stay queued: b can be cancelled and a
        # cannot have finished
        assert srv.cancel(b) == lib.RS_OK
        assert srv.cancel(b) == lib.RS_ERR_INVALID  # unknown now
        with pytest.raises(lib.RSError) as ei:
            lib.rs_serve_wait(srv.handle, a, 0)
        assert ei.value.status in (lib.RS_ERR_TIMEOUT,)
        srv.release_builds()
        res = srv.wait(a)
        assert res["status"] == lib.RS_OK
        assert srv.cancel(a) == lib.RS_ERR_INVALID  # finished and released
        empty = dict(r, quat=np.zeros((0, 4)), trans=np.zeros((0, 3)))
        e = srv.wait(_submit(lib, srv, prots, ligs, params, empty))
        assert e["status"] == lib.RS_OK and e["E"].shape == (0,)
        st = srv.stats()
        assert st["done"] == 2 and st["queued"] == 0
    finally:
        srv.close()
