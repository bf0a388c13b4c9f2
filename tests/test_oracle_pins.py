"""Pins of the FP64 oracle against mathematics that does not come from the oracle:
closed forms, brute force on the full n^3 tensor, exact symmetries, error bounds
and finite differences.  CPU only."""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.interpolate import RegularGridInterpolator

import oracle as O
import workloads as W


# --------------------------------------------------------------------------- sinc
def test_sinc_substitution_identity():
    """(1/sqrt(pi)) int_R cosh(u) exp(-rho^2 sinh^2 u) du = 1/rho: the integral the
    quadrature discretises (Sec. 2, Gaussian representation of 1/r)."""
    for rho in (0.01, 0.3, 1.0):
        U = math.asinh(10.0 / rho) + 1.0     # integrand < e^-100 beyond
        val, _ = integrate.quad(lambda u: math.cosh(u) * math.exp(-(rho * math.sinh(u)) ** 2),
                                -U, U, limit=400, epsabs=0, epsrel=1e-12)
        assert abs(val / math.sqrt(math.pi) * rho - 1.0) < 1e-9


@pytest.mark.parametrize("b,R_l,tol", [(32.0, 20, 1e-6), (64.0, 20, 4e-6)])
def test_sinc_table_reproduces_inverse_r(b, R_l, tol):
    """sum_k a_k exp(-t_k^2 r^2) = 1/r on [r_min, 2 sqrt(3) b] (Sec. 2, Eq. sinc and
    its error bound): checked against the closed form 1/r on points the table
    builder never sampled."""
    tab = O.sinc_table(b, 3.0, R_l)
    r = np.random.default_rng(5).uniform(tab.r_min, tab.box_len, 5000)
    s = (tab.a[None, :] * np.exp(-np.outer(r * r, tab.t ** 2))).sum(axis=1)
    err = np.abs(s * r - 1.0).max()
    assert err < tol
    assert err <= tab.quad_err * 1.0001 + 1e-15
    # structure: t_0 = 0, t increasing, positive weights, long part = R_l widest terms
    assert tab.t[0] == 0.0 and np.all(np.diff(tab.t) > 0) and np.all(tab.a > 0)
    assert tab.is_long.sum() == R_l and np.all(tab.is_long[:R_l])
    # narrowest long-range Gaussian: t * sigma = tau = 4 (sigma bounds the support)
    assert abs(tab.t[R_l - 1] * 3.0 - 4.0) < 1e-9


def test_sinc_error_decays_with_step():
    """Exponential convergence in the number of terms (Sec. 2 bound C e^{-beta sqrt K})."""
    e = [O.sinc_table(32.0, 3.0, R).quad_err for R in (8, 12, 16, 20)]
    assert all(e[i + 1] < 0.5 * e[i] for i in range(3))


def test_short_range_cutoff_definition():
    tab = O.sinc_table(32.0, 3.0, 20)
    ts, as_ = tab.t[~tab.is_long], tab.a[~tab.is_long]
    f = lambda r: r * (as_ * np.exp(-(r * ts) ** 2)).sum()
    assert f(tab.r_c) <= 1e-9 * 1.000001
    assert f(tab.r_c * 0.999) > 1e-9
    assert 2.0 < tab.r_c < 3.0      # inside sigma: feasible poses get no short-range term


# ----------------------------------------------------------- full-tensor checks
def _full_long_tensor(model):
    """P_l[i,j,k] = sum_m z_m sum_{k long} a_k exp(-t_k^2 |x_ijk - x_m|^2): the
    collective long-range potential on the grid from its 3-D definition
    (Sec. 2, Eq. Long-Range_Sum), without using separability."""
    x = O.grid_nodes(model.n, model.b)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    tl = model.table.t[model.table.is_long]
    al = model.table.a[model.table.is_long]
    T = np.zeros(X.shape)
    for m in range(model.prot_xyz.shape[0]):
        d2 = (X - model.prot_xyz[m, 0]) ** 2 + (Y - model.prot_xyz[m, 1]) ** 2 + (Z - model.prot_xyz[m, 2]) ** 2
        for tk, ak in zip(tl, al):
            T += model.prot_q[m] * ak * np.exp(-tk * tk * d2)
    return T


def test_per_factor_interpolation_equals_trilinear_on_full_tensor():
    w = W.tiny(seed=1, N=3, n=17, b=8.0)
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l)
    T = _full_long_tensor(m)
    x = O.grid_nodes(m.n, m.b)
    interp = RegularGridInterpolator((x, x, x), T, method="linear")
    pts = np.random.default_rng(2).uniform(-m.b * 0.99, m.b * 0.99, (200, 3))
    ref = interp(pts)
    pl, _, _, _ = O.potential(m, pts)
    assert np.abs(pl - ref).max() <= 1e-12 * np.abs(T).max()


def test_node_value_closed_form():
    """A point on a grid node gets z * sum_{k long} a_k exp(-t_k^2 d^2)."""
    w = W.tiny(seed=3, N=1, n=33, b=8.0)
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l)
    x = O.grid_nodes(m.n, m.b)
    node = np.array([[x[5], x[20], x[29]], [x[16], x[16], x[3]]])
    d2 = ((node - w.prot_xyz[0]) ** 2).sum(axis=1)
    tl, al = m.table.t[m.table.is_long], m.table.a[m.table.is_long]
    expect = w.prot_q[0] * (al[None, :] * np.exp(-np.outer(d2, tl * tl))).sum(axis=1)
    pl, _, _, _ = O.potential(m, node)
    assert np.allclose(pl, expect, rtol=1e-13, atol=0)


def test_brute_force_energy_tiny():
    """E_RS of a few poses against explicit loops: trilinear interpolation of the full
    tensor by its 8 corners, short range by an explicit pair loop with the cutoff."""
    w = W.tiny(seed=4, N=3, L=2, P=4, n=17, b=8.0, sigma=0.5)
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l)
    T = _full_long_tensor(m)
    h = m.h
    ts, as_ = m.table.t[~m.table.is_long], m.table.a[~m.table.is_long]
    res = O.pose_energies(m, w.lig_xyz, w.lig_q, w.quat, w.trans)
    R = O.quat_to_rot(w.quat)
    y = w.lig_xyz - w.lig_xyz.mean(axis=0)
    for p in range(w.P):
        E = 0.0
        for j in range(w.L):
            xj = R[p] @ y[j] + w.trans[p]
            s = (xj + m.b) / h
            i0 = np.minimum(np.floor(s).astype(int), m.n - 2)
            f = s - i0
            val = 0.0
            for c in range(8):
                o = [(c >> a) & 1 for a in range(3)]
                wgt = 1.0
                for a in range(3):
                    wgt *= f[a] if o[a] else 1 - f[a]
                val += wgt * T[i0[0] + o[0], i0[1] + o[1], i0[2] + o[2]]
            for mm in range(w.N):
                d = math.sqrt(((xj - w.prot_xyz[mm]) ** 2).sum())
                if d < m.table.r_c:
                    val += w.prot_q[mm] * sum(ak * math.exp(-(tk * d) ** 2) for tk, ak in zip(ts, as_))
            E += w.lig_q[j] * val
        assert abs(E - res["E"][p]) <= 1e-12 * max(1.0, abs(E))


# ------------------------------------------------------------------ invariants
def _signed_perms():
    import itertools
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1.0, -1.0), repeat=3):
            S = np.zeros((3, 3))
            for r, c in enumerate(perm):
                S[r, c] = signs[r]
            yield S


def test_octahedral_symmetry_exact():
    """The node grid is symmetric under the 48 signed axis permutations; applying
    one jointly to both clusters leaves E_RS unchanged."""
    w = W.plain_small(P=6)
    x = O.posed_atoms(w.lig_xyz, O.quat_to_rot(w.quat), w.trans)
    base = None
    for S in _signed_perms():
        m = O.build_model(w.prot_xyz @ S.T, w.prot_q, w.n, w.b, w.sigma, w.R_l)
        E = O.energies_from_atoms(m, x @ S.T, w.lig_q)["E"]
        if base is None:
            base = E
        else:
            assert np.abs(E - base).max() <= 1e-12 * np.abs(base).max()


def test_translation_by_grid_steps_exact():
    w = W.plain_small(P=6)
    m0 = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l)
    x = O.posed_atoms(w.lig_xyz, O.quat_to_rot(w.quat), w.trans)
    E0 = O.energies_from_atoms(m0, x, w.lig_q)["E"]
    shift = np.array([3, -2, 1]) * m0.h
    m1 = O.build_model(w.prot_xyz + shift, w.prot_q, w.n, w.b, w.sigma, w.R_l)
    E1 = O.energies_from_atoms(m1, x + shift, w.lig_q)["E"]
    assert np.abs(E1 - E0).max() <= 1e-11 * np.abs(E0).max()


def test_quaternion_sign_and_charge_sign():
    w = W.plain_small(P=20)
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l)
    a = O.pose_energies(m, w.lig_xyz, w.lig_q, w.quat, w.trans)["E"]
    b = O.pose_energies(m, w.lig_xyz, w.lig_q, -w.quat, w.trans)["E"]
    c = O.pose_energies(m, w.lig_xyz, -w.lig_q, w.quat, w.trans)["E"]
    assert np.array_equal(a, b)
    assert np.allclose(c, -a, rtol=0, atol=1e-15)


def test_rs_energy_within_coulomb_error_bound():
    """|E_RS - E_C| <= sum_{j,m} |q_j z_m| (eps_q / r_jm + 3 h^2/4 sum_{k long} a_k t_k^2
    + cutoff tail): quadrature error (Sec. 2 bound) plus the trilinear interpolation
    error of the long-range kernel (h^2/8 per axis times max |second derivative|
    <= 2 a_k t_k^2), for feasible poses, also after a joint continuous rotation."""
    w = W.plain_small(P=60)
    rng = np.random.default_rng(9)
    Rj = O.quat_to_rot(W.shoemake_quaternions(rng, 1))[0]
    for rot in (np.eye(3), Rj):
        prot = w.prot_xyz @ rot.T
        m = O.build_model(prot, w.prot_q, w.n, w.b, w.sigma, w.R_l)
        x = O.posed_atoms(w.lig_xyz, O.quat_to_rot(w.quat), w.trans) @ rot.T
        r = O.energies_from_atoms(m, x, w.lig_q)
        d = np.linalg.norm(x[:, :, None, :] - prot[None, None], axis=-1)
        Ec = (w.lig_q[None, :, None] * w.prot_q[None, None, :] / d).sum(axis=(1, 2))
        tab = m.table
        tl, al = tab.t[tab.is_long], tab.a[tab.is_long]
        interp = 0.75 * m.h ** 2 * (al * tl * tl).sum()
        qz = np.abs(w.lig_q)[None, :, None] * np.abs(w.prot_q)[None, None, :]
        bound = (qz * (tab.quad_err / d + interp + 1e-9 / tab.r_c)).sum(axis=(1, 2))
        feas = r["flags"] == 0
        assert feas.sum() > 10
        assert np.all(np.abs(r["E"] - Ec)[feas] <= bound[feas])


# ------------------------------------------------------------------- reduction
def test_reduction_full_rank_is_exact():
    w = W.tiny(seed=6, N=3, n=17, b=8.0, P=10)
    m_c = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l)
    m_t = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l, tucker_cap=17, eps_r=0.0)
    assert m_t.ranks == (17, 17, 17)
    a = O.pose_energies(m_c, w.lig_xyz, w.lig_q, w.quat, w.trans)["E"]
    b = O.pose_energies(m_t, w.lig_xyz, w.lig_q, w.quat, w.trans)["E"]
    assert np.abs(a - b).max() <= 1e-11 * np.abs(a).max()


def test_reduction_core_is_projection_of_full_tensor():
    """beta = P_l x1 V1^T x2 V2^T x3 V3^T with P_l built from its 3-D definition, and
    V^(l) satisfies Z Z^T V = V diag(s^2) (left singular vectors of the weighted
    factor matrix)."""
    w = W.tiny(seed=7, N=3, n=17, b=8.0)
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l, tucker_cap=5,
                      keep_canonical=True)
    T = _full_long_tensor(m)
    proj = np.einsum("ijk,ia,jb,kc->abc", T, m.V[0], m.V[1], m.V[2])
    assert np.abs(proj - m.beta).max() <= 1e-11 * np.abs(m.beta).max()
    wgt = np.abs(m.xi) ** (1 / 3)
    for ax in range(3):
        Z = m.U[ax] * wgt[None, :]
        G = Z @ Z.T
        s2 = m.svals[ax][: m.V[ax].shape[1]] ** 2
        res = G @ m.V[ax] - m.V[ax] * s2[None, :]
        assert np.abs(res).max() <= 1e-10 * s2[0]
        assert np.allclose(m.V[ax].T @ m.V[ax], np.eye(m.V[ax].shape[1]), atol=1e-12)


def test_reduction_error_bound():
    """|phi_can(x) - phi_tucker(x)| <= ||P - P_r||_F <= sum_l (sum_{i>r_l} s_i^2)^(1/2)
    prod_{l' != l} ||Z^(l')||_2 (projector splitting; ||A (.) B||_2 <= ||A||_2 ||B||_2;
    trilinear weights have unit-bounded Frobenius norm)."""
    w = W.plain_small(P=40)
    m = O.build_model(w.prot_xyz, w.prot_q, 65, w.b, w.sigma, w.R_l, tucker_cap=8,
                      keep_canonical=True)
    tails = [math.sqrt((s[m.V[ax].shape[1]:] ** 2).sum()) for ax, s in enumerate(m.svals)]
    norms = [s[0] for s in m.svals]
    bound = sum(tails[ax] * np.prod([norms[o] for o in range(3) if o != ax]) for ax in range(3))
    x = O.posed_atoms(w.lig_xyz, O.quat_to_rot(w.quat), w.trans).reshape(-1, 3)
    m_c = O.RSModel("canonical", m.n, m.b, m.sigma, m.table, m.prot_xyz, m.prot_q, U=m.U, xi=m.xi)
    a, _, _, _ = O.potential(m_c, x)
    b, _, _, _ = O.potential(m, x)
    assert np.abs(a - b).max() <= bound
    assert np.abs(a - b).max() > 0


def test_reduced_rank_grows_slowly_with_N():
    """Theorem 2.2: the epsilon-rank of the long-range part is almost independent of N."""
    rng = np.random.default_rng(11)
    ranks = []
    for N in (20, 80, 320):
        prot = W.ball_uniform(rng, N, 10.0)
        zq = rng.normal(0, 0.3, N)
        tab = O.sinc_table(16.0, 3.0, 12)
        U, xi = O.long_range_factors(prot, zq, tab, 129, 16.0)
        wgt = np.abs(xi) ** (1 / 3)
        s = np.linalg.svd(U[0] * wgt[None, :], compute_uv=False)
        ranks.append(int((s > 1e-6 * s[0]).sum()))
    # 16x more atoms: the rank grows by well under 2x and stays far below N * R_l
    assert ranks[2] < 1.5 * ranks[0] and ranks[2] < 0.05 * 320 * 12


# -------------------------------------------------------------------- gradients
def _fd_grad(fn, rotvec, trans, eps_t=1e-4, eps_w=1e-4):
    P = rotvec.shape[0]
    gt, gw = np.zeros((P, 3)), np.zeros((P, 3))
    for a in range(3):
        e = np.zeros(3); e[a] = eps_t
        gt[:, a] = (fn(rotvec, trans + e) - fn(rotvec, trans - e)) / (2 * eps_t)
        e = np.zeros(3); e[a] = eps_w
        gw[:, a] = (fn(rotvec + e, trans) - fn(rotvec - e, trans)) / (2 * eps_w)
    return gt, gw


def _rv2q(w):
    th = np.linalg.norm(w, axis=1)
    s = np.where(th > 0, np.sin(th / 2) / np.where(th > 0, th, 1), 0.5)
    return np.concatenate([np.cos(th / 2)[:, None], w * s[:, None]], axis=1)


def test_coulomb_gradient_matches_fd():
    w = W.plain_small(P=12)
    rv = W.random_rotvecs(np.random.default_rng(1), 12)
    E, dt, dw = O.coulomb_gradients(w.prot_xyz, w.prot_q, w.lig_xyz, w.lig_q, rv, w.trans)
    fn = lambda r, t: O.coulomb_energies(w.prot_xyz, w.prot_q, w.lig_xyz, w.lig_q, _rv2q(r), t)
    ft, fw = _fd_grad(fn, rv, w.trans)
    assert np.allclose(E, fn(rv, w.trans), rtol=1e-12)
    assert np.abs(dt - ft).max() <= 1e-6 * np.abs(dt).max()
    assert np.abs(dw - fw).max() <= 1e-6 * np.abs(dw).max()


@pytest.mark.parametrize("tucker", [0, 12])
def test_rs_gradient_matches_fd(tucker):
    """Exact adjoint of the piecewise-trilinear energy vs central differences,
    on poses whose atoms stay away from grid planes by more than the FD step."""
    w = W.plain_small(P=60)
    m = O.build_model(w.prot_xyz, w.prot_q, 129, w.b, w.sigma, w.R_l, tucker_cap=tucker)
    rv = W.random_rotvecs(np.random.default_rng(2), w.P)
    R = O.rotvec_to_rot(rv)
    x = O.posed_atoms(w.lig_xyz, R, w.trans)
    s = (x + m.b) / m.h
    gap = np.abs(s - np.round(s)).min(axis=(1, 2)) * m.h
    keep = gap > 5e-3
    assert keep.sum() >= 5
    rv, tr = rv[keep], w.trans[keep]
    g = O.pose_gradients(m, w.lig_xyz, w.lig_q, rv, tr)
    fn = lambda r, t: O.pose_energies(m, w.lig_xyz, w.lig_q, _rv2q(r), t)["E"]
    ft, fw = _fd_grad(fn, rv, tr)
    assert np.allclose(g["E"], fn(rv, tr), rtol=1e-12, atol=1e-15)
    sc = np.maximum(np.abs(g["dE_dt"]).max(), np.abs(g["dE_dw"]).max())
    assert np.abs(g["dE_dt"] - ft).max() <= 1e-6 * sc
    assert np.abs(g["dE_dw"] - fw).max() <= 1e-6 * sc


def test_left_jacobian_first_order():
    rng = np.random.default_rng(3)
    w = W.random_rotvecs(rng, 5, 3.0)
    d = rng.normal(size=(5, 3)) * 1e-6
    lhs = O.rotvec_to_rot(w + d)
    J = O.left_jacobian(w)
    from scipy.linalg import expm
    for p in range(5):
        jd = J[p] @ d[p]
        K = np.array([[0, -jd[2], jd[1]], [jd[2], 0, -jd[0]], [-jd[1], jd[0], 0]])
        rhs = expm(K) @ O.rotvec_to_rot(w[p:p + 1])[0]
        assert np.abs(lhs[p] - rhs).max() < 1e-11
    # Rodrigues against the matrix exponential
    for p in range(5):
        v = w[p]
        K = np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])
        assert np.allclose(expm(K), O.rotvec_to_rot(w[p:p + 1])[0], atol=1e-13)


def test_quaternion_matches_rotvec():
    rng = np.random.default_rng(4)
    w = W.random_rotvecs(rng, 7)
    assert np.allclose(O.quat_to_rot(_rv2q(w)), O.rotvec_to_rot(w), atol=1e-13)


# --------------------------------------------------------------------- flags, pgd
def test_flags_brute_force():
    w = W.plain_small(P=200)
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l)
    x = O.posed_atoms(w.lig_xyz, O.quat_to_rot(w.quat), w.trans)
    d = np.linalg.norm(x[:, :, None, :] - w.prot_xyz[None, None], axis=-1).min(axis=(1, 2))
    r = O.energies_from_atoms(m, x, w.lig_q)
    assert np.array_equal((r["flags"] & O.FLAG_CLASH) > 0, d < w.sigma)
    assert 0 < (d < w.sigma).sum() < w.P


def test_out_of_grid_flag_and_clamp():
    w = W.tiny(seed=8, N=2, n=17, b=8.0)
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l)
    x = np.array([[[9.0, 0.0, 0.0]], [[8.0, 0.0, 0.0]], [[7.9, 0.0, 0.0]]])
    r = O.energies_from_atoms(m, x, np.array([1.0]))
    assert r["flags"][0] & O.FLAG_OUT_OF_GRID
    assert not (r["flags"][1] & O.FLAG_OUT_OF_GRID)
    assert not (r["flags"][2] & O.FLAG_OUT_OF_GRID)
    assert abs(r["E_long"][0] - r["E_long"][1]) < 1e-15   # clamped to the edge node


def test_pgd_step_monotone_and_feasible():
    w = W.plain_small(P=40)
    m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l)
    rv = W.random_rotvecs(np.random.default_rng(5), w.P)
    st = O.pgd_step(m, w.lig_xyz, w.lig_q, rv, w.trans)
    assert np.all(st["E"] <= st["E_start"])
    acc = st["accepted"] >= 0
    assert acc.sum() > 0
    q = _rv2q(st["rotvec"][acc])
    r = O.pose_energies(m, w.lig_xyz, w.lig_q, q, st["trans"][acc])
    assert np.all(r["flags"] == 0)
    assert np.allclose(r["E"], st["E"][acc], rtol=1e-12)


def test_topk_feasible():
    E = np.array([3.0, -1.0, -5.0, 2.0, -7.0])
    f = np.array([0, 0, 1, 0, 0], dtype=np.uint8)
    assert list(O.feasible_topk(E, f, 3)) == [4, 1, 3]
