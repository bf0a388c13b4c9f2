"""Pins of the oracle's finite-difference force (Sec. 3.3, Eq. differ_ligand) and of
its rigid-cluster resultants (Sec. 5.2, Eq. Field_Xcenter and Eq. Field_phi) against
closed forms, the Coulomb law, the exact adjoint and an exact grid symmetry.
CPU only."""
import numpy as np
import pytest

import oracle as O
import workloads as W


def _one_charge_model(x_m, z, n=65, b=16.0, sigma=1.0, R_l=12):
    return O.build_model(np.array([x_m]), np.array([z]), n, b, sigma, R_l)


def test_fd_at_nodes_closed_form():
    """A single ligand atom on a grid node, h = the grid step: x and x - h e_i are
    nodes, where the interpolant is exact, so F_i = q z (g(d_0) - g(d_i)) / h with
    g(r) = sum_{k long} a_k exp(-t_k^2 r^2) (no short range beyond r_c)."""
    x = O.grid_nodes(65, 16.0)
    x_m = np.array([x[20] + 0.37, x[31] - 0.81, x[26] + 0.13])
    z, q = 0.7, -1.3
    m = _one_charge_model(x_m, z)
    node = np.array([x[40], x[37], x[45]])
    assert np.linalg.norm(node - x_m) - m.h > m.table.r_c
    out = O.fd_forces(m, node[None, :], np.array([q]), np.zeros((1, 3)), node[None, :])
    tl, al = m.table.t[m.table.is_long], m.table.a[m.table.is_long]
    g = lambda p: (al * np.exp(-(tl * tl) * ((p - x_m) ** 2).sum())).sum()
    expect = np.array([q * z * (g(node) - g(node - m.h * e)) / m.h for e in np.eye(3)])
    assert out["h"] == m.h
    assert np.allclose(out["Fsum"][0], expect, rtol=1e-11, atol=0)
    # one atom sits at the centre: all of its force is translational
    assert np.array_equal(out["F0"][0], out["Fsum"][0])
    assert np.all(out["Fphi"][0] == 0.0) and np.all(out["M"][0] == 0.0)
    assert out["E"][0] == pytest.approx(q * z * g(node), rel=1e-13)


def test_fd_at_nodes_follows_coulomb():
    """The same quotient against the Coulomb law: the nodes carry only the sinc
    quadrature error (<= 3e-7 of 1/r here), so F_i matches
    q z (1/d_0 - 1/d_i) / h to that error times d/h."""
    x = O.grid_nodes(129, 32.0)
    x_m = np.array([0.21, -0.43, 0.05])
    z, q = 1.0, 0.6
    m = O.build_model(x_m[None, :], np.array([z]), 129, 32.0, 3.0, 20)
    rng = np.random.default_rng(4)
    for _ in range(6):
        node = x[rng.integers(70, 100, 3)]
        d0 = np.linalg.norm(node - x_m)
        d = np.array([np.linalg.norm(node - m.h * e - x_m) for e in np.eye(3)])
        out = O.fd_forces(m, node[None, :], np.array([q]), np.zeros((1, 3)), node[None, :])
        cl = q * z * (1 / d0 - 1 / d) / m.h
        # each value is within (quad_err + 1e-9) / r of q z / r (1e-9: the short-range
        # tail beyond r_c, which the long-range part carries)
        tol = 2.0 * (m.table.quad_err + 1e-9) * abs(q * z) / min(d0, d.min()) / m.h
        assert np.abs(out["Fsum"][0] - cl).max() <= tol
        # and the quotient points uphill in energy: F . (x - x_m) has the sign of -q z
        assert np.sign(out["Fsum"][0] @ (node - x_m)) == -np.sign(q * z)


@pytest.mark.parametrize("tucker", [0, 12])
def test_fd_inside_a_cell_equals_exact_adjoint(tucker):
    """Within one interpolation cell the trilinear interpolant is linear along each
    axis, so for a step that stays inside the cell the backward quotient is the exact
    derivative: Fsum = dE/dt and J_l(w)^T M = dE/dw of the adjoint (feasible poses,
    whose atoms keep more than r_c from the protein, where the short range is zero)."""
    w = W.plain_small(P=40)
    m = O.build_model(w.prot_xyz, w.prot_q, 129, w.b, w.sigma, w.R_l, tucker_cap=tucker)
    rv = W.random_rotvecs(np.random.default_rng(2), w.P)
    hfd = 1e-6
    x = O.posed_atoms(w.lig_xyz, O.rotvec_to_rot(rv), w.trans)
    s = (x + m.b) / m.h
    keep = (s - np.floor(s)).min(axis=(1, 2)) * m.h > 10 * hfd
    keep &= O.min_distances(m.prot_xyz, x.reshape(-1, 3)).reshape(w.P, -1).min(axis=1) > m.table.r_c + 1e-3
    assert keep.sum() >= 20
    rv, tr = rv[keep], w.trans[keep]
    fd = O.fd_forces(m, w.lig_xyz, w.lig_q, rv, tr, h=hfd)
    ex = O.pose_gradients(m, w.lig_xyz, w.lig_q, rv, tr)
    assert np.array_equal(fd["E"], ex["E"]) or np.allclose(fd["E"], ex["E"], rtol=1e-13)
    sc = np.abs(ex["dE_dt"]).max()
    # rounding of phi(x) - phi(x - h e): ~1e-16 |phi| / h
    tol = 1e-16 * np.abs(ex["S_ref"]).max() / hfd * 50
    assert np.abs(fd["Fsum"] - ex["dE_dt"]).max() <= tol, (np.abs(fd["Fsum"] - ex["dE_dt"]).max(), tol, sc)
    scw = np.abs(ex["dE_dw"]).max()
    assert np.abs(fd["dE_dw"] - ex["dE_dw"]).max() <= tol * 10, (np.abs(fd["dE_dw"] - ex["dE_dw"]).max(), scw)


def test_fd_projection_on_an_axis_symmetric_case():
    """Two ligand atoms at +-a e_x about the centre and one protein charge on the x
    axis; the charge's y and z are node coordinates and the atoms' lie half a step
    above them, so x and x - h e_y (x - h e_z) are mirror images about the charge's
    plane, on a grid that is symmetric about it: the y and z quotients vanish and
    each atom's force lies along x, i.e. along v_l.  Then F0 = Fsum, Fphi = 0 and
    M = 0 (Eq. Field_Xcenter takes all of it)."""
    x = O.grid_nodes(65, 16.0)
    h = x[1] - x[0]
    x_m = np.array([x[10] + 0.3, x[33], x[30]])
    m = _one_charge_model(x_m, 1.0)
    a = 1.7
    lig = np.array([[a, 0.0, 0.0], [-a, 0.0, 0.0]])
    t = np.array([[x[44] + 0.41 * h, x[33] + h / 2, x[30] + h / 2]])
    out = O.fd_forces(m, lig, np.array([0.8, -0.3]), np.zeros((1, 3)), t)
    F = out["Fsum"][0]
    assert abs(F[0]) > 1e-4 and abs(F[1]) < 1e-12 * abs(F[0]) and abs(F[2]) < 1e-12 * abs(F[0])
    assert np.allclose(out["F0"][0], F, rtol=1e-12, atol=1e-14 * abs(F[0]))
    assert np.abs(out["Fphi"][0]).max() < 1e-11 * abs(F[0])
    assert np.abs(out["M"][0]).max() < 1e-11 * abs(F[0])
    assert out["r0"] == pytest.approx(a, rel=1e-15)


def test_fd_projection_tangential_case():
    """The same pair rotated by w = (pi/2) e_z lies along y; with the protein charge
    far out on the x axis the forces are (nearly) perpendicular to the pair, so the
    tangential resultant carries them: F0 has no x part, Fphi has no y part, and
    r0 * (Fphi_x) relates to the moment M_z = a (F_{1,x} - F_{2,x}) as the moment of
    the tangential parts moved to radius r0 = a."""
    x = O.grid_nodes(65, 16.0)
    h = x[1] - x[0]
    zc = x[30] + h / 2
    x_m = np.array([x[5], x[32] + 0.11, zc])
    m = _one_charge_model(x_m, -1.0)
    a = 1.2
    lig = np.array([[a, 0.0, 0.0], [-a, 0.0, 0.0]])
    rv = np.array([[0.0, 0.0, np.pi / 2]])
    t = np.array([[x[40] + 0.3 * h, x[32] + 0.37 * h, zc]])
    q = np.array([0.9, 0.4])
    out = O.fd_forces(m, lig, q, rv, t)
    # per-atom forces from single-atom calls (an atom alone sits at its own centre)
    R = O.rotvec_to_rot(rv)[0]
    ry = (R @ lig.T).T
    Fl = [O.fd_forces(m, np.zeros((1, 3)), q[l:l + 1], np.zeros((1, 3)), (t[0] + ry[l])[None, :])["Fsum"][0]
          for l in range(2)]
    # v_1 = +e_y, v_2 = -e_y: radial = y parts, tangential = x and z parts
    assert np.allclose(out["F0"][0], [0.0, Fl[0][1] + Fl[1][1], 0.0], rtol=1e-12, atol=1e-15)
    assert np.allclose(out["Fphi"][0], [Fl[0][0] + Fl[1][0], 0.0, Fl[0][2] + Fl[1][2]], rtol=1e-12, atol=1e-15)
    Mz = a * (-Fl[0][0] + Fl[1][0])  # r_1 x F_1 + r_2 x F_2 with r_1 = a e_y, r_2 = -a e_y
    assert out["M"][0][2] == pytest.approx(Mz, rel=1e-12)
    assert np.allclose(out["Fsum"][0], Fl[0] + Fl[1], rtol=1e-12, atol=1e-15)


def test_fd_cyclic_axis_permutation_exact():
    """A cyclic permutation of the axes maps the node grid onto itself and each
    backward difference onto another one; applied jointly to the protein, the
    ligand and the translation, every resultant permutes as a vector."""
    w = W.plain_small(P=5)
    S = np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]], dtype=np.float64)  # (x,y,z) -> (z,x,y)
    rv = W.random_rotvecs(np.random.default_rng(9), 5)
    m0 = O.build_model(w.prot_xyz, w.prot_q, 129, w.b, w.sigma, w.R_l, tucker_cap=10)
    m1 = O.build_model(w.prot_xyz @ S.T, w.prot_q, 129, w.b, w.sigma, w.R_l, tucker_cap=10)
    a = O.fd_forces(m0, w.lig_xyz, w.lig_q, rv, w.trans)
    # R' = S R S^T is exp of [S w]x; the ligand frame maps by S
    b = O.fd_forces(m1, w.lig_xyz @ S.T, w.lig_q, rv @ S.T, w.trans @ S.T)
    sc = np.abs(a["Fsum"]).max()
    assert np.abs(a["E"] - b["E"]).max() <= 1e-11 * np.abs(a["E"]).max()
    for k in ("Fsum", "F0", "Fphi", "M", "dE_dw"):
        assert np.abs(a[k] @ S.T - b[k]).max() <= 1e-9 * sc, k
