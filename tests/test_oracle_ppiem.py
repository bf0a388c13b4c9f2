"""Pins of the oracle's pose scan (Algorithm PPIEM, Sec. 3.4 steps A0-A7): the contact
offset of step A3 against distances from a k-d tree, closed forms, the direction grid,
and the minima of a scan whose answer follows from symmetry.  CPU only."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def test_direction_grid():
    U = O.ppiem_directions(6, 12)
    assert U.shape == (72, 3)
    assert np.allclose(np.linalg.norm(U, axis=1), 1.0, atol=1e-15)
    # index a * n_phi + b: polar angle (a + 1/2) pi / 6, azimuth 2 pi b / 12
    a, b = 4, 7
    th, ph = (a + 0.5) * math.pi / 6, b * 2 * math.pi / 12
    assert np.allclose(U[a * 12 + b], [math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    # no direction is repeated and the set is symmetric under z -> -z
    assert len({tuple(np.round(u, 12)) for u in U}) == 72
    Um = U * np.array([1, 1, -1])
    assert all(np.abs(U - v).sum(axis=1).min() < 1e-12 for v in Um)


def test_euler_grid_quaternions():
    q = W.euler_grid_quaternions(4)
    assert q.shape == (32, 4) and np.allclose(np.linalg.norm(q, axis=1), 1.0)
    # ZYZ: R = Rz(alpha) Ry(beta) Rz(gamma), alpha slowest
    Rz = lambda t: np.array([[math.cos(t), -math.sin(t), 0], [math.sin(t), math.cos(t), 0], [0, 0, 1]])
    Ry = lambda t: np.array([[math.cos(t), 0, math.sin(t)], [0, 1, 0], [-math.sin(t), 0, math.cos(t)]])
    st = math.pi / 2
    i, k, g = 3, 1, 2
    R = Rz(i * st) @ Ry((k + 0.5) * st) @ Rz(g * st)
    assert np.allclose(O.quat_to_rot(q[(i * 2 + k) * 4 + g][None])[0], R, atol=1e-15)


def test_contact_on_the_axis_closed_form():
    # one protein atom 5 A out along u, one ligand atom: contact at s = 5 + sigma
    u = np.array([[0.6, 0.0, 0.8]])
    x_P = np.array([1.0, -2.0, 0.5])
    s = O.contact_offsets(x_P + 5.0 * u, 3.0, np.zeros((1, 3)), np.array([[1.0, 0, 0, 0]]), x_P, u)
    assert s[0] == pytest.approx(8.0, abs=1e-13)
    # an atom 4 A off the line is never met: no contact
    off = x_P + 5.0 * u + 4.0 * np.array([0.8, 0.0, -0.6])
    s = O.contact_offsets(off, 3.0, np.zeros((1, 3)), np.array([[1.0, 0, 0, 0]]), x_P, u)
    assert s[0] == -np.inf


def test_contact_is_first_touch_from_outside():
    """At s* the closest ligand-protein distance is sigma; it stays >= sigma for every
    s > s* (checked on a grid out to 40 A) and drops below sigma just inside s*."""
    w = W.plain_small(P=1)
    rng = np.random.default_rng(3)
    quat = W.shoemake_quaternions(rng, 12)
    u = O.ppiem_directions(4, 6)[rng.integers(0, 24, 12)]
    x_P = w.prot_xyz.mean(axis=0)
    s = O.contact_offsets(w.prot_xyz, w.sigma, w.lig_xyz, quat, x_P, u)
    assert np.all(np.isfinite(s))

    def dmin(p, sv):
        x = O.posed_atoms(w.lig_xyz, O.quat_to_rot(quat[p:p + 1]), (x_P + sv * u[p])[None])[0]
        return O.min_distances(w.prot_xyz, x).min()

    for p in range(12):
        assert dmin(p, s[p]) == pytest.approx(w.sigma, abs=1e-9)
        assert dmin(p, s[p] - 1e-3) < w.sigma
        for sv in s[p] + np.linspace(1e-6, 40.0, 400):
            assert dmin(p, sv) >= w.sigma - 1e-12


def test_scan_finds_the_symmetric_minimum():
    """Protein: +1 at the origin and -1 at (6, 0, 0); ligand: one +1 atom.  The scan's
    lowest local minimum faces the negative charge (azimuth 0, polar angle next to
    pi/2); the two polar rows beside the equator are mirror images (the node grid and
    the protein are symmetric under z -> -z), so the tie goes to the lower index."""
    m = O.build_model(np.array([[0.0, 0, 0], [6.0, 0, 0]]), np.array([1.0, -1.0]), 65, 16.0, 3.0, 12)
    for nt, nph in ((6, 12), (8, 16)):
        r = O.ppiem_scan(m, np.zeros((1, 3)), np.array([1.0]), np.array([[1.0, 0, 0, 0]]), nt, nph)
        mins = np.nonzero(r["is_min"])[0]
        lowest = mins[np.argmin(r["E_best"][mins])]
        assert lowest == (nt // 2 - 1) * nph
        mirror = (nt // 2) * nph
        assert r["E_best"][lowest] == r["E_best"][mirror] and not r["is_min"][mirror]
        # the pose returned is the contact pose of that direction, just outside sigma
        x = r["x_P"] + (r["s"][lowest, 0] + 1e-6 * 3.0) * r["dirs"][lowest]
        d = O.min_distances(m.prot_xyz, x[None])[0]
        assert 3.0 < d < 3.0 + 1e-5
        assert r["E"][lowest, 0] < 0 and r["flags"][lowest, 0] == 0


def test_scan_directions_without_contact():
    # a lone protein atom: lines farther than sigma from it never touch
    m = O.build_model(np.array([[0.0, 0, 0]]), np.array([1.0]), 33, 8.0, 1.0, 8)
    lig = np.array([[2.0, 0, 0], [-2.0, 0, 0]])
    r = O.ppiem_scan(m, lig, np.array([0.3, -0.3]), np.array([[1.0, 0, 0, 0]]), 4, 8)
    none = ~np.isfinite(r["s"][:, 0])
    assert none.any() and (~none).any()
    assert np.all(r["flags"][none, 0] == 4) and np.all(np.isinf(r["E"][none, 0]))
    assert np.all(r["rot_best"][none] == -1)
