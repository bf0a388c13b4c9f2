"""Pins of the oracle's projected-gradient step (Sec. 3.4, Eq. Energy_Min, with the
step rule read as: normalised steps of 0.1 A in translation and 0.02 rad in rotation,
at most five halvings, accept the first trial that is feasible with E_trial <= E,
else keep the pose).

Nothing here uses the oracle's own gradient.  Step directions come from central
differences of the pose energy (itself pinned by brute force elsewhere) and from
exact symmetry: a protein charge on the mid-plane y = h/2 of a grid cell makes the
grid's trilinear interpolant symmetric under y -> h - y, and a function linear in y
on [0, h] with equal end values is constant, so inside that cell the gradient has
no y (or z) component and the trial points, their distances to the protein and the
accepted halving level follow from one-dimensional geometry.  CPU only."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O

N_GRID, B, SIGMA, R_L = 65, 8.0, 3.0, 20     # h = 0.25 A
H = 2 * B / (N_GRID - 1)
ETA_T, ETA_R, MAX_HALVINGS = 0.1, 0.02, 5     # the step rule's constants


def _model(xyz, q):
    return O.build_model(np.asarray(xyz, float), np.asarray(q, float), N_GRID, B, SIGMA, R_L)


def _quat(w):
    """Rotation vector -> unit quaternion (w, x, y, z), through scipy (scalar last)."""
    x = Rotation.from_rotvec(np.atleast_2d(w)).as_quat()
    return np.concatenate([x[:, 3:], x[:, :3]], axis=1)


def _energy(m, lig, lq, w, t):
    r = O.pose_energies(m, lig, lq, _quat(w), np.atleast_2d(t))
    return r["E"][0], r["flags"][0]


def _fd_grad(m, lig, lq, w, t, d=1e-6):
    """Central differences of the pose energy in (t, w)."""
    g = np.zeros(6)
    for k in range(6):
        e = np.zeros(6)
        e[k] = d
        ep = _energy(m, lig, lq, w + e[3:], t + e[:3])[0]
        em = _energy(m, lig, lq, w - e[3:], t - e[:3])[0]
        g[k] = (ep - em) / (2 * d)
    return g[:3], g[3:]


def _step(m, lig, lq, w, t):
    st = O.pgd_step(m, lig, lq, np.atleast_2d(w), np.atleast_2d(t))
    return {k: (v[0] if isinstance(v, np.ndarray) else v) for k, v in st.items()}


def _single_charge_case(gap):
    """One protein charge +1 at the cell centre (h/2, h/2, h/2) and a one-atom ligand
    of charge -1 on the line y = z = h/2 + const inside the same y/z cell, at distance
    sigma + gap from the charge.  The gradient points along +x (attraction), so every
    trial moves the atom straight towards the charge by 0.1 * 2^-s."""
    c = np.full(3, H / 2)
    m = _model([c], [1.0])
    dy, dz = -0.02, 0.03
    dx = np.sqrt((SIGMA + gap) ** 2 - dy * dy - dz * dz)
    t = c + np.array([dx, dy, dz])
    return m, np.zeros((1, 3)), np.array([-1.0]), t, c


def _trial_distance(t, c, s):
    return np.linalg.norm(t - np.array([ETA_T * 0.5 ** s, 0, 0]) - c)


def test_step_is_normalised_gradient_descent():
    """A full step is taken when it is feasible and lowers E: the translation moves
    by exactly 0.1 A against dE/dt and the rotation vector by exactly 0.02 rad
    against dE/dw (directions from central differences of the energy)."""
    prot = [[1.2, -0.7, 0.4], [-2.3, 1.1, -0.6], [0.3, 2.2, 1.7]]
    m = _model(prot, [1.0, -0.6, 0.8])
    lig = np.array([[0.9, 0.1, -0.3], [-0.8, -0.2, 0.4]])
    lq = np.array([-0.7, 0.45])
    w = np.array([0.31, -0.52, 0.17])
    t = np.array([4.61, 2.73, 3.37])
    st = _step(m, lig, lq, w, t)
    assert st["accepted"] == 0
    gt, gw = _fd_grad(m, lig, lq, w, t)
    assert np.linalg.norm(gt) > 1e-3 and np.linalg.norm(gw) > 1e-3
    dt, dw = st["trans"] - t, st["rotvec"] - w
    assert abs(np.linalg.norm(dt) - ETA_T) < 1e-13
    assert abs(np.linalg.norm(dw) - ETA_R) < 1e-13
    assert np.abs(dt + ETA_T * gt / np.linalg.norm(gt)).max() < 1e-7
    assert np.abs(dw + ETA_R * gw / np.linalg.norm(gw)).max() < 1e-7
    # the returned energy is the energy of the returned pose, and it went down
    e_new, f_new = _energy(m, lig, lq, st["rotvec"], st["trans"])
    assert f_new == 0 and abs(e_new - st["E"]) < 1e-14 and st["E"] < st["E_start"]


@pytest.mark.parametrize("gap,level", [(0.03, 2), (0.004, MAX_HALVINGS)])
def test_halving_level_for_infeasible_trials(gap, level):
    """At distance sigma + gap the trials clash until the step 0.1 * 2^-level is
    short enough: sigma + 0.03 is reached at the second halving (0.025 A) and
    sigma + 0.004 only at the last one (0.003125 A)."""
    m, lig, lq, t, c = _single_charge_case(gap)
    d = [_trial_distance(t, c, s) for s in range(level + 1)]
    assert all(x < SIGMA for x in d[:-1]) and d[-1] > SIGMA
    gt, _ = _fd_grad(m, lig, lq, np.zeros(3), t)
    assert abs(gt[1]) < 1e-9 * abs(gt[0]) and abs(gt[2]) < 1e-9 * abs(gt[0]) and gt[0] > 0
    st = _step(m, lig, lq, np.zeros(3), t)
    assert st["accepted"] == level
    assert np.abs(st["trans"] - (t - [ETA_T * 0.5 ** level, 0, 0])).max() < 1e-12
    assert np.array_equal(st["rotvec"], np.zeros(3))       # one atom: no torque, no turn
    e2, f2 = _energy(m, lig, lq, np.zeros(3), st["trans"])
    assert f2 == 0 and abs(e2 - st["E"]) < 1e-14 and st["E"] <= st["E_start"]


def test_keeps_pose_when_all_levels_fail():
    """At distance sigma + 0.002 every trial down to 0.1 * 2^-5 = 0.003125 A clashes
    (the sixth halving, 0.0016 A, would not): the pose and its energy are kept."""
    m, lig, lq, t, c = _single_charge_case(0.002)
    assert all(_trial_distance(t, c, s) < SIGMA for s in range(MAX_HALVINGS + 1))
    assert _trial_distance(t, c, MAX_HALVINGS + 1) > SIGMA
    st = _step(m, lig, lq, np.zeros(3), t)
    assert st["accepted"] == -1
    assert np.array_equal(st["trans"], t) and np.array_equal(st["rotvec"], np.zeros(3))
    assert st["E"] == st["E_start"]


def test_rejects_trial_that_raises_energy():
    """Two charges +1 at (+-6, h/2, h/2) and a charge +1 near the midpoint: along x the
    interpolated potential is symmetric about the node x = 0 and linear on each side,
    so from x = 0.04 the full step (to x = -0.06) raises E although it is feasible,
    and the first halving (to x = -0.01) lowers it."""
    yz = H / 2
    m = _model([[-6.0, yz, yz], [6.0, yz, yz]], [1.0, 1.0])
    lig, lq = np.zeros((1, 3)), np.array([1.0])
    t = np.array([0.04, yz - 0.02, yz + 0.03])
    e0, f0 = _energy(m, lig, lq, np.zeros(3), t)
    e_full, f_full = _energy(m, lig, lq, np.zeros(3), t - [ETA_T, 0, 0])
    e_half, f_half = _energy(m, lig, lq, np.zeros(3), t - [ETA_T / 2, 0, 0])
    assert f0 == 0 and f_full == 0 and f_half == 0
    assert e_full > e0 > e_half
    gt, _ = _fd_grad(m, lig, lq, np.zeros(3), t)
    assert gt[0] > 0 and abs(gt[1]) < 1e-9 * gt[0] and abs(gt[2]) < 1e-9 * gt[0]
    st = _step(m, lig, lq, np.zeros(3), t)
    assert st["accepted"] == 1
    assert np.abs(st["trans"] - (t - [ETA_T / 2, 0, 0])).max() < 1e-12
    assert abs(st["E"] - e_half) < 1e-14


def test_equal_energy_is_accepted():
    """A ligand without charge has E = 0 and a zero gradient everywhere: the (zero)
    step gives E_trial = E, which the rule accepts at the first level."""
    m = _model([[1.0, 0.5, -0.5]], [1.0])
    lig = np.array([[0.5, 0.0, 0.0], [-0.5, 0.0, 0.0]])
    lq = np.zeros(2)
    w, t = np.array([0.2, 0.1, -0.3]), np.array([5.3, 0.7, -1.2])
    st = _step(m, lig, lq, w, t)
    assert st["E_start"] == 0.0 and st["E"] == 0.0
    assert st["accepted"] == 0
    assert np.array_equal(st["trans"], t) and np.array_equal(st["rotvec"], w)


@pytest.mark.parametrize("kw,which", [
    ({"eta_t": ETA_R, "eta_r": ETA_T}, "normalised"),   # step lengths swapped
    ({"max_halvings": MAX_HALVINGS + 1}, "keep"),       # one halving too many
])
def test_pins_catch_mistaken_step_rules(kw, which):
    """The checks above fail for a step rule with the wrong constants."""
    if which == "normalised":
        prot = [[1.2, -0.7, 0.4], [-2.3, 1.1, -0.6], [0.3, 2.2, 1.7]]
        m = _model(prot, [1.0, -0.6, 0.8])
        lig = np.array([[0.9, 0.1, -0.3], [-0.8, -0.2, 0.4]])
        lq = np.array([-0.7, 0.45])
        w, t = np.array([0.31, -0.52, 0.17]), np.array([4.61, 2.73, 3.37])
        st = O.pgd_step(m, lig, lq, w[None], t[None], **kw)
        assert abs(np.linalg.norm(st["trans"][0] - t) - ETA_T) > 1e-3
    else:
        m, lig, lq, t, _ = _single_charge_case(0.002)
        st = O.pgd_step(m, lig, lq, np.zeros((1, 3)), t[None], **kw)
        assert st["accepted"][0] != -1
