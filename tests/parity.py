"""Helpers shared by the GPU parity tests: tolerances and comparisons."""
import numpy as np

import oracle as O

E_TOL = 1e-5      # per-pose energy, relative to max(|E|, 1e-2 S)
G_TOL = 1e-4      # gradients, relative to max(|g|, 1e-2 * sum of per-atom magnitudes)
# Two evaluation paths of the library (the tensor-core W form, ~2^-33 per
# contraction, and the float-pair W form, ~2^-47) on the same poses: per-pose
# energies relative to max(|E|, median |E|).  Set for the earlier 2^-31 slicing
# (four slices); the five-slice scheme's rounding is four times smaller.
PATH_TOL = 1e-8


def energy_errors(E_gpu, ref):
    scale = O.tolerance_scale(ref["E"], ref["S_ref"])
    return np.abs(np.asarray(E_gpu) - ref["E"]) / scale


def assert_energies(E_gpu, ref, tol=E_TOL):
    err = energy_errors(E_gpu, ref)
    worst = int(np.argmax(err))
    assert err.max() <= tol, (f"max rel err {err.max():.3e} at pose {worst}: gpu {E_gpu[worst]!r} "
                              f"oracle {ref['E'][worst]!r}")
    return err


def assert_flags(flags_gpu, ref):
    fg = np.asarray(flags_gpu).astype(np.uint8)
    bad = np.nonzero(fg != ref["flags"])[0]
    assert bad.size == 0, f"{bad.size} flag mismatches, first {bad[:5]}: gpu {fg[bad[:5]]} oracle {ref['flags'][bad[:5]]}"


def assert_topk(E_gpu, flags_gpu, ref, k=10, tie=2e-5):
    """Top-k feasible poses by energy agree; poses whose oracle energies differ by less
    than tie * scale are interchangeable."""
    a = O.feasible_topk(np.asarray(E_gpu), np.asarray(flags_gpu), k)
    b = O.feasible_topk(ref["E"], ref["flags"], k)
    if np.array_equal(a, b):
        return
    scale = O.tolerance_scale(ref["E"], ref["S_ref"])
    Eb = ref["E"][b]
    for i, (x, y) in enumerate(zip(a, b)):
        if x != y:
            assert abs(ref["E"][x] - ref["E"][y]) <= tie * max(scale[x], scale[y]), (i, x, y)
    kth = Eb[-1]
    assert set(a) == set(b) or np.all(np.abs(ref["E"][np.setxor1d(a, b)] - kth) <= tie * scale.max())


def assert_gradients(gt, gw, ref, keep=None, tol=G_TOL):
    gt, gw = np.asarray(gt), np.asarray(gw)
    st = np.maximum(np.linalg.norm(ref["dE_dt"], axis=1), 1e-2 * ref["T_ref"])
    sw = np.maximum(np.linalg.norm(ref["dE_dw"], axis=1), 1e-2 * ref["W_ref"])
    et = np.abs(gt - ref["dE_dt"]).max(axis=1) / st
    ew = np.abs(gw - ref["dE_dw"]).max(axis=1) / sw
    if keep is not None:
        et, ew = et[keep], ew[keep]
    assert et.max() <= tol, f"translation gradient rel err {et.max():.3e}"
    assert ew.max() <= tol, f"rotation gradient rel err {ew.max():.3e}"
    return et, ew


def away_from_planes(model, lig_xyz, R, trans, eps=1e-5):
    """Poses whose atoms all sit farther than eps (in cell units) from a grid plane:
    there the interpolant is differentiable and both sides pick the same cell."""
    x = O.posed_atoms(lig_xyz, R, trans)
    s = (x + model.b) / model.h
    frac = s - np.floor(s)
    return np.all((frac > eps) & (frac < 1 - eps), axis=(1, 2))


def path_errors(E, E_ref):
    E, E_ref = np.asarray(E, dtype=np.float64), np.asarray(E_ref, dtype=np.float64)
    if E_ref.size == 0:
        return np.zeros(0)
    scale = np.maximum(np.abs(E_ref), max(np.median(np.abs(E_ref)), 1e-300))
    return np.abs(E - E_ref) / scale


def assert_paths_agree(E, E_ref, flags=None, flags_ref=None, tol=PATH_TOL):
    """Energies of two library paths agree to tol; flags (decided by the same short-range
    code on every path) are identical."""
    err = path_errors(E, E_ref)
    if err.size:
        worst = int(np.argmax(err))
        assert err[worst] <= tol, f"paths differ by {err[worst]:.3e} at pose {worst}: {E[worst]!r} vs {E_ref[worst]!r}"
    if flags is not None:
        assert np.array_equal(np.asarray(flags), np.asarray(flags_ref))
    return err
