"""Plain FP64 oracle (numpy) for RS-tensor electrostatic energies of rigid ligand poses.

TEST INFRASTRUCTURE ONLY -- see the package docstring.  Nothing here is blocked,
fused or reordered beyond the paper's definitions; library primitives (numpy
SVD, a k-d tree for neighbour lists) serve as single steps.

Paper: arXiv 2510.26611 (Benner, Khoromskij, Khoromskaia, Stein).

Readings of the paper taken here (the paper leaves them open):
* Grid: n nodes x_i = -b + i*h, h = 2b/(n-1) on [-b, b] (Sec. 2, grid Omega_n;
  the paper's h = 2b/n with even n is replaced by a node grid for odd n).
* Sinc quadrature for 1/r (Sec. 2, Eq. sinc): the substitution t = sinh(u) of
  1/r = (2/sqrt(pi)) int_0^inf exp(-r^2 t^2) dt, trapezoid rule with step h_s
  in box-scaled units rho = r / (2 sqrt(3) b); the k = 0 term has t = 0.
  Long range = the R_l widest terms (Sec. 2, Eq. Split_Tens), h_s chosen so
  the narrowest long-range Gaussian has t*sigma = tau (TEP step 2: sigma bounds
  the long-range support from below).  K_max from r_min.
* Collocation: factor entries are point values of the Gaussians at the grid
  nodes, atoms at their exact (off-grid) positions (Sec. 2, Eq. Total_Sum and
  Eq. Long-Range_Sum with the shift taken exactly).
* Off-grid ligand atoms: trilinear interpolation of the grid tensor, done per
  axis on each rank-1 term (equal by multilinearity); atoms outside [-b, b]
  are clamped to the edge cell and flagged.
* Short range: each protein atom's short-range Gaussians, summed analytically
  for pairs closer than the cutoff r_c (Def. 2.1, the cumulated local part).
* RHOSVD (Sec. 1 and Sec. 4.1): Z = U diag(|xi|^(1/3)), V = leading r left
  singular vectors, r = min(cap, #{s_i > eps_r s_1}); core
  beta = sum_r xi_r (V1^T u1_r) o (V2^T u2_r) o (V3^T u3_r).
* Poses: unit quaternion (w,x,y,z) or rotation vector about the ligand's
  geometric centre, plus the centre's position (Sec. 3.4, transformation
  F = R o T).  Gradient with respect to the rotation vector uses the SO(3)
  left Jacobian.
* vdW constraint (Sec. 3.4, Eq. Energy_Min): feasible iff every ligand-protein
  distance is >= sigma.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "SincTable", "sinc_table", "grid_nodes", "interp_weights", "ligand_frame",
    "quat_to_rot", "rotvec_to_rot", "left_jacobian", "posed_atoms",
    "long_range_factors", "rhosvd", "RSModel", "build_model", "potential",
    "short_range", "min_distances", "energies_from_atoms", "pose_energies", "pose_gradients",
    "coulomb_energies", "coulomb_gradients", "pgd_step", "feasible_topk", "fd_forces",
    "ppiem_directions", "contact_offsets", "ppiem_scan", "box_cells", "local_box_model",
    "complex_energies", "add_and_compress",
    "FLAG_CLASH", "FLAG_OUT_OF_GRID", "tolerance_scale",
]

FLAG_CLASH = 1          # some ligand atom is closer than sigma to a protein atom
FLAG_OUT_OF_GRID = 2    # some ligand atom lies outside [-b, b]^3


# ----------------------------------------------------------------------------
# Sinc quadrature (Sec. 2, Eq. sinc; range split Eq. Split_Tens; TEP step 2)
# ----------------------------------------------------------------------------
@dataclass
class SincTable:
    t: np.ndarray            # (K+1,) Gaussian exponents, 1/Angstrom; t[0] = 0
    a: np.ndarray            # (K+1,) weights, 1/Angstrom
    is_long: np.ndarray      # (K+1,) bool, True for the R_l widest terms
    h_s: float               # quadrature step in the sinh variable
    box_len: float           # scaling length 2*sqrt(3)*b
    r_c: float               # short-range cutoff
    quad_err: float          # max |r * sum_k a_k exp(-t_k^2 r^2) - 1| on [r_min, box_len]
    r_min: float


def _short_sum(t, a, r):
    return (a[None, :] * np.exp(-np.outer(r * r, t * t))).sum(axis=1)


def sinc_table(b: float, sigma: float, R_l: int, r_min: float = 0.5, tau: float = 4.0,
               short_tol: float = 1e-9) -> SincTable:
    """Sum-of-Gaussians for 1/r by sinc quadrature (Sec. 2, Eq. sinc).

    1/r = (2/sqrt(pi)) int_0^inf exp(-r^2 t^2) dt (Sec. 2, the Gaussian integral
    representation of the Newton kernel).  With t = sinh(u)/box_len this becomes
    (1/box_len)(1/sqrt(pi)) int_R cosh(u) exp(-rho^2 sinh^2 u) du, rho = r/box_len;
    the trapezoid rule with step h_s, folded over +-k, gives the nodes and weights.
    """
    if R_l < 2:
        raise ValueError("R_l must be >= 2")
    box_len = 2.0 * math.sqrt(3.0) * b
    h_s = math.asinh(tau * box_len / sigma) / (R_l - 1)
    K = int(math.ceil(math.asinh(tau * box_len / r_min) / h_s))
    K = max(K, R_l - 1)
    k = np.arange(K + 1, dtype=np.float64)
    t_hat = np.sinh(k * h_s)
    a_hat = 2.0 * h_s * np.cosh(k * h_s) / math.sqrt(math.pi)
    a_hat[0] = h_s / math.sqrt(math.pi)
    t = t_hat / box_len
    a = a_hat / box_len
    is_long = np.arange(K + 1) < R_l

    # measured quadrature error on [r_min, box_len]
    r = np.geomspace(r_min, box_len, 20001)
    quad_err = float(np.abs(r * _short_sum(t, a, r) - 1.0).max())

    # short-range cutoff: last r where r * (short-range sum) exceeds short_tol
    ts, as_ = t[~is_long], a[~is_long]
    r_c = 0.0
    if ts.size:
        rr = np.linspace(1e-3, box_len, 200001)
        f = rr * _short_sum(ts, as_, rr)
        above = np.nonzero(f > short_tol)[0]
        if above.size:
            lo, hi = rr[above[-1]], rr[min(above[-1] + 1, rr.size - 1)]
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                if mid * _short_sum(ts, as_, np.array([mid]))[0] > short_tol:
                    lo = mid
                else:
                    hi = mid
            r_c = hi
    return SincTable(t, a, is_long, h_s, box_len, r_c, quad_err, r_min)


# ----------------------------------------------------------------------------
# Grid, interpolation, poses (Sec. 2 grid; Sec. 3.2 atoms off the grid; Sec. 3.4)
# ----------------------------------------------------------------------------
def grid_nodes(n: int, b: float) -> np.ndarray:
    """Node coordinates x_i = -b + i*h, h = 2b/(n-1) (Sec. 2, grid Omega_n)."""
    return -b + np.arange(n, dtype=np.float64) * (2.0 * b / (n - 1))


def interp_weights(c: np.ndarray, n: int, b: float):
    """Cell index i, fraction f in [0,1], inside flag, for coordinates c.
    s = (c + b)/h; i = min(floor(s), n-2) clamped at 0; f = s - i clamped to [0,1]."""
    h = 2.0 * b / (n - 1)
    s = (c + b) / h
    i = np.floor(s).astype(np.int64)
    i = np.clip(i, 0, n - 2)
    f = s - i
    inside = (s >= 0.0) & (s <= n - 1)
    f = np.clip(f, 0.0, 1.0)
    return i, f, inside


def ligand_frame(lig_xyz: np.ndarray) -> np.ndarray:
    """Ligand coordinates relative to its unweighted geometric centre (Sec. 3.4)."""
    lig = np.asarray(lig_xyz, dtype=np.float64)
    return lig - lig.mean(axis=0)


def quat_to_rot(q: np.ndarray) -> np.ndarray:
    """Rotation matrices of (normalised) quaternions (w, x, y, z); shape (P, 3, 3)."""
    q = np.asarray(q, dtype=np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _hat(w: np.ndarray) -> np.ndarray:
    K = np.zeros(w.shape[:-1] + (3, 3))
    K[..., 0, 1], K[..., 0, 2] = -w[..., 2], w[..., 1]
    K[..., 1, 0], K[..., 1, 2] = w[..., 2], -w[..., 0]
    K[..., 2, 0], K[..., 2, 1] = -w[..., 1], w[..., 0]
    return K


def rotvec_to_rot(w: np.ndarray) -> np.ndarray:
    """R = exp([w]x) (Rodrigues), with Taylor coefficients for small angles."""
    w = np.asarray(w, dtype=np.float64)
    th = np.linalg.norm(w, axis=-1)
    K = _hat(w)
    small = th < 1e-4
    ths = np.where(small, 1.0, th)
    A = np.where(small, 1 - th ** 2 / 6 + th ** 4 / 120, np.sin(ths) / ths)
    B = np.where(small, 0.5 - th ** 2 / 24 + th ** 4 / 720, (1 - np.cos(ths)) / ths ** 2)
    I = np.broadcast_to(np.eye(3), K.shape)
    return I + A[..., None, None] * K + B[..., None, None] * (K @ K)


def left_jacobian(w: np.ndarray) -> np.ndarray:
    """SO(3) left Jacobian J_l(w) = I + (1-cos t)/t^2 [w]x + (t - sin t)/t^3 [w]x^2
    (Sola et al. 2018, "A micro Lie theory"); exp(w + d) = exp(J_l d) exp(w) + O(d^2)."""
    w = np.asarray(w, dtype=np.float64)
    th = np.linalg.norm(w, axis=-1)
    K = _hat(w)
    small = th < 1e-4
    ths = np.where(small, 1.0, th)
    B = np.where(small, 0.5 - th ** 2 / 24 + th ** 4 / 720, (1 - np.cos(ths)) / ths ** 2)
    C = np.where(small, 1.0 / 6 - th ** 2 / 120 + th ** 4 / 5040, (ths - np.sin(ths)) / ths ** 3)
    I = np.broadcast_to(np.eye(3), K.shape)
    return I + B[..., None, None] * K + C[..., None, None] * (K @ K)


def posed_atoms(lig_xyz: np.ndarray, R: np.ndarray, trans: np.ndarray) -> np.ndarray:
    """x_j = R y_j + t for every pose; y = ligand coordinates about its centre."""
    y = ligand_frame(lig_xyz)
    return np.einsum("pij,lj->pli", R, y) + np.asarray(trans, dtype=np.float64)[:, None, :]


# ----------------------------------------------------------------------------
# Long-range canonical factors (Sec. 2 Eq. Long-Range_Sum; TEP step 3)
# ----------------------------------------------------------------------------
def long_range_factors(prot_xyz, prot_q, table: SincTable, n: int, b: float, galerkin: bool = False):
    """U^(l)[i, (m,k)] = exp(-t_k^2 (x_i - x_m^l)^2) over the long-range terms and
    weights xi_(m,k) = z_m a_k: the rank N*R_l canonical sum of shifted
    long-range Gaussians (Sec. 2, Eq. Long-Range_Sum; TEP step 3).
    galerkin: the entries are instead the Gaussians' averages over the node's cell
    [x_i - h/2, x_i + h/2] (the projection of Sec. 2, Eq. galten, per axis),
    sqrt(pi)/(2 t h) (erf(t (d + h/2)) - erf(t (d - h/2))), and 1 for t = 0."""
    from scipy.special import erf, erfc
    x = grid_nodes(n, b)
    h = 2.0 * b / (n - 1)
    prot_xyz = np.asarray(prot_xyz, dtype=np.float64)
    tl, al = table.t[table.is_long], table.a[table.is_long]
    N, Rl = prot_xyz.shape[0], tl.size
    U = []
    for ax in range(3):
        d = x[:, None, None] - prot_xyz[None, :, ax, None]
        if not galerkin:
            U.append(np.exp(-(tl[None, None, :] ** 2) * d * d).reshape(n, N * Rl))
            continue
        t = tl[None, None, :]
        ts = np.where(t > 0, t, 1.0)
        A, B = ts * (d - 0.5 * h), ts * (d + 0.5 * h)
        # erf(B) - erf(A) without cancellation in the tails: through erfc when both
        # arguments have the same sign
        diff = np.where(A >= 0, erfc(np.abs(A)) - erfc(np.abs(B)),
                        np.where(B <= 0, erfc(np.abs(B)) - erfc(np.abs(A)), erf(B) - erf(A)))
        avg = math.sqrt(math.pi) / (2.0 * ts * h) * diff
        U.append(np.where(t > 0, avg, 1.0).reshape(n, N * Rl))
    xi = (np.asarray(prot_q, dtype=np.float64)[:, None] * al[None, :]).ravel()
    return U, xi


def rhosvd(U, xi, cap: int, eps_r: float = 1e-7):
    """Reduced HOSVD of the canonical tensor sum_r xi_r u1_r o u2_r o u3_r
    (Sec. 1 and Sec. 4.1, canonical-to-Tucker by RHOSVD; TEP step 4).

    Returns (V list, beta, singular values list)."""
    w = np.abs(xi) ** (1.0 / 3.0)
    V, svals = [], []
    for ax in range(3):
        Z = U[ax] * w[None, :]
        # SVD of the wide Z through a QR of Z^T (Z = R^T Q^T): same left singular
        # vectors and singular values, without forming the right factor of Z.
        if Z.shape[1] > Z.shape[0]:
            Rt = np.linalg.qr(Z.T, mode="r").T
            Ul, s, _ = np.linalg.svd(Rt)
        else:
            Ul, s, _ = np.linalg.svd(Z, full_matrices=False)
        r = int(np.count_nonzero(s > eps_r * s[0]))
        if cap > 0:
            r = min(r, cap)
        V.append(Ul[:, :r].copy())
        svals.append(s)
    C = [V[ax].T @ U[ax] for ax in range(3)]
    beta = np.einsum("ar,br,cr,r->abc", C[0], C[1], C[2], xi, optimize=True)
    return V, beta, svals


@dataclass
class RSModel:
    kind: str                       # "canonical" or "tucker"
    n: int
    b: float
    sigma: float
    table: SincTable
    prot_xyz: np.ndarray
    prot_q: np.ndarray
    U: list = field(default_factory=list)     # canonical factors (n x R) x3
    xi: np.ndarray | None = None
    V: list = field(default_factory=list)     # Tucker factors (n x r_l) x3
    beta: np.ndarray | None = None
    svals: list = field(default_factory=list)
    # a local model (scheme C): per axis the interpolation cells [lo, hi] it covers;
    # a point outside them is flagged out of grid
    cells: tuple | None = None

    @property
    def h(self) -> float:
        return 2.0 * self.b / (self.n - 1)

    @property
    def ranks(self):
        if self.kind == "tucker":
            return tuple(v.shape[1] for v in self.V)
        return (self.xi.size,)


def build_model(prot_xyz, prot_q, n: int, b: float, sigma: float, R_l: int,
                tucker_cap: int = 0, eps_r: float = 1e-7, r_min: float = 0.5,
                tau: float = 4.0, keep_canonical: bool = False, galerkin: bool = False) -> RSModel:
    """Algorithm TEP (Sec. 3.4): sinc table, shifted long-range Gaussians,
    optional rank reduction.  tucker_cap = 0 keeps the unreduced canonical form;
    galerkin takes cell averages for the factor entries (collocation otherwise)."""
    table = sinc_table(b, sigma, R_l, r_min=r_min, tau=tau)
    U, xi = long_range_factors(prot_xyz, prot_q, table, n, b, galerkin=galerkin)
    m = RSModel("canonical", n, b, sigma, table, np.asarray(prot_xyz, np.float64),
                np.asarray(prot_q, np.float64), U=U, xi=xi)
    if tucker_cap > 0:
        V, beta, sv = rhosvd(U, xi, tucker_cap, eps_r)
        m.kind, m.V, m.beta, m.svals = "tucker", V, beta, sv
        if not keep_canonical:
            m.U, m.xi = [], None
    return m


def box_cells(model: RSModel, lo, hi):
    """Interpolation cells [c_lo, c_hi] per axis that cover the box [lo, hi] (A)."""
    out = []
    for ax in range(3):
        c0 = int(min(max(math.floor((lo[ax] + model.b) / model.h), 0), model.n - 2))
        c1 = int(min(max(math.ceil((hi[ax] + model.b) / model.h) - 1, c0), model.n - 2))
        out.append((c0, c1))
    return tuple(out)


def local_box_model(model: RSModel, lo, hi, eps: float = 1e-7, cap: int = 32) -> RSModel:
    """Scheme (C) of Sec. 3.2 (Table 1): the global Tucker potential restricted to the
    grid nodes of the box [lo, hi] and re-truncated there by an HOSVD of the restricted
    node tensor T_Pi: per axis the leading left singular vectors of its mode
    unfolding, rank r = #{s_i > eps s_1} (at most cap), core = T_Pi projected on them.
    The factor rows outside the box are zero; points outside its cells are flagged.
    The node-tensor error is at most sqrt(sum over axes of the dropped s_i^2)."""
    assert model.kind == "tucker"
    cells = box_cells(model, lo, hi)
    rows = [np.arange(c0, c1 + 2) for c0, c1 in cells]           # the cells' nodes
    Vr = [model.V[ax][rows[ax]] for ax in range(3)]
    T = np.einsum("abc,ia,jb,kc->ijk", model.beta, Vr[0], Vr[1], Vr[2], optimize=True)
    U, svals = [], []
    for ax in range(3):
        M = np.moveaxis(T, ax, 0).reshape(T.shape[ax], -1)
        Ul, sv, _ = np.linalg.svd(M, full_matrices=False)
        r = int(np.count_nonzero(sv > eps * sv[0])) if sv[0] > 0 else 0
        r = max(1, min(r, cap))
        U.append(Ul[:, :r])
        svals.append(sv)
    core = np.einsum("ijk,ia,jb,kc->abc", T, U[0], U[1], U[2], optimize=True)
    V = []
    for ax in range(3):
        F = np.zeros((model.n, U[ax].shape[1]))
        F[rows[ax]] = U[ax]
        V.append(F)
    dropped = math.sqrt(sum(float((sv[U[ax].shape[1]:] ** 2).sum()) for ax, sv in enumerate(svals)))
    out = RSModel("tucker", model.n, model.b, model.sigma, model.table, model.prot_xyz, model.prot_q,
                  V=V, beta=core, svals=svals, cells=cells)
    out.trunc_bound = dropped
    out.node_tensor_norm = float(np.linalg.norm(T))
    return out


# ----------------------------------------------------------------------------
# Point evaluation (Sec. 2 entry evaluation; Lemma 3.3; Eq. Gradients_Tens)
# ----------------------------------------------------------------------------
def _lerp_rows(M, i, f):
    return (1.0 - f)[:, None] * M[i] + f[:, None] * M[i + 1]


def _long_range(model: RSModel, pts: np.ndarray, grad: bool, chunk: int | None = None):
    """Trilinear interpolation of the long-range grid tensor at points, done per
    rank-1 term as a product of per-axis linear interpolations."""
    P = pts.shape[0]
    if chunk is None:  # points per batch: bounded memory for large canonical ranks
        chunk = 256 if model.kind == "canonical" else 16384
    h = model.h
    phi = np.zeros(P)
    g = np.zeros((P, 3)) if grad else None
    for s0 in range(0, P, chunk):
        p = pts[s0:s0 + chunk]
        ifs = [interp_weights(p[:, ax], model.n, model.b) for ax in range(3)]
        mats = model.U if model.kind == "canonical" else model.V
        vals, ders = [], []
        for ax in range(3):
            i, f, inside = ifs[ax]
            vals.append(_lerp_rows(mats[ax], i, f))
            if grad:
                d = (mats[ax][i + 1] - mats[ax][i]) / h
                ders.append(np.where(inside[:, None], d, 0.0))
        if model.kind == "canonical":
            xi = model.xi[None, :]
            phi[s0:s0 + chunk] = (xi * vals[0] * vals[1] * vals[2]).sum(axis=1)
            if grad:
                g[s0:s0 + chunk, 0] = (xi * ders[0] * vals[1] * vals[2]).sum(axis=1)
                g[s0:s0 + chunk, 1] = (xi * vals[0] * ders[1] * vals[2]).sum(axis=1)
                g[s0:s0 + chunk, 2] = (xi * vals[0] * vals[1] * ders[2]).sum(axis=1)
        else:
            # phi = sum_a v1_a sum_b v2_b sum_c beta_abc v3_c (nested sums of the
            # Tucker entry evaluation; the c-sum is a matrix product)
            B = model.beta
            r1, r2, r3 = B.shape
            Bm = B.reshape(r1 * r2, r3).T

            def contract(x1, x2, x3):
                t = (x3 @ Bm).reshape(-1, r1, r2)
                return ((t * x2[:, None, :]).sum(axis=2) * x1).sum(axis=1)

            phi[s0:s0 + chunk] = contract(*vals)
            if grad:
                g[s0:s0 + chunk, 0] = contract(ders[0], vals[1], vals[2])
                g[s0:s0 + chunk, 1] = contract(vals[0], ders[1], vals[2])
                g[s0:s0 + chunk, 2] = contract(vals[0], vals[1], ders[2])
    return phi, g


def short_range(model: RSModel, pts: np.ndarray, grad: bool = False):
    """Short-range part at points: sum over protein atoms closer than r_c of
    z_m sum_{k short} a_k exp(-t_k^2 d^2) (Def. 2.1, cumulated local tensors)."""
    from scipy.spatial import cKDTree
    tab = model.table
    ts, as_ = tab.t[~tab.is_long], tab.a[~tab.is_long]
    P = pts.shape[0]
    phi = np.zeros(P)
    g = np.zeros((P, 3)) if grad else None
    if ts.size == 0 or tab.r_c <= 0.0:
        return phi, g
    tp = cKDTree(model.prot_xyz)
    tq = cKDTree(pts)
    S = tq.sparse_distance_matrix(tp, tab.r_c, output_type="coo_matrix")
    i, m = S.row, S.col
    diff = pts[i] - model.prot_xyz[m]
    d2 = (diff * diff).sum(axis=1)
    keep = d2 < tab.r_c * tab.r_c
    i, m, diff, d2 = i[keep], m[keep], diff[keep], d2[keep]
    e = as_[None, :] * np.exp(-np.outer(d2, ts * ts))         # (pairs, K_s)
    val = model.prot_q[m] * e.sum(axis=1)
    np.add.at(phi, i, val)
    if grad:
        dv = model.prot_q[m] * (e * (-2.0 * ts * ts)[None, :]).sum(axis=1)
        np.add.at(g, i, dv[:, None] * diff)
    return phi, g


def potential(model: RSModel, pts: np.ndarray, grad: bool = False):
    """Long-range (Lemma 3.3) and short-range parts of the RS potential at points."""
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
    pl, gl = _long_range(model, pts, grad)
    ps, gs = short_range(model, pts, grad)
    return pl, ps, gl, gs


def min_distances(prot_xyz: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Distance from each point to its nearest protein atom."""
    from scipy.spatial import cKDTree
    d, _ = cKDTree(prot_xyz).query(pts, k=1)
    return d


# ----------------------------------------------------------------------------
# Pose energies and gradients (Algorithm PLIE; Sec. 3.3 forces; Sec. 4.2)
# ----------------------------------------------------------------------------
def _flags(model: RSModel, x: np.ndarray) -> np.ndarray:
    P, L, _ = x.shape
    flat = x.reshape(-1, 3)
    dmin = min_distances(model.prot_xyz, flat).reshape(P, L).min(axis=1)
    ok = (flat >= -model.b) & (flat <= model.b)
    if model.cells is not None:
        for ax in range(3):
            i, _, _ = interp_weights(flat[:, ax], model.n, model.b)
            lo, hi = model.cells[ax]
            ok[:, ax] &= (i >= lo) & (i <= hi)
    inside = np.all(ok, axis=1).reshape(P, L).all(axis=1)
    flags = np.zeros(P, dtype=np.uint8)
    flags[dmin < model.sigma] |= FLAG_CLASH
    flags[~inside] |= FLAG_OUT_OF_GRID
    return flags, dmin


def energies_from_atoms(model: RSModel, x: np.ndarray, lig_q) -> dict:
    """E_p = sum_j q_j (phi_long + phi_short)(x_j) for posed atoms x (P, L, 3)
    (Sec. 3.4, PLIE steps 2-3; Lemma 3.3, Eq. EnergySum_ligand) and vdW flags."""
    x = np.asarray(x, dtype=np.float64)
    q = np.asarray(lig_q, dtype=np.float64)
    P, L, _ = x.shape
    pl, ps, _, _ = potential(model, x.reshape(-1, 3))
    pl, ps = pl.reshape(P, L), ps.reshape(P, L)
    flags, dmin = _flags(model, x)
    return {"E_long": (q[None, :] * pl).sum(axis=1),
            "E": (q[None, :] * (pl + ps)).sum(axis=1),
            "S_ref": np.abs(q[None, :] * (pl + ps)).sum(axis=1),
            "flags": flags, "dmin": dmin}


def pose_energies(model: RSModel, lig_xyz, lig_q, quat, trans, chunk: int = 2048):
    """Algorithm PLIE for a batch of poses: sample the potential at the posed ligand
    atoms and take the charge-weighted sum (Sec. 3.4, PLIE steps 2-3;
    Lemma 3.3, Eq. EnergySum_ligand), plus the short-range part and vdW flags."""
    quat = np.asarray(quat, dtype=np.float64)
    trans = np.asarray(trans, dtype=np.float64)
    P = quat.shape[0]
    out = {k: np.zeros(P) for k in ("E", "E_long", "S_ref", "dmin")}
    out["flags"] = np.zeros(P, dtype=np.uint8)
    for s0 in range(0, P, chunk):
        sl = slice(s0, min(P, s0 + chunk))
        x = posed_atoms(lig_xyz, quat_to_rot(quat[sl]), trans[sl])
        r = energies_from_atoms(model, x, lig_q)
        for k in out:
            out[k][sl] = r[k]
    return out


def add_and_compress(models, cap: int, eps_r: float = 1e-7) -> RSModel:
    """Add-and-compress (Sec. 3.4, Algorithm TEP step 4; Sec. 5.1, the complex of
    Eq. EnergySum_Mcomplex): the long-range Tucker tensors of several molecules on one
    grid, T = sum_p beta_p x_1 V1_p x_2 V2_p x_3 V3_p, summed and re-truncated.  Per
    axis the factor matrices side by side are orthonormalised, [V_l^(1) ... V_l^(P)] =
    Q_l R_l (thin QR), so that T = C x_l Q_l exactly with
    C = sum_p beta_p x_l R_l[:, columns of p]; an HOSVD of the small core C keeps per
    axis the leading left singular vectors of its mode unfolding (r = #{s_i > eps_r
    s_1}, at most cap): V_l = Q_l U_l, core = C x_l U_l^T.  The short range is that of
    the union of the molecules' atoms (their sinc table is shared)."""
    m0 = models[0]
    for m in models:
        assert m.kind == "tucker" and m.n == m0.n and m.b == m0.b and m.sigma == m0.sigma
        assert np.array_equal(m.table.t, m0.table.t) and np.array_equal(m.table.a, m0.table.a)
    Q, Rf, cols = [], [], []
    for ax in range(3):
        A = np.concatenate([m.V[ax] for m in models], axis=1)
        q, r = np.linalg.qr(A)
        Q.append(q)
        Rf.append(r)
        cols.append(np.cumsum([0] + [m.V[ax].shape[1] for m in models]))
    C = np.zeros(tuple(q.shape[1] for q in Q))
    for p, m in enumerate(models):
        Rp = [Rf[ax][:, cols[ax][p]:cols[ax][p + 1]] for ax in range(3)]
        C += np.einsum("abc,ia,jb,kc->ijk", m.beta, Rp[0], Rp[1], Rp[2], optimize=True)
    U, svals = [], []
    for ax in range(3):
        M = np.moveaxis(C, ax, 0).reshape(C.shape[ax], -1)
        Ul, sv, _ = np.linalg.svd(M, full_matrices=False)
        r = int(np.count_nonzero(sv > eps_r * sv[0])) if sv[0] > 0 else 0
        r = max(1, min(r, cap))
        U.append(Ul[:, :r])
        svals.append(sv)
    core = np.einsum("ijk,ia,jb,kc->abc", C, U[0], U[1], U[2], optimize=True)
    V = [Q[ax] @ U[ax] for ax in range(3)]
    xyz = np.concatenate([m.prot_xyz for m in models], axis=0)
    q = np.concatenate([m.prot_q for m in models], axis=0)
    out = RSModel("tucker", m0.n, m0.b, m0.sigma, m0.table, xyz, q, V=V, beta=core, svals=svals)
    out.trunc_bound = math.sqrt(sum(float((sv[U[ax].shape[1]:] ** 2).sum()) for ax, sv in enumerate(svals)))
    return out


def complex_energies(models, lig_xyz, lig_q, quat, trans) -> dict:
    """A molecular complex M_1..M_{P-1} against a ligand molecule (Sec. 5.1, Eq.
    EnergySum_Mcomplex): E_p = sum_j q_j (sum over the molecules of their RS
    potentials)(x_j); a pose is flagged when it is flagged against any molecule."""
    quat = np.asarray(quat, dtype=np.float64)
    trans = np.asarray(trans, dtype=np.float64)
    q = np.asarray(lig_q, dtype=np.float64)
    x = posed_atoms(lig_xyz, quat_to_rot(quat), trans)
    P, L, _ = x.shape
    phi = np.zeros((P, L))
    flags = np.zeros(P, dtype=np.uint8)
    for m in models:
        pl, ps, _, _ = potential(m, x.reshape(-1, 3))
        phi += (pl + ps).reshape(P, L)
        flags |= _flags(m, x)[0]
    return {"E": (q[None, :] * phi).sum(axis=1), "S_ref": np.abs(q[None, :] * phi).sum(axis=1), "flags": flags}


def pose_gradients(model: RSModel, lig_xyz, lig_q, rotvec, trans, chunk: int = 1024):
    """Energy and exact gradient with respect to (translation, rotation vector):
    dE/dt = sum_j q_j grad phi(x_j);  dE/dw = J_l(w)^T sum_j q_j (R y_j) x grad phi(x_j)
    (the derivative of Eq. EnergySum_ligand under x_j = R(w) y_j + t; Sec. 3.3 and
    Sec. 4.2 force on a rigid cluster, taken exactly rather than by projection)."""
    rotvec = np.asarray(rotvec, dtype=np.float64)
    trans = np.asarray(trans, dtype=np.float64)
    q = np.asarray(lig_q, dtype=np.float64)
    y = ligand_frame(lig_xyz)
    P, L = rotvec.shape[0], q.size
    out = {"E": np.zeros(P), "dE_dt": np.zeros((P, 3)), "dE_dw": np.zeros((P, 3)),
           "flags": np.zeros(P, dtype=np.uint8), "S_ref": np.zeros(P), "T_ref": np.zeros(P),
           "W_ref": np.zeros(P)}
    for s0 in range(0, P, chunk):
        sl = slice(s0, min(P, s0 + chunk))
        R = rotvec_to_rot(rotvec[sl])
        ry = np.einsum("pij,lj->pli", R, y)
        x = ry + trans[sl][:, None, :]
        pl, ps, gl, gs = potential(model, x.reshape(-1, 3), grad=True)
        phi = (pl + ps).reshape(-1, L)
        gphi = (gl + gs).reshape(-1, L, 3)
        out["E"][sl] = (q[None, :] * phi).sum(axis=1)
        out["S_ref"][sl] = np.abs(q[None, :] * phi).sum(axis=1)
        qg = q[None, :, None] * gphi
        out["dE_dt"][sl] = qg.sum(axis=1)
        tau = np.cross(ry, qg).sum(axis=1)
        out["dE_dw"][sl] = np.einsum("pji,pj->pi", left_jacobian(rotvec[sl]), tau)
        # gradient scales: sum_j |q_j| |grad phi_j| and sum_j |q_j| |R y_j| |grad phi_j|
        gn = np.linalg.norm(qg, axis=2)
        out["T_ref"][sl] = gn.sum(axis=1)
        out["W_ref"][sl] = (gn * np.linalg.norm(ry, axis=2)).sum(axis=1)
        out["flags"][sl], _ = _flags(model, x)
    return out


# ----------------------------------------------------------------------------
# The paper's finite-difference force (Sec. 3.3, Eq. differ_ligand) and its
# resultants on a rigid cluster (Sec. 5.2, Eq. Field_Xcenter and Eq. Field_phi)
# ----------------------------------------------------------------------------
def fd_forces(model: RSModel, lig_xyz, lig_q, rotvec, trans, h: float | None = None,
              r0: float | None = None, chunk: int = 512):
    """Per-atom forces by the backward difference of Eq. differ_ligand and their
    rigid-cluster resultants.

    For ligand atom l at x_l and axis i:  F_{l,i} = q_l (phi(x_l) - phi(x_l - h e_i)) / h,
    phi the RS potential (long range + short range), h the grid step unless given.
    The quotient is taken as printed, so F_l approximates +grad_x of the energy.
    With r_l = x_l - x0 (x0 = the ligand's geometric centre = the translation),
    v_l = r_l / |r_l|:
      radial part      F_rad,l = (F_l . v_l) v_l   (F_l itself when |r_l| = 0)
      tangential part  F_tan,l = F_l - F_rad,l
      F0   = sum_l F_rad,l                         (Eq. Field_Xcenter)
      Fphi = sum_l (|r_l| / r0) F_tan,l            (Eq. Field_phi: each tangential
             part moved along v_l to radius r0 and scaled to keep its moment)
      M    = sum_l r_l x F_l                       (moment about x0; the 3-D form of
             summing the moved tangential parts along the sphere: r0 sum_l v_l x
             (|r_l|/r0) F_tan,l)
    and Fsum = sum_l F_l, dE_dw = J_l(w)^T M (the rotation-vector derivative that M
    stands for).  r0 defaults to the RMS distance of the ligand atoms from x0 (when
    that is 0 every atom sits at x0 and Fphi = 0)."""
    rotvec = np.asarray(rotvec, dtype=np.float64)
    trans = np.asarray(trans, dtype=np.float64)
    q = np.asarray(lig_q, dtype=np.float64)
    y = ligand_frame(lig_xyz)
    if h is None:
        h = model.h
    if r0 is None:
        r0 = math.sqrt(float((y * y).sum(axis=1).mean()))
    P, L = rotvec.shape[0], q.size
    out = {k: np.zeros((P, 3)) for k in ("Fsum", "F0", "Fphi", "M", "dE_dw")}
    out["E"] = np.zeros(P)
    # scales for tolerances: sum_l |q_l phi_l|, sum_l |F_l| and sum_l |r_l| |F_l|
    out["S_ref"], out["T_ref"], out["W_ref"] = np.zeros(P), np.zeros(P), np.zeros(P)
    out["flags"] = np.zeros(P, dtype=np.uint8)
    out["h"], out["r0"] = h, r0
    for s0 in range(0, P, chunk):
        sl = slice(s0, min(P, s0 + chunk))
        ry = np.einsum("pij,lj->pli", rotvec_to_rot(rotvec[sl]), y)
        x = ry + trans[sl][:, None, :]
        pl, ps, _, _ = potential(model, x.reshape(-1, 3))
        phi0 = (pl + ps).reshape(-1, L)
        F = np.zeros(x.shape)
        for i in range(3):
            xs = x.copy()
            xs[..., i] -= h
            pl, ps, _, _ = potential(model, xs.reshape(-1, 3))
            F[..., i] = q[None, :] * (phi0 - (pl + ps).reshape(-1, L)) / h
        rn = np.linalg.norm(ry, axis=2)
        at_centre = rn == 0.0
        v = ry / np.where(at_centre, 1.0, rn)[..., None]
        F_rad = np.where(at_centre[..., None], F, (F * v).sum(axis=2)[..., None] * v)
        F_tan = F - F_rad
        out["E"][sl] = (q[None, :] * phi0).sum(axis=1)
        out["S_ref"][sl] = np.abs(q[None, :] * phi0).sum(axis=1)
        out["Fsum"][sl] = F.sum(axis=1)
        out["F0"][sl] = F_rad.sum(axis=1)
        scale = rn / r0 if r0 > 0.0 else np.zeros_like(rn)  # r0 = 0: every atom at x0
        out["Fphi"][sl] = (scale[..., None] * F_tan).sum(axis=1)
        fn = np.linalg.norm(F, axis=2)
        out["T_ref"][sl] = fn.sum(axis=1)
        out["W_ref"][sl] = (fn * rn).sum(axis=1)
        M = np.cross(ry, F).sum(axis=1)
        out["M"][sl] = M
        out["dE_dw"][sl] = np.einsum("pji,pj->pi", left_jacobian(rotvec[sl]), M)
        out["flags"][sl], _ = _flags(model, x)
    return out


# ----------------------------------------------------------------------------
# Pose scan of Algorithm PPIEM (Sec. 3.4, steps A0-A7)
# ----------------------------------------------------------------------------
def ppiem_directions(n_theta: int, n_phi: int) -> np.ndarray:
    """Orbit positions of the ligand centre around the protein centre (A0, A5): unit
    vectors at polar angles (a + 1/2) pi / n_theta and azimuths 2 pi b / n_phi,
    index a * n_phi + b."""
    th = (np.arange(n_theta) + 0.5) * math.pi / n_theta
    ph = np.arange(n_phi) * 2.0 * math.pi / n_phi
    T, F = np.meshgrid(th, ph, indexing="ij")
    return np.stack([np.sin(T) * np.cos(F), np.sin(T) * np.sin(F), np.cos(T)], axis=-1).reshape(-1, 3)


def contact_offsets(prot_xyz, sigma: float, lig_xyz, quat, x_P, u):
    """Step A3: the ligand (rotated by quat about its centre) approaches the protein
    along the line x_P + s u from s = +inf; the result is the first s at which some
    ligand-protein distance reaches sigma, i.e. the largest upper end of the
    intervals {s : |x_P + s u + R y_j - x_m| < sigma} over all atom pairs:
      w = x_m - x_P - R y_j,  c = u . w,  q = |w|^2 - c^2 (squared distance of x_m
      from atom j's line),  s_jm = c + sqrt(sigma^2 - q)  for q < sigma^2.
    Brute force over all pairs; -inf where no pair blocks.  quat (P, 4), u (P, 3)."""
    prot = np.asarray(prot_xyz, np.float64)
    y = ligand_frame(lig_xyz)
    R = quat_to_rot(quat)
    u = np.asarray(u, np.float64)
    P = u.shape[0]
    out = np.full(P, -np.inf)
    s2 = sigma * sigma
    for p in range(P):
        ry = R[p] @ y.T                                   # (3, L)
        w = prot[:, None, :] - (np.asarray(x_P)[None, None, :] + ry.T[None, :, :])   # (N, L, 3)
        c = w @ u[p]
        q = (w * w).sum(axis=2) - c * c
        hit = q < s2
        if hit.any():
            out[p] = (c[hit] + np.sqrt(s2 - q[hit])).max()
    return out


def ppiem_scan(model: RSModel, lig_xyz, lig_q, quats, n_theta: int, n_phi: int, x_P=None,
               margin: float = 1e-6):
    """Steps A2-A6 of Algorithm PPIEM for every orbit direction u_d (A5) and every
    self-rotation q_r (A4): the contact offset s*_dr (A3), the pose
    (q_r, x_P + (s*_dr + margin sigma) u_d) just outside contact, its energy and flags.
    A6 reads as: per direction the lowest feasible energy over the self-rotations
    (ties: lowest r), then the directions whose lowest energy is a local minimum over
    their grid neighbours (a +- 1 in theta without wrap, b +- 1 in phi with wrap;
    ties broken by the lower direction index).  x_P defaults to the protein's
    geometric centre (A2).  A direction with no contact has s* = -inf, energy +inf
    and flag 4."""
    quats = np.asarray(quats, np.float64)
    U = ppiem_directions(n_theta, n_phi)
    D, Rn = U.shape[0], quats.shape[0]
    if x_P is None:
        x_P = model.prot_xyz.mean(axis=0)
    x_P = np.asarray(x_P, np.float64)
    qq = np.tile(quats, (D, 1))
    uu = np.repeat(U, Rn, axis=0)
    s = contact_offsets(model.prot_xyz, model.sigma, lig_xyz, qq, x_P, uu)
    E = np.full(D * Rn, np.inf)
    S_ref = np.zeros(D * Rn)      # tolerance scale sum_j |q_j phi_j| of each pose
    flags = np.full(D * Rn, 4, dtype=np.uint8)
    ok = np.isfinite(s)
    if ok.any():
        t = x_P[None, :] + (s[ok] + margin * model.sigma)[:, None] * uu[ok]
        ev = pose_energies(model, lig_xyz, lig_q, qq[ok], t)
        E[ok], flags[ok], S_ref[ok] = ev["E"], ev["flags"], ev["S_ref"]
    E2, F2 = E.reshape(D, Rn), flags.reshape(D, Rn)
    Ef = np.where(F2 == 0, E2, np.inf)
    best = np.argmin(Ef, axis=1)                         # first index among equal minima
    E_best = Ef[np.arange(D), best]
    best = np.where(np.isfinite(E_best), best, -1)
    is_min = np.zeros(D, dtype=bool)
    for a in range(n_theta):
        for b in range(n_phi):
            d = a * n_phi + b
            if not np.isfinite(E_best[d]):
                continue
            nbs = [a2 * n_phi + b for a2 in (a - 1, a + 1) if 0 <= a2 < n_theta]
            nbs += [a * n_phi + (b - 1) % n_phi, a * n_phi + (b + 1) % n_phi]
            is_min[d] = all(E_best[d] < E_best[e] or (E_best[d] == E_best[e] and d < e)
                            for e in nbs if e != d)
    return {"dirs": U, "s": s.reshape(D, Rn), "E": E2, "flags": F2, "E_best": E_best,
            "rot_best": best, "is_min": is_min, "x_P": x_P, "S_ref": S_ref.reshape(D, Rn)}


# ----------------------------------------------------------------------------
# Direct Coulomb (Sec. 3.1, Eq. EnergyLatSum_mixed and Eq. EnergySum_partial;
# forces Sec. 3.3)
# ----------------------------------------------------------------------------
def coulomb_energies(prot_xyz, prot_q, lig_xyz, lig_q, quat, trans, chunk: int = 64):
    """E(M,L) = sum_l sum_m z_l z_m / |x_m - x_l| (Eq. EnergyLatSum_mixed)."""
    prot_xyz = np.asarray(prot_xyz, np.float64)
    zq = np.asarray(prot_q, np.float64)
    q = np.asarray(lig_q, np.float64)
    P = len(quat)
    E = np.zeros(P)
    for s0 in range(0, P, chunk):
        sl = slice(s0, min(P, s0 + chunk))
        x = posed_atoms(lig_xyz, quat_to_rot(np.asarray(quat)[sl]), np.asarray(trans)[sl])
        d = np.linalg.norm(x[:, :, None, :] - prot_xyz[None, None], axis=-1)
        E[sl] = (q[None, :, None] * zq[None, None, :] / d).sum(axis=(1, 2))
    return E


def coulomb_gradients(prot_xyz, prot_q, lig_xyz, lig_q, rotvec, trans):
    """Analytic gradient of E(M,L) w.r.t. (t, w): grad_x phi = -sum_m z_m (x-x_m)/|x-x_m|^3
    (Sec. 3.3, the field E_M), chained through x_j = R(w) y_j + t as in pose_gradients."""
    prot_xyz = np.asarray(prot_xyz, np.float64)
    zq = np.asarray(prot_q, np.float64)
    q = np.asarray(lig_q, np.float64)
    rotvec = np.asarray(rotvec, np.float64)
    y = ligand_frame(lig_xyz)
    R = rotvec_to_rot(rotvec)
    ry = np.einsum("pij,lj->pli", R, y)
    x = ry + np.asarray(trans, np.float64)[:, None, :]
    diff = x[:, :, None, :] - prot_xyz[None, None]
    d = np.linalg.norm(diff, axis=-1)
    E = (q[None, :, None] * zq[None, None, :] / d).sum(axis=(1, 2))
    gphi = -(zq[None, None, :, None] * diff / d[..., None] ** 3).sum(axis=2)
    qg = q[None, :, None] * gphi
    dt = qg.sum(axis=1)
    tau = np.cross(ry, qg).sum(axis=1)
    dw = np.einsum("pji,pj->pi", left_jacobian(rotvec), tau)
    return E, dt, dw


# ----------------------------------------------------------------------------
# Constrained minimisation step (Sec. 3.4, Eq. Energy_Min) and ranking
# ----------------------------------------------------------------------------
def pgd_step(model: RSModel, lig_xyz, lig_q, rotvec, trans, eta_t: float = 0.1,
             eta_r: float = 0.02, max_halvings: int = 5):
    """One projected-gradient step on (t, w) for arg min E s.t. dist >= sigma
    (Eq. Energy_Min): normalised steps of length eta_t (Angstrom) and eta_r (rad);
    the step is halved up to max_halvings times until the trial pose is feasible
    with E_trial <= E; otherwise the pose is kept."""
    rotvec = np.asarray(rotvec, np.float64).copy()
    trans = np.asarray(trans, np.float64).copy()
    cur = pose_gradients(model, lig_xyz, lig_q, rotvec, trans)
    gt, gw = cur["dE_dt"], cur["dE_dw"]
    nt = np.linalg.norm(gt, axis=1)
    nw = np.linalg.norm(gw, axis=1)
    dt = np.where(nt[:, None] > 0, -eta_t * gt / np.where(nt > 0, nt, 1)[:, None], 0.0)
    dw = np.where(nw[:, None] > 0, -eta_r * gw / np.where(nw > 0, nw, 1)[:, None], 0.0)
    P = rotvec.shape[0]
    done = np.zeros(P, dtype=bool)
    new_t, new_w, new_E = trans.copy(), rotvec.copy(), cur["E"].copy()
    accepted = np.full(P, -1, dtype=np.int64)
    for s in range(max_halvings + 1):
        idx = np.nonzero(~done)[0]
        if idx.size == 0:
            break
        sc = 0.5 ** s
        tt = trans[idx] + sc * dt[idx]
        ww = rotvec[idx] + sc * dw[idx]
        quat = _rotvec_to_quat(ww)
        ev = pose_energies(model, lig_xyz, lig_q, quat, tt)
        ok = (ev["flags"] == 0) & (ev["E"] <= cur["E"][idx])
        acc = idx[ok]
        new_t[acc], new_w[acc], new_E[acc] = tt[ok], ww[ok], ev["E"][ok]
        accepted[acc] = s
        done[acc] = True
    return {"trans": new_t, "rotvec": new_w, "E": new_E, "accepted": accepted,
            "E_start": cur["E"], "dE_dt": gt, "dE_dw": gw}


def _rotvec_to_quat(w: np.ndarray) -> np.ndarray:
    th = np.linalg.norm(w, axis=-1)
    small = th < 1e-8
    ths = np.where(small, 1.0, th)
    s = np.where(small, 0.5 - th ** 2 / 48, np.sin(ths / 2) / ths)
    return np.concatenate([np.cos(th / 2)[:, None], w * s[:, None]], axis=1)


def feasible_topk(E: np.ndarray, flags: np.ndarray, k: int = 10) -> np.ndarray:
    """Indices of the k lowest-energy feasible poses (flags == 0), ascending E."""
    idx = np.nonzero(np.asarray(flags) == 0)[0]
    order = idx[np.argsort(np.asarray(E)[idx], kind="stable")]
    return order[:k]


def tolerance_scale(E_ref: np.ndarray, S_ref: np.ndarray) -> np.ndarray:
    """Per-pose error denominator max(|E_ref|, 1e-2 * S_ref), S_ref = sum_j |q_j phi(x_j)|."""
    return np.maximum(np.abs(E_ref), 1e-2 * np.asarray(S_ref))
