"""Seeded generators for protein-shaped point-charge clusters, ligands and pose batches.

Shapes follow the paper's setting (Sec. 3.1, a large cluster M and a small
rigid cluster L; Sec. 3.4, poses = rotation about the ligand's geometric centre
plus a translation of that centre).  The paper's own protein (Sec. 4.2, 379
atoms) is not available, so these recipes stand in for it:

* ``plain_small``  : N=200 charges uniform in a 20 A ball, 10 % set to +-1;
                     L=20 ligand atoms in a 5 A ball; n=257 on [-32,32]^3;
                     1000 poses on a 25 A shell.
* ``plain_protein``: N=3000 sites of a jittered 1.5 A lattice in an ellipsoid
                     (20,14,10) A, 8 % at +-1; L=50; n=1025 on [-64,64]^3;
                     1e5 poses with |t| in [10,30] A.
* ``batch_pairs``  : uneven protein/ligand pairs (N log-uniform [500,20000],
                     L uniform [10,200], n matched to the box).
* ``pgd_start``    : N=10000, L=100, n=2049, feasible starting poses.

Everything is float64 numpy.  Quaternions are unit, stored (w, x, y, z).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "Workload", "ball_uniform", "mixed_charges", "shoemake_quaternions",
    "shell_translations", "ellipsoid_lattice", "sphere_lattice",
    "plain_small", "plain_protein", "batch_pairs", "pgd_start", "tiny", "euler_grid_quaternions",
    "random_rotvecs", "serve_pool", "serve_request", "poisson_arrivals", "WORKLOADS",
]


@dataclass
class Workload:
    name: str
    prot_xyz: np.ndarray          # (N, 3) float64, Angstrom
    prot_q: np.ndarray            # (N,)   float64, e
    lig_xyz: np.ndarray           # (L, 3) float64, ligand frame (not re-centred)
    lig_q: np.ndarray             # (L,)   float64
    quat: np.ndarray              # (P, 4) float64 unit quaternions (w, x, y, z)
    trans: np.ndarray             # (P, 3) float64 position of the ligand centre
    n: int                        # grid nodes per axis
    b: float                      # box half-width: grid spans [-b, b]^3
    sigma: float = 3.0            # van der Waals distance
    R_l: int = 20                 # long-range sinc terms
    tucker_cap: int = 0           # 0: keep the unreduced canonical long-range part
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.prot_xyz.shape[0])

    @property
    def L(self) -> int:
        return int(self.lig_xyz.shape[0])

    @property
    def P(self) -> int:
        return int(self.quat.shape[0])

    def subset(self, idx) -> "Workload":
        idx = np.asarray(idx)
        return Workload(self.name, self.prot_xyz, self.prot_q, self.lig_xyz, self.lig_q,
                        self.quat[idx], self.trans[idx], self.n, self.b, self.sigma,
                        self.R_l, self.tucker_cap, dict(self.meta))


def _unit_vectors(rng: np.random.Generator, count: int) -> np.ndarray:
    v = rng.standard_normal((count, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def ball_uniform(rng: np.random.Generator, count: int, radius: float) -> np.ndarray:
    """Points uniform in a ball: uniform direction, radius R*u^(1/3)."""
    d = _unit_vectors(rng, count)
    r = radius * rng.random(count) ** (1.0 / 3.0)
    return d * r[:, None]


def mixed_charges(rng: np.random.Generator, count: int, std: float, frac_unit: float) -> np.ndarray:
    """N(0, std) partial charges with a random fraction replaced by +-1."""
    q = rng.normal(0.0, std, count)
    k = int(round(frac_unit * count))
    if k > 0:
        idx = rng.choice(count, size=k, replace=False)
        q[idx] = rng.choice(np.array([-1.0, 1.0]), size=k)
    return q


def shoemake_quaternions(rng: np.random.Generator, count: int) -> np.ndarray:
    """Uniform random unit quaternions (Shoemake 1992), returned as (w, x, y, z)."""
    u1, u2, u3 = rng.random(count), rng.random(count), rng.random(count)
    a, c = np.sqrt(1.0 - u1), np.sqrt(u1)
    x = a * np.sin(2 * np.pi * u2)
    y = a * np.cos(2 * np.pi * u2)
    z = c * np.sin(2 * np.pi * u3)
    w = c * np.cos(2 * np.pi * u3)
    return np.stack([w, x, y, z], axis=1)


def shell_translations(rng: np.random.Generator, count: int, r_lo: float, r_hi: float) -> np.ndarray:
    """Uniform directions; radius uniform in [r_lo, r_hi] (a thin shell when equal)."""
    d = _unit_vectors(rng, count)
    r = r_lo + (r_hi - r_lo) * rng.random(count)
    return d * r[:, None]


def random_rotvecs(rng: np.random.Generator, count: int, max_angle: float = math.pi) -> np.ndarray:
    """Rotation vectors with uniform axis and angle uniform in [0, max_angle)."""
    return _unit_vectors(rng, count) * (max_angle * rng.random(count))[:, None]


def ellipsoid_lattice(rng: np.random.Generator, count: int, semi_axes, spacing: float,
                      jitter: float) -> np.ndarray:
    """The ``count`` sites of a cubic lattice nearest the centre in ellipsoidal norm,
    each jittered uniformly in [-jitter, jitter] per coordinate."""
    ax = np.asarray(semi_axes, dtype=np.float64)
    m = int(math.ceil(ax.max() / spacing)) + 2
    g = np.arange(-m, m + 1) * spacing
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    en = np.sqrt(((pts / ax) ** 2).sum(axis=1))
    order = np.lexsort((pts[:, 2], pts[:, 1], pts[:, 0], en))
    pts = pts[order[:count]].copy()
    pts += rng.uniform(-jitter, jitter, pts.shape)
    return pts


def sphere_lattice(rng: np.random.Generator, count: int, spacing: float = 1.5,
                   jitter: float = 0.25) -> tuple[np.ndarray, float]:
    """``count`` jittered lattice sites nearest the centre of a sphere of radius
    spacing*(3*count/(4*pi))^(1/3); returns (points, radius)."""
    r = spacing * (3.0 * count / (4.0 * math.pi)) ** (1.0 / 3.0)
    pts = ellipsoid_lattice(rng, count, (r, r, r), spacing, jitter)
    return pts, r


def tiny(seed: int = 0, N: int = 3, L: int = 2, P: int = 4, n: int = 17, b: float = 8.0,
         R_l: int = 8, sigma: float = 1.0) -> Workload:
    """Very small cases for brute-force checks (full n^3 tensors fit in memory)."""
    rng = np.random.default_rng(seed)
    prot = ball_uniform(rng, N, 2.5)
    zq = rng.normal(0.0, 0.5, N)
    lig = ball_uniform(rng, L, 1.0)
    lq = rng.normal(0.0, 0.5, L)
    quat = shoemake_quaternions(rng, P)
    trans = shell_translations(rng, P, 3.5, 4.5)
    return Workload("tiny", prot, zq, lig, lq, quat, trans, n, b, sigma, R_l, 0,
                    {"seed": seed})


def plain_small(seed: int = 0, P: int = 1000) -> Workload:
    rng = np.random.default_rng(seed)
    prot = ball_uniform(rng, 200, 20.0)
    zq = mixed_charges(rng, 200, 0.3, 0.10)
    lig = ball_uniform(rng, 20, 5.0)
    lq = rng.normal(0.0, 0.3, 20)
    quat = shoemake_quaternions(rng, P)
    trans = shell_translations(rng, P, 25.0, 25.0)
    return Workload("plain_small", prot, zq, lig, lq, quat, trans, n=257, b=32.0,
                    sigma=3.0, R_l=20, tucker_cap=0, meta={"seed": seed})


def plain_protein(seed: int = 1, P: int = 100_000, tucker_cap: int = 20) -> Workload:
    rng = np.random.default_rng(seed)
    prot = ellipsoid_lattice(rng, 3000, (20.0, 14.0, 10.0), 1.5, 0.25)
    zq = mixed_charges(rng, 3000, 0.3, 0.08)
    r_lig = 5.0 * (50.0 / 20.0) ** (1.0 / 3.0)
    lig = ball_uniform(rng, 50, r_lig)
    lq = rng.normal(0.0, 0.3, 50)
    quat = shoemake_quaternions(rng, P)
    trans = shell_translations(rng, P, 10.0, 30.0)
    return Workload("plain_protein", prot, zq, lig, lq, quat, trans, n=1025, b=64.0,
                    sigma=3.0, R_l=20, tucker_cap=tucker_cap, meta={"seed": seed})


_N_CHOICES = (513, 1025, 2049, 4097)


def batch_pairs(seed: int = 2, pairs: int = 64, P: int = 10_000, tucker_cap: int = 20,
                n_max: int = 4097) -> list[Workload]:
    """Uneven protein-ligand pairs; n picked by quartile of the box half-width b."""
    rng = np.random.default_rng(seed)
    out = []
    bs = []
    for p in range(pairs):
        N = int(round(math.exp(rng.uniform(math.log(500.0), math.log(20000.0)))))
        L = int(rng.integers(10, 201))
        prot, r_p = sphere_lattice(rng, N)
        zq = mixed_charges(rng, N, 0.3, 0.08)
        r_l = 5.0 * (L / 20.0) ** (1.0 / 3.0)
        lig = ball_uniform(rng, L, r_l)
        lq = rng.normal(0.0, 0.3, L)
        quat = shoemake_quaternions(rng, P)
        trans = shell_translations(rng, P, r_p, r_p + 2.0 * r_l + 3.0)
        b = r_p + 2.0 * r_l + 8.0
        bs.append(b)
        out.append(Workload(f"pair{p:02d}", prot, zq, lig, lq, quat, trans, n=0, b=b,
                            sigma=3.0, R_l=20, tucker_cap=tucker_cap,
                            meta={"seed": seed, "pair": p}))
    qs = np.quantile(np.asarray(bs), [0.25, 0.5, 0.75])
    for w in out:
        k = int(np.searchsorted(qs, w.b, side="right"))
        w.n = min(_N_CHOICES[k], n_max)
    return out


def pgd_start(seed: int = 3, P: int = 4096, N: int = 10000, L: int = 100, n: int = 2049,
              tucker_cap: int = 20, feasible=None) -> Workload:
    """Starting poses for projected gradient descent.  ``feasible`` is an optional
    callable (quat, trans) -> bool mask used for rejection sampling."""
    rng = np.random.default_rng(seed)
    prot, r_p = sphere_lattice(rng, N)
    zq = mixed_charges(rng, N, 0.3, 0.08)
    r_l = 5.0 * (L / 20.0) ** (1.0 / 3.0)
    lig = ball_uniform(rng, L, r_l)
    lq = rng.normal(0.0, 0.3, L)
    b = r_p + 2.0 * r_l + 8.0
    quats, transs, got = [], [], 0
    while got < P:
        m = 2 * (P - got) + 64
        qq = shoemake_quaternions(rng, m)
        tt = shell_translations(rng, m, r_p, r_p + 2.0 * r_l + 3.0)
        if feasible is not None:
            ok = np.asarray(feasible(qq, tt), dtype=bool)
            qq, tt = qq[ok], tt[ok]
        quats.append(qq)
        transs.append(tt)
        got += len(qq)
    quat = np.concatenate(quats)[:P]
    trans = np.concatenate(transs)[:P]
    return Workload("pgd_start", prot, zq, lig, lq, quat, trans, n=n, b=b, sigma=3.0,
                    R_l=20, tucker_cap=tucker_cap, meta={"seed": seed})


_SERVE_N_CHOICES = (1025, 2049, 4097, 8193, 16385)
_SERVE_L_MAX = 200


def serve_pool(seed: int = 5, proteins: int = 64, n_max: int = 16385, tucker_cap: int = 20) -> list[dict]:
    """Proteins of a serving stream: N log-uniform in [500, 20000] on jittered lattice
    spheres, charges as elsewhere; the box fits the largest ligand of the stream
    (L = 200) and the grid n is picked by quintile of the box half-width b from
    1025 ... 16385 (capped at n_max)."""
    rng = np.random.default_rng(seed)
    r_l_max = 5.0 * (_SERVE_L_MAX / 20.0) ** (1.0 / 3.0)
    out = []
    for p in range(proteins):
        N = int(round(math.exp(rng.uniform(math.log(500.0), math.log(20000.0)))))
        prot, r_p = sphere_lattice(rng, N)
        zq = mixed_charges(rng, N, 0.3, 0.08)
        out.append({"id": p + 1, "xyz": prot, "q": zq, "r_p": r_p,
                    "b": r_p + 2.0 * r_l_max + 8.0, "sigma": 3.0, "R_l": 20,
                    "tucker_cap": tucker_cap})
    qs = np.quantile(np.asarray([e["b"] for e in out]), [0.2, 0.4, 0.6, 0.8])
    for e in out:
        k = int(np.searchsorted(qs, e["b"], side="right"))
        e["n"] = min(_SERVE_N_CHOICES[k], n_max)
    return out


def serve_request(rng: np.random.Generator, prot: dict, P: int = 2048) -> dict:
    """One docking request against a pool protein: a new ligand (L uniform in
    [10, 200], ball of radius 5 (L/20)^(1/3), charges N(0, 0.3)) and P poses
    (uniform rotations, centres on the shell outside the protein)."""
    L = int(rng.integers(10, _SERVE_L_MAX + 1))
    r_l = 5.0 * (L / 20.0) ** (1.0 / 3.0)
    return {"lig_xyz": ball_uniform(rng, L, r_l), "lig_q": rng.normal(0.0, 0.3, L),
            "quat": shoemake_quaternions(rng, P),
            "trans": shell_translations(rng, P, prot["r_p"], prot["r_p"] + 2.0 * r_l + 3.0)}


def euler_grid_quaternions(m_L: int) -> np.ndarray:
    """Self-rotations of the ligand for a pose scan with angular step 2 pi / m_L
    (m_L even): ZYZ Euler angles alpha, gamma in {2 pi i / m_L} and beta at the
    midpoints (k + 1/2) 2 pi / m_L of [0, pi]; m_L^3 / 2 unit quaternions (w, x, y, z),
    alpha slowest."""
    if m_L < 2 or m_L % 2:
        raise ValueError("m_L must be even and >= 2")
    step = 2.0 * math.pi / m_L
    out = []
    for i in range(m_L):
        for k in range(m_L // 2):
            for g in range(m_L):
                a, b, c = i * step, (k + 0.5) * step, g * step
                # q = q_z(a) q_y(b) q_z(c)
                ca, sa = math.cos(a / 2), math.sin(a / 2)
                cb, sb = math.cos(b / 2), math.sin(b / 2)
                cc, sc = math.cos(c / 2), math.sin(c / 2)
                w = ca * cb * cc - sa * cb * sc
                x = ca * sb * sc - sa * sb * cc
                y = ca * sb * cc + sa * sb * sc
                z = ca * cb * sc + sa * cb * cc
                out.append((w, x, y, z))
    return np.asarray(out, dtype=np.float64)


def poisson_arrivals(rng: np.random.Generator, rate: float, duration: float) -> np.ndarray:
    """Arrival times (s) of a Poisson stream of the given rate over [0, duration)."""
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return np.asarray(out)
        out.append(t)


WORKLOADS = {
    "plain_small": plain_small,
    "plain_protein": plain_protein,
}
