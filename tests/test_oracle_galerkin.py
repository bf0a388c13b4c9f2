"""Pins of the oracle's Galerkin factors (Sec. 2, Eq. galten: projection of the
Gaussians on the cells): each entry against numerical quadrature of the cell
integral, the collocation limit as the cell shrinks, and the long-range potential
against the Coulomb law.  CPU only."""
import math

import numpy as np
from scipy import integrate

import oracle as O
import workloads as W


def test_galerkin_entries_are_cell_averages():
    tab = O.sinc_table(16.0, 1.0, 12)
    x_m = np.array([[0.37, -1.2, 2.05]])
    n, b = 33, 16.0
    h = 2 * b / (n - 1)
    U, _ = O.long_range_factors(x_m, np.array([1.0]), tab, n, b, galerkin=True)
    x = O.grid_nodes(n, b)
    tl = tab.t[tab.is_long]
    rng = np.random.default_rng(0)
    for _ in range(40):
        ax, i, k = rng.integers(0, 3), rng.integers(0, n), rng.integers(0, tl.size)
        f = lambda s: math.exp(-(tl[k] * (s - x_m[0, ax])) ** 2)
        val, _ = integrate.quad(f, x[i] - h / 2, x[i] + h / 2, epsabs=0, epsrel=1e-13)
        assert abs(U[ax][i, k] - val / h) <= 1e-11 * abs(val / h) + 1e-300, (ax, i, k, U[ax][i, k], val / h)


def test_galerkin_tends_to_collocation():
    # a finer grid (smaller cells) brings the averages to the node values: O(t^2 h^2)
    tab = O.sinc_table(16.0, 1.0, 12)
    x_m = np.array([[0.37, -1.2, 2.05]])
    errs = []
    wide = tab.t[tab.is_long] <= 0.5  # t h <= 1/2 already on the coarsest grid (h = 1)
    for n in (33, 65, 129):
        Ug, _ = O.long_range_factors(x_m, np.array([1.0]), tab, n, 16.0, galerkin=True)
        Uc, _ = O.long_range_factors(x_m, np.array([1.0]), tab, n, 16.0)
        errs.append(max(np.abs(Ug[a][:, wide] - Uc[a][:, wide]).max() for a in range(3)))
    assert errs[1] < errs[0] / 3.5 and errs[2] < errs[1] / 3.5


def test_galerkin_long_range_follows_coulomb():
    # far from the charge the long-range potential is 1/r; cell averaging adds the
    # O(h^2) smoothing of each Gaussian, small against 1/r at these distances
    w = W.plain_small(P=1)
    m = O.build_model(w.prot_xyz[:1], np.array([1.0]), 129, 32.0, 3.0, 20, galerkin=True)
    rng = np.random.default_rng(1)
    x = w.prot_xyz[0] + rng.normal(size=(200, 3)) * 6.0
    x = x[(np.linalg.norm(x - w.prot_xyz[0], axis=1) > 6.0) & np.all(np.abs(x) < 31.0, axis=1)]
    pl, _, _, _ = O.potential(m, x)
    r = np.linalg.norm(x - w.prot_xyz[0], axis=1)
    assert np.abs(pl * r - 1.0).max() < 2e-3
