"""Pins of the oracle's molecular-complex energy (Sec. 5.1, Eq. EnergySum_Mcomplex):
linearity of the RS construction in the charges makes the complex of two molecules
equal to the one molecule built on their union, and a complex of one molecule is the
molecule itself.  CPU only."""
import numpy as np

import oracle as O
import workloads as W


def test_complex_of_split_molecule_equals_union():
    w = W.plain_small(P=64)
    half = w.prot_xyz.shape[0] // 2
    kw = dict(n=129, b=w.b, sigma=w.sigma, R_l=w.R_l)
    m1 = O.build_model(w.prot_xyz[:half], w.prot_q[:half], **kw)
    m2 = O.build_model(w.prot_xyz[half:], w.prot_q[half:], **kw)
    mu = O.build_model(w.prot_xyz, w.prot_q, **kw)
    c = O.complex_energies([m1, m2], w.lig_xyz, w.lig_q, w.quat, w.trans)
    u = O.pose_energies(mu, w.lig_xyz, w.lig_q, w.quat, w.trans)
    assert np.abs(c["E"] - u["E"]).max() <= 1e-12 * np.abs(u["S_ref"]).max()
    assert np.array_equal(c["flags"], u["flags"])


def test_complex_of_one_molecule():
    w = W.plain_small(P=32)
    m = O.build_model(w.prot_xyz, w.prot_q, 129, w.b, w.sigma, w.R_l, tucker_cap=10)
    c = O.complex_energies([m], w.lig_xyz, w.lig_q, w.quat, w.trans)
    e = O.pose_energies(m, w.lig_xyz, w.lig_q, w.quat, w.trans)
    assert np.array_equal(c["E"], e["E"]) and np.array_equal(c["flags"], e["flags"])
