"""GB300-native range-separated (RS) tensor electrostatics for rigid ligand poses.

Implements the data-parallel path of arXiv 2510.26611 (Algorithms TEP and PLIE,
the vdW constraint of Eq. Energy_Min, and the rigid-body gradient) as CUDA
kernels for sm_103a behind the C ABI in include/rs.h.  ``lib`` is the thin
ctypes binding; importing it builds and loads librs.so.
"""
from importlib import import_module

__all__ = ["lib"]


def __getattr__(name):
    if name == "lib":
        return import_module(".lib", __name__)
    raise AttributeError(name)
