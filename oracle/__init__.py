"""FP64 CPU oracle for the range-separated (RS) tensor energy of rigid ligand poses.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA path is checked against.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the library
``paper_2510_26611_gb300`` never does, and the two share no code.

Every function cites the passage of the paper (arXiv 2510.26611, "Fast
tensor-based electrostatic energy calculations in the perspective of
protein-ligand docking problem") that it follows.
"""
from .rs_oracle import *  # noqa: F401,F403
