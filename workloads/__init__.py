"""Seeded synthetic inputs shared by the tests, the oracle and the benchmark.

This package draws random numbers and places points; it holds none of the
electrostatics (no sinc quadrature, no factors, no energies).
"""
from .synth import *  # noqa: F401,F403
