"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This package holds workload geometry and value distributions only: octree node
lists, cell densities sampled at cell centres, random moment fields and probe
selections. It contains none of the interaction arithmetic (no moments, no
Green's-function derivatives, no contractions); both the oracle and the CUDA
library compute those independently from these inputs.
"""
from .inputs import *  # noqa: F401,F403
