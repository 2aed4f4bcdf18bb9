"""Seeded synthetic inputs (meshes, bathymetry, initial states, forcing tracks).

Shared by the oracle-side tests and the CUDA-side tests/bench; holds no
shallow-water tendency or time-integration arithmetic.
"""
