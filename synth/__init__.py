"""Seeded synthetic inputs (geometry, densities, octree U-lists).

Shared by the tests, the benchmark and the oracle checks.  Holds none of the
layer-potential arithmetic: only the surfaces and structures the sums run over.
"""
