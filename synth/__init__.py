"""Seeded synthetic inputs (scanner geometry, spectral tables, phantoms, Poisson data).

This package holds input preparation only: it is shared by the tests, the
benchmark and the oracle's own checks, and contains none of the reconstruction
method's steps.
"""
