"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

Holds none of the method's arithmetic: only constructions of test matrices
A = U0 diag(sigma) V0^T (+ 1 c^T) (+ noise) with prescribed spectra, and
their storage-precision roundings.
"""
