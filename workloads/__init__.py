"""Seeded synthetic inputs (H, S, n_occ) shared by the tests, the bench and the oracle checks.

This package builds inputs only. It holds none of the solver's arithmetic: no S^{-1/2}, no
purification, no density matrix. The construction data it returns (Haar factors, the exact
generalised spectrum, the eigen-factors of S) let the oracle side write closed forms.
"""
from .synthetic import (  # noqa: F401
    Problem,
    haar_orthogonal,
    make_config0,
    make_config1,
    make_config2,
    make_batch_config3,
    make_spectrum_problem,
    make_request_stream,
    make_request_problem,
    make_small_diag,
    make_random_small,
    make_geometry_step,
    make_banded,
)
