"""Seeded synthetic problem generators shared by the oracle and the CUDA path.

This package only *builds inputs*: matrices with prescribed spectra, finite-element
cell matrices, approximate inverses, initial guesses and arrival streams.  It holds
none of the eigensolver's arithmetic (no Chebyshev recurrence, no Rayleigh-Ritz,
no residuals).  Every generator is a pure function of its arguments and a seed,
so the oracle and the GPU path receive identical bytes.
"""
from .dense import (orthogonal, config1_spectrum, dense_from_spectrum, dense_config1,
                    dense_config2, toy_standard, toy_generalized, gaussian_block)
from .fe import (gll_1d, fe_mesh, fe_problem, fe_1d_matrices, fe_config3, fe_kpoint_problem,
                 fe_config4_list, fe_scf_chain)

__all__ = ["orthogonal", "config1_spectrum", "dense_from_spectrum", "dense_config1",
           "dense_config2", "toy_standard", "toy_generalized", "gaussian_block",
           "gll_1d", "fe_mesh", "fe_problem", "fe_1d_matrices", "fe_config3",
           "fe_kpoint_problem", "fe_config4_list", "fe_scf_chain"]
