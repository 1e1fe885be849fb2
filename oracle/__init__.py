"""FP64 CPU oracle for ChFSI and R-ChFSI (test infrastructure only).

A plain, slow, obviously correct NumPy/SciPy restatement of the paper's method, used to
check the CUDA path.  Only the test suite, the smoke check and the CPU-baseline leg of
the benchmark may import it; the library itself never does.  It shares no code with the
CUDA path: both read their inputs from the `workloads` generators.

Contents and what they follow:
    chebyshev   scaled/shifted Chebyshev polynomials and the sigma-scaled recurrence
                coefficients (Section 2.1, Eq. for the ChFSI recurrence; a_k, b_k, c_k of
                Section 3.2.1)
    filters     Algorithm 2 (ChFSI filter) and Algorithm 3 (R-ChFSI filter), plus the
                eigenvalue recurrence (Proposition 3.3)
    rr          Rayleigh-Ritz for a non-orthogonal basis and the residual (Section 2.1,
                Algorithm 1 steps 2-3)
    lanczos     k-step Lanczos upper bound of the filter operator's spectrum
    solver      Algorithm 1 with either filter
    fe          global assembly A = sum_c P_c^T A_c P_c of a cell-matrix operator
    angles      maximum principal angle (Definition 2.1)
"""
from . import chebyshev, filters, rr, lanczos, solver, fe, angles  # noqa: F401
