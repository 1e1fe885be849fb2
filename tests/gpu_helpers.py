"""Shared helpers of the GPU parity tests: building the library and running the oracle on the
same seeded inputs."""
import numpy as np

import workloads as wl
from oracle import filters, rr

from paper_2503_22652_gb300 import build as B
from paper_2503_22652_gb300 import Solver


def ensure_built():
    B.build()


def relfro(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dense_case(m, N, seed=3, generalized=False, dense_dinv=False, perturbed=False):
    """A random symmetric problem with a spread spectrum plus inputs of one filter call."""
    rng = np.random.default_rng(seed)
    lam = np.sort(rng.uniform(-1.0, 9.0, m))
    A = wl.dense_from_spectrum(wl.orthogonal(m, seed + 1), lam)
    case = {"A": A, "B": None, "Dinv": None, "Dinv_dense": None, "A_filter": None}
    if generalized:
        c = wl.dense_config2(m=m, seed_q=seed + 1)
        case["A"], case["B"], case["Dinv"] = c["A"], c["B"], c["Dinv"]
    if dense_dinv:
        g = wl.toy_generalized(1e-3, m=m, n=max(2, N // 2))
        case["A"], case["B"], case["Dinv_dense"] = g["A"], g["B"], g["Dinv_dense"]
    if perturbed:
        E = rng.standard_normal((m, m))
        case["A_filter"] = case["A"] + 1e-3 * (E + E.T) / np.linalg.norm(E + E.T, 2)
    X = rng.standard_normal((m, N))
    L = np.sort(rng.uniform(-1.0, 2.0, N))
    # filter bounds that bracket the spectrum of the filter operator D^-1 A~ (so the Chebyshev
    # polynomial is bounded on it): lmin below, lmax above, lT at the 30% point
    F = case["A_filter"] if case["A_filter"] is not None else case["A"]
    if case["Dinv"] is not None:
        H = case["Dinv"][:, None] * F
    elif case["Dinv_dense"] is not None:
        H = case["Dinv_dense"] @ F
    else:
        H = F
    ev = np.sort(np.real(np.linalg.eigvals(H)))
    span = ev[-1] - ev[0]
    case["bounds"] = (ev[0] - 0.05 * span, ev[0] + 0.3 * span, ev[-1] + 0.02 * span)
    L = np.sort(rng.uniform(ev[0], ev[0] + 0.3 * span, N))
    Bm = case["B"] if case["B"] is not None else np.eye(m)
    W = case["A"] @ X - (Bm @ X) * L[None, :]
    case.update(X=X, L=L, W=W)
    return case


def oracle_ops(case):
    F = case["A_filter"] if case["A_filter"] is not None else case["A"]
    if case["Dinv"] is not None:
        d = case["Dinv"]
        Dinv = lambda R: d[:, None] * R  # noqa: E731
    elif case["Dinv_dense"] is not None:
        Dd = case["Dinv_dense"]
        Dinv = lambda R: Dd @ R  # noqa: E731
    else:
        Dinv = lambda R: R  # noqa: E731
    AD = lambda R: F @ Dinv(R)  # noqa: E731
    H = lambda Y: Dinv(F @ Y)  # noqa: E731
    return AD, Dinv, H


def make_solver(case, N, precision="fp64", method="rchfsi", **kw):
    m = case["A"].shape[0]
    s = Solver(m, nev=max(1, N // 2), block=N, precision=precision, method=method, **kw)
    s.set_dense(case["A"], B=case["B"], Dinv=case["Dinv"], Dinv_dense=case["Dinv_dense"],
                A_filter=case["A_filter"])
    return s


def round_mantissa(x, bits, mode="nearest"):
    """Round float64 values to `bits` explicit mantissa bits (bits = 23 is FP32 precision,
    10 TF32, 7 BF16); mode "truncate" drops the low bits (round toward zero)."""
    m, e = np.frexp(x)
    scale = 2.0 ** (bits + 1)
    if mode == "truncate":
        q = np.trunc(m * scale)
    else:
        q = np.round(m * scale)
    return np.ldexp(q / scale, e)


def lowp_reference(case, p, bits_op, bits_r, r_mode, lmin, lT, lmax):
    """Oracle Algorithm 3 whose product consumes the operator rounded to `bits_op` mantissa bits and
    R_Y rounded to `bits_r` bits (the inputs the tensor cores / FP32 units see)."""
    _, Dinv, _ = oracle_ops(case)
    d = case["Dinv"]
    F = case["A"] if case["A_filter"] is None else case["A_filter"]
    Ad = F * d[None, :] if d is not None else F
    Ar = round_mantissa(Ad, bits_op)
    ADr = lambda R: Ar @ round_mantissa(round_mantissa(R, 23), bits_r, r_mode)  # noqa: E731
    return filters.rchfsi_filter(ADr, Dinv, case["X"], case["L"], case["W"], lmin, lT, lmax, p)
