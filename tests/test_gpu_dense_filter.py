"""Parity of the CUDA dense filters (Algorithms 2 and 3) with the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import filters
from gpu_helpers import ensure_built, dense_case, oracle_ops, make_solver, relfro, lowp_reference

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12   # relative Frobenius error of the FP64 filter


@pytest.fixture(scope="module", autouse=True)
def _build():
    ensure_built()


CASES = [
    dict(m=200, N=24),                        # standard problem, ragged tiles
    dict(m=333, N=40, generalized=True),      # dense B, diagonal D^-1
    dict(m=256, N=17, dense_dinv=True),       # dense approximate inverse (Section 4.1 toy form)
    dict(m=150, N=9, perturbed=True),         # perturbed filter matrix
]


@pytest.mark.parametrize("cfg", CASES, ids=lambda c: "-".join("%s%s" % kv for kv in c.items()))
@pytest.mark.parametrize("p", [1, 2, 7, 20])
def test_rchfsi_filter_fp64_parity(cfg, p):
    case = dense_case(**cfg)
    AD, Dinv, _ = oracle_ops(case)
    lmin, lT, lmax = case["bounds"]
    ref = filters.rchfsi_filter(AD, Dinv, case["X"], case["L"], case["W"], lmin, lT, lmax, p)
    s = make_solver(case, cfg["N"])
    got = s.filter(case["X"], case["L"], case["W"], lmin, lT, lmax, p)
    assert relfro(got, ref) <= FP64_TOL


@pytest.mark.parametrize("cfg", CASES[:3], ids=["std", "gen", "densedinv"])
def test_chfsi_filter_fp64_parity(cfg):
    case = dense_case(**cfg)
    _, _, H = oracle_ops(case)
    ref = filters.chfsi_filter(H, case["X"], *case["bounds"], 12)
    s = make_solver(case, cfg["N"])
    got = s.chfsi_filter(case["X"], *case["bounds"], 12)
    assert relfro(got, ref) <= FP64_TOL


# Tolerances for the reduced-precision filters, relative to ||Y_p - X Lambda_p|| (the part of Y_p
# that the low-precision recurrence produces).  The oracle sees the same rounded operator and the
# same rounding of R_Y as the GPU; what remains is FP32 accumulation (u = 6e-8 times sqrt(K)
# growth, K <= 333) and the FP32 storage of R between steps, amplified over p steps, plus the
# occasional different rounding of an R_Y entry that sits on a rounding boundary.
LOWP = {"fp32": (23, 23, "nearest", 2e-5), "tf32": (10, 10, "truncate", 2e-3), "bf16": (7, 7, "nearest", 2e-2)}


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
@pytest.mark.parametrize("cfg", [dict(m=512, N=64, generalized=True), dict(m=333, N=40), dict(m=200, N=24)],
                         ids=["gen512x64", "std333x40", "std200x24"])
def test_rchfsi_filter_lowp_parity(prec, cfg):
    case = dense_case(**cfg)
    bits_op, bits_r, mode, tol = LOWP[prec]
    (lmin, lT, lmax), p = case["bounds"], 10
    ref = lowp_reference(case, p, bits_op, bits_r, mode, lmin, lT, lmax)
    s = make_solver(case, cfg["N"], precision=prec)
    got = s.filter(case["X"], case["L"], case["W"], lmin, lT, lmax, p)
    from oracle.filters import lambda_p
    base = case["X"] * lambda_p(case["L"], lmin, lT, lmax, p)[None, :]
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref - base)
    assert err <= tol, err


def test_filter_accepts_device_pointers():
    torch = pytest.importorskip("torch")
    case = dense_case(m=200, N=24)
    AD, Dinv, _ = oracle_ops(case)
    ref = filters.rchfsi_filter(AD, Dinv, case["X"], case["L"], case["W"], *case["bounds"], 6)
    s = make_solver(case, 24)
    dev = lambda a: torch.from_numpy(a).cuda()  # noqa: E731
    got = s.filter(dev(case["X"]), dev(case["L"]), dev(case["W"]), *case["bounds"], 6)
    assert got.is_cuda
    assert relfro(got.cpu().numpy(), ref) <= FP64_TOL


def test_filter_rejects_bad_bounds():
    from paper_2503_22652_gb300 import RChFSIError
    case = dense_case(m=64, N=4)
    s = make_solver(case, 4)
    with pytest.raises(RChFSIError) as e:
        s.filter(case["X"], case["L"], case["W"], 5.0, 3.0, 9.5, 4)
    assert e.value.code == -1
    with pytest.raises(RChFSIError):
        s.filter(case["X"], case["L"], case["W"], -1.0, 3.0, 2.0, 4)
