"""rchfsi_filter_step_tf32_static: the allocation-free TF32 filter step.

Some callers cannot let a library allocate device memory (a serving loop that must not call
cudaMalloc after start-up, an application whose memory belongs to its own pool allocator).  For them
the library has one entry point whose scratch lives in a fixed, file-scope device array.  This test
calls it through the C ABI, twice in a row, and checks its results against the regular entry point
(rchfsi_filter in TF32), which runs the same recurrence with its own cudaMalloc'd scratch.

The file is named to be collected last, so a run that stops at the first failure has already run
every other test; it also passes when run alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as wl
from oracle.chebyshev import affine, recurrence_coefficients
from oracle.filters import lambda_p
from gpu_helpers import ensure_built

pytestmark = pytest.mark.gpu

# Same tolerance as the TF32 filter parity tests: error relative to ||Y_p - X Lambda_p||.
TF32_TOL = 2e-3


def _tf32_rna(t):
    """Round FP32 values to TF32 (10 explicit mantissa bits), nearest, ties away from zero -- the
    rounding the library applies to its TF32 copy of the operator."""
    import torch
    b = t.contiguous().view(torch.int32)
    b = (b + 0x1000) & ~0x1FFF
    return b.view(torch.float32)


def _scalars(lmin, lT, lmax, p):
    """e, c, sigma_1 and the (a_k, b_k, c_k) of the degree loop, from the oracle's definitions."""
    e, cc, s1 = affine(lmin, lT, lmax)
    return e, cc, s1, recurrence_coefficients(lmin, lT, lmax, p)


def _lambda_rows(lam, e, cc, s1, co):
    """Lambda_d = C_d(Lambda) for d = 0..p, same recurrence as the library's host table."""
    rows = [np.ones_like(lam), (s1 / e) * (lam - cc)]
    for (a, b, c) in co:
        lx, ly = rows[-2], rows[-1]
        rows.append(a * ly * lam - a * cc * ly + c * lx)
    return rows


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    ensure_built()
    from paper_2503_22652_gb300 import _lib, Solver
    lib = _lib.load()
    m, N = 1000, 120
    c = wl.dense_config2(m=m)
    rng = np.random.default_rng(7)
    X = rng.standard_normal((m, N))
    L = np.sort(rng.uniform(-1.0, 0.5, N))
    W = c["A"] @ X - (c["B"] @ X) * L[None, :]
    d = c["Dinv"]
    ev = np.sort(np.real(np.linalg.eigvals(d[:, None] * c["A"])))
    span = ev[-1] - ev[0]
    bounds = (ev[0] - 0.05 * span, ev[0] + 0.3 * span, ev[-1] + 0.02 * span)
    solver = Solver(m, nev=N // 2, block=N, precision="tf32")
    solver.set_dense(c["A"], B=c["B"], Dinv=d)
    return dict(torch=torch, lib=lib, _lib=_lib, solver=solver, m=m, N=N, c=c, X=X, L=L, W=W, d=d,
                bounds=bounds)


def _step(S, Ad, Ry, Rx, Wc, lam_row, a, b, c, out):
    torch, lib = S["torch"], S["lib"]
    m, N = S["m"], S["N"]
    lam = torch.from_numpy(np.ascontiguousarray(lam_row)).cuda()
    rc = lib.rchfsi_filter_step_tf32_static(Ad.data_ptr(), m, Ry.data_ptr(), None if Rx is None else Rx.data_ptr(),
                                            Wc.data_ptr(), lam.data_ptr(), a, b, c, m, N, m, out.data_ptr(),
                                            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        buf = C.create_string_buffer(512)
        lib.rchfsi_last_error(None, buf, 512)
        raise AssertionError("rc=%d: %s" % (rc, buf.value.decode()))
    return out


def test_static_scratch_step_matches_filter_two_calls(setup):
    S = setup
    torch = S["torch"]
    m, N, X, L, W, d = S["m"], S["N"], S["X"], S["L"], S["W"], S["d"]
    lmin, lT, lmax = S["bounds"]
    e, cc, s1, co = _scalars(lmin, lT, lmax, 3)
    rows = _lambda_rows(L, e, cc, s1, co)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    # inputs as the regular path forms them: A D^-1 rounded to TF32, R_Y = (sigma_1/e) W, W in FP32,
    # column-major blocks (leading dimension m)
    Ad = _tf32_rna((dev(S["c"]["A"]) * dev(d)[None, :]).float())
    Wt = dev(W).t().contiguous()                       # N x m row-major = column-major m x N
    Ry0 = (Wt * (s1 / e)).float().contiguous()
    Wc = Wt.float().contiguous()
    out1 = torch.empty_like(Ry0)
    out2 = torch.empty_like(Ry0)
    # call 1: degree-2 step (R_X = 0), call 2: degree-3 step
    _step(S, Ad, Ry0, None, Wc, rows[1], co[0][0], co[0][1], co[0][2], out1)
    _step(S, Ad, out1, Ry0, Wc, rows[2], co[1][0], co[1][1], co[1][2], out2)
    torch.cuda.synchronize()
    for deg, R in ((2, out1), (3, out2)):
        Rn = R.double().t().cpu().numpy()               # back to row-major m x N
        got = d[:, None] * Rn + X * rows[deg][None, :]
        ref = S["solver"].filter(X, L, W, lmin, lT, lmax, deg)
        base = X * lambda_p(L, lmin, lT, lmax, deg)[None, :]
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref - base)
        assert err <= TF32_TOL, (deg, err)


def _last_error(lib):
    buf = C.create_string_buffer(512)
    lib.rchfsi_last_error(None, buf, 512)
    return buf.value


def test_static_scratch_rejects_oversized_problem(setup):
    S = setup
    torch, lib = S["torch"], S["lib"]
    # 65 row tiles of 128 and one 256-wide column tile: on any GPU with >= 130 SMs the product is
    # split over K at least twice, and two splits of 8200 x 256 partials already exceed the array
    m, N = 8200, 256
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    if sms // ((m + 127) // 128) < 2:
        pytest.skip("this GPU would not split the product over K")
    assert 2 * m * N > S["_lib"].STATIC_SCRATCH_FLOATS
    A = torch.zeros(m, m, dtype=torch.float32, device="cuda")
    R = torch.zeros(N, m, dtype=torch.float32, device="cuda")
    out = torch.zeros(N, m, dtype=torch.float32, device="cuda")
    lam = torch.zeros(N, dtype=torch.float64, device="cuda")
    rc = lib.rchfsi_filter_step_tf32_static(A.data_ptr(), m, R.data_ptr(), None, None, lam.data_ptr(), 1.0, 0.0,
                                            0.0, m, N, m, out.data_ptr(), None)
    assert rc == S["_lib"].ERR_INVALID_ARG
    assert b"static limit" in _last_error(lib)


def test_static_scratch_rejects_partial_overlap(setup):
    """out may be Rx itself, but an out that overlaps part of Ry, W or Rx is refused before any
    kernel runs."""
    S = setup
    torch, lib = S["torch"], S["lib"]
    m, N = 256, 32
    A = torch.zeros(m, m, dtype=torch.float32, device="cuda")
    big = torch.zeros(4 * N * m, dtype=torch.float32, device="cuda")
    Ry, W, Rx = big[:N * m], big[N * m:2 * N * m], big[2 * N * m:3 * N * m]
    lam = torch.zeros(N, dtype=torch.float64, device="cuda")

    def call(out_ptr, rx_ptr):
        return lib.rchfsi_filter_step_tf32_static(A.data_ptr(), m, Ry.data_ptr(), rx_ptr, W.data_ptr(),
                                                  lam.data_ptr(), 1.0, 0.0, 0.0, m, N, m, out_ptr, None)

    shifted = big.data_ptr() + 4 * 4   # 4 floats into Ry: overlaps Ry
    assert call(shifted, None) == S["_lib"].ERR_INVALID_ARG
    assert b"overlap" in _last_error(lib)
    assert call(W.data_ptr() + 64, None) == S["_lib"].ERR_INVALID_ARG   # overlaps W
    assert call(Rx.data_ptr() + 16, Rx.data_ptr()) == S["_lib"].ERR_INVALID_ARG   # part of Rx
    assert call(Rx.data_ptr(), Rx.data_ptr()) == S["_lib"].OK   # out is Rx itself: allowed
    torch.cuda.synchronize()
