"""The request loop (rchfsi_server_create / rchfsi_submit / rchfsi_poll): requests admitted while
others run give the same result as alone, warm starts keep the subspace on the device, and the HBM
budget admits requests in arrival order."""
import time

import numpy as np
import pytest

import workloads as wl
from gpu_helpers import ensure_built

from paper_2503_22652_gb300 import Server, Solver, RChFSIError

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    ensure_built()


def _problem(m, seed, shift=0.0):
    lam = np.linspace(-1.0, 10.0, m) + shift
    lam[20:] += 0.3
    A = wl.dense_from_spectrum(wl.orthogonal(m, seed), lam)
    return A, lam


def _wait(srv, tickets, timeout=120.0, want_vectors=False):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t, want_vectors=want_vectors)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout, "requests did not finish"
        time.sleep(0.01)
    return out


def test_mix_equals_alone():
    specs = [(300, 11, "tf32"), (400, 12, "fp64"), (256, 13, "bf16"), (350, 14, "fp32"), (300, 15, "tf32")]
    srv = Server(slots=3)
    tickets = []
    for m, seed, prec in specs:
        A, _ = _problem(m, seed)
        X0 = wl.gaussian_block(m, 24, seed=seed)
        tickets.append(srv.submit(m, 20, 24, X0=X0, dense={"A": A}, precision=prec, degree=12, max_iter=80,
                                  tol=1e-9))
    res = _wait(srv, tickets)
    for t, (m, seed, prec) in zip(tickets, specs):
        r = res[t]
        assert r["status"] == 0, r
        A, lam = _problem(m, seed)
        s = Solver(m, nev=20, block=24, degree=12, precision=prec, max_iter=80, tol=1e-9)
        s.set_dense(A)
        _, ev, _, st = s.solve(wl.gaussian_block(m, 24, seed=seed))
        np.testing.assert_allclose(r["evals"][:20], ev[:20], rtol=0, atol=1e-10 * 11)
        np.testing.assert_allclose(r["evals"][:20], lam[:20], rtol=0, atol=1e-9 * 11)
        assert r["latency_ms"] >= r["queue_ms"] >= 0.0
    srv.close()


def test_warm_start_reuses_subspace():
    m = 400
    A, _ = _problem(m, 21)
    srv = Server(slots=1)
    X0 = wl.gaussian_block(m, 24, seed=3)
    t1 = srv.submit(m, 20, 24, X0=X0, dense={"A": A}, precision="tf32", degree=12, tol=1e-9, warm_key=7)
    r1 = _wait(srv, [t1])[t1]
    # a 1e-4 perturbation of the operator, started from the kept subspace (no X0)
    E = np.random.default_rng(5).standard_normal((m, m))
    A2 = A + 1e-4 * (E + E.T) / np.linalg.norm(E + E.T, 2)
    t2 = srv.submit(m, 20, 24, X0=None, dense={"A": A2}, precision="tf32", degree=12, tol=1e-9, warm_key=7)
    r2 = _wait(srv, [t2])[t2]
    assert r1["status"] == 0 and r2["status"] == 0
    assert r2["iterations"] < r1["iterations"]
    ref = np.linalg.eigvalsh(A2)[:20]
    np.testing.assert_allclose(r2["evals"][:20], ref, rtol=0, atol=1e-9 * 11)
    srv.close()


def test_budget_admission_and_errors():
    m = 300
    A, lam = _problem(m, 31)
    # a budget below one request's footprint still runs requests, one at a time
    srv = Server(slots=4, hbm_budget_bytes=1)
    ts = [srv.submit(m, 10, 16, X0=wl.gaussian_block(m, 16, seed=k), dense={"A": A}, precision="tf32",
                     degree=10, tol=1e-9) for k in range(3)]
    res = _wait(srv, ts)
    for t in ts:
        assert res[t]["status"] == 0
        np.testing.assert_allclose(res[t]["evals"][:10], lam[:10], rtol=0, atol=1e-9 * 11)
    # requests queue behind one another: the last one waited for the earlier ones
    assert res[ts[-1]]["queue_ms"] > 0.0
    # a request without X0 and without a warm start fails cleanly
    t = srv.submit(m, 10, 16, X0=None, dense={"A": A}, precision="tf32", degree=10)
    r = _wait(srv, [t])[t]
    assert r["status"] == -1
    with pytest.raises(KeyError):
        srv.poll(123456)
    srv.close()


def test_concurrent_fe_requests_of_different_widths():
    """FE requests whose tensor-core launches use different tile widths (shared-memory plans) run
    concurrently in several slots: every one succeeds and equals its solve alone."""
    probs = [(wl.fe_problem(3), 6, 10, "tf32"), (wl.fe_problem(3, seed_wells=9), 20, 48, "bf16"),
             (wl.fe_problem(2), 8, 16, "tf32"), (wl.fe_problem(3, seed_wells=10), 30, 96, "tf32")]
    srv = Server(slots=4)
    tickets = []
    for p, nev, blk, prec in probs:
        fe = dict(cell_dofs=p["cell_dofs"], A_cells=p["A_cells"], B_cells=p["B_cell"], Dinv=p["Dinv"])
        tickets.append(srv.submit(p["m"], nev, blk, X0=wl.gaussian_block(p["m"], blk, seed=blk), fe=fe,
                                  precision=prec, degree=20, max_iter=150))
    res = _wait(srv, tickets)
    srv.close()
    for t, (p, nev, blk, prec) in zip(tickets, probs):
        r = res[t]
        assert r["status"] == 0, r["error"]
        s = Solver(p["m"], nev=nev, block=blk, degree=20, precision=prec, max_iter=150)
        s.set_fe(p["cell_dofs"], p["A_cells"], p["B_cell"], p["Dinv"])
        _, ev, _, st = s.solve(wl.gaussian_block(p["m"], blk, seed=blk))
        np.testing.assert_allclose(r["evals"][:nev], ev[:nev], rtol=0, atol=1e-9 * np.abs(ev[:nev]).max())
