"""GB300 (sm_103a) R-ChFSI eigensolver: Python binding of the C ABI in include/rchfsi.h.

The binding only marshals arguments: NumPy arrays (host memory) and torch tensors (host or CUDA
memory) are passed to the library as raw pointers; every step of the method runs in
librchfsi.so.  Blocks are (m, N) float64 arrays in row-major (C) order; for complex Hermitian
problems (field="complex") blocks, A and the FE cell matrices A_c are complex128 (interleaved
real/imaginary parts) while B, B_c and D^-1 stay real.

    from paper_2503_22652_gb300 import Solver
    s = Solver(m, nev=50, block=60, degree=20, precision="tf32")
    s.set_dense(A, B=None, Dinv=None)
    X, evals, resid, stats = s.solve(X0)
"""
import ctypes as C

import numpy as np

from . import _lib
from ._lib import (rchfsi_params, rchfsi_operator, rchfsi_stats, rchfsi_request, rchfsi_result,  # noqa: F401
                   PRECISIONS, METHOD_RCHFSI, METHOD_CHFSI, OK, PENDING)

__all__ = ["Solver", "Server", "RChFSIError", "load_library", "ptr", "solve_batch"]


class RChFSIError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_lib.load().rchfsi_strerror(code).decode(), code, msg))
        self.code = code


def load_library():
    return _lib.load()


def ptr(a):
    """Raw address of a NumPy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    raise TypeError("expected a numpy array or torch tensor, got %r" % type(a))


def _check_arr(a, shape, name, dtype=np.float64):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags.c_contiguous:
            a = np.ascontiguousarray(a, dtype=dtype)
        if tuple(a.shape) != tuple(shape) and a.size != int(np.prod(shape)):
            raise ValueError("%s: expected shape %s, got %s" % (name, shape, a.shape))
        return a
    # torch tensor
    if not a.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if a.is_complex() != (dtype == np.complex128) or a.element_size() != np.dtype(dtype).itemsize:
        raise ValueError("%s: expected a %s tensor" % (name, np.dtype(dtype).name))
    if a.numel() != int(np.prod(shape)):
        raise ValueError("%s: expected %s elements" % (name, int(np.prod(shape))))
    if a.is_cuda:
        # the library reads device inputs on its own stream: torch's pending writes to this tensor
        # (a clone, a copy from the host) must have landed first
        import torch
        torch.cuda.current_stream(a.device).synchronize()
    return a


def _is_cuda(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def _empty_like_kind(ref, shape, dtype=np.float64):
    if _is_cuda(ref):
        import torch
        tdt = torch.complex128 if dtype == np.complex128 else torch.float64
        return torch.empty(shape, dtype=tdt, device=ref.device)
    return np.empty(shape, dtype=dtype)


class Solver:
    """One rchfsi handle (rchfsi_create / rchfsi_destroy)."""

    def __init__(self, m, nev, block, degree=20, precision="fp64", method="rchfsi", max_iter=100,
                 min_iter=0, tol=1e-8, lanczos_steps=10, stall_iters=0, bounds=None,
                 hbm_budget_bytes=0, stream=None, rr_mode=None, eig_mode=None, field="real"):
        self.lib = _lib.load()
        p = rchfsi_params()
        self.lib.rchfsi_params_default(C.byref(p))
        if rr_mode is not None:
            p.rr_mode = _lib.RR_MODES[rr_mode] if isinstance(rr_mode, str) else int(rr_mode)
        if eig_mode is not None:
            p.eig_mode = _lib.EIG_MODES[eig_mode] if isinstance(eig_mode, str) else int(eig_mode)
        p.m, p.nev, p.block, p.degree = int(m), int(nev), int(block), int(degree)
        p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        p.method = METHOD_CHFSI if method == "chfsi" else METHOD_RCHFSI
        p.max_iter, p.min_iter, p.tol = int(max_iter), int(min_iter), float(tol)
        p.lanczos_steps, p.stall_iters = int(lanczos_steps), int(stall_iters)
        if bounds is not None:
            p.fixed_bounds = 1
            p.lmin, p.lT, p.lmax = (float(b) for b in bounds)
        p.hbm_budget_bytes = int(hbm_budget_bytes)
        self.complex = field == "complex"
        p.field = _lib.COMPLEX if self.complex else _lib.REAL
        self.dt = np.complex128 if self.complex else np.float64  # dtype of blocks and of A / A_c
        self.params = p
        self.m, self.N = int(m), int(block)
        h = C.c_void_p()
        self._check(self.lib.rchfsi_create(C.byref(h), C.byref(p), stream), None)
        self.h = h
        self._keep = []

    def _check(self, rc, h, allow=()):
        if rc != OK and rc not in allow:
            buf = C.create_string_buffer(1024)
            self.lib.rchfsi_last_error(h, buf, 1024)
            raise RChFSIError(rc, buf.value.decode(errors="replace"))
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.rchfsi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, **kw):
        p = self.params
        for k, v in kw.items():
            if k == "precision" and isinstance(v, str):
                v = PRECISIONS[v]
            if k == "method":
                v = METHOD_CHFSI if v == "chfsi" else METHOD_RCHFSI
            if k == "rr_mode" and isinstance(v, str):
                v = _lib.RR_MODES[v]
            if k == "eig_mode" and isinstance(v, str):
                v = _lib.EIG_MODES[v]
            if k == "bounds":
                p.fixed_bounds = 0 if v is None else 1
                if v is not None:
                    p.lmin, p.lT, p.lmax = (float(b) for b in v)
                continue
            setattr(p, k, v)
        self._check(self.lib.rchfsi_set_params(self.h, C.byref(p)), self.h)

    # ------------------------------------------------------------ operators
    def set_dense(self, A, B=None, Dinv=None, Dinv_dense=None, A_filter=None):
        m = self.m
        A = _check_arr(A, (m, m), "A", self.dt)
        B = _check_arr(B, (m, m), "B")
        Dinv = _check_arr(Dinv, (m,), "Dinv")
        Dinv_dense = _check_arr(Dinv_dense, (m, m), "Dinv_dense")
        A_filter = _check_arr(A_filter, (m, m), "A_filter")
        op = rchfsi_operator()
        op.kind, op.field, op.m = _lib.OP_DENSE, self.params.field, m
        op.A, op.B, op.Dinv, op.Dinv_dense, op.A_filter = (ptr(A), ptr(B), ptr(Dinv), ptr(Dinv_dense),
                                                           ptr(A_filter))
        self._check(self.lib.rchfsi_set_operator(self.h, C.byref(op)), self.h)

    def set_fe(self, cell_dofs, A_cells, B_cells, Dinv):
        cell_dofs = np.ascontiguousarray(cell_dofs, dtype=np.int32) if isinstance(cell_dofs, np.ndarray) \
            else cell_dofs
        nC, nc = cell_dofs.shape
        shared = tuple(B_cells.shape) == (nc, nc)
        A_cells = _check_arr(A_cells, (nC, nc, nc), "A_cells", self.dt)
        B_cells = _check_arr(B_cells, (nc, nc) if shared else (nC, nc, nc), "B_cells")
        Dinv = _check_arr(Dinv, (self.m,), "Dinv")
        op = rchfsi_operator()
        op.kind, op.field, op.m = _lib.OP_FE_CELL, self.params.field, self.m
        op.n_cells, op.n_c, op.B_cells_shared = nC, nc, 1 if shared else 0
        op.cell_dofs, op.A_cells, op.B_cells, op.Dinv = ptr(cell_dofs), ptr(A_cells), ptr(B_cells), ptr(Dinv)
        self._check(self.lib.rchfsi_set_operator(self.h, C.byref(op)), self.h)

    # ------------------------------------------------------------ the method
    def filter(self, X, lam, W, lmin, lT, lmax, degree, out=None):
        """Algorithm 3 (rchfsi_filter)."""
        X = _check_arr(X, (self.m, self.N), "X", self.dt)
        W = _check_arr(W, (self.m, self.N), "W", self.dt)
        lam = _check_arr(lam, (self.N,), "Lambda")
        if out is None:
            out = _empty_like_kind(X, (self.m, self.N), self.dt)
        self._check(self.lib.rchfsi_filter(self.h, ptr(X), ptr(lam), ptr(W), lmin, lT, lmax, int(degree),
                                           ptr(out)), self.h)
        return out

    def chfsi_filter(self, X, lmin, lT, lmax, degree, out=None):
        """Algorithm 2 (rchfsi_chfsi_filter)."""
        X = _check_arr(X, (self.m, self.N), "X", self.dt)
        if out is None:
            out = _empty_like_kind(X, (self.m, self.N), self.dt)
        self._check(self.lib.rchfsi_chfsi_filter(self.h, ptr(X), lmin, lT, lmax, int(degree), ptr(out)),
                    self.h)
        return out

    def residual(self, X, lam):
        X = _check_arr(X, (self.m, self.N), "X", self.dt)
        lam = _check_arr(lam, (self.N,), "Lambda")
        W = _empty_like_kind(X, (self.m, self.N), self.dt)
        r = np.empty(self.N)
        self._check(self.lib.rchfsi_residual(self.h, ptr(X), ptr(lam), ptr(W), ptr(r)), self.h)
        return W, r

    def rayleigh_ritz(self, Y):
        Y = _check_arr(Y, (self.m, self.N), "Y", self.dt)
        X = _empty_like_kind(Y, (self.m, self.N), self.dt)
        ev = np.empty(self.N)
        self._check(self.lib.rchfsi_rayleigh_ritz(self.h, ptr(Y), ptr(X), ptr(ev)), self.h)
        return X, ev

    def lanczos_bounds(self, v0, steps=10):
        v0 = _check_arr(v0, (self.m,), "v0", self.dt)
        lmax, nA = C.c_double(), C.c_double()
        self._check(self.lib.rchfsi_lanczos_bounds(self.h, ptr(v0), int(steps), C.byref(lmax), C.byref(nA)),
                    self.h)
        return lmax.value, nA.value

    def solve(self, X0, allow_not_converged=False, inplace=False):
        """Algorithm 1 (rchfsi_solve).  Returns (X, evals, rel_resid, stats_dict).  With inplace=True
        X0 itself (C-contiguous float64 host array, e.g. pinned memory, or a CUDA tensor) is the
        rchfsi_solve in/out block and receives the Ritz vectors; otherwise a copy is."""
        if inplace:
            if isinstance(X0, np.ndarray) and (X0.dtype != self.dt or not X0.flags.c_contiguous
                                               or not X0.flags.writeable):
                raise ValueError("inplace solve needs a writable C-contiguous %s array" % np.dtype(self.dt).name)
            X = X0
        else:
            X = X0.copy() if isinstance(X0, np.ndarray) else X0.clone()
        X = _check_arr(X, (self.m, self.N), "X0", self.dt)
        ev = np.empty(self.N)
        res = np.empty(self.N)
        hist = np.full(self.params.max_iter + 1, np.nan)
        st = rchfsi_stats()
        st.history = hist.ctypes.data
        allow = (_lib.ERR_NOT_CONVERGED, _lib.ERR_STAGNATED) if allow_not_converged else ()
        rc = self._check(self.lib.rchfsi_solve(self.h, ptr(X), ptr(ev), ptr(res), C.byref(st)), self.h, allow)
        stats = {k: getattr(st, k) for k, _ in rchfsi_stats._fields_ if k != "history"}
        stats["status"] = rc
        stats["history"] = hist[: st.iterations + 1].copy()
        return X, ev, res, stats


def solve_batch(solvers, X0s, allow_not_converged=False):
    """rchfsi_solve_batch: solve several problems together (one Solver each, distinct handles).
    Returns a list of (X, evals, rel_resid, stats_dict) as Solver.solve does."""
    lib = _lib.load()
    n = len(solvers)
    Xs, evs, ress, hists = [], [], [], []
    sts = (rchfsi_stats * n)()
    for i, (s, X0) in enumerate(zip(solvers, X0s)):
        X = X0.copy() if isinstance(X0, np.ndarray) else X0.clone()
        X = _check_arr(X, (s.m, s.N), "X0", s.dt)
        Xs.append(X)
        evs.append(np.empty(s.N))
        ress.append(np.empty(s.N))
        hists.append(np.full(s.params.max_iter + 1, np.nan))
        sts[i].history = hists[-1].ctypes.data
    hs = (C.c_void_p * n)(*[s.h for s in solvers])
    xp = (C.c_void_p * n)(*[ptr(X) for X in Xs])
    ep = (C.c_void_p * n)(*[e.ctypes.data for e in evs])
    rp = (C.c_void_p * n)(*[r.ctypes.data for r in ress])
    rc = lib.rchfsi_solve_batch(hs, n, xp, ep, rp, sts)
    allow = (OK, _lib.ERR_NOT_CONVERGED, _lib.ERR_STAGNATED) if allow_not_converged else (OK,)
    if rc not in allow:
        bad = next((i for i in range(n) if sts[i].status != OK), 0)
        buf = C.create_string_buffer(1024)
        lib.rchfsi_last_error(solvers[bad].h, buf, 1024)
        raise RChFSIError(rc, buf.value.decode(errors="replace"))
    out = []
    for i in range(n):
        st = {k: getattr(sts[i], k) for k, _ in rchfsi_stats._fields_ if k != "history"}
        st["history"] = hists[i][: sts[i].iterations + 1].copy()
        out.append((Xs[i], evs[i], ress[i], st))
    return out


class Server:
    """Request loop (rchfsi_server_create / rchfsi_submit / rchfsi_poll)."""

    def __init__(self, slots=2, hbm_budget_bytes=0):
        self.lib = _lib.load()
        h = C.c_void_p()
        rc = self.lib.rchfsi_server_create(C.byref(h), int(slots), int(hbm_budget_bytes))
        if rc != OK:
            raise RChFSIError(rc, "server_create")
        self.h = h
        self._pending = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.rchfsi_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, m, nev, block, X0=None, warm_key=0, dense=None, fe=None, **params):
        """dense = dict(A=, B=, Dinv=) or fe = dict(cell_dofs=, A_cells=, B_cells=, Dinv=).
        Array arguments are copied by the library before this returns."""
        lib = self.lib
        rq = rchfsi_request()
        p = rq.params
        lib.rchfsi_params_default(C.byref(p))
        p.m, p.nev, p.block = int(m), int(nev), int(block)
        cplx = params.pop("field", "real") == "complex"
        dt = np.complex128 if cplx else np.float64
        p.field = _lib.COMPLEX if cplx else _lib.REAL
        for k, v in params.items():
            if k == "precision" and isinstance(v, str):
                v = PRECISIONS[v]
            setattr(p, k, v)
        keep = []
        op = rq.op
        op.m, op.field = int(m), p.field
        if dense is not None:
            op.kind = _lib.OP_DENSE
            for k in ("A", "B", "Dinv"):
                a = dense.get(k)
                if a is not None:
                    a = np.ascontiguousarray(a, dtype=dt if k == "A" else np.float64)
                    keep.append(a)
                    setattr(op, k, a.ctypes.data)
        else:
            op.kind = _lib.OP_FE_CELL
            dofs = np.ascontiguousarray(fe["cell_dofs"], dtype=np.int32)
            Ac = np.ascontiguousarray(fe["A_cells"], dtype=dt)
            Bc = np.ascontiguousarray(fe["B_cells"], dtype=np.float64)
            Dv = np.ascontiguousarray(fe["Dinv"], dtype=np.float64)
            keep += [dofs, Ac, Bc, Dv]
            op.n_cells, op.n_c = dofs.shape
            op.B_cells_shared = 1 if Bc.ndim == 2 else 0
            op.cell_dofs, op.A_cells, op.B_cells, op.Dinv = (dofs.ctypes.data, Ac.ctypes.data, Bc.ctypes.data,
                                                             Dv.ctypes.data)
        if X0 is not None:
            X0 = np.ascontiguousarray(X0, dtype=dt)
            keep.append(X0)
            rq.X0 = X0.ctypes.data
        rq.warm_key = int(warm_key)
        t = C.c_uint64()
        rc = lib.rchfsi_submit(self.h, C.byref(rq), C.byref(t))
        if rc != OK:
            raise RChFSIError(rc, "submit")
        self._pending[t.value] = (int(m), int(block), dt)
        return t.value

    def poll(self, ticket, want_vectors=False):
        """None while pending, else dict(status, iterations, max_rel_residual, latency_ms,
        queue_ms, evals[, X])."""
        m, N, dt = self._pending[ticket]
        res = rchfsi_result()
        ev = np.empty(N)
        res.evals = ev.ctypes.data
        X = np.empty((m, N), dtype=dt) if want_vectors else None
        if X is not None:
            res.X = X.ctypes.data
        rc = self.lib.rchfsi_poll(self.h, int(ticket), C.byref(res))
        if rc == PENDING:
            return None
        if rc != OK:
            raise RChFSIError(rc, "poll")
        del self._pending[ticket]
        out = {"status": res.status, "iterations": res.iterations, "max_rel_residual": res.max_rel_residual,
               "latency_ms": res.latency_ms, "queue_ms": res.queue_ms, "evals": ev,
               "error": res.error.decode(errors="replace")}
        if X is not None:
            out["X"] = X
        return out


def _solver_profile(self, enable=True):
    """rchfsi_profile: start (True) or stop (False) the per-kernel-class device timers."""
    self._check(self.lib.rchfsi_profile(self.h, 1 if enable else 0), self.h)


def _solver_profile_read(self, cls):
    """rchfsi_profile_read: dict(ms, launches, flops, bytes) of one kernel class ("all" = launch count)."""
    idx = len(_lib.KERNEL_CLASSES) if cls == "all" else _lib.KERNEL_CLASSES[cls]
    ms, fl, by = C.c_double(), C.c_double(), C.c_double()
    n = C.c_int64()
    self._check(self.lib.rchfsi_profile_read(self.h, idx, C.byref(ms), C.byref(n), C.byref(fl), C.byref(by)),
                self.h)
    return {"ms": ms.value, "launches": n.value, "flops": fl.value, "bytes": by.value}


Solver.profile = _solver_profile
Solver.profile_read = _solver_profile_read
