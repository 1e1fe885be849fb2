"""Finite-element test problems on a periodic uniform hexahedral mesh.

Discretisation (the paper gives none; this is the construction used for the synthetic
stand-ins of its DFT-FE benchmarks): periodic cube of n^3 cells of size h = 0.5, Q4
Lagrange elements with 5 Gauss-Lobatto-Legendre (GLL) nodes per direction, so the mesh
has m = (4n)^3 dofs and each cell couples n_c = 125 of them.

Cell matrices, integrated with 6-point Gauss-Legendre quadrature per direction:
    stiffness  K_c = int grad(phi_i) . grad(phi_j)
    mass       M_c = int phi_i phi_j                     (B, the consistent mass)
    potential  V_c = int V(r) phi_i phi_j
    A_c = 0.5 K_c + V_c                                  (real, Gamma point)
    A_c(k) = 0.5 K_c - i sum_d k_d int phi_i d_d phi_j + 0.5 |k|^2 M_c + V_c   (Bloch k-point)
The approximate inverse of B is the inverse of the GLL-lumped (diagonal) mass.
V(r) = -sum_i d_i exp(-|r - c_i|^2 / (2 w_i^2)) with minimum-image distances.

Local node order inside a cell: l = (lz*5 + ly)*5 + lx.  Global dof order:
dof = (gz*4n + gy)*4n + gx with g = 4*cell + local (mod 4n).  Cells are numbered
c = (cz*n + cy)*n + cx.
"""
import numpy as np

NQ = 6          # Gauss-Legendre points per direction
P = 4           # polynomial degree
NP = P + 1      # nodes per direction
NC = NP ** 3    # nodes per cell


def gll_1d():
    """The 5 GLL nodes on [-1, 1] and their weights (closed form)."""
    s = np.sqrt(3.0 / 7.0)
    x = np.array([-1.0, -s, 0.0, s, 1.0])
    w = np.array([1.0 / 10.0, 49.0 / 90.0, 32.0 / 45.0, 49.0 / 90.0, 1.0 / 10.0])
    return x, w


def _lagrange(nodes, xi):
    """Values and derivatives of the Lagrange basis on `nodes` at points `xi`:
    returns (len(xi), len(nodes)) arrays."""
    k = len(nodes)
    phi = np.ones((len(xi), k))
    dphi = np.zeros((len(xi), k))
    for a in range(k):
        others = [b for b in range(k) if b != a]
        den = np.prod([nodes[a] - nodes[b] for b in others])
        for b in others:
            phi[:, a] *= (xi - nodes[b])
        for skip in others:
            term = np.ones(len(xi))
            for b in others:
                if b != skip:
                    term = term * (xi - nodes[b])
            dphi[:, a] += term
        phi[:, a] /= den
        dphi[:, a] /= den
    return phi, dphi


def fe_1d_matrices(h=0.5):
    """1D element mass M1, stiffness K1 and first-derivative G1[a,b] = int phi_a phi_b'
    on an element of length h (6-point Gauss-Legendre)."""
    nodes, _ = gll_1d()
    xq, wq = np.polynomial.legendre.leggauss(NQ)
    phi, dphi = _lagrange(nodes, xq)
    jac = 0.5 * h
    m1 = (phi * wq[:, None]).T @ phi * jac
    k1 = (dphi * wq[:, None]).T @ dphi / jac
    g1 = (phi * wq[:, None]).T @ dphi
    return m1, k1, g1


def fe_mesh(n):
    """Connectivity of the periodic n^3 Q4 mesh: (n^3, 125) int32 array of global dofs."""
    g = 4 * n
    c = np.arange(n)
    cz, cy, cx = np.meshgrid(c, c, c, indexing="ij")
    l = np.arange(NP)
    lz, ly, lx = np.meshgrid(l, l, l, indexing="ij")
    gx = (4 * cx.reshape(-1, 1) + lx.reshape(1, -1)) % g
    gy = (4 * cy.reshape(-1, 1) + ly.reshape(1, -1)) % g
    gz = (4 * cz.reshape(-1, 1) + lz.reshape(1, -1)) % g
    return ((gz * g + gy) * g + gx).astype(np.int32)


def _wells(n_wells, box, seed, depth=(2.0, 5.0), width=(0.3, 0.8)):
    r = np.random.default_rng(seed)
    d = r.uniform(*depth, n_wells)
    w = r.uniform(*width, n_wells)
    c = r.uniform(0.0, box, (n_wells, 3))
    return d, w, c


def potential(points, wells, box):
    """V at (k, 3) points for the well parameters (d, w, c), minimum-image distances."""
    d, w, c = wells
    v = np.zeros(points.shape[0])
    for i in range(len(d)):
        dx = points - c[i][None, :]
        dx -= box * np.round(dx / box)
        v -= d[i] * np.exp(-(dx * dx).sum(1) / (2.0 * w[i] ** 2))
    return v


def _kron3(z, y, x):
    return np.kron(z, np.kron(y, x))


def fe_problem(n, seed_wells=6, n_wells=8, h=0.5, wells=None, kpoint=None, v_scale=1.0,
               chunk=512):
    """Assemble the cell matrices of the periodic Q4 problem with n^3 cells.

    Returns dict(n, m, h, box, cell_dofs (C,125) int32, A_cells (C,125,125) float64 or
    complex128, B_cell (125,125) float64 shared by all cells, Dinv (m,) float64,
    wells).  `kpoint` = (kx, ky, kz) adds the Bloch terms (complex Hermitian problem);
    `wells=None` draws the 8 seeded wells, `v_scale=0` gives the separable V = 0 case.
    """
    box = n * h
    m1, k1, g1 = fe_1d_matrices(h)
    stiff = _kron3(k1, m1, m1) + _kron3(m1, k1, m1) + _kron3(m1, m1, k1)
    mass = _kron3(m1, m1, m1)
    cells = fe_mesh(n)
    ncell = n ** 3
    if wells is None:
        wells = _wells(n_wells, box, seed_wells)
    nodes, wgll = gll_1d()
    xq, wq = np.polynomial.legendre.leggauss(NQ)
    phi, _ = _lagrange(nodes, xq)
    jac = 0.5 * h
    # 3D quadrature: point q = (qz*6 + qy)*6 + qx
    phi3 = _kron3(phi, phi, phi)                      # (216, 125)
    w3 = _kron3(wq, wq, wq) * jac ** 3                # (216,)
    qz, qy, qx = np.meshgrid(xq, xq, xq, indexing="ij")
    ref = np.stack([qx.ravel(), qy.ravel(), qz.ravel()], 1)
    cidx = np.arange(ncell)
    origin = np.stack([cidx % n, (cidx // n) % n, cidx // (n * n)], 1) * h
    base = 0.5 * stiff
    cplx = kpoint is not None
    if cplx:
        k = np.asarray(kpoint, dtype=np.float64)
        grad_terms = k[0] * _kron3(m1, m1, g1) + k[1] * _kron3(m1, g1, m1) + k[2] * _kron3(g1, m1, m1)
        base = base + 0.5 * float(k @ k) * mass - 1j * grad_terms
    a_cells = np.empty((ncell, NC, NC), dtype=np.complex128 if cplx else np.float64)
    for s in range(0, ncell, chunk):
        e = min(ncell, s + chunk)
        pts = origin[s:e, None, :] + (ref[None, :, :] + 1.0) * jac       # (b, 216, 3)
        v = potential(pts.reshape(-1, 3), wells, box).reshape(e - s, -1) * v_scale
        vc = np.einsum("qi,bq,qj->bij", phi3, v * w3[None, :], phi3, optimize=True)
        a_cells[s:e] = base[None] + vc
    # GLL-lumped diagonal mass
    dl = _kron3(wgll, wgll, wgll) * jac ** 3
    dvec = np.zeros((4 * n) ** 3)
    np.add.at(dvec, cells.ravel(), np.tile(dl, ncell))
    return {"n": n, "m": (4 * n) ** 3, "h": h, "box": box, "cell_dofs": cells,
            "A_cells": a_cells, "B_cell": mass, "Dinv": 1.0 / dvec, "wells": wells,
            "kpoint": None if kpoint is None else tuple(float(t) for t in kpoint)}


def fe_config3(n=16, **kw):
    """Real FE problem: 16^3 cells (m = 262,144 dofs), 8 seeded wells."""
    return fe_problem(n, **kw)


def fe_kpoint_problem(n, kappa, **kw):
    """Complex Hermitian Bloch problem at k = (2 pi / L) kappa."""
    box = n * kw.get("h", 0.5)
    return fe_problem(n, kpoint=2.0 * np.pi / box * np.asarray(kappa), **kw)


def fe_scf_chain(n, steps, seed_wells=6, seed_pert=100, rel=0.01, kpoint=None):
    """A sequence of FE problems whose well depths drift by a seeded relative perturbation `rel`
    per step (each step perturbs the previous one), as in the successive operators of an outer
    self-consistency loop.  kpoint as in fe_problem."""
    box = n * 0.5
    d, w, c = _wells(8, box, seed_wells)
    r = np.random.default_rng(seed_pert)
    out = []
    for _ in range(steps):
        out.append(fe_problem(n, wells=(d.copy(), w, c), kpoint=kpoint))
        d = d * (1.0 + rel * r.standard_normal(d.shape))
    return out


def fe_config4_list(n_problems=16, seed=7, nmin=8, nmax=20, nev_range=(100, 800)):
    """Specs of the batched k-point workload: cells per dimension, nev, block N and the
    reduced Bloch vector kappa in [-0.5, 0.5)^3 for each problem (matrices are built
    on demand with fe_kpoint_problem)."""
    r = np.random.default_rng(seed)
    out = []
    for _ in range(n_problems):
        n = int(r.integers(nmin, nmax + 1))
        nev = int(r.integers(nev_range[0], nev_range[1] + 1))
        out.append({"n": n, "nev": nev, "block": int(np.ceil(1.2 * nev / 16.0) * 16),
                    "kappa": r.uniform(-0.5, 0.5, 3)})
    return out
