"""Dense test problems with prescribed spectra.

* Toy problems of Section 4.1 ("Controlled numerical experiments on dense random
  matrices"): A = Q diag(lambda) Q^T with lambda_j = 1 + 3(j-1)/(n-1) for the n wanted
  pairs and 5 + 0.2(j-n-1) for the rest; perturbed filter matrix A + eps E; generalized
  pencil with B sharing the eigenbasis of A (eigenvalues of B linear in [1, 5]) and an
  approximate inverse D^-1 = B^-1 + zeta E with ||E||_2 = 1.
* Dense benchmark problems: a standard problem with spectrum linspace(-1, 10) and a gap
  of 0.05 after the 50th eigenvalue, and a generalized problem with a dense SPD B whose
  diagonal is prescribed, so that D^-1 = diag(B)^-1 is a meaningful approximate inverse.

Matrices are float64, C-contiguous, symmetric to the last bit (the upper triangle is
mirrored).  Nothing here runs the eigensolver.
"""
import numpy as np


def _rng(seed):
    return np.random.default_rng(seed)


def _symmetrize(a):
    a = np.triu(a)
    return a + np.triu(a, 1).T


def orthogonal(m, seed):
    """Random orthogonal m x m matrix: Householder QR of an i.i.d. N(0,1) matrix
    (the paper's dgeqrf/dorgqr construction), with the sign of each column fixed
    by diag(R) > 0 so the result is a deterministic function of the seed."""
    g = _rng(seed).standard_normal((m, m))
    q, r = np.linalg.qr(g)
    q *= np.sign(np.diag(r))[None, :]
    return np.ascontiguousarray(q)


def dense_from_spectrum(q, lam):
    """A = Q diag(lam) Q^T, symmetrised."""
    return _symmetrize((q * lam[None, :]) @ q.T)


def config1_spectrum(m=1000, gap_after=50, gap=0.05, lo=-1.0, hi=10.0):
    """lambda_j = lo + (hi-lo)(j-1)/(m-1) + gap*[j > gap_after]  (1-based j)."""
    lam = np.linspace(lo, hi, m)
    lam[gap_after:] += gap
    return lam


def dense_config1(m=1000, seed=1):
    """Standard problem A = Q diag(lambda) Q^T, B = I, D = I.  Returns a dict with the
    exact spectrum (ascending)."""
    lam = config1_spectrum(m)
    q = orthogonal(m, seed)
    return {"A": dense_from_spectrum(q, lam), "B": None, "Dinv": None, "lam": lam, "Q": q}


def dense_config2(m=4000, seed_q=1, seed_q2=3, seed_s=4, seed_g=5, t=0.1, variant="a",
                  smin=0.5, smax=50.0):
    """Dense generalized problem A u = lambda B u with D^-1 = diag(B)^-1.

    A: as the standard problem (spectrum linspace(-1, 10) with the gap after index 50).
    variant "a": B = S^1/2 (I + t G) S^1/2, S log-uniform in [smin, smax], G = Q2 diag(U[-1,1]) Q2^T
                 with its diagonal set to zero, so diag(B) = S exactly and B is SPD
                 (||G|| <= 2, t = 0.1).
    variant "b": B = Q2 diag(mu) Q2^T with mu log-uniform in [smin, smax] (literal reading).
    Returns dict(A, B, Dinv) with Dinv = 1 / diag(B).
    """
    lam = config1_spectrum(m)
    a = dense_from_spectrum(orthogonal(m, seed_q), lam)
    q2 = orthogonal(m, seed_q2)
    if variant == "a":
        s = np.exp(_rng(seed_s).uniform(np.log(smin), np.log(smax), m))
        g = dense_from_spectrum(q2, _rng(seed_g).uniform(-1.0, 1.0, m))
        np.fill_diagonal(g, 0.0)
        r = np.sqrt(s)
        b = _symmetrize((np.eye(m) + t * g) * r[:, None] * r[None, :])
        np.fill_diagonal(b, s)
    elif variant == "b":
        mu = np.exp(_rng(seed_s).uniform(np.log(smin), np.log(smax), m))
        b = dense_from_spectrum(q2, mu)
    else:
        raise ValueError(variant)
    return {"A": a, "B": b, "Dinv": 1.0 / np.diag(b).copy()}


def _unit_symmetric(m, seed):
    """E = (F + F^T)/2 with F_ij ~ N(0,1), scaled so that ||E||_2 = 1."""
    f = _rng(seed).standard_normal((m, m))
    e = _symmetrize(0.5 * (f + f.T))
    return e / np.abs(np.linalg.eigvalsh(e)).max()


def toy_spectrum(m=1000, n=10):
    j = np.arange(1, m + 1, dtype=np.float64)
    return np.where(j <= n, 1.0 + 3.0 * (j - 1) / (n - 1), 5.0 + 0.2 * (j - n - 1))


def toy_standard(eps, m=1000, n=10, seed=1, seed_e=11):
    """Standard toy problem (B = I) with perturbed filter matrix A~ = A + eps E."""
    lam = toy_spectrum(m, n)
    q = orthogonal(m, seed)
    a = dense_from_spectrum(q, lam)
    a_f = a + eps * _unit_symmetric(m, seed_e) if eps else a.copy()
    return {"A": a, "A_filter": a_f, "B": None, "Dinv": None, "lam": lam, "Q": q,
            "lmin": lam[0] - 0.05, "lT": 0.5 * (lam[n - 1] + lam[n]), "lmax": lam[-1] + 0.1}


def toy_generalized(zeta, m=1000, n=10, seed=1, seed_e=12):
    """Generalized toy problem: B shares the eigenbasis Q of A (same seed), eigenvalues
    b_j = 1 + 4(j-1)/(m-1); approximate inverse D^-1 = B^-1 + zeta E, ||E||_2 = 1 (dense).
    The generalized eigenvalues are a_j / b_j; the bounds follow the same recipe as the
    standard toy problem applied to those eigenvalues."""
    lam_a = toy_spectrum(m, n)
    bj = 1.0 + 4.0 * np.arange(m) / (m - 1)
    q = orthogonal(m, seed)
    a = dense_from_spectrum(q, lam_a)
    b = dense_from_spectrum(q, bj)
    binv = dense_from_spectrum(q, 1.0 / bj)
    dinv = binv + zeta * _unit_symmetric(m, seed_e) if zeta else binv
    gen = lam_a / bj
    srt = np.sort(gen)
    return {"A": a, "B": b, "Dinv_dense": dinv, "Binv": binv, "lam": srt, "Q": q,
            "lmin": srt[0] - 0.05, "lT": 0.5 * (srt[n - 1] + srt[n]), "lmax": srt[-1] + 0.1}


def gaussian_block(m, n, seed=2, dtype=np.float64):
    """Initial guess X0: i.i.d. N(0,1) entries (complex: independent real and imaginary
    parts, each N(0, 1/2))."""
    r = _rng(seed)
    if np.issubdtype(dtype, np.complexfloating):
        return (r.standard_normal((m, n)) + 1j * r.standard_normal((m, n))) / np.sqrt(2.0)
    return r.standard_normal((m, n))
