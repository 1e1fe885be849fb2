"""Maximum principal angle between subspaces (Definition 2.1).

tan angle(X, Y) = || X_perp^H Y (X^H Y)^+ || with X, X_perp orthonormal bases of the
subspace and its complement; pi/2 when X^H Y is rank deficient.
"""
import numpy as np


def max_angle(Xbasis, Ybasis):
    Qx, _ = np.linalg.qr(Xbasis, mode="complete")
    q = Xbasis.shape[1]
    X, Xp = Qx[:, :q], Qx[:, q:]
    Qy, _ = np.linalg.qr(Ybasis)
    G = X.conj().T @ Qy
    if np.linalg.matrix_rank(G) < Qy.shape[1]:
        return np.pi / 2
    t = np.linalg.norm(Xp.conj().T @ Qy @ np.linalg.pinv(G), 2)
    return float(np.arctan(t))
