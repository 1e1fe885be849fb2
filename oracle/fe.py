"""Global operator of a cell-matrix (finite-element) discretisation.

A = sum_c P_c^T A_c P_c, where P_c picks the cell's dofs (duplicate entries summed).
This is the plain definition of the element-level operator whose product the paper
evaluates cell by cell with batched GEMMs (Remark in Section 4.2).
"""
import numpy as np
import scipy.sparse as sp


def assemble(cell_dofs, cell_mats, m):
    """cell_mats: (C, nc, nc) array, or a single (nc, nc) matrix shared by all cells."""
    C, nc = cell_dofs.shape
    if cell_mats.ndim == 2:
        cell_mats = np.broadcast_to(cell_mats, (C, nc, nc))
    rows = np.repeat(cell_dofs, nc, axis=1).ravel()
    cols = np.tile(cell_dofs, (1, nc)).ravel()
    return sp.csr_matrix((cell_mats.reshape(-1), (rows, cols)), shape=(m, m))
