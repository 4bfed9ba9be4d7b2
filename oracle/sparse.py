"""Scalar sparse views of the block Jacobian (Eq. JacSys, Sec. 2).

The Jacobian is J = [A C1 Q1; C2 -H 0; Q2 0 T] with the unknown order
[u; t; p] of Eq. JacSys.  Blocks arrive from the input generator as BSR
triples; here they become scipy CSR matrices of scalars.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def csr(B) -> sp.csr_matrix:
    """Scalar CSR of a BSR block (row_ptr, col_idx, val[nnzb, br, bc])."""
    m = sp.bsr_matrix((B.val, B.col_idx, B.row_ptr),
                      shape=(B.n_brows * B.br, B.n_bcols * B.bc))
    return m.tocsr()


def blocks(P) -> dict:
    return {k: csr(v) for k, v in P.blocks().items()}


def jacobian(P, blk: dict | None = None) -> sp.csr_matrix:
    """J of Eq. JacSys: rows (u, t, p), columns (u, t, p)."""
    b = blk or blocks(P)
    return sp.bmat([[b["A"], b["C1"], b["Q1"]],
                    [b["C2"], -b["H"], None],
                    [b["Q2"], None, b["T"]]], format="csr")


def split(P, x: np.ndarray):
    nu, nt = 3 * P.n_node, 3 * P.n_face
    return x[:nu], x[nu:nu + nt], x[nu + nt:]
