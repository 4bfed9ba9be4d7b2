"""Approximate Schur complements of the two restriction orderings.

* Alg. 1 (cpt_tpu):  H~ = Bdiag(H, 3),  T~ = diag(T),
                     S~ = A + C1 H~^-1 C2 - Q1 T~^-1 Q2      (Eq. appSchur_1)
* Alg. 3 (cpt_tup):  H~ = Bdiag(H, 3),  S1 = A + C1 H~^-1 C2  (Eq. Schur1_2),
                     S~2 = T - FS(Q2, S1, Q1)                 (Eq. app_Schur2_2)
  with the algebraic fixed-stress diagonal of Eq. FS_algebraic (Remark
  rem:FS): [S_K]_k = Q2^(k)T (S1^(k))^-1 Q1^(k), S1^(k) the principal
  submatrix of S1 on K^(k) = nz(Q1 column k) U nz(Q2 row k).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import sparse as osp


class SingularBlock(RuntimeError):
    pass


def htilde_blocks(P, Hs: sp.csr_matrix | None = None) -> np.ndarray:
    """The 3x3 diagonal blocks of H, one per face (Bdiag(H,3), Alg. 1)."""
    Hs = osp.csr(P.H) if Hs is None else Hs
    out = np.zeros((P.n_face, 3, 3))
    coo = Hs.tocoo()
    r, c = coo.row, coo.col
    keep = (r // 3) == (c // 3)
    np.add.at(out, (r[keep] // 3, r[keep] % 3, c[keep] % 3), coo.data[keep])
    return out


def htilde_inv(P, Hs=None) -> sp.csr_matrix:
    """H~^-1 as a block-diagonal sparse matrix (3x3 blocks)."""
    Hb = htilde_blocks(P, Hs)
    if len(Hb) == 0:
        return sp.csr_matrix((0, 0))
    det = np.linalg.det(Hb)
    scale = np.abs(Hb).reshape(len(Hb), -1).max(axis=1)
    bad = ~(np.abs(det) > 1e-300) | (np.abs(det) <= 1e-14 * np.maximum(scale, 1e-300) ** 3)
    if np.any(bad):
        raise SingularBlock(f"singular H~ block at faces {np.nonzero(bad)[0][:8]}")
    Hi = np.linalg.inv(Hb)
    return sp.csr_matrix(sp.block_diag(list(Hi), format="csr"))


def s1(P, blk=None) -> sp.csr_matrix:
    """S1 = A + C1 H~^-1 C2 (Eq. Schur1_2, Alg. 3)."""
    b = blk or osp.blocks(P)
    return (b["A"] + b["C1"] @ htilde_inv(P, b["H"]) @ b["C2"]).tocsr()


def t_diag(P, blk=None) -> np.ndarray:
    b = blk or osp.blocks(P)
    return b["T"].diagonal()


def s_tilde(P, blk=None, S1=None) -> sp.csr_matrix:
    """S~ = A + C1 H~^-1 C2 - Q1 T~^-1 Q2 with T~ = diag(T) (Eq. appSchur_1)."""
    b = blk or osp.blocks(P)
    S1 = s1(P, b) if S1 is None else S1
    Tti = sp.diags(1.0 / t_diag(P, b))
    return (S1 - b["Q1"] @ Tti @ b["Q2"]).tocsr()


def fixed_stress(P, S1: sp.csr_matrix, blk=None) -> np.ndarray:
    """Diagonal of S_K by Eq. FS_algebraic.

    For each face k: K1 = indices of the nonzero entries of column k of Q1,
    K2 = those of row k of Q2, K = sorted(K1 U K2).  If K2 is empty the entry
    is 0.  Otherwise [S_K]_k = Q2[k, K] . solve(S1[K, K], Q1[K, k]).
    """
    b = blk or osp.blocks(P)
    Q1c = b["Q1"].tocsc()
    Q2r = b["Q2"].tocsr()
    S1r = S1.tocsr()
    nf = P.n_face
    out = np.zeros(nf)
    for k in range(nf):
        c0, c1 = Q1c.indptr[k], Q1c.indptr[k + 1]
        K1 = Q1c.indices[c0:c1][Q1c.data[c0:c1] != 0.0]
        r0, r1 = Q2r.indptr[k], Q2r.indptr[k + 1]
        K2 = Q2r.indices[r0:r1][Q2r.data[r0:r1] != 0.0]
        if K2.size == 0:
            continue
        K = np.union1d(K1, K2)
        Sk = S1r[K][:, K].toarray()
        q1 = np.asarray(b["Q1"][K, k].todense()).ravel()
        q2 = np.asarray(Q2r[k, K].todense()).ravel()
        y = sla.lu_solve(sla.lu_factor(Sk), q1)
        out[k] = q2 @ y
    return out


def fixed_stress_geometric(P, omega: np.ndarray, kbar: np.ndarray, dt: float, blk=None) -> np.ndarray:
    """Diagonal of the geometric fixed stress (Eq. FS): the volume |Omega_k|
    of the cells around face k over their bulk modulus Kbar_k, in the units
    and sign of Q2 S1^-1 Q1 here: Q2 carries -Q1^T / dt on open faces, so
    [S_K]_k = -|Omega_k| / (Kbar_k dt).  Faces whose row of Q2 is zero get 0,
    the index rule of the algebraic form."""
    b = blk or osp.blocks(P)
    Q2r = b["Q2"].tocsr()
    out = np.zeros(P.n_face)
    for k in range(P.n_face):
        r0, r1 = Q2r.indptr[k], Q2r.indptr[k + 1]
        if np.any(Q2r.data[r0:r1] != 0.0):
            out[k] = -omega[k] / (kbar[k] * dt)
    return out


def s2_tilde(P, S1: sp.csr_matrix, blk=None, sk: np.ndarray | None = None) -> sp.csr_matrix:
    """S~2 = T - S_K (Eq. app_Schur2_2), S_K diagonal: the algebraic fixed
    stress, or the given diagonal ``sk`` (e.g. the geometric form)."""
    b = blk or osp.blocks(P)
    d = fixed_stress(P, S1, b) if sk is None else sk
    return (b["T"] - sp.diags(d)).tocsr()
