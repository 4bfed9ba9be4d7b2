"""Plain dense definitions for tiny cases (pins for the oracle).

* ``solve``: x = J^-1 b, the exact block solve of Eq. ex_Jac_appl.
* ``schur_exact_tpu``: S = A + C1 H~^-1 C2 - Q1 T^-1 Q2 (Eq. Schur_1).
* ``schur2_exact``: S2 = T - Q2 S1^-1 Q1 (Eq. Schur2_2).
* ``m1_matrix`` / ``m2_matrix``: the preconditioners written as the products
  of block factors in Eq. P1 and Eq. P2 (in the permuted orders of
  Eq. Q1 / Eq. Q2, mapped back to [u; t; p]).
* ``m2_factors`` / ``m2_star_matrix``: the three factors of Eq. P2 and the
  incomplete form D2^-1 L2^-1 (the last two factors only).
"""
from __future__ import annotations

import numpy as np

from . import schur
from . import sparse as osp


def solve(P, b=None) -> np.ndarray:
    J = osp.jacobian(P).toarray()
    return np.linalg.solve(J, P.b if b is None else b)


def blocks_dense(P):
    return {k: v.toarray() for k, v in osp.blocks(P).items()}


def hinv_dense(P):
    return schur.htilde_inv(P).toarray()


def schur_exact_tpu(P):
    d = blocks_dense(P)
    Hi = hinv_dense(P)
    return d["A"] + d["C1"] @ Hi @ d["C2"] - d["Q1"] @ np.linalg.solve(d["T"], d["Q2"])


def schur2_exact(P):
    d = blocks_dense(P)
    Hi = hinv_dense(P)
    S1 = d["A"] + d["C1"] @ Hi @ d["C2"]
    return d["T"] - d["Q2"] @ np.linalg.solve(S1, d["Q1"])


def m1_matrix(P, S_tilde: np.ndarray | None = None, T: np.ndarray | None = None):
    """Eq. P1 in the order (t, p, u): M1^-1 = U1^-1 D1^-1 L1^-1, returned in
    the [u; t; p] order of Eq. JacSys."""
    d = blocks_dense(P)
    Hi = hinv_dense(P)
    Tm = d["T"] if T is None else T
    Ti = np.linalg.inv(Tm)
    St = S_tilde if S_tilde is not None else (
        d["A"] + d["C1"] @ Hi @ d["C2"] - d["Q1"] @ np.diag(1.0 / np.diag(d["T"])) @ d["Q2"])
    nt, npp, nu = d["H"].shape[0], d["T"].shape[0], d["A"].shape[0]
    I_t, I_p, I_u = np.eye(nt), np.eye(npp), np.eye(nu)
    Z = np.zeros
    U = np.block([[I_t, Z((nt, npp)), Hi @ d["C2"]],
                  [Z((npp, nt)), I_p, -Ti @ d["Q2"]],
                  [Z((nu, nt)), Z((nu, npp)), I_u]])
    D = np.block([[-Hi, Z((nt, npp)), Z((nt, nu))],
                  [Z((npp, nt)), Ti, Z((npp, nu))],
                  [Z((nu, nt)), Z((nu, npp)), np.linalg.inv(St)]])
    L = np.block([[I_t, Z((nt, npp)), Z((nt, nu))],
                  [Z((npp, nt)), I_p, Z((npp, nu))],
                  [d["C1"] @ Hi, -d["Q1"] @ Ti, I_u]])
    M_tpu = U @ D @ L
    # permutation Q1 maps [u; t; p] -> [t; p; u]
    perm = np.concatenate([np.arange(nu, nu + nt), np.arange(nu + nt, nu + nt + npp),
                           np.arange(nu)])
    Q = np.eye(nu + nt + npp)[perm]
    return Q.T @ M_tpu @ Q


def m2_factors(P, S1_inv: np.ndarray | None = None, S2_tilde: np.ndarray | None = None):
    """The factors (U2^-1, D2^-1, L2^-1) of Eq. P2 in the (t, u, p) order of
    Eq. Q2, and the permutation matrix Q with Q [u; t; p] = [t; u; p]."""
    d = blocks_dense(P)
    Hi = hinv_dense(P)
    S1 = d["A"] + d["C1"] @ Hi @ d["C2"]
    S1i = np.linalg.inv(S1) if S1_inv is None else S1_inv
    if S2_tilde is None:
        S2_tilde = schur.s2_tilde(P, schur.s1(P)).toarray()
    S2i = np.linalg.inv(S2_tilde)
    nt, npp, nu = d["H"].shape[0], d["T"].shape[0], d["A"].shape[0]
    I_t, I_p, I_u = np.eye(nt), np.eye(npp), np.eye(nu)
    Z = np.zeros
    U = np.block([[I_t, Hi @ d["C2"], -Hi @ d["C2"] @ S1i @ d["Q1"]],
                  [Z((nu, nt)), I_u, -S1i @ d["Q1"]],
                  [Z((npp, nt)), Z((npp, nu)), I_p]])
    D = np.block([[-Hi, Z((nt, nu)), Z((nt, npp))],
                  [Z((nu, nt)), S1i, Z((nu, npp))],
                  [Z((npp, nt)), Z((npp, nu)), S2i]])
    L = np.block([[I_t, Z((nt, nu)), Z((nt, npp))],
                  [d["C1"] @ Hi, I_u, Z((nu, npp))],
                  [-d["Q2"] @ S1i @ d["C1"] @ Hi, -d["Q2"] @ S1i, I_p]])
    perm = np.concatenate([np.arange(nu, nu + nt), np.arange(nu), np.arange(nu + nt, nu + nt + npp)])
    Q = np.eye(nu + nt + npp)[perm]
    return U, D, L, Q


def m2_matrix(P, S1_inv: np.ndarray | None = None, S2_tilde: np.ndarray | None = None):
    """Eq. P2 in the order (t, u, p), returned in the [u; t; p] order."""
    U, D, L, Q = m2_factors(P, S1_inv, S2_tilde)
    return Q.T @ (U @ D @ L) @ Q


def m2_star_matrix(P, S1_inv: np.ndarray | None = None, S2_tilde: np.ndarray | None = None):
    """The incomplete factorisation D2^-1 L2^-1 of Eq. P2, in [u; t; p]."""
    U, D, L, Q = m2_factors(P, S1_inv, S2_tilde)
    return Q.T @ (D @ L) @ Q
