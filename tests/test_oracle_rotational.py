"""Rotational near-null modes for the elasticity AMG, an oracle option.

Smoothed aggregation with the six rigid-body modes as candidates (three
translations, three rotations; Vanek, Mandel and Brezina) instead of the
three translations the CUDA path uses.  The pins fix the tentative
prolongator; the last test measures what the option buys (the figures the
design notes quote: t-u-p iterations and the size of the first coarse
operator).
"""
import numpy as np
import scipy.sparse as sp

import fracgen
from oracle import sparse as osp
from oracle.amg import AMG, AmgOptions, rigid_modes, tentative_nullspace
from oracle.fgmres import fgmres
from oracle.precond import BlockPreconditioner
from oracle import schur


def coords(P):
    N1 = P.N + 1
    g = P.node_grid
    return np.stack([g % N1, (g // N1) % N1, g // (N1 * N1)], 1) / P.N


def test_rigid_modes_are_the_kernel_of_an_unconstrained_element():
    """The candidates are rigid motions: the unit hexahedron's stiffness
    annihilates all six (and the translations alone span only three)."""
    K = fracgen.hex8_stiffness(0.25)
    X = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], float)
    Z = rigid_modes(X)
    assert np.linalg.matrix_rank(Z) == 6
    assert np.abs(K @ Z).max() <= 1e-14 * np.abs(K).max()


def test_tentative_prolongator_reproduces_the_modes_on_every_aggregate():
    """P_tent Z_c = Z on the rows of every aggregate whose coarse dofs are all
    alive, P_tent has orthonormal columns, and an aggregate too small for six
    modes (a single node: rank 3) keeps exactly its live part.  A lost
    rotation column, an unnormalised Q or a swapped component fail it."""
    P = fracgen.generate("planes64", N=8)
    S1 = schur.s1(P)
    A = AMG(S1, 3, AmgOptions(coarse_max=20), near_null=rigid_modes(coords(P)))
    L = A.levels[0]
    Z = rigid_modes(coords(P))
    Pt, Zc, dead = tentative_nullspace(L.agg, L.nc, 3, Z)
    G = (Pt.T @ Pt).toarray()
    live = ~dead
    assert np.allclose(G[np.ix_(live, live)], np.eye(live.sum()), atol=1e-13)
    assert not G[np.ix_(dead, dead)].any()
    rec = Pt @ Zc
    agg = L.agg
    nodes_full = np.array([i for i in range(len(agg)) if agg[i] >= 0 and not dead[6 * agg[i]:6 * agg[i] + 6].any()])
    rows = (3 * nodes_full[:, None] + np.arange(3)).ravel()
    assert nodes_full.size > 0.5 * len(agg)
    assert np.allclose(rec[rows], Z[rows], rtol=0, atol=1e-12 * np.abs(Z).max())
    # a one-node aggregate carries three live dofs (its translations span the
    # rotations' values at one point); two nodes carry five (the rotation
    # about the line through them moves neither)
    for m, n_dead in ((1, 3), (2, 1)):
        Pt1, Zc1, d1 = tentative_nullspace(np.zeros(m, dtype=np.int64), 1, 3, Z[:3 * m])
        assert d1.sum() == n_dead and np.allclose(Pt1 @ Zc1, Z[:3 * m], atol=1e-14)


def test_coarse_operators_have_six_by_six_blocks_and_stay_galerkin():
    P = fracgen.generate("planes64", N=8)
    S1 = schur.s1(P)
    A = AMG(S1, 3, AmgOptions(coarse_max=20), near_null=rigid_modes(coords(P)))
    assert [L.B for L in A.levels] == [3] + [6] * (len(A.levels) - 1)
    L0, L1 = A.levels[0], A.levels[1]
    ref = (L0.R @ L0.S @ L0.P).toarray()
    dead = np.abs(ref).sum(axis=1) == 0
    ref[dead, dead] = 1.0
    assert np.allclose(L1.S.toarray(), ref, atol=1e-12 * np.abs(ref).max())


def test_rotational_modes_cut_iterations_and_grow_the_coarse_operator():
    """Three planes at 16^3, t-u-p, FGMRES to 1e-8: 45 iterations with the
    translations, 39 with the rigid modes, while the first coarse operator
    stores about four times the scalars (6 x 6 instead of 3 x 3 blocks)."""
    P = fracgen.generate("planes64", N=16)
    J = osp.jacobian(P)
    out = {}
    for name, nn in (("translations", None), ("rigid", rigid_modes(coords(P)))):
        M = BlockPreconditioner(P, "tup", u_near_null=nn)
        r = fgmres(lambda v: J @ v, M, P.b, 1e-8, 400)
        assert r.relres <= 1e-8
        out[name] = (r.iters, M.u_inv.levels[1].S.nnz)
    assert out["translations"][0] == 45 and out["rigid"][0] == 39
    growth = out["rigid"][1] / out["translations"][1]
    assert 3.5 < growth < 4.5
