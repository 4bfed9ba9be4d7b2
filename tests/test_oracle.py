"""Pins of the CPU oracle against what the paper and the mathematics fix:
the exact solution (Eq. ex_Jac_appl), the algebraic forms Eq. P1 / Eq. P2 of
Alg. 2 / Alg. 4, the exactness limit M^-1 = J^-1, Prop. 3.1, GMRES theory,
the greedy-MIS theorem, the Chebyshev polynomial and the fixed-stress
bound."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import fracgen
from oracle import amg as oamg
from oracle import dense, rng, schur
from oracle.adjoint import operator_matrix as adjoint_operator
from oracle import sparse as osp
from oracle.amg import AMG, AmgOptions
from oracle.fgmres import fgmres
from oracle.precond import BlockPreconditioner

from fields import assert_fields

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_oracle_rng_reference_outputs():
    ref = [int(l, 16) for l in open(os.path.join(GOLD, "splitmix64_seed0.txt"))
           if l.strip() and not l.startswith("#")]
    assert [int(v) for v in rng.rand_u64(0, 0, np.arange(4))] == ref
    u = rng.uniform(7, 3, np.arange(100000))
    assert u.min() >= 0 and u.max() < 1 and abs(u.mean() - 0.5) < 5e-3


@pytest.fixture(scope="module")
def small_mixed():
    # 4^3 cells, three central planes, stick/slip/open mix; ~840 unknowns
    return fracgen.generate("planes64", N=4, seed=2)


@pytest.mark.parametrize("variant", ["tpu", "tup"])
def test_fgmres_matches_dense_solution(tiny, variant):
    J = osp.jacobian(tiny)
    xs = dense.solve(tiny)
    M = BlockPreconditioner(tiny, variant, opt=AmgOptions(coarse_max=64))
    r = fgmres(lambda v: J @ v, M, tiny.b, tol=1e-12, maxit=300)
    # the true residual floors near eps * || |J| |x| || / ||b|| ~ 1e-10 here
    # (tractions are ~1e7 times the displacements); the solution is tighter
    assert r.relres <= 1e-9
    # every field (u, t, p) on its own scale, not the t-dominated whole norm
    assert_fields(tiny, r.x, xs, 1e-11, f"{variant} x vs dense")


@pytest.mark.parametrize("variant", ["tpu", "tup", "tup_star"])
def test_algorithm_equals_block_factor_form(small_mixed, variant):
    """Alg. 2 (Alg. 4) with exact inner solves is the operator of Eq. P1
    (Eq. P2); the incomplete form is the product D2^-1 L2^-1 of Eq. P2's
    last two factors."""
    P = small_mixed
    assert set(np.unique(P.state)) == {0, 1, 2}
    M = BlockPreconditioner(P, variant, "exact", "exact")
    Md = {"tpu": dense.m1_matrix, "tup": dense.m2_matrix, "tup_star": dense.m2_star_matrix}[variant](P)
    rs = np.random.default_rng(5)
    for _ in range(3):
        w = rs.standard_normal(P.n)
        a, b = M(w), Md @ w
        assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b)


@pytest.mark.parametrize("variant", ["tpu", "tup"])
def test_exact_factors_give_one_iteration(variant):
    """All faces open: H is block diagonal, so H~ = H; with the exact Schur
    complements S (Eq. Schur_1) or S2 (Eq. Schur2_2) the inexact LDU of
    Eq. LDU1/LDU2 is exact, M^-1 = J^-1, and FGMRES stops after one step."""
    P = fracgen.generate("planes64", N=4, p_stick=0.0, p_slip=0.0, seed=1)
    assert np.all(P.state == 2)
    J = osp.jacobian(P)
    if variant == "tpu":
        M = BlockPreconditioner(P, "tpu", "exact", "exact",
                                u_matrix=sp.csr_matrix(dense.schur_exact_tpu(P)))
    else:
        M = BlockPreconditioner(P, "tup", "exact", "exact",
                                p_matrix=sp.csr_matrix(dense.schur2_exact(P)))
    r = fgmres(lambda v: J @ v, M, P.b, tol=1e-10, maxit=20)
    assert r.iters == 1 and r.relres <= 1e-9


def test_incomplete_tup_with_exact_factors_is_unipotent():
    """Exact pieces (all faces open, exact S2): Q2 J Q2^T = L2 D2 U2, so
    M2*^-1 J = Q2^T U2 Q2 exactly.  With every face open C2 = 0, and U2 - I
    keeps only its (u, p) block S1^-1 Q1: E = M2*^-1 J - I is non-zero with
    E^2 = 0, so the minimal polynomial is (z - 1)^2 and GMRES stops after
    exactly two steps (the complete M2 takes one)."""
    P = fracgen.generate("planes64", N=4, p_stick=0.0, p_slip=0.0, seed=1)
    J = osp.jacobian(P)
    M = BlockPreconditioner(P, "tup_star", "exact", "exact",
                            p_matrix=sp.csr_matrix(dense.schur2_exact(P)))
    E = adjoint_operator(M, P.n) @ J.toarray() - np.eye(P.n)
    nu, nt = 3 * P.n_node, 3 * P.n_face
    # u and p carry different units: rescale u by the size of the (u, p)
    # block so that every block of E is dimensionless
    su = np.abs(E[:nu, nu + nt:]).max()
    assert su > 0
    d = np.ones(P.n)
    d[:nu] = su
    E = E / d[:, None] * d[None, :]
    off = E.copy()
    off[:nu, nu + nt:] = 0.0
    assert np.abs(off).max() <= 1e-10
    assert np.abs(E @ E).max() <= 1e-10
    r = fgmres(lambda v: J @ v, M, P.b, tol=1e-10, maxit=20)
    assert r.iters == 2 and r.relres <= 1e-9


def test_complete_tup_is_U2_inverse_times_incomplete(small_mixed):
    """M2^-1 = U2^-1 M2*^-1 (Eq. P2) with the AMG V-cycles as the inner
    S~1^-1 and S~2^-1: the two algorithms differ by exactly Eq. P2's first
    factor, built from the V-cycle operators column by column."""
    P = small_mixed
    opt = AmgOptions(coarse_max=20)
    Mc = BlockPreconditioner(P, "tup", opt=opt, opt_p=AmgOptions(coarse_max=8))
    Ms = BlockPreconditioner(P, "tup_star", opt=opt, opt_p=AmgOptions(coarse_max=8))
    nu = 3 * P.n_node
    S1i = adjoint_operator(Ms.u_inv, nu)
    S2 = np.linalg.inv(adjoint_operator(Ms.p_inv, P.n_face))
    U, _, _, Q = dense.m2_factors(P, S1_inv=S1i, S2_tilde=S2)
    rs = np.random.default_rng(9)
    for _ in range(3):
        w = rs.standard_normal(P.n)
        a, b = Mc(w), Q.T @ (U @ (Q @ Ms(w)))
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(a)


def test_prop31_unit_eigenvalues_tpu(small_mixed):
    """Prop. 3.1: M1^-1 J has the eigenvalue 1 with multiplicity >= n_p."""
    P = small_mixed
    J = osp.jacobian(P).toarray()
    ev = np.linalg.eigvals(dense.m1_matrix(P) @ J)
    assert np.sum(np.abs(ev - 1.0) < 1e-7) >= P.n_p


def test_S1_positive_definite_and_S2_symmetric(small_mixed):
    """S1 is positive definite in every state; S~2 is symmetric (Sec. 3.2)."""
    P = small_mixed
    S1 = schur.s1(P).toarray()
    assert np.linalg.eigvalsh(0.5 * (S1 + S1.T)).min() > 0
    S2 = schur.s2_tilde(P, schur.s1(P)).toarray()
    assert np.abs(S2 - S2.T).max() <= 1e-14 * np.abs(S2).max()


def test_fixed_stress_sign_and_bound():
    """With p^l = 0 the flux derivative F_u vanishes, Q2 = -Psi(Q1^T)/dt, and
    for S1 SPD the local diagonal of Eq. FS_algebraic is negative on open
    faces, zero elsewhere, and bounded by the exact diag(Q2 S1^-1 Q1):
    (S1_KK)^-1 <= (S1^-1)_KK in the Loewner order."""
    P = fracgen.generate("planes64", N=4, p_stick=0.7, p_slip=0.0, pl_scale=0.0, seed=3)
    S1 = schur.s1(P)
    assert abs(S1 - S1.T).max() <= 1e-12 * abs(S1).max()
    sk = schur.fixed_stress(P, S1)
    d = dense.blocks_dense(P)
    exact = np.diag(d["Q2"] @ np.linalg.solve(S1.toarray(), d["Q1"]))
    open_ = P.state == 2
    assert open_.any() and np.all(sk[open_] < 0) and np.all(sk[~open_] == 0)
    assert np.all(np.abs(sk[open_]) <= np.abs(exact[open_]) * (1 + 1e-12))


def test_fixed_stress_index_set_is_the_union():
    """Eq. FS_algebraic takes S1 on K = nz(Q1 column k) U nz(Q2 row k).
    With p^l != 0 the flux derivative F_u puts neighbouring open faces'
    copies into row k of Q2, so K2 = nz(Q2 row k) reaches beyond
    K1 = nz(Q1 column k) and K1 beyond K2 (a stick face next to an open
    one).  Zero every coupling of S1 between K and the rest: S1' is then
    block diagonal on (K, rest), Q1 column k lives on K1 and Q2 row k on
    K2, so (Q2 S1'^-1 Q1)_kk = Q2[k, K] S1[K, K]^-1 Q1[K, k] exactly, and
    the oracle's local diagonal on S1' must equal that dense product.  With
    K = K1 or K = K2 alone it does not."""
    P = fracgen.generate("planes64", N=4, p_stick=0.5, p_slip=0.2, seed=3)
    b = osp.blocks(P)
    Q1c, Q2r = b["Q1"].tocsc(), b["Q2"].tocsr()
    S1 = schur.s1(P, b).tolil()
    d = dense.blocks_dense(P)
    tested = 0
    for k in range(P.n_face):
        K1 = Q1c.indices[Q1c.indptr[k]:Q1c.indptr[k + 1]][Q1c.data[Q1c.indptr[k]:Q1c.indptr[k + 1]] != 0]
        K2 = Q2r.indices[Q2r.indptr[k]:Q2r.indptr[k + 1]][Q2r.data[Q2r.indptr[k]:Q2r.indptr[k + 1]] != 0]
        if np.setdiff1d(K1, K2).size == 0 or np.setdiff1d(K2, K1).size == 0:
            continue
        K = np.union1d(K1, K2)
        rest = np.setdiff1d(np.arange(S1.shape[0]), K)
        Sp = S1.tocsr().copy().tolil()
        for i in K:
            Sp[i, rest] = 0.0
            Sp[rest, i] = 0.0
        Sp = Sp.tocsr()
        Sp.eliminate_zeros()
        exact = d["Q2"][k] @ np.linalg.solve(Sp.toarray(), d["Q1"][:, k])
        got = schur.fixed_stress(P, Sp, b)[k]
        assert abs(got - exact) <= 1e-10 * abs(exact), (k, got, exact)
        # the same product over K1 or K2 alone misses part of it
        for part in (K1, K2):
            alt = d["Q2"][k, part] @ np.linalg.solve(Sp[part][:, part].toarray(), d["Q1"][part, k])
            assert abs(alt - exact) > 1e-6 * abs(exact)
        tested += 1
        if tested == 3:
            break
    assert tested == 3


def test_fgmres_identity_preconditioner_distinct_eigenvalues():
    """GMRES on a diagonal matrix with k distinct eigenvalues terminates in k
    steps (minimal polynomial of degree k)."""
    k = 5
    d = np.repeat(np.arange(1.0, k + 1), 40)
    b = np.random.default_rng(0).standard_normal(d.size)
    r = fgmres(lambda v: d * v, lambda v: v, b, tol=1e-13, maxit=50)
    assert r.iters == k
    assert np.linalg.norm(r.x - b / d) <= 1e-12 * np.linalg.norm(b / d)


def _parallel_mis2(W, keys):
    """The fixed-priority parallel rule: a node joins when its key is the
    largest among undecided nodes within distance 2; nodes within distance 2
    of a new root drop out."""
    n = W.shape[0]
    A = (W != 0).astype(int).tolil()
    A.setdiag(1)
    A = A.tocsr()
    deg = np.diff(W.indptr)
    und = deg > 0
    root = np.zeros(n, bool)
    kf = keys.astype(np.float64)
    while und.any():
        m1 = np.array([kf[A.indices[A.indptr[v]:A.indptr[v + 1]]][und[A.indices[A.indptr[v]:A.indptr[v + 1]]]].max()
                       if und[A.indices[A.indptr[v]:A.indptr[v + 1]]].any() else -1.0 for v in range(n)])
        m2 = np.array([m1[A.indices[A.indptr[v]:A.indptr[v + 1]]].max() for v in range(n)])
        new = und & (kf == m2)
        root |= new
        near = (A @ new.astype(int)) > 0
        near2 = (A @ near.astype(int)) > 0
        und &= ~near2
    return root


def test_mis2_greedy_equals_parallel_rule_and_is_maximal():
    rs = np.random.default_rng(11)
    for trial in range(4):
        n = 120
        M = sp.random(n, n, density=0.03, random_state=rs, format="csr")
        W = (M + M.T).tocsr()
        W.setdiag(0)
        W.eliminate_zeros()
        keys = oamg.priority_keys(n, trial, 0)
        # float64 keeps the order of these 64-bit keys: top bits are random
        assert len(np.unique(keys.astype(np.float64))) == n
        g = oamg.mis2_greedy(W, keys)
        p = _parallel_mis2(W, keys)
        assert np.array_equal(g, p)
        A = (W != 0).astype(int)
        A2 = ((A + A @ A) > 0).astype(int).tolil()
        A2.setdiag(0)
        A2 = A2.tocsr()
        r = np.nonzero(g)[0]
        assert A2[r][:, r].nnz == 0                      # distance >= 3 apart
        deg = np.diff(W.indptr)
        cover = (A2 @ g.astype(int) > 0) | g
        assert np.all(cover[deg > 0])                     # maximal


def test_aggregates_and_tentative_prolongator():
    P = fracgen.generate("planes64", N=6)
    S = schur.s1(P)
    W = oamg.strength_graph(S, 3, 0, AmgOptions())
    root = oamg.mis2_greedy(W, oamg.priority_keys(W.shape[0], 0, 0))
    agg, nc = oamg.aggregate(W, root)
    deg = np.diff(W.indptr)
    assert np.all(agg[deg > 0] >= 0) and np.all(agg[deg == 0] == -1)
    assert nc == root.sum()
    # every node is the root or a strong neighbour of a node assigned in round 1
    Pt = oamg.tentative(agg, nc, 3)
    assert np.allclose((Pt.T @ Pt).toarray(), np.eye(3 * nc), atol=1e-14)
    ones = np.tile([1.0, 0.0, 0.0], nc)
    v = Pt @ ones
    has = np.repeat(agg >= 0, 3)
    # piecewise constant per aggregate in the x component
    vx = v[0::3]
    for a in range(min(nc, 20)):
        vals = vx[agg == a]
        assert np.allclose(vals, vals[0])


def test_chebyshev_error_polynomial_closed_form():
    """Two Chebyshev steps on D^-1 S = diag(lam) from zero guess leave the
    error e = T_2((theta - lam)/delta) / T_2(theta/delta) * e0."""
    lam_true = np.linspace(0.05, 2.0, 30)
    S = sp.diags(lam_true).tocsr()
    a = AMG.__new__(AMG)
    a.opt = AmgOptions()
    L = oamg.Level(S=S, B=1, n=30, Dinv=np.ones((30, 1, 1)), lam=2.0)
    f = np.random.default_rng(2).standard_normal(30)
    x = a._cheb(L, f, None)
    e0 = f / lam_true
    e = e0 - x
    hi = 1.1 * 2.0
    lo = 0.1 * hi
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    T2 = lambda z: 2 * z * z - 1
    assert np.allclose(e, T2((theta - lam_true) / delta) / T2(theta / delta) * e0, rtol=1e-12, atol=1e-14)


def test_vcycle_symmetric_for_symmetric_operator():
    """With the same polynomial smoother before and after the correction and
    R = P^T, the V-cycle is a symmetric operator when S is symmetric."""
    P = fracgen.generate("planes64", N=8, p_stick=1.0, p_slip=0.0)
    S = schur.s1(P)
    amg = AMG(S, 3, AmgOptions(coarse_max=40))
    assert len(amg.levels) >= 2
    for L in amg.levels[1:]:
        assert abs(L.S - L.S.T).max() <= 1e-10 * abs(L.S).max()
    rs = np.random.default_rng(4)
    x, y = rs.standard_normal(S.shape[0]), rs.standard_normal(S.shape[0])
    assert np.isclose(x @ amg(y), y @ amg(x), rtol=1e-10)
    # and it reduces the error of the pure elasticity operator
    e = rs.standard_normal(S.shape[0])
    for _ in range(5):
        e = e - amg(S @ e)
    e2 = e - amg(S @ e)
    assert np.linalg.norm(e2) < 0.9 * np.linalg.norm(e)


def test_amg_numeric_rebuild_on_kept_aggregates():
    """The numeric rebuild (kept aggregates, new values): on the same S it is
    the original hierarchy; on 2 S every recomputed piece scales exactly
    (D^-1 halves, lambda, P and the tentative prolongator stay, the Galerkin
    operators and the coarsest solve double), so the V-cycle halves; a rebuild
    that kept any old value would not."""
    P = fracgen.generate("planes64", N=8, seed=3)
    S1 = schur.s1(P)
    opt = AmgOptions(coarse_max=20)
    a = AMG(S1, 3, opt)
    assert len(a.levels) >= 3
    same = AMG(S1, 3, opt, aggregates=a.aggregates())
    dbl = AMG((2.0 * S1).tocsr(), 3, opt, aggregates=a.aggregates())
    f = np.random.default_rng(4).standard_normal(S1.shape[0])
    x = a(f)
    assert np.array_equal(same(f), x)
    assert np.linalg.norm(2.0 * dbl(f) - x) <= 1e-14 * np.linalg.norm(x)
    for La, Ld in zip(a.levels[:-1], dbl.levels[:-1]):
        assert La.lam == pytest.approx(Ld.lam, rel=1e-13)
        assert abs(Ld.P - La.P).max() <= 1e-14 * abs(La.P).max()


def test_geometric_fixed_stress():
    """Eq. FS in the units of Q2 S1^-1 Q1: on a case whose only face
    coupling in Q2 is -Q1^T / dt (p^l = 0 removes F_u), the algebraic and
    geometric diagonals share sign and support, and agree within the order of
    magnitude their derivation allows (|Omega| / K against the local
    compliance seen through Q1); faces with a zero row of Q2 get 0."""
    P = fracgen.generate("planes64", N=8, seed=2, pl_scale=0.0)
    S1 = schur.s1(P)
    alg = schur.fixed_stress(P, S1)
    h = 1.0 / P.N
    omega = np.full(P.n_face, 2.0 * h ** 3)
    kbar = P.Ebar_face / (3.0 * (1.0 - 2.0 * P.nu))
    geo = schur.fixed_stress_geometric(P, omega, kbar, P.dt)
    open_ = P.state == 2
    assert np.array_equal(geo != 0, alg != 0) and np.array_equal(geo != 0, open_)
    assert np.all(geo[open_] < 0) and np.all(alg[open_] < 0)
    ratio = geo[open_] / alg[open_]
    assert 0.1 < np.median(ratio) < 10.0
    S2 = schur.s2_tilde(P, S1, sk=geo)
    assert np.abs(S2 - S2.T).max() <= 1e-14 * np.abs(S2).max()


@pytest.mark.parametrize("variant", ["tpu", "tup"])
def test_block_preconditioners_agree_with_block_jacobi_gmres(tiny, variant):
    """Both preconditioned solves reach the solution that GMRES with the plain
    block-Jacobi preconditioner of J reaches (3x3 node blocks of A, 3x3 face
    blocks of -H, the diagonal of T), in a small fraction of its iterations."""
    J = osp.jacobian(tiny)
    Jd = J.toarray()
    nu, nt = 3 * tiny.n_node, 3 * tiny.n_face
    groups = [np.arange(i, i + 3) for i in range(0, nu + nt, 3)]
    groups += [np.array([k]) for k in range(nu + nt, J.shape[0])]
    inv = [np.linalg.inv(Jd[np.ix_(g, g)]) for g in groups]

    def jacobi(v):
        out = np.empty_like(v)
        for g, Bi in zip(groups, inv):
            out[g] = Bi @ v[g]
        return out

    rj = fgmres(lambda v: J @ v, jacobi, tiny.b, tol=1e-12, maxit=1500)
    M = BlockPreconditioner(tiny, variant, opt=AmgOptions(coarse_max=64))
    rp = fgmres(lambda v: J @ v, M, tiny.b, tol=1e-12, maxit=300)
    xs = dense.solve(tiny)
    assert rj.relres <= 1e-9 and rp.relres <= 1e-9
    assert np.linalg.norm(rj.x - rp.x) <= 1e-10 * np.linalg.norm(xs)
    assert 4 * rp.iters < rj.iters


def test_smoothed_prolongator_lowers_energy_and_keeps_translations():
    """One damped-Jacobi smoothing step of P_tent (omega in (0, 2/lambda))
    lowers the energy trace(P^T S P) of every column of the SPD elasticity
    Schur complement, and keeps the rigid translations exactly on nodes whose
    rows of S annihilate them (interior nodes, all neighbours aggregated)."""
    P = fracgen.generate("planes64", N=6)
    S = schur.s1(P)
    amg = AMG(S, 3, AmgOptions(coarse_max=10))
    L = amg.levels[0]
    Pt = oamg.tentative(L.agg, L.nc, 3)
    e_t = np.einsum("ij,ij->j", Pt.toarray(), (S @ Pt).toarray())
    e_s = np.einsum("ij,ij->j", L.P.toarray(), (S @ L.P).toarray())
    assert np.all(e_s < e_t)
    size = np.bincount(L.agg[L.agg >= 0], minlength=L.nc).astype(float)
    for comp in range(3):
        c = np.zeros(3 * L.nc)
        c[comp::3] = np.sqrt(size)
        t = np.zeros(S.shape[0])
        t[comp::3] = 1.0
        St = S @ t
        rows = np.nonzero(np.abs(St) <= 1e-12 * abs(S).max())[0]
        rows = rows[np.repeat(L.agg >= 0, 3)[rows]]
        Sa = S[rows]
        keep = [r for k, r in enumerate(rows)
                if np.all(np.repeat(L.agg >= 0, 3)[Sa.indices[Sa.indptr[k]:Sa.indptr[k + 1]]])]
        assert len(keep) > 0
        assert np.allclose((L.P @ c)[keep], t[keep], atol=1e-12)


def test_power_estimate_of_the_jacobi_spectrum():
    """The power estimate of lambda_max(D^-1 S): on a diagonal operator with
    known eigenvalues it converges to the largest (gap ratio 0.9^15 after 15
    steps); on the elasticity Schur complement of a stick/slip/open case it
    lies below the spectral radius of D^-1 S (dense eigenvalues) and within
    10% of it."""
    lam = np.concatenate([np.linspace(0.1, 0.9, 40), [1.0]])
    S = sp.diags(lam).tocsr()
    est = oamg.power_lambda(S, np.ones((41, 1, 1)), 1, 0, AmgOptions())
    assert 0.9 < est <= 1.0 + 1e-14
    P = fracgen.generate("planes64", N=5)
    assert set(np.unique(P.state)) >= {1}
    S1 = schur.s1(P)
    D = oamg.diag_blocks(oamg.to_bsr(S1, 3), 3)
    Dinv = np.linalg.inv(D)
    est = oamg.power_lambda(S1, Dinv, 3, 0, AmgOptions())
    M = sp.block_diag(list(Dinv), format="csr") @ S1
    rho = np.abs(np.linalg.eigvals(M.toarray())).max()
    assert 0.9 * rho <= est <= rho * (1 + 1e-10)


def test_strength_graph_classic_cases():
    """Strength of connection, scalar case: the 1D Laplacian couples every
    neighbour with weight 1/4; the anisotropic 2D Laplacian -u_xx - eps u_yy
    keeps the y couplings only while eps^2 / (2 + 2 eps)^2 exceeds theta^2
    (theta0 = 0.08: eps = 0.1 weak, eps = 0.5 strong); the graph does not
    change under a symmetric positive diagonal scaling D S D."""
    n = 12
    L1 = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
    W = oamg.strength_graph(L1, 1, 0, AmgOptions())
    assert W.nnz == 2 * (n - 1)
    assert np.allclose(W.data, 0.25)
    m = 6
    I = sp.identity(m)
    T1 = sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1])
    for eps, strong_y in ((0.1, False), (0.5, True)):
        # -u_xx - eps u_yy on an m x m grid, x fastest; diagonal 2 + 2 eps
        Ax = sp.kron(I, T1)
        Ay = sp.kron(T1, I)
        A = (Ax + eps * Ay).tocsr()
        W = oamg.strength_graph(A, 1, 0, AmgOptions()).tocoo()
        dx = np.abs(W.row - W.col)
        assert np.all((dx == 1) | (dx == m))
        assert (dx == 1).sum() == 2 * m * (m - 1)
        assert ((dx == m).sum() > 0) == strong_y
    rs = np.random.default_rng(4)
    P = fracgen.generate("planes64", N=4, seed=2)
    S = schur.s1(P)
    d = np.repeat(rs.uniform(0.5, 2.0, S.shape[0] // 3), 3)
    Ds = sp.diags(d)
    W1 = oamg.strength_graph(S, 3, 0, AmgOptions())
    W2 = oamg.strength_graph((Ds @ S @ Ds).tocsr(), 3, 0, AmgOptions())
    assert (W1 != 0).toarray().tolist() == (W2 != 0).toarray().tolist()


def test_aggregates_are_rooted_balls_of_radius_two():
    """MIS-2 aggregation: every aggregate holds exactly one root, and each of
    its nodes is the root, a strong neighbour of it, or a strong neighbour of
    such a neighbour within the same aggregate (radius <= 2, connected)."""
    P = fracgen.generate("planes64", N=6)
    S = schur.s1(P)
    W = oamg.strength_graph(S, 3, 0, AmgOptions())
    root = oamg.mis2_greedy(W, oamg.priority_keys(W.shape[0], 0, 0))
    agg, nc = oamg.aggregate(W, root)
    roots = np.nonzero(root)[0]
    assert np.array_equal(np.sort(agg[roots]), np.arange(nc))
    for a in range(nc):
        members = np.nonzero(agg == a)[0]
        r = roots[agg[roots] == a]
        assert len(r) == 1
        r = r[0]
        nb1 = set(W.indices[W.indptr[r]:W.indptr[r + 1]]) & set(members)
        for i in members:
            if i == r or i in nb1:
                continue
            ni = set(W.indices[W.indptr[i]:W.indptr[i + 1]])
            assert ni & nb1, (a, i)


def test_stick_jacobian_is_a_symmetric_saddle_point(tiny):
    """All faces in stick: the (u, t) part [A C1; C2 -H] of the assembled J is
    symmetric (C2 = C1^T) with exactly n_u positive and n_t negative
    eigenvalues (Sylvester: A is SPD once the constrained dofs are removed, and
    the Schur complement -(H + C1^T A^-1 C1) is negative definite), which a
    wrong sign of H or a misplaced block would break."""
    assert np.all(tiny.state == 0)
    J = osp.jacobian(tiny)
    nu, nt = 3 * tiny.n_node, 3 * tiny.n_face
    K = J[:nu + nt, :nu + nt].toarray()
    assert np.abs(K - K.T).max() <= 1e-12 * np.abs(K).max()
    # inertia is kept by the congruence |diag K|^-1/2 K |diag K|^-1/2, which
    # brings the traction rows (~1e7 times the displacement scale) to O(1)
    d = 1.0 / np.sqrt(np.abs(np.diag(K)))
    ev = np.linalg.eigvalsh(K * d[:, None] * d[None, :])
    assert np.abs(ev).min() > 1e-3
    assert (ev > 0).sum() == nu and (ev < 0).sum() == nt
