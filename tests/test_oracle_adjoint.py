"""Pins of the oracle's adjoint: the transposed preconditioners and V-cycle
equal the transposes of the forward operators (built column by column), and
the adjoint FGMRES reaches the dense solution of J^T lambda = g; the gradient
of 0.5 ||p - p_obs||^2 with respect to b is lambda (central differences)."""
import numpy as np
import pytest

import fracgen
from oracle import adjoint, dense
from oracle import sparse as osp
from oracle.amg import AMG, AmgOptions
from oracle import schur
from oracle.fgmres import fgmres
from oracle.precond import BlockPreconditioner


@pytest.fixture(scope="module")
def small():
    return fracgen.generate("planes64", N=4, seed=2)


def test_transposed_vcycle_is_the_transpose(small):
    S1 = schur.s1(small)
    amg = AMG(S1, 3, AmgOptions(coarse_max=20))
    assert len(amg.levels) >= 2
    n = S1.shape[0]
    B = adjoint.operator_matrix(amg, n)
    Bt = adjoint.operator_matrix(amg.vcycle_t, n)
    assert np.abs(Bt - B.T).max() <= 1e-10 * np.abs(B).max()


@pytest.mark.parametrize("variant", ["tpu", "tup", "tup_star"])
@pytest.mark.parametrize("inner", ["amg", "exact"])
def test_transposed_preconditioner_is_the_transpose(small, variant, inner):
    M = BlockPreconditioner(small, variant, inner, inner, opt=AmgOptions(coarse_max=20),
                            opt_p=AmgOptions(coarse_max=8))
    Mt = adjoint.AdjointPreconditioner(M)
    n = small.n
    Md = adjoint.operator_matrix(M, n)
    Mtd = adjoint.operator_matrix(Mt, n)
    assert np.abs(Mtd - Md.T).max() <= 1e-9 * np.abs(Md).max()


@pytest.mark.parametrize("variant", ["tpu", "tup", "tup_star"])
def test_adjoint_solve_matches_dense(variant):
    P = fracgen.generate("tiny8")
    g = np.zeros(P.n)
    g[-P.n_face:] = np.random.default_rng(1).standard_normal(P.n_face)
    M = BlockPreconditioner(P, variant, opt=AmgOptions(coarse_max=64))
    r = adjoint.solve_adjoint(P, M, g, tol=1e-12, maxit=300)
    lam = adjoint.dense_adjoint(P, g)
    assert np.linalg.norm(r.x - lam) <= 1e-9 * np.linalg.norm(lam)


def test_gradient_wrt_rhs_by_central_differences():
    P = fracgen.generate("planes64", N=4, seed=5)
    J = osp.jacobian(P).toarray()
    b = P.b.copy()
    p_obs = np.random.default_rng(2).standard_normal(P.n_face)

    def loss(bb):
        x = np.linalg.solve(J, bb)
        return 0.5 * np.sum((x[-P.n_face:] - p_obs) ** 2)

    x = np.linalg.solve(J, b)
    g = np.zeros(P.n)
    g[-P.n_face:] = x[-P.n_face:] - p_obs
    lam = adjoint.dense_adjoint(P, g)
    rs = np.random.default_rng(3)
    for _ in range(5):
        d = rs.standard_normal(P.n)
        h = 1e-6
        fd = (loss(b + h * d) - loss(b - h * d)) / (2 * h)
        assert abs(fd - lam @ d) <= 1e-5 * abs(lam @ d)


def _phi(P, a, lam_p, x):
    """lambda_p^T (T(a) x_p + Q2(a) x_u) with the blocks regenerated at a."""
    Pa = fracgen.generate(P.cfg, aperture=a)
    b = osp.blocks(Pa)
    nu, nt = 3 * Pa.n_node, 3 * Pa.n_face
    return lam_p @ (b["T"] @ x[nu + nt:] + b["Q2"] @ x[:nu])


def test_aperture_derivative_entries_by_central_differences():
    """The generator's d T / d a and d Q2 / d a entries against central
    differences of the blocks regenerated at perturbed apertures."""
    P = fracgen.generate("planes64", N=6, p_stick=0.4, p_slip=0.2, seed=7)
    rs = np.random.default_rng(8)
    x = rs.standard_normal(P.n)
    lam = rs.standard_normal(P.n)
    lam_p = lam[-P.n_face:]
    g = -adjoint.aperture_gradient(P, x, lam)      # = lambda^T (dK/da) x per face
    for _ in range(4):
        d = rs.standard_normal(P.n_face) * P.aperture
        h = 1e-4
        fd = (_phi(P, P.aperture + h * d, lam_p, x) - _phi(P, P.aperture - h * d, lam_p, x)) / (2 * h)
        assert abs(fd - g @ d) <= 1e-6 * (abs(fd) + 1e-300)


def test_aperture_gradient_of_loss_dense():
    """dL/da for L = 0.5 ||p - p_obs||^2 by the adjoint formula against
    central differences of the dense solve (step 1e-6 relative)."""
    P = fracgen.generate("planes64", N=4, p_stick=0.4, p_slip=0.3, seed=9)
    p_obs = np.random.default_rng(1).standard_normal(P.n_face)

    def loss(a):
        Pa = fracgen.generate(P.cfg, aperture=a)
        x = np.linalg.solve(osp.jacobian(Pa).toarray(), Pa.b)
        return 0.5 * np.sum((x[-P.n_face:] - p_obs) ** 2), x

    L0, x = loss(P.aperture)
    gvec = np.zeros(P.n)
    gvec[-P.n_face:] = x[-P.n_face:] - p_obs
    lam = adjoint.dense_adjoint(P, gvec)
    grad = adjoint.aperture_gradient(P, x, lam)
    rs = np.random.default_rng(2)
    for _ in range(5):
        d = rs.standard_normal(P.n_face) * P.aperture
        h = 1e-6
        fd = (loss(P.aperture + h * d)[0] - loss(P.aperture - h * d)[0]) / (2 * h)
        assert abs(fd - grad @ d) <= 1e-5 * abs(grad @ d)
