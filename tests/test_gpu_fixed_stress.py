"""Geometric fixed stress (Eq. FS) through fc_set_geometric_fs against the
oracle: the S~2 it builds, the t-u-p preconditioner on it, a solve, and the
switch back to the algebraic form (Eq. FS_algebraic)."""
import numpy as np
import pytest

import fracgen
from oracle import schur
from oracle import sparse as osp
from oracle.amg import AmgOptions
from oracle.fgmres import fgmres
from oracle.precond import BlockPreconditioner

from fields import assert_fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CM, CMP = 50, 30


@pytest.fixture(scope="module")
def fs():
    import paper_2112_12397_gb300 as m
    m.load(build_if_missing=True)
    assert torch.cuda.is_available()
    return m


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def geometry(P):
    h = 1.0 / P.N
    omega = np.full(P.n_face, 2.0 * h ** 3)
    kbar = P.Ebar_face / (3.0 * (1.0 - 2.0 * P.nu))
    return omega, kbar


def to_csr(rp, ci, val, shape):
    import scipy.sparse as sp
    nbr, nbc, br, bc = shape
    return sp.bsr_matrix((val, ci, rp), shape=(nbr * br, nbc * bc)).tocsr()


@pytest.mark.parametrize("name,over", [("rects128", dict(N=16)), ("network96", dict(N=16, spacing=4))])
def test_geometric_fixed_stress_matches_oracle(fs, name, over):
    P = fracgen.generate(name, **over)
    ctx = fs.context_for(P, fs.default_options(coarse_max=CM, coarse_max_p=CMP, variants=2))
    omega, kbar = geometry(P)
    ctx.set_geometric_fs(torch.from_numpy(omega).cuda(), torch.from_numpy(kbar).cuda(), P.dt)
    ctx.update(fs.device_blocks(P), P.n_node, P.n_face)
    sk = schur.fixed_stress_geometric(P, omega, kbar, P.dt)
    assert np.abs(ctx.fixed_stress() - sk).max() <= 1e-14 * np.abs(sk).max()
    S1 = schur.s1(P)
    S2 = schur.s2_tilde(P, S1, sk=sk)
    g = ctx.get_bsr(fs.FC_M_S2TILDE)
    got = to_csr(*g[:3], g[3])
    assert abs(got - S2).max() <= 1e-12 * abs(S2).max()
    # t-u-p with the geometric S~2: the update rebuilt its hierarchy on the
    # aggregates of the algebraic setup
    opt, optp = AmgOptions(coarse_max=CM), AmgOptions(coarse_max=CMP)
    from oracle.amg import AMG
    p_aggs = AMG(schur.s2_tilde(P, S1), 1, optp).aggregates()
    M = BlockPreconditioner(P, "tup", opt=opt, opt_p=optp, p_matrix=S2, p_aggregates=p_aggs)
    w = np.random.default_rng(6).standard_normal(P.n)
    v = torch.zeros(P.n, dtype=torch.float64, device="cuda")
    ctx.apply_prec("tup", torch.from_numpy(w).cuda(), v)
    assert_fields(P, v.cpu().numpy(), M(w), 1e-10, "geometric FS tup M^-1 w")
    J = osp.jacobian(P)
    b = torch.from_numpy(P.b).cuda()
    x = torch.zeros_like(b)
    rc, it, rr = ctx.solve("tup", b, x, 1e-8, 600, allow_fail=True)
    ref = fgmres(lambda q: J @ q, M, P.b, 1e-8, 600)
    assert abs(it - ref.iters) <= 1
    assert_fields(P, x.cpu().numpy(), ref.x, 1e-8, "geometric FS tup x")
    # back to the algebraic form
    ctx.set_geometric_fs(None)
    ctx.setup(fs.device_blocks(P), P.n_node, P.n_face)
    alg = schur.fixed_stress(P, S1)
    assert np.abs(ctx.fixed_stress() - alg).max() <= 1e-10 * np.abs(alg).max()
    ctx.close()


def test_geometric_fixed_stress_argument_checks(fs):
    P = fracgen.generate("tiny8")
    ctx = fs.Context(fs.default_options())
    om = torch.ones(P.n_face, dtype=torch.float64, device="cuda")
    with pytest.raises(fs.FcError) as e:
        ctx.set_geometric_fs(om, om, P.dt)          # before the first setup
    assert e.value.code == fs.FC_NOT_SETUP
    ctx.setup(fs.device_blocks(P), P.n_node, P.n_face)
    with pytest.raises(fs.FcError) as e:
        ctx.set_geometric_fs(om, om, 0.0)
    assert e.value.code == fs.FC_BAD_ARG
    ctx.close()
