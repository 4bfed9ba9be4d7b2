"""fc_update: numeric refresh of the setup for new block values on the same
patterns (the next Newton iteration with unchanged contact states, or new
apertures and current pressures, which change T and Q2).

The oracle's counterpart rebuilds every AMG hierarchy on the aggregates of
the first setup (``AMG(..., aggregates=...)``); with the GPU aggregates equal
to the oracle's (pinned elsewhere), preconditioner applications agree to
1e-10 and solves to the usual +-1 iteration / 1e-8 solution difference.
"""
import dataclasses

import numpy as np
import pytest

import fracgen
from oracle import schur
from oracle import sparse as osp
from oracle.amg import AMG, AmgOptions
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


def cuda(v):
    return torch.from_numpy(np.ascontiguousarray(v)).cuda()


def first_aggregates(P, opt, optp):
    """Aggregates of the four hierarchies of the first setup (oracle)."""
    blk = osp.blocks(P)
    S1 = schur.s1(P, blk)
    St = schur.s_tilde(P, blk, S1)
    S2 = schur.s2_tilde(P, S1, blk)
    return {"tpu": (AMG(St, 3, opt).aggregates(), AMG(blk["T"], 1, optp).aggregates()),
            "tup": (AMG(S1, 3, opt).aggregates(), AMG(S2, 1, optp).aggregates())}


def newton_pair():
    """A 16^3 ten-rectangle instance and the same mesh and states with new
    apertures and current pressures (T and Q2 change) and a stiffer A (S1
    changes too)."""
    P = fracgen.generate("rects128", N=16)
    a2 = P.aperture * np.exp(0.3 * np.random.default_rng(5).standard_normal(P.n_face))
    Q = fracgen.generate("rects128", N=16, aperture=a2, pl_scale=2.0)
    A = dataclasses.replace(Q.A, val=Q.A.val * 1.1)
    Q = dataclasses.replace(Q, A=A)
    return P, Q


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_update_with_identical_blocks_keeps_everything(fs, precision):
    P = fracgen.generate("rects128", N=16)
    ctx = fs.context_for(P, fs.default_options(precision=precision, coarse_max=CM, coarse_max_p=CMP))
    b = cuda(P.b)
    before = []
    for variant in ("tpu", "tup", "tup_star"):
        v = torch.zeros_like(b)
        ctx.apply_prec(variant, b, v)
        before.append(v.cpu().numpy())
    ctx.update(fs.device_blocks(P), P.n_node, P.n_face)
    for variant, v0 in zip(("tpu", "tup", "tup_star"), before):
        v = torch.zeros_like(b)
        ctx.apply_prec(variant, b, v)
        assert np.array_equal(v.cpu().numpy(), v0)
    ctx.close()


@pytest.mark.parametrize("variant", ["tpu", "tup", "tup_star"])
def test_update_matches_oracle_on_kept_aggregates(fs, variant):
    P, Q = newton_pair()
    opt, optp = AmgOptions(coarse_max=CM), AmgOptions(coarse_max=CMP)
    ctx = fs.context_for(P, fs.default_options(coarse_max=CM, coarse_max_p=CMP))
    ctx.update(fs.device_blocks(Q), Q.n_node, Q.n_face)
    aggs = first_aggregates(P, opt, optp)["tpu" if variant == "tpu" else "tup"]
    M = BlockPreconditioner(Q, variant, opt=opt, opt_p=optp, u_aggregates=aggs[0], p_aggregates=aggs[1])
    w = np.random.default_rng(2).standard_normal(Q.n)
    v = torch.zeros(Q.n, dtype=torch.float64, device="cuda")
    ctx.apply_prec(variant, cuda(w), v)
    assert_fields(Q, v.cpu().numpy(), M(w), 1e-10, f"update {variant} M^-1 w")
    J = osp.jacobian(Q)
    b = cuda(Q.b)
    x = torch.zeros_like(b)
    star = variant == "tup_star"
    rc, it, rr = ctx.solve(variant, b, x, 1e-8, 400, allow_fail=star)
    ref = fgmres(lambda q: J @ q, M, Q.b, 1e-8, 400)
    assert abs(it - ref.iters) <= 1
    assert_fields(Q, x.cpu().numpy(), ref.x, 1e-8, f"update {variant} x")
    true = np.linalg.norm(Q.b - J @ x.cpu().numpy()) / np.linalg.norm(Q.b)
    assert true <= (3e-8 if star else 1e-8)
    ctx.close()


def test_update_in_mixed_precision_reaches_tol_and_adjoint_follows(fs):
    P, Q = newton_pair()
    ctx = fs.context_for(P, fs.default_options(precision="mixed", coarse_max=CM, coarse_max_p=CMP))
    b = cuda(P.b)
    x = torch.zeros_like(b)
    ctx.solve("tup", b, x, 1e-8, 400)
    ctx.solve_adjoint("tup", b, x, 1e-8, 400)     # builds the transposed data
    ctx.update(fs.device_blocks(Q), Q.n_node, Q.n_face)
    J = osp.jacobian(Q)
    for variant in ("tpu", "tup"):
        bq = cuda(Q.b)
        xq = torch.zeros_like(bq)
        ctx.solve(variant, bq, xq, 1e-8, 400)
        assert np.linalg.norm(Q.b - J @ xq.cpu().numpy()) / np.linalg.norm(Q.b) <= 1e-8
        lam = torch.zeros_like(bq)
        ctx.solve_adjoint(variant, bq, lam, 1e-8, 400)
        assert np.linalg.norm(Q.b - J.T @ lam.cpu().numpy()) / np.linalg.norm(Q.b) <= 1e-8
    ctx.close()


def test_update_rejects_a_changed_pattern_and_stays_usable(fs):
    P = fracgen.generate("rects128", N=16)
    R = fracgen.generate("rects128", N=16, seed=3)          # other rectangles and states
    ctx = fs.context_for(P, fs.default_options(coarse_max=CM, coarse_max_p=CMP))
    if R.n_face == P.n_face and R.n_node == P.n_node:
        with pytest.raises(fs.FcError) as e:
            ctx.update(fs.device_blocks(R), R.n_node, R.n_face)
        assert e.value.code == fs.FC_BAD_ARG and "pattern" in str(e.value)
    else:
        with pytest.raises(fs.FcError) as e:
            ctx.update(fs.device_blocks(R), R.n_node, R.n_face)
        assert e.value.code == fs.FC_BAD_ARG
    b = cuda(P.b)
    x = torch.zeros_like(b)
    rc, it, rr = ctx.solve("tup", b, x, 1e-8, 400)
    assert rr <= 1e-8
    ctx.close()


def test_update_before_setup_is_refused(fs):
    P = fracgen.generate("tiny8")
    ctx = fs.Context(fs.default_options())
    with pytest.raises(fs.FcError) as e:
        ctx.update(fs.device_blocks(P), P.n_node, P.n_face)
    assert e.value.code == fs.FC_NOT_SETUP
    ctx.close()
