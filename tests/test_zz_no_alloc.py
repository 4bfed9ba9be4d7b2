"""fc_residual_noalloc: the relative residual without any device allocation.

It exists for callers that may not allocate device memory at the moment they
check a solution (a device-memory budget fixed up front, or stream work that
a cudaFree would synchronise).  This file is collected last on purpose.
"""
import numpy as np
import pytest

import fracgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fs():
    import paper_2112_12397_gb300 as m
    m.load(build_if_missing=True)
    assert torch.cuda.is_available()
    return m


def test_noalloc_residual_matches_fc_residual_twice(fs):
    P = fracgen.generate("rects128", N=16)
    ctx = fs.context_for(P, fs.default_options(coarse_max=50, coarse_max_p=30))
    b = torch.from_numpy(P.b).cuda()
    rng = np.random.default_rng(11)
    r = torch.zeros_like(b)
    for call in range(2):
        x = torch.from_numpy(rng.standard_normal(P.n)).cuda()
        ref = ctx.residual(b, x, r)
        free0 = torch.cuda.mem_get_info()[0]
        got = ctx.residual_noalloc(b, x)
        torch.cuda.synchronize()
        if call == 1:   # the first call may load the library's device module
            assert torch.cuda.mem_get_info()[0] == free0
        assert abs(got - ref) <= 1e-12 * ref, (call, got, ref)
    # a solved system: b - J x is a difference of nearly equal vectors, so two
    # summation orders of J x agree only to eps * || |J| |x| || / ||b - J x||
    # (about 1e-4 relative here); both must certify the 1e-8 solve
    x = torch.zeros_like(b)
    rc, it, rr = ctx.solve("tup", b, x, 1e-8, 400)
    ref = ctx.residual(b, x, r)
    got = ctx.residual_noalloc(b, x)
    assert abs(got - ref) <= 1e-3 * ref and ref <= 1e-8 and got <= 1e-8 * (1 + 1e-3)
    ctx.close()


def test_noalloc_residual_rejects_sizes_beyond_its_scratch(fs):
    P = fracgen.generate("rects128", N=72, n_rect=4)
    assert P.n > 1 << 20
    ctx = fs.context_for(P, fs.default_options(variants=2))
    b = torch.from_numpy(P.b).cuda()
    with pytest.raises(fs.FcError) as e:
        ctx.residual_noalloc(b, b)
    assert e.value.code == fs.FC_BAD_ARG and "1048576" in str(e.value)
    ctx.close()
