"""The device generator (fc_generate) against the host generator of the test
suite: the same seeded instance, assembled independently.

* integer data (node split, face geometry and copies, contact states, roller
  dofs, every block's row pointers and columns) identical;
* block values within 1e-14 of each block's largest entry (the two sides sum
  the same terms in other orders and evaluate exp / log / cos in their own
  libraries);
* b identical (2 U - 1 from the same counter draws);
* a system set up from the device blocks solves like one set up from the
  host blocks (iterations equal, every field of x within 1e-10).
"""
import numpy as np
import pytest

import fracgen

from fields import assert_fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    # name: (preset, overrides, seed)
    "tiny8": ("tiny8", {}, 0),
    "planes8": ("planes64", dict(N=8), 0),
    "planes7_ragged": ("planes64", dict(N=7), 4),
    "rects16": ("rects128", dict(N=16), 0),
    "rects16_seed2": ("rects128", dict(N=16), 2),
    "rects12_many": ("rects128", dict(N=12, n_rect=25), 1),
    "network16": ("network96", dict(N=16, spacing=4), 0),
    "no_fractures": ("rects128", dict(N=10, n_rect=0), 0),
    "all_open": ("planes64", dict(N=6, p_stick=0.0, p_slip=0.0), 3),
    "all_slip_beta": ("planes64", dict(N=6, p_stick=0.0, p_slip=1.0, beta=0.5, k_scale=4.0), 5),
}


@pytest.fixture(scope="module")
def fs():
    import paper_2112_12397_gb300 as m
    m.load(build_if_missing=True)
    assert torch.cuda.is_available()
    return m


def host(t):
    return t.cpu().numpy()


def compare(P, inst, what):
    assert (inst.n_node, inst.n_face, inst.n) == (P.n_node, P.n_face, P.n), what
    assert np.array_equal(host(inst.field("node_grid")), P.node_grid), what
    assert np.array_equal(host(inst.field("face_geom")).reshape(-1, 4), P.face_geom.reshape(-1, 4)), what
    assert np.array_equal(host(inst.field("face_copies")).reshape(-1, 2, 4), P.face_copies.reshape(-1, 2, 4)), what
    assert np.array_equal(host(inst.field("state")), P.state), what
    assert np.array_equal(host(inst.field("dirichlet")).astype(bool), P.dirichlet.astype(bool).ravel()), what
    if P.n_face:
        a = host(inst.field("aperture"))
        assert np.max(np.abs(a - P.aperture) / P.aperture) <= 1e-15, what
        e = host(inst.field("ebar"))
        assert np.max(np.abs(e - P.Ebar_face) / P.Ebar_face) <= 1e-15, what
        assert np.array_equal(host(inst.field("pl")), P.pl), what
    for name, (rp, ci, val, nbr, nbc, br, bc) in inst.blocks().items():
        B = getattr(P, name)
        assert (nbr, nbc, br, bc) == (B.n_brows, B.n_bcols, B.br, B.bc), (what, name)
        assert np.array_equal(host(rp), B.row_ptr), (what, name, "row pointers")
        assert np.array_equal(host(ci), B.col_idx), (what, name, "columns")
        v = host(val).reshape(B.val.shape)
        scale = np.abs(B.val).max() if B.val.size else 0.0
        if scale > 0:
            err = np.abs(v - B.val).max() / scale
            assert err <= 1e-14, (what, name, err)
    assert np.array_equal(host(inst.b), P.b), what


@pytest.mark.parametrize("name", sorted(CASES))
def test_device_instance_equals_host_instance(fs, name):
    preset, over, seed = CASES[name]
    P = fracgen.generate(preset, seed=seed, **over)
    inst = fs.generate(preset, seed=seed, **over)
    compare(P, inst, name)
    inst.close()


def test_apertures_given_by_the_caller(fs):
    """Apertures passed in (a perturbed set, as for the adjoint workload's
    p_obs) give the host generator's instance for the same apertures; a
    count that does not match the layout is refused."""
    P0 = fracgen.generate("planes64", N=8, seed=1)
    a = P0.aperture * np.exp(0.1 * np.random.default_rng(3).standard_normal(P0.n_face))
    P = fracgen.generate("planes64", N=8, seed=1, aperture=a)
    inst = fs.generate("planes64", seed=1, N=8, aperture=torch.from_numpy(a))
    compare(P, inst, "apertures in")
    inst.close()
    with pytest.raises(fs.FcError) as e:
        fs.generate("planes64", seed=1, N=8, aperture=torch.from_numpy(a[:-1]))
    assert e.value.code == fs.FC_BAD_ARG


def test_bad_configurations_are_refused(fs):
    for over in (dict(N=1), dict(p_stick=0.8, p_slip=0.5), dict(layout=7)):
        with pytest.raises(fs.FcError) as e:
            fs.generate("planes64", **over)
        assert e.value.code == fs.FC_BAD_ARG
    with pytest.raises(fs.FcError):
        fs.generate("network96", N=16, spacing=0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_setup_from_device_instance_solves_like_host_blocks(fs, precision):
    P = fracgen.generate("rects128", N=16)
    inst = fs.generate("rects128", N=16)
    opt = dict(precision=precision, coarse_max=50, coarse_max_p=30)
    ch = fs.context_for(P, fs.default_options(**opt))
    cd = fs.Context(fs.default_options(**opt))
    cd.setup(inst.blocks(), inst.n_node, inst.n_face)
    b = torch.from_numpy(P.b).cuda()
    for variant in ("tpu", "tup"):
        xh, xd = torch.zeros_like(b), torch.zeros_like(b)
        _, ith, _ = ch.solve(variant, b, xh, 1e-8, 400)
        _, itd, rrd = cd.solve(variant, inst.b, xd, 1e-8, 400)
        assert ith == itd and rrd <= 1e-8
        assert_fields(P, host(xd), host(xh), 1e-10, f"{precision} {variant} x from device blocks")
    for c in (ch, cd):
        c.close()
    inst.close()


def test_full_size_rects128(fs):
    """The 128^3 bench instance (6.7M unknowns, 58M blocks of A): patterns
    identical and values within 1e-14, compared on the device."""
    P = fracgen.generate("rects128")
    inst = fs.generate("rects128")
    assert (inst.n_node, inst.n_face) == (P.n_node, P.n_face)
    for name, (rp, ci, val, nbr, nbc, br, bc) in inst.blocks().items():
        B = getattr(P, name)
        assert torch.equal(rp, torch.from_numpy(B.row_ptr).cuda()), name
        assert torch.equal(ci, torch.from_numpy(B.col_idx).cuda()), name
        ref = torch.from_numpy(np.ascontiguousarray(B.val).reshape(-1)).cuda()
        if ref.numel():
            assert float((val - ref).abs().max() / ref.abs().max()) <= 1e-14, name
    assert torch.equal(inst.b, torch.from_numpy(P.b).cuda())
    inst.close()
