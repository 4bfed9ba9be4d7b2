"""The per-field comparison used by the parity tests: it sees a relative
error confined to the displacements (or pressures) that a whole-vector norm,
dominated by the tractions, does not."""
import numpy as np
import pytest

import fracgen
from oracle import dense

from fields import assert_fields, field_errors


def test_field_errors_see_what_the_whole_norm_hides(tiny):
    xs = dense.solve(tiny)
    nu, nt = 3 * tiny.n_node, 3 * tiny.n_face
    u, t, p = xs[:nu], xs[nu:nu + nt], xs[nu + nt:]
    # the tractions dominate the norm of the exact solution by orders of
    # magnitude (b = U(-1, 1) in every entry)
    assert np.linalg.norm(t) > 1e4 * np.linalg.norm(u)
    for sl, f in ((slice(0, nu), "u"), (slice(nu + nt, None), "p")):
        y = xs.copy()
        y[sl] *= 1.0 + 5e-4
        assert np.linalg.norm(y - xs) / np.linalg.norm(xs) < 1e-8      # hidden in the whole norm
        e = field_errors(tiny, y, xs)
        assert abs(e[f][0] - 5e-4) < 1e-12 and abs(e[f][1] - 5e-4) < 1e-12
        with pytest.raises(AssertionError):
            assert_fields(tiny, y, xs, 1e-8)
    assert_fields(tiny, xs, xs, 0.0)


def test_zero_and_empty_fields():
    P = fracgen.generate("rects128", N=6, n_rect=0)
    assert P.n_face == 0
    x = np.random.default_rng(0).standard_normal(P.n)
    assert set(field_errors(P, x, x)) == {"u"}
    Q = fracgen.generate("tiny8")
    z = np.zeros(Q.n)
    z[0] = 1.0                                    # t and p references exactly zero
    y = z.copy()
    y[-1] = 1e-9                                  # judged against the whole norm
    e = field_errors(Q, y, z)
    assert e["t"] == (0.0, 0.0) and abs(e["p"][0] - 1e-9) < 1e-20
