"""Per-field comparison of vectors in the unknown order [u; t; p] of
Eq. JacSys.

The three fields live on very different scales: with b = U(-1, 1) in every
entry the tractions of a solution are 1e5-1e6 times the displacements (H is
of order h^3 / E, so H~^-1 is large), and the pressures sit in between.  A
relative difference of the whole vector is therefore a statement about t
alone.  Every parity check of a solution, a preconditioner application or an
adjoint compares the three blocks separately, each against its own norm:

    rel2(f)  = ||a_f - r_f|| / ||r_f||
    relmax(f) = max |a_f - r_f| / max |r_f|

A block whose reference is exactly zero is compared against the norm of the
whole reference vector instead (so a zero block must come out as zero to the
same relative accuracy).  Empty blocks (no fracture faces) are skipped.
"""
from __future__ import annotations

import numpy as np

FIELDS = ("u", "t", "p")


def split(n_node: int, n_face: int, v: np.ndarray):
    nu, nt = 3 * n_node, 3 * n_face
    return {"u": v[:nu], "t": v[nu:nu + nt], "p": v[nu + nt:nu + nt + n_face]}


def field_errors(P, got, ref) -> dict:
    """{field: (rel2, relmax)} for the u, t and p blocks of two vectors."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape == (3 * P.n_node + 4 * P.n_face,)
    whole = float(np.linalg.norm(ref))
    wmax = float(np.abs(ref).max()) if ref.size else 0.0
    g, r = split(P.n_node, P.n_face, got), split(P.n_node, P.n_face, ref)
    out = {}
    for f in FIELDS:
        if r[f].size == 0:
            continue
        d = g[f] - r[f]
        nr = float(np.linalg.norm(r[f]))
        mr = float(np.abs(r[f]).max())
        out[f] = (float(np.linalg.norm(d)) / (nr if nr > 0 else max(whole, 1e-300)),
                  float(np.abs(d).max()) / (mr if mr > 0 else max(wmax, 1e-300)))
    return out


def assert_fields(P, got, ref, tol: float, what: str = "") -> dict:
    """Assert rel2 <= tol and relmax <= tol on every non-empty field; returns
    the errors for reporting."""
    e = field_errors(P, got, ref)
    bad = {f: v for f, v in e.items() if not (v[0] <= tol and v[1] <= tol)}
    assert not bad, f"{what}: per-field errors above {tol:g}: " + ", ".join(
        f"{f} rel2 {v[0]:.2e} relmax {v[1]:.2e}" for f, v in e.items())
    return e
