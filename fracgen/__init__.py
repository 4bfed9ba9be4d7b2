"""Seeded synthetic inputs: the fractured-cube block Jacobian and right-hand side.

This package is the input recipe shared by the CPU oracle and the CUDA
library.  It holds no solver arithmetic.  The C source ``gen.c`` assembles the
blocks of the Jacobian ``[A C1 Q1; C2 -H 0; Q2 0 T]`` of Eq. JacSys /
Eq. block_def (Sec. 2) on an N^3 unit-cube hexahedral grid with conforming
planar fractures, a median-E0 lognormal Young's modulus field, seeded contact
states and seeded fracture data.

``generate(cfg)`` returns a :class:`Problem` whose blocks are plain numpy BSR
triples ``(row_ptr int32, col_idx int32, val float64[nnzb, br, bc])``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libfracgen.so")


def build(force: bool = False) -> str:
    """Compile gen.c into an in-tree shared library with the host compiler."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Cfg(C.Structure):
    _fields_ = [("N", C.c_int32), ("layout", C.c_int32), ("n_rect", C.c_int32),
                ("spacing", C.c_int32), ("p_stick", C.c_double), ("p_slip", C.c_double),
                ("sigma_E", C.c_double), ("aperture_sigma", C.c_double),
                ("seed", C.c_uint64), ("aperture_in", C.POINTER(C.c_double)),
                ("beta", C.c_double), ("k_scale", C.c_double), ("pl_scale", C.c_double)]


class _Bsr(C.Structure):
    _fields_ = [("n_brows", C.c_int32), ("n_bcols", C.c_int32), ("br", C.c_int32),
                ("bc", C.c_int32), ("nnzb", C.c_int64), ("row_ptr", C.POINTER(C.c_int32)),
                ("col_idx", C.POINTER(C.c_int32)), ("val", C.POINTER(C.c_double))]


class _Prob(C.Structure):
    _fields_ = [("N", C.c_int32), ("n_node", C.c_int32), ("n_face", C.c_int32),
                ("n_rect_eff", C.c_int32),
                ("h", C.c_double), ("dt", C.c_double), ("mu", C.c_double), ("E0", C.c_double),
                ("nu", C.c_double), ("C_f0", C.c_double), ("beta", C.c_double),
                ("tan_theta", C.c_double),
                ("A", _Bsr), ("C1", _Bsr), ("Q1", _Bsr), ("C2", _Bsr), ("H", _Bsr),
                ("Q2", _Bsr), ("T", _Bsr),
                ("b", C.POINTER(C.c_double)), ("state", C.POINTER(C.c_int8)),
                ("dirichlet", C.POINTER(C.c_int8)), ("node_grid", C.POINTER(C.c_int32)),
                ("face_geom", C.POINTER(C.c_int32)), ("face_copies", C.POINTER(C.c_int32)),
                ("aperture", C.POINTER(C.c_double)), ("pl", C.POINTER(C.c_double)),
                ("E_cell", C.POINTER(C.c_double)), ("Ebar_face", C.POINTER(C.c_double)),
                ("ups_face", C.POINTER(C.c_double)), ("rects", C.POINTER(C.c_int32)),
                ("rects_q1", C.POINTER(C.c_int32)),
                ("n_dk", C.c_int64), ("dk_face", C.POINTER(C.c_int32)), ("dk_row", C.POINTER(C.c_int32)),
                ("dk_col", C.POINTER(C.c_int32)), ("dk_block", C.POINTER(C.c_int8)),
                ("dk_comp", C.POINTER(C.c_int8)), ("dk_val", C.POINTER(C.c_double))]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.fg_generate.argtypes = [C.POINTER(_Cfg), C.POINTER(_Prob)]
        _lib.fg_generate.restype = C.c_int
        _lib.fg_free.argtypes = [C.POINTER(_Prob)]
        _lib.fg_rand_u64.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
        _lib.fg_rand_u64.restype = C.c_uint64
        _lib.fg_uniform.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
        _lib.fg_uniform.restype = C.c_double
        _lib.fg_normal.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
        _lib.fg_normal.restype = C.c_double
        _lib.fg_hex8_stiffness.argtypes = [C.c_double, C.POINTER(C.c_double)]
        _lib.fg_problem_size.restype = C.c_size_t
        _lib.fg_config_size.restype = C.c_size_t
        assert _lib.fg_problem_size() == C.sizeof(_Prob), "fg_problem layout mismatch"
        assert _lib.fg_config_size() == C.sizeof(_Cfg), "fg_config layout mismatch"
    return _lib


@dataclass
class Config:
    """Generator parameters.  ``layout``: 0 one x-plane at N/2, 1 three central
    planes, 2 ``n_rect`` seeded rectangles, 3 planes every ``spacing`` cells."""
    N: int
    layout: int
    p_stick: float
    p_slip: float
    sigma_E: float
    aperture_sigma: float
    n_rect: int = 0
    spacing: int = 0
    seed: int = 0
    name: str = ""
    beta: float = 0.0
    k_scale: float = 0.0
    pl_scale: float = 1.0


# Synthetic stand-ins for the paper's workloads (Sec. 4): unit cube, planar
# fractures, mixed contact states.
PRESETS = {
    # 8^3, one x-plane, all stick, sigma_E 0.5, aperture 1e-3 (~2.7k unknowns)
    "tiny8": Config(8, 0, 1.0, 0.0, 0.5, 0.0, name="tiny8"),
    # 64^3, three intersecting central planes, 60/30/10 (~0.91M unknowns)
    "planes64": Config(64, 1, 0.6, 0.3, 1.0, 0.5, name="planes64"),
    # 128^3, ten seeded rectangles, 60/30/10 (~6.6M unknowns)
    "rects128": Config(128, 2, 0.6, 0.3, 1.0, 0.5, n_rect=10, name="rects128"),
    # 96^3, planes every 8 cells on all axes, 50/40/10 (~5.0M unknowns)
    "network96": Config(96, 3, 0.5, 0.4, 1.0, 0.5, spacing=8, name="network96"),
}


def preset(name: str, **over) -> Config:
    c = PRESETS[name]
    d = dict(c.__dict__)
    d.update(over)
    return Config(**d)


@dataclass
class Bsr:
    n_brows: int
    n_bcols: int
    br: int
    bc: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray            # (nnzb, br, bc) float64

    @property
    def nnzb(self) -> int:
        return int(self.col_idx.shape[0])


@dataclass
class Problem:
    cfg: Config
    N: int
    h: float
    dt: float
    mu: float
    E0: float
    nu: float
    C_f0: float
    beta: float
    tan_theta: float
    n_node: int
    n_face: int
    A: Bsr
    C1: Bsr
    Q1: Bsr
    C2: Bsr
    H: Bsr
    Q2: Bsr
    T: Bsr
    b: np.ndarray
    state: np.ndarray
    dirichlet: np.ndarray
    node_grid: np.ndarray
    face_geom: np.ndarray
    face_copies: np.ndarray
    aperture: np.ndarray
    pl: np.ndarray
    E_cell: np.ndarray
    Ebar_face: np.ndarray
    ups_face: np.ndarray
    rects: np.ndarray
    dk: dict = field(default_factory=dict)      # derivative entries d K / d a_face
    extra: dict = field(default_factory=dict)

    @property
    def n_u(self) -> int:
        return 3 * self.n_node

    @property
    def n_t(self) -> int:
        return 3 * self.n_face

    @property
    def n_p(self) -> int:
        return self.n_face

    @property
    def n(self) -> int:
        return self.n_u + self.n_t + self.n_p

    def blocks(self):
        return dict(A=self.A, C1=self.C1, Q1=self.Q1, C2=self.C2, H=self.H, Q2=self.Q2, T=self.T)


def _arr(ptr, n, dtype):
    if n == 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


def _bsr(m: _Bsr) -> Bsr:
    nnzb = int(m.nnzb)
    rp = _arr(m.row_ptr, m.n_brows + 1, np.int32)
    ci = _arr(m.col_idx, nnzb, np.int32)
    val = _arr(m.val, nnzb * m.br * m.bc, np.float64).reshape(nnzb, m.br, m.bc)
    return Bsr(int(m.n_brows), int(m.n_bcols), int(m.br), int(m.bc), rp, ci, val)


def generate(cfg: Config | str, aperture: np.ndarray | None = None, **over) -> Problem:
    """Assemble one seeded instance.  ``aperture`` (n_face, metres) overrides
    the drawn apertures (used for perturbed-aperture and derivative runs)."""
    if isinstance(cfg, str):
        cfg = preset(cfg, **over)
    elif over:
        d = dict(cfg.__dict__)
        d.update(over)
        cfg = Config(**d)
    lib = _load()
    c = _Cfg(cfg.N, cfg.layout, cfg.n_rect, cfg.spacing, cfg.p_stick, cfg.p_slip,
             cfg.sigma_E, cfg.aperture_sigma, cfg.seed, None, cfg.beta, cfg.k_scale, cfg.pl_scale)
    keep = None
    if aperture is not None:
        keep = np.ascontiguousarray(aperture, dtype=np.float64)
        c.aperture_in = keep.ctypes.data_as(C.POINTER(C.c_double))
    p = _Prob()
    rc = lib.fg_generate(C.byref(c), C.byref(p))
    if rc != 0:
        raise ValueError(f"fg_generate failed for {cfg}")
    try:
        nn, nf = int(p.n_node), int(p.n_face)
        if keep is not None and keep.shape[0] != nf:
            raise ValueError(f"aperture has {keep.shape[0]} entries, expected {nf}")
        nfr = int(p.n_rect_eff)
        rects = np.zeros((nfr, 6), dtype=np.int32)
        if nfr:
            rects[:, :5] = _arr(p.rects, 5 * nfr, np.int32).reshape(nfr, 5)
            rects[:, 5] = _arr(p.rects_q1, nfr, np.int32)
        out = Problem(
            cfg=cfg, N=int(p.N), h=p.h, dt=p.dt, mu=p.mu, E0=p.E0, nu=p.nu, C_f0=p.C_f0,
            beta=p.beta, tan_theta=p.tan_theta, n_node=nn, n_face=nf,
            A=_bsr(p.A), C1=_bsr(p.C1), Q1=_bsr(p.Q1), C2=_bsr(p.C2), H=_bsr(p.H),
            Q2=_bsr(p.Q2), T=_bsr(p.T),
            b=_arr(p.b, 3 * nn + 4 * nf, np.float64),
            state=_arr(p.state, nf, np.int8),
            dirichlet=_arr(p.dirichlet, 3 * nn, np.int8).astype(bool),
            node_grid=_arr(p.node_grid, nn, np.int32),
            face_geom=_arr(p.face_geom, 4 * nf, np.int32).reshape(nf, 4),
            face_copies=_arr(p.face_copies, 8 * nf, np.int32).reshape(nf, 2, 4),
            aperture=_arr(p.aperture, nf, np.float64),
            pl=_arr(p.pl, nf, np.float64),
            E_cell=_arr(p.E_cell, cfg.N ** 3, np.float64),
            Ebar_face=_arr(p.Ebar_face, nf, np.float64),
            ups_face=_arr(p.ups_face, nf, np.float64),
            rects=rects,
            dk=dict(face=_arr(p.dk_face, int(p.n_dk), np.int32), block=_arr(p.dk_block, int(p.n_dk), np.int8),
                    row=_arr(p.dk_row, int(p.n_dk), np.int32), col=_arr(p.dk_col, int(p.n_dk), np.int32),
                    comp=_arr(p.dk_comp, int(p.n_dk), np.int8), val=_arr(p.dk_val, int(p.n_dk), np.float64)),
        )
    finally:
        lib.fg_free(C.byref(p))
    return out


def hex8_stiffness(nu: float) -> np.ndarray:
    """24x24 stiffness of the unit trilinear hexahedron with E = 1."""
    lib = _load()
    K = np.zeros(576, dtype=np.float64)
    lib.fg_hex8_stiffness(nu, K.ctypes.data_as(C.POINTER(C.c_double)))
    return K.reshape(24, 24)


def rand_u64(seed: int, stream: int, i: int) -> int:
    return int(_load().fg_rand_u64(seed, stream, i))


def uniform(seed: int, stream: int, i: int) -> float:
    return float(_load().fg_uniform(seed, stream, i))
