"""Python binding of libfracsolve (include/fracsolve.h): argument marshalling only.

Every step of the solve runs in the CUDA library; this module converts torch
tensors and numpy arrays to the plain pointers and sizes of the C-ABI and
raises on non-zero status codes.  It fails loudly when the library or a CUDA
device is missing: there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libfracsolve.so")

FC_OK, FC_NOT_CONVERGED, FC_BREAKDOWN, FC_SINGULAR_BLOCK, FC_NAN, FC_BAD_ARG, \
    FC_CUDA_ERROR, FC_OOM, FC_INTERNAL, FC_NOT_SETUP = range(10)
FC_TPU, FC_TUP, FC_TUP_STAR = 0, 1, 2
FC_FP64, FC_MIXED = 0, 1
FC_H_TPU_U, FC_H_TPU_P, FC_H_TUP_U, FC_H_TUP_P = range(4)
FC_M_LEVEL, FC_M_PROLONG, FC_M_S1, FC_M_STILDE, FC_M_S2TILDE = range(5)
VARIANTS = {"tpu": FC_TPU, "tup": FC_TUP, "tup_star": FC_TUP_STAR}

# exported symbols declared by include/fracsolve.h
SYMBOLS = ["fc_default_gen_config", "fc_generate", "fc_generate_error", "fc_instance_free",
           "fc_default_options", "fc_create", "fc_setup", "fc_setup_host", "fc_update", "fc_set_geometric_fs", "fc_spmv", "fc_residual", "fc_residual_noalloc",
           "fc_apply_prec", "fc_solve", "fc_spmv_adjoint", "fc_apply_prec_adjoint", "fc_solve_adjoint",
           "fc_vcycle_adjoint", "fc_aperture_gradient",
           "fc_solve_host", "fc_num_levels", "fc_get_bsr", "fc_get_aggregates", "fc_vcycle",
           "fc_get_fixed_stress", "fc_krylov_basis", "fc_profile", "fc_kernel_stats", "fc_launch_count", "fc_destroy",
           "fc_strerror", "fc_last_error"]
(FC_K_SMOOTH0, FC_K_JAC, FC_K_CGS, FC_K_VCYCLE, FC_K_PREC, FC_K_RESID0, FC_K_RESTRICT0, FC_K_PROLONG0,
 FC_K_COARSE0, FC_K_VCYCLE_P) = range(10)


class FcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fracsolve status {code}: {msg}")
        self.code = code


class fc_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("variants", C.c_int32), ("theta0", C.c_double),
                ("theta_decay", C.c_double), ("coarse_max", C.c_int32), ("coarse_max_p", C.c_int32),
                ("max_levels", C.c_int32), ("max_ratio", C.c_double), ("power_steps", C.c_int32),
                ("omega_num", C.c_double), ("cheb_degree", C.c_int32), ("cheb_hi", C.c_double),
                ("cheb_lo", C.c_double), ("amg_seed", C.c_uint64), ("max_restarts", C.c_int32),
                ("verbose", C.c_int32), ("coarse_graphs", C.c_int32)]


class fc_bsr(C.Structure):
    _fields_ = [("n_brows", C.c_int32), ("n_bcols", C.c_int32), ("br", C.c_int32), ("bc", C.c_int32),
                ("nnzb", C.c_int64), ("d_row_ptr", C.c_void_p), ("d_col_idx", C.c_void_p),
                ("d_val", C.c_void_p)]


class fc_blocks(C.Structure):
    _fields_ = [("A", fc_bsr), ("C1", fc_bsr), ("Q1", fc_bsr), ("C2", fc_bsr), ("H", fc_bsr),
                ("Q2", fc_bsr), ("T", fc_bsr), ("n_node", C.c_int32), ("n_face", C.c_int32)]


LIB_HOOKS_PATH = os.path.join(_HERE, "lib", "libfracsolve_testhooks.so")

FC_GEN_PLANE_X, FC_GEN_PLANES_XYZ, FC_GEN_RECTS, FC_GEN_NETWORK = range(4)
# the four workload families by name: (layout, cells per side)
GEN_PRESETS = {"tiny8": (FC_GEN_PLANE_X, 8), "planes64": (FC_GEN_PLANES_XYZ, 64),
               "rects128": (FC_GEN_RECTS, 128), "network96": (FC_GEN_NETWORK, 96)}


class fc_gen_config(C.Structure):
    _fields_ = [("N", C.c_int32), ("layout", C.c_int32), ("n_rect", C.c_int32), ("spacing", C.c_int32),
                ("p_stick", C.c_double), ("p_slip", C.c_double), ("sigma_E", C.c_double),
                ("aperture_sigma", C.c_double), ("pl_scale", C.c_double), ("beta", C.c_double),
                ("k_scale", C.c_double), ("d_aperture", C.c_void_p), ("n_aperture", C.c_int32)]


class fc_instance(C.Structure):
    _fields_ = [("J", fc_blocks), ("d_b", C.c_void_p), ("n", C.c_int64), ("n_node", C.c_int32),
                ("n_face", C.c_int32), ("grid_n", C.c_int32), ("h", C.c_double), ("dt", C.c_double),
                ("nu", C.c_double), ("d_state", C.c_void_p), ("d_dirichlet", C.c_void_p),
                ("d_aperture", C.c_void_p), ("d_pl", C.c_void_p), ("d_ebar", C.c_void_p),
                ("d_face_geom", C.c_void_p), ("d_face_copies", C.c_void_p), ("d_node_grid", C.c_void_p),
                ("owner", C.c_void_p)]


_lib = None
_lib_hooks = None


def load(build_if_missing: bool = False):
    """Load the shared library (optionally building it first)."""
    global _lib
    if _lib is None:
        _lib = _open(LIB_PATH, build_if_missing)
    return _lib


def load_test_hooks():
    """The test build of the library: the same entry points, and it honours
    test variables read at setup that send small problems down the paths
    large ones take (FS_SPGEMM_FORCE_LONG: the SpGEMM's long-row and chunked
    kernels; FS_SELL_FORCE_JAG: jagged sliced ELL everywhere; FS_JAG_LANES:
    the lanes per row of the fused prolongation) or keep the prolongation and
    the first post-smoothing step apart (FS_FUSE_PROLONG=0).  Only tests use
    it."""
    global _lib_hooks
    if _lib_hooks is None:
        _lib_hooks = _open(LIB_HOOKS_PATH, False)
    return _lib_hooks


def _open(path: str, build_if_missing: bool):
    if not os.path.exists(path):
        if build_if_missing:
            from . import build as _b
            _b.build()
        else:
            raise FileNotFoundError(f"{path} is missing: run __graft_entry__.build() first")
    lib = C.CDLL(path)
    vp, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    pi32, pi64, pd, pint = C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_double), C.POINTER(C.c_int)
    sig = {
        "fc_default_gen_config": (None, [C.POINTER(fc_gen_config), C.c_int, C.c_int]),
        "fc_generate": (C.c_int, [C.POINTER(fc_gen_config), C.c_uint64, vp, C.POINTER(C.POINTER(fc_instance))]),
        "fc_generate_error": (C.c_char_p, []),
        "fc_instance_free": (None, [C.POINTER(fc_instance)]),
        "fc_default_options": (None, [C.POINTER(fc_options)]),
        "fc_create": (C.c_int, [C.POINTER(vp), C.POINTER(fc_options), vp]),
        "fc_setup": (C.c_int, [vp, C.POINTER(fc_blocks)]),
        "fc_setup_host": (C.c_int, [vp, C.POINTER(fc_blocks)]),
        "fc_update": (C.c_int, [vp, C.POINTER(fc_blocks)]),
        "fc_set_geometric_fs": (C.c_int, [vp, vp, vp, d]),
        "fc_spmv": (C.c_int, [vp, vp, vp]),
        "fc_residual": (C.c_int, [vp, vp, vp, vp, pd]),
        "fc_residual_noalloc": (C.c_int, [vp, vp, vp, pd]),
        "fc_apply_prec": (C.c_int, [vp, C.c_int, vp, vp]),
        "fc_solve": (C.c_int, [vp, C.c_int, vp, vp, d, C.c_int, pint, pd]),
        "fc_solve_host": (C.c_int, [vp, C.c_int, vp, vp, d, C.c_int, pint, pd]),
        "fc_spmv_adjoint": (C.c_int, [vp, vp, vp]),
        "fc_apply_prec_adjoint": (C.c_int, [vp, C.c_int, vp, vp]),
        "fc_solve_adjoint": (C.c_int, [vp, C.c_int, vp, vp, d, C.c_int, pint, pd]),
        "fc_vcycle_adjoint": (C.c_int, [vp, C.c_int, vp, vp]),
        "fc_aperture_gradient": (C.c_int, [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "fc_num_levels": (C.c_int, [vp, C.c_int, pint]),
        "fc_get_bsr": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, pi32, pi32, pi32, pi32, pi64, vp, vp, vp]),
        "fc_get_aggregates": (C.c_int, [vp, C.c_int, C.c_int, vp, pd]),
        "fc_vcycle": (C.c_int, [vp, C.c_int, vp, vp]),
        "fc_get_fixed_stress": (C.c_int, [vp, vp]),
        "fc_krylov_basis": (C.c_int, [vp, pint, vp]),
        "fc_profile": (C.c_int, [vp, C.c_int]),
        "fc_kernel_stats": (C.c_int, [vp, C.c_int, pi64, pd, pd]),
        "fc_launch_count": (C.c_ulonglong, []),
        "fc_destroy": (None, [vp]),
        "fc_strerror": (C.c_char_p, [C.c_int]),
        "fc_last_error": (C.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def variant_bit(variant: str) -> int:
    """The fc_options.variants bit whose setup a variant needs (the
    incomplete t-u-p form runs on the t-u-p setup)."""
    v = VARIANTS[variant]
    return 1 << (FC_TUP if v == FC_TUP_STAR else v)


def default_options(**over) -> fc_options:
    o = fc_options()
    load().fc_default_options(C.byref(o))
    for k, v in over.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": FC_FP64, "mixed": FC_MIXED}[v]
        setattr(o, k, v)
    return o


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _host_ptr(a) -> int:
    """Address of a contiguous host array (numpy or CPU tensor)."""
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return int(a.ctypes.data)
    assert a.device.type == "cpu" and a.is_contiguous()
    return int(a.data_ptr())


class Context:
    """One fc_ctx bound to the current CUDA device and a CUDA stream."""

    def __init__(self, options: fc_options | None = None, stream=None, lib=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("fracsolve needs a CUDA device; no CPU path exists")
        self.lib = lib or load()
        self.opt = options or default_options()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        self._check(self.lib.fc_create(C.byref(h), C.byref(self.opt), C.c_void_p(self.stream.cuda_stream)), None)
        self.h = h
        self._keep = None
        self.n = 0

    def _check(self, rc, h, ok=(FC_OK,)):
        if rc not in ok:
            msg = self.lib.fc_last_error(h).decode() if h else ""
            raise FcError(rc, (self.lib.fc_strerror(rc).decode() + (": " + msg if msg else "")))
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.fc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ setup
    @staticmethod
    def _blocks(blocks: dict, n_node: int, n_face: int) -> fc_blocks:
        J = fc_blocks()
        for name in ("A", "C1", "Q1", "C2", "H", "Q2", "T"):
            rp, ci, val, nbr, nbc, br, bc = blocks[name]
            m = getattr(J, name)
            m.n_brows, m.n_bcols, m.br, m.bc = nbr, nbc, br, bc
            m.nnzb = int(ci.numel())
            m.d_row_ptr, m.d_col_idx, m.d_val = _ptr(rp), _ptr(ci), _ptr(val)
        J.n_node, J.n_face = n_node, n_face
        return J

    def setup(self, blocks: dict, n_node: int, n_face: int):
        """blocks: name -> (row_ptr, col_idx, val, n_brows, n_bcols, br, bc) with
        int32/int32/float64 CUDA tensors."""
        J = self._blocks(blocks, n_node, n_face)
        self._check(self.lib.fc_setup(self.h, C.byref(J)), self.h)
        self.n = 3 * n_node + 4 * n_face
        self.n_node, self.n_face = n_node, n_face

    def setup_host(self, blocks: dict, n_node: int, n_face: int):
        """fc_setup_host: the same blocks dict with int32/int32/float64 CPU
        tensors or numpy arrays (pinned memory makes the copies
        asynchronous)."""
        J = fc_blocks()
        for name in ("A", "C1", "Q1", "C2", "H", "Q2", "T"):
            rp, ci, val, nbr, nbc, br, bc = blocks[name]
            m = getattr(J, name)
            m.n_brows, m.n_bcols, m.br, m.bc = nbr, nbc, br, bc
            m.nnzb = int(ci.numel() if hasattr(ci, "numel") else ci.size)
            m.d_row_ptr, m.d_col_idx, m.d_val = (_host_ptr(a) for a in (rp, ci, val))
        J.n_node, J.n_face = n_node, n_face
        self._check(self.lib.fc_setup_host(self.h, C.byref(J)), self.h)
        self.n = 3 * n_node + 4 * n_face
        self.n_node, self.n_face = n_node, n_face

    def update(self, blocks: dict, n_node: int, n_face: int):
        """fc_update: numeric refresh for new values on the patterns of the
        last setup."""
        J = self._blocks(blocks, n_node, n_face)
        self._check(self.lib.fc_update(self.h, C.byref(J)), self.h)
        self.n_node, self.n_face = n_node, n_face

    def set_geometric_fs(self, omega=None, kbar=None, dt: float = 0.0):
        """fc_set_geometric_fs: per-face cell volume and bulk modulus (CUDA
        float64 tensors) for the geometric fixed stress; None restores the
        algebraic form.  Takes effect at the next setup or update."""
        if omega is None:
            self._check(self.lib.fc_set_geometric_fs(self.h, None, None, 0.0), self.h)
        else:
            self._check(self.lib.fc_set_geometric_fs(self.h, _ptr(omega), _ptr(kbar), dt), self.h)

    # ------------------------------------------------------------ apply
    def spmv(self, x, y):
        self._check(self.lib.fc_spmv(self.h, _ptr(x), _ptr(y)), self.h)

    def residual(self, b, x, r) -> float:
        rr = C.c_double(0)
        self._check(self.lib.fc_residual(self.h, _ptr(b), _ptr(x), _ptr(r), C.byref(rr)), self.h)
        return rr.value

    def residual_noalloc(self, b, x) -> float:
        """Relative residual with no device allocation (library-held scratch,
        n <= 1048576); see fc_residual_noalloc."""
        rr = C.c_double(0)
        self._check(self.lib.fc_residual_noalloc(self.h, _ptr(b), _ptr(x), C.byref(rr)), self.h)
        return rr.value

    def apply_prec(self, variant: str, w, v):
        self._check(self.lib.fc_apply_prec(self.h, VARIANTS[variant], _ptr(w), _ptr(v)), self.h)

    def solve(self, variant: str, b, x, tol: float = 1e-8, maxit: int = 500, allow_fail: bool = False):
        it, rr = C.c_int(0), C.c_double(0)
        ok = (FC_OK, FC_NOT_CONVERGED, FC_BREAKDOWN) if allow_fail else (FC_OK,)
        rc = self._check(self.lib.fc_solve(self.h, VARIANTS[variant], _ptr(b), _ptr(x), tol, maxit,
                                           C.byref(it), C.byref(rr)), self.h, ok)
        return rc, it.value, rr.value

    def solve_host(self, variant: str, b: np.ndarray, x: np.ndarray, tol: float = 1e-8, maxit: int = 500,
                   allow_fail: bool = False):
        it, rr = C.c_int(0), C.c_double(0)
        ok = (FC_OK, FC_NOT_CONVERGED, FC_BREAKDOWN) if allow_fail else (FC_OK,)
        bp = b.ctypes.data if isinstance(b, np.ndarray) else b.data_ptr()
        xp = x.ctypes.data if isinstance(x, np.ndarray) else x.data_ptr()
        rc = self._check(self.lib.fc_solve_host(self.h, VARIANTS[variant], C.c_void_p(bp), C.c_void_p(xp), tol,
                                                maxit, C.byref(it), C.byref(rr)), self.h, ok)
        return rc, it.value, rr.value

    # ------------------------------------------------------------ adjoint
    def spmv_adjoint(self, x, y):
        self._check(self.lib.fc_spmv_adjoint(self.h, _ptr(x), _ptr(y)), self.h)

    def apply_prec_adjoint(self, variant: str, w, v):
        self._check(self.lib.fc_apply_prec_adjoint(self.h, VARIANTS[variant], _ptr(w), _ptr(v)), self.h)

    def solve_adjoint(self, variant: str, g, lam, tol: float = 1e-8, maxit: int = 500, allow_fail: bool = False):
        it, rr = C.c_int(0), C.c_double(0)
        ok = (FC_OK, FC_NOT_CONVERGED, FC_BREAKDOWN) if allow_fail else (FC_OK,)
        rc = self._check(self.lib.fc_solve_adjoint(self.h, VARIANTS[variant], _ptr(g), _ptr(lam), tol, maxit,
                                                   C.byref(it), C.byref(rr)), self.h, ok)
        return rc, it.value, rr.value

    def vcycle_adjoint(self, hier: int, f, x):
        self._check(self.lib.fc_vcycle_adjoint(self.h, hier, _ptr(f), _ptr(x)), self.h)

    def aperture_gradient(self, dk: dict, x, lam, grad):
        """dk: device tensors face_ptr (int64), block (int8), row, col (int32),
        comp (int8), val (float64); see fc_aperture_gradient."""
        self._check(self.lib.fc_aperture_gradient(
            self.h, _ptr(dk["face_ptr"]), _ptr(dk["block"]), _ptr(dk["row"]), _ptr(dk["col"]), _ptr(dk["comp"]),
            _ptr(dk["val"]), _ptr(x), _ptr(lam), _ptr(grad)), self.h)

    # ------------------------------------------------------------ inspection
    def num_levels(self, hier: int) -> int:
        n = C.c_int(0)
        self._check(self.lib.fc_num_levels(self.h, hier, C.byref(n)), self.h)
        return n.value

    def get_bsr(self, kind: int, hier: int = 0, level: int = 0):
        nbr, nbc, br, bc = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        nnz = C.c_int64()
        self._check(self.lib.fc_get_bsr(self.h, kind, hier, level, C.byref(nbr), C.byref(nbc), C.byref(br),
                                        C.byref(bc), C.byref(nnz), None, None, None), self.h)
        rp = np.zeros(nbr.value + 1, np.int32)
        ci = np.zeros(nnz.value, np.int32)
        val = np.zeros(nnz.value * br.value * bc.value, np.float64)
        self._check(self.lib.fc_get_bsr(self.h, kind, hier, level, None, None, None, None, None,
                                        C.c_void_p(rp.ctypes.data), C.c_void_p(ci.ctypes.data),
                                        C.c_void_p(val.ctypes.data)), self.h)
        return rp, ci, val.reshape(nnz.value, br.value, bc.value), (nbr.value, nbc.value, br.value, bc.value)

    def get_aggregates(self, hier: int, level: int, nb: int):
        agg = np.zeros(max(nb, 1), np.int32)
        lam = C.c_double(0)
        self._check(self.lib.fc_get_aggregates(self.h, hier, level, C.c_void_p(agg.ctypes.data), C.byref(lam)),
                    self.h)
        return agg[:nb], lam.value

    def vcycle(self, hier: int, f, x):
        self._check(self.lib.fc_vcycle(self.h, hier, _ptr(f), _ptr(x)), self.h)

    def krylov_basis(self):
        """The Arnoldi basis of the last FGMRES cycle as a (k, n) CUDA tensor."""
        import torch
        k = C.c_int(0)
        self._check(self.lib.fc_krylov_basis(self.h, C.byref(k), None), self.h)
        V = torch.empty((k.value, self.n), dtype=torch.float64, device="cuda")
        if k.value:
            self._check(self.lib.fc_krylov_basis(self.h, C.byref(k), _ptr(V)), self.h)
        return V

    def profile(self, enable: bool = True):
        self._check(self.lib.fc_profile(self.h, 1 if enable else 0), self.h)

    def kernel_stats(self, kernel: int):
        n, ms, b = C.c_int64(0), C.c_double(0), C.c_double(0)
        self._check(self.lib.fc_kernel_stats(self.h, kernel, C.byref(n), C.byref(ms), C.byref(b)), self.h)
        return n.value, ms.value, b.value

    def fixed_stress(self) -> np.ndarray:
        out = np.zeros(max(self.n_face, 1))
        self._check(self.lib.fc_get_fixed_stress(self.h, C.c_void_p(out.ctypes.data)), self.h)
        return out[:self.n_face]


def launch_count() -> int:
    return int(load().fc_launch_count())


def device_blocks(problem, device="cuda"):
    """Marshal a generated problem's numpy BSR blocks into CUDA tensors in the
    layout fc_setup expects."""
    import torch
    out = {}
    for name, B in problem.blocks().items():
        out[name] = (torch.from_numpy(B.row_ptr).to(device), torch.from_numpy(B.col_idx).to(device),
                     torch.from_numpy(np.ascontiguousarray(B.val).reshape(-1)).to(device),
                     B.n_brows, B.n_bcols, B.br, B.bc)
    return out


def device_dk(problem, device="cuda"):
    """Marshal a problem's aperture-derivative entries (sorted by face) and
    the per-face offsets into CUDA tensors."""
    import torch
    d = problem.dk
    fptr = np.zeros(problem.n_face + 1, dtype=np.int64)
    np.add.at(fptr, d["face"] + 1, 1)
    fptr = np.cumsum(fptr)
    return {"face_ptr": torch.from_numpy(fptr).to(device),
            **{k: torch.from_numpy(np.ascontiguousarray(d[k])).to(device)
               for k in ("block", "row", "col", "comp", "val")}}


def context_for(problem, options: fc_options | None = None, stream=None, lib=None) -> Context:
    ctx = Context(options, stream, lib)
    blocks = device_blocks(problem)
    ctx.setup(blocks, problem.n_node, problem.n_face)
    return ctx


# ------------------------------------------------------------------ device generator
class _DeviceArray:
    """A view of library-owned device memory for torch.as_tensor (no copy)."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr,
                                         "data": (int(ptr or 0), False), "version": 3}


_TYPESTR = {"i4": "<i4", "f8": "<f8", "i1": "|i1"}


def gen_config(preset: str, **over) -> fc_gen_config:
    """fc_gen_config of a workload family (tiny8, planes64, rects128,
    network96) with field overrides (N, p_stick, p_slip, sigma_E,
    aperture_sigma, pl_scale, n_rect, spacing, beta, k_scale)."""
    layout, N = GEN_PRESETS[preset]
    c = fc_gen_config()
    load().fc_default_gen_config(C.byref(c), layout, int(over.pop("N", N)))
    for k, v in over.items():
        setattr(c, k, v)
    return c


class Instance:
    """A seeded instance assembled on the device by fc_generate.  The blocks
    and vectors are torch views of memory the library owns; they stay valid
    until close()."""

    def __init__(self, cfg: fc_gen_config, seed: int = 0, stream=None, aperture=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("fc_generate needs a CUDA device; no CPU path exists")
        self.lib = load()
        self._aper = None
        if aperture is not None:
            self._aper = aperture.to(device="cuda", dtype=torch.float64).contiguous()
            cfg.d_aperture = self._aper.data_ptr()
            cfg.n_aperture = self._aper.numel()
        st = stream if stream is not None else torch.cuda.current_stream()
        p = C.POINTER(fc_instance)()
        rc = self.lib.fc_generate(C.byref(cfg), int(seed), C.c_void_p(st.cuda_stream), C.byref(p))
        if rc != FC_OK:
            raise FcError(rc, self.lib.fc_strerror(rc).decode() + ": " + self.lib.fc_generate_error().decode())
        self._p = p
        self.inst = p.contents
        self.n_node, self.n_face, self.n = self.inst.n_node, self.inst.n_face, self.inst.n
        self.h, self.dt, self.nu = self.inst.h, self.inst.dt, self.inst.nu

    def _view(self, ptr, n, t):
        import torch
        if n == 0:
            dt = {"i4": torch.int32, "f8": torch.float64, "i1": torch.int8}[t]
            return torch.zeros(0, dtype=dt, device="cuda")
        return torch.as_tensor(_DeviceArray(ptr, n, _TYPESTR[t]), device="cuda")

    def blocks(self) -> dict:
        """name -> (row_ptr, col_idx, val, n_brows, n_bcols, br, bc), the
        layout Context.setup takes."""
        out = {}
        for name in ("A", "C1", "Q1", "C2", "H", "Q2", "T"):
            m = getattr(self.inst.J, name)
            out[name] = (self._view(m.d_row_ptr, m.n_brows + 1, "i4"), self._view(m.d_col_idx, m.nnzb, "i4"),
                         self._view(m.d_val, m.nnzb * m.br * m.bc, "f8"), m.n_brows, m.n_bcols, m.br, m.bc)
        return out

    @property
    def b(self):
        return self._view(self.inst.d_b, self.n, "f8")

    def field(self, name: str):
        """Per-face or per-copy arrays: state, dirichlet, aperture, pl, ebar,
        face_geom (4 per face), face_copies (8 per face), node_grid."""
        nf, nn = self.n_face, self.n_node
        ptr, n, t = {"state": (self.inst.d_state, nf, "i1"), "dirichlet": (self.inst.d_dirichlet, 3 * nn, "i1"),
                     "aperture": (self.inst.d_aperture, nf, "f8"), "pl": (self.inst.d_pl, nf, "f8"),
                     "ebar": (self.inst.d_ebar, nf, "f8"), "face_geom": (self.inst.d_face_geom, 4 * nf, "i4"),
                     "face_copies": (self.inst.d_face_copies, 8 * nf, "i4"),
                     "node_grid": (self.inst.d_node_grid, nn, "i4")}[name]
        return self._view(ptr, n, t)

    def close(self):
        if getattr(self, "_p", None):
            self.lib.fc_instance_free(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def generate(preset: str, seed: int = 0, stream=None, aperture=None, **over) -> Instance:
    """fc_generate for a workload family with overrides (see gen_config)."""
    return Instance(gen_config(preset, **over), seed, stream, aperture)
