"""The C-ABI library builds, loads without a GPU and exports every symbol its
header declares; the binding refuses to run without CUDA (no CPU path)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fracsolve.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char|unsigned long long)\s*\*?\s*(fc_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2112_12397_gb300 import build as b
    path = b.build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("fc_create", "fc_setup", "fc_apply_prec", "fc_solve", "fc_destroy", "fc_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_binding_lists_every_declared_symbol():
    import paper_2112_12397_gb300 as fs
    assert sorted(fs.SYMBOLS) == declared_functions()


def test_host_only_entry_points(lib):
    import paper_2112_12397_gb300 as fs
    fs.load()
    o = fs.default_options()
    assert o.precision == fs.FC_FP64 and o.cheb_degree == 2 and o.coarse_max == 200
    assert abs(o.omega_num - 4.0 / 3.0) < 1e-15
    assert fs.load().fc_strerror(fs.FC_SINGULAR_BLOCK) == b"singular block"


def test_no_cpu_fallback():
    import torch
    import paper_2112_12397_gb300 as fs
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        fs.Context()


def test_create_without_device_reports_cuda_error(lib):
    import torch
    import paper_2112_12397_gb300 as fs
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    rc = fs.load().fc_create(C.byref(h), None, None)
    assert rc == fs.FC_CUDA_ERROR and not h.value
