"""Host-side checks of the C ABI (no GPU compute): the library builds, loads
and exports every function that include/eth.h declares; argument validation
rejects bad input before touching the device."""
import ctypes

import pytest

from paper_2303_10233_gb300 import build as B
from paper_2303_10233_gb300 import eth


@pytest.fixture(scope="module")
def lib():
    B.build()
    return eth.load()


def test_exports_every_header_function(lib):
    names = eth.header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_sizes_and_defaults(lib):
    assert eth.sizes(16) == (1089, 289, 256, 2723)
    assert eth.sizes(256)[3] == 657923
    assert lib.eth_sizes(0, None, None, None) == -1
    o = eth.make_opts()
    assert o.tol == 1e-6 and o.restart == 50 and o.c_stage == 10.0


def test_create_rejects_bad_sizes_without_device(lib):
    h = ctypes.c_void_p()
    for n in (0, 1, 3, 9, 100000):
        rc = lib.eth_grid_create(n, -1.0, 1.0, -1.0, 1.0, 0, None, ctypes.byref(h))
        assert rc == 1 and not h.value
    rc = lib.eth_grid_create(8, 1.0, -1.0, -1.0, 1.0, 0, None, ctypes.byref(h))
    assert rc == 1
    assert b"empty domain" in lib.eth_last_error()
    assert lib.eth_set_coefficients(None, 1.0, None) == 1
    assert lib.eth_apply(None, 0, 0, None, None) == 1
    assert lib.eth_status_string(4) == b"not converged"


def _header_struct_fields(name):
    """Field names of `typedef struct { ... } name;` in include/eth.h, in order."""
    import re
    src = open(eth.HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", src)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        parts = decl.split(None, 1)
        fields += [f.strip() for f in parts[1].split(",")]
    return fields


@pytest.mark.parametrize("cname,pytype", [("eth_opts", "Opts"), ("eth_stats", "Stats")])
def test_binding_structs_match_header(cname, pytype):
    """The ctypes mirrors of eth_opts / eth_stats list the header's fields in order."""
    ours = [f for f, _ in getattr(eth, pytype)._fields_]
    assert ours == _header_struct_fields(cname)


class _FakeCuda:
    """Stand-in for a CUDA float64 tensor (no GPU here): what the binding's checks read."""

    def __init__(self, numel, device="cuda:0"):
        import torch
        self.is_cuda = True
        self.dtype = torch.float64
        self.device = torch.device(device)
        self._n = numel

    def is_contiguous(self):
        return True

    def numel(self):
        return self._n

    def data_ptr(self):
        return 0


def test_binding_checks_lengths_and_devices_before_the_call():
    """The C ABI takes raw pointers and cannot check lengths: the binding must refuse a
    short tensor or one on another device before calling into the library."""
    import torch
    nt = eth.sizes(16)[3]
    assert eth._ptr(_FakeCuda(nt), nt, torch.device("cuda:0")) is not None
    with pytest.raises(ValueError):
        eth._ptr(_FakeCuda(nt - 1), nt, torch.device("cuda:0"))
    with pytest.raises(ValueError):
        eth._ptr(_FakeCuda(nt, "cuda:1"), nt, torch.device("cuda:0"))
    with pytest.raises(TypeError):
        eth._ptr(torch.zeros(nt, dtype=torch.float64))          # host tensor
    with pytest.raises(ValueError):
        eth.apply_k_dot_static(16, 1.0, _FakeCuda(nt - 5), _FakeCuda(nt), _FakeCuda(1))
