"""The allocation-free K apply (eth_apply_k_dot_static) against the handle-based
entry point: the same y = K x (to the rounding of the element arithmetic) and
the fused <K x, x> of its own output, on two calls in a row (the shared static
scratch keeps the previous call's contents, which the entry point must not
depend on).

This file is collected last on purpose: callers that cannot allocate device
memory use this entry point, and a failure here should not hide the results
of the rest of the suite."""
import numpy as np
import pytest

from paper_2303_10233_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eth():
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_10233_gb300 import eth as E
    return E


@pytest.mark.parametrize("n", [16, 70])
@pytest.mark.parametrize("fp32", [False, True])
def test_static_scratch_apply_matches_handle_apply(eth, n, fp32):
    w = W.mms(n, seed=0, nu=0.7)
    G = eth.problem(w)
    rng = np.random.default_rng(100 + n)
    for call in range(2):
        x = torch.as_tensor(rng.standard_normal(G.nt), device="cuda")
        ref = G.apply("K", x, fp32=fp32)
        y = torch.empty_like(x)
        dot = torch.zeros(1, dtype=torch.float64, device="cuda")
        eth.apply_k_dot_static(n, w["nu"], x, y, dot, fp32=fp32)
        torch.cuda.synchronize()
        tol = 5e-5 if fp32 else 1e-13
        scale = float(torch.abs(ref).max())
        assert float(torch.abs(y - ref).max()) <= tol * scale
        # the fused dot is <K x, x> of this call's own output (FP64 products and sums)
        dref = float(torch.dot(y, x))
        assert abs(float(dot[0]) - dref) <= 1e-10 * max(1.0, float((y.abs() * x.abs()).sum()))
    G.close()


def test_static_scratch_rejects_oversize(eth):
    """Through the C ABI directly: n = 4096 needs more element tiles than the static
    scratch holds, and the entry point refuses it before touching the buffers."""
    import ctypes
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    L = eth.load()
    rc = L.eth_apply_k_dot_static(4096, -1.0, 1.0, -1.0, 1.0, 1.0, 0, p, p, p,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1 and b"static scratch" in L.eth_last_error()
    with pytest.raises(ValueError):   # the Python wrapper checks the tensor length first
        eth.apply_k_dot_static(16, 1.0, x, x, x)
