"""Host logic of the masked grids (no GPU): the node roles the CUDA library assigns on
the host equal the oracle's (Sec. 3, Test problem 3: Dirichlet walls and inflow, the
natural outflow edge without its two wall corners, inactive nodes fixed), on the step,
the channel, an enclosed full mask and a mask with a hole."""
import os

import numpy as np
import pytest

from oracle import step
from paper_2303_10233_gb300 import workloads as W

LIB = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2303_10233_gb300", "_lib", "libeth.so")
pytestmark = pytest.mark.skipif(not os.path.exists(LIB), reason="CUDA library not built")


def _check(w, x_out):
    from paper_2303_10233_gb300 import eth
    g = step.MaskedGrid(w["nx"], w["ny"], w["h"], w["x0"], w["y0"], w["active"], x_out=x_out)
    fx, dr, qa = eth.mask_roles(w["nx"], w["ny"], w["active"], outflow=x_out is not None)
    assert np.array_equal(fx, g.fixed)
    assert np.array_equal(dr, g.dirichlet)
    assert np.array_equal(qa, g.q1_active)


@pytest.mark.parametrize("m", [1, 2, 4])
def test_step_roles(m):
    w = W.step(m)
    _check(w, 5.0)


@pytest.mark.parametrize("m", [1, 3])
def test_channel_roles(m):
    w = W.channel(m)
    _check(w, 2.0)


def test_enclosed_and_holed_masks():
    n = 6
    act = np.ones((n, n), dtype=bool)
    _check({"nx": n, "ny": n, "h": 1.0 / 3, "x0": -1.0, "y0": -1.0, "active": act}, None)
    act[2:4, 1:3] = False      # an obstacle inside the channel
    _check({"nx": n, "ny": n, "h": 1.0 / 3, "x0": -1.0, "y0": -1.0, "active": act}, -1.0 + 6 / 3)


def test_bad_arguments_rejected():
    import ctypes
    from paper_2303_10233_gb300 import eth
    act = np.ones(4, dtype=np.uint8)
    L = eth.load()
    assert L.eth_mask_roles(0, 2, act.ctypes.data_as(ctypes.c_void_p), 1, None, None, None) == 1
    assert L.eth_mask_roles(2, 2, act.ctypes.data_as(ctypes.c_void_p), 2, None, None, None) == 1
    assert L.eth_mask_roles(2, 2, None, 1, None, None, None) == 1



def test_masked_grid_arguments_rejected_on_the_host():
    """eth_mgrid_create and the masked-grid calls reject bad arguments before any device
    work (the checks run on machines without a GPU)."""
    import ctypes
    from paper_2303_10233_gb300 import eth
    L = eth.load()
    act = np.ones(12, dtype=np.uint8)
    none = np.zeros(12, dtype=np.uint8)
    h = ctypes.c_void_p()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert L.eth_mgrid_create(0, 2, 0.5, 0.0, 0.0, p(act), 1, None, ctypes.byref(h)) == 1
    assert L.eth_mgrid_create(6, 2, -1.0, 0.0, 0.0, p(act), 1, None, ctypes.byref(h)) == 1
    assert L.eth_mgrid_create(6, 2, 0.5, 0.0, 0.0, p(act), 2, None, ctypes.byref(h)) == 1
    assert L.eth_mgrid_create(6, 2, 0.5, 0.0, 0.0, p(none), 1, None, ctypes.byref(h)) == 1
    assert L.eth_mgrid_create(6, 2, 0.5, 0.0, 0.0, None, 1, None, ctypes.byref(h)) == 1
    assert L.eth_mgrid_create(6, 2, 0.5, 0.0, 0.0, p(act), 1, None, None) == 1
    assert b"active" in L.eth_last_error() or b"NULL" in L.eth_last_error()
    assert L.eth_mgrid_apply(None, 0, None, None) == 1
    assert L.eth_mgrid_solve(None, None, None, None, None) == 1
    assert L.eth_mgrid_picard(None, None, None, 5, None, None, None, None) == 1
    assert L.eth_mgrid_sizes(None, None, None, None, None) == 1
