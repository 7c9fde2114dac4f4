"""Tile shapes of the fused K apply and the tile autotuner.

Every node sums its element contributions in one fixed order whatever the
tile, so K x is bitwise the same for tiles of 32 x 4, 32 x 8 and 32 x 16
elements and for the persistent pipelined 32 x 8 kernel; the fused dot
<Kx, x> agrees to rounding; a solve with the autotuner on reports the tile it
chose and reaches the tolerance like one with the default tile.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def eth():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_10233_gb300 import eth as E
    E.load()
    return E


@pytest.mark.parametrize("kind,n", [("stokes", 40), ("oseen", 66), ("stokes", 128)])
def test_apply_independent_of_tile(eth, kind, n):
    from paper_2303_10233_gb300 import workloads as W
    w = W.mms(n, seed=3) if kind == "stokes" else W.oseen_cavity(n, nu=1 / 50, seed=3)
    G = eth.problem(w)
    g = torch.Generator().manual_seed(5)
    x = torch.randn(G.nt, generator=g, dtype=torch.float64).cuda()
    ys = {}
    for rows, pers in ((4, False), (8, False), (16, False), (8, True)):
        G.set_tile(rows, pers)
        for fp32 in (True, False):
            ys[(rows, pers, fp32)] = G.apply("K", x, fp32=fp32)
    for fp32 in (True, False):
        for key in ((4, False), (16, False), (8, True)):
            assert torch.equal(ys[key + (fp32,)], ys[(8, False, fp32)]), (key, fp32)
    G.close()


@pytest.mark.parametrize("n", [30, 256])
def test_persistent_apply_and_solve(eth, n):
    """Persistent kernel: K x bitwise equal to the one-tile-per-CTA entry; MINRES converges with its fused dot."""
    from paper_2303_10233_gb300 import workloads as W
    w = W.mms(n, seed=2)
    G = eth.problem(w)
    g = torch.Generator().manual_seed(7)
    x = torch.randn(G.nt, generator=g, dtype=torch.float64).cuda()
    y0 = torch.empty_like(x); d0 = torch.zeros(1, dtype=torch.float64, device="cuda")
    eth.apply_k_dot_static(n, w["nu"], x, y0, d0, fp32=True)
    G.set_tile(8, True)
    u, p, st = G.solve(tol=1e-6, autotune=0)
    assert st["tile_persistent"] == 1 and st["status"] == 0
    y1 = G.apply("K", x, fp32=True)
    assert torch.equal(y0, y1)
    ref = float((y0 * x).sum())
    assert abs(float(d0) - ref) <= 1e-13 * float((y0 * x).abs().sum())
    G.close()


def test_set_tile_rejects(eth):
    G = eth.Grid(16)
    with pytest.raises(eth.EthError):
        G.set_tile(5)
    with pytest.raises(eth.EthError):
        G.set_tile(4, True)
    with pytest.raises(eth.EthError):
        G.set_tile(40, 2)
    G.set_tile(0)
    G.close()


def test_autotuned_solve(eth):
    from paper_2303_10233_gb300 import workloads as W
    w = W.mms(96, seed=1)
    G = eth.problem(w)
    u0, p0, st0 = G.solve(tol=1e-8, autotune=0)
    assert st0["tile_rows"] == 8 and st0["tile_persistent"] == 2   # default: warp strips of 8 element rows
    G.set_tile(0)
    u1, p1, st1 = G.solve(tol=1e-8, autotune=1)
    assert (st1["tile_rows"] in (4, 8, 16) and st1["tile_persistent"] in (0, 1)) or \
        (st1["tile_rows"] in (2, 4, 8, 16) and st1["tile_persistent"] == 2)
    assert st1["status"] == 0 and st1["relres_true"] <= 1e-8
    scale = float(torch.linalg.norm(u0))
    assert float(torch.linalg.norm(u1 - u0)) <= 1e-6 * scale
    G.close()
