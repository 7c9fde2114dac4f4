"""The seeded-input module's step and channel inputs (element mask and inflow data) follow
the oracle's Test problem 3 recipe (Sec. 3): D = [-1, 0) x [0, 1] U [0, 5] x [-1, 1] on
square elements of side 1/m, u = (4y(1 - y), 0) on the inflow edge; the channel
[0, 2] x [-1, 1] with u = (1 - y^2, 0)."""
import numpy as np
import pytest

from oracle import step
from paper_2303_10233_gb300 import workloads as W


@pytest.mark.parametrize("m", [1, 2, 4])
def test_step_inputs_match_oracle_recipe(m):
    w = W.step(m)
    g = step.step_grid(m)
    assert np.array_equal(w["active"], g.active)
    assert np.abs(w["ubc"] - step.step_inflow(g)).max() == 0.0
    wc = W.channel(m)
    gc = step.channel_grid(m, 2.0)
    assert np.array_equal(wc["active"], gc.active)
    assert np.abs(wc["ubc"] - step.inflow_data(gc, lambda y: 1.0 - y ** 2)).max() == 0.0
