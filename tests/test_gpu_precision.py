"""16-bit storage of the distributions (deviations f_i - w_i rho0 in FP16
with a power-of-two scale, or BF16) against the FP64 oracle: the error of the
drag and torque after the flow around a sedimenting spheroid has developed.

Workload: 32^3 periodic box, tau = 1, spheroid (4, 2, 2) in a random pose,
F_ext = 1e-5 along x with the counter force (small enough that no node is
covered or uncovered in the run, so both sides follow the same geometry),
1200 steps (about 8 diffusion times of the box).  Errors at the end:
drag |U - U_ref| / |U_ref| (the drag coefficient F / U has the same relative
error) and torque |T - T_ref| / (|F_ext| a), a = 4 the long semi-axis.
Bars: FP32 1e-5 (the plain path's bar); FP16 (scale 2^14, 11-bit significand)
1e-3, the mixed-storage target, measured 6.2e-4; BF16 (8-bit significand, each
stored value rounded by up to 2^-9 of itself every step) misses that target,
measured 1.6e-3, and is held to 2.5e-3 so that a regression still shows."""
import math

import numpy as np
import pytest

from lb_inputs import single_32
from oracle import oracle as O

pytestmark = pytest.mark.gpu

L = pytest.importorskip("paper_2403_05443_gb300.lbsph")

STEPS = 1200
_ref = {}


def _reference():
    if not _ref:
        boxes, parts = single_32(seed=0, force=1e-5)
        o = O.Sim(boxes[0], parts[0], nthreads=8)
        o.step(STEPS)
        _ref.update(o.particle(0))
    return _ref


@pytest.mark.parametrize("precision,bar", [(L.LB_FP32, 1e-5), (L.LB_FP16, 1e-3), (L.LB_BF16, 2.5e-3)])
def test_drag_and_torque_error_of_the_storage_format(precision, bar):
    boxes, parts = single_32(seed=0, force=1e-5)
    sim = L.Simulation(boxes, parts, precision=precision, max_semi=4)
    sim.step(STEPS)
    g, r = sim.particle(0, 0), _reference()
    drag = float(np.linalg.norm(g["U"] - r["U"]) / np.linalg.norm(r["U"]))
    torque = float(np.linalg.norm(g["T"] - r["T"]) / (1e-5 * 4.0))
    print("storage", precision, "drag error", drag, "torque error", torque)
    assert drag <= bar and torque <= bar
