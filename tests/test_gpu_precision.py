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
1e-3, the mixed-storage target, measured 6.1e-4; BF16 (8-bit significand, each
stored value rounded by up to 2^-9 of itself every step) misses that target,
measured 1.5e-3, and is held to 2.5e-3 so that a regression still shows.

The same measurement on the first two benchmark workloads at their own
forces: config 1 (the 32^3 box above at |F_ext| = 1e-4, 1200 steps) and one box
of the orientation sweep (64^3, tau = 0.8, spheroid (8,4,4) at 45 degrees to
|F_ext| = 5e-4, 3000 steps, about three diffusion times L^2 / (4 pi^2 nu)),
where the spheroid moves and covers nodes.  Measured (means over the last 500
steps): FP32 2.3e-6 / 1.7e-5, FP16 2.5e-4 / 9.0e-4, BF16 9.8e-4 / 8.6e-3.  FP16
meets the mixed-storage target of 1e-3 on both (bar 1e-3); BF16 meets it on
config 1 only and is held to 1.5e-3 / 1.2e-2 so that a regression shows.  The
FP32 path is held to 3e-5 on the 3000-step run: the counter force spreads
|F_ext| / N = 2e-9 per node, whose per-population increments (~1e-11) lie a
few FP32 units in the last place below the stored deviations of the far field,
so their rounding is correlated between nodes of nearly equal deviations.

The second test is the squirmer batch of the benchmark's second workload
(2000 steps, the swimming velocity and flow field per storage format against
the oracle): there BF16 stays within 1e-3 on the velocity (5.8e-4)."""
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


_wref = {}


def _workload(name):
    from lb_inputs import sweep_8x64
    if name == "config1":
        boxes, parts = single_32(seed=0)
        return [boxes[0]], [parts[0]], 1200, 4
    boxes, parts = sweep_8x64(seed=0)
    return [boxes[3]], [parts[3]], 3000, 8


AVG = 500          # steady values: means over the last AVG steps, read every 25


def _mean_tail(step, read, steps):
    step(steps - AVG)
    acc = []
    for _ in range(AVG // 25):
        step(25)
        acc.append(read())
    return {k: np.mean([a[k] for a in acc], axis=0) for k in ("U", "Om", "T")}


def _workload_reference(name):
    if name not in _wref:
        boxes, parts, steps, _ = _workload(name)
        o = O.Sim(boxes[0], parts[0], nthreads=16)
        _wref[name] = _mean_tail(o.step, lambda: o.particle(0), steps)
    return _wref[name]


BARS = {("config1", L.LB_FP32): 1e-5, ("config2", L.LB_FP32): 3e-5,
        ("config1", L.LB_FP16): 1e-3, ("config2", L.LB_FP16): 1e-3,
        ("config1", L.LB_BF16): 1.5e-3, ("config2", L.LB_BF16): 1.2e-2}


@pytest.mark.parametrize("name", ["config1", "config2"])
@pytest.mark.parametrize("precision", [L.LB_FP32, L.LB_FP16, L.LB_BF16])
def test_drag_error_on_the_benchmark_workloads(name, precision):
    """Steady velocity and torque, averaged over the last 500 steps on both sides
    (a moving spheroid's drag jumps by 1e-3 of itself when it covers a node,
    and the two sides may cover one at steps a few apart)."""
    boxes, parts, steps, ms = _workload(name)
    sim = L.Simulation(boxes, parts, precision=precision, max_semi=ms)
    g = _mean_tail(sim.step, lambda: sim.particle(0, 0), steps)
    r = _workload_reference(name)
    sim.close()
    F = float(np.linalg.norm(parts[0][0]["F_ext"]))
    a = max(parts[0][0]["semi"])
    drag = float(np.linalg.norm(g["U"] - r["U"]) / np.linalg.norm(r["U"]))
    torque = float(np.linalg.norm(g["T"] - r["T"]) / (F * a))
    rot = float(np.linalg.norm(g["Om"] - r["Om"]) * a / np.linalg.norm(r["U"]))
    bar = BARS[(name, precision)]
    print(name, "storage", precision, "drag error", drag, "torque error", torque, "rotation error", rot)
    assert drag <= bar and torque <= bar and rot <= bar


def test_squirmer_batch_swimming_speed_and_flow_per_storage_format():
    """The 32-box squirmer batch (boxes of 48-128 nodes a side, squirmer (6,3,3),
    B1 = 1e-3, B2/B1 in {-2, 0, 2}, tau = 1) run for 2000 steps in FP32, FP16
    and BF16 storage; the swimming velocity and the flow field of the six 48^3
    boxes against the FP64 oracle, the velocities of all 32 boxes against FP32.
    A squirmer is force-free: its swimming speed is where a drag error shows.
    Bars (measured): velocity FP32 1e-5 (1.4e-7), FP16 1e-3 (3.5e-5), BF16
    1e-3 (5.8e-4); flow field normwise FP32 1e-5 (1.4e-6), FP16 1e-3 (1.6e-4),
    BF16 2.5e-2 (1.1e-2: the 8-bit significand shows in the slow far field)."""
    from lb_inputs import squirmer_batch
    boxes, parts = squirmer_batch(seed=0)
    steps = 2000
    small = [i for i, b in enumerate(boxes) if b["nx"] == 48]
    U, fields = {}, {}
    for prec in (L.LB_FP32, L.LB_FP16, L.LB_BF16):
        sim = L.Simulation(boxes, parts, precision=prec, max_semi=6)
        sim.step(steps)
        U[prec] = np.array([sim.particle(bi, 0)["U"] for bi in range(len(boxes))])
        fields[prec] = {bi: sim.field("u", bi) for bi in small}
        sim.close()
    Uo, fo = {}, {}
    for bi in small:
        o = O.Sim(boxes[bi], parts[bi], nthreads=16)
        o.step(steps)
        Uo[bi] = o.particle(0)["U"]
        fo[bi] = np.moveaxis(o.moments()[1], -1, 0)
    bars = {L.LB_FP32: (1e-5, 1e-5), L.LB_FP16: (1e-3, 1e-3), L.LB_BF16: (1e-3, 2.5e-2)}
    speed = np.linalg.norm(U[L.LB_FP32], axis=1)
    for prec, (bar_u, bar_f) in bars.items():
        du = max(float(np.linalg.norm(U[prec][bi] - Uo[bi]) / np.linalg.norm(Uo[bi])) for bi in small)
        dall = float((np.linalg.norm(U[prec] - U[L.LB_FP32], axis=1) / speed).max())
        df = max(float(np.abs(fields[prec][bi] - fo[bi]).max() / np.abs(fo[bi]).max()) for bi in small)
        print("storage", prec, "velocity vs oracle", du, "vs FP32 (all boxes)", dall, "flow field", df)
        assert du <= bar_u and dall <= max(bar_u, 1e-6) and df <= bar_f
