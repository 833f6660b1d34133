"""One time step of the 16-bit storage paths (FP16 with its power-of-two scale,
BF16) against the FP64 oracle started from the same stored distributions.

Both sides start from the populations the GPU holds (read back through
lb_get_fields, which reconstructs them independently of the kernels that
advance the run); the GPU then computes the step in FP32 and rounds every
stored population once to the storage format.  So each population after the
step is within one unit in the last place of that format of the oracle's FP64
value (2^-7 of its size for BF16's 8-bit significand, 2^-10 for FP16's 11-bit
one), plus FP32 round-off: 1e-6 of the largest deviation where the bulk tile
computes on deviations, 4e-7 rho0 within two nodes of a particle, where the
links, the remap and the momentum exchange work on whole populations (up to
rho0 / 3).  On a link the rounded value is the stored one and the read-back
adds the moving wall's term 6 w rho0 c.u_b to it, so next to a wall or a
particle the relative bound applies to |ref| + 6 w rho0 |u_b|.  A wrong shift, a wrong lane or row end, a wrong wall or particle
link moves a value by the size of a deviation and fails the bound by orders of
magnitude.

The field is random per node (no smoothness hides a neighbour mix-up); the
batch holds a periodic box whose rows do not line up with warps (nx = 40: five
8-node groups per row), with a moving particle and a squirmer, and two channels
with moving walls (the wall links are handled in the bulk tile), one of them
with rows that do line up with warps (nx = 32: the x wrap by shuffle)."""
import math

import numpy as np
import pytest

from lb_inputs import box, particle, random_quaternion, rng
from oracle import oracle as O
from parity_util import direction_map, oracle_df_gpu_layout

pytestmark = pytest.mark.gpu

L = pytest.importorskip("paper_2403_05443_gb300.lbsph")


def _case():
    g = rng(41)
    boxes = [box(40, 24, 32, 0.9, counter_force=1),
             box(24, 20, 16, 1.0, walls=1, wall_u_lo=(0.01, 0.0, 0.0), wall_u_hi=(-0.01, 0.0, 0.002)),
             box(32, 20, 24, 1.2, walls=1, wall_u_lo=(0.0, 0.0, 0.004), wall_u_hi=(0.008, 0.0, 0.0))]
    parts = [[particle((4.5, 2.5, 2.0), (10.3, 11.1, 9.7), random_quaternion(g), U=(0.01, -0.004, 0.002),
                       Om=(0.0, 0.001, -0.002), F_ext=(2e-4, -1e-4, 5e-5)),
              particle((3.0, 2.0, 2.0), (29.2, 12.6, 23.9), random_quaternion(g), U=(-0.005, 0.0, 0.006),
                       B1=1e-3, B2=2e-3)],
             [particle((3.0, 2.0, 2.0), (12.4, 9.8, 8.3), random_quaternion(g), U=(0.0, 0.003, -0.004))],
             [particle((3.5, 2.5, 2.0), (20.6, 10.3, 11.2), random_quaternion(g), U=(0.004, 0.002, 0.0))]]
    return boxes, parts


def _random_field(b, seed):
    g = np.random.default_rng(seed)
    shape = (b["nz"], b["ny"], b["nx"])
    return g.normal(0.0, 0.01, (3,) + shape), g.normal(0.0, 0.005, shape)


def _oracle_from_gpu(sim, bi, b, parts):
    """An oracle run whose pre-collision populations are the GPU's."""
    o = O.Sim(b, parts, nthreads=8)
    _sync(o, sim, bi, b)
    return o


def _sync(o, sim, bi, b):
    _, w = O.lattice()
    perm = direction_map()
    df = sim.field("df", bi)                                   # [19 gpu][nz][ny][nx]
    f = np.zeros((b["nz"], b["ny"], b["nx"], 19))
    f[..., perm] = np.moveaxis(df.astype(np.float64), 0, -1)
    f += w[None, None, None, :] * b["rho0"]
    f[o.owner() != 0] = 0.0
    o.set_f(f)


def _near_particles(owner, r=2):
    """Nodes within r nodes (per axis, periodically) of a particle's solid node."""
    near = owner > 0
    for ax in range(3):
        grown = near.copy()
        for s in range(1, r + 1):
            grown |= np.roll(near, s, axis=ax) | np.roll(near, -s, axis=ax)
        near = grown
    return near


def _check(sim, bi, o, b, rel, label):
    got = sim.field("df", bi).astype(np.float64)
    ref = oracle_df_gpu_layout(o, b["rho0"])
    err = np.abs(got - ref)
    near = _near_particles(o.owner())
    # largest bounce-back term: w <= 1/18 on links; |c.u_b| <= |u_b|_1, with
    # u_b = U + Omega x r + slip of the particles below 0.03
    uw = max(sum(abs(v) for v in b["wall_u_lo"]), sum(abs(v) for v in b["wall_u_hi"])) if b["walls"] else 0.0
    link = np.zeros(near.shape)
    link[near] = 6.0 / 18.0 * b["rho0"] * 0.03
    if b["walls"]:
        link[:, [1, b["ny"] - 2], :] = np.maximum(link[:, [1, b["ny"] - 2], :], 6.0 / 18.0 * b["rho0"] * uw)
    bound = rel * (np.abs(ref) + link[None]) + np.where(near, 4e-7 * b["rho0"], 1e-6 * np.abs(ref).max())[None]
    ratio = err / bound
    k = np.unravel_index(int(np.argmax(ratio)), err.shape)
    print(label, "max |err| / bound", float(ratio.max()), "at", k, "err", float(err[k]), "ref", float(ref[k]),
          "near", bool(near[k[1:]]), "bulk max", float(ratio[:, ~near].max()), "max |dev|", float(np.abs(ref).max()))
    assert float(ratio.max()) <= 1.0, (label, k)


@pytest.mark.parametrize("precision,rel", [(L.LB_FP16, 2.0 ** -10), (L.LB_BF16, 2.0 ** -7)])
def test_one_step_is_the_oracle_rounded_once(precision, rel):
    boxes, parts = _case()
    maxs = int(math.ceil(max(max(p["semi"]) for ps in parts for p in ps)))
    sim = L.Simulation(boxes, parts, precision=precision, max_semi=maxs)
    for bi, b in enumerate(boxes):
        u, d = _random_field(b, 100 + bi)
        sim.init_fluid(bi, u, d)
    orcs = [_oracle_from_gpu(sim, bi, b, parts[bi]) for bi, b in enumerate(boxes)]
    # the first step (collision of the stored initial field), then a streaming
    # step from the resynchronised populations
    for step in range(2):
        sim.step(1)
        for bi, b in enumerate(boxes):
            orcs[bi].step(1)
            _check(sim, bi, orcs[bi], b, rel, f"precision {precision} box {bi} step {step + 1}")
            _sync(orcs[bi], sim, bi, b)
