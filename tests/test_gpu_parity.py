"""Parity of the CUDA path (called through the C ABI) with the FP64 CPU oracle.

Bars:
  * occupancy maps and boundary-link lists: bit-exact for the same FP64 pose
    (both sides evaluate Eq. ellipsoidsurface in the same FP64 operation order);
  * FP32 path: normwise relative error max|x - x_ref| / max|x_ref| <= 1e-5 per
    field and step for the deviations f_i - w_i rho0, u, F and T; the centre and
    the quaternion to 1e-5 of the distance travelled / angle turned (+1e-9).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from lb_inputs import (box, particle, rng, random_pose, random_quaternion, single_32, sweep_8x64,
                       axis_angle_quaternion)
from parity_util import gpu_links_as_set, normwise, oracle_df_gpu_layout, oracle_links_as_set

pytestmark = pytest.mark.gpu

L = pytest.importorskip("paper_2403_05443_gb300.lbsph")

TOL_FIELD = 1e-5
TOL_FT = 1e-5


def _sim(boxes, parts, **kw):
    ms = max([max(p["semi"]) for pl in parts for p in pl] + [1.0])
    return L.Simulation(boxes, parts, max_semi=int(math.ceil(ms)), **kw)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(12))
def test_solid_map_and_links_bit_exact(seed):
    g = rng(1000 + seed)
    n = [int(v) for v in g.choice([16, 20, 24, 32], size=3)]
    n[0] = 4 * (n[0] // 4)
    semi = [float(v) for v in g.uniform(1.5, 5.0, 3)]
    c, q = random_pose(g, min(n), margin=-1)       # anywhere: exercises periodic wrap
    b = box(*n, 1.0)
    p = particle(semi, c, q)
    gpu = _sim([b], [[p]])
    orc = O.Sim(b, [p], nthreads=4)
    solid = gpu.field("solid")
    assert np.array_equal(solid, orc.owner())
    assert gpu_links_as_set(gpu) == oracle_links_as_set(orc)


@pytest.mark.parametrize("seed", range(16))
def test_solid_map_bit_exact_for_thin_long_and_subnode_shapes(seed):
    """The occupancy map over a wider range of shapes: semi-axes from 0.6 to
    14 nodes with aspect ratios up to 12 (rows far from the body are skipped
    and the root bands are one node wide only when every semi-axis is at least
    one node; below that the wide bands), random poses anywhere in the box."""
    g = rng(1300 + seed)
    if seed % 4 == 3:
        semi = [float(v) for v in g.uniform(0.6, 1.0, 3)]
    else:
        a = float(g.uniform(3.0, 14.0))
        semi = [a, a / float(g.uniform(1.0, 12.0)), a / float(g.uniform(1.0, 12.0))]
        semi = [max(s_, 1.0) for s_ in semi]
    n = [int(v) for v in g.choice([40, 48], size=3)]          # the bounding cube (34 nodes at most) fits
    c, q = random_pose(g, min(n), margin=-1)
    b = box(*n, 1.0)
    p = particle(semi, c, q)
    gpu = _sim([b], [[p]])
    orc = O.Sim(b, [p], nthreads=4)
    assert np.array_equal(gpu.field("solid"), orc.owner())
    assert gpu_links_as_set(gpu) == oracle_links_as_set(orc)


@pytest.mark.parametrize("seed", range(4))
def test_links_bit_exact_for_a_quaternion_off_unit_norm(seed):
    """Both sides divide the input quaternion by its norm (Eq. vectrotn assumes
    |q| = 1), with the same FP64 operations: a pose given with |q| = 1 + 9e-7
    (inside the 1e-6 the library accepts) still gives identical solid nodes
    and links."""
    g = rng(1100 + seed)
    semi = [float(v) for v in g.uniform(2.0, 5.0, 3)]
    c, q = random_pose(g, 24, margin=-1)
    q = [v * (1.0 + 9e-7) for v in q]
    b = box(24, 24, 24, 1.0)
    p = particle(semi, c, q)
    gpu = _sim([b], [[p]])
    orc = O.Sim(b, [p], nthreads=4)
    assert np.array_equal(gpu.field("solid"), orc.owner())
    assert gpu_links_as_set(gpu) == oracle_links_as_set(orc)


def test_drag_matrix_matches_oracle():
    g = rng(5)
    b = box(32, 28, 36, 1.0)
    p = particle((5.5, 3.0, 2.5), (10.3, 20.7, 30.1), random_quaternion(g))
    gpu = _sim([b], [[p]])
    orc = O.Sim(b, [p], nthreads=4)
    Z, Zr = gpu.drag(), orc.zeta()
    assert np.abs(Z - Zr).max() <= 1e-12 * np.abs(Zr).max()


# ---------------------------------------------------------------------------
def _compare_run(boxes, parts, steps, every=1, tol_field=TOL_FIELD, tol_ft=TOL_FT, ft_scale="self", **kw):
    """Run the GPU and the oracle side by side, comparing every `every` steps.
    F and T are compared normwise against their own size (ft_scale "self") or,
    where the net force or torque is a small residual of its parts
    (F = F0 - zeta (U', Omega')), against the size of its parts (ft_scale
    "links"): the link sum F0 for the force, and for the torque the larger of
    T0 and F0 times the long semi-axis (the link forces' lever arm), whose
    round-off the residual carries."""
    gpu = _sim(boxes, parts, **kw)
    orcs = [O.Sim(b, pl, nthreads=8) for b, pl in zip(boxes, parts)]
    worst = {"df": 0.0, "u": 0.0, "F": 0.0, "T": 0.0, "x": 0.0, "q": 0.0}
    x0 = [[np.array(p["x"], float) for p in pl] for pl in parts]
    q0 = [[np.array(p.get("q", (1, 0, 0, 0)), float) for p in pl] for pl in parts]
    hist = {bi: {"F": [], "Fr": [], "T": [], "Tr": [], "F0r": [], "T0r": []} for bi in range(len(boxes))}
    done = 0
    while done < steps:
        k = min(every, steps - done)
        gpu.step(k)
        for o in orcs:
            o.step(k)
        done += k
        for bi, (b, o) in enumerate(zip(boxes, orcs)):
            df = gpu.field("df", bi)
            ref = oracle_df_gpu_layout(o, b.get("rho0", 1.0))
            worst["df"] = max(worst["df"], normwise(df, ref))
            _, ur = o.moments()
            u = gpu.field("u", bi)
            worst["u"] = max(worst["u"], normwise(u, np.moveaxis(ur, -1, 0)))
            for pi in range(len(parts[bi])):
                r = gpu.particle(bi, pi)
                s = o.particle(pi)
                hist[bi]["F"].append(r["F"]); hist[bi]["Fr"].append(s["F"])
                hist[bi]["T"].append(r["T"]); hist[bi]["Tr"].append(s["T"])
                hist[bi]["F0r"].append(s["F0"]); hist[bi]["T0r"].append(s["T0"])
                moved = float(np.abs(s["x"] - x0[bi][pi]).max())
                turned = 2.0 * math.acos(min(1.0, abs(float(s["q"] @ q0[bi][pi]))))
                worst["x"] = max(worst["x"], float(np.abs(r["x"] - s["x"]).max()) / (1e-5 * moved + 1e-9))
                worst["q"] = max(worst["q"], float(np.abs(r["q"] - s["q"]).max()) / (1e-5 * turned + 1e-9))
    for bi in hist:
        if hist[bi]["F"]:
            for q in ("F", "T"):
                got, ref = np.array(hist[bi][q]), np.array(hist[bi][q + "r"])
                if ft_scale == "links":
                    den = float(np.abs(np.array(hist[bi][q + "0r"])).max())
                    if q == "T":   # the link forces act at lever arms up to the long semi-axis
                        arm = max(max(p["semi"]) for p in parts[bi])
                        den = max(den, arm * float(np.abs(np.array(hist[bi]["F0r"])).max()))
                    worst[q] = max(worst[q], float(np.abs(got - ref).max()) / max(den, 1e-30))
                else:
                    worst[q] = max(worst[q], normwise(got, ref))
    print("parity", worst)
    assert worst["df"] <= tol_field and worst["u"] <= tol_field
    assert worst["F"] <= tol_ft and worst["T"] <= tol_ft
    assert worst["x"] <= 1.0 and worst["q"] <= 1.0       # in units of the bar above
    return gpu, orcs, worst


def test_single_spheroid_32_every_step():
    """32^3, tau = 1, spheroid (4,2,2), random pose, F_ext = 1e-4 with counter force:
    every field and particle value every step for 200 steps."""
    boxes, parts = single_32(seed=0)
    _compare_run(boxes, parts, steps=200, every=1)


@pytest.mark.parametrize("seed", [1, 2])
def test_single_spheroid_other_seeds(seed):
    boxes, parts = single_32(seed=seed)
    _compare_run(boxes, parts, steps=120, every=10)


def test_fast_particle_covers_and_uncovers_nodes():
    """A particle launched at |U| ~ 0.04 crosses nodes every few steps: the remap
    (covered / uncovered nodes, mass return) runs on both sides."""
    g = rng(9)
    b = box(24, 20, 28, 0.9)
    p = particle((4.5, 2.5, 2.0), (10.3, 9.1, 11.7), random_quaternion(g), U=(0.03, -0.02, 0.025),
                 Om=(0.004, 0.006, -0.005), density=5.0)
    _compare_run([b], [[p]], steps=60, every=3)


@pytest.mark.parametrize("didt_mode", [1, 2])
def test_inertia_rate_modes_spinning_triaxial_body(didt_mode):
    """The two other forms of I(t+1) in Eq. Tdiscrete: the finite difference
    (mode 1) and the predictor-corrector (mode 2: the solve is repeated with
    I of the predicted orientation), on a fast-spinning triaxial body under an
    external torque, which turns it by several degrees."""
    g = rng(13)
    b = box(24, 24, 28, 0.9, didt_mode=didt_mode)
    p = particle((5.5, 3.5, 2.5), (11.7, 12.2, 13.9), random_quaternion(g), Om=(0.004, -0.006, 0.008),
                 T_ext=(2e-3, 1e-3, -1.5e-3), density=3.0)
    _compare_run([b], [[p]], steps=60, every=6, didt_mode=didt_mode)


@pytest.mark.parametrize("semi", [(2.5, 5.0, 5.0), (5.5, 3.5, 2.0)])
def test_oblate_and_triaxial_bodies(semi):
    """An oblate spheroid (body x the short symmetry axis) and a triaxial
    ellipsoid (Sec. IV), settling and turning under a force and a torque."""
    g = rng(14)
    b = box(28, 28, 28, 1.0, counter_force=1)
    p = particle(semi, (13.6, 14.3, 13.2), random_quaternion(g), F_ext=(1e-3, -5e-4, 2e-4),
                 T_ext=(2e-3, 0.0, -1e-3))
    _compare_run([b], [[p]], steps=60, every=6)


def _close_pair(lub_cut):
    """A sphere and a spheroid pushed together from a gap of 0.89 lattice units
    (to 0.68 without, 0.72 with the lubrication correction): their bounding
    cubes overlap, nodes between them have links to both surfaces, and nodes
    are covered and uncovered next to both."""
    b = box(40, 32, 32, 0.9, counter_force=1, lub_cut=lub_cut)
    qB = axis_angle_quaternion((0.2, 0.3, 1.0), 0.15)
    pA = particle((3.5, 3.5, 3.5), (14.3, 15.8, 16.1), U=(0.01, 0, 0), F_ext=(3e-3, 0, 0), density=2.0)
    pB = particle((4.5, 2.5, 2.0), (23.15, 16.2, 15.9), qB, U=(-0.01, 0.001, 0), F_ext=(-3e-3, 5e-4, 0), density=2.0)
    return b, [pA, pB]


@pytest.mark.parametrize("lub_cut", [0.0, 1.0])
def test_close_particles_with_overlapping_cubes(lub_cut):
    """Multiple particles within reach of each other: the nodes
    between two bodies are updated once, with bounce-back on both surfaces, the
    remap and the momentum-exchange sums going to the body each link or node
    belongs to; with lub_cut > 0 the lubrication correction (Nguyen-Ladd, the
    squeeze force the lattice does not resolve below the cut-off gap) enters
    both solves.  Every field and particle value every 4 steps for 80 steps."""
    b, parts = _close_pair(lub_cut)
    _compare_run([b], [parts], steps=80, every=4)


def test_close_particles_links_and_owner_bit_exact():
    b, parts = _close_pair(1.0)
    gpu = _sim([b], [parts])
    orc = O.Sim(b, parts, nthreads=4)
    for k in range(3):
        assert np.array_equal(gpu.field("solid"), orc.owner())
        for p in range(2):
            assert gpu_links_as_set(gpu, 0, p) == oracle_links_as_set(orc, p)
        gpu.step(20)
        orc.step(20)


def test_cluster_of_three_particles():
    """A chain of three bodies within reach of each other: one cluster whose
    critical parts run one after the other once all its boundary work is done;
    a fourth particle far away stays on its own."""
    g = rng(15)
    b = box(56, 32, 36, 1.0, counter_force=1, lub_cut=2.0 / 3.0)
    parts = [particle((3.0, 3.0, 3.0), (10.2, 15.7, 17.9), F_ext=(2e-3, 0, 0), U=(0.008, 0, 0)),
             particle((4.0, 2.5, 2.5), (18.9, 16.3, 18.2), random_quaternion(g), U=(0.0, 0.004, 0)),
             particle((3.0, 3.0, 3.0), (27.6, 15.9, 18.3), F_ext=(-2e-3, 0, 0), U=(-0.008, 0, 0)),
             particle((2.5, 2.5, 2.5), (47.4, 16.1, 6.2), random_quaternion(g), F_ext=(0, 1e-3, 0))]
    _compare_run([b], [parts], steps=60, every=6)


@pytest.mark.parametrize("tau", [0.7, 1.3])
def test_ghost_mode_collision(tau):
    """The paper's collision (Sec. II.A: the non-equilibrium part projected on
    the hydrodynamic modes and relaxed with tau, ghost modes set to
    equilibrium; lb_options.collision = 1, FP32 storage) with a particle
    covering and uncovering nodes, a counter force and a moving wall: every
    field and particle value every 5 steps for 60 steps against the oracle's
    form of the same scheme."""
    g = rng(16)
    b = box(24, 22, 28, tau, counter_force=1, walls=1, wall_u_lo=(-0.005, 0, 0), wall_u_hi=(0.005, 0, 0.001),
            collision=1)
    p = particle((4.5, 2.5, 2.0), (11.3, 10.7, 13.9), random_quaternion(g), U=(0.02, -0.01, 0.015),
                 Om=(0.003, 0.004, -0.002), F_ext=(1e-3, 0, 0), density=3.0)
    _compare_run([b], [[p]], steps=60, every=5, collision=1)


def test_channel_walls_with_particle():
    """Moving walls (Couette) plus a free spheroid; nx = 20 is not a multiple of 128
    (rows shorter than a warp), ny not a power of two."""
    b = box(20, 22, 24, 1.0, walls=1, wall_u_lo=(-0.01, 0, 0), wall_u_hi=(0.01, 0.0, 0.002))
    p = particle((5.0, 2.5, 2.5), (10.2, 10.6, 12.3), axis_angle_quaternion((0.3, 0.2, 1.0), 0.7))
    _compare_run([b], [[p]], steps=80, every=8)


def test_squirmer():
    """A squirmer is force- and torque-free: its F and T are residuals of slip
    terms (Eq. squirmer) about 100 times larger, evaluated in FP32 on the GPU and
    in FP64 by the oracle, so the bar on F and T is 5e-5 of their own size."""
    b = box(28, 28, 28, 1.0)
    p = particle((6.0, 3.0, 3.0), (14.2, 13.9, 14.1), random_quaternion(rng(11)), B1=1e-3, B2=2e-3)
    _compare_run([b], [[p]], steps=60, every=6, tol_ft=5e-5)


def test_uneven_batch_of_boxes():
    """Three boxes of different shapes in one launch (ragged rows and tails),
    one of them empty of particles, one with two particles."""
    g = rng(12)
    boxes = [box(48, 20, 24, 0.8, counter_force=1), box(16, 36, 20, 1.2),
             box(36, 32, 28, 1.0, body_force=(1e-6, 0, -2e-6))]
    parts = [[particle((4.0, 2.0, 2.0), (20.5, 10.2, 12.1), random_quaternion(g), F_ext=(2e-4, 0, 0))],
             [],
             [particle((3.0, 3.0, 3.0), (8.3, 8.1, 7.7), random_quaternion(g), U=(0.01, 0, 0)),
              particle((4.0, 3.0, 2.0), (26.2, 22.9, 20.4), random_quaternion(g), F_ext=(0, 1e-4, 0))]]
    _compare_run(boxes, parts, steps=40, every=8)


def test_sweep_8x64_bench_workload_sampled():
    """The benchmark workload (8 boxes of 64^3, tau = 0.8, spheroid (8,4,4)) in the
    same launch configuration, checked against the oracle for its first steps."""
    boxes, parts = sweep_8x64(seed=0)
    _compare_run(boxes, parts, steps=6, every=3)


def test_squirmer_batch_bench_workload_sampled():
    """The 32-box batch the benchmark's second workload times (23.5 M nodes,
    boxes of 48-128 nodes a side, one squirmer each, tau = 1) in one launch,
    every field of every box and every particle against the oracle after 6 and
    12 steps.  A squirmer's net force and torque are residuals of its link sums
    (its torque is zero by symmetry up to the lattice's discreteness), so they
    are held to 1e-5 of the size of their parts (ft_scale "links").  Not
    earlier: in the first
    steps the flow is only the slip's first kick (deviations of a few 1e-4
    next to the surface), and the link arithmetic on whole populations (up to
    rho0 / 3, FP32 round-off of a few 1e-9) is then 1e-5 of the field."""
    from lb_inputs import squirmer_batch
    boxes, parts = squirmer_batch(seed=0)
    _compare_run(boxes, parts, steps=12, every=6, ft_scale="links")


def test_largest_particle_the_bounding_cube_allows():
    """Semi-axis 29, the largest lb_create accepts: h = 31, cube side
    S = 2h + 2 = 64, one full 64-bit word per cube row; the box is just as
    large in y and z; random pose."""
    g = rng(14)
    b = box(68, 64, 64, 0.9, counter_force=1)
    p = particle((29.0, 9.0, 8.5), (33.7, 31.2, 32.9), random_quaternion(g), F_ext=(1e-4, -5e-5, 2e-5))
    # no external torque: the net torque is a residual of the link torque
    _compare_run([b], [[p]], steps=6, every=3, ft_scale="links")


def test_fields_before_first_step_are_rest_state():
    boxes, parts = single_32(seed=3)
    gpu = _sim(boxes, parts)
    f = gpu.field("f")
    _, w = L.lb_lattice()
    solid = gpu.field("solid") != 0
    fl = ~solid
    assert np.allclose(f[:, fl], w[:, None].astype(np.float32), rtol=0, atol=0)
    assert (f[:, solid] == 0).all()


def test_runs_are_bitwise_reproducible_and_step_kernel_matches_separate_kernels():
    # integer accumulators make every schedule of the same compiled code
    # bitwise reproducible; the persistent step kernel and the separate kernels
    # are two compilations of the same source, which may contract a * b + c
    # differently, so they agree to FP32 round-off
    boxes, parts = single_32(seed=4)
    outs = []
    for separate in (False, False, True, True):
        g = _sim(boxes, parts, separate_kernels=separate)
        g.step(70)
        outs.append((g.field("df"), g.records()))
    for a, b in ((0, 1), (2, 3)):
        assert np.array_equal(outs[a][0], outs[b][0]) and np.array_equal(outs[a][1], outs[b][1])
    assert normwise(outs[0][0], outs[2][0].astype(np.float64)) < 1e-5
    assert np.abs(outs[0][1] - outs[2][1]).max() <= 1e-6 * max(1.0, np.abs(outs[2][1]).max())


def test_invalid_particles_rejected():
    b = box(32, 32, 32, 1.0)
    with pytest.raises(L.LBError):
        _sim([b], [[particle((40.0, 2.0, 2.0), (16, 16, 16))]])   # larger than max_semi / the box
    with pytest.raises(L.LBError):
        _sim([b], [[particle((4.0, 2.0, 2.0), (16, 16, 16), q=(1.0, 1.0, 0.0, 0.0))]])
    g = L.Simulation([b], [[particle((4.0, 2.0, 2.0), (16, 16, 16))]], max_semi=8)
    g.step(1)
    with pytest.raises(L.LBError) as e:
        g.set_particles(0, [particle((4.0, 2.0, 2.0), (16, 16, 16))])
    assert e.value.status == 8


def test_autotune_keeps_results_bitwise_and_picks_a_candidate():
    """The launch-shape candidates (blocks per particle, units per fetch)
    compute the same values bit for bit, so a tuned run equals an untuned run
    of the same number of steps."""
    boxes = [box(48, 20, 24, 0.8, counter_force=1), box(32, 36, 20, 1.2)]
    g = rng(21)
    parts = [[particle((4.0, 2.0, 2.0), (20.5, 10.2, 12.1), random_quaternion(g), F_ext=(2e-4, 0, 0))],
             [particle((3.0, 2.5, 2.0), (15.3, 18.1, 9.7), random_quaternion(g), F_ext=(0, 1e-4, 0))]]
    a = _sim(boxes, parts)
    (fetch, gx, advanced), ms = L.lb_autotune(a.ctx, 5)
    assert fetch in (1, 2, 4, 8) and gx >= 1 and np.all(ms[6:] > 0) and ms[3] > 0
    a.step(9)
    b = _sim(boxes, parts)
    b.step(advanced + 9)
    for bi in range(2):
        assert np.array_equal(a.field("df", bi), b.field("df", bi))
        assert np.array_equal(a.records(bi), b.records(bi))


def test_autotune_with_large_particles_keeps_results_bitwise():
    """Semi-axis 7 (cube side 20, 400 rows): the tuner may not try fewer blocks
    per particle than cover every cube row with a thread (one block of 256
    threads would leave rows 256-399 of each cube undone), and every candidate
    it tries must leave the run bit for bit where an untuned run is."""
    g = rng(23)
    boxes = [box(64, 48, 48, 0.9, counter_force=1)]
    parts = [[particle((7.0, 3.0, 2.5), (20.5, 21.2, 19.1), random_quaternion(g), F_ext=(2e-4, -1e-4, 0)),
              particle((6.0, 3.0, 3.0), (48.3, 30.1, 38.7), random_quaternion(g), F_ext=(0, 1e-4, 1e-4))]]
    a = _sim(boxes, parts)
    (fetch, gx, advanced), ms = L.lb_autotune(a.ctx, 5)
    assert ms[0] == 0.0 and gx >= 2
    a.step(7)
    b = _sim(boxes, parts)
    b.step(advanced + 7)
    assert np.array_equal(a.field("df"), b.field("df"))
    assert np.array_equal(a.records(), b.records())


def test_async_record_copies_match_synchronous_reads():
    """A pipelined loop (each step's F_ext from its own pinned slot, each step's
    records copied into their own pinned slot by lb_get_force_torque_async, one
    wait at the end), and lb_step_io doing the same in one call, give the
    records a synchronous loop reads step by step."""
    torch = pytest.importorskip("torch")
    boxes, parts = single_32(seed=6)
    K = 12
    ft = torch.empty((K, 1, 6), dtype=torch.float64, pin_memory=True)
    for k in range(K):
        ft[k, 0] = torch.tensor([1e-4 * (1 + 0.1 * k), -2e-5 * k, 0.0, 0.0, 1e-6 * k, 0.0], dtype=torch.float64)
    recs = torch.empty((K, 1, L.LB_RECORD_DOUBLES), dtype=torch.float64, pin_memory=True)
    a = _sim(boxes, parts)
    b = _sim(boxes, parts)
    a.step(3)
    b.step(3)
    ftn = ft.numpy()
    for k in range(K):
        L.lb_set_external(a.ctx, -1, ftn[k])
        a.step(1)
        L.lb_get_force_torque_async(a.ctx, -1, 1, recs[k].data_ptr())
    L.lb_synchronize(a.ctx)
    for k in range(K):
        L.lb_set_external(b.ctx, -1, ftn[k])
        b.step(1)
        assert np.array_equal(recs[k].numpy(), b.records())
    # the inputs of every step took effect (F_ext enters the records' force)
    assert not np.array_equal(recs[0].numpy(), recs[-1].numpy())
    # the same loop queued by the library in one call
    c = _sim(boxes, parts)
    c.step(3)
    recs_io = torch.empty_like(recs)
    L.lb_step_io(c.ctx, K, ft.data_ptr(), recs_io.data_ptr())
    L.lb_synchronize(c.ctx)
    assert np.array_equal(recs_io.numpy(), recs.numpy())
    assert np.array_equal(c.records(), recs[-1].numpy())
    # pageable host memory: the per-step copy path, same records
    d = _sim(boxes, parts)
    d.step(3)
    ft_pageable = np.array(ft.numpy())
    recs_pageable = np.zeros(recs.shape)
    L.lb_step_io(d.ctx, K, ft_pageable.ctypes.data, recs_pageable.ctypes.data)
    L.lb_synchronize(d.ctx)
    assert np.array_equal(recs_pageable, recs.numpy())
    # device memory: the step kernel reads and writes it directly as well
    g = _sim(boxes, parts)
    g.step(3)
    ft_dev, recs_dev = ft.cuda(), torch.zeros(recs.shape, dtype=torch.float64, device="cuda")
    L.lb_step_io(g.ctx, K, ft_dev.data_ptr(), recs_dev.data_ptr())
    L.lb_synchronize(g.ctx)
    assert np.array_equal(recs_dev.cpu().numpy(), recs.numpy())
    # forces only, records only
    h = _sim(boxes, parts)
    h.step(3)
    L.lb_step_io(h.ctx, K, ft.data_ptr(), None)
    L.lb_synchronize(h.ctx)
    assert np.array_equal(h.records(), recs[-1].numpy())
    with pytest.raises(L.LBError):
        L.lb_step_io(h.ctx, -1, None, None)
    # from the very first step (the first collision runs as separate kernels)
    e = _sim(boxes, parts)
    f = _sim(boxes, parts)
    recs_first = torch.empty_like(recs)
    L.lb_step_io(e.ctx, K, ft.data_ptr(), recs_first.data_ptr())
    L.lb_synchronize(e.ctx)
    for k in range(K):
        L.lb_set_external(f.ctx, -1, ftn[k])
        f.step(1)
        assert np.array_equal(recs_first[k].numpy(), f.records())


def test_steps_capture_into_a_cuda_graph_and_replay():
    """lb_step on a capturing stream records the persistent step kernel (and its
    counter reset) into a CUDA graph; replaying a graph of an even number of
    steps (the two distribution buffers come back to the same parity) continues
    the run exactly as direct calls do."""
    torch = pytest.importorskip("torch")
    boxes, parts = single_32(seed=7)
    s = torch.cuda.Stream()
    sp = L.stream_handle(s)
    a = _sim(boxes, parts)
    b = _sim(boxes, parts)
    a.step(2, stream=sp)
    b.step(2, stream=sp)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        L.lb_step(a.ctx, 8, sp)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    b.step(24, stream=sp)
    L.lb_synchronize(b.ctx)
    assert np.array_equal(a.records(), b.records())
    assert np.array_equal(a.field("df"), b.field("df"))
