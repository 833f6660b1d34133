"""Parity of the warm-start entry points (lb_stokes_field, lb_init_fluid with
and without the stress part, lb_mlp_features, lb_resistance_targets,
lb_warm_velocities), called through the C ABI, with the FP64 reference
oracle/warmstart.py and the FP64 LB oracle.

Bars: the steady flow of the lattice fluid and its density within 1e-4
normwise (FP32 DFTs of length <= 40 against numpy's FP64 FFT: each pass adds
a few FP32 roundings per term; the per-mode solve is FP64 on both sides); a run started
from lb_init_fluid within the bars of the plain runs (1e-5 normwise on the
deviations, u, F and T every few steps); features, targets and velocities
within FP32 rounding (2e-6 normwise)."""
import math

import numpy as np
import pytest

from lb_inputs import box, particle, random_quaternion, rng
from oracle import oracle as O
from oracle import warmstart as W
from parity_util import direction_map, normwise, oracle_df_gpu_layout

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_2403_05443_gb300.lbsph")
SU = pytest.importorskip("paper_2403_05443_gb300.surrogate")


def _case():
    g = rng(31)
    b = box(40, 24, 36, 0.9, counter_force=1)
    parts = [particle((4.5, 2.5, 2.0), (9.3, 9.1, 10.7), random_quaternion(g), F_ext=(2e-4, -1e-4, 5e-5)),
             particle((3.0, 2.0, 2.0), (29.2, 15.6, 27.9), random_quaternion(g), F_ext=(-5e-5, 1e-4, 1e-4))]
    return b, parts


def _sim(b, parts):
    return L.Simulation([b], [parts], max_semi=int(math.ceil(max(max(p["semi"]) for p in parts))))


def _gpu_stokes(sim, b):
    N = b["nx"] * b["ny"] * b["nz"]
    u = torch.zeros(3 * N, dtype=torch.float32, device="cuda")
    d = torch.zeros(N, dtype=torch.float32, device="cuda")
    L.lb_stokes_field(sim.ctx, 0, u.data_ptr(), d.data_ptr())
    return u, d


def test_stokes_field_matches_reference():
    b, parts = _case()
    sim = _sim(b, parts)
    ud, dd = _gpu_stokes(sim, b)
    u = ud.cpu().numpy().reshape(3, b["nz"], b["ny"], b["nx"])
    d = dd.cpu().numpy().reshape(b["nz"], b["ny"], b["nx"])
    owner = sim.field("solid")
    mu = b["rho0"] * (b["tau"] - 0.5) / 3.0
    ref, dref = W.stokes_field(b["nx"], b["ny"], b["nz"], owner, [p["F_ext"] for p in parts], mu, counter=True,
                               density=True, tau=b["tau"], rho0=b["rho0"])
    err, derr = normwise(u, ref), normwise(d, dref)
    print("stokes error", err, derr)
    assert err <= 1e-4 and derr <= 1e-4


@pytest.mark.parametrize("shape,tau", [((32, 16, 64), 0.8), ((64, 24, 32), 0.8), ((32, 16, 64), 0.52),
                                       ((64, 24, 32), 1.45)])
def test_stokes_field_with_power_of_two_edges_matches_reference(shape, tau):
    """Power-of-two edges take the radix-2 FFT pass (one edge of the second box
    does not, and keeps the transform by definition).  At tau = 0.52 the
    per-mode denominator 1 - (1 - omega) cos(theta) falls to about 0.04 near
    theta = pi, where its FP32 terms lose most digits: the bar still holds."""
    nx, ny, nz = shape
    g = rng(37)
    b = box(nx, ny, nz, tau, counter_force=1)
    parts = [particle((4.5, 2.5, 2.0), (nx * 0.3, ny * 0.45, nz * 0.4), random_quaternion(g), F_ext=(2e-4, -1e-4, 5e-5)),
             particle((3.0, 2.0, 2.0), (nx * 0.75, ny * 0.55, nz * 0.8), random_quaternion(g), F_ext=(-5e-5, 1e-4, 1e-4))]
    sim = _sim(b, parts)
    ud, dd = _gpu_stokes(sim, b)
    u = ud.cpu().numpy().reshape(3, nz, ny, nx)
    d = dd.cpu().numpy().reshape(nz, ny, nx)
    mu = b["rho0"] * (b["tau"] - 0.5) / 3.0
    ref, dref = W.stokes_field(nx, ny, nz, sim.field("solid"), [p["F_ext"] for p in parts], mu, counter=True,
                               density=True, tau=b["tau"], rho0=b["rho0"])
    err, derr = normwise(u, ref), normwise(d, dref)
    print("stokes error", shape, tau, err, derr)
    assert err <= 1e-4 and derr <= 1e-4


def test_run_from_initial_fluid_matches_oracle():
    """Start both sides from f = f_eq(rho0 + drho, u) of the Stokes flow and its
    pressure and compare every field
    and particle value over 40 steps."""
    b, parts = _case()
    sim = _sim(b, parts)
    ud, dd = _gpu_stokes(sim, b)
    L.lb_init_fluid(sim.ctx, 0, ud.data_ptr(), ud.numel() * 4, dd.data_ptr(), True, False)
    u = ud.cpu().numpy().astype(np.float64).reshape(3, b["nz"], b["ny"], b["nx"])
    d = dd.cpu().numpy().astype(np.float64).reshape(b["nz"], b["ny"], b["nx"])
    o = O.Sim(b, parts, nthreads=8)
    co, wo = O.lattice()
    f = o.f()
    fluid = o.owner() == 0
    feq = W.equilibrium_f(u, b["rho0"] + d, co, wo)
    f[fluid] = feq[fluid]
    o.set_f(f)
    # before the first collision the read-back is the initial field itself
    assert normwise(sim.field("df"), oracle_df_gpu_layout(o, b["rho0"])) <= 1e-6
    worst = {"df": 0.0, "u": 0.0, "F": 0.0}
    for _ in range(8):
        sim.step(5)
        o.step(5)
        worst["df"] = max(worst["df"], normwise(sim.field("df"), oracle_df_gpu_layout(o, b["rho0"])))
        _, ur = o.moments()
        worst["u"] = max(worst["u"], normwise(sim.field("u"), np.moveaxis(ur, -1, 0)))
        for p in range(2):
            worst["F"] = max(worst["F"], normwise(sim.particle(0, p)["F"], o.particle(p)["F"]))
    print("warm-start parity", worst)
    assert worst["df"] <= 1e-5 and worst["u"] <= 1e-5 and worst["F"] <= 1e-5


def test_features_targets_and_velocities_match_reference():
    g = np.random.default_rng(5)
    n = 50
    e = g.normal(0, 1, (n, 3))
    e /= np.linalg.norm(e, axis=1, keepdims=True)
    geom = np.column_stack([g.uniform(2, 9, n), g.uniform(2, 4, n), g.uniform(0.1, 0.25, n), g.uniform(24, 64, n),
                            e, np.ones(n)])
    A = g.normal(0, 1, (n, 6, 6))
    M = np.einsum("nik,njk->nij", A, A) * 1e-3 + 1e-2 * np.eye(6)
    FT = g.normal(0, 1e-4, (n, 6))
    gd = torch.from_numpy(geom).cuda()
    x = torch.zeros((n, 8), dtype=torch.float32, device="cuda")
    SU.lb_mlp_features(gd.data_ptr(), n, x.data_ptr())
    Md = torch.from_numpy(M.reshape(n, 36)).cuda()
    Rh = torch.zeros((n, 36), dtype=torch.float32, device="cuda")
    SU.lb_resistance_targets(Md.data_ptr(), gd.data_ptr(), n, Rh.data_ptr())
    FTd = torch.from_numpy(FT).cuda()
    UW = torch.zeros((n, 6), dtype=torch.float64, device="cuda")
    SU.lb_warm_velocities(Rh.data_ptr(), gd.data_ptr(), FTd.data_ptr(), n, UW.data_ptr())
    torch.cuda.synchronize()
    assert normwise(x.cpu().numpy(), W.features(geom)) <= 2e-7
    Rref = W.targets(M, geom)
    assert normwise(Rh.cpu().numpy().reshape(n, 6, 6), Rref) <= 2e-6
    Rf = Rh.cpu().numpy().astype(np.float64)
    assert normwise(UW.cpu().numpy(), W.warm_velocities(Rf, geom, FT)) <= 1e-10


def test_run_from_initial_fluid_with_stress_matches_oracle():
    """lb_init_fluid with the non-equilibrium stress part (tau = 0.9, where the
    collision keeps part of it): the stored start equals the oracle's f_eq +
    stress_f, and a run from it follows the oracle's run from the same start."""
    b, parts = _case()
    sim = _sim(b, parts)
    ud, dd = _gpu_stokes(sim, b)
    L.lb_init_fluid(sim.ctx, 0, ud.data_ptr(), ud.numel() * 4, dd.data_ptr(), True, True)
    u = ud.cpu().numpy().astype(np.float64).reshape(3, b["nz"], b["ny"], b["nx"])
    d = dd.cpu().numpy().astype(np.float64).reshape(b["nz"], b["ny"], b["nx"])
    o = O.Sim(b, parts, nthreads=8)
    co, wo = O.lattice()
    f = o.f()
    fluid = o.owner() == 0
    rho = b["rho0"] + d
    start = W.equilibrium_f(u, rho, co, wo) + W.stress_f(u, rho, b["tau"], co, wo)
    f[fluid] = start[fluid]
    o.set_f(f)
    assert normwise(sim.field("df"), oracle_df_gpu_layout(o, b["rho0"])) <= 1e-6
    # the stress part is a visible share of the start
    plain = W.equilibrium_f(u, rho, co, wo)
    share = np.abs(start - plain)[fluid].max() / np.abs(plain - wo * b["rho0"])[fluid].max()
    assert share > 1e-2
    worst = {"df": 0.0, "F": 0.0}
    for _ in range(8):
        sim.step(5)
        o.step(5)
        worst["df"] = max(worst["df"], normwise(sim.field("df"), oracle_df_gpu_layout(o, b["rho0"])))
        for p in range(2):
            worst["F"] = max(worst["F"], normwise(sim.particle(0, p)["F"], o.particle(p)["F"]))
    print("stress warm-start parity", worst, "stress share", share)
    assert worst["df"] <= 1e-5 and worst["F"] <= 1e-5
