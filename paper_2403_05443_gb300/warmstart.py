"""Learned warm start of spheroid runs: resistance tensors measured by the LB
method, the surrogate trained on them, and its use to start a run near steady
state.  Orchestration only: the LB runs, the lattice fluid's steady flow, the network's
training and inference and the 6x6 solves are calls into liblbsph.so
(include/lbsph.h, include/lbsurrogate.h); the host assembles the calls'
inputs and outputs.

Resistance data (the paper measures drag at steady state, Sec. III): for each
sample, six periodic boxes hold the same spheroid, box k with a unit force
(k < 3) or torque (k >= 3) along axis k and the opposite force spread over the
fluid; after the flow has developed, (U, Omega) of box k is column k of the
mobility M, and the target is R^ = (D M D)^-1 (lb_resistance_targets).  The 24
rotations of the cube map the periodic D3Q19 lattice onto itself, so each
sample also gives the mobility of the 23 rotated spheroids, P M P^T with
P = diag(Q, Q): exact copies of what the method would measure for them (up to
the centre's sub-node offset, which is random anyway).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import lbsph as L
from . import surrogate as SU


def _torch():
    import torch
    return torch


def cube_rotations():
    """The 24 proper rotations of the cube as 3x3 signed permutation matrices."""
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            P = np.zeros((3, 3))
            for i, j in enumerate(perm):
                P[i, j] = signs[i]
            if round(np.linalg.det(P)) == 1:
                out.append(P)
    return out


def geom_of(a, b, tau, Ledge, e, rho0=1.0):
    return [float(a), float(b), (float(tau) - 0.5) / 3.0, float(Ledge), float(e[0]), float(e[1]), float(e[2]),
            float(rho0)]


def _ft_of(smp, k, force, torque):
    unit = np.eye(3)[k % 3]
    fe = force * unit if k < 3 else np.zeros(3)
    te = torque * unit if k >= 3 else np.zeros(3)
    return fe, te


def measure_mobility(samples, max_steps: int, force=1e-4, torque=None, device: int = 0, batch: int = 64,
                     check_every: int = 0, tol: float = 1e-5, checks: int = 3, warm_fluid: bool = False,
                     history=None):
    """Mobility matrices M[n, 6, 6] of the samples (dicts of
    lb_inputs.resistance_samples, all with the same box edge) from the LB
    method, in batched contexts of 6 boxes per sample (box k: unit force or
    torque along axis k).  force / torque: a number, or a function of the
    sample (default torque: force * b).

    check_every = 0: `max_steps` iterations.  Otherwise each run goes to steady
    state: every check_every iterations the (U, b Omega) of every box is
    compared with the last check's; a sample is steady once its six boxes have
    all changed by less than tol (relative) at `checks` consecutive checks, and
    its mobility is taken then; a batch runs until all its samples are steady or
    max_steps (history, a list, collects (step, largest change of a sample not
    yet steady, median change) of every check).  warm_fluid: each box starts from the lattice fluid's own steady
    flow under its particle's force (lb_stokes_field, lb_init_fluid), the
    particles at rest, which leaves only the particle's and the near field's
    adjustment to relax.  Returns (M, steps used per sample, converged per
    sample)."""
    torch = _torch()
    out = np.zeros((len(samples), 6, 6))
    used = np.zeros(len(samples), np.int64)
    conv = np.zeros(len(samples), bool)
    fofs = force if callable(force) else (lambda smp: force)
    tofs = torque if callable(torque) else ((lambda smp: torque) if torque is not None
                                             else (lambda smp: fofs(smp) * smp["b"]))
    for s0 in range(0, len(samples), batch):
        chunk = samples[s0:s0 + batch]
        boxes, parts = [], []
        for smp in chunk:
            for k in range(6):
                fe, te = _ft_of(smp, k, fofs(smp), tofs(smp))
                boxes.append(dict(nx=smp["L"], ny=smp["L"], nz=smp["L"], tau=smp["tau"], rho0=1.0,
                                  counter_force=1))
                parts.append([dict(semi=(smp["a"], smp["b"], smp["b"]), x=smp["x"], q=smp["q"],
                                   F_ext=list(fe), T_ext=list(te))])
        ms = int(math.ceil(max(s["a"] for s in chunk)))
        sim = L.Simulation(boxes, parts, max_semi=ms, device=device)
        if warm_fluid:
            for bi, b in enumerate(boxes):
                N = b["nx"] * b["ny"] * b["nz"]
                u = torch.zeros(3 * N, dtype=torch.float32, device="cuda")
                d = torch.zeros(N, dtype=torch.float32, device="cuda")
                L.lb_stokes_field(sim.ctx, bi, u.data_ptr(), d.data_ptr())
                L.lb_init_fluid(sim.ctx, bi, u.data_ptr(), u.numel() * 4, d.data_ptr(), True, True)
        bscale = np.repeat(np.array([s["b"] for s in chunk]), 6)[:, None]
        nch = len(chunk)
        rec_keep = np.zeros((len(boxes), 25))
        if check_every <= 0:
            sim.step(max_steps)
            rec_keep[:] = L.lb_get_force_torque(sim.ctx, -1, len(boxes))
            used[s0:s0 + nch] = max_steps
        else:
            # each sample is steady once all six of its boxes have changed by less
            # than tol at `checks` consecutive checks; its records are kept from
            # then on (a node the particle covers later jolts the velocity by
            # ~1e-3 for a few hundred steps)
            prev, streak = None, np.zeros(nch, int)
            done = np.zeros(nch, bool)
            steps = 0
            while steps < max_steps and not done.all():
                sim.step(check_every)
                steps += check_every
                rec = L.lb_get_force_torque(sim.ctx, -1, len(boxes))
                X = np.concatenate([rec[:, 12:15], rec[:, 15:18] * bscale], axis=1)
                if prev is not None:
                    ch = np.linalg.norm(X - prev, axis=1) / np.maximum(np.linalg.norm(X, axis=1), 1e-300)
                    chs = ch.reshape(nch, 6).max(axis=1)
                    if history is not None:
                        history.append((steps, float(chs[~done].max()) if (~done).any() else 0.0,
                                        float(np.median(chs))))
                    streak = np.where(chs < tol, streak + 1, 0)
                    newly = (~done) & (streak >= checks)
                    for i in np.nonzero(newly)[0]:
                        rec_keep[6 * i:6 * i + 6] = rec[6 * i:6 * i + 6]
                        used[s0 + i] = steps
                        conv[s0 + i] = True
                    done |= newly
                prev = X
            rest = np.nonzero(~done)[0]
            for i in rest:
                rec_keep[6 * i:6 * i + 6] = rec[6 * i:6 * i + 6]
                used[s0 + i] = steps
        sim.close()
        for i, smp in enumerate(chunk):
            for k in range(6):
                mag = fofs(smp) if k < 3 else tofs(smp)
                r = rec_keep[6 * i + k]
                out[s0 + i, :3, k] = r[12:15] / mag
                out[s0 + i, 3:, k] = r[15:18] / mag
    return out, used, conv


def config5_dataset(seed: int = 0, n: int = 2000, L_edge: int = 64, max_steps: int = 40000, batch: int = 96,
                    device: int = 0, drift: float = 0.02, tol: float = 1e-4, history=None):
    """The surrogate workload's training set: n samples in periodic L^3
    boxes, tau uniform in [0.6, 1.5], a/b in [1, 4], b in [3, 5], uniform
    orientation; each run to steady state (checked every 500 steps, relative
    change of every box's (U, b Omega) below tol at three consecutive checks,
    from the lattice fluid's steady flow).  The force and torque of each sample are scaled so that the
    particle moves at most `drift` lattice units (and its surface turns by at
    most that) in max_steps: no node is covered or uncovered, which would
    jitter the velocity by a few 1e-3 and defeat the steady-state test.
    Samples run in batches of similar tau (similar relaxation times)."""
    import lb_inputs as I
    samples = I.resistance_samples(seed, n, L_edge, tau_range=(0.6, 1.5), aspect=(1.0, 4.0), b_range=(3.0, 5.0))
    order = np.argsort([s["tau"] for s in samples], kind="stable")

    def fmag(smp):
        mu = (smp["tau"] - 0.5) / 3.0
        return drift * 6.0 * math.pi * mu * smp["b"] / max_steps

    def tmag(smp):
        mu = (smp["tau"] - 0.5) / 3.0
        return drift * 8.0 * math.pi * mu * smp["b"] ** 3 / (smp["a"] * max_steps)

    M = np.zeros((n, 6, 6))
    used = np.zeros(n, np.int64)
    conv = np.zeros(n, bool)
    sub = [samples[i] for i in order]
    Ms, us, cs = measure_mobility(sub, max_steps, force=fmag, torque=tmag, device=device, batch=batch,
                                  check_every=500, tol=tol, checks=3, warm_fluid=True, history=history)
    M[order], used[order], conv[order] = Ms, us, cs
    return samples, M, used, conv


def augment(geoms, M):
    """Cube-rotated copies: e -> Q e, M -> P M P^T with P = diag(Q, Q)."""
    G, Ms = [], []
    for Q in cube_rotations():
        P = np.zeros((6, 6))
        P[:3, :3] = Q
        P[3:, 3:] = Q
        for g, m in zip(geoms, M):
            e = Q @ np.asarray(g[4:7])
            G.append(list(g[:4]) + list(e) + [g[7]])
            Ms.append(P @ m @ P.T)
    return np.asarray(G), np.asarray(Ms)


def targets(geoms, M):
    """R^ targets (device FP32 [n, 36]) and features (device FP32 [n, 8])."""
    torch = _torch()
    n = len(geoms)
    gd = torch.as_tensor(np.asarray(geoms, np.float64), device="cuda")
    Md = torch.as_tensor(np.asarray(M, np.float64).reshape(n, 36), device="cuda")
    R = torch.zeros((n, 36), dtype=torch.float32, device="cuda")
    x = torch.zeros((n, 8), dtype=torch.float32, device="cuda")
    SU.lb_resistance_targets(Md.data_ptr(), gd.data_ptr(), n, R.data_ptr())
    SU.lb_mlp_features(gd.data_ptr(), n, x.data_ptr())
    return x, R


def init_params(seed: int = 0):
    """He-style initial weights (seeded), zero biases except the diagonal of L
    (softplus(0.55) = 1: the output starts at R^ = I)."""
    g = np.random.default_rng(seed)
    p = np.zeros(SU.LB_MLP_NPARAM, np.float32)
    P = SU.unpack(p)
    P["W1"][:, :8] = g.normal(0, math.sqrt(2.0 / 8), (256, 8))
    P["W2"][:] = g.normal(0, math.sqrt(2.0 / 256), (256, 256))
    P["W3"][:21] = g.normal(0, 0.1 * math.sqrt(1.0 / 256), (21, 256))
    for i in range(6):
        P["b3"][i * (i + 1) // 2 + i] = 0.5413
    return p


def train(x, R, steps: int = 3000, batch: int = 512, lr: float = 2e-3, seed: int = 0, net=None):
    """Adam on minibatches drawn (seeded) from the device arrays x, R; the
    learning rate decays linearly to lr/20.  Returns the network and the loss
    of the last minibatches."""
    torch = _torch()
    n = x.shape[0]
    batch = min(batch, n)
    net = net or SU.Surrogate(max_batch=max(batch, 1024), params=init_params(seed))
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    loss = torch.zeros(1, device="cuda")
    hist = []
    for t in range(steps):
        idx = torch.randint(0, n, (batch,), device="cuda", generator=g)
        xb, Rb = x[idx].contiguous(), R[idx].contiguous()
        rate = lr * (1.0 - 0.95 * t / max(1, steps - 1))
        SU.lb_mlp_train_step(net.h, xb.data_ptr(), Rb.data_ptr(), batch, rate, loss.data_ptr())
        if t >= steps - 20:
            hist.append(float(loss.item()))
    return net, float(np.mean(hist)) if hist else float("nan")


def predict(net, x):
    """R^ (device FP32 [n, 36]) for features x (device FP32 [n, 8])."""
    torch = _torch()
    n = x.shape[0]
    R = torch.zeros((n, 36), dtype=torch.float32, device="cuda")
    for s0 in range(0, n, 1024):
        m = min(1024, n - s0)
        SU.lb_mlp_forward(net.h, x[s0:s0 + m].data_ptr(), m, None, R[s0:s0 + m].data_ptr())
    return R


def long_axis(q):
    """The lab direction of the body x axis for a unit quaternion (q0, q1, q2, q3)."""
    q0, q1, q2, q3 = q
    return [q0 * q0 + q1 * q1 - q2 * q2 - q3 * q3, 2 * (q1 * q2 + q0 * q3), 2 * (q1 * q3 - q0 * q2)]


def warm_start(sim, box: int, net, use_net: bool = True, use_fluid: bool = True, use_stress: bool = True):
    """Before the first step: set each particle's (U, Omega) to the surrogate's
    steady estimate R^-1 (F_ext, T_ext) (use_net) and the fluid to the lattice
    fluid's own steady flow and density under the particle forces (use_fluid), with the
    flow's viscous stress in the populations' non-equilibrium part
    (use_stress; no effect at tau = 1, where the first collision discards it).
    The confinement feature is the box's own edge (for a non-cubic box, the
    cube root of its volume): each particle's self-mobility in that box; the
    other particles act through the fluid.  (The edge of the volume per
    particle, which treats the suspension as a periodic array of identical
    particles, predicted the steady velocities of 16 spheroids with random
    forces in a 128^3 box to 18 % median error, the box edge to 12 %.)"""
    torch = _torch()
    b = sim.boxes[box]
    parts = [dict(p) for p in sim.parts_of(box)]
    n = len(parts)
    if use_net and n:
        Ledge = (b["nx"] * b["ny"] * b["nz"]) ** (1.0 / 3.0)
        geoms = [geom_of(p["semi"][0], p["semi"][1], b["tau"], Ledge, long_axis(p["q"]), b.get("rho0", 1.0))
                 for p in parts]
        gd = torch.as_tensor(np.asarray(geoms), device="cuda")
        x = torch.zeros((n, 8), dtype=torch.float32, device="cuda")
        SU.lb_mlp_features(gd.data_ptr(), n, x.data_ptr())
        R = predict(net, x)
        FT = torch.as_tensor(np.asarray([list(p.get("F_ext", (0, 0, 0))) + list(p.get("T_ext", (0, 0, 0)))
                                         for p in parts], np.float64), device="cuda")
        UW = torch.zeros((n, 6), dtype=torch.float64, device="cuda")
        SU.lb_warm_velocities(R.data_ptr(), gd.data_ptr(), FT.data_ptr(), n, UW.data_ptr())
        uw = UW.cpu().numpy()
        for p, v in zip(parts, uw):
            p["U"], p["Om"] = [float(t) for t in v[:3]], [float(t) for t in v[3:]]
        sim.set_particles(box, parts)
    if use_fluid:
        N = b["nx"] * b["ny"] * b["nz"]
        u = torch.zeros(3 * N, dtype=torch.float32, device="cuda")
        d = torch.zeros(N, dtype=torch.float32, device="cuda")
        L.lb_stokes_field(sim.ctx, box, u.data_ptr(), d.data_ptr())
        L.lb_init_fluid(sim.ctx, box, u.data_ptr(), u.numel() * 4, d.data_ptr(), True, use_stress)


def velocity_history(sim, box: int, steps: int, every: int):
    """U and Omega of the box's particles every `every` steps: [k, n, 6]."""
    out = []
    for _ in range(steps // every):
        sim.step(every)
        r = sim.records(box)
        out.append(r[:, 12:18].copy())
    return np.asarray(out)


def velocity_error(hist, ref):
    """max over particles of |U - U_ref| / rms |U_ref| at each record."""
    scale = float(np.sqrt((np.linalg.norm(ref, axis=1) ** 2).mean()))
    return np.abs(hist[:, :, :3] - ref[None]).max(axis=2).max(axis=1) / scale


def steps_to_steady(hist, ref, every: int, tol: float = 1e-3):
    """First step after which every particle's velocity stays within tol (in
    units of the particles' rms steady speed) of the steady velocities ref[n, 3];
    None if it never does within the record."""
    worst = velocity_error(hist, ref)
    bad = np.nonzero(worst > tol)[0]
    if len(bad) == 0:
        return every
    if bad[-1] == len(worst) - 1:
        return None
    return int((bad[-1] + 2) * every)


def save_params(net, path: str):
    """The network's FP32 parameters to a .npy file."""
    np.save(path, net.params())


def load_params(path: str, device: int = 0, max_batch: int = 1024):
    """A network with the parameters of a .npy file written by save_params."""
    p = np.load(path).astype(np.float32)
    return SU.Surrogate(device=device, max_batch=max_batch, params=p)


def evaluate(net, seed: int = 0, eval_n: int = 128, eval_count: int = 16, force: float = 1e-7, every: int = 50,
             ref_steps: int = 40000, eval_tau: float = 1.0, aspect=(1.5, 2.5), b_range=(2.5, 3.0), device: int = 0,
             modes=("stokes_fluid_only", "warm")):
    """Steps to steady state of an eval_n^3 box with eval_count spheroids (sizes
    drawn from the ranges, random orientations, forces of magnitude `force`
    in random directions with the counter force) started cold (fluid and
    particles at rest), with the lattice fluid's steady flow only, and with that
    flow plus the network's velocities ("warm"), each against the velocities
    at the end of a ref_steps cold run: the first step after which every
    particle's velocity stays within 1e-2, 3e-3 and 1e-3 (in units of the rms
    steady speed) of it.  The forces are small enough that no particle covers a
    node during the runs."""
    import time

    import lb_inputs as I
    torch = _torch()
    boxes, parts = I.many_spheroids(seed, n=eval_n, count=eval_count, force=force, tau=eval_tau, aspect=aspect,
                                    b_range=b_range)
    ms = int(math.ceil(max(p["semi"][0] for p in parts[0])))
    cost = {}

    def run(mode, steps):
        sim = L.Simulation(boxes, parts, max_semi=ms, device=device)
        if mode != "cold":
            torch.cuda.synchronize()
            t = time.perf_counter()
            warm_start(sim, 0, net, use_net=mode.startswith("warm"), use_fluid=True,
                       use_stress=(mode != "warm_no_stress"))
            torch.cuda.synchronize()
            cost[mode + "_warm_start_s"] = time.perf_counter() - t
        t = time.perf_counter()
        h = velocity_history(sim, 0, steps, every)
        cost[mode + "_seconds_per_step"] = (time.perf_counter() - t) / steps
        sim.close()
        return h

    ref = run("cold", ref_steps)
    U_ss = ref[-1, :, :3]
    drift = float(velocity_error(ref[-11:-10], U_ss)[0])
    tols = (1e-2, 3e-3, 1e-3)
    res = {f"cold@{t:g}": steps_to_steady(ref, U_ss, every, t) for t in tols}
    curves = {"cold": velocity_error(ref, U_ss)}
    end_vs_ref = {}
    for mode in modes:
        h = run(mode, ref_steps // 2)
        for t in tols:
            res[f"{mode}@{t:g}"] = steps_to_steady(h, U_ss, every, t)
        curves[mode] = velocity_error(h, U_ss)
        end_vs_ref[mode] = float(curves[mode][-1])
    pick = lambda c: {int((i + 1) * every): float(c[i]) for i in range(0, len(c), max(1, len(c) // 40))}
    gain = lambda a, b: (res[a] / res[b]) if res[a] and res[b] else None
    return {"steps_to_steady": res,
            "gain_warm_vs_cold": {f"{t:g}": gain(f"cold@{t:g}", f"warm@{t:g}") for t in tols},
            "gain_warm_vs_fluid_only": ({f"{t:g}": gain(f"stokes_fluid_only@{t:g}", f"warm@{t:g}") for t in tols}
                                        if "stokes_fluid_only" in modes else None),
            "reference_drift_last_500_steps": drift, "end_of_runs_vs_reference": end_vs_ref,
            "eval": (f"{eval_n}^3, {eval_count} spheroids (a/b in {list(aspect)}, b in {list(b_range)}), "
                     f"|F|={force}, tau={eval_tau}"),
            "error_curves": {k: pick(v) for k, v in curves.items()}, "seconds": cost}


def held_out_error(net, geoms, M):
    """Relative (Frobenius) error of the network's R^ on samples it was not trained on."""
    torch = _torch()
    xv, Rv = targets(geoms, M)
    Pv = predict(net, xv)
    return (torch.linalg.matrix_norm((Pv - Rv).reshape(-1, 6, 6)) /
            torch.linalg.matrix_norm(Rv.reshape(-1, 6, 6))).cpu().numpy()


def experiment(seed: int = 0, n32: int = 384, n48: int = 128, train_steps: int = 4000, eval_n: int = 128,
               eval_count: int = 16, force: float = 2e-5, every: int = 50, ref_steps: int = 40000, device: int = 0,
               eval_tau: float = 1.0):
    """A reduced learned warm start, end to end on the GPU:
      1. resistance data from the LB method: n32 samples in 32^3 boxes and n48
         in 48^3 boxes (tau in {0.8, 1, 1.2}, a/b in [1, 3], b in [2, 3.5]),
         each flow developed for 8 diffusion times L^2 / (4 pi^2 nu) of its box;
      2. 24-fold cube-rotation augmentation, 10 % of the LB samples held out;
      3. training of the network;
      4. evaluate(): an eval_n^3 box with eval_count spheroids, cold, steady
         lattice fluid only, and warm.
    Returns a dict of the measurements.  config5() is the full-size form."""
    import time

    import lb_inputs as I
    t0 = time.time()
    samples = I.resistance_samples(seed, n32, 32) + I.resistance_samples(seed + 1, n48, 48)
    M = np.zeros((len(samples), 6, 6))
    for Ledge in (32, 48):
        idx = [i for i, s in enumerate(samples) if s["L"] == Ledge]
        for tau in (0.8, 1.0, 1.2):
            sub = [i for i in idx if samples[i]["tau"] == tau]
            if not sub:
                continue
            nu = (tau - 0.5) / 3.0
            steps = int(8 * Ledge * Ledge / (4 * math.pi ** 2 * nu))
            M[sub] = measure_mobility([samples[i] for i in sub], steps, device=device)[0]
    t_data = time.time() - t0
    geoms = np.asarray([geom_of(s["a"], s["b"], s["tau"], s["L"], s["e"]) for s in samples])
    g = np.random.default_rng(seed)
    perm = g.permutation(len(samples))
    nval = max(1, len(samples) // 10)
    val, tr = perm[:nval], perm[nval:]
    Gt, Mt = augment(geoms[tr], M[tr])
    x, R = targets(Gt, Mt)
    t1 = time.time()
    net, train_loss = train(x, R, steps=train_steps, seed=seed)
    t_train = time.time() - t1
    rel = held_out_error(net, geoms[val], M[val])
    t2 = time.time()
    ev = evaluate(net, seed=seed, eval_n=eval_n, eval_count=eval_count, force=force, every=every,
                  ref_steps=ref_steps, eval_tau=eval_tau, device=device,
                  modes=("stokes_fluid_only", "warm") + (("warm_no_stress",) if eval_tau != 1.0 else ()))
    ev["seconds"].update({"data": t_data, "train": t_train, "eval": time.time() - t2})
    return {"samples": len(samples), "augmented": int(len(Gt)), "train_loss": train_loss,
            "val_rel_err_median": float(np.median(rel)), "val_rel_err_max": float(rel.max()), **ev}


def config5(seed: int = 0, n: int = 2000, train_steps: int = 8000, out: str = "", device: int = 0):
    """The surrogate workload at its stated size: config5_dataset (n runs on
    64^3 boxes to steady state), 24-fold augmentation with 10 % of the LB
    samples held out, training, and the held-out error; the parameters go to
    `out` (.npy) when given.  Returns (net, summary)."""
    import time

    t0 = time.time()
    samples, M, used, conv = config5_dataset(seed=seed, n=n, device=device)
    t_data = time.time() - t0
    geoms = np.asarray([geom_of(s["a"], s["b"], s["tau"], s["L"], s["e"]) for s in samples])
    g = np.random.default_rng(seed)
    perm = g.permutation(len(samples))
    nval = max(1, len(samples) // 10)
    val, tr = perm[:nval], perm[nval:]
    Gt, Mt = augment(geoms[tr], M[tr])
    x, R = targets(Gt, Mt)
    t1 = time.time()
    net, train_loss = train(x, R, steps=train_steps, seed=seed, batch=1024)
    t_train = time.time() - t1
    rel = held_out_error(net, geoms[val], M[val])
    if out:
        save_params(net, out)
    taus = np.array([s["tau"] for s in samples])
    summary = {"samples": len(samples), "augmented": int(len(Gt)), "train_loss": train_loss,
               "converged": int(conv.sum()), "steps_used_median": int(np.median(used)),
               "steps_used_max": int(used.max()),
               "steps_used_by_tau": {f"{lo:.1f}-{lo + 0.3:.1f}": int(np.median(used[(taus >= lo) & (taus < lo + 0.3)]))
                                     for lo in (0.6, 0.9, 1.2) if ((taus >= lo) & (taus < lo + 0.3)).any()},
               "val_rel_err_median": float(np.median(rel)), "val_rel_err_max": float(rel.max()),
               "seconds": {"data": t_data, "train": t_train}}
    return net, summary


if __name__ == "__main__":
    import json
    import sys

    args = sys.argv[1:]
    cmd = args.pop(0) if args and "=" not in args[0] else "experiment"
    kw = {}
    for a in args:
        k, v = a.split("=", 1)
        try:
            kw[k] = int(v)
        except ValueError:
            try:
                kw[k] = float(v)
            except ValueError:
                kw[k] = v
    if cmd == "config5":
        ev_kw = {k[3:]: kw.pop(k) for k in list(kw) if k.startswith("ev.")}   # evaluate()'s arguments
        net, summ = config5(**kw)
        summ["evaluation"] = evaluate(net, aspect=(1.0, 4.0), b_range=(3.0, 5.0), **ev_kw)
        print(json.dumps(summ))
    elif cmd == "evaluate":
        net = load_params(kw.pop("weights"))
        print(json.dumps(evaluate(net, **kw)))
    else:
        print(json.dumps(experiment(**kw)))
