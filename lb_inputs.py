"""Seeded synthetic workloads, shared by the oracle tests and the CUDA path.

This module holds no arithmetic of the method: it only draws random numbers
and fills in the parameters of each workload (box sizes, relaxation time,
particle semi-axes, positions, orientations, forces).  Both sides receive the
same plain dictionaries:

  box      = dict(nx, ny, nz, tau, rho0, body_force, counter_force, walls,
                  wall_u_lo, wall_u_hi, didt_mode)
  particle = dict(semi, x, q, U, Om, density, F_ext, T_ext, B1, B2)

Workloads (all D3Q19, lattice units, rho0 = 1, fluid initially at rest):
  single_32     32^3 periodic, tau = 1, one prolate spheroid (4,2,2), density 1,
                centre = box centre + U(-0.5,0.5)^3, random unit quaternion,
                F_ext = (1e-4, 0, 0) with the opposite force spread over the fluid.
  sweep_8x64    8 periodic 64^3 boxes, tau = 0.8, spheroid (8,4,4), long axis at
                theta in {0,15,...,90, random} degrees to the force, |F| = 5e-4.
  shear_channel 128 x 64 x 128, walls at y = 0 and y = 63 moving at -/+0.01 in x.
  squirmer_batch 32 periodic cubes, edges drawn from {48,64,96,128}, squirmer (6,3,3).
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(seed))


def random_quaternion(g: np.random.Generator) -> list:
    """Uniform random unit quaternion (q0, q1, q2, q3) by Shoemake's subgroup
    algorithm (Graphics Gems III, 1992): three uniforms u1, u2, u3."""
    u1, u2, u3 = g.random(3)
    a, b = math.sqrt(1.0 - u1), math.sqrt(u1)
    t1, t2 = 2.0 * math.pi * u2, 2.0 * math.pi * u3
    q = [b * math.cos(t2), a * math.sin(t1), a * math.cos(t1), b * math.sin(t2)]
    if q[0] < 0.0:
        q = [-v for v in q]
    return q


def axis_angle_quaternion(axis, angle: float) -> list:
    """Unit quaternion of a rotation by `angle` about `axis`."""
    ax = np.asarray(axis, dtype=np.float64)
    ax = ax / np.linalg.norm(ax)
    s = math.sin(0.5 * angle)
    return [math.cos(0.5 * angle), s * ax[0], s * ax[1], s * ax[2]]


def box(nx, ny, nz, tau, rho0=1.0, body_force=(0.0, 0.0, 0.0), counter_force=0, walls=0,
        wall_u_lo=(0.0, 0.0, 0.0), wall_u_hi=(0.0, 0.0, 0.0), didt_mode=0, lub_cut=0.0, collision=0) -> dict:
    return dict(nx=int(nx), ny=int(ny), nz=int(nz), tau=float(tau), rho0=float(rho0),
                body_force=list(map(float, body_force)), counter_force=int(counter_force),
                walls=int(walls), wall_u_lo=list(map(float, wall_u_lo)),
                wall_u_hi=list(map(float, wall_u_hi)), didt_mode=int(didt_mode), lub_cut=float(lub_cut),
                collision=int(collision))


def particle(semi, x, q=(1.0, 0.0, 0.0, 0.0), U=(0.0, 0.0, 0.0), Om=(0.0, 0.0, 0.0), density=1.0,
             F_ext=(0.0, 0.0, 0.0), T_ext=(0.0, 0.0, 0.0), B1=0.0, B2=0.0) -> dict:
    return dict(semi=list(map(float, semi)), x=list(map(float, x)), q=list(map(float, q)),
                U=list(map(float, U)), Om=list(map(float, Om)), density=float(density),
                F_ext=list(map(float, F_ext)), T_ext=list(map(float, T_ext)),
                B1=float(B1), B2=float(B2))


def single_32(seed: int = 0, n: int = 32, semi=(4.0, 2.0, 2.0), force=1e-4, tau=1.0):
    """One spheroid in a periodic n^3 box with a counter body force."""
    g = rng(seed)
    centre = [0.5 * n + v for v in g.uniform(-0.5, 0.5, size=3)]
    q = random_quaternion(g)
    b = box(n, n, n, tau, counter_force=1)
    p = particle(semi, centre, q, F_ext=(force, 0.0, 0.0))
    return [b], [[p]]


SWEEP_ANGLES = (0.0, 15.0, 30.0, 45.0, 60.0, 75.0, 90.0, None)


def sweep_8x64(seed: int = 0, n: int = 64, semi=(8.0, 4.0, 4.0), force=5e-4, tau=0.8):
    """Eight boxes; the long axis of box k sits at SWEEP_ANGLES[k] to the force
    (the last one random); every centre is jittered by U(-0.5,0.5)^3."""
    g = rng(seed)
    boxes, parts = [], []
    for ang in SWEEP_ANGLES:
        centre = [0.5 * n + v for v in g.uniform(-0.5, 0.5, size=3)]
        if ang is None:
            q = random_quaternion(g)
        else:
            q = axis_angle_quaternion((0.0, 0.0, 1.0), math.radians(ang))
        boxes.append(box(n, n, n, tau, counter_force=1))
        parts.append([particle(semi, centre, q, F_ext=(force, 0.0, 0.0))])
    return boxes, parts


def shear_channel(seed: int = 0, semi=(8.0, 4.0, 4.0), nx=128, ny=64, nz=128, u_wall=0.01, tau=1.0):
    """Walls at y = 0 and y = ny-1 moving at -u_wall and +u_wall along x, one
    neutrally buoyant spheroid at the centre, orientation drawn off the vorticity
    axis (z)."""
    g = rng(seed)
    while True:
        q = random_quaternion(g)
        # body x axis = first column of the rotation; keep it away from z
        ez = 2.0 * (q[1] * q[3] - q[0] * q[2])
        if abs(ez) < 0.9:
            break
    centre = [0.5 * nx, 0.5 * (ny - 1), 0.5 * nz]
    b = box(nx, ny, nz, tau, walls=1, wall_u_lo=(-u_wall, 0, 0), wall_u_hi=(u_wall, 0, 0))
    return [b], [[particle(semi, centre, q)]]


def squirmer_batch(seed: int = 0, nbox: int = 32, edges=(48, 64, 96, 128), semi=(6.0, 3.0, 3.0),
                   B1=1e-3, betas=(-2.0, 0.0, 2.0), tau=1.0):
    g = rng(seed)
    boxes, parts = [], []
    for _ in range(nbox):
        n = int(g.choice(edges))
        beta = float(g.choice(betas))
        centre = [0.5 * n + v for v in g.uniform(-0.5, 0.5, size=3)]
        q = random_quaternion(g)
        boxes.append(box(n, n, n, tau))
        parts.append([particle(semi, centre, q, B1=B1, B2=beta * B1)])
    return boxes, parts


def random_pose(g: np.random.Generator, n: int, margin: float):
    """Random centre inside [margin, n - margin)^3 (or anywhere if margin <= 0,
    to exercise periodic wrap) and a random unit quaternion."""
    if margin > 0:
        c = g.uniform(margin, n - margin, size=3)
    else:
        c = g.uniform(0.0, n, size=3)
    return [float(v) for v in c], random_quaternion(g)


def unit_vector(g: np.random.Generator) -> list:
    """Uniform random direction (normalised Gaussian triple)."""
    v = g.normal(0.0, 1.0, 3)
    return [float(x) for x in v / np.linalg.norm(v)]


def long_axis_quaternion(e) -> list:
    """A unit quaternion turning the body x axis onto the unit vector e (the
    roll about e is irrelevant for a spheroid with b = c)."""
    e = np.asarray(e, np.float64)
    ax = np.cross([1.0, 0.0, 0.0], e)
    s = np.linalg.norm(ax)
    if s < 1e-12:
        return [1.0, 0.0, 0.0, 0.0] if e[0] > 0 else [0.0, 0.0, 0.0, 1.0]
    return axis_angle_quaternion(ax, math.atan2(s, e[0]))


def resistance_samples(seed: int, n: int, L: int, taus=(0.8, 1.0, 1.2), aspect=(1.0, 3.0), b_range=(2.0, 3.5),
                       tau_range=None):
    """n spheroids for resistance runs in periodic L^3 boxes: aspect ratio
    r = a/b and b uniform in the ranges, tau drawn from taus (or uniform in
    tau_range when given), long axis e uniform on the sphere, centre = box
    centre + U(-0.5,0.5)^3.  The surrogate workload's training set is
    resistance_samples(seed, 2000, 64, tau_range=(0.6, 1.5), aspect=(1, 4),
    b_range=(3, 5))."""
    g = rng(seed)
    out = []
    for _ in range(n):
        r = float(g.uniform(*aspect))
        b = float(g.uniform(*b_range))
        tau = float(g.uniform(*tau_range)) if tau_range is not None else float(g.choice(taus))
        e = unit_vector(g)
        centre = [0.5 * L + v for v in g.uniform(-0.5, 0.5, size=3)]
        out.append(dict(a=r * b, b=b, tau=tau, L=int(L), e=e, q=long_axis_quaternion(e), x=centre))
    return out


def many_spheroids(seed: int = 0, n: int = 128, count: int = 16, aspect=(1.5, 2.5), b_range=(2.5, 3.0),
                   force=2e-5, tau=1.0, gap: int = 2, max_semi=None, margin: int = 2):
    """`count` spheroids in one periodic n^3 box with random orientations and
    external forces of magnitude `force` in random directions (counter body
    force on the fluid).  Sizes first (aspect ratio and b uniform in the
    ranges), then centres by rejection sampling so that the bounding cubes,
    of side 2 (ceil(semi) + margin) + 2 (or of the common max_semi when
    given), keep `gap` nodes between them (periodically)."""
    g = rng(seed)
    sizes = []
    for _ in range(count):
        r = float(g.uniform(*aspect))
        b = float(g.uniform(*b_range))
        sizes.append((r * b, b))
    side = [2 * (int(math.ceil(a if max_semi is None else max_semi)) + margin) + 2 for a, _ in sizes]
    centres = []
    for k in range(count):
        for _ in range(100000):
            c = g.uniform(0.0, n, size=3)
            ok = True
            for j, d in enumerate(centres):
                dd = np.abs(c - d)
                dd = np.minimum(dd, n - dd)
                if np.all(dd < 0.5 * (side[k] + side[j]) + gap):
                    ok = False
                    break
            if ok:
                centres.append(c)
                break
        else:
            raise RuntimeError("no room for the spheroids")
    parts = []
    for (a, b), c in zip(sizes, centres):
        e = unit_vector(g)
        f = unit_vector(g)
        parts.append(particle((a, b, b), [float(v) for v in c], long_axis_quaternion(e),
                              F_ext=[force * v for v in f]))
    return [box(n, n, n, tau, counter_force=1)], [parts]
