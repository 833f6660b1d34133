"""Pins of the oracle's lattice, equilibrium and fluid update (Sec. II.A, Eq. 1-4).

Each check is fixed by mathematics the paper relies on, not by the oracle:
isotropy of the D3Q19 weights, the moments that Eq. 4 is built to reproduce,
the viscosity relation nu = (tau - 1/2)/3, exact conservation, and the exactness
of half-way bounce-back for linear (Couette) flow.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O
from lb_inputs import box


def test_d3q19_velocity_set():
    c, w = O.lattice()
    vecs = {tuple(v) for v in c}
    assert len(vecs) == 19
    lens = sorted(int(np.dot(v, v)) for v in c)
    assert lens.count(0) == 1 and lens.count(1) == 6 and lens.count(2) == 12
    for v, wi in zip(c, w):
        assert wi == {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}[int(np.dot(v, v))]


def test_d3q19_isotropy():
    c, w = O.lattice()
    c = c.astype(float)
    d = np.eye(3)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs(np.einsum("i,ia->a", w, c)).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib->ab", w, c, c) - d / 3.0).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib,ic->abc", w, c, c, c)).max() < 1e-15
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.abs(m4 - iso).max() < 1e-15


@pytest.mark.parametrize("rho,u", [(1.0, (0, 0, 0)), (1.03, (0.01, -0.02, 0.005)), (0.97, (-0.03, 0.0, 0.04))])
def test_equilibrium_moments(rho, u):
    """Eq. 4 reproduces rho, rho u and rho (c_s^2 I + u u) exactly (Eq. 1-2)."""
    c, _ = O.lattice()
    c = c.astype(float)
    f = O.feq(rho, u)
    u = np.asarray(u, float)
    assert abs(f.sum() - rho) < 1e-14
    assert np.abs(f @ c - rho * u).max() < 1e-15
    P = np.einsum("i,ia,ib->ab", f, c, c)
    assert np.abs(P - rho * (np.eye(3) / 3.0 + np.outer(u, u))).max() < 1e-14


def _shear_wave_rate(tau, ny=64, steps=400, U0=1e-4):
    c, w = O.lattice()
    b = box(2, ny, 2, tau)
    s = O.Sim(b, [], nthreads=1)
    y = np.arange(ny)
    f = np.zeros((2, ny, 2, 19))
    for j in range(ny):
        f[:, j, :, :] = O.feq(1.0, (U0 * math.sin(2 * math.pi * j / ny), 0.0, 0.0))
    s.set_f(f.ravel())
    basis = np.sin(2 * math.pi * y / ny)
    amps = []
    for _ in range(steps):
        s.step(1)
        _, u = s.moments()
        amps.append(2.0 / ny * (u[0, :, 0, 0] @ basis))
    amps = np.array(amps)
    t = np.arange(1, steps + 1)
    sl = slice(50, None)  # skip the start-up transient of the f_eq initialisation
    rate = -np.polyfit(t[sl], np.log(amps[sl]), 1)[0]
    return rate / (2 * math.pi / ny) ** 2


@pytest.mark.parametrize("tau", [0.8, 1.0, 1.4])
def test_shear_wave_viscosity(tau):
    """Decay of u_x = U0 sin(k y) is exp(-nu k^2 t), nu = (tau - 1/2)/3 (Sec. II.A)."""
    nu = _shear_wave_rate(tau)
    assert abs(nu / ((tau - 0.5) / 3.0) - 1.0) < 5e-3


def test_conservation_no_particle():
    """Without particles or force, total mass and momentum are exact invariants."""
    g = np.random.default_rng(1)
    b = box(6, 5, 7, 0.77)
    s = O.Sim(b, [], nthreads=2)
    _, w = O.lattice()
    f = w[None, :] * (1.0 + 0.01 * g.standard_normal((6 * 5 * 7, 19)))
    s.set_f(f.ravel())
    m0, p0 = s.fluid_mass(), s.fluid_momentum()
    s.step(40)
    assert abs(s.fluid_mass() - m0) < 1e-12 * m0
    assert np.abs(s.fluid_momentum() - p0).max() < 1e-13


def test_tau_one_relaxes_to_equilibrium_and_streams_along_c():
    """At tau = 1 the post-collision state is f_eq, which then moves along +c_i
    (Eq. 3): f_i(x, 1) = f_eq_i(rho, u at x - c_i)."""
    g = np.random.default_rng(2)
    n = (5, 4, 3)
    b = box(*n, 1.0)
    s = O.Sim(b, [], nthreads=1)
    c, w = O.lattice()
    f0 = w[None, :] * (1.0 + 0.02 * g.standard_normal((n[0] * n[1] * n[2], 19)))
    s.set_f(f0.ravel())
    rho, u = s.moments()
    s.step(1)
    f1 = s.f()
    for z, y, x in itertools.product(range(n[2]), range(n[1]), range(n[0])):
        for i in range(19):
            xs, ys, zs = (x - c[i, 0]) % n[0], (y - c[i, 1]) % n[1], (z - c[i, 2]) % n[2]
            fe = O.feq(rho[zs, ys, xs], u[zs, ys, xs])[i]
            assert abs(f1[z, y, x, i] - fe) < 1e-15


def test_body_force_momentum_per_step():
    """Guo forcing adds exactly g per fluid node per step and no mass."""
    g3 = np.array([1e-5, -2e-5, 3e-6])
    b = box(4, 6, 5, 0.9, body_force=g3)
    s = O.Sim(b, [], nthreads=1)
    m0, p0 = s.fluid_mass(), s.fluid_momentum()
    s.step(7)
    N = 4 * 6 * 5
    assert abs(s.fluid_mass() - m0) < 1e-12
    assert np.abs(s.fluid_momentum() - (p0 + 7 * N * g3)).max() < 1e-14


@pytest.mark.parametrize("tau", [0.7, 1.0, 1.6])
def test_couette_profile_exact(tau):
    """Half-way bounce-back on moving walls gives the exact linear profile, walls
    half a link outside the first fluid node (Sec. II.B, link bounce-back)."""
    ny, uw = 10, 0.01
    b = box(2, ny, 2, tau, walls=1, wall_u_lo=(-uw, 0, 0), wall_u_hi=(uw, 0, 0))
    s = O.Sim(b, [], nthreads=1)
    s.step(6000)
    _, u = s.moments()
    y = np.arange(1, ny - 1)
    expect = -uw + 2 * uw * (y - 0.5) / (ny - 2)
    assert np.abs(u[0, 1:ny - 1, 0, 0] - expect).max() < 1e-10
    assert np.abs(u[0, 1:ny - 1, 0, 1:]).max() < 1e-13


# ---------------------------------------------------------------------------
# The paper's collision (Sec. II.A: one relaxation time for the non-conserved
# hydrodynamic modes, instantaneous relaxation of the non-hydrodynamic ones),
# box option collision = 1.

def _uniform_collision(tau, collision, g=(2e-5, -1e-5, 3e-5), seed=3):
    """One step of a spatially uniform random non-equilibrium state in a
    periodic box: streaming maps the uniform post-collision state onto itself,
    so f(t+1) is the post-collision distribution of every node."""
    c, w = O.lattice()
    rng = np.random.default_rng(seed)
    f0 = O.feq(1.02, (0.01, -0.02, 0.015)) + 1e-3 * w * rng.standard_normal(19)
    b = box(3, 3, 3, tau, body_force=g, collision=collision)
    s = O.Sim(b, [], nthreads=1)
    s.set_f(np.tile(f0, 27))
    s.step(1)
    return f0, s.f()[0, 0, 0]


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.4])
def test_ghost_mode_collision_keeps_only_the_relaxed_stress(tau):
    c, w = O.lattice()
    c = c.astype(float)
    g = np.array([2e-5, -1e-5, 3e-5])
    f0, fs = _uniform_collision(tau, 1, g)
    rho = f0.sum()
    u = (f0 @ c + 0.5 * g) / rho
    feq = O.feq(rho, u)
    S = (1 - 0.5 / tau) * w * (3 * (c @ g - u @ g) + 9 * (c @ u) * (c @ g))
    d = fs - feq - S
    # the hydrodynamic Hermite modes of D3Q19 beyond mass: w_i c_ia and
    # w_i (c_ia c_ib - delta_ab / 3)
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    H = np.stack([w * c[:, a] for a in range(3)] +
                 [w * (c[:, a] * c[:, b] - (a == b) / 3.0) for a, b in pairs], axis=1)
    coef, *_ = np.linalg.lstsq(H, d, rcond=None)
    assert np.abs(d - H @ coef).max() < 1e-15                     # no ghost content left
    Pn = np.einsum("i,ia,ib->ab", f0 - feq, c, c)
    Ps = np.einsum("i,ia,ib->ab", d, c, c)
    assert np.abs(Ps - (1 - 1 / tau) * Pn).max() < 1e-15          # the stress relaxed by 1 - 1/tau
    assert np.abs(d @ c - (1 - 1 / tau) * ((f0 - feq) @ c)).max() < 1e-16
    assert abs(fs.sum() - rho) < 1e-15
    assert np.abs(fs @ c - (f0 @ c + g)).max() < 1e-15            # momentum + the force
    # BGK keeps (1 - 1/tau) of the ghost content of f - feq, so the two differ
    _, fb = _uniform_collision(tau, 0, g)
    db = fb - feq - S
    cb, *_ = np.linalg.lstsq(H, db, rcond=None)
    assert np.abs(db - H @ cb).max() > 1e-6 * abs(1 - 1 / tau)


def test_ghost_mode_collision_equals_bgk_at_tau_one():
    _, f1 = _uniform_collision(1.0, 1)
    _, f0 = _uniform_collision(1.0, 0)
    assert np.abs(f1 - f0).max() < 1e-16


@pytest.mark.parametrize("tau", [0.8, 1.4])
def test_ghost_mode_collision_viscosity(tau):
    """The shear viscosity is still (tau - 1/2)/3: the shear-wave decay."""
    c, w = O.lattice()
    ny, U0 = 64, 1e-4
    b = box(2, ny, 2, tau, collision=1)
    s = O.Sim(b, [], nthreads=1)
    f = np.zeros((2, ny, 2, 19))
    for j in range(ny):
        f[:, j, :, :] = O.feq(1.0, (U0 * math.sin(2 * math.pi * j / ny), 0.0, 0.0))
    s.set_f(f.ravel())
    basis = np.sin(2 * math.pi * np.arange(ny) / ny)
    amps = []
    for _ in range(400):
        s.step(1)
        amps.append(2.0 / ny * (s.moments()[1][0, :, 0, 0] @ basis))
    t = np.arange(1, 401)
    rate = -np.polyfit(t[50:], np.log(np.array(amps)[50:]), 1)[0] / (2 * math.pi / ny) ** 2
    assert abs(rate / ((tau - 0.5) / 3.0) - 1.0) < 0.005
