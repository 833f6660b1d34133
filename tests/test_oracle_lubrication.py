"""Pins of the oracle's lubrication correction between close particles (the
Nguyen-Ladd correction of the moving-boundary method the paper builds on,
Sec. II.B).  Readings (oracle/lb_oracle.c, orc_lubrication_pair): gap and radii
along the line of centres, R(n) = (n^T A n)^(-1/2) with A of
Eq. ellipsoidsurface; below the cut-off gap h_c the squeeze force of two
spheres of radii R_p, R_q that the lattice no longer resolves,
-6 pi mu R^2 (1/h - 1/h_c) (n . (U_p - U_q)) n with R = R_p R_q / (R_p + R_q), is
added; h >= 0.1; explicit, antisymmetric, its coefficient capped at the
reduced mass.

Pinned by:
  * closed forms of the geometry (sphere gap |d| - 2a; a spheroid's radius a
    along its axis and b across it) and of the force's structure
    (antisymmetry, no tangential part, zero beyond h_c, the cap);
  * combined momentum conserved to round-off with two particles inside the
    cut-off (internal forces);
  * the squeeze flow of two spheres approaching at a fixed speed: between
    gaps of 0.55 and 0.30 lattice units the corrected force grows as the
    asymptotic two-sphere resistance 6 pi mu a (V_rel/2) (a/(2h) + (9/20)
    ln(a/h)) (Brenner 1961; Jeffrey and Onishi 1984) does, within 25 %, while
    the uncorrected lattice force has levelled off (below half of that
    growth; below a gap of about a quarter node the lattice force is no longer
    a squeeze force at all).
"""
import math

import numpy as np
import pytest

from lb_inputs import box, particle, random_quaternion, rng
from oracle import oracle as O

MU = 1.0 / 6.0


def _body(semi, x, q=(1, 0, 0, 0), U=(0, 0, 0), M=100.0):
    return dict(semi=semi, x=x, q=q, U=U, M=M)


def test_gap_and_radii_closed_forms():
    L = (64, 64, 64)
    a = 3.5
    f, h = O.lubrication_pair(_body((a, a, a), (10, 10, 10)), _body((a, a, a), (10, 17.3, 10)), L, MU, 1.0)
    assert abs(h - (7.3 - 2 * a)) < 1e-14
    # spheroid (6, 3, 3): radius a along its axis, b across it
    _, h = O.lubrication_pair(_body((6.0, 3.0, 3.0), (10, 10, 10)), _body((2.0, 2.0, 2.0), (18.5, 10, 10)), L, MU, 1.0)
    assert abs(h - (8.5 - 6.0 - 2.0)) < 1e-14
    _, h = O.lubrication_pair(_body((6.0, 3.0, 3.0), (10, 10, 10)), _body((2.0, 2.0, 2.0), (10, 10, 15.5)), L, MU, 1.0)
    assert abs(h - (5.5 - 3.0 - 2.0)) < 1e-14
    # the same spheroid turned by 90 degrees about z: its axis along y
    qz = [math.cos(math.pi / 4), 0.0, 0.0, math.sin(math.pi / 4)]
    _, h = O.lubrication_pair(_body((6.0, 3.0, 3.0), (10, 10, 10), q=qz), _body((2.0, 2.0, 2.0), (10, 18.5, 10)),
                              L, MU, 1.0)
    assert abs(h - 0.5) < 1e-12
    # minimum image across the periodic boundary
    _, h = O.lubrication_pair(_body((a, a, a), (1.0, 5, 5)), _body((a, a, a), (57.5, 5, 5)), L, MU, 1.0)
    assert abs(h - (7.5 - 2 * a)) < 1e-12


def test_force_structure():
    L = (64, 64, 64)
    g = rng(40)
    A = _body((4.0, 2.5, 2.0), [20.0, 20.0, 20.0], random_quaternion(g), U=[1e-3, -2e-3, 5e-4], M=80.0)
    B = _body((3.0, 3.0, 2.0), [20.0, 26.0, 21.0], random_quaternion(g), U=[-1e-3, 1e-3, 0.0], M=50.0)
    fa, h = O.lubrication_pair(A, B, L, MU, 2.0)
    fb, hb = O.lubrication_pair(B, A, L, MU, 2.0)
    assert 0.0 < h < 2.0 and abs(h - hb) < 1e-12
    assert np.allclose(fa, -fb, rtol=0, atol=1e-18)          # equal and opposite
    n = (np.array(B["x"]) - np.array(A["x"])) / np.linalg.norm(np.array(B["x"]) - np.array(A["x"]))
    assert np.linalg.norm(np.cross(fa, n)) < 1e-15 * np.linalg.norm(fa)   # along the line of centres
    vn = n @ (np.array(A["U"]) - np.array(B["U"]))
    assert abs(vn) > 1e-4 and -(fa @ n) / vn > 0           # opposes the normal relative motion
    # a tangential relative velocity gives none
    At = dict(A, U=list(np.array(B["U"]) + np.cross(n, [0.3, -0.2, 0.9]) * 1e-3))
    ft, _ = O.lubrication_pair(At, B, L, MU, 2.0)
    assert np.abs(ft).max() < 1e-18
    # none beyond the cut-off
    f0, _ = O.lubrication_pair(A, B, L, MU, 0.5 * h)
    assert np.abs(f0).max() == 0.0
    # capped at the reduced mass for very light bodies (stops the approach in one step)
    fl, _ = O.lubrication_pair(dict(A, M=1e-3), dict(B, M=1e-3), L, MU, 2.0)
    assert abs(-(fl @ n) / vn - 0.5e-3) < 1e-15


def test_momentum_conserved_with_lubrication():
    g = rng(41)
    b = box(28, 24, 24, 0.9, lub_cut=2.0 / 3.0)
    p1 = particle((4.0, 2.5, 2.5), (9.3, 11.8, 12.1), random_quaternion(g), U=(0.004, 0.0, 0.0), density=2.0)
    p2 = particle((3.0, 3.0, 3.0), (17.6, 12.4, 11.7), random_quaternion(g), U=(-0.004, 0.001, 0.0), density=2.0)
    s = O.Sim(b, [p1, p2], nthreads=2)

    def total():
        P = s.fluid_momentum().copy()
        for p in range(2):
            P += s.mass(p) * s.particle(p)["U"] + s.pending(p)[0]
        return P

    P0 = total()
    for _ in range(40):
        s.step(1)
        assert np.abs(total() - P0).max() < 1e-12 * np.abs(P0).max()


def _squeeze(cut, a=4.0, V=0.002, h0=1.5, steps=320):
    b = box(48, 32, 32, 1.0, lub_cut=cut)
    pa = particle((a, a, a), (24 - a - h0 / 2 + 0.13, 16.2, 15.9), U=(V, 0, 0), density=1e7)
    pb = particle((a, a, a), (24 + a + h0 / 2 + 0.13, 16.2, 15.9), U=(-V, 0, 0), density=1e7)
    s = O.Sim(b, [pa, pb], nthreads=8)
    hs, F = [], []
    for _ in range(steps):
        s.step(1)
        A, B = s.particle(0), s.particle(1)
        hs.append(B["x"][0] - A["x"][0] - 2 * a)
        F.append(A["F"][0])
    return np.array(hs), np.array(F)


def _mean_near(hs, F, h, w=0.025):
    sel = np.abs(hs - h) < w
    assert sel.sum() >= 5
    return float(F[sel].mean())


@pytest.mark.slow
def test_squeeze_flow_of_two_spheres_follows_the_lubrication_law():
    a, V = 4.0, 0.002
    full = lambda h: -6 * math.pi * MU * a * V * (a / (2 * h) + 0.45 * math.log(a / h))
    h1, h2 = 0.55, 0.30
    want = full(h2) - full(h1)
    hs, F = _squeeze(2.0 / 3.0)
    got = _mean_near(hs, F, h2) - _mean_near(hs, F, h1)
    hs0, F0 = _squeeze(0.0)
    got0 = _mean_near(hs0, F0, h2) - _mean_near(hs0, F0, h1)
    print("force increase", got, "asymptotic law", want, "uncorrected", got0)
    assert want < 0 and abs(got / want - 1.0) < 0.25
    assert abs(got0) < abs(want) / 2
