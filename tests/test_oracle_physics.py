"""Physics pins of the coupled oracle against the paper's closed forms (Sec. III).

Small boxes, so each check states how the closed form is used:
  * rotation in simple shear: a sphere spins at half the vorticity; a spheroid in
    the flow-gradient plane turns at the Jeffery rates gamma/(r^2+1) (long axis
    along the flow) and gamma r^2/(r^2+1) (long axis along the gradient), Eq. jeffery;
  * sedimentation: the periodic-image correction of a Stokeslet array is
    shape independent at leading order, so U_end-on - U_broadside is compared
    with Eq. settlingvel without it, and the inclined spheroid's lateral drift
    follows from the two principal velocities (Eq. drift);
  * squirmers: swimming speed of Eq. squirmervel (sphere limit 2 B1/3),
    independent of B2.
Tolerances cover the first-order accuracy of link bounce-back at these small
radii (Sec. III.A, III.E).
"""
import math

import numpy as np
import pytest

from oracle import analytic as A
from oracle import oracle as O
from lb_inputs import axis_angle_quaternion, box, particle

pytestmark = pytest.mark.slow


def _couette_init(s, ny, uw):
    f = np.zeros((s.nz, ny, s.nx, 19))
    for y in range(ny):
        u = -uw + 2 * uw * (y - 0.5) / (ny - 2)
        f[:, y, :, :] = O.feq(1.0, (u, 0.0, 0.0))
    s.set_f(f.ravel())


def _shear_rate(semi, q, nx=32, ny=34, nz=32, uw=0.01, steps=700):
    b = box(nx, ny, nz, 1.0, walls=1, wall_u_lo=(-uw, 0, 0), wall_u_hi=(uw, 0, 0))
    s = O.Sim(b, [particle(semi, (nx / 2, (ny - 1) / 2, nz / 2), q)])
    _couette_init(s, ny, uw)
    gam = 2 * uw / (ny - 2)
    Om = []
    for _ in range(steps // 50):
        s.step(50)
        Om.append(s.particle(0)["Om"][2])
    e = O.rotate(s.particle(0)["q"], (1.0, 0.0, 0.0))
    return np.array(Om), gam, math.atan2(e[1], e[0])


def test_sphere_rotates_at_half_vorticity():
    Om, gam, _ = _shear_rate((4.0, 4.0, 4.0), (1, 0, 0, 0), steps=500)
    assert abs(Om[-1] - Om[-2]) < 0.01 * abs(Om[-1])        # steady
    assert abs(Om[-1] / (-gam / 2) - 1.0) < 0.05


def test_spheroid_jeffery_rates_in_flow_gradient_plane():
    r = 2.0

    def jeffery_rate(gam, phi):   # in-plane Eq. jeffery, phi from the flow direction
        return -gam * (r * r * math.sin(phi) ** 2 + math.cos(phi) ** 2) / (r * r + 1)

    Om_flow, gam, phi_f = _shear_rate((6.0, 3.0, 3.0), (1, 0, 0, 0))
    Om_grad, _, phi_g = _shear_rate((6.0, 3.0, 3.0), axis_angle_quaternion((0, 0, 1), math.pi / 2))
    assert -0.2 < phi_f < 0 and 1.2 < phi_g < math.pi / 2   # it turned with the vorticity
    assert abs(Om_flow[-1] / jeffery_rate(gam, phi_f) - 1.0) < 0.1
    assert abs(Om_grad[-1] / jeffery_rate(gam, phi_g) - 1.0) < 0.1
    assert 2.8 < Om_grad[-1] / Om_flow[-1] < 4.6             # about r^2 = 4


def _settle(semi, q, L=28, F=1e-4, steps=2000):
    b = box(L, L, L, 1.0, counter_force=1)
    s = O.Sim(b, [particle(semi, (L / 2 + 0.25, L / 2 - 0.125, L / 2 + 0.375), q, F_ext=(F, 0.0, 0.0))])
    hist = []
    for _ in range(steps // 100):
        s.step(100)
        hist.append(s.particle(0)["U"].copy())
    return np.array(hist), s.particle(0)


def test_sedimenting_spheroid_oberbeck_anisotropy_and_drift():
    a, b = 6.0, 3.0
    F, mu = 1e-4, 1.0 / 6.0
    end, _ = _settle((a, b, b), (1, 0, 0, 0), F=F)
    broad, _ = _settle((a, b, b), axis_angle_quaternion((0, 0, 1), math.pi / 2), F=F)
    incl, last = _settle((a, b, b), axis_angle_quaternion((0, 0, 1), math.pi / 4), F=F)
    for h in (end, broad, incl):
        assert np.abs(h[-1] - h[-2]).max() < 5e-3 * np.abs(h[-1]).max()
    cpar, cperp = A.oberbeck_coefficients(A.eccentricity(a, b))
    want = F / (6 * math.pi * mu * a) * (1 / cpar - 1 / cperp)
    got = end[-1][0] - broad[-1][0]
    assert got > 0                                           # end-on settles faster (Sec. III.A)
    assert abs(got / want - 1.0) < 0.25
    # Stokes linearity with the principal velocities of the aligned runs (how the
    # paper builds its drift prediction, Sec. III.B): at 45 degrees
    # U_x = (U_par + U_perp)/2 and the lateral drift is (U_par - U_perp)/2.  The
    # lateral part is a small difference of two discretised shapes, hence 25 %.
    assert abs(incl[-1][0] / (0.5 * (end[-1][0] + broad[-1][0])) - 1.0) < 0.015
    lateral = incl[-1][1]
    assert lateral > 0                                       # drifts towards the long axis
    assert abs(lateral / (0.5 * got) - 1.0) < 0.25
    # the inclined spheroid keeps its orientation (Sec. III.B)
    q0 = axis_angle_quaternion((0, 0, 1), math.pi / 4)
    assert np.abs(O.rotate(last["q"], (1, 0, 0)) - O.rotate(q0, (1, 0, 0))).max() < 1e-4


@pytest.mark.parametrize("semi,L", [((4.0, 4.0, 4.0), 24), ((6.0, 3.0, 3.0), 32)])
def test_squirmer_speed(semi, L):
    """The swimmer crosses nodes every few hundred steps, so its speed ripples by
    a few per cent; the pin uses the mean over steps 400-1200.  At these radii
    link bounce-back puts the slip half a link off the surface (Sec. III.E)."""
    B1 = 1e-3
    speeds = []
    for beta in (0.0, 2.0):
        b = box(L, L, L, 1.0)
        s = O.Sim(b, [particle(semi, (L / 2, L / 2, L / 2), (1, 0, 0, 0), B1=B1, B2=beta * B1)])
        s.step(400)
        U = []
        for _ in range(40):
            s.step(20)
            U.append(s.particle(0)["U"].copy())
        U = np.array(U)
        speeds.append(U[:, 0].mean())
        assert np.abs(U[:, 1:]).max() < 1e-6 * U[:, 0].mean()    # swims along +e only
    want = A.squirmer_speed(B1, semi[0], semi[1])
    assert abs(speeds[0] / want - 1.0) < 0.12
    assert abs(speeds[1] / speeds[0] - 1.0) < 0.05        # independent of B2 (Sec. III.D)


def test_closed_form_limits():
    """Sphere limits of the closed forms and the Jeffery period from Eq. jeffery."""
    cpar, cperp = A.oberbeck_coefficients(A.eccentricity(1.0, 0.9999999))
    assert abs(cpar - 1) < 1e-6 and abs(cperp - 1) < 1e-6
    assert abs(A.squirmer_speed(1.0, 1.0, 1.0) - 2 / 3) < 1e-12
    assert abs(A.squirmer_speed(1.0, 1.0, 0.99999) - 2 / 3) < 1e-4
    assert A.drift_angle(0.0, 2.0, 1.0) == 0.0
    assert abs(A.drift_angle(math.pi / 2 - 1e-9, 2.0, 1.0)) < 1e-7
    # Jeffery: integrate Eq. jeffery in the flow-gradient plane for one period
    r, gam = 2.0, 1e-2
    beta = (r * r - 1) / (r * r + 1)
    G = np.zeros((3, 3))
    G[0, 1] = gam                                            # u_x = gam * y
    T = A.jeffery_period(r, gam)
    t, e = A.jeffery_orbit([1.0, 0.0, 0.0], G, beta, T, T / 20000)
    assert np.abs(e[-1] - e[0]).max() < 1e-6
    half = np.argmin(np.abs(t - T / 2))
    assert np.abs(e[half] + e[0]).max() < 1e-3               # half a period flips the axis
    # a 3-D orbit (axis off the vorticity axis): the orbit constant is constant
    # along the integrated Eq. jeffery, and an orbit of another aspect ratio
    # does not keep it
    for r in (2.0, 3.0):
        beta = (r * r - 1) / (r * r + 1)
        T = A.jeffery_period(r, gam)
        e0 = np.array([0.5, 0.3, 0.8]) / np.linalg.norm([0.5, 0.3, 0.8])
        t, e = A.jeffery_orbit(e0, G, beta, 1.5 * T, T / 20000)
        C = A.jeffery_orbit_constant(e, r)
        assert np.ptp(C) < 1e-6 * C.mean()
        assert np.ptp(A.jeffery_orbit_constant(e, 1.1 * r)) > 0.05 * C.mean()
        assert abs(A.jeffery_aspect_from_period(T, gam) - r) < 1e-12


def _settle_sphere(a, L, F, mu_tau=1.0, tol=2e-5, max_steps=20000):
    """Steady settling velocity of a sphere under F_ext in a periodic L^3 box
    with the counter body force (zero total momentum, as in sedimentation)."""
    b = box(L, L, L, mu_tau, counter_force=1)
    s = O.Sim(b, [particle((a, a, a), (L / 2 + 0.25, L / 2 - 0.125, L / 2 + 0.375), F_ext=(F, 0.0, 0.0))])
    prev = None
    for _ in range(max_steps // 100):
        s.step(100)
        U = s.particle(0)["U"][0]
        if prev is not None and abs(U - prev) < tol * abs(U):
            return U
        prev = U
    raise AssertionError("no steady state")


def test_sphere_settling_absolute_scale_against_hasimoto():
    """Absolute drag, not a difference of orientations: the change of a
    sphere's settling velocity between two periodic boxes is fixed by the
    Stokeslet image sum (Hasimoto's constant, Sec. III.A) and the fluid's
    viscosity mu = rho0 (tau - 1/2)/3 alone; the sphere's own, discretisation-
    dependent hydrodynamic radius only enters the O((a/L)^3) terms (a +-10 %
    radius moves the expected value by under 2 %).  A wrong viscosity, force
    scale or momentum-exchange factor shows up in full."""
    a, F, mu = 3.0, 1e-4, 1.0 / 6.0
    L1, L2 = 20, 28
    U1, U2 = _settle_sphere(a, L1, F), _settle_sphere(a, L2, F)
    U0 = A.stokes_velocity(F, mu, a)
    want = U0 * (A.hasimoto_series(a, L2) - A.hasimoto_series(a, L1))
    # leading term alone, shape independent: 2.8373 F / (6 pi mu) (1/L1 - 1/L2)
    lead = A.hasimoto_velocity(F, mu, a, L2) - A.hasimoto_velocity(F, mu, a, L1)
    assert abs(want / lead - 1.0) < 0.1
    assert U2 > U1 > 0
    assert abs((U2 - U1) / want - 1.0) < 0.05
    # each box on its own, with the input radius (the hydrodynamic radius of a
    # link-bounce-back sphere of radius 3 differs by a few per cent)
    for U, Lb in ((U1, L1), (U2, L2)):
        assert abs(U / (U0 * A.hasimoto_series(a, Lb)) - 1.0) < 0.12
