"""Pins of the oracle's fluid-particle coupling (Sec. II.B-C, Appendix steps 3-9).

Fixed by the method's own conservation laws rather than by the oracle's code:
  * combined momentum of fluid + particle (+ the pending remap impulse) is
    conserved exactly, with or without nodes being covered and uncovered
    (Sec. II.B: "combined momentum ... is conserved");
  * fluid mass is conserved around a particle at rest;
  * the drag matrices of Eq. drag1-drag4 form one symmetric positive
    semi-definite 6x6 matrix, isotropic for a sphere centred on a node;
  * the new velocities satisfy Eq. Fdiscrete / Eq. Tdiscrete.
"""
import numpy as np
import pytest

from oracle import oracle as O
from lb_inputs import box, particle, rng, random_quaternion


def _total_momentum(s):
    P = s.fluid_momentum().copy()
    for p in range(s.np):
        st = s.particle(p)
        dP = s.pending(p)[0]
        P += s.mass(p) * st["U"] + dP
    return P


@pytest.mark.parametrize("semi", [(3.5, 3.5, 3.5), (4.5, 2.5, 2.0)])
def test_momentum_conserved_with_cover_uncover(semi):
    """A fast particle crossing many nodes: fluid + particle + pending impulse is
    constant to round-off (the remap's covered/uncovered bookkeeping included)."""
    g = rng(3)
    s = O.Sim(box(20, 18, 22, 0.9), [particle(semi, (10.3, 9.1, 11.7), random_quaternion(g),
                                               U=(0.03, -0.02, 0.025), Om=(0.004, 0.006, -0.005),
                                               density=5.0)],
              nthreads=2)
    P0 = _total_momentum(s)
    changed = 0
    for _ in range(60):
        own = s.owner()
        s.step(1)
        changed += int((s.owner() != own).sum())
        assert np.abs(_total_momentum(s) - P0).max() < 1e-12 * np.abs(P0).max()
    assert changed > 20  # the particle really covered and uncovered nodes


def test_momentum_conserved_with_external_and_counter_force():
    s = O.Sim(box(16, 16, 16, 1.0, counter_force=1),
              [particle((4.0, 2.0, 2.0), (8.2, 7.9, 8.4), random_quaternion(rng(4)), F_ext=(1e-3, -2e-3, 5e-4))],
              nthreads=2)
    for _ in range(10):
        s.step(10)
        # round-off of summing N*19 populations of order w_i (total mass 4096)
        assert np.abs(_total_momentum(s)).max() < 1e-12


def test_fluid_mass_conserved_around_resting_particle():
    g = rng(5)
    s = O.Sim(box(14, 14, 14, 0.8), [particle((4.0, 3.0, 2.5), (7.1, 6.8, 7.3), random_quaternion(g),
                                               density=1e12)], nthreads=2)
    _, w = O.lattice()
    own = s.owner().ravel()
    f = w[None, :] * (1.0 + 0.01 * g.standard_normal((own.size, 19)))
    s.set_f(f.ravel())
    m0 = s.fluid_mass()
    s.step(50)
    assert abs(s.fluid_mass() - m0) < 1e-10 * m0


@pytest.mark.parametrize("seed", range(4))
def test_drag_matrix_symmetric_psd(seed):
    g = rng(60 + seed)
    semi = [float(v) for v in g.uniform(2.0, 5.0, 3)]
    s = O.Sim(box(18, 18, 18, 1.0), [particle(semi, g.uniform(0, 18, 3), random_quaternion(g))], nthreads=2)
    Z = s.zeta(0)
    assert np.allclose(Z, Z.T, atol=1e-12)
    assert np.linalg.eigvalsh(Z).min() > -1e-10
    assert np.allclose(Z[3:, :3], Z[:3, 3:].T, atol=1e-12)


def test_drag_matrix_sphere_isotropic():
    s = O.Sim(box(17, 17, 17, 1.0), [particle((4.2, 4.2, 4.2), (8, 8, 8))], nthreads=1)
    Z = s.zeta(0)
    k = Z[0, 0]
    assert k > 0
    assert np.allclose(Z[:3, :3], k * np.eye(3), atol=1e-12)
    assert np.abs(Z[:3, 3:]).max() < 1e-12
    assert np.allclose(Z[3:, 3:], Z[3, 3] * np.eye(3), atol=1e-10)
    # zeta^{FU} = (2 rho0 / c_s^2) sum_b w_b c_b c_b: its trace is 6 * sum_b w_b |c_b|^2
    node, cv = s.links()
    w = np.array([{1: 1 / 18, 2: 1 / 36}[int(v @ v)] for v in cv])
    assert abs(np.trace(Z[:3, :3]) - 6.0 * (w * (cv * cv).sum(1)).sum()) < 1e-10


def test_implicit_update_satisfies_discrete_equations():
    """U(t+1), Omega(t+1) satisfy Eq. Fdiscrete / Eq. Tdiscrete with the reported
    F = F0 - zeta U' - zeta Omega' and the analytic dI/dt (dt = 1)."""
    g = rng(6)
    Fe, Te = np.array([2e-4, -1e-4, 3e-4]), np.array([1e-3, 2e-3, -1e-3])
    s = O.Sim(box(18, 18, 18, 0.9), [particle((5.0, 2.5, 2.0), (9.3, 8.7, 9.1), random_quaternion(g),
                                               F_ext=Fe, T_ext=Te, Om=(0.001, -0.002, 0.0015))], nthreads=2)
    s.step(3)
    for _ in range(3):
        before = s.particle(0)
        dP, dL = s.pending(0)[:2]
        s.step(1)
        after = s.particle(0)
        M = s.mass(0)
        assert np.allclose(M * (after["U"] - before["U"]), after["F"] + Fe + dP, rtol=0, atol=1e-14)
        a, b, c = 5.0, 2.5, 2.0
        Ib = M / 5 * np.array([b * b + c * c, a * a + c * c, a * a + b * b])
        I = O.inertia_lab(before["q"], Ib)
        dI = O.inertia_rate(before["q"], before["Om"], Ib)
        lhs = I @ (after["Om"] - before["Om"]) + dI @ after["Om"]
        assert np.allclose(lhs, after["T"] + Te + dL, rtol=0, atol=1e-12)


def test_force_is_momentum_exchange_of_the_links():
    """F of Eq. Fsplit equals the fluid's momentum loss at the links: with no
    remap events and no body force, dP_fluid = -F each step (Eq. fb summed)."""
    g = rng(7)
    s = O.Sim(box(16, 16, 16, 1.0), [particle((4.0, 2.5, 2.5), (8.1, 7.7, 8.3), random_quaternion(g),
                                               F_ext=(1e-3, 0, 0), density=50.0)], nthreads=2)
    for _ in range(5):
        p0 = s.fluid_momentum()
        own0 = s.owner()
        s.step(1)
        if not np.array_equal(own0, s.owner()):
            continue
        assert np.allclose(s.fluid_momentum() - p0, -s.particle(0)["F"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("semi", [(3.5, 3.5, 3.5), (4.5, 2.5, 2.0)])
def test_fluid_mass_with_pending_remap_mass_conserved(semi):
    """Mass through covered / uncovered nodes (Appendix step 8, with the
    reading that the remap's net mass is returned uniformly, without momentum,
    at the collision two iterations later).  A fast passive particle crosses
    many nodes; each iteration:
      * the link bounce-back of a rigid body moves no mass (its w_b c_b . u_b
        terms cancel between the two ends of every lattice line through the
        solid), collision and streaming conserve it, so the fluid's mass
        changes by exactly the mass returned at this collision minus the mass
        taken by this remap;
      * the remap mass handed over for return is the previous remap's;
      * fluid mass + the two pending amounts is constant to round-off.
    A dropped or wrongly signed return, or one at another iteration, breaks one
    of these."""
    g = rng(31)
    s = O.Sim(box(20, 18, 22, 0.9), [particle(semi, (10.3, 9.1, 11.7), random_quaternion(g),
                                               U=(0.03, -0.02, 0.025), Om=(0.004, 0.006, -0.005),
                                               density=5.0)],
              nthreads=2)
    _, w = O.lattice()
    # start from a perturbed fluid so that covered nodes carry mass other than rho0
    own = s.owner().ravel()
    f = w[None, :] * (1.0 + 0.02 * g.standard_normal((own.size, 19)))
    s.set_f(f.ravel())
    M = [s.fluid_mass()]
    pend = [s.pending(0)]
    for _ in range(60):
        s.step(1)
        M.append(s.fluid_mass())
        pend.append(s.pending(0))
    dm = np.array([p[2] for p in pend])
    ret = np.array([p[3] for p in pend])
    M = np.array(M)
    assert np.count_nonzero(dm[1:]) > 15                      # the remap really moved mass
    assert np.abs(dm).max() > 0.5                             # whole nodes' worth
    eps = 1e-13 * M[0]
    for t in range(1, len(M)):
        assert ret[t] == dm[t - 1]                            # handed over one iteration later
        assert abs((M[t] - M[t - 1]) - (ret[t - 1] - dm[t])) < eps
        assert abs((M[t] + dm[t] + ret[t]) - (M[0] + dm[0] + ret[0])) < eps
