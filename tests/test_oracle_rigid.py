"""Pins of the oracle's rigid-body pieces (Sec. II.C-D): quaternion product and
rotation (Eq. vectrotn), lab-frame inertia (Eq. Irot), its time derivative
(Eq. Irotdiff with Eq. qevolution), the exponential-map update (Eq. qnplus0-1)
and the Gaussian elimination used for Eq. Fdiscrete / Eq. Tdiscrete.

References are an independent rotation library (scipy), numpy's LAPACK solver,
closed forms ([Omega]x I - I [Omega]x, rotation angle n|Omega|) and finite
differences.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as O
from lb_inputs import rng, random_quaternion


def _R(q):
    return Rotation.from_quat([q[1], q[2], q[3], q[0]])


def _skew(w):
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])


@pytest.mark.parametrize("seed", range(5))
def test_rotation_matches_library(seed):
    g = rng(seed)
    q = random_quaternion(g)
    s = g.standard_normal(3)
    assert np.allclose(O.rotate(q, s), _R(q).apply(s), atol=1e-14)


@pytest.mark.parametrize("seed", range(5))
def test_hamilton_product_composes_rotations(seed):
    g = rng(10 + seed)
    a, b = random_quaternion(g), random_quaternion(g)
    ab = O.quat_mul(a, b)
    assert np.allclose(_R(ab).as_matrix(), (_R(a) * _R(b)).as_matrix(), atol=1e-14)


@pytest.mark.parametrize("seed", range(5))
def test_lab_inertia_is_R_I_RT(seed):
    g = rng(20 + seed)
    q = random_quaternion(g)
    Ib = g.uniform(1, 10, 3)
    R = _R(q).as_matrix()
    assert np.allclose(O.inertia_lab(q, Ib), R @ np.diag(Ib) @ R.T, atol=1e-12)


@pytest.mark.parametrize("seed", range(5))
def test_inertia_rate_closed_form_and_finite_difference(seed):
    """Eq. Irotdiff equals [Omega]x I - I [Omega]x and the central difference of
    Eq. Irot along q(t) = exp(Omega t / 2) q."""
    g = rng(30 + seed)
    q = random_quaternion(g)
    Om = g.standard_normal(3) * 0.3
    Ib = g.uniform(1, 10, 3)
    dI = O.inertia_rate(q, Om, Ib)
    I = O.inertia_lab(q, Ib)
    W = _skew(Om)
    assert np.allclose(dI, W @ I - I @ W, atol=1e-12)
    h = 1e-5
    qp = (Rotation.from_rotvec(Om * h) * _R(q)).as_quat()
    qm = (Rotation.from_rotvec(-Om * h) * _R(q)).as_quat()
    Ip = O.inertia_lab([qp[3], *qp[:3]], Ib)
    Im = O.inertia_lab([qm[3], *qm[:3]], Ib)
    assert np.allclose(dI, (Ip - Im) / (2 * h), atol=1e-8)
    # the backward difference of Eq. Irot (the paper's finite-difference option)
    # agrees to first order in dt
    assert np.allclose(dI, (I - Im) / h, atol=1e-4)


def test_quaternion_update_constant_rate():
    """With constant Omega the update rotates by exactly n |Omega| about Omega."""
    q0 = random_quaternion(rng(40))
    Om = np.array([0.013, -0.021, 0.007])
    q = np.array(q0)
    n = 2000
    for _ in range(n):
        q = O.quat_step(q, Om)
    want = Rotation.from_rotvec(Om * n) * _R(q0)
    assert np.allclose(_R(q).as_matrix(), want.as_matrix(), atol=1e-11)


def test_quaternion_update_unit_norm():
    """Eq. qnplus0-1 keep |q| = 1 without renormalisation (Sec. II.C)."""
    g = rng(41)
    q = np.array(random_quaternion(g))
    Oms = g.standard_normal((100000, 3)) * 0.05
    for k in range(Oms.shape[0]):
        q = O.quat_step(q, Oms[k])
    assert abs(np.linalg.norm(q) - 1.0) < 1e-13


def test_zero_rotation_is_identity():
    q = random_quaternion(rng(42))
    assert np.array_equal(O.quat_step(q, [0.0, 0.0, 0.0]), np.asarray(q))


@pytest.mark.parametrize("seed", range(5))
def test_gauss_solve_matches_lapack(seed):
    g = rng(50 + seed)
    A = g.standard_normal((6, 6)) + 6 * np.eye(6)
    b = g.standard_normal(6)
    x = O.gauss_solve(A, b)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-12, atol=1e-12)


def test_gauss_solve_needs_pivoting():
    A = np.array([[1e-20, 1.0, 0, 0, 0, 0], [1.0, 1.0, 0, 0, 0, 0]] + [[0] * i + [1.0] + [0] * (5 - i) for i in range(2, 6)])
    b = np.array([1.0, 2.0, 3, 4, 5, 6])
    assert np.allclose(O.gauss_solve(A, b), np.linalg.solve(A, b), rtol=1e-12)


def test_body_inertia_of_spheroid():
    """Sec. II.D: I = diag(M(b^2+c^2)/5, M(a^2+c^2)/5, M(a^2+b^2)/5) with
    M = density * 4/3 pi a b c (continuum volume)."""
    from lb_inputs import box, particle
    s = O.Sim(box(24, 24, 24, 1.0), [particle((5.0, 3.0, 2.0), (12, 12, 12), density=1.3)], nthreads=1)
    M = s.mass(0)
    assert abs(M - 1.3 * 4 / 3 * math.pi * 30) < 1e-12


def _free_step_L_error(mode, q, Ib, Om):
    """Relative change of the angular momentum I(q) Omega over one step of a
    free body (no drag, no torque), which the exact dynamics conserves."""
    M = 4.0
    L0 = O.inertia_lab(q, Ib) @ Om
    _, Wn = O.rigid_solve(M, Ib, q, (0, 0, 0), Om, np.zeros(36), (0, 0, 0), (0, 0, 0), mode=mode)
    qn = O.quat_step(q, 0.5 * (np.asarray(Om) + Wn))
    return float(np.linalg.norm(O.inertia_lab(qn, Ib) @ Wn - L0) / np.linalg.norm(L0))


def test_predictor_corrector_conserves_angular_momentum_to_higher_order():
    """Sec. II.D: replacing I(t+1) by I(t) + dI/dt (Eq. Irotdiff) leaves a
    one-step angular-momentum error of second order in |Omega| dt; the
    predictor-corrector (I(t+1) from the predicted orientation, Eq. Irot) is of
    third order.  Halving Omega divides the errors by 4 and by 8."""
    g = rng(21)
    q = random_quaternion(g)
    Ib = np.array([1.0, 2.0, 3.5])                      # triaxial
    ax = np.array([0.3, 1.0, -0.6]) / np.linalg.norm([0.3, 1.0, -0.6])
    e0 = [_free_step_L_error(0, q, Ib, w * ax) for w in (0.02, 0.01, 0.005)]
    e2 = [_free_step_L_error(2, q, Ib, w * ax) for w in (0.02, 0.01, 0.005)]
    for k in range(2):
        assert 3.6 < e0[k] / e0[k + 1] < 4.4
        assert 7.2 < e2[k] / e2[k + 1] < 8.8
    assert e2[0] < 0.05 * e0[0]


def test_predictor_corrector_limits():
    """An isotropic body has I(q) = I for every q: dI/dt = 0 and I(q_p) = I, so
    all three modes give the same solution to round-off.  For an anisotropic
    body with drag, mode 2 differs from mode 0 by O(|Omega|^2) (the second-order
    term of I(t+1) that Eq. Irotdiff drops)."""
    g = rng(22)
    q = random_quaternion(g)
    A = g.standard_normal((6, 6))
    Z = A @ A.T * 0.05 + np.eye(6) * 0.1                # a drag matrix: SPD
    rF, rT = g.standard_normal(3) * 1e-4, g.standard_normal(3) * 1e-4
    U0 = g.standard_normal(3) * 1e-3
    ax = g.standard_normal(3)
    ax /= np.linalg.norm(ax)
    Iso = np.array([2.0, 2.0, 2.0])
    Om = 0.03 * ax
    I0 = O.inertia_lab(q, Iso)
    sols = [O.rigid_solve(5.0, Iso, q, U0, Om, Z, rF, rT, Iprev=I0, mode=m) for m in (0, 1, 2)]
    for m in (1, 2):
        assert np.allclose(np.concatenate(sols[m]), np.concatenate(sols[0]), rtol=0, atol=1e-14)
    # no velocity-independent forces: every velocity scales with Omega(t)
    Ib = np.array([1.0, 2.0, 3.5])
    d, x = [], []
    for w in (0.02, 0.01, 0.005):
        x0 = np.concatenate(O.rigid_solve(5.0, Ib, q, w * U0, w * ax, Z, (0, 0, 0), (0, 0, 0), mode=0))
        x2 = np.concatenate(O.rigid_solve(5.0, Ib, q, w * U0, w * ax, Z, (0, 0, 0), (0, 0, 0), mode=2))
        d.append(float(np.abs(x2 - x0).max()))
        x.append(float(np.abs(x0).max()))
    for k in range(2):
        assert 3.6 < (d[k] / x[k]) / (d[k + 1] / x[k + 1]) * 2 < 4.4
