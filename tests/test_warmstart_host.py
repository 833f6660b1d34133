"""Host-side pieces of the warm-start driver (no GPU): the cube rotations used
to augment the LB-measured mobilities, the augmentation itself, the long-axis
direction of a quaternion and the steps-to-steady criterion."""
import math

import numpy as np
import pytest

pytest.importorskip("torch")
from lb_inputs import long_axis_quaternion, resistance_samples  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2403_05443_gb300 import warmstart as W  # noqa: E402


def test_cube_rotations_are_the_24_proper_ones():
    R = W.cube_rotations()
    assert len(R) == 24
    keys = {tuple(np.round(Q).astype(int).ravel()) for Q in R}
    assert len(keys) == 24
    for Q in R:
        assert np.allclose(Q @ Q.T, np.eye(3)) and round(np.linalg.det(Q)) == 1
        assert set(np.abs(Q).ravel()) <= {0.0, 1.0}


def test_augmentation_rotates_axis_and_mobility_consistently():
    """For the mobility of an axisymmetric body, M = P M_body P^T depends on e
    only through e e^T: rotating e and M by the same cube rotation keeps the
    relation (checked against a mobility built from its own axis)."""
    g = np.random.default_rng(0)
    e = g.normal(size=3)
    e /= np.linalg.norm(e)

    def mobility(e):
        ee = np.outer(e, e)
        M = np.zeros((6, 6))
        M[:3, :3] = 2.0 * ee + 1.0 * (np.eye(3) - ee)
        M[3:, 3:] = 0.5 * ee + 0.3 * (np.eye(3) - ee)
        return M

    geom = [[6.0, 3.0, 0.1, 32.0, e[0], e[1], e[2], 1.0]]
    G, Ms = W.augment(geom, [mobility(e)])
    assert G.shape == (24, 8) and Ms.shape == (24, 6, 6)
    for gk, Mk in zip(G, Ms):
        assert np.allclose(Mk, mobility(gk[4:7]))
        assert np.allclose(gk[:4], geom[0][:4]) and gk[7] == geom[0][7]


def test_long_axis_of_the_generated_quaternions():
    for s in resistance_samples(3, 20, 32):
        assert np.allclose(W.long_axis(s["q"]), s["e"], atol=1e-12)
        assert np.allclose(O.rotate(s["q"], (1.0, 0.0, 0.0)), s["e"], atol=1e-12)
    assert np.allclose(W.long_axis(long_axis_quaternion([-1.0, 0.0, 0.0])), [-1.0, 0.0, 0.0])


def test_steps_to_steady_criterion():
    ref = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    every = 10
    errs = [0.5, 0.1, 0.02, 0.0005, 0.002, 0.0004, 0.0002]
    hist = np.zeros((len(errs), 2, 6))
    scale = math.sqrt((1.0 + 4.0) / 2)
    for k, e in enumerate(errs):
        hist[k, :, :3] = ref
        hist[k, 1, 1] += e * scale
    # the error leaves the band once (record 4) and stays inside from record 5
    assert W.steps_to_steady(hist, ref, every, 1e-3) == 60
    assert W.steps_to_steady(hist, ref, every, 1e-1) == 30
    assert W.steps_to_steady(hist[:5], ref, every, 1e-3) is None
