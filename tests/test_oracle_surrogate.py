"""Pins of the surrogate's FP64 reference (oracle/surrogate.py) against things
other than itself: finite differences of its loss, PyTorch's BF16 conversion,
closed forms of the output head and of the first Adam step, and LAPACK."""
import numpy as np
import pytest

from oracle import surrogate as S


def _params(seed, scale=0.2):
    g = np.random.default_rng(seed)
    P = {"W1": g.normal(0, scale, (256, 16)), "b1": g.normal(0, 0.1, 256), "W2": g.normal(0, scale / 8, (256, 256)),
         "b2": g.normal(0, 0.1, 256), "W3": g.normal(0, scale / 8, (32, 256)), "b3": g.normal(0, 0.3, 32)}
    P["W1"][:, 8:] = 0.0
    P["W3"][21:] = 0.0
    P["b3"][21:] = 0.0
    return S.pack(P)


def _batch(seed, n):
    g = np.random.default_rng(seed)
    x = g.normal(0, 1, (n, 8))
    A = g.normal(0, 1, (n, 6, 6))
    Rt = np.einsum("nik,njk->nij", A, A) / 6 + np.eye(6)
    return x, Rt


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(0)
    v = np.concatenate([g.normal(0, 1, 5000), g.normal(0, 1e-30, 100), g.normal(0, 1e30, 100),
                        [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 65504.0, -3.0e-39]]).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(S.bf16(v), ref)


def test_head_closed_form_at_zero_outputs():
    """y = 0 gives L = softplus(0) I = ln 2 I and R^ = (ln 2)^2 I."""
    L, R = S.head(np.zeros((3, 21)))
    assert np.allclose(L, np.log(2.0) * np.eye(6))
    assert np.allclose(R, np.log(2.0) ** 2 * np.eye(6), rtol=0, atol=1e-15)


def test_head_is_spd_and_lower_triangular_fill_is_row_major():
    y = np.arange(21, dtype=float)[None, :] * 0.1 - 1.0
    L, R = S.head(y)
    assert L[0, 1, 0] == pytest.approx(y[0, 1]) and L[0, 5, 4] == pytest.approx(y[0, 19])
    assert L[0, 2, 2] == pytest.approx(np.log1p(np.exp(y[0, 5])))
    assert np.allclose(R[0], R[0].T) and np.linalg.eigvalsh(R[0]).min() > 0


@pytest.mark.parametrize("emulate", [False, True])
def test_gradient_against_central_differences(emulate):
    """The chain rule of loss_grad against central differences of the FP64
    loss (emulate=False), on entries of every parameter block; with BF16
    emulation the gradient stays close to the FP64 one."""
    p = _params(1)
    x, Rt = _batch(2, 7)
    loss, g = S.loss_grad(p, x, Rt, emulate=emulate)
    if emulate:
        _, g64 = S.loss_grad(p, x, Rt, emulate=False)
        assert np.abs(g - g64).max() <= 0.05 * np.abs(g64).max()
        return
    rng = np.random.default_rng(3)
    for name, (o, shape) in S.OFF.items():
        size = int(np.prod(shape))
        live = [k for k in range(size) if not (name == "W1" and k % 16 >= 8) and not (name == "W3" and k // 256 >= 21)
                and not (name == "b3" and k >= 21)]
        for k in rng.choice(live, 6, replace=False):
            h = 1e-6 * max(1.0, abs(p[o + k]))
            pp, pm = p.copy(), p.copy()
            pp[o + k] += h
            pm[o + k] -= h
            fd = (S.loss_grad(pp, x, Rt)[0] - S.loss_grad(pm, x, Rt)[0]) / (2 * h)
            assert fd == pytest.approx(g[o + k], rel=1e-5, abs=1e-10 * abs(loss) + 1e-14), (name, k)


def test_padding_gets_zero_gradient():
    p = _params(4)
    x, Rt = _batch(5, 9)
    _, g = S.loss_grad(p, x, Rt)
    G = S.unpack(g)
    assert np.all(G["W1"][:, 8:] == 0) and np.all(G["W3"][21:] == 0) and np.all(G["b3"][21:] == 0)


def test_first_adam_step_closed_form():
    """At step 1 the bias-corrected moments are g and g^2, so the update is
    lr g / (|g| + eps)."""
    g = np.random.default_rng(6).normal(0, 1, 100)
    p = np.ones(100)
    p1, _, _ = S.adam_step(p, g, np.zeros(100), np.zeros(100), 1, 1e-3)
    assert np.allclose(p1, 1.0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_spd_solve_and_invert_against_lapack_identities():
    g = np.random.default_rng(7)
    A = g.normal(0, 1, (5, 6, 6))
    R = np.einsum("nik,njk->nij", A, A) + 6 * np.eye(6)
    f = g.normal(0, 1, (5, 6))
    u = S.spd_solve(R, f)
    assert np.allclose(np.einsum("nij,nj->ni", R, u), f, atol=1e-12)
    Ri = S.spd_invert(R)
    assert np.allclose(np.einsum("nij,njk->nik", R, Ri), np.eye(6), atol=1e-12)
