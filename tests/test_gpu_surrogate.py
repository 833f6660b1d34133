"""Parity of the surrogate's CUDA path (tcgen05 GEMM, network forward and
backward, Adam, 6x6 solves), called through the C ABI, with the FP64 reference
oracle/surrogate.py on the same seeded inputs.

Bars:
  * GEMM: products of BF16 operands are exact in FP32 and the tensor core sums
    them in FP32, so |C - C_ref| <= K * 2^-23 * (|A| |B|^T) elementwise (a
    generous multiple of the FP32 summation bound), C_ref the FP64 product of
    the same BF16 operands.
  * Network with the reference rounding to BF16 where the CUDA path holds BF16:
    the remaining differences are FP32 sums and rare rounding-boundary flips,
    where the two sums of an activation straddle a BF16 rounding boundary and
    round one BF16 unit apart.  One flip of a second-layer activation h moves an
    output by at most max|W3| * 2^-8 * max|h|; outputs are held to four such
    flips plus 1e-5 (normwise), R^ = L L^T to twice that, and gradients to 5e-3
    normwise per parameter block.
"""
import numpy as np
import pytest

from oracle import surrogate as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
SU = pytest.importorskip("paper_2403_05443_gb300.surrogate")


def _bf16_dev(a):
    """(device BF16 tensor, the same values as float64 numpy)."""
    t = torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).cuda()
    return t, t.float().cpu().numpy().astype(np.float64)


def _normwise(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-30))


@pytest.mark.parametrize("M,N,K,transA,transB,bias,relu", [
    (200, 48, 100, False, False, True, True),
    (128, 256, 256, False, False, False, False),
    (1, 1, 1, False, False, True, False),
    (300, 300, 1000, True, True, True, False),
    (37, 16, 64, True, False, False, True),
    # transposed operands whose strides allow 16-byte staging loads, with
    # partial tiles in M (8 rows of a third tile), N (200 of 208) and K
    (264, 200, 136, True, True, True, True),
])
def test_gemm_matches_fp64_product_of_the_same_bf16_operands(M, N, K, transA, transB, bias, relu):
    g = np.random.default_rng(M * 7 + N * 3 + K)
    A = g.normal(0, 1, (M, K))
    B = g.normal(0, 1, (N, K))
    # storage: A row-major (M x K) or column-major; B row-major (N x K) or as B^T (K x N)
    At, Av = _bf16_dev(A.T if transA else A)
    Bt, Bv = _bf16_dev(B.T if transB else B)
    Av = Av.T if transA else Av
    Bv = Bv.T if transB else Bv
    a_sm, a_sk = (1, M) if transA else (K, 1)
    b_sn, b_sk = (1, N) if transB else (K, 1)
    bias_v = g.normal(0, 1, N).astype(np.float32)
    bt = torch.from_numpy(bias_v).cuda() if bias else None
    C32 = torch.full((M, N), np.nan, dtype=torch.float32, device="cuda")
    C16 = torch.zeros((M, N), dtype=torch.bfloat16, device="cuda")
    SU.lb_gemm_bf16(At.data_ptr(), a_sm, a_sk, Bt.data_ptr(), b_sn, b_sk, M, N, K,
                    bt.data_ptr() if bias else None, int(relu), C32.data_ptr(), C16.data_ptr(), N, 1)
    SU.lb_gemm_status()
    ref = S.gemm(Av, Bv, bias_v.astype(np.float64) if bias else None, relu)
    got = C32.cpu().numpy().astype(np.float64)
    bound = K * 2.0 ** -23 * (np.abs(Av) @ np.abs(Bv).T + (np.abs(bias_v) if bias else 0.0)) + 1e-30
    assert np.all(np.abs(got - ref) <= bound)
    assert np.array_equal(C16.float().cpu().numpy(), S.bf16(got).astype(np.float32))


def _params(seed):
    g = np.random.default_rng(seed)
    P = {"W1": g.normal(0, 0.35, (256, 16)), "b1": g.normal(0, 0.1, 256), "W2": g.normal(0, 0.06, (256, 256)),
         "b2": g.normal(0, 0.1, 256), "W3": g.normal(0, 0.06, (32, 256)), "b3": g.normal(0, 0.3, 32)}
    return S.pack(P).astype(np.float32).astype(np.float64)


def _batch(seed, n):
    g = np.random.default_rng(seed)
    x = g.normal(0, 1, (n, 8)).astype(np.float32)
    A = g.normal(0, 1, (n, 6, 6))
    Rt = (np.einsum("nik,njk->nij", A, A) / 6 + np.eye(6)).astype(np.float32)
    return x, Rt


def _padded(p):
    """The parameters as the library keeps them (padding forced to zero)."""
    P = S.unpack(p.copy())
    P["W1"][:, 8:] = 0.0
    P["W3"][21:] = 0.0
    P["b3"][21:] = 0.0
    return S.pack(P)


@pytest.mark.parametrize("n", [1, 130, 1000])
def test_forward_and_gradients_match_reference(n):
    p = _params(10 + n)
    x, Rt = _batch(20 + n, n)
    net = SU.Surrogate(max_batch=1024, params=p.astype(np.float32))
    assert np.array_equal(net.params(), _padded(p).astype(np.float32))
    xd, Rd = torch.from_numpy(x).cuda(), torch.from_numpy(Rt.reshape(n, 36)).cuda()
    y = torch.zeros((n, 21), device="cuda")
    R = torch.zeros((n, 36), device="cuda")
    SU.lb_mlp_forward(net.h, xd.data_ptr(), n, y.data_ptr(), R.data_ptr())
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros(SU.LB_MLP_NPARAM, device="cuda")
    SU.lb_mlp_loss_grad(net.h, xd.data_ptr(), Rd.data_ptr(), n, loss.data_ptr(), grad.data_ptr())
    torch.cuda.synchronize()
    SU.lb_gemm_status()
    pp = _padded(p)
    f = S.forward(pp, x.astype(np.float64), emulate=True)
    flip = np.abs(f["W3"]).max() * 2.0 ** -8 * np.abs(f["H2"]).max() / np.abs(f["Y"][:, :21]).max()
    tol = 4 * flip + 1e-5
    ey = _normwise(y.cpu().numpy(), f["Y"][:, :21])
    eR = _normwise(R.cpu().numpy().reshape(n, 6, 6), f["R"])
    print("forward errors", ey, eR, "bar", tol)
    assert ey <= tol and eR <= 2 * tol
    lref, gref = S.loss_grad(pp, x.astype(np.float64), Rt.astype(np.float64), emulate=True)
    assert float(loss.item()) == pytest.approx(lref, rel=2e-4)
    G, Gr = S.unpack(grad.cpu().numpy().astype(np.float64)), S.unpack(gref)
    errs = {k: _normwise(G[k], Gr[k]) for k in G}
    print("gradient errors", errs)
    assert all(e <= 5e-3 for e in errs.values()), errs


def test_one_adam_step_matches_reference():
    n = 256
    p = _params(3)
    x, Rt = _batch(4, n)
    net = SU.Surrogate(max_batch=n, params=p.astype(np.float32))
    xd, Rd = torch.from_numpy(x).cuda(), torch.from_numpy(Rt.reshape(n, 36)).cuda()
    lr = 1e-3
    SU.lb_mlp_train_step(net.h, xd.data_ptr(), Rd.data_ptr(), n, lr)
    got = net.params().astype(np.float64)
    pp = _padded(p)
    _, g = S.loss_grad(pp, x.astype(np.float64), Rt.astype(np.float64), emulate=True)
    ref, _, _ = S.adam_step(pp, g, np.zeros_like(pp), np.zeros_like(pp), 1, lr)
    big = np.abs(g) > 1e-3 * np.abs(g).max()
    assert np.abs(got - ref)[big].max() <= 2e-2 * lr
    assert np.abs(got - ref).max() <= 2.0 * lr + 1e-7


def test_training_reduces_the_loss():
    """Fitting a fixed batch: the loss falls by more than 10x in 300 Adam steps."""
    n = 512
    g = np.random.default_rng(8)
    x = g.uniform(-1, 1, (n, 8)).astype(np.float32)
    # a smooth SPD target: diagonal entries depending on the features
    Rt = np.zeros((n, 6, 6), np.float32)
    for i in range(6):
        Rt[:, i, i] = 1.0 + 0.5 * np.tanh(x[:, i % 8]) + 0.2 * x[:, (i + 3) % 8] ** 2
    p = _params(9) * 0.5
    net = SU.Surrogate(max_batch=n, params=p.astype(np.float32))
    xd, Rd = torch.from_numpy(x).cuda(), torch.from_numpy(Rt.reshape(n, 36)).cuda()
    loss = torch.zeros(1, device="cuda")
    SU.lb_mlp_loss_grad(net.h, xd.data_ptr(), Rd.data_ptr(), n, loss.data_ptr())
    l0 = float(loss.item())
    for _ in range(300):
        SU.lb_mlp_train_step(net.h, xd.data_ptr(), Rd.data_ptr(), n, 2e-3)
    SU.lb_mlp_loss_grad(net.h, xd.data_ptr(), Rd.data_ptr(), n, loss.data_ptr())
    l1 = float(loss.item())
    print("loss", l0, "->", l1)
    assert l1 < 0.1 * l0


def test_spd_solve_and_invert_match_reference():
    g = np.random.default_rng(12)
    n = 77
    A = g.normal(0, 1, (n, 6, 6))
    R = (np.einsum("nik,njk->nij", A, A) + 3 * np.eye(6)).astype(np.float32)
    f = g.normal(0, 1, (n, 6))
    Rd = torch.from_numpy(R.reshape(n, 36)).cuda()
    fd = torch.from_numpy(f).cuda()
    ud = torch.zeros((n, 6), dtype=torch.float64, device="cuda")
    SU.lb_spd_solve6(Rd.data_ptr(), fd.data_ptr(), ud.data_ptr(), n)
    Md = torch.from_numpy(R.astype(np.float64).reshape(n, 36)).cuda()
    SU.lb_spd_invert6(Md.data_ptr(), n)
    torch.cuda.synchronize()
    assert _normwise(ud.cpu().numpy(), S.spd_solve(R.astype(np.float64), f)) <= 1e-10
    assert _normwise(Md.cpu().numpy().reshape(n, 6, 6), S.spd_invert(R.astype(np.float64))) <= 1e-10
