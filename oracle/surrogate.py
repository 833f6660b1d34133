"""FP64 reference of the resistance-tensor surrogate: the network, its loss,
its gradients by the chain rule, one Adam step and the 6x6 SPD solves.

Test infrastructure only: the tests, __graft_entry__.smoke() and bench.py's CPU
baseline use it; the product path never does.  It shares no code with the CUDA
library.

Network (fixed shape, as the library defines it): x (8 features, padded with
zeros to 16) -> h1 = relu(W1 x + b1) (256) -> h2 = relu(W2 h1 + b2) (256) ->
y = W3 h2 + b3 (21 used of 32).  The 21 outputs fill a lower-triangular L row
by row (diagonal through softplus) and the prediction is R^ = L L^T, an SPD
6x6 resistance tensor in units of the radius-b sphere: R^ = D^-1 R D^-1 with
D = diag(sqrt(6 pi mu b) I3, sqrt(8 pi mu b^3) I3), so that the translation
block is in units of 6 pi mu b, the rotation block of 8 pi mu b^3 and the
coupling blocks of sqrt(48) pi mu b^2 (oracle/warmstart.py: scales, targets).  Loss: mean over samples of mean over the 36
entries of (R^ - R_target)^2.

With emulate=True the reference rounds to BF16 at exactly the points where
the CUDA path holds BF16 values (the inputs, the weight copies, the hidden
activations and the back-propagated signals that feed the next product), so
that both sides take the same ReLU decisions; products are then exact FP64
sums of the rounded operands.  With emulate=False it is the plain FP64
network.  Parity pinned by: finite differences of the loss, the closed form of
the head at y = 0, BF16 rounding against PyTorch's conversion, and the first
Adam step's closed form (tests/test_oracle_surrogate.py).
"""
from __future__ import annotations

import numpy as np

NIN, NINP, NH, NOUT, NOUTP = 8, 16, 256, 21, 32
OFF = {"W1": (0, (256, 16)), "b1": (4096, (256,)), "W2": (4352, (256, 256)), "b2": (69888, (256,)),
       "W3": (70144, (32, 256)), "b3": (78336, (32,))}
NPARAM = 78368


def unpack(p):
    p = np.asarray(p, np.float64)
    return {k: p[o:o + int(np.prod(s))].reshape(s) for k, (o, s) in OFF.items()}


def pack(d):
    out = np.zeros(NPARAM)
    for k, (o, s) in OFF.items():
        out[o:o + int(np.prod(s))] = np.asarray(d[k], np.float64).reshape(-1)
    return out


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(x))


def softplus(y):
    return np.where(y > 20.0, y, np.log1p(np.exp(np.minimum(y, 20.0))))


def sigmoid(y):
    return 1.0 / (1.0 + np.exp(-y))


def tri_index():
    """(i, j) of each of the 21 outputs: the lower triangle row by row."""
    return [(i, j) for i in range(6) for j in range(i + 1)]


def head(y):
    """L (diagonal softplus) and R^ = L L^T from outputs y[n, 21]."""
    n = y.shape[0]
    L = np.zeros((n, 6, 6))
    for t, (i, j) in enumerate(tri_index()):
        L[:, i, j] = softplus(y[:, t]) if i == j else y[:, t]
    return L, np.einsum("nik,njk->nij", L, L)


def forward(params, x, emulate=False):
    r = bf16 if emulate else (lambda a: np.asarray(a, np.float64))
    P = unpack(params)
    n = x.shape[0]
    X = np.zeros((n, NINP))
    X[:, :NIN] = x
    X = r(X)
    W1, W2, W3 = r(P["W1"]), r(P["W2"]), r(P["W3"])
    H1 = r(np.maximum(X @ W1.T + P["b1"], 0.0))
    H2 = r(np.maximum(H1 @ W2.T + P["b2"], 0.0))
    Y = H2 @ W3.T + P["b3"]
    L, R = head(Y[:, :NOUT])
    return {"X": X, "H1": H1, "H2": H2, "Y": Y, "L": L, "R": R, "W1": W1, "W2": W2, "W3": W3}


def loss_grad(params, x, Rt, emulate=False):
    """(loss, gradient vector in the parameter layout) by the chain rule."""
    r = bf16 if emulate else (lambda a: np.asarray(a, np.float64))
    f = forward(params, x, emulate)
    n = x.shape[0]
    Rt = np.asarray(Rt, np.float64).reshape(n, 6, 6)
    D = f["R"] - Rt
    loss = float((D ** 2).sum() / (36.0 * n))
    dR = 2.0 * D / (36.0 * n)
    dL = 2.0 * np.einsum("nik,nkj->nij", dR, f["L"])     # dR symmetric
    dY = np.zeros((n, NOUTP))
    for t, (i, j) in enumerate(tri_index()):
        dY[:, t] = dL[:, i, j] * (sigmoid(f["Y"][:, t]) if i == j else 1.0)
    dY16 = r(dY)
    g = {}
    g["W3"] = dY16.T @ f["H2"]
    g["b3"] = dY.sum(0)
    dH2 = (dY16 @ f["W3"]) * (f["H2"] > 0)
    g["b2"] = dH2.sum(0)
    dH2 = r(dH2)
    g["W2"] = dH2.T @ f["H1"]
    dH1 = (dH2 @ f["W2"]) * (f["H1"] > 0)
    g["b1"] = dH1.sum(0)
    dH1 = r(dH1)
    g["W1"] = dH1.T @ f["X"]
    return loss, pack(g)


def adam_step(params, grad, m1, m2, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected moments); returns (params, m1, m2)."""
    m1 = b1 * m1 + (1.0 - b1) * grad
    m2 = b2 * m2 + (1.0 - b2) * grad * grad
    mh = m1 / (1.0 - b1 ** step)
    vh = m2 / (1.0 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m1, m2


def spd_solve(R, f):
    """u with R u = f, per sample (R [n,6,6] symmetrised first)."""
    R = np.asarray(R, np.float64).reshape(-1, 6, 6)
    R = 0.5 * (R + np.transpose(R, (0, 2, 1)))
    return np.stack([np.linalg.solve(a, b) for a, b in zip(R, np.asarray(f, np.float64).reshape(-1, 6))])


def spd_invert(M):
    M = np.asarray(M, np.float64).reshape(-1, 6, 6)
    inv = np.linalg.inv(M)
    return 0.5 * (inv + np.transpose(inv, (0, 2, 1)))


def gemm(A, B, bias=None, relu=False):
    """C = A B^T (+ bias) (ReLU): the plain definition."""
    C = np.asarray(A, np.float64) @ np.asarray(B, np.float64).T
    if bias is not None:
        C = C + np.asarray(bias, np.float64)
    return np.maximum(C, 0.0) if relu else C
