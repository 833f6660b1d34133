"""FP64 reference of the warm-start pieces: the periodic Stokes flow of the
particles' forces, the equilibrium initial fluid, the network's input
features and the scaling of resistance tensors.

Test infrastructure only (tests, smoke, bench baselines); shares no code with
the CUDA library.

Stokes flow on the periodic lattice: mu Lap u - grad p + g = 0, div u = 0,
solved mode by mode with numpy's FFT as the transform.  With kt_d =
2 sin(pi k_d / n_d), |kt|^2 is the symbol of the 7-point Laplacian and the
flow is u^ = (g^ - kt (kt . g^) / |kt|^2) / (mu |kt|^2), u^(0) = 0.  g puts
each particle's F_ext uniformly on the fluid nodes next to it (a face
neighbour is its solid node), and the body force plus
(with counter_force) -sum F_ext / N_fluid on the fluid nodes; the mean flow
on the fluid nodes is then shifted so that fluid and particle momenta add up to
zero (the total momentum of a run started from rest).  Pinned by the
single-mode closed form, the projection (divergence-free in the lattice
symbol), the closed form of a curl-free force's pressure and the symmetry of
the periodic Green's function
(tests/test_oracle_warmstart.py).

Steady state of the lattice fluid itself (lb_steady_solve): the linear
D3Q19 BGK dynamics with Guo forcing solved exactly mode by mode (a 4 x 4 system
in the conserved moments); pinned by the oracle's own lattice step written as a
per-mode transfer, by the direct solve of the 19-population fixed point, and
by its long-wavelength (Stokes) limit and a closed form at tau = 1.

Non-equilibrium start (stress_f): the first-order Chapman-Enskog part of the
populations of a viscous flow, pinned by its moments (none in mass and
momentum, the viscous stress in the second moment, a closed form for a shear
wave) and by the LB's own decay of a shear wave, which it starts on the decaying
mode (tests/test_oracle_warmstart.py).

Scaling: D = diag(s_t I3, s_r I3), s_t^2 = 6 pi mu b, s_r^2 = 8 pi mu b^3
(mu = rho0 nu); the network predicts R^ = D^-1 R D^-1, so a radius-b sphere in
free space has R^ = I (Stokes drag 6 pi mu b and torque 8 pi mu b^3).
"""
from __future__ import annotations

import numpy as np


def stokes_field(nx, ny, nz, owner, F_ext, mu, counter=False, body=(0.0, 0.0, 0.0), MU=None, rho0=1.0,
                 density=False, tau=None):
    """u[3, nz, ny, nx]; owner[nz, ny, nx] (0 fluid, p+1 particle p, -1 wall);
    F_ext[np, 3].  The fluid's mean is then shifted so that rho0 sum_fluid u +
    sum_p M_p U_p = 0 (MU[np, 3] = M_p U_p; zero if None).  With density=True
    returns (u, drho), drho the pressure's density deviation with zero sum over
    the fluid nodes.  With tau given, the flow and density are the lattice
    fluid's own steady state (lb_steady_solve) instead of the 7-point Stokes
    solve."""
    owner = np.asarray(owner)
    F = np.asarray(F_ext, np.float64).reshape(-1, 3)
    g = np.zeros((3, nz, ny, nx))
    fluid = owner == 0
    nfl = int(fluid.sum())
    for k in range(3):
        gk = np.zeros((nz, ny, nx))
        gk[fluid] = body[k] - (F[:, k].sum() / nfl if (counter and nfl) else 0.0)
        shell = shell_owner(owner)
        for p in range(F.shape[0]):
            m = shell == p + 1
            if m.any():
                gk[m] += F[p, k] / m.sum()
        g[k] = gk
    if tau is not None:
        from .oracle import lattice
        c, w = lattice()
        u, d_lb = lb_steady_solve(g, tau, rho0, c, w)
    else:
        u = stokes_solve(g, mu)
    P = np.zeros(3) if MU is None else np.asarray(MU, np.float64).reshape(-1, 3).sum(0)
    for k in range(3):
        u[k][fluid] += (-P[k] / rho0 - u[k][fluid].sum()) / nfl
    if not density:
        return u
    d = d_lb if tau is not None else pressure_density(g)
    d[fluid] -= d[fluid].sum() / nfl
    return u, d


def _modes(shape):
    """k vectors [nz, ny, nx, 3] (x, y, z components) of the periodic DFT grid."""
    nz, ny, nx = shape
    kz, ky, kx = [2 * np.pi * np.arange(m) / m for m in (nz, ny, nx)]
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    return np.stack([KX, KY, KZ], -1)


def lb_step_transfer(k, tau, c, w):
    """One step of the linear lattice fluid (BGK, no force) on the Fourier mode
    k: f^_i <- e_i [(1 - omega) f^_i + omega f^eq_i(f^)], e_i = exp(-i k.c_i),
    f^eq_i = w_i (drho^ + 3 c_i . j^) (deviations, rho0 = 1, linear).  19 x 19."""
    c = np.asarray(c, np.float64)
    om = 1.0 / tau
    e = np.exp(-1j * (c @ np.asarray(k, np.float64)))
    Qm = np.asarray(w)[:, None] * (1.0 + 3.0 * c @ c.T)
    return e[:, None] * ((1.0 - om) * np.eye(len(w)) + om * Qm)


def lb_steady_bruteforce(gh, k, tau, c, w):
    """Steady populations of the linear lattice fluid under the force mode
    gh (3 complex) at wave vector k, by solving the 19 x 19 fixed point
    f^ = e (f^ - omega (f^ - f^eq) + (1 - omega/2) F^) with Guo's force term
    F_i = 3 w_i c_i . g and the velocity u = j + g/2 (rho0 = 1); returns
    (drho^, u^)."""
    c = np.asarray(c, np.float64)
    om = 1.0 / tau
    e = np.exp(-1j * (c @ np.asarray(k, np.float64)))
    w = np.asarray(w)
    Qm = w[:, None] * (1.0 + 3.0 * c @ c.T)
    T = e[:, None] * ((1.0 - om) * np.eye(len(w)) + om * Qm)
    # f^eq carries u = j + g/2: its g part, and the force term, are the source
    src = e * (om * 3.0 * w * (c @ gh) / 2.0 + (1.0 - om / 2.0) * 3.0 * w * (c @ gh))
    f = np.linalg.solve(np.eye(len(w)) - T, src)
    return f.sum(), c.T @ f + gh / 2.0


def lb_steady_solve(g, tau, rho0, c, w):
    """Exact steady state of the linear lattice fluid (D3Q19 BGK with Guo
    forcing, rho0, omega = 1/tau) under the periodic force density
    g[3, nz, ny, nx]: the pre-collision populations are the post-collision ones
    streamed, f^_i = e_i f^*_i, so f^_i = h_i (omega f^eq_i + (1 - omega/2) F^_i)
    with h_i = e_i / (1 - (1 - omega) e_i), and their moments (drho, u) solve,
    mode by mode,
      D0 drho - 3 rho0 omega H1 . u = 3 (1 - omega/2) H1 . g
      -omega H1 drho + rho0 D2 u = g/2 + 3 (1 - omega/2) H2 g
    with H1 = sum w_i c_i h_i, H2 = sum w_i c_i c_i^T h_i,
    D0 = sum w_i (1 - e_i) / (1 - (1 - omega) e_i) (= 1 - omega sum w_i h_i) and
    D2 = sum 3 w_i c_i c_i^T (1 - e_i) / (1 - (1 - omega) e_i) (= I - 3 omega H2).
    The k = 0 mode (mean flow, mass) is set to zero.  Returns (u, drho)."""
    g = np.asarray(g, np.float64)
    shape = g.shape[1:]
    K = _modes(shape)
    c = np.asarray(c, np.float64)
    om = 1.0 / tau
    gh = np.stack([np.fft.fftn(g[a]) for a in range(3)], -1)
    H1 = np.zeros(shape + (3,), complex)
    H2 = np.zeros(shape + (3, 3), complex)
    D0 = np.zeros(shape, complex)
    D2 = np.zeros(shape + (3, 3), complex)
    for ci, wi in zip(c, w):
        th = K @ ci
        e = np.exp(-1j * th)
        den = 1.0 - (1.0 - om) * e
        h = e / den
        one_minus_e = 2.0 * np.sin(th / 2.0) ** 2 + 1j * np.sin(th)
        q = one_minus_e / den
        cc = np.outer(ci, ci)
        H1 += wi * h[..., None] * ci
        H2 += wi * h[..., None, None] * cc
        D0 += wi * q
        D2 += 3.0 * wi * q[..., None, None] * cc
    M = np.zeros(shape + (4, 4), complex)
    M[..., 0, 0] = D0
    M[..., 0, 1:] = -3.0 * rho0 * om * H1
    M[..., 1:, 0] = -om * H1
    M[..., 1:, 1:] = rho0 * D2
    r = np.zeros(shape + (4,), complex)
    r[..., 0] = 3.0 * (1.0 - om / 2.0) * np.einsum("...a,...a->...", H1, gh)
    r[..., 1:] = gh / 2.0 + 3.0 * (1.0 - om / 2.0) * np.einsum("...ab,...b->...a", H2, gh)
    M[(0,) * len(shape)] = np.eye(4)
    r[(0,) * len(shape)] = 0.0
    x = np.linalg.solve(M, r[..., None])[..., 0]
    u = np.stack([np.real(np.fft.ifftn(x[..., 1 + a])) for a in range(3)])
    drho = np.real(np.fft.ifftn(x[..., 0]))
    return u, drho


def pressure_density(g):
    """drho = p / c_s^2 = 3 p of the Stokes pressure, grad_c p = P_long g with
    the central difference: p^ = -i (s . g^) / |s|^2, s_d = sin(2 pi k_d / n_d),
    p^ = 0 where |s| = 0."""
    _, nz, ny, nx = g.shape
    s = [np.broadcast_to(np.sin(2 * np.pi * np.arange(nx) / nx)[None, None, :], (nz, ny, nx)),
         np.broadcast_to(np.sin(2 * np.pi * np.arange(ny) / ny)[None, :, None], (nz, ny, nx)),
         np.broadcast_to(np.sin(2 * np.pi * np.arange(nz) / nz)[:, None, None], (nz, ny, nx))]
    s2 = s[0] ** 2 + s[1] ** 2 + s[2] ** 2
    gh = [np.fft.fftn(g[c]) for c in range(3)]
    ph = -1j * (s[0] * gh[0] + s[1] * gh[1] + s[2] * gh[2]) / np.where(s2 > 1e-12, s2, 1.0)
    ph[s2 <= 1e-12] = 0.0
    return 3.0 * np.real(np.fft.ifftn(ph))


def shell_owner(owner):
    """For each fluid node, the particle (p + 1) owning one of its 6 face
    neighbours (periodic), 0 if none; with several, the first in the order
    -x, -y, -z, +x, +y, +z."""
    owner = np.asarray(owner)
    out = np.zeros_like(owner)
    for sh in (1, -1):
        for a in (2, 1, 0):             # x, y, z of an [nz, ny, nx] array
            nb = np.roll(owner, sh, axis=a)
            out = np.where((out == 0) & (nb > 0), nb, out)
    return np.where(owner == 0, out, 0)


def stokes_solve(g, mu):
    """Periodic lattice Stokes flow of a force density g[3, nz, ny, nx]."""
    _, nz, ny, nx = g.shape
    kz = 2 * np.sin(np.pi * np.arange(nz) / nz)[:, None, None]
    ky = 2 * np.sin(np.pi * np.arange(ny) / ny)[None, :, None]
    kx = 2 * np.sin(np.pi * np.arange(nx) / nx)[None, None, :]
    k = [np.broadcast_to(kx, (nz, ny, nx)), np.broadcast_to(ky, (nz, ny, nx)), np.broadcast_to(kz, (nz, ny, nx))]
    k2 = k[0] ** 2 + k[1] ** 2 + k[2] ** 2
    gh = [np.fft.fftn(g[c]) for c in range(3)]
    safe = np.where(k2 > 0, k2, 1.0)
    proj = (k[0] * gh[0] + k[1] * gh[1] + k[2] * gh[2]) / safe
    u = np.zeros_like(g)
    for c in range(3):
        uh = (gh[c] - k[c] * proj) / (mu * safe)
        uh[k2 == 0] = 0.0
        u[c] = np.real(np.fft.ifftn(uh))
    return u


def equilibrium_f(u, rho, c, w):
    """f_i = w_i rho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u) for u[3, ...] and a
    density rho (scalar or [...]): the second-order equilibrium; returns
    [..., 19] in the order of the table (c, w) given."""
    u = np.moveaxis(np.asarray(u, np.float64), 0, -1)
    cu = u @ np.asarray(c, np.float64).T
    uu = (u * u).sum(-1, keepdims=True)
    rho = np.asarray(rho, np.float64)[..., None] if np.ndim(rho) else rho
    return np.asarray(w) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu)


def stress_f(u, rho, tau, c, w):
    """First-order (Chapman-Enskog) non-equilibrium populations of a viscous
    flow u[3, nz, ny, nx]: f_i = -3 tau rho w_i (c_ia c_ib - delta_ab / 3)
    d_a u_b, with d_a the periodic central difference; returns [..., 19] in the
    order of the table (c, w).  Its second moment is -tau rho c_s^2 (grad u +
    grad u^T) and its zeroth and first moments vanish."""
    u = np.asarray(u, np.float64)
    # grad[a][b] = d_a u_b; axis of x in an [nz, ny, nx] array is 2
    axis = {0: 2, 1: 1, 2: 0}
    grad = np.zeros((3, 3) + u.shape[1:])
    for a in range(3):
        for b in range(3):
            grad[a, b] = 0.5 * (np.roll(u[b], -1, axis=axis[a]) - np.roll(u[b], 1, axis=axis[a]))
    c = np.asarray(c, np.float64)
    div = grad[0, 0] + grad[1, 1] + grad[2, 2]
    out = np.zeros(u.shape[1:] + (len(w),))
    rho = np.asarray(rho, np.float64)
    for i in range(len(w)):
        q = -div / 3.0
        for a in range(3):
            for b in range(3):
                q = q + c[i, a] * c[i, b] * grad[a, b]
        out[..., i] = -3.0 * tau * rho * w[i] * q
    return out


def features(geom):
    """Network inputs from geom[n, 8] = (a, b, nu, L, e, rho0)."""
    g = np.asarray(geom, np.float64).reshape(-1, 8)
    sg = np.where(g[:, 6] < 0, -1.0, 1.0)
    x = np.stack([g[:, 0] / g[:, 1] - 2.0, g[:, 1] - 3.0, (g[:, 2] - 1.0 / 6.0) * 10.0, g[:, 1] / g[:, 3] * 10.0 - 1.0,
                  sg * g[:, 4], sg * g[:, 5], sg * g[:, 6], np.ones(len(g))], axis=1)
    return x


def scales(geom):
    g = np.asarray(geom, np.float64).reshape(-1, 8)
    mu = g[:, 7] * g[:, 2]
    b = g[:, 1]
    st, sr = np.sqrt(6 * np.pi * mu * b), np.sqrt(8 * np.pi * mu * b ** 3)
    return np.stack([st, st, st, sr, sr, sr], axis=1)


def targets(M, geom):
    """R^ = (D M D)^-1, symmetrised, from measured mobilities M[n, 6, 6]."""
    d = scales(geom)
    A = d[:, :, None] * np.asarray(M, np.float64).reshape(-1, 6, 6) * d[:, None, :]
    R = np.linalg.inv(A)
    return 0.5 * (R + np.transpose(R, (0, 2, 1)))


def warm_velocities(Rhat, geom, FT):
    """(U, Omega) = D^-1 R^^-1 D^-1 (F, T)."""
    d = scales(geom)
    R = np.asarray(Rhat, np.float64).reshape(-1, 6, 6)
    R = 0.5 * (R + np.transpose(R, (0, 2, 1)))
    f = np.asarray(FT, np.float64).reshape(-1, 6) / d
    return np.stack([np.linalg.solve(a, b) for a, b in zip(R, f)]) / d
