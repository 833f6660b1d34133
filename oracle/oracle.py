"""Python handle on the FP64 CPU oracle (oracle/lb_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py.  Nothing in the CUDA package imports
it, and it imports nothing from the CUDA package.

The oracle follows the paper's Appendix steps 1-10 in order (see lb_oracle.c).
This module only marshals arguments; every step of the method runs in C.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lb_oracle.c")
_HDR = os.path.join(_HERE, "lb_oracle.h")
_LIBS = {19: os.path.join(_HERE, "_build", "liboracle.so"), 27: os.path.join(_HERE, "_build", "liboracle27.so")}
_LIB = _LIBS[19]


def _build_one(q: int, force: bool) -> str:
    out = _LIBS[q]
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-ffp-contract=off",
           "-fPIC", "-shared", *(["-DORC_D3Q27"] if q == 27 else []), "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FMA contraction): the D3Q19
    library and, from the same source, the D3Q27 one."""
    _build_one(27, force)
    return _build_one(19, force)


class OrcBox(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("tau", C.c_double), ("rho0", C.c_double),
                ("body_force", C.c_double * 3), ("counter_force", C.c_int),
                ("walls", C.c_int), ("wall_u_lo", C.c_double * 3),
                ("wall_u_hi", C.c_double * 3), ("didt_mode", C.c_int), ("lub_cut", C.c_double),
                ("collision", C.c_int)]


class OrcParticle(C.Structure):
    _fields_ = [("semi", C.c_double * 3), ("x", C.c_double * 3), ("q", C.c_double * 4),
                ("U", C.c_double * 3), ("Om", C.c_double * 3), ("density", C.c_double),
                ("F_ext", C.c_double * 3), ("T_ext", C.c_double * 3),
                ("B1", C.c_double), ("B2", C.c_double)]


_libs = {}
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


def lib(q: int = 19):
    """The oracle library of the D3Q19 (q = 19) or D3Q27 (q = 27) lattice."""
    if q not in _LIBS:
        raise ValueError(f"no oracle for D3Q{q}")
    if q not in _libs:
        build()
        _libs[q] = C.CDLL(_LIBS[q])
        L = _libs[q]
        L.orc_q.restype = C.c_int
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(OrcBox), C.POINTER(OrcParticle), C.c_int, C.c_int]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_step.restype = C.c_int
        L.orc_time.argtypes = [C.c_void_p]
        L.orc_time.restype = C.c_long
        L.orc_lattice.argtypes = [_I, _D]
        for name in ("orc_get_f", "orc_set_f"):
            getattr(L, name).argtypes = [C.c_void_p, _D]
        L.orc_get_moments.argtypes = [C.c_void_p, _D, _D]
        L.orc_get_owner.argtypes = [C.c_void_p, _I]
        L.orc_total_fluid_mass.argtypes = [C.c_void_p]
        L.orc_total_fluid_mass.restype = C.c_double
        L.orc_total_fluid_momentum.argtypes = [C.c_void_p, _D]
        for name in ("orc_get_particle", "orc_get_pending", "orc_get_zeta"):
            getattr(L, name).argtypes = [C.c_void_p, C.c_int, _D]
        L.orc_get_links.argtypes = [C.c_void_p, C.c_int, _I, _I, C.c_int]
        L.orc_get_links.restype = C.c_int
        L.orc_mass.argtypes = [C.c_void_p, C.c_int]
        L.orc_mass.restype = C.c_double
        L.orc_feq.argtypes = [C.c_double, _D, _D]
        L.orc_quat_mul.argtypes = [_D, _D, _D]
        L.orc_rotate.argtypes = [_D, _D, _D]
        L.orc_inertia_lab.argtypes = [_D, _D, _D]
        L.orc_inertia_rate.argtypes = [_D, _D, _D, _D]
        L.orc_quat_step.argtypes = [_D, _D, _D]
        L.orc_gauss_solve.argtypes = [C.c_int, _D, _D, _D]
        L.orc_gauss_solve.restype = C.c_int
        L.orc_inside_value.argtypes = [_D, _D, _D, _I, _I, _I]
        L.orc_inside_value.restype = C.c_double
        L.orc_squirmer_slip.argtypes = [_D, _D, C.c_double, C.c_double, _D, _D]
        L.orc_rigid_solve.argtypes = [C.c_double, _D, _D, _D, _D, _D, _D, _D, _D, C.c_int, _D, _D]
        L.orc_rigid_solve.restype = C.c_int
        L.orc_lubrication_pair.argtypes = [_D, _D, _D, _D, C.c_double, _D, _D, _D, _D, C.c_double, _I, _I,
                                           C.c_double, C.c_double, _D, _D]
        assert L.orc_q() == q
    return _libs[q]


def _dp(a):
    return a.ctypes.data_as(_D)


def _ip(a):
    return a.ctypes.data_as(_I)


def _f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None:
        assert a.size == n, (a.shape, n)
    return a


# ----------------------------------------------------------------------------
def lattice(q: int = 19):
    """D3Q19 (or D3Q27) velocities c[q,3] and weights w[q] in the oracle's own order."""
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q)
    lib(q).orc_lattice(_ip(c), _dp(w))
    return c, w


def feq(rho, u, q: int = 19):
    out = np.zeros(q)
    lib(q).orc_feq(float(rho), _dp(_f64(u, 3)), _dp(out))
    return out


def quat_mul(a, b):
    out = np.zeros(4)
    lib().orc_quat_mul(_dp(_f64(a, 4)), _dp(_f64(b, 4)), _dp(out))
    return out


def rotate(q, s):
    out = np.zeros(3)
    lib().orc_rotate(_dp(_f64(q, 4)), _dp(_f64(s, 3)), _dp(out))
    return out


def inertia_lab(q, Ibody):
    out = np.zeros(9)
    lib().orc_inertia_lab(_dp(_f64(q, 4)), _dp(_f64(Ibody, 3)), _dp(out))
    return out.reshape(3, 3)


def inertia_rate(q, Om, Ibody):
    out = np.zeros(9)
    lib().orc_inertia_rate(_dp(_f64(q, 4)), _dp(_f64(Om, 3)), _dp(_f64(Ibody, 3)), _dp(out))
    return out.reshape(3, 3)


def quat_step(q, Om_mean):
    out = np.zeros(4)
    lib().orc_quat_step(_dp(_f64(q, 4)), _dp(_f64(Om_mean, 3)), _dp(out))
    return out


def gauss_solve(A, b):
    A = _f64(A)
    n = A.shape[0]
    x = np.zeros(n)
    rc = lib().orc_gauss_solve(n, _dp(A), _dp(_f64(b, n)), _dp(x))
    if rc != 0:
        raise np.linalg.LinAlgError(f"orc_gauss_solve failed ({rc})")
    return x


def inside_value(semi, q, xc, X, L, periodic=(1, 1, 1)):
    Xa = np.ascontiguousarray(np.asarray(X, dtype=np.int32))
    La = np.ascontiguousarray(np.asarray(L, dtype=np.int32))
    Pa = np.ascontiguousarray(np.asarray(periodic, dtype=np.int32))
    return lib().orc_inside_value(_dp(_f64(semi, 3)), _dp(_f64(q, 4)), _dp(_f64(xc, 3)),
                                  _ip(Xa), _ip(La), _ip(Pa))


def squirmer_slip(semi, q, B1, B2, r):
    out = np.zeros(3)
    lib().orc_squirmer_slip(_dp(_f64(semi, 3)), _dp(_f64(q, 4)), float(B1), float(B2),
                            _dp(_f64(r, 3)), _dp(out))
    return out


def rigid_solve(M, Ibody, q, U, Om, zeta, rF, rT, Iprev=None, mode=0):
    """Appendix steps 4-5 for one body (Eq. Fdiscrete / Eq. Tdiscrete, dt = 1):
    (U(t+1), Omega(t+1)) for drag matrix zeta (6x6) and velocity-independent
    forces rF, rT; mode 0 analytic dI/dt, 1 finite difference (Iprev = I(t-1)),
    2 predictor-corrector."""
    Un, Wn = np.zeros(3), np.zeros(3)
    Ip = _f64(Iprev if Iprev is not None else np.zeros(9), 9)
    rc = lib().orc_rigid_solve(float(M), _dp(_f64(Ibody, 3)), _dp(_f64(q, 4)), _dp(_f64(U, 3)), _dp(_f64(Om, 3)),
                               _dp(_f64(zeta, 36)), _dp(_f64(rF, 3)), _dp(_f64(rT, 3)), _dp(Ip), int(mode),
                               _dp(Un), _dp(Wn))
    if rc:
        raise ArithmeticError("singular system")
    return Un, Wn


def lubrication_pair(a: dict, b: dict, L, mu, h_cut, periodic=(1, 1, 1)):
    """(force on a, gap) of the lubrication correction between particle
    dicts a and b (semi, q, x, U, M)."""
    f, h = np.zeros(3), np.zeros(1)
    lib().orc_lubrication_pair(_dp(_f64(a["semi"], 3)), _dp(_f64(a["q"], 4)), _dp(_f64(a["x"], 3)),
                               _dp(_f64(a["U"], 3)), float(a["M"]), _dp(_f64(b["semi"], 3)), _dp(_f64(b["q"], 4)),
                               _dp(_f64(b["x"], 3)), _dp(_f64(b["U"], 3)), float(b["M"]),
                               _ip(np.asarray(L, np.int32)), _ip(np.asarray(periodic, np.int32)), float(mu),
                               float(h_cut), _dp(f), _dp(h))
    return f, float(h[0])


# ----------------------------------------------------------------------------
class Sim:
    """One box of fluid with its particles, stepped by the oracle.

    box: dict with nx, ny, nz, tau, rho0, body_force, counter_force, walls,
    wall_u_lo, wall_u_hi, didt_mode, and lattice (19, the default, or 27).
    particles: list of dicts with semi, x, q, U, Om, density, F_ext, T_ext, B1,
    B2.
    """

    def __init__(self, box: dict, particles=(), nthreads: int | None = None):
        self.Q = int(box.get("lattice", 19) or 19)
        L = self._L = lib(self.Q)
        b = OrcBox()
        b.nx, b.ny, b.nz = int(box["nx"]), int(box["ny"]), int(box["nz"])
        b.tau = float(box["tau"])
        b.rho0 = float(box.get("rho0", 1.0))
        b.body_force[:] = list(box.get("body_force", (0.0, 0.0, 0.0)))
        b.counter_force = int(box.get("counter_force", 0))
        b.walls = int(box.get("walls", 0))
        b.wall_u_lo[:] = list(box.get("wall_u_lo", (0.0, 0.0, 0.0)))
        b.wall_u_hi[:] = list(box.get("wall_u_hi", (0.0, 0.0, 0.0)))
        b.didt_mode = int(box.get("didt_mode", 0))
        b.lub_cut = float(box.get("lub_cut", 0.0))
        b.collision = int(box.get("collision", 0))
        ps = (OrcParticle * max(1, len(particles)))()
        for k, p in enumerate(particles):
            ps[k].semi[:] = list(p["semi"])
            ps[k].x[:] = list(p["x"])
            ps[k].q[:] = list(p.get("q", (1.0, 0.0, 0.0, 0.0)))
            ps[k].U[:] = list(p.get("U", (0.0, 0.0, 0.0)))
            ps[k].Om[:] = list(p.get("Om", (0.0, 0.0, 0.0)))
            ps[k].density = float(p.get("density", 1.0))
            ps[k].F_ext[:] = list(p.get("F_ext", (0.0, 0.0, 0.0)))
            ps[k].T_ext[:] = list(p.get("T_ext", (0.0, 0.0, 0.0)))
            ps[k].B1 = float(p.get("B1", 0.0))
            ps[k].B2 = float(p.get("B2", 0.0))
        if nthreads is None:
            nthreads = int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1))
        self.nthreads = nthreads
        self._h = L.orc_create(C.byref(b), ps, len(particles), nthreads)
        if not self._h:
            raise ValueError("oracle rejected the box or particles (overlap or bad size)")
        self.nx, self.ny, self.nz = b.nx, b.ny, b.nz
        self.N = b.nx * b.ny * b.nz
        self.np = len(particles)

    def close(self):
        if getattr(self, "_h", None):
            self._L.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        rc = self._L.orc_step(self._h, int(n))
        if rc:
            raise RuntimeError(f"oracle step failed with code {rc}")

    @property
    def time(self) -> int:
        return self._L.orc_time(self._h)

    def f(self):
        """Pre-collision f, shape (nz, ny, nx, Q), oracle direction order."""
        out = np.zeros(self.N * self.Q)
        self._L.orc_get_f(self._h, _dp(out))
        return out.reshape(self.nz, self.ny, self.nx, self.Q)

    def set_f(self, f):
        self._L.orc_set_f(self._h, _dp(_f64(f, self.N * self.Q)))

    def moments(self):
        rho = np.zeros(self.N)
        u = np.zeros(self.N * 3)
        self._L.orc_get_moments(self._h, _dp(rho), _dp(u))
        return rho.reshape(self.nz, self.ny, self.nx), u.reshape(self.nz, self.ny, self.nx, 3)

    def owner(self):
        o = np.zeros(self.N, dtype=np.int32)
        self._L.orc_get_owner(self._h, _ip(o))
        return o.reshape(self.nz, self.ny, self.nx)

    def fluid_mass(self) -> float:
        return self._L.orc_total_fluid_mass(self._h)

    def fluid_momentum(self):
        out = np.zeros(3)
        self._L.orc_total_fluid_momentum(self._h, _dp(out))
        return out

    def particle(self, p: int = 0) -> dict:
        out = np.zeros(25)
        self._L.orc_get_particle(self._h, p, _dp(out))
        return {"F0": out[0:3], "T0": out[3:6], "F": out[6:9], "T": out[9:12],
                "U": out[12:15], "Om": out[15:18], "x": out[18:21], "q": out[21:25],
                "raw": out}

    def pending(self, p: int = 0):
        """(dP, dL, dm, dm_return) of the remap terms still to be applied."""
        out = np.zeros(8)
        self._L.orc_get_pending(self._h, p, _dp(out))
        return out[0:3], out[3:6], out[6], out[7]

    def zeta(self, p: int = 0):
        out = np.zeros(36)
        self._L.orc_get_zeta(self._h, p, _dp(out))
        return out.reshape(6, 6)

    def mass(self, p: int = 0) -> float:
        return self._L.orc_mass(self._h, p)

    def links(self, p: int = 0):
        """Boundary links (node index, c_b) of particle p."""
        n = self._L.orc_get_links(self._h, p, None, None, 0)
        node = np.zeros(max(n, 1), dtype=np.int32)
        cv = np.zeros(max(n, 1) * 3, dtype=np.int32)
        self._L.orc_get_links(self._h, p, _ip(node), _ip(cv), n)
        return node[:n], cv[: 3 * n].reshape(n, 3)


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
