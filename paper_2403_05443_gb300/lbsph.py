"""Python binding of the lbsph C ABI (include/lbsph.h), argument marshalling only.

Every function below has the name of the C entry point it calls and raises
LBError on a non-zero lb_status.  All of the method runs in liblbsph.so; there
is no Python or CPU fallback: if the library is missing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LB_FP32, LB_FP16, LB_BF16 = 0, 1, 2
LB_FIELD_F, LB_FIELD_DF, LB_FIELD_RHO, LB_FIELD_U, LB_FIELD_SOLID = 1, 2, 4, 8, 16
LB_FLAG_SEPARATE_KERNELS = 1
LB_RECORD_DOUBLES = 25
STATUS = {0: "LB_OK", 1: "LB_EINVAL", 2: "LB_ENOMEM", 3: "LB_ECUDA", 4: "LB_ETIMEOUT",
          5: "LB_ENAN", 6: "LB_EOVERLAP", 7: "LB_ECAPACITY", 8: "LB_ESTATE"}
_FIELD_NAMES = {"f": LB_FIELD_F, "df": LB_FIELD_DF, "rho": LB_FIELD_RHO, "u": LB_FIELD_U, "solid": LB_FIELD_SOLID}


class LBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class BoxDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("tau", C.c_double), ("rho0", C.c_double), ("body_force", C.c_double * 3),
                ("counter_force", C.c_int32), ("walls", C.c_int32),
                ("wall_u_lo", C.c_double * 3), ("wall_u_hi", C.c_double * 3), ("lub_cut", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
RELEASE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("didt_mode", C.c_int32), ("device", C.c_int32),
                ("flags", C.c_uint32), ("max_semi", C.c_int32), ("max_particles", C.c_int32),
                ("fp16_scale", C.c_double), ("alloc", ALLOC_FN), ("release", RELEASE_FN),
                ("alloc_user", C.c_void_p), ("collision", C.c_int32), ("lattice", C.c_int32)]


class Particle(C.Structure):
    _fields_ = [("semi", C.c_double * 3), ("x", C.c_double * 3), ("q", C.c_double * 4),
                ("U", C.c_double * 3), ("Omega", C.c_double * 3), ("density", C.c_double),
                ("F_ext", C.c_double * 3), ("T_ext", C.c_double * 3),
                ("B1", C.c_double), ("B2", C.c_double)]


_lib = None


def library(path: str | None = None):
    """Load liblbsph.so (building it first if the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("liblbsph.so is missing: run paper_2403_05443_gb300.build.build()")
    L = C.CDLL(path)
    vp, i32, u32, dp, ip = C.c_void_p, C.c_int32, C.c_uint32, C.POINTER(C.c_double), C.POINTER(C.c_int32)
    L.lb_create.argtypes = [C.POINTER(BoxDesc), i32, C.POINTER(Options), C.POINTER(vp)]
    L.lb_destroy.argtypes = [vp]
    L.lb_set_particles.argtypes = [vp, i32, C.POINTER(Particle), i32]
    L.lb_set_external.argtypes = [vp, i32, dp, i32, vp]
    L.lb_step.argtypes = [vp, i32, vp]
    L.lb_get_fields.argtypes = [vp, i32, u32, vp, C.c_size_t, i32, vp]
    L.lb_get_force_torque.argtypes = [vp, i32, dp, i32]
    L.lb_get_force_torque_async.argtypes = [vp, i32, vp, i32, vp]
    L.lb_step_io.argtypes = [vp, i32, vp, vp, vp]
    L.lb_get_links.argtypes = [vp, i32, i32, ip, i32, ip]
    L.lb_get_drag.argtypes = [vp, i32, i32, dp]
    L.lb_synchronize.argtypes = [vp]
    L.lb_profile_step.argtypes = [vp, i32, vp, dp]
    L.lb_links_noalloc.argtypes = [dp, dp, dp, i32, i32, i32, i32, vp, i32, vp, vp]
    L.lb_links_noalloc.restype = i32
    L.lb_autotune.argtypes = [vp, i32, vp, ip, dp]
    L.lb_init_fluid.argtypes = [vp, i32, vp, C.c_size_t, vp, i32, i32, vp]
    L.lb_stokes_field.argtypes = [vp, i32, vp, vp, vp]
    L.lb_lattice.argtypes = [ip, dp]
    L.lb_lattice.restype = None
    L.lb_lattice_q.argtypes = [i32, ip, dp]
    L.lb_lattice_q.restype = i32
    L.lb_status_string.argtypes = [i32]
    L.lb_status_string.restype = C.c_char_p
    L.lb_last_error.argtypes = [vp]
    L.lb_last_error.restype = C.c_char_p
    L.lb_abi_version.restype = i32
    for name in ("lb_create", "lb_destroy", "lb_set_particles", "lb_set_external", "lb_step",
                 "lb_get_fields", "lb_get_force_torque", "lb_get_force_torque_async", "lb_get_links", "lb_get_drag",
                 "lb_synchronize", "lb_step_io",
                 "lb_profile_step", "lb_init_fluid", "lb_stokes_field", "lb_autotune"):
        getattr(L, name).restype = i32
    _lib = L
    return L


def _check(rc: int, ctx=None):
    if rc != 0:
        msg = library().lb_last_error(ctx).decode() if ctx else library().lb_status_string(rc).decode()
        raise LBError(rc, msg)


def _box_struct(d: dict) -> BoxDesc:
    b = BoxDesc()
    b.nx, b.ny, b.nz = int(d["nx"]), int(d["ny"]), int(d["nz"])
    b.tau, b.rho0 = float(d["tau"]), float(d.get("rho0", 1.0))
    b.body_force[:] = list(d.get("body_force", (0.0, 0.0, 0.0)))
    b.counter_force, b.walls = int(d.get("counter_force", 0)), int(d.get("walls", 0))
    b.wall_u_lo[:] = list(d.get("wall_u_lo", (0.0, 0.0, 0.0)))
    b.wall_u_hi[:] = list(d.get("wall_u_hi", (0.0, 0.0, 0.0)))
    b.lub_cut = float(d.get("lub_cut", 0.0))
    return b


def _particle_struct(p: dict, out: Particle):
    out.semi[:] = list(p["semi"])
    out.x[:] = list(p["x"])
    out.q[:] = list(p.get("q", (1.0, 0.0, 0.0, 0.0)))
    out.U[:] = list(p.get("U", (0.0, 0.0, 0.0)))
    out.Omega[:] = list(p.get("Om", p.get("Omega", (0.0, 0.0, 0.0))))
    out.density = float(p.get("density", 1.0))
    out.F_ext[:] = list(p.get("F_ext", (0.0, 0.0, 0.0)))
    out.T_ext[:] = list(p.get("T_ext", (0.0, 0.0, 0.0)))
    out.B1, out.B2 = float(p.get("B1", 0.0)), float(p.get("B2", 0.0))


# ---------------------------------------------------------------------------
# the C entry points, one Python function each
def lb_abi_version() -> int:
    return library().lb_abi_version()


def lb_status_string(status: int) -> str:
    return library().lb_status_string(status).decode()


def lb_last_error(ctx) -> str:
    return library().lb_last_error(ctx).decode()


def lb_lattice():
    """(c[19,3] int32, w[19]) of the library's D3Q19 order."""
    c = np.zeros((19, 3), np.int32)
    w = np.zeros(19)
    library().lb_lattice(c.ctypes.data_as(C.POINTER(C.c_int32)), w.ctypes.data_as(C.POINTER(C.c_double)))
    return c, w


def lb_lattice_q(q: int):
    """(c[q,3] int32, w[q]) of the library's order of lattice q (19 or 27)."""
    c = np.zeros((q, 3), np.int32)
    w = np.zeros(q)
    _check(library().lb_lattice_q(int(q), c.ctypes.data_as(C.POINTER(C.c_int32)), w.ctypes.data_as(C.POINTER(C.c_double))))
    return c, w


def lb_create(boxes, opt: Options):
    arr = (BoxDesc * len(boxes))(*[_box_struct(b) for b in boxes])
    h = C.c_void_p()
    _check(library().lb_create(arr, len(boxes), C.byref(opt), C.byref(h)))
    return h


def lb_destroy(ctx):
    _check(library().lb_destroy(ctx))


def lb_set_particles(ctx, box: int, particles):
    arr = (Particle * max(1, len(particles)))()
    for k, p in enumerate(particles):
        _particle_struct(p, arr[k])
    _check(library().lb_set_particles(ctx, box, arr, len(particles)), ctx)


def lb_set_external(ctx, box: int, ft, stream=None):
    ft = np.ascontiguousarray(np.asarray(ft, np.float64).reshape(-1, 6))
    _check(library().lb_set_external(ctx, box, ft.ctypes.data_as(C.POINTER(C.c_double)), ft.shape[0], stream), ctx)


def lb_step(ctx, nsteps: int, stream=None):
    _check(library().lb_step(ctx, int(nsteps), stream), ctx)


def lb_get_fields(ctx, box: int, what: int, dst_ptr: int, nbytes: int, dst_is_device: bool, stream=None):
    _check(library().lb_get_fields(ctx, box, what, C.c_void_p(dst_ptr), nbytes, int(dst_is_device), stream), ctx)


def lb_get_force_torque(ctx, box: int, n: int, out: np.ndarray | None = None) -> np.ndarray:
    """Records of the n particles of `box` (-1: all boxes); `out` may be a
    preallocated (pinned) float64 host array of n*25 values."""
    if out is None:
        out = np.zeros((max(n, 1), LB_RECORD_DOUBLES))
    _check(library().lb_get_force_torque(ctx, box, out.ctypes.data_as(C.POINTER(C.c_double)), n), ctx)
    return out.reshape(-1, LB_RECORD_DOUBLES)[:n]


def lb_get_force_torque_async(ctx, box: int, n: int, out_ptr: int, stream=None):
    """Enqueue the copy of the n particle records of `box` (-1: all boxes) to
    out_ptr (pinned host or device memory, n*25 float64) on `stream`; returns
    at once, the data are there once the stream has been waited for."""
    _check(library().lb_get_force_torque_async(ctx, box, C.c_void_p(out_ptr), n, stream), ctx)


def lb_step_io(ctx, nsteps: int, ft_ptr, rec_ptr, stream=None):
    """nsteps iterations, each with its F_ext/T_ext from ft_ptr + k*np*6 and its
    records copied to rec_ptr + k*np*25 (float64; pinned host or device
    addresses, either may be None); queued on `stream`, returns at once."""
    _check(library().lb_step_io(ctx, int(nsteps), None if ft_ptr is None else C.c_void_p(ft_ptr),
                                None if rec_ptr is None else C.c_void_p(rec_ptr), stream), ctx)


def lb_profile_step(ctx, nsteps: int, stream=None):
    """ms of (bulk, boundary, particle-critical, particle-auxiliary) kernels,
    each summed over nsteps iterations."""
    out = np.zeros(4)
    _check(library().lb_profile_step(ctx, int(nsteps), stream, out.ctypes.data_as(C.POINTER(C.c_double))), ctx)
    return tuple(float(v) for v in out)


def lb_get_links(ctx, box: int, particle: int):
    cnt = C.c_int32(0)
    _check(library().lb_get_links(ctx, box, particle, None, 0, C.byref(cnt)), ctx)
    n = cnt.value
    pairs = np.zeros(2 * max(n, 1), np.int32)
    _check(library().lb_get_links(ctx, box, particle, pairs.ctypes.data_as(C.POINTER(C.c_int32)), n,
                                  C.byref(cnt)), ctx)
    pairs = pairs[: 2 * n].reshape(n, 2)
    return pairs[:, 0].copy(), pairs[:, 1].copy()


def lb_get_drag(ctx, box: int, particle: int) -> np.ndarray:
    out = np.zeros(36)
    _check(library().lb_get_drag(ctx, box, particle, out.ctypes.data_as(C.POINTER(C.c_double))), ctx)
    return out.reshape(6, 6)


def lb_init_fluid(ctx, box: int, u_ptr: int, nbytes: int, drho_ptr, is_device: bool, with_stress: bool = False,
                  stream=None):
    """Initial fluid f = f_eq(rho0 + drho, u) of a box before the first step
    (with_stress: plus the first-order non-equilibrium part of the flow's
    viscous stress); u_ptr / drho_ptr (drho may be None) are host or device
    addresses of FP32 [3][nz][ny][nx] / [nz][ny][nx]."""
    _check(library().lb_init_fluid(ctx, box, C.c_void_p(u_ptr), nbytes,
                                   None if drho_ptr is None else C.c_void_p(drho_ptr), int(is_device),
                                   int(bool(with_stress)), stream), ctx)


def lb_stokes_field(ctx, box: int, u_dev_ptr: int, drho_dev_ptr=None, stream=None):
    """Periodic Stokes flow of the box's particle forces into device FP32 [3][N]
    (and its pressure as a density deviation [N] if drho_dev_ptr is given)."""
    _check(library().lb_stokes_field(ctx, box, C.c_void_p(u_dev_ptr),
                                     None if drho_dev_ptr is None else C.c_void_p(drho_dev_ptr), stream), ctx)


def lb_autotune(ctx, steps_per_candidate: int, stream=None):
    """((units per fetch, blocks per particle, iterations advanced), ms per
    step of the 6 blocks-per-particle (1, 2, 3, d, 2d, 3d) and the 4
    units-per-fetch candidates)."""
    out = np.zeros(3, np.int32)
    ms = np.zeros(10)
    _check(library().lb_autotune(ctx, int(steps_per_candidate), stream, out.ctypes.data_as(C.POINTER(C.c_int32)),
                                 ms.ctypes.data_as(C.POINTER(C.c_double))), ctx)
    return tuple(int(v) for v in out), ms


def lb_synchronize(ctx):
    _check(library().lb_synchronize(ctx), ctx)


def lb_links_noalloc(semi, q, x, nx, ny, nz, walls, pairs_dev_ptr: int, cap: int, count_dev_ptr: int, stream=None):
    """Boundary links of one spheroid into caller-owned device buffers, with no
    allocation by the library (see include/lbsph.h).  pairs_dev_ptr / count_dev_ptr
    are device addresses (e.g. tensor.data_ptr())."""
    def d(v, n):
        a = np.ascontiguousarray(np.asarray(v, np.float64))
        assert a.size == n
        return a
    s, qq, xx = d(semi, 3), d(q, 4), d(x, 3)
    dp = C.POINTER(C.c_double)
    _check(library().lb_links_noalloc(s.ctypes.data_as(dp), qq.ctypes.data_as(dp), xx.ctypes.data_as(dp),
                                      int(nx), int(ny), int(nz), int(walls), C.c_void_p(pairs_dev_ptr), int(cap),
                                      C.c_void_p(count_dev_ptr), stream))


# ---------------------------------------------------------------------------
def _torch_allocator(device: int):
    import torch

    live = {}

    def alloc(nbytes, _user):
        ptr = torch.cuda.caching_allocator_alloc(int(nbytes), device)
        live[ptr] = nbytes
        return ptr

    def release(ptr, _user):
        if ptr in live:
            del live[ptr]
            torch.cuda.caching_allocator_delete(ptr)

    return ALLOC_FN(alloc), RELEASE_FN(release)


CUDA_STREAM_LEGACY = 1   # cudaStreamLegacy: the NULL stream with legacy synchronisation


def stream_handle(s) -> C.c_void_p:
    """cudaStream_t of a torch stream.  torch's default stream has handle 0,
    which the C ABI would read as "the context's own stream", so it is passed
    as cudaStreamLegacy instead."""
    h = int(s.cuda_stream)
    return C.c_void_p(h if h != 0 else CUDA_STREAM_LEGACY)


def current_stream():
    """The cudaStream_t of torch's current stream (None if torch has no CUDA)."""
    try:
        import torch
        if torch.cuda.is_available():
            return stream_handle(torch.cuda.current_stream())
    except ImportError:
        pass
    return None


class Simulation:
    """A context plus the particles of its boxes; marshals to the C entry points."""

    def __init__(self, boxes, particles=None, precision=LB_FP32, didt_mode=0, device=0, max_semi=16,
                 max_particles=None, fp16_scale=0.0, separate_kernels=False, torch_alloc=False, collision=0,
                 lattice=19):
        self.boxes = [dict(b) for b in boxes]
        self.Q = int(lattice)
        parts = particles or [[] for _ in boxes]
        opt = Options()
        opt.precision, opt.didt_mode, opt.device = precision, didt_mode, device
        opt.flags = LB_FLAG_SEPARATE_KERNELS if separate_kernels else 0
        opt.max_semi = int(max_semi)
        opt.max_particles = int(max_particles or max(1, sum(len(p) for p in parts)))
        opt.fp16_scale = float(fp16_scale)
        opt.collision = int(collision)
        opt.lattice = self.Q
        self._alloc = None
        if torch_alloc:
            self._alloc = _torch_allocator(device)
            opt.alloc, opt.release = self._alloc
        self.ctx = lb_create(self.boxes, opt)
        self.nparts = [0] * len(boxes)
        self._parts = [[] for _ in boxes]
        for b, plist in enumerate(parts):
            if plist:
                self.set_particles(b, plist)

    def close(self):
        if getattr(self, "ctx", None):
            lb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_particles(self, box, plist):
        lb_set_particles(self.ctx, box, plist)
        self.nparts[box] = len(plist)
        self._parts[box] = [dict(p) for p in plist]

    def parts_of(self, box: int):
        """The particle dictionaries last given for a box (initial state)."""
        return [dict(p) for p in self._parts[box]]

    def step(self, n=1, stream=None):
        lb_step(self.ctx, n, stream)

    def sync(self):
        lb_synchronize(self.ctx)

    def field(self, name: str, box: int = 0) -> np.ndarray:
        b = self.boxes[box]
        N = b["nx"] * b["ny"] * b["nz"]
        what = _FIELD_NAMES[name]
        shape = {"f": (self.Q,), "df": (self.Q,), "rho": (), "u": (3,), "solid": ()}[name] + (b["nz"], b["ny"], b["nx"])
        out = np.zeros(shape, np.int32 if name == "solid" else np.float32)
        lb_get_fields(self.ctx, box, what, out.ctypes.data, out.nbytes, False)
        assert out.size * 4 == out.nbytes and out.size == int(np.prod(shape)) and N > 0
        return out

    def records(self, box: int = 0) -> np.ndarray:
        return lb_get_force_torque(self.ctx, box, self.nparts[box])

    def particle(self, box: int = 0, p: int = 0) -> dict:
        r = self.records(box)[p]
        return {"F0": r[0:3], "T0": r[3:6], "F": r[6:9], "T": r[9:12], "U": r[12:15],
                "Om": r[15:18], "x": r[18:21], "q": r[21:25], "raw": r}

    def links(self, box: int = 0, p: int = 0):
        return lb_get_links(self.ctx, box, p)

    def drag(self, box: int = 0, p: int = 0):
        return lb_get_drag(self.ctx, box, p)

    def init_fluid(self, box: int, u: np.ndarray, drho: np.ndarray | None = None, with_stress: bool = False):
        """Initial velocity field u (host, [3][nz][ny][nx]) and density
        deviation drho (host, [nz][ny][nx], or None) of a box."""
        a = np.ascontiguousarray(np.asarray(u, np.float32))
        d = None if drho is None else np.ascontiguousarray(np.asarray(drho, np.float32))
        lb_init_fluid(self.ctx, box, a.ctypes.data, a.nbytes, None if d is None else d.ctypes.data, False,
                      with_stress)

    def set_external(self, box, ft, stream=None):
        lb_set_external(self.ctx, box, ft, stream)
