"""Python binding of include/lbsurrogate.h (argument marshalling only).

Every function named lb_* calls the C entry point of the same name in
liblbsph.so and raises LBError on a non-zero status.  Device buffers are
passed as integer addresses (e.g. torch.Tensor.data_ptr()); the tensor-core
products, the loss, the backward pass, the Adam step and the 6x6 solves all run
in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .lbsph import LBError, library

LB_MLP_IN, LB_MLP_IN_PAD, LB_MLP_HID, LB_MLP_OUT, LB_MLP_OUT_PAD = 8, 16, 256, 21, 32
LB_MLP_NPARAM = 256 * 16 + 256 + 256 * 256 + 256 + 32 * 256 + 32
LB_MLP_MAX_BATCH = 65536

# offsets of the parameter block (FP32, row-major [out][in])
OFF = {"W1": (0, (256, 16)), "b1": (4096, (256,)), "W2": (4352, (256, 256)), "b2": (69888, (256,)),
       "W3": (70144, (32, 256)), "b3": (78336, (32,))}

_bound = False


def _lib():
    global _bound
    L = library()
    if _bound:
        return L
    vp, i32, i64, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_float
    L.lb_gemm_bf16.argtypes = [vp, i64, i64, vp, i64, i64, i32, i32, i32, vp, i32, vp, vp, i64, i64, vp]
    L.lb_gemm_status.argtypes = []
    L.lb_mlp_create.argtypes = [i32, i32, C.POINTER(vp)]
    L.lb_mlp_destroy.argtypes = [vp]
    L.lb_mlp_set_params.argtypes = [vp, C.POINTER(C.c_float)]
    L.lb_mlp_get_params.argtypes = [vp, C.POINTER(C.c_float)]
    L.lb_mlp_forward.argtypes = [vp, vp, i32, vp, vp, vp]
    L.lb_mlp_loss_grad.argtypes = [vp, vp, vp, i32, vp, vp, vp]
    L.lb_mlp_train_step.argtypes = [vp, vp, vp, i32, f32, vp, vp]
    L.lb_spd_solve6.argtypes = [vp, vp, vp, i32, vp]
    L.lb_spd_invert6.argtypes = [vp, i32, vp]
    L.lb_mlp_features.argtypes = [vp, i32, vp, vp]
    L.lb_resistance_targets.argtypes = [vp, vp, i32, vp, vp]
    L.lb_warm_velocities.argtypes = [vp, vp, vp, i32, vp, vp]
    for n in ("lb_gemm_bf16", "lb_gemm_status", "lb_mlp_create", "lb_mlp_destroy", "lb_mlp_set_params",
              "lb_mlp_get_params", "lb_mlp_forward", "lb_mlp_loss_grad", "lb_mlp_train_step", "lb_spd_solve6",
              "lb_spd_invert6", "lb_mlp_features", "lb_resistance_targets", "lb_warm_velocities"):
        getattr(L, n).restype = i32
    _bound = True
    return L


def _check(rc: int, what: str):
    if rc != 0:
        raise LBError(rc, f"{what}: {library().lb_status_string(rc).decode()}")


def _p(x):
    return None if x is None else C.c_void_p(int(x))


def lb_gemm_bf16(A, a_sm, a_sk, B, b_sn, b_sk, M, N, K, bias=None, relu=0, C32=None, C16=None, c_sm=0, c_sn=1,
                 stream=None):
    _check(_lib().lb_gemm_bf16(_p(A), a_sm, a_sk, _p(B), b_sn, b_sk, M, N, K, _p(bias), int(relu), _p(C32), _p(C16),
                               c_sm, c_sn, stream), "lb_gemm_bf16")


def lb_gemm_status():
    _check(_lib().lb_gemm_status(), "lb_gemm_status")


def lb_mlp_create(device: int = 0, max_batch: int = 4096):
    h = C.c_void_p()
    _check(_lib().lb_mlp_create(device, max_batch, C.byref(h)), "lb_mlp_create")
    return h


def lb_mlp_destroy(m):
    _check(_lib().lb_mlp_destroy(m), "lb_mlp_destroy")


def lb_mlp_set_params(m, params: np.ndarray):
    a = np.ascontiguousarray(np.asarray(params, np.float32).reshape(-1))
    assert a.size == LB_MLP_NPARAM
    _check(_lib().lb_mlp_set_params(m, a.ctypes.data_as(C.POINTER(C.c_float))), "lb_mlp_set_params")


def lb_mlp_get_params(m) -> np.ndarray:
    a = np.zeros(LB_MLP_NPARAM, np.float32)
    _check(_lib().lb_mlp_get_params(m, a.ctypes.data_as(C.POINTER(C.c_float))), "lb_mlp_get_params")
    return a


def lb_mlp_forward(m, x_dev, n, y_dev=None, R_dev=None, stream=None):
    _check(_lib().lb_mlp_forward(m, _p(x_dev), n, _p(y_dev), _p(R_dev), stream), "lb_mlp_forward")


def lb_mlp_loss_grad(m, x_dev, Rt_dev, n, loss_dev, grad_dev=None, stream=None):
    _check(_lib().lb_mlp_loss_grad(m, _p(x_dev), _p(Rt_dev), n, _p(loss_dev), _p(grad_dev), stream),
           "lb_mlp_loss_grad")


def lb_mlp_train_step(m, x_dev, Rt_dev, n, lr, loss_dev=None, stream=None):
    _check(_lib().lb_mlp_train_step(m, _p(x_dev), _p(Rt_dev), n, float(lr), _p(loss_dev), stream),
           "lb_mlp_train_step")


def lb_spd_solve6(R_dev, f_dev, u_dev, n, stream=None):
    _check(_lib().lb_spd_solve6(_p(R_dev), _p(f_dev), _p(u_dev), n, stream), "lb_spd_solve6")


def lb_spd_invert6(M_dev, n, stream=None):
    _check(_lib().lb_spd_invert6(_p(M_dev), n, stream), "lb_spd_invert6")


def lb_mlp_features(geom_dev, n, x_dev, stream=None):
    _check(_lib().lb_mlp_features(_p(geom_dev), n, _p(x_dev), stream), "lb_mlp_features")


def lb_resistance_targets(M_dev, geom_dev, n, Rhat_dev, stream=None):
    _check(_lib().lb_resistance_targets(_p(M_dev), _p(geom_dev), n, _p(Rhat_dev), stream), "lb_resistance_targets")


def lb_warm_velocities(Rhat_dev, geom_dev, FT_dev, n, UW_dev, stream=None):
    _check(_lib().lb_warm_velocities(_p(Rhat_dev), _p(geom_dev), _p(FT_dev), n, _p(UW_dev), stream),
           "lb_warm_velocities")


def unpack(params: np.ndarray) -> dict:
    """Views of the named blocks of a parameter vector."""
    return {k: params[o:o + int(np.prod(s))].reshape(s) for k, (o, s) in OFF.items()}


class Surrogate:
    """An lb_mlp handle with its parameters."""

    def __init__(self, device: int = 0, max_batch: int = 4096, params: np.ndarray | None = None):
        self.h = lb_mlp_create(device, max_batch)
        if params is not None:
            lb_mlp_set_params(self.h, params)

    def close(self):
        if getattr(self, "h", None):
            lb_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        return lb_mlp_get_params(self.h)
