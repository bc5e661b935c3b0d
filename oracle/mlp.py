"""ctypes front end of the FP64 CPU oracle of the transport-data surrogate
(mlp_oracle.c): forward pass, mean-squared-error gradient and Adam.

TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the benchmark's
CPU-baseline leg import this module; the library never does, and this module
imports nothing from the library.  The arithmetic is in the C file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mlp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_mlp.so")
_lock = threading.Lock()
_lib = None

NI, NH, NO = 2, 128, 6
OFF = dict(W1=0, b1=NH * NI, W2=NH * NI + NH, b2=NH * NI + NH + NH * NH,
           W3=NH * NI + 2 * NH + NH * NH, b3=NH * NI + 2 * NH + NH * NH + NO * NH)
N_PARAMS = OFF["b3"] + NO
SHAPES = dict(W1=(NH, NI), b1=(NH,), W2=(NH, NH), b2=(NH,), W3=(NO, NH), b3=(NO,))

PD = C.POINTER(C.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            L.orc_mlp_n_params.restype = C.c_int
            L.orc_mlp_forward.argtypes = [PD, PD, C.c_int, PD]
            L.orc_mlp_loss_grad.argtypes = [PD, PD, PD, C.c_int, PD]
            L.orc_mlp_loss_grad.restype = C.c_double
            L.orc_mlp_adam.argtypes = [PD, PD, PD, PD, C.c_int, C.c_double, C.c_double, C.c_double,
                                       C.c_double]
            L.orc_mlp_train.argtypes = [PD, PD, PD, C.c_int, PD, PD, C.c_int, C.c_int, C.c_double,
                                        C.c_double, C.c_double, C.c_double]
            L.orc_mlp_train.restype = C.c_double
            assert L.orc_mlp_n_params() == N_PARAMS
            _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, np.float64)
    return a, a.ctypes.data_as(PD)


def unpack(theta):
    return {k: np.asarray(theta[OFF[k]:OFF[k] + int(np.prod(s))]).reshape(s) for k, s in SHAPES.items()}


def pack(parts: dict) -> np.ndarray:
    th = np.zeros(N_PARAMS)
    for k, s in SHAPES.items():
        th[OFF[k]:OFF[k] + int(np.prod(s))] = np.asarray(parts[k], np.float64).ravel()
    return th


def forward(theta, x):
    th, pt = _d(theta)
    xx, px = _d(x)
    n = xx.shape[0]
    y = np.zeros((n, NO))
    lib().orc_mlp_forward(pt, px, n, y.ctypes.data_as(PD))
    return y


def loss_grad(theta, x, t):
    th, pt = _d(theta)
    xx, px = _d(x)
    tt, ptt = _d(t)
    g = np.zeros(N_PARAMS)
    loss = lib().orc_mlp_loss_grad(pt, px, ptt, xx.shape[0], g.ctypes.data_as(PD))
    return loss, g


def adam(theta, m, v, g, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In place on float64 arrays theta, m, v."""
    for a in (theta, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    gg, pg = _d(g)
    lib().orc_mlp_adam(theta.ctypes.data_as(PD), m.ctypes.data_as(PD), v.ctypes.data_as(PD), pg, step, lr,
                       beta1, beta2, eps)


def train(theta, m, v, step0, x, t, n_steps, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In place; returns the loss before the last update."""
    xx, px = _d(x)
    tt, ptt = _d(t)
    return lib().orc_mlp_train(theta.ctypes.data_as(PD), m.ctypes.data_as(PD), v.ctypes.data_as(PD), step0,
                               px, ptt, xx.shape[0], n_steps, lr, beta1, beta2, eps)
