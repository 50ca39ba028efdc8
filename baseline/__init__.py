"""CPU condensed-dense baseline (a comparison baseline, not product code).

The condensed-space interior-point method of Section III (dense M of Eq. 7,
dense Cholesky, Mehrotra predictor-corrector) on the host cores with OpenMP:
the analogue of the "CPU dense" columns of the paper's Tables II-V.  The
benchmark times it beside the GPU solver as context; its tests compare it
with the oracle.  The CUDA package never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "libcpu_dense.so")
STATUS_OK = 0


def build(force: bool = False) -> str:
    """Compile cpu_dense.c into libcpu_dense.so (gcc -O3 -fopenmp)."""
    src = os.path.join(_HERE, "cpu_dense.c")
    hdr = os.path.join(_HERE, "cpu_dense.h")
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(src),
                                                                          os.path.getmtime(hdr)):
        subprocess.check_call(["gcc", "-O3", "-march=native", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", _LIB, src, "-lm"])
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [("ns", ctypes.c_int), ("nu", ctypes.c_int), ("N", ctypes.c_int),
                ("a_ptr", ctypes.c_void_p), ("a_idx", ctypes.c_void_p), ("a_val", ctypes.c_void_p),
                ("B", ctypes.c_void_p),
                ("q_ptr", ctypes.c_void_p), ("q_idx", ctypes.c_void_p), ("q_val", ctypes.c_void_p),
                ("qf_ptr", ctypes.c_void_p), ("qf_idx", ctypes.c_void_p), ("qf_val", ctypes.c_void_p),
                ("R", ctypes.c_void_p),
                ("xl", ctypes.c_void_p), ("xu", ctypes.c_void_p), ("ul", ctypes.c_void_p), ("uu", ctypes.c_void_p)]


class _Options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("tau", ctypes.c_double),
                ("threads", ctypes.c_int)]


class _Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("threads", ctypes.c_int),
                ("mu", ctypes.c_double), ("res_d", ctypes.c_double), ("res_p", ctypes.c_double),
                ("res", ctypes.c_double), ("t_form_s", ctypes.c_double), ("t_factor_s", ctypes.c_double)]


_handle = None


def _lib():
    global _handle
    if _handle is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.cpd_solve.restype = ctypes.c_int
        lib.cpd_solve.argtypes = [ctypes.POINTER(_Problem), ctypes.c_void_p, ctypes.POINTER(_Options),
                                  ctypes.c_void_p, ctypes.POINTER(_Stats)]
        _handle = lib
    return _handle


def _csr(m, n):
    m = sp.csr_matrix(m, dtype=np.float64, shape=(n, n))
    m.sort_indices()
    return (np.ascontiguousarray(m.indptr, dtype=np.int32), np.ascontiguousarray(m.indices, dtype=np.int32),
            np.ascontiguousarray(m.data, dtype=np.float64))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def solve(plant, x0, *, tol: float = 1e-8, max_iter: int = 100, tau: float = 0.995, threads: int = 0):
    """Run the CPU condensed-dense IPM.  Returns dict(u, stats, status)."""
    ns, nu, N = plant.ns, plant.nu, plant.N
    a, q, qf = _csr(plant.A, ns), _csr(plant.Q, ns), _csr(plant.Qf, ns)
    B = np.asfortranarray(np.asarray(plant.B, dtype=np.float64).reshape(ns, nu))
    R = np.asfortranarray(np.asarray(plant.R, dtype=np.float64).reshape(nu, nu))
    vec = [np.ascontiguousarray(v, dtype=np.float64) for v in (plant.xl, plant.xu, plant.ul, plant.uu)]
    pb = _Problem(ns, nu, N, _p(a[0]), _p(a[1]), _p(a[2]), _p(B), _p(q[0]), _p(q[1]), _p(q[2]),
                  _p(qf[0]), _p(qf[1]), _p(qf[2]), _p(R), _p(vec[0]), _p(vec[1]), _p(vec[2]), _p(vec[3]))
    op = _Options(tol, max_iter, tau, threads)
    xb = np.ascontiguousarray(x0, dtype=np.float64)
    u = np.zeros(nu * N)
    st = _Stats()
    rc = _lib().cpd_solve(ctypes.byref(pb), _p(xb), ctypes.byref(op), _p(u), ctypes.byref(st))
    return {"u": u, "status": rc, "stats": {k: getattr(st, k) for k, _ in _Stats._fields_}}
