"""ctypes binding of liblqmpc.so (argument marshalling only).

Every computation runs in the CUDA library; this module converts numpy /
torch arguments to pointers and status codes to exceptions.  If the shared
library is missing or no CUDA device is usable, calls raise -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblqmpc.so")

FP64, MIXED_BF16, MIXED_TF32, FP32, FP32X2 = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": FP64, "bf16": MIXED_BF16, "tf32": MIXED_TF32, "fp32": FP32, "fp32x2": FP32X2}

STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "KKT matrix not positive definite",
          4: "iteration limit reached", 5: "infeasible", 6: "non-finite iterate",
          7: "iterative refinement stalled", 8: "device wait timed out", 9: "unsupported option or size"}

EXPORTS = ["lqmpc_default_options", "lqmpc_status_str", "lqmpc_setup", "lqmpc_set_options",
           "lqmpc_solve", "lqmpc_solve_device", "lqmpc_solve_batch", "lqmpc_free",
           "lqmpc_get_gstack", "lqmpc_get_hessian", "lqmpc_gamma_mv", "lqmpc_gamma_tmv",
           "lqmpc_form_kkt", "lqmpc_kkt_solve", "lqmpc_get_trace", "lqmpc_get_duals",
           "lqmpc_kernel_launches", "lqmpc_form_kkt_noalloc", "lqmpc_solve_warm", "lqmpc_mlp_create",
           "lqmpc_mlp_set_bounds", "lqmpc_mlp_get_params", "lqmpc_mlp_set_params", "lqmpc_mlp_grad",
           "lqmpc_mlp_train", "lqmpc_mlp_infer", "lqmpc_mlp_free", "lqmpc_autotune",
           "lqmpc_solve_batch_warm", "lqmpc_setup_general"]


class LqmpcError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, 'unknown')} ({code})")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("precision", ctypes.c_int),
                ("refine_max", ctypes.c_int), ("refine_tol", ctypes.c_double), ("fallback", ctypes.c_int),
                ("tau", ctypes.c_double), ("verbose", ctypes.c_int)]


class General(ctypes.Structure):
    _fields_ = [("S", ctypes.c_void_p), ("w", ctypes.c_void_p), ("nc", ctypes.c_int), ("E", ctypes.c_void_p),
                ("F", ctypes.c_void_p), ("gl", ctypes.c_void_p), ("gu", ctypes.c_void_p), ("K", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("refine_steps", ctypes.c_int), ("fallbacks", ctypes.c_int),
                ("status", ctypes.c_int), ("mu", ctypes.c_double), ("res_primal", ctypes.c_double),
                ("res_dual", ctypes.c_double), ("t_total_ms", ctypes.c_double), ("t_kkt_ms", ctypes.c_double),
                ("t_syrk_tc_ms", ctypes.c_double), ("t_syrk_cc_ms", ctypes.c_double),
                ("syrk_tc_launches", ctypes.c_int), ("syrk_cc_launches", ctypes.c_int),
                ("t_syrk_fp64_ms", ctypes.c_double), ("syrk_fp64_launches", ctypes.c_int),
                ("t_syrk_tc3_ms", ctypes.c_double), ("syrk_tc3_launches", ctypes.c_int),
                ("t_potrf32_ms", ctypes.c_double), ("potrf32_launches", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH):
    """Load liblqmpc.so (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"liblqmpc.so not built ({path}); run paper_2209_13049_b300.build")
    lib = ctypes.CDLL(path)
    P, I, D, VP = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    lib.lqmpc_default_options.restype = Options
    lib.lqmpc_status_str.restype = ctypes.c_char_p
    lib.lqmpc_status_str.argtypes = [I]
    lib.lqmpc_setup.restype = I
    lib.lqmpc_setup.argtypes = [ctypes.POINTER(P), I, I, I, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P,
                                ctypes.POINTER(Options), VP]
    lib.lqmpc_setup_general.restype = I
    lib.lqmpc_setup_general.argtypes = [ctypes.POINTER(P), I, I, I, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P,
                                        ctypes.POINTER(General), ctypes.POINTER(Options), VP]
    lib.lqmpc_set_options.restype = I
    lib.lqmpc_set_options.argtypes = [P, ctypes.POINTER(Options)]
    for name in ("lqmpc_solve", "lqmpc_solve_device"):
        f = getattr(lib, name)
        f.restype = I
        f.argtypes = [P, P, P, ctypes.POINTER(Stats)]
    lib.lqmpc_solve_batch.restype = I
    lib.lqmpc_solve_batch.argtypes = [P, I, P, P, P]
    lib.lqmpc_solve_batch_warm.restype = I
    lib.lqmpc_solve_batch_warm.argtypes = [P, I, P, P, D, P, P]
    lib.lqmpc_free.restype = None
    lib.lqmpc_free.argtypes = [P]
    for name in ("lqmpc_get_gstack", "lqmpc_get_hessian", "lqmpc_get_duals"):
        f = getattr(lib, name)
        f.restype = I
        f.argtypes = [P, P]
    for name in ("lqmpc_gamma_mv", "lqmpc_gamma_tmv"):
        f = getattr(lib, name)
        f.restype = I
        f.argtypes = [P, P, P]
    lib.lqmpc_form_kkt.restype = I
    lib.lqmpc_form_kkt.argtypes = [P, P, P, I, P]
    lib.lqmpc_form_kkt_noalloc.restype = I
    lib.lqmpc_form_kkt_noalloc.argtypes = [P, P, P, P]
    lib.lqmpc_kkt_solve.restype = I
    lib.lqmpc_kkt_solve.argtypes = [P, P, P, I, P, P, P, ctypes.POINTER(I)]
    lib.lqmpc_kernel_launches.restype = ctypes.c_ulonglong
    lib.lqmpc_kernel_launches.argtypes = []
    lib.lqmpc_get_trace.restype = I
    lib.lqmpc_get_trace.argtypes = [P, P, I, ctypes.POINTER(I)]
    lib.lqmpc_solve_warm.restype = I
    lib.lqmpc_solve_warm.argtypes = [P, P, P, D, P, ctypes.POINTER(Stats)]
    lib.lqmpc_mlp_create.restype = I
    lib.lqmpc_mlp_create.argtypes = [ctypes.POINTER(P), I, I, I, I, ctypes.c_ulonglong, VP]
    lib.lqmpc_mlp_set_bounds.restype = I
    lib.lqmpc_mlp_set_bounds.argtypes = [P, P, P]
    for name in ("lqmpc_mlp_get_params", "lqmpc_mlp_set_params"):
        f = getattr(lib, name)
        f.restype = I
        f.argtypes = [P, P]
    lib.lqmpc_mlp_grad.restype = I
    lib.lqmpc_mlp_grad.argtypes = [P, P, P, I, P, ctypes.POINTER(D)]
    lib.lqmpc_mlp_train.restype = I
    lib.lqmpc_mlp_train.argtypes = [P, P, P, I, I, I, ctypes.c_float, ctypes.c_ulonglong, P]
    lib.lqmpc_mlp_infer.restype = I
    lib.lqmpc_mlp_infer.argtypes = [P, P, I, P]
    lib.lqmpc_mlp_free.restype = None
    lib.lqmpc_mlp_free.argtypes = [P]
    lib.lqmpc_autotune.restype = I
    lib.lqmpc_autotune.argtypes = [P, I, ctypes.c_char_p]
    _lib = lib
    return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _csr(m, n):
    m = sp.csr_matrix(m, dtype=np.float64, shape=(n, n))
    m.sort_indices()
    return (np.ascontiguousarray(m.indptr, dtype=np.int32), np.ascontiguousarray(m.indices, dtype=np.int32),
            np.ascontiguousarray(m.data, dtype=np.float64))


def default_options(**kw) -> Options:
    o = load().lqmpc_default_options()
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        setattr(o, k, v)
    return o


def _check(code: int, where: str):
    if code != 0:
        raise LqmpcError(code, where)


class Solver:
    """One plant's solver context (wraps lqmpc_setup / lqmpc_free)."""

    def __init__(self, plant, options: Options | None = None, stream=None, **kw):
        lib = load()
        self.plant = plant
        self.ns, self.nu, self.N = plant.ns, plant.nu, plant.N
        self.n = self.nu * self.N
        o = options or default_options(**kw)
        a, q, qf = _csr(plant.A, self.ns), _csr(plant.Q, self.ns), _csr(plant.Qf, self.ns)
        B = np.asfortranarray(np.asarray(plant.B, dtype=np.float64).reshape(self.ns, self.nu))
        R = np.asfortranarray(np.asarray(plant.R, dtype=np.float64).reshape(self.nu, self.nu))
        vec = [_f64(v) for v in (plant.xl, plant.xu, plant.ul, plant.uu)]
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0))
        # internal (lifted) state dimension: general rows and, with K, the inputs
        self.ns_int = self.ns
        if getattr(plant, "general", False):
            nc = plant.nc

            def col(m, r, c):
                return None if m is None else np.asfortranarray(np.asarray(m, dtype=np.float64).reshape(r, c))
            self._gen = {"S": col(plant.S, self.ns, self.nu),
                         "w": None if plant.w is None else _f64(np.asarray(plant.w).reshape(self.N, self.ns)),
                         "E": col(plant.E, nc, self.ns) if nc else None, "F": col(plant.F, nc, self.nu) if nc else None,
                         "gl": _f64(plant.gl) if nc else None, "gu": _f64(plant.gu) if nc else None,
                         "K": col(plant.K, self.nu, self.ns)}
            gd = self._gen
            g = General(_p(gd["S"]), _p(gd["w"]), nc, _p(gd["E"]), _p(gd["F"]), _p(gd["gl"]), _p(gd["gu"]),
                        _p(gd["K"]))
            self.ns_int = self.ns + nc + (self.nu if plant.K is not None else 0)
            code = lib.lqmpc_setup_general(ctypes.byref(h), self.ns, self.nu, self.N, _p(a[0]), _p(a[1]), _p(a[2]),
                                           _p(B), _p(q[0]), _p(q[1]), _p(q[2]), _p(qf[0]), _p(qf[1]), _p(qf[2]),
                                           _p(R), _p(vec[0]), _p(vec[1]), _p(vec[2]), _p(vec[3]), ctypes.byref(g),
                                           ctypes.byref(o), st)
            _check(code, "lqmpc_setup_general")
        else:
            code = lib.lqmpc_setup(ctypes.byref(h), self.ns, self.nu, self.N, _p(a[0]), _p(a[1]), _p(a[2]), _p(B),
                                   _p(q[0]), _p(q[1]), _p(q[2]), _p(qf[0]), _p(qf[1]), _p(qf[2]), _p(R),
                                   _p(vec[0]), _p(vec[1]), _p(vec[2]), _p(vec[3]), ctypes.byref(o), st)
            _check(code, "lqmpc_setup")
        self.h = h
        self.options = o

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            load().lqmpc_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, **kw):
        o = Options.from_buffer_copy(self.options)
        for k, v in kw.items():
            if k == "precision" and isinstance(v, str):
                v = PRECISIONS[v]
            setattr(o, k, v)
        _check(load().lqmpc_set_options(self.h, ctypes.byref(o)), "lqmpc_set_options")
        self.options = o

    def solve(self, x0, check: bool = True):
        x0 = _f64(x0)
        u = np.zeros(self.n)
        st = Stats()
        code = load().lqmpc_solve(self.h, _p(x0), _p(u), ctypes.byref(st))
        if check and code not in (0,):
            raise LqmpcError(code, "lqmpc_solve")
        return u, st.as_dict()

    def solve_device(self, x0_dev, u_dev, check: bool = True):
        """x0_dev, u_dev: CUDA float64 torch tensors (ns and nu*N elements)."""
        st = Stats()
        code = load().lqmpc_solve_device(self.h, ctypes.c_void_p(x0_dev.data_ptr()),
                                         ctypes.c_void_p(u_dev.data_ptr()), ctypes.byref(st))
        if check and code != 0:
            raise LqmpcError(code, "lqmpc_solve_device")
        return st.as_dict()

    def get_gstack(self):
        G = np.zeros((self.N, self.nu, self.ns_int))
        _check(load().lqmpc_get_gstack(self.h, _p(G)), "lqmpc_get_gstack")
        return np.transpose(G, (0, 2, 1)).copy()          # (N, ns, nu)

    def get_hessian(self):
        H = np.zeros((self.n, self.n), order="F")
        _check(load().lqmpc_get_hessian(self.h, _p(H)), "lqmpc_get_hessian")
        return np.asarray(H)

    def gamma_mv(self, v):
        v = _f64(v)
        out = np.zeros(self.ns_int * self.N)
        _check(load().lqmpc_gamma_mv(self.h, _p(v), _p(out)), "lqmpc_gamma_mv")
        return out

    def gamma_tmv(self, w):
        w = _f64(w)
        out = np.zeros(self.n)
        _check(load().lqmpc_gamma_tmv(self.h, _p(w), _p(out)), "lqmpc_gamma_tmv")
        return out

    def form_kkt(self, sigx, sigu, precision="fp64"):
        p = PRECISIONS[precision] if isinstance(precision, str) else precision
        M = np.zeros((self.n, self.n), order="F")
        _check(load().lqmpc_form_kkt(self.h, _p(_f64(sigx)), _p(_f64(sigu)), p, _p(M)), "lqmpc_form_kkt")
        return np.asarray(M)

    def solve_warm(self, x0, u_init, mu0: float = 0.0, check: bool = True):
        """Warm-started solve from the guess u_init (nu*N); returns (u, stats)."""
        u = np.zeros(self.n)
        st = Stats()
        code = load().lqmpc_solve_warm(self.h, _p(_f64(x0)), _p(_f64(u_init)), float(mu0), _p(u), ctypes.byref(st))
        if check and code != 0:
            raise LqmpcError(code, "lqmpc_solve_warm")
        return u, st.as_dict()

    def form_kkt_noalloc(self, sigx, sigu, M):
        """FP64 M into the CUDA tensor M (n x n, read column-major) from CUDA
        tensors sigx (ns*N) and sigu (n); allocates nothing and does not wait
        for the context's stream."""
        for name, t, size in (("sigx", sigx, self.ns_int * self.N), ("sigu", sigu, self.n),
                              ("M", M, self.n * self.n)):
            if not (t.is_cuda and str(t.dtype) == "torch.float64" and t.is_contiguous() and t.numel() == size):
                raise ValueError(f"{name}: contiguous float64 CUDA tensor of {size} elements expected")
        _check(load().lqmpc_form_kkt_noalloc(self.h, sigx.data_ptr(), sigu.data_ptr(), M.data_ptr()),
               "lqmpc_form_kkt_noalloc")

    def kkt_solve(self, sigx, sigu, rhs, precision="fp64", want_L=False, check=True):
        p = PRECISIONS[precision] if isinstance(precision, str) else precision
        x = np.zeros(self.n)
        L = np.zeros((self.n, self.n), order="F") if want_L else None
        steps = ctypes.c_int(0)
        code = load().lqmpc_kkt_solve(self.h, _p(_f64(sigx)), _p(_f64(sigu)), p, _p(_f64(rhs)), _p(x), _p(L),
                                      ctypes.byref(steps))
        if check:
            _check(code, "lqmpc_kkt_solve")
        return {"x": x, "L": None if L is None else np.asarray(L), "refine_steps": steps.value, "status": code}

    def get_trace(self, max_rows=None):
        max_rows = max_rows or (self.options.max_iter + 1)
        tr = np.zeros((max_rows, 8))
        rows = ctypes.c_int(0)
        _check(load().lqmpc_get_trace(self.h, _p(tr), max_rows, ctypes.byref(rows)), "lqmpc_get_trace")
        return tr[: rows.value].copy()

    def get_duals(self):
        z = np.zeros(2 * self.ns_int * self.N + 2 * self.n)
        _check(load().lqmpc_get_duals(self.h, _p(z)), "lqmpc_get_duals")
        return z


def kernel_launches() -> int:
    """Cumulative count of CUDA kernels launched by the library in this process."""
    return int(load().lqmpc_kernel_launches())


def autotune(solvers, cache_path=None):
    """Autotune the launch shapes of batches like this one (lqmpc_autotune)."""
    k = len(solvers)
    hs = (ctypes.c_void_p * k)(*[s.h.value for s in solvers])
    _check(load().lqmpc_autotune(ctypes.cast(hs, ctypes.c_void_p), k,
                                 None if cache_path is None else str(cache_path).encode()), "lqmpc_autotune")


def solve_batch(solvers, x0s, check: bool = True, u_inits=None, mu0: float = 0.0):
    """Solve every (solver, x0) pair in one lockstep batch (lqmpc_solve_batch);
    with u_inits, every instance starts from its guess (lqmpc_solve_batch_warm)."""
    lib = load()
    k = len(solvers)
    x0a = [_f64(x) for x in x0s]
    us = [np.zeros(s.n) for s in solvers]
    hs = (ctypes.c_void_p * k)(*[s.h.value for s in solvers])
    xp = (ctypes.c_void_p * k)(*[x.ctypes.data for x in x0a])
    up = (ctypes.c_void_p * k)(*[u.ctypes.data for u in us])
    stats = (Stats * k)()
    if u_inits is None:
        code = lib.lqmpc_solve_batch(ctypes.cast(hs, ctypes.c_void_p), k, ctypes.cast(xp, ctypes.c_void_p),
                                     ctypes.cast(up, ctypes.c_void_p), ctypes.cast(stats, ctypes.c_void_p))
        where = "lqmpc_solve_batch"
    else:
        ga = [_f64(g) for g in u_inits]
        gp = (ctypes.c_void_p * k)(*[g.ctypes.data for g in ga])
        code = lib.lqmpc_solve_batch_warm(ctypes.cast(hs, ctypes.c_void_p), k, ctypes.cast(xp, ctypes.c_void_p),
                                          ctypes.cast(gp, ctypes.c_void_p), float(mu0),
                                          ctypes.cast(up, ctypes.c_void_p), ctypes.cast(stats, ctypes.c_void_p))
        where = "lqmpc_solve_batch_warm"
    if check and code != 0:
        raise LqmpcError(code, where)
    return us, [s.as_dict() for s in stats], code


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


class MLP:
    """The warm-start network (lqmpc_mlp_*): n_in -> n_hidden -> n_hidden -> n_out."""

    def __init__(self, n_in: int, n_hidden: int, n_out: int, max_batch: int, seed: int = 0, stream=None):
        self.n_in, self.n_hidden, self.n_out = n_in, n_hidden, n_out
        self.h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0))
        _check(load().lqmpc_mlp_create(ctypes.byref(self.h), n_in, n_hidden, n_out, max_batch, seed, st),
               "lqmpc_mlp_create")

    @property
    def n_params(self) -> int:
        i, h, o = self.n_in, self.n_hidden, self.n_out
        return h * i + h + h * h + h + o * h + o

    def set_bounds(self, lo, hi):
        _check(load().lqmpc_mlp_set_bounds(self.h, _p(_f64(lo)), _p(_f64(hi))), "lqmpc_mlp_set_bounds")

    def get_params(self):
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(load().lqmpc_mlp_get_params(self.h, _p(out)), "lqmpc_mlp_get_params")
        return out

    def set_params(self, flat):
        _check(load().lqmpc_mlp_set_params(self.h, _p(_f32(flat))), "lqmpc_mlp_set_params")

    def grad(self, X, U):
        X, U = _f32(X), _f32(U)
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = ctypes.c_double(0.0)
        _check(load().lqmpc_mlp_grad(self.h, _p(X), _p(U), X.shape[0], _p(g), ctypes.byref(loss)), "lqmpc_mlp_grad")
        return g, loss.value

    def train(self, X, U, epochs: int, batch: int, lr: float, seed: int = 0):
        X, U = _f32(X), _f32(U)
        losses = np.zeros(max(epochs, 1))
        _check(load().lqmpc_mlp_train(self.h, _p(X), _p(U), X.shape[0], epochs, batch, float(lr), seed, _p(losses)),
               "lqmpc_mlp_train")
        return losses[:epochs]

    def infer(self, X):
        X = _f64(X)
        out = np.zeros((X.shape[0], self.n_out))
        _check(load().lqmpc_mlp_infer(self.h, _p(X), X.shape[0], _p(out)), "lqmpc_mlp_infer")
        return out

    def close(self):
        if self.h:
            load().lqmpc_mlp_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
