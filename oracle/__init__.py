"""Oracle for the condensed-space IPM hot path (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA product path never imports,
links or executes anything here, and this package imports nothing from the
CUDA package (the seeded input generators live in a module of their own that
holds no arithmetic of the method).

Contents, each a plain FP64 restatement of the paper:

* ``ipm_solve``      -- Mehrotra predictor-corrector IPM on the uncondensed
                        problem (Eq. 1, Eqs. 4-6), Riccati recursion per Newton
                        step; plain C in ``ipm.c``.
* ``gstack``         -- the blocks A^k B of the state-elimination matrix (the
                        bold-B matrix of Section II, Eq. 2), by repeated products.
* ``condensed``      -- Gamma (bold B without its zero first block row),
                        y = Phi xbar, H and h of the dense QP (Eq. 3), by
                        simulating unit impulses and multiplying out.
* ``kkt_matrix``     -- the condensed KKT matrix H + J' Sigma J of Eq. 7 with
                        J = [Gamma; -Gamma; I; -I].
* ``kkt_entries``    -- selected entries of the same matrix from the G-stack,
                        for sizes where the dense product is too slow.
* ``kkt_check``      -- the KKT conditions (Eq. 5) of a candidate (u, z).

Parity unpinned: none.  Every function here has a pin in
``tests/test_oracle_*.py`` (brute force, LQR closed form, scalar closed form,
impulse-response identities, quadratic-form identities, KKT invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "liboracle.so")
TRACE_W = 6
STATUS_OK, STATUS_NOT_PD, STATUS_MAXITER, STATUS_NAN = 0, 3, 4, 6


def build(force: bool = False) -> str:
    """Compile ipm.c into liboracle.so (plain C, gcc -O3)."""
    src = os.path.join(_HERE, "ipm.c")
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        subprocess.check_call(["gcc", "-O3", "-march=native", "-fPIC", "-shared", "-std=c11",
                               "-o", _LIB, src, "-lm"])
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [("ns", ctypes.c_int), ("nu", ctypes.c_int), ("N", ctypes.c_int),
                ("a_ptr", ctypes.c_void_p), ("a_idx", ctypes.c_void_p), ("a_val", ctypes.c_void_p),
                ("B", ctypes.c_void_p),
                ("q_ptr", ctypes.c_void_p), ("q_idx", ctypes.c_void_p), ("q_val", ctypes.c_void_p),
                ("qf_ptr", ctypes.c_void_p), ("qf_idx", ctypes.c_void_p), ("qf_val", ctypes.c_void_p),
                ("R", ctypes.c_void_p),
                ("xl", ctypes.c_void_p), ("xu", ctypes.c_void_p),
                ("ul", ctypes.c_void_p), ("uu", ctypes.c_void_p),
                ("S", ctypes.c_void_p), ("w", ctypes.c_void_p), ("nc", ctypes.c_int),
                ("E", ctypes.c_void_p), ("F", ctypes.c_void_p), ("gl", ctypes.c_void_p),
                ("gu", ctypes.c_void_p)]


class _Options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("tau", ctypes.c_double),
                ("u_init", ctypes.c_void_p), ("mu0", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("m", ctypes.c_int),
                ("mu", ctypes.c_double), ("res_d", ctypes.c_double), ("res_p", ctypes.c_double),
                ("res", ctypes.c_double), ("hnorm", ctypes.c_double), ("dnorm", ctypes.c_double)]


_lib_handle = None


def _lib():
    global _lib_handle
    if _lib_handle is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.orc_ipm_solve.restype = ctypes.c_int
        lib.orc_ipm_solve.argtypes = [ctypes.POINTER(_Problem), ctypes.c_void_p,
                                      ctypes.POINTER(_Options), ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.POINTER(_Stats), ctypes.c_void_p]
        _lib_handle = lib
    return _lib_handle


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _csr(m, n):
    m = sp.csr_matrix(m, dtype=np.float64, shape=(n, n))
    m.sort_indices()
    return (np.ascontiguousarray(m.indptr, dtype=np.int32),
            np.ascontiguousarray(m.indices, dtype=np.int32),
            np.ascontiguousarray(m.data, dtype=np.float64))


def _general_arrays(plant, ns, nu, N, nc):
    """The optional data of Eq. 1 as C-ordered FP64 arrays (None when absent).
    A feedback K is not the oracle's business: it reparametrises the inputs
    (u = K x + v) without changing the problem or its minimiser."""
    def col(m, r, c):
        return None if m is None else np.asfortranarray(np.asarray(m, dtype=np.float64).reshape(r, c))
    out = {"S": col(getattr(plant, "S", None), ns, nu),
           "w": None if getattr(plant, "w", None) is None else
           np.ascontiguousarray(np.asarray(plant.w, dtype=np.float64).reshape(N, ns)),
           "E": None, "F": None, "gl": None, "gu": None}
    if nc:
        out["E"] = col(plant.E, nc, ns)
        out["F"] = col(plant.F, nc, nu)
        out["gl"] = np.ascontiguousarray(plant.gl, dtype=np.float64).reshape(nc)
        out["gu"] = np.ascontiguousarray(plant.gu, dtype=np.float64).reshape(nc)
    return out


def ipm_solve(plant, x0, *, tol: float = 1e-8, max_iter: int = 100, tau: float = 0.995,
              want_trace: bool = False, u_init=None, mu0: float = 0.0):
    """Run the oracle IPM (cold, or warm-started from the guess u_init with
    complementarity mu0).  Returns dict(u, x, z, stats, trace)."""
    ns, nu, N = plant.ns, plant.nu, plant.N
    n = nu * N
    keep = []
    a = _csr(plant.A, ns)
    q = _csr(plant.Q, ns)
    qf = _csr(plant.Qf, ns)
    B = np.asfortranarray(np.asarray(plant.B, dtype=np.float64).reshape(ns, nu))
    R = np.asfortranarray(np.asarray(plant.R, dtype=np.float64).reshape(nu, nu))
    vecs = [np.ascontiguousarray(v, dtype=np.float64) for v in (plant.xl, plant.xu, plant.ul, plant.uu)]
    keep += [a, q, qf, B, R, vecs]
    nc = getattr(plant, "nc", 0)
    gen = _general_arrays(plant, ns, nu, N, nc)
    keep.append(gen)
    pb = _Problem(ns, nu, N, _ptr(a[0]), _ptr(a[1]), _ptr(a[2]), _ptr(B),
                  _ptr(q[0]), _ptr(q[1]), _ptr(q[2]), _ptr(qf[0]), _ptr(qf[1]), _ptr(qf[2]),
                  _ptr(R), _ptr(vecs[0]), _ptr(vecs[1]), _ptr(vecs[2]), _ptr(vecs[3]),
                  _ptr(gen["S"]), _ptr(gen["w"]), nc, _ptr(gen["E"]), _ptr(gen["F"]), _ptr(gen["gl"]),
                  _ptr(gen["gu"]))
    ui = None if u_init is None else np.ascontiguousarray(u_init, dtype=np.float64).reshape(n)
    keep.append(ui)
    op = _Options(tol, max_iter, tau, _ptr(ui), mu0)
    xb = np.ascontiguousarray(x0, dtype=np.float64)
    u = np.zeros(n)
    x = np.zeros(ns * N)
    z = np.zeros(2 * ns * N + 2 * n + 2 * nc * N)
    st = _Stats()
    tr = np.zeros((max_iter + 1, TRACE_W)) if want_trace else None
    rc = _lib().orc_ipm_solve(ctypes.byref(pb), _ptr(xb), ctypes.byref(op), _ptr(u), _ptr(x),
                              _ptr(z), ctypes.byref(st), _ptr(tr))
    stats = {k: getattr(st, k) for k, _ in _Stats._fields_}
    out = {"u": u, "x": x.reshape(N, ns), "z": z, "stats": stats, "status": rc}
    if want_trace:
        out["trace"] = tr[: st.iters + 1].copy()
    return out


# ---------------------------------------------------------------------------
# Plain definitions (numpy, FP64)
# ---------------------------------------------------------------------------

def gstack(plant) -> np.ndarray:
    """G[k] = A^k B for k = 0..N-1 (Section II, blocks of bold B), shape (N, ns, nu)."""
    A = plant.A
    G = np.zeros((plant.N, plant.ns, plant.nu))
    cur = np.asarray(plant.B, dtype=np.float64).copy()
    for k in range(plant.N):
        G[k] = cur
        cur = A @ cur
    return G


def simulate(plant, x0, u) -> np.ndarray:
    """States x_1..x_N of x_{t+1} = A x_t + B u_t from x_0 = x0, shape (N, ns)."""
    x = np.asarray(x0, dtype=np.float64).copy()
    u = np.asarray(u, dtype=np.float64).reshape(plant.N, plant.nu)
    out = np.zeros((plant.N, plant.ns))
    for t in range(plant.N):
        x = plant.A @ x + plant.B @ u[t]
        out[t] = x
    return out


def condensed(plant, x0):
    """Gamma (ns*N x nu*N), y = Phi x0 (ns*N), H and h of Eq. 3.

    Gamma's column (t, c) is the state response to a unit impulse on input c at
    time t (the reduction x = Phi xbar + Gamma u of Section II); H = Gamma' Qbar
    Gamma + Rbar and h = Gamma' Qbar y with Qbar = blkdiag(Q, ..., Q, Qf)."""
    ns, nu, N = plant.ns, plant.nu, plant.N
    n = nu * N
    zero = np.zeros(ns)
    Gam = np.zeros((ns * N, n))
    for t in range(N):
        for c in range(nu):
            e = np.zeros(n)
            e[t * nu + c] = 1.0
            Gam[:, t * nu + c] = simulate(plant, zero, e).reshape(-1)
    y = simulate(plant, x0, np.zeros(n)).reshape(-1)
    Qd = plant.dense("Q")
    Qfd = plant.dense("Qf")
    Qbar = sp.block_diag([sp.csr_matrix(Qd)] * (N - 1) + [sp.csr_matrix(Qfd)], format="csr")
    Rbar = np.kron(np.eye(N), np.asarray(plant.R))
    QG = Qbar @ Gam
    H = Gam.T @ QG + Rbar
    h = Gam.T @ (Qbar @ y)
    return Gam, y, H, h


def kkt_matrix(plant, sigx, sigu, Gam=None, H=None):
    """M = H + Gamma' diag(sigx) Gamma + diag(sigu)  (Eq. 7 with J = [Gamma; -Gamma; I; -I],
    the two Gamma row blocks' Sigma summed into sigx)."""
    if Gam is None or H is None:
        Gam, _, H, _ = condensed(plant, np.zeros(plant.ns))
    return H + Gam.T @ (np.asarray(sigx)[:, None] * Gam) + np.diag(sigu)


def kkt_entries(plant, sigx, sigu, pairs, G=None, H=None):
    """Entries M[j, k] for the (j, k) in `pairs`, from the G-stack:
    M[j,k] = H[j,k] + sum_{rows} Gamma[row, j] sigx[row] Gamma[row, k] + [j==k] sigu[j],
    with Gamma[(r, i), (t, c)] = (A^{r-t} B)[i, c] for r >= t (states x_{r+1})."""
    ns, nu, N = plant.ns, plant.nu, plant.N
    if G is None:
        G = gstack(plant)
    sx = np.asarray(sigx).reshape(N, ns)
    out = np.zeros(len(pairs))
    for q, (j, k) in enumerate(pairs):
        tj, cj = divmod(j, nu)
        tk, ck = divmod(k, nu)
        acc = 0.0
        for r in range(max(tj, tk), N):
            acc += np.dot(G[r - tj][:, cj] * sx[r], G[r - tk][:, ck])
        out[q] = (H[j, k] if H is not None else 0.0) + acc + (sigu[j] if j == k else 0.0)
    return out


def hessian_entries(plant, pairs, G=None):
    """Entries of H = Gamma' Qbar Gamma + Rbar from the G-stack (any Q, Qf)."""
    ns, nu, N = plant.ns, plant.nu, plant.N
    if G is None:
        G = gstack(plant)
    Q = plant.csr("Q")
    Qf = plant.csr("Qf")
    R = np.asarray(plant.R)
    out = np.zeros(len(pairs))
    for q, (j, k) in enumerate(pairs):
        tj, cj = divmod(j, nu)
        tk, ck = divmod(k, nu)
        acc = 0.0
        for r in range(max(tj, tk), N):
            W = Qf if r == N - 1 else Q
            acc += np.dot(G[r - tj][:, cj], W @ G[r - tk][:, ck])
        if tj == tk:
            acc += R[cj, ck]
        out[q] = acc
    return out


def adjoint_gradient(plant, xtraj, w):
    """g = Gamma' w for w over state rows (N, ns), by the backward recursion
    p_N = w_N, p_t = w_t + A' p_{t+1}, g_t = B' p_{t+1}."""
    N = plant.N
    w = np.asarray(w).reshape(N, plant.ns)
    At = plant.A.T
    p = np.zeros(plant.ns)
    g = np.zeros((N, plant.nu))
    for t in range(N - 1, -1, -1):
        p = w[t] + (At @ p if t < N - 1 else 0.0)
        g[t] = plant.B.T @ p
    return g.reshape(-1)


def kkt_check(plant, x0, u, z=None):
    """KKT quantities (Eq. 5) of a candidate u (and duals z = [z_xu, z_xl, z_uu, z_ul]).

    Returns a dict with max primal violation, and, when z is given, the
    stationarity residual ||Hu + h + J'z||_inf, complementarity max |s_i z_i|
    and its mean over the finite one-sided constraints (the mu of the
    interior-point stop test), with s the slacks of u."""
    ns, nu, N = plant.ns, plant.nu, plant.N
    n = nu * N
    x = simulate(plant, x0, u)
    uu = np.asarray(u).reshape(N, nu)
    viol = max(
        np.max(np.where(np.isfinite(plant.xu), x - plant.xu, 0.0), initial=0.0),
        np.max(np.where(np.isfinite(plant.xl), plant.xl - x, 0.0), initial=0.0),
        np.max(np.where(np.isfinite(plant.uu), uu - plant.uu, 0.0), initial=0.0),
        np.max(np.where(np.isfinite(plant.ul), plant.ul - uu, 0.0), initial=0.0))
    out = {"primal_violation": float(viol)}
    if z is not None:
        z = np.asarray(z)
        SX = ns * N
        z1, z2 = z[:SX].reshape(N, ns), z[SX:2 * SX].reshape(N, ns)
        z3, z4 = z[2 * SX:2 * SX + n].reshape(N, nu), z[2 * SX + n:].reshape(N, nu)
        Q = plant.csr("Q")
        Qf = plant.csr("Qf")
        w = np.zeros((N, ns))
        for t in range(N):
            W = Qf if t == N - 1 else Q
            w[t] = W @ x[t] + z1[t] - z2[t]
        g = adjoint_gradient(plant, x, w) + (uu @ np.asarray(plant.R).T).reshape(-1) \
            + (z3 - z4).reshape(-1)
        s1 = np.where(np.isfinite(plant.xu), plant.xu - x, np.inf)
        s2 = np.where(np.isfinite(plant.xl), x - plant.xl, np.inf)
        s3 = np.where(np.isfinite(plant.uu), plant.uu - uu, np.inf)
        s4 = np.where(np.isfinite(plant.ul), uu - plant.ul, np.inf)
        comp, csum, m = 0.0, 0.0, 0
        for s_, z_ in ((s1, z1), (s2, z2), (s3, z3), (s4, z4)):
            fin = np.isfinite(s_)
            if fin.any():
                comp = max(comp, float(np.max(np.abs(s_[fin] * z_[fin]))))
                csum += float(np.sum(np.abs(s_[fin] * z_[fin])))
                m += int(fin.sum())
        out["stationarity"] = float(np.max(np.abs(g)))
        out["complementarity"] = comp
        out["complementarity_mean"] = csum / m if m else 0.0
        out["dual_min"] = float(min(z1.min(initial=0), z2.min(initial=0), z3.min(initial=0),
                                    z4.min(initial=0)))
    return out
