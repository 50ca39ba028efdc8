"""Independent references that pin the oracle (test helpers, numpy FP64).

None of these shares code with the oracle's IPM: each is a textbook or
brute-force statement of the same optimum.
"""
from __future__ import annotations

import itertools

import numpy as np


def simulate(A, B, x0, u, N):
    """x_1..x_N of x_{t+1} = A x_t + B u_t (dense A, B)."""
    A = np.asarray(A.toarray() if hasattr(A, "toarray") else A, dtype=np.float64)
    x = np.asarray(x0, dtype=np.float64)
    u = np.asarray(u).reshape(N, -1)
    out = []
    for t in range(N):
        x = A @ x + B @ u[t]
        out.append(x)
    return np.array(out)


def dense_qp(plant, x0):
    """Dense reduced QP (Eq. 3) built independently: Gamma by unit impulses,
    H = sum over stages of Gamma_t' Q_t Gamma_t + Rbar, h likewise."""
    ns, nu, N = plant.ns, plant.nu, plant.N
    n = nu * N
    Ad = plant.dense("A")
    Q, Qf, R = plant.dense("Q"), plant.dense("Qf"), np.asarray(plant.R)
    cols = []
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        cols.append(simulate(Ad, plant.B, np.zeros(ns), e, N).reshape(-1))
    Gam = np.array(cols).T
    y = simulate(Ad, plant.B, x0, np.zeros(n), N).reshape(-1)
    H = np.kron(np.eye(N), R)
    h = np.zeros(n)
    for t in range(N):
        W = Qf if t == N - 1 else Q
        Gt = Gam[t * ns:(t + 1) * ns]
        H += Gt.T @ W @ Gt
        h += Gt.T @ W @ y[t * ns:(t + 1) * ns]
    return Gam, y, H, h


def dense_qp_general(plant, x0):
    """Dense reduced QP of Eq. 1 with its general data, written out directly:
    x_t = y_t + Gamma_t u (y the free response, disturbance included, x_0 =
    xbar), the cost 1/2 sum x'Q x + 1/2 sum u'R u + sum_t x_t' S u_t expanded
    in u, and the general rows E x_t + F u_t as rows in u with offsets.
    Returns Gam, y, H, h and the general rows [(g, lo, hi)]."""
    ns, nu, N = plant.ns, plant.nu, plant.N
    n = nu * N
    Ad = plant.dense("A")
    B = np.asarray(plant.B, dtype=np.float64)
    w = np.zeros((N, ns)) if plant.w is None else np.asarray(plant.w, dtype=np.float64).reshape(N, ns)
    cols = []
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        cols.append(simulate(Ad, B, np.zeros(ns), e, N).reshape(-1))
    Gam = np.array(cols).T
    x = np.asarray(x0, dtype=np.float64)
    y = []
    for t in range(N):
        x = Ad @ x + w[t]
        y.append(x)
    y = np.concatenate(y)
    Q, Qf, R = plant.dense("Q"), plant.dense("Qf"), np.asarray(plant.R)
    H = np.kron(np.eye(N), R)
    h = np.zeros(n)
    for t in range(N):
        W = Qf if t == N - 1 else Q
        Gt = Gam[t * ns:(t + 1) * ns]
        H += Gt.T @ W @ Gt
        h += Gt.T @ W @ y[t * ns:(t + 1) * ns]

    def state(t):        # x_t = off + G u  (t = 0..N)
        if t == 0:
            return np.asarray(x0, dtype=np.float64), np.zeros((ns, n))
        return y[(t - 1) * ns:t * ns], Gam[(t - 1) * ns:t * ns]

    def sel(t):          # u_t = P u
        P = np.zeros((nu, n))
        P[:, t * nu:(t + 1) * nu] = np.eye(nu)
        return P

    if plant.S is not None:
        S = np.asarray(plant.S, dtype=np.float64).reshape(ns, nu)
        for t in range(N):
            off, G = state(t)
            P = sel(t)
            C = G.T @ S @ P
            H += C + C.T
            h += P.T @ S.T @ off
    rows = []
    if plant.E is not None:
        E = np.asarray(plant.E, dtype=np.float64).reshape(-1, ns)
        F = np.asarray(plant.F, dtype=np.float64).reshape(-1, nu)
        for t in range(N):
            off, G = state(t)
            Gr = E @ G + F @ sel(t)
            o = E @ off
            for r in range(E.shape[0]):
                rows.append((Gr[r], plant.gl[r] - o[r], plant.gu[r] - o[r]))
    return Gam, y, H, h, rows


def brute_force(plant, x0, tol=1e-9):
    """Unique minimiser of the strictly convex QP by enumerating every
    active-set pattern of the two-sided rows (free / at upper / at lower),
    solving the equality-constrained KKT system densely and keeping the
    pattern that is primal and dual feasible.  Tiny instances only."""
    if getattr(plant, "general", False):
        Gam, y, H, h, grows = dense_qp_general(plant, x0)
    else:
        Gam, y, H, h = dense_qp(plant, x0)
        grows = []
    ns, nu, N = plant.ns, plant.nu, plant.N
    n = nu * N
    rows = []   # (row vector g, lower bound, upper bound) for lo <= g u <= hi
    for t in range(N):
        for i in range(ns):
            k = t * ns + i
            if np.isfinite(plant.xl[i]) or np.isfinite(plant.xu[i]):
                rows.append((Gam[k], plant.xl[i] - y[k], plant.xu[i] - y[k]))
    for t in range(N):
        for c in range(nu):
            e = np.zeros(n)
            e[t * nu + c] = 1.0
            if np.isfinite(plant.ul[c]) or np.isfinite(plant.uu[c]):
                rows.append((e, plant.ul[c], plant.uu[c]))
    rows += grows
    choices = []
    for (_, lo, hi) in rows:
        ch = [0]
        if np.isfinite(hi):
            ch.append(1)
        if np.isfinite(lo):
            ch.append(-1)
        choices.append(ch)
    best = None
    for pattern in itertools.product(*choices):
        act = [(k, s) for k, s in enumerate(pattern) if s != 0]
        m = len(act)
        if m > n:
            continue
        Aw = np.array([rows[k][0] * (1.0 if s > 0 else -1.0) for k, s in act]).reshape(m, n)
        bw = np.array([rows[k][2] if s > 0 else -rows[k][1] for k, s in act])
        K = np.zeros((n + m, n + m))
        K[:n, :n] = H
        K[:n, n:] = Aw.T
        K[n:, :n] = Aw
        rhs = np.concatenate([-h, bw])
        try:
            if m and np.linalg.matrix_rank(Aw) < m:
                continue
            sol = np.linalg.solve(K, rhs)
        except np.linalg.LinAlgError:
            continue
        u, lam = sol[:n], sol[n:]
        if m and lam.min() < -tol:
            continue
        ok = True
        for (g, lo, hi) in rows:
            v = g @ u
            if (np.isfinite(hi) and v > hi + tol) or (np.isfinite(lo) and v < lo - tol):
                ok = False
                break
        if ok:
            best = (u, act)
            break
    return best


def lqr(plant, x0):
    """Finite-horizon discrete LQR (textbook backward Riccati, P_N = Qf):
    K_t = -(R + B'P B)^{-1} B'P A, P_t = Q + A'P(A + B K_t), u_t = K_t x_t."""
    A = plant.dense("A")
    B = np.asarray(plant.B)
    Q, Qf, R = plant.dense("Q"), plant.dense("Qf"), np.asarray(plant.R)
    P = Qf
    Ks = [None] * plant.N
    for t in range(plant.N - 1, -1, -1):
        K = -np.linalg.solve(R + B.T @ P @ B, B.T @ P @ A)
        Ks[t] = K
        P = Q + A.T @ P @ (A + B @ K)
    x = np.asarray(x0, dtype=np.float64)
    us = []
    for t in range(plant.N):
        u = Ks[t] @ x
        us.append(u)
        x = A @ x + B @ u
    return np.concatenate(us)


def scalar_closed_form(a, b, qf, r, xbar, xl, xu, ul, uu):
    """ns = nu = N = 1: minimise 1/2 qf x1^2 + 1/2 r u^2, x1 = a xbar + b u,
    xl <= x1 <= xu, ul <= u <= uu.  A strictly convex 1-D problem: the
    minimiser is the unconstrained one clipped to the feasible interval."""
    u_unc = -qf * a * b * xbar / (qf * b * b + r)
    lo_x, hi_x = (xl - a * xbar) / b, (xu - a * xbar) / b
    if b < 0:
        lo_x, hi_x = hi_x, lo_x
    lo, hi = max(ul, lo_x), min(uu, hi_x)
    assert lo <= hi
    return min(max(u_unc, lo), hi)
