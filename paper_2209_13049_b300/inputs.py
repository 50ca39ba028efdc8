"""Seeded synthetic inputs: plants, bounds and initial states.

This module holds problem data only and none of the solver's arithmetic, so
that the CUDA path, the oracle tests and the benchmark draw identical inputs
from it without sharing any code of the method.

The plants are explicit-Euler finite-difference heat equations, the class of
PDE-constrained control problem the paper solves (Section V-A, Eq. 8, where the
boundary temperatures are the inputs and only interior temperatures are
states).  Sizes follow the paper's problem statement (Eq. 1): ns states,
nu inputs, horizon N.

Recipe (stated once here, repeated in the design notes):

* ``heat1d(ns, nu)``: A = I + a*L1 with L1 the 1-D Dirichlet Laplacian
  stencil [1, -2, 1] and a = 0.1; actuator k sits at state index
  (2k+1)*ns // (2*nu) with gain B[i_k, k] = a.
* ``heat2d(g, nu)``: ns = g*g interior nodes, A = I + a*L2 (5-point stencil,
  a = 0.1).  The ring of 4g ghost (boundary) nodes is walked counter-clockwise
  (bottom, right, top, left) and cut into nu contiguous arcs of equal length;
  arc k has temperature u_k and B[i, k] = a * (number of ghost neighbours of
  node i in arc k).
* ``x0_uniform``: x0 ~ U(-0.8, 0.8) (1-D plants).
* ``x0_gaussians``: a sum of 8 Gaussian bumps, centres ~ U[0,1]^2,
  widths ~ U[0.05, 0.2], amplitudes ~ U[0,1], rescaled so max(x0) = 0.9.
* Q = I, R = 0.1*I, Qf = Q; 1-D bounds x in [-1,1], u in [-2,2];
  2-D bounds x in [0,1], u in [-5,5].
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np
import scipy.sparse as sp

ALPHA = 0.1


@dataclass
class Plant:
    """Data of one box-constrained LQ-MPC problem (Eq. 1 with S=0, E=F=0, w=0).

    A, Q, Qf are ns x ns (scipy CSR or dense ndarray), B is ns x nu, R is
    nu x nu.  Bounds are per-state / per-input vectors; +-inf means absent.
    """

    ns: int
    nu: int
    N: int
    A: object
    B: np.ndarray
    Q: object
    R: np.ndarray
    Qf: object
    xl: np.ndarray
    xu: np.ndarray
    ul: np.ndarray
    uu: np.ndarray
    kind: str = "custom"
    meta: dict = field(default_factory=dict)
    # general data of Eq. 1 (None: absent): cross term S (ns x nu), disturbance
    # w (N x ns), general constraints gl <= E x_t + F u_t <= gu (E: nc x ns,
    # F: nc x nu), and a stabilising feedback K (nu x ns) for the elimination
    # u_t = K x_t + v_t (Section II; it changes the arithmetic, not u*)
    S: Optional[np.ndarray] = None
    w: Optional[np.ndarray] = None
    E: Optional[np.ndarray] = None
    F: Optional[np.ndarray] = None
    gl: Optional[np.ndarray] = None
    gu: Optional[np.ndarray] = None
    K: Optional[np.ndarray] = None

    @property
    def n(self) -> int:
        return self.nu * self.N

    @property
    def nc(self) -> int:
        return 0 if self.E is None else int(np.asarray(self.E).shape[0])

    @property
    def general(self) -> bool:
        return any(v is not None for v in (self.S, self.w, self.E, self.K))

    def dense(self, name: str) -> np.ndarray:
        m = getattr(self, name)
        return m.toarray() if sp.issparse(m) else np.asarray(m, dtype=np.float64)

    def csr(self, name: str) -> sp.csr_matrix:
        m = getattr(self, name)
        return sp.csr_matrix(m, dtype=np.float64)


def _laplacian_1d(ns: int) -> sp.csr_matrix:
    main = -2.0 * np.ones(ns)
    off = np.ones(ns - 1)
    return sp.diags([off, main, off], [-1, 0, 1], format="csr")


def heat1d(ns: int, nu: int, N: int, *, alpha: float = ALPHA, xb: float = 1.0,
           ub: float = 2.0, r: float = 0.1) -> Plant:
    """1-D heat plant with nu point actuators (x in [-xb,xb], u in [-ub,ub])."""
    A = (sp.identity(ns, format="csr") + alpha * _laplacian_1d(ns)).tocsr()
    B = np.zeros((ns, nu))
    for k in range(nu):
        B[(2 * k + 1) * ns // (2 * nu), k] = alpha
    Q = sp.identity(ns, format="csr")
    return Plant(ns, nu, N, A, B, Q, r * np.eye(nu), Q.copy(),
                 -xb * np.ones(ns), xb * np.ones(ns), -ub * np.ones(nu), ub * np.ones(nu),
                 kind="heat1d", meta={"alpha": alpha})


def ghost_ring(g: int):
    """Ghost nodes of a g x g grid in counter-clockwise order.

    Returns a list of (interior neighbour index) for each of the 4g ghost nodes;
    grid node (i, j) (row i, column j) has state index i*g + j.
    """
    ring = []
    for j in range(g):                 # bottom side, row -1
        ring.append(0 * g + j)
    for i in range(g):                 # right side, column g
        ring.append(i * g + (g - 1))
    for j in range(g - 1, -1, -1):     # top side, row g
        ring.append((g - 1) * g + j)
    for i in range(g - 1, -1, -1):     # left side, column -1
        ring.append(i * g + 0)
    return ring


def heat2d(g: int, nu: int, N: int, *, alpha: float = ALPHA, r: float = 0.1) -> Plant:
    """2-D heat plant on a g x g interior grid with nu boundary-arc inputs."""
    ns = g * g
    L1 = _laplacian_1d(g)
    I = sp.identity(g, format="csr")
    L2 = (sp.kron(I, L1) + sp.kron(L1, I)).tocsr()
    A = (sp.identity(ns, format="csr") + alpha * L2).tocsr()
    B = np.zeros((ns, nu))
    ring = ghost_ring(g)
    P = len(ring)
    for p, node in enumerate(ring):
        k = (p * nu) // P
        B[node, k] += alpha
    Q = sp.identity(ns, format="csr")
    return Plant(ns, nu, N, A, B, Q, r * np.eye(nu), Q.copy(),
                 np.zeros(ns), np.ones(ns), -5.0 * np.ones(nu), 5.0 * np.ones(nu),
                 kind="heat2d", meta={"alpha": alpha, "g": g})


# Table I of the paper (3-D copper cube): time step, mesh size, density,
# specific heat, conductivity, weights and bounds
CUBE_DT, CUBE_DW = 0.1, 0.02
CUBE_RHO, CUBE_CP, CUBE_K = 8960.0, 386.0, 400.0
CUBE_XL, CUBE_XU, CUBE_UL, CUBE_UU, CUBE_XHAT = 200.0, 550.0, 300.0, 500.0, 300.0
CUBE_SETPOINT = 400.0


def heat3d_cube(g: int, T: int, *, setpoint: float = CUBE_SETPOINT) -> Plant:
    """The paper's 3-D temperature control problem (Section V-A, Eq. 8,
    Table I) on a g x g x g interior grid with horizon T.

    Explicit Euler in time and the 7-point finite-difference Laplacian in
    space give A = I + a*L3 with a = dt*k/(rho*cp*dw^2); the six faces are
    Dirichlet boundaries whose temperatures are the nu = 6 inputs (the
    boundary is not a state), so an interior node next to face f gets
    B[node, f] = a.  The set point d of Eq. 8 is not given in the paper; it is
    the constant `setpoint` (K), and the problem is written in deviations
    from it (x - d, u - d), the form of Eq. 1, which has no linear cost terms:
    the uniform state at d with every face at d is a fixed point of the
    discretised dynamics (each row of [A B] sums to one), Q = q*I and
    R = r*I with q = 10 dw^2 and r = dw^2/10 weigh the deviations, and the
    bounds of Table I move by -d.  Node (i, j, l) is state (i*g + j)*g + l;
    faces are i = 0, i = g-1, j = 0, j = g-1, l = 0, l = g-1 in that order.
    """
    ns = g ** 3
    a = CUBE_DT * CUBE_K / (CUBE_RHO * CUBE_CP * CUBE_DW ** 2)
    L1 = _laplacian_1d(g)
    I = sp.identity(g, format="csr")
    L3 = (sp.kron(sp.kron(I, I), L1) + sp.kron(sp.kron(I, L1), I) + sp.kron(sp.kron(L1, I), I)).tocsr()
    A = (sp.identity(ns, format="csr") + a * L3).tocsr()
    B = np.zeros((ns, 6))
    idx = np.arange(ns)
    i, j, l = idx // (g * g), (idx // g) % g, idx % g
    for f, on in enumerate((i == 0, i == g - 1, j == 0, j == g - 1, l == 0, l == g - 1)):
        B[on, f] += a
    q, r = 10.0 * CUBE_DW ** 2, 0.1 * CUBE_DW ** 2
    Q = q * sp.identity(ns, format="csr")
    d = setpoint
    return Plant(ns, 6, T, A, B, Q, r * np.eye(6), Q.copy(),
                 (CUBE_XL - d) * np.ones(ns), (CUBE_XU - d) * np.ones(ns),
                 (CUBE_UL - d) * np.ones(6), (CUBE_UU - d) * np.ones(6),
                 kind="heat3d_cube", meta={"alpha": a, "g": g, "setpoint": d})


def x0_cube(g: int, setpoint: float = CUBE_SETPOINT) -> np.ndarray:
    """The cube's initial temperature (Table I: 300 K everywhere) as a
    deviation from the set point."""
    return (CUBE_XHAT - setpoint) * np.ones(g ** 3)


def x0_uniform(ns: int, seed: int, lo: float = -0.8, hi: float = 0.8) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=ns)


def x0_gaussians(g: int, seed: int, n_bumps: int = 8, peak: float = 0.9) -> np.ndarray:
    """Smooth nonnegative field on the g x g grid, max value `peak`."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.0, 1.0, size=(n_bumps, 2))
    w = rng.uniform(0.05, 0.2, size=n_bumps)
    a = rng.uniform(0.0, 1.0, size=n_bumps)
    t = (np.arange(g) + 0.5) / g
    yy, xx = np.meshgrid(t, t, indexing="ij")       # row i ~ y, column j ~ x
    f = np.zeros((g, g))
    for k in range(n_bumps):
        f += a[k] * np.exp(-((xx - c[k, 0]) ** 2 + (yy - c[k, 1]) ** 2) / (2.0 * w[k] ** 2))
    f *= peak / f.max()
    return f.reshape(-1).copy()


def random_small(ns: int, nu: int, N: int, seed: int, *, xb: float = 1.0, ub: float = 1.0,
                 dense_q: bool = False, stable: float = 0.9) -> Plant:
    """Random dense plant for tiny oracle pins (non-symmetric A, dense B)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((ns, ns))
    rad = max(abs(np.linalg.eigvals(A)))
    A *= stable / rad
    B = rng.standard_normal((ns, nu))
    if dense_q:
        F = rng.standard_normal((ns, ns))
        Q = F @ F.T / ns + 0.5 * np.eye(ns)
        F = rng.standard_normal((ns, ns))
        Qf = F @ F.T / ns + 1.0 * np.eye(ns)
        F = rng.standard_normal((nu, nu))
        R = F @ F.T / nu + 0.2 * np.eye(nu)
    else:
        Q = np.eye(ns)
        Qf = np.eye(ns)
        R = 0.1 * np.eye(nu)
    return Plant(ns, nu, N, A, B, Q, R, Qf,
                 -xb * np.ones(ns), xb * np.ones(ns), -ub * np.ones(nu), ub * np.ones(nu),
                 kind="random")


# ---------------------------------------------------------------------------
# Named workloads (sizes of the five benchmark configurations)
# ---------------------------------------------------------------------------

def config_1d_small(seed: int = 0):
    """ns=50 1-D plant, nu=5, N=10; x0 ~ U(-0.8,0.8) from `seed`."""
    p = heat1d(50, 5, 10)
    return p, x0_uniform(50, seed)


def config_2d_32(seed: int = 0, N: int = 50):
    """32x32 2-D plant (ns=1024), nu=10, N=50; x0 = 8-Gaussian field."""
    p = heat2d(32, 10, N)
    return p, x0_gaussians(32, seed)


def config_2d_100(seed: int = 0, N: int = 50):
    """100x100 2-D plant (ns=10000), nu=20, N=50; x0 = 8-Gaussian field."""
    p = heat2d(100, 20, N)
    return p, x0_gaussians(100, seed)


def batch_instances(count: int = 256, master_seed: int = 0):
    """Uneven batch: coin-flip 1-D (ns~U{200..2000}) or 2-D (g~U{15..44}) plants,
    nu~U{2..16}, N~U{10..50}; bounds and x0 as in the 1-D / 2-D recipes."""
    rng = np.random.default_rng(master_seed)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    out = []
    for s in seeds:
        r = np.random.default_rng(int(s))
        nu = int(r.integers(2, 17))
        N = int(r.integers(10, 51))
        if r.integers(0, 2) == 0:
            ns = int(r.integers(200, 2001))
            p = heat1d(ns, nu, N)
            x0 = x0_uniform(ns, int(s))
        else:
            g = int(r.integers(15, 45))
            p = heat2d(g, nu, N)
            x0 = x0_gaussians(g, int(s))
        out.append((p, x0))
    return out
