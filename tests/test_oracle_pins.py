"""Pins of the oracle against references other than itself (CPU only).

Each test would fail for a plausible mistake in the oracle: a dropped or
sign-flipped term, a transposed A, a wrong stage index, a wrong step rule.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import pins
from paper_2209_13049_b300 import inputs
from paper_2209_13049_b300.inputs import Plant


def _tiny(seed, ns=2, nu=1, N=3, xb=0.5, ub=0.4, dense_q=True):
    return inputs.random_small(ns, nu, N, seed, xb=xb, ub=ub, dense_q=dense_q)


# ---------------------------------------------------------------- IPM optimum


def _double_integrator(N=3, ub=0.5, r=0.1):
    A = np.array([[1.0, 0.5], [0.0, 1.0]])
    B = np.array([[0.125], [0.5]])
    return Plant(2, 1, N, A, B, np.eye(2), np.array([[r]]), np.eye(2),
                 -np.ones(2), np.ones(2), -ub * np.ones(1), ub * np.ones(1))


def _feasible_cases(make, draws, count):
    """(plant, x0, brute-force optimum, active rows) for the first `count`
    feasible draws; infeasible draws (no KKT point) are skipped."""
    out = []
    for p, x0 in draws:
        bf = pins.brute_force(p, x0)
        if bf is not None:
            out.append((p, x0, bf[0], bf[1]))
        if len(out) == count:
            break
    return out


def _di_draws():
    rng = np.random.default_rng(0)
    for _ in range(40):
        yield _double_integrator(), rng.uniform([0.3, 0.2], [0.95, 0.9])


def _random_draws():
    for seed in range(40):
        p = _tiny(seed)
        yield p, np.random.default_rng(100 + seed).uniform(-0.45, 0.45, size=p.ns)


def test_ipm_matches_brute_force_active_bounds():
    """Brute-force active-set enumeration gives the exact minimiser; these
    double-integrator cases have state and input bounds that bind."""
    cases = _feasible_cases(None, _di_draws(), 8)
    assert len(cases) == 8
    assert sum(len(c[3]) for c in cases) >= 10
    for p, x0, ubf, _ in cases:
        r = oracle.ipm_solve(p, x0, tol=1e-12)
        assert r["status"] == oracle.STATUS_OK
        np.testing.assert_allclose(r["u"], ubf, rtol=0, atol=1e-8)


def test_ipm_matches_brute_force_random_dense():
    """Random non-symmetric A, dense Q, Qf, R (a transposed A or a wrong Qf
    stage would change the optimum)."""
    cases = _feasible_cases(None, _random_draws(), 8)
    assert len(cases) == 8
    for p, x0, ubf, _ in cases:
        r = oracle.ipm_solve(p, x0, tol=1e-12)
        assert r["status"] == oracle.STATUS_OK
        np.testing.assert_allclose(r["u"], ubf, rtol=0, atol=1e-8)


def test_ipm_matches_brute_force_two_inputs():
    draws = ((inputs.random_small(2, 2, 2, 50 + s, xb=0.4, ub=0.3, dense_q=True),
              np.random.default_rng(s).uniform(-0.35, 0.35, size=2)) for s in range(20))
    cases = _feasible_cases(None, draws, 3)
    assert len(cases) == 3
    for p, x0, ubf, _ in cases:
        r = oracle.ipm_solve(p, x0, tol=1e-12)
        np.testing.assert_allclose(r["u"], ubf, rtol=0, atol=1e-8)


@pytest.mark.parametrize("seed", range(4))
def test_ipm_unbounded_equals_lqr(seed):
    """With every bound absent the QP is the finite-horizon LQR problem."""
    p = inputs.random_small(4, 2, 6, seed, dense_q=True)
    p.xl, p.xu = np.full(4, -np.inf), np.full(4, np.inf)
    p.ul, p.uu = np.full(2, -np.inf), np.full(2, np.inf)
    x0 = np.random.default_rng(seed).standard_normal(4)
    r = oracle.ipm_solve(p, x0, tol=1e-12)
    assert r["stats"]["m"] == 0
    np.testing.assert_allclose(r["u"], pins.lqr(p, x0), rtol=0, atol=1e-11)


def test_ipm_inactive_bounds_equal_lqr_heat1d():
    """1-D heat plant with loose finite bounds: the optimum is the LQR law."""
    p = inputs.heat1d(20, 3, 8, xb=50.0, ub=50.0)
    x0 = inputs.x0_uniform(20, 3)
    r = oracle.ipm_solve(p, x0, tol=1e-13)
    assert r["status"] == 0
    np.testing.assert_allclose(r["u"], pins.lqr(p, x0), rtol=0, atol=1e-9)


@pytest.mark.parametrize("case", [
    (0.9, 0.5, 2.0, 0.1, 1.0, -0.5, 0.5, -1.0, 1.0),    # state bound active
    (0.9, -0.5, 2.0, 0.1, 1.0, -0.8, 0.8, -0.3, 0.3),   # input bound active, b < 0
    (0.5, 1.0, 1.0, 1.0, 0.2, -1.0, 1.0, -1.0, 1.0),    # interior optimum
])
def test_ipm_scalar_closed_form(case):
    a, b, qf, r_, xbar, xl, xu, ul, uu = case
    p = Plant(1, 1, 1, np.array([[a]]), np.array([[b]]), np.array([[1.0]]), np.array([[r_]]),
              np.array([[qf]]), np.array([xl]), np.array([xu]), np.array([ul]), np.array([uu]))
    r = oracle.ipm_solve(p, np.array([xbar]), tol=1e-13)
    ref = pins.scalar_closed_form(a, b, qf, r_, xbar, xl, xu, ul, uu)
    assert abs(r["u"][0] - ref) < 1e-10


def test_ipm_kkt_invariants_heat1d():
    """Stationarity, feasibility, nonnegative duals and complementarity at the
    returned point of the ns=50 1-D configuration."""
    p, x0 = inputs.config_1d_small(0)
    r = oracle.ipm_solve(p, x0, tol=1e-10)
    k = oracle.kkt_check(p, x0, r["u"], r["z"])
    assert r["status"] == 0
    assert k["primal_violation"] <= 1e-12
    assert k["stationarity"] <= 1e-9
    assert k["dual_min"] >= 0.0
    assert k["complementarity"] <= 1e-8


def test_ipm_kkt_invariants_active_heat2d_small():
    """A small 2-D plant where the lower state bound binds."""
    p = inputs.heat2d(6, 4, 8)
    x0 = inputs.x0_gaussians(6, 1)
    r = oracle.ipm_solve(p, x0, tol=1e-11)
    k = oracle.kkt_check(p, x0, r["u"], r["z"])
    x = oracle.simulate(p, x0, r["u"])
    assert r["status"] == 0
    assert np.sum(x < 1e-7) > 0
    assert k["primal_violation"] <= 1e-12 and k["stationarity"] <= 1e-9
    assert k["complementarity"] <= 1e-9


def test_kkt_check_mean_complementarity_is_the_ipm_mu():
    """The checker's mean complementarity, from the bound distances of the
    simulated trajectory, equals the oracle's own final mu = s'z / m (its
    slack variables), up to the primal residual left at the stop."""
    for p, x0 in (inputs.config_1d_small(1), (inputs.heat2d(6, 4, 8), inputs.x0_gaussians(6, 1))):
        r = oracle.ipm_solve(p, x0, tol=1e-10)
        k = oracle.kkt_check(p, x0, r["u"], r["z"])
        assert r["status"] == 0
        np.testing.assert_allclose(k["complementarity_mean"], r["stats"]["mu"], rtol=1e-3)
        assert k["complementarity"] >= k["complementarity_mean"]


def test_ipm_trace_monotone_and_steps_valid():
    p, x0 = inputs.config_1d_small(2)
    r = oracle.ipm_solve(p, x0, want_trace=True)
    tr = r["trace"]
    assert np.all(tr[:-1, 5] > 0) and np.all(tr[:-1, 5] <= 1)
    assert np.all(tr[:-1, 3] > 0) and np.all(tr[:-1, 3] <= 1)
    assert np.all(np.diff(tr[:, 0]) < 0)          # mu decreases every iteration


def test_ipm_status_codes_match_abi_numbering():
    """The oracle's status numbers equal the C-ABI's (documented values)."""
    assert (oracle.STATUS_OK, oracle.STATUS_NOT_PD, oracle.STATUS_MAXITER, oracle.STATUS_NAN) == (0, 3, 4, 6)


def test_ipm_maxiter_on_infeasible():
    """x0 far outside what the inputs can correct: the QP is infeasible and the
    iteration must end with MAXITER or NAN, never a false OK."""
    p = _tiny(0, xb=0.1, ub=0.01)
    r = oracle.ipm_solve(p, np.array([5.0, -5.0]), max_iter=40)
    assert r["status"] in (oracle.STATUS_MAXITER, oracle.STATUS_NAN)


# ------------------------------------------------------ condensed operators


def test_gstack_is_toeplitz_expansion_of_impulse_response():
    """Gamma's block (r, t) equals A^{r-t} B (the structure the paper notes in
    its conclusions: all data of J sits in its first nu columns)."""
    p = inputs.heat2d(5, 3, 6)
    G = oracle.gstack(p)
    Gam, _, _, _ = oracle.condensed(p, np.zeros(p.ns))
    for r in range(p.N):
        for t in range(p.N):
            blk = Gam[r * p.ns:(r + 1) * p.ns, t * p.nu:(t + 1) * p.nu]
            if t <= r:
                np.testing.assert_allclose(blk, G[r - t], rtol=1e-14, atol=1e-300)
            else:
                assert not blk.any()


def test_condensed_reproduces_dynamics():
    """Phi xbar + Gamma u equals a direct simulation of the dynamics."""
    p = inputs.random_small(3, 2, 5, 7)
    x0 = np.array([0.3, -0.2, 0.1])
    u = np.random.default_rng(1).standard_normal(p.n)
    Gam, y, _, _ = oracle.condensed(p, x0)
    np.testing.assert_allclose(y + Gam @ u, oracle.simulate(p, x0, u).reshape(-1), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("dense_q", [False, True])
def test_condensed_objective_identity(dense_q):
    """1/2 u'Hu + h'u + c equals the sparse objective of Eq. 1 for any u;
    checked at several u so H and h are both pinned (with the constant c
    from u = 0)."""
    p = inputs.random_small(3, 2, 5, 11, dense_q=dense_q)
    x0 = np.array([0.4, 0.1, -0.3])
    Gam, y, H, h = oracle.condensed(p, x0)
    Q, Qf, R = p.dense("Q"), p.dense("Qf"), np.asarray(p.R)

    def sparse_obj(u):
        x = oracle.simulate(p, x0, u)
        uu = u.reshape(p.N, p.nu)
        v = sum(0.5 * x[t] @ (Qf if t == p.N - 1 else Q) @ x[t] for t in range(p.N))
        return v + sum(0.5 * uu[t] @ R @ uu[t] for t in range(p.N))

    c = sparse_obj(np.zeros(p.n))
    rng = np.random.default_rng(2)
    for _ in range(5):
        u = rng.standard_normal(p.n)
        assert abs(0.5 * u @ H @ u + h @ u + c - sparse_obj(u)) < 1e-11 * (1 + abs(c))


def test_condensed_matches_independent_dense_build():
    p = inputs.random_small(3, 2, 4, 3, dense_q=True)
    x0 = np.array([0.2, 0.5, -0.1])
    G1, y1, H1, h1 = oracle.condensed(p, x0)
    G2, y2, H2, h2 = pins.dense_qp(p, x0)
    np.testing.assert_allclose(G1, G2, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(H1, H2, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(h1, h2, rtol=1e-12, atol=1e-14)


def test_kkt_matrix_matches_matrix_free_product():
    """M v = H v + Gamma'(Sigma_x (Gamma v)) + Sigma_u v, with Gamma v by
    simulation and Gamma' w by the adjoint recursion (no explicit Gamma)."""
    p = inputs.heat2d(4, 3, 5)
    rng = np.random.default_rng(4)
    sigx = rng.uniform(0, 10, p.ns * p.N)
    sigu = rng.uniform(0, 10, p.n)
    M = oracle.kkt_matrix(p, sigx, sigu)
    Gam, _, H, _ = oracle.condensed(p, np.zeros(p.ns))
    for _ in range(3):
        v = rng.standard_normal(p.n)
        Gv = oracle.simulate(p, np.zeros(p.ns), v).reshape(-1)
        mv = H @ v + oracle.adjoint_gradient(p, None, sigx * Gv) + sigu * v
        np.testing.assert_allclose(M @ v, mv, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(M, M.T, rtol=0, atol=1e-12)
    np.linalg.cholesky(M)          # positive definite (Eq. 7)


def test_kkt_entries_match_dense_definition():
    p = inputs.heat1d(12, 2, 5)
    rng = np.random.default_rng(5)
    sigx = rng.uniform(0, 3, p.ns * p.N)
    sigu = rng.uniform(0, 3, p.n)
    Gam, _, H, _ = oracle.condensed(p, np.zeros(p.ns))
    M = oracle.kkt_matrix(p, sigx, sigu, Gam, H)
    pairs = [(j, k) for j in range(p.n) for k in range(p.n)]
    e = oracle.kkt_entries(p, sigx, sigu, pairs, H=H)
    np.testing.assert_allclose(e, M.reshape(-1), rtol=1e-13, atol=1e-14)
    hq = oracle.hessian_entries(p, pairs)
    np.testing.assert_allclose(hq, H.reshape(-1), rtol=1e-13, atol=1e-15)


def test_dimensions_of_figure1_instance():
    """Fig. 1's instance (nx=5, nu=3, T=5): the condensed system is n_u T = 15
    square, J has (n_x + n_u) T two-sided rows (conclusions), and the dense QP
    has 2 T (n_x + n_u) one-sided inequalities (Section II)."""
    p = inputs.random_small(5, 3, 5, 0)
    Gam, y, H, h = oracle.condensed(p, np.zeros(5))
    M = oracle.kkt_matrix(p, np.ones(25), np.ones(15), Gam, H)
    assert M.shape == (15, 15)
    assert Gam.shape[0] + p.n == (5 + 3) * 5
    r = oracle.ipm_solve(p, np.zeros(5))
    assert r["stats"]["m"] == 2 * 5 * (5 + 3)


# ----------------------------------------- planted mistakes are caught (CPU)


def test_planted_transpose_is_caught_by_objective_identity():
    """Plant a transposed A in the oracle's condensing step: the objective
    identity against the true dynamics must fail."""
    p = inputs.random_small(3, 2, 4, 9)
    x0 = np.array([0.4, 0.1, -0.3])
    wrong = inputs.random_small(3, 2, 4, 9)
    wrong.A = p.A.T.copy()
    _, _, H, h = oracle.condensed(wrong, x0)
    Q, R = p.dense("Q"), np.asarray(p.R)
    u = np.random.default_rng(0).standard_normal(p.n)
    x = oracle.simulate(p, x0, u)
    true = sum(0.5 * x[t] @ Q @ x[t] for t in range(p.N)) + 0.5 * u @ np.kron(np.eye(p.N), R) @ u
    x00 = oracle.simulate(p, x0, np.zeros(p.n))
    c = sum(0.5 * x00[t] @ Q @ x00[t] for t in range(p.N))
    assert abs(0.5 * u @ H @ u + h @ u + c - true) > 1e-6


def test_planted_sign_error_is_caught_by_brute_force():
    """Flip the sign of A's off-diagonal in the oracle's input: its optimum no
    longer matches the brute-force optimum of the true problem."""
    p, x0, ubf, _ = _feasible_cases(None, _di_draws(), 1)[0]
    bad = _double_integrator()
    bad.A = np.array([[1.0, -0.5], [0.0, 1.0]])
    r = oracle.ipm_solve(bad, x0, tol=1e-12)
    assert np.max(np.abs(r["u"] - ubf)) > 1e-4


def test_cube_plant_follows_table_1_and_the_oracle_meets_kkt():
    """The 3-D cube generator against Table I's constants (a = dt k /
    (rho cp dw^2), six face inputs, q = 10 dw^2, r = dw^2 / 10) and the fixed
    point of the deviation form (the uniform set-point state with every face
    at the set point stays put); the oracle's solution of a small cube meets
    the KKT conditions of Eq. 5."""
    from paper_2209_13049_b300 import inputs
    p = inputs.heat3d_cube(3, 12)
    a = 0.1 * 400.0 / (8960.0 * 386.0 * 0.02 ** 2)
    assert abs(p.meta["alpha"] - a) <= 1e-15
    A = p.dense("A")
    assert np.allclose(np.diag(A), 1.0 - 6 * a)
    centre = (1 * 3 + 1) * 3 + 1                     # the one node with no face neighbour
    assert np.all(p.B[centre] == 0.0)
    assert np.allclose(p.B.sum(axis=0), 9 * a)      # nine nodes touch each face
    assert np.allclose(A.sum(axis=1) + p.B.sum(axis=1), 1.0)
    assert np.allclose(p.dense("Q"), 10 * 0.02 ** 2 * np.eye(27))
    assert np.allclose(p.R, 0.1 * 0.02 ** 2 * np.eye(6))
    assert np.allclose(p.xl, -200.0) and np.allclose(p.uu, 100.0)
    x0 = inputs.x0_cube(3)
    assert np.allclose(x0, -100.0)
    r = oracle.ipm_solve(p, x0, tol=1e-11)
    assert r["status"] == 0
    k = oracle.kkt_check(p, x0, r["u"], r["z"])
    assert k["primal_violation"] <= 1e-9 and k["dual_min"] >= 0.0
    scale = 1.0 + float(np.max(np.abs(p.R @ r["u"].reshape(-1, 6).T)))
    assert k["stationarity"] <= 1e-9 * scale and k["complementarity"] <= 1e-8


# ------------------------------------------------- general data of Eq. 1


def _general(seed, ns=2, nu=1, N=3, nc=2, xb=np.inf, ub=0.6, cross=True, dist=True, cons=True):
    """Random plant with the general data of Eq. 1: a cross term S with the
    joint stage weight [Q S; S' R] positive definite, a disturbance w, and nc
    general rows E x_t + F u_t."""
    rng = np.random.default_rng(seed)
    p = inputs.random_small(ns, nu, N, seed, xb=1.0, ub=ub, dense_q=True)
    Mj = rng.standard_normal((ns + nu, ns + nu))
    W = Mj @ Mj.T / (ns + nu) + 0.3 * np.eye(ns + nu)
    p.Q, p.R = W[:ns, :ns], W[ns:, ns:]
    if cross:
        p.S = W[:ns, ns:].copy()
    if dist:
        p.w = 0.3 * rng.standard_normal((N, ns))
    if cons:
        p.E = rng.standard_normal((nc, ns))
        p.F = rng.standard_normal((nc, nu))
        p.gl = -rng.uniform(0.2, 0.6, nc)
        p.gu = rng.uniform(0.2, 0.6, nc)
    p.xl, p.xu = np.full(ns, -xb), np.full(ns, xb)
    return p


def test_general_data_unconstrained_equals_dense_minimiser():
    """No finite bound or row: the oracle's optimum with S and w equals
    -H^-1 h of the dense QP written out independently (a dropped cross term,
    a transposed S or a disturbance at the wrong stage changes it)."""
    for seed in range(4):
        p = _general(seed, ns=3, nu=2, N=5, ub=np.inf, cons=False)
        x0 = np.random.default_rng(seed).uniform(-1, 1, 3)
        _, _, H, h, _ = pins.dense_qp_general(p, x0)
        r = oracle.ipm_solve(p, x0, tol=1e-12)
        assert r["status"] == 0 and r["stats"]["m"] == 0
        np.testing.assert_allclose(r["u"], -np.linalg.solve(H, h), rtol=0, atol=1e-10)


def test_general_constraints_match_brute_force():
    """General rows gl <= E x_t + F u_t <= gu (t = 0..N-1, the first on the
    fixed x_0) with binding rows, cross term and disturbance, against the
    brute-force active-set optimum."""
    found, active = 0, 0
    for seed in range(30):
        p = _general(seed)
        x0 = np.random.default_rng(200 + seed).uniform(-0.5, 0.5, 2)
        bf = pins.brute_force(p, x0)
        if bf is None:
            continue
        r = oracle.ipm_solve(p, x0, tol=1e-12)
        assert r["status"] == 0, seed
        np.testing.assert_allclose(r["u"], bf[0], rtol=0, atol=1e-8)
        found += 1
        active += len(bf[1])
        if found == 6:
            break
    assert found == 6 and active >= 6


def test_cross_term_and_disturbance_with_state_bounds_match_brute_force():
    found = 0
    for seed in range(30):
        p = _general(50 + seed, xb=0.5, cons=False)
        x0 = np.random.default_rng(300 + seed).uniform(-0.4, 0.4, 2)
        bf = pins.brute_force(p, x0)
        if bf is None or not bf[1]:
            continue
        r = oracle.ipm_solve(p, x0, tol=1e-12)
        assert r["status"] == 0
        np.testing.assert_allclose(r["u"], bf[0], rtol=0, atol=1e-8)
        found += 1
        if found == 4:
            break
    assert found == 4


def test_general_rows_kkt_and_duals():
    """At the oracle's optimum the general rows hold, their duals are
    nonnegative and complementary to the row slacks, and rows that cut the
    unconstrained optimum bind (nc = nu with F invertible: every row value is
    reachable, so the problem is feasible)."""
    p = _general(7, ns=4, nu=2, N=6, nc=2, ub=np.inf)
    x0 = np.random.default_rng(1).uniform(-0.5, 0.5, 4)
    _, _, H, h, _ = pins.dense_qp_general(p, x0)
    u0 = -np.linalg.solve(H, h).reshape(p.N, p.nu)
    xs, c0 = x0.copy(), []
    for t in range(p.N):
        c0.append(p.E @ xs + p.F @ u0[t])
        xs = p.dense("A") @ xs + p.B @ u0[t] + p.w[t]
    c0 = np.array(c0)
    p.gu = c0.max(axis=0) - 0.3 * np.ptp(c0, axis=0)
    p.gl = np.full(p.nc, -np.inf)
    r = oracle.ipm_solve(p, x0, tol=1e-12)
    assert r["status"] == 0
    n, SX, nc = p.n, p.ns * p.N, p.nc
    z5 = r["z"][2 * SX + 2 * n:2 * SX + 2 * n + nc * p.N].reshape(p.N, nc)
    z6 = r["z"][2 * SX + 2 * n + nc * p.N:].reshape(p.N, nc)
    xs = np.vstack([x0, r["x"][:-1]])
    u = r["u"].reshape(p.N, p.nu)
    c = xs @ p.E.T + u @ p.F.T
    assert np.all(c <= p.gu + 1e-9)
    assert z5.min() >= 0 and np.all(z6 == 0.0)
    assert np.max(np.abs(z5 * (p.gu - c))) <= 1e-9
    assert z5.max() > 1e-3                       # rows bind
