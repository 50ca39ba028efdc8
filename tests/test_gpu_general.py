"""The general problem data of Eq. 1 (Section II) through lqmpc_setup_general:
cross term S, disturbance w, general rows gl <= E x_t + F u_t <= gu, and a
stabilising feedback K (u_t = K x_t + v_t), against the oracle, which
states the same problem directly (no lifting, no feedback).

Without K the lifted solver runs the oracle's method on the same problem, so
the FP64 path takes the oracle's iterates (iteration count, mu_k) and the
usual bars hold (FP64 1e-10, mixed 1e-6, relative).  With K the solver's
variable is v and its start differs (v = 0 instead of the box midpoint of
u), so only the optimum is compared, both run to 1e-11: the problems here
are not degenerate, and the optimum is unique (R > 0).
"""
import numpy as np
import pytest

import oracle
import pins
from paper_2209_13049_b300 import binding, build, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.load()


def rel(u, ref):
    return float(np.max(np.abs(u - ref)) / max(1.0, np.max(np.abs(ref))))


def heat1d_general(with_k=False):
    """1-D heat plant (ns = 60, nu = 4, N = 12) with a cross term, a
    disturbance, and three general rows: the mean temperature of each third
    of the rod plus one input each, bounded so that they bind (the input can
    always meet its row: the problem stays feasible)."""
    p = inputs.heat1d(60, 4, 12)
    rng = np.random.default_rng(5)
    p.S = 0.02 * rng.standard_normal((60, 4))          # [Q S; S' R] > 0: |S| << sqrt(1 * 0.1)
    p.w = 0.01 * rng.standard_normal((12, 60))
    E = np.zeros((3, 60))
    for r in range(3):
        E[r, 20 * r:20 * (r + 1)] = 1.0 / 20
    F = np.zeros((3, 4))
    F[0, 0], F[1, 1], F[2, 3] = 1.0, 1.0, -1.0
    p.E, p.F = E, F
    p.gl, p.gu = np.array([-0.1, -np.inf, -0.1]), np.array([0.1, 0.05, np.inf])
    if with_k:
        p.K = -0.5 * p.B.T                               # A + B K stays stable
    return p, inputs.x0_uniform(60, 9)


def random_general(seed, with_k=False):
    """Dense non-symmetric A, joint stage weight with cross term, disturbance,
    two general rows (nc = nu, F invertible: every row value reachable) with
    bounds cutting the unconstrained optimum; no box bounds."""
    rng = np.random.default_rng(seed)
    ns, nu, N = 6, 2, 9
    p = inputs.random_small(ns, nu, N, seed, xb=np.inf, ub=np.inf, dense_q=True)
    Mj = rng.standard_normal((ns + nu, ns + nu))
    W = Mj @ Mj.T / (ns + nu) + 0.3 * np.eye(ns + nu)
    p.Q, p.R, p.S = W[:ns, :ns], W[ns:, ns:], W[:ns, ns:].copy()
    p.w = 0.2 * rng.standard_normal((N, ns))
    p.E, p.F = rng.standard_normal((2, ns)), rng.standard_normal((2, nu)) + 2.0 * np.eye(nu)
    x0 = rng.uniform(-0.6, 0.6, ns)
    E, F = p.E, p.F
    p.E = None                                    # the unconstrained optimum first
    _, _, H, h, _ = pins.dense_qp_general(p, x0)
    u = (-np.linalg.solve(H, h)).reshape(N, nu)
    p.E = E
    xs, c = x0.copy(), []
    for t in range(N):
        c.append(E @ xs + F @ u[t])
        xs = p.dense("A") @ xs + p.B @ u[t] + p.w[t]
    c = np.array(c)
    p.gl = np.array([-np.inf, c[:, 1].min() + 0.3 * np.ptp(c[:, 1])])
    p.gu = np.array([c[:, 0].max() - 0.3 * np.ptp(c[:, 0]), np.inf])
    if with_k:
        p.K = 0.1 * np.random.default_rng(1000 + seed).standard_normal((nu, ns))
    return p, x0


CASES = [("heat1d", lambda k=False: heat1d_general(k)), ("random3", lambda k=False: random_general(3, k)),
         ("random8", lambda k=False: random_general(8, k))]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_fp64_general_takes_the_oracle_iterates(name, make):
    p, x0 = make()
    ref8 = oracle.ipm_solve(p, x0, tol=1e-8, want_trace=True)
    ref12 = oracle.ipm_solve(p, x0, tol=1e-11)
    assert ref8["status"] == 0 and ref12["status"] == 0
    s = binding.Solver(p, precision="fp64")
    u, st = s.solve(x0)
    assert st["status"] == 0
    assert st["iters"] == ref8["stats"]["iters"]
    np.testing.assert_allclose(s.get_trace()[:, 0], ref8["trace"][:, 0], rtol=1e-6)
    assert rel(u, ref8["u"]) <= 1e-8
    s.set_options(tol=1e-11)
    u12, _ = s.solve(x0)
    assert rel(u12, ref12["u"]) <= 1e-10
    # the general rows bind at the optimum (so their duals are exercised)
    nc = p.nc
    z = ref12["z"]
    SX = p.ns * p.N
    zg = z[2 * SX + 2 * p.n:]
    assert zg.size == 2 * nc * p.N and zg.max() > 1e-6


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_mixed_general_matches_oracle(name, make, precision):
    p, x0 = make()
    ref8 = oracle.ipm_solve(p, x0, tol=1e-8)
    u, st = binding.Solver(p, precision=precision).solve(x0)
    assert st["status"] == 0
    assert rel(u, ref8["u"]) <= 1e-6


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_feedback_k_reaches_the_oracle_optimum(name, make, precision):
    """u_t = K x_t + v_t: the solver runs in v with A + B K and returns u."""
    p, x0 = make(True)
    ref = oracle.ipm_solve(p, x0, tol=1e-11)     # the oracle ignores K: same problem in u
    assert ref["status"] == 0
    s = binding.Solver(p, precision=precision, tol=1e-11)
    u, st = s.solve(x0)
    assert st["status"] == 0
    assert rel(u, ref["u"]) <= (1e-8 if precision == "fp64" else 1e-6)
    # the input bounds hold on u (they are lifted rows with K)
    U = u.reshape(p.N, p.nu)
    assert np.all(U <= p.uu + 1e-9) and np.all(U >= p.ul - 1e-9)
    with pytest.raises(binding.LqmpcError) as e:
        s.solve_warm(x0, u)
    assert e.value.code == 9


def test_general_and_plain_contexts_in_one_batch():
    items = [heat1d_general(), random_general(3), random_general(8, True),
             (inputs.heat1d(40, 3, 10), inputs.x0_uniform(40, 1))]
    refs = [oracle.ipm_solve(p, x0, tol=1e-11)["u"] for p, x0 in items]
    for precision, bar in (("fp64", 1e-8), ("fp32", 1e-6)):
        solvers = [binding.Solver(p, precision=precision, tol=1e-11) for p, _ in items]
        us, stats, code = binding.solve_batch(solvers, [x for _, x in items])
        assert code == 0
        for k in range(len(items)):
            assert rel(us[k], refs[k]) <= bar, (precision, k)


def test_x0_is_read_for_the_plant_states_only():
    """x0 holds the plant's ns states; the lifted rows (general rows, and the
    inputs with K) start at zero and nothing past x0[ns-1] is read: an x0
    that is a view into a buffer with NaN after it solves like a plain one."""
    for with_k in (False, True):
        p, x0 = random_general(8, with_k)
        buf = np.full(p.ns + 64, np.nan)
        buf[:p.ns] = x0
        ref = binding.Solver(p, precision="fp64", tol=1e-10).solve(x0)[0]
        for precision in ("fp64", "fp32"):
            s = binding.Solver(p, precision=precision, tol=1e-10)
            u, st = s.solve(buf[:p.ns])
            assert st["status"] == 0
            assert rel(u, ref) <= (1e-12 if precision == "fp64" else 1e-6)
        solvers = [binding.Solver(p, precision="fp32", tol=1e-10) for _ in range(2)]
        us, stats, code = binding.solve_batch(solvers, [buf[:p.ns], x0])
        assert code == 0
        for k in range(2):
            assert rel(us[k], ref) <= 1e-6


def test_general_setup_rejects_bad_rows():
    p, _ = heat1d_general()
    p.gl = np.array([0.3, -np.inf, -0.3])        # gl > gu in row 0
    with pytest.raises(binding.LqmpcError) as e:
        binding.Solver(p)
    assert e.value.code == 1
    p, _ = heat1d_general()
    p.S = p.S.copy()
    p.S[3, 1] = np.nan
    with pytest.raises(binding.LqmpcError):
        binding.Solver(p)
