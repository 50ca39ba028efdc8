"""Parity at the full sizes of the benchmark workloads, in the launch
configuration bench.py times, against stored oracle solutions
(tests/golden/make_golden.py, which calls only the oracle):

* the 100 x 100 heat plant (ns = 10000, nu = 20, N = 50; M is 1000 x 1000,
  factored by the queued dataflow Cholesky in the FP32 tier and the
  cooperative FP64 Cholesky in the FP64 tier);
* the uneven 256-instance batch, eight instances sampled;
* the learned warm start on the 32 x 32 plant with the 1024-512-512-500
  network, on held-out initial states.

Bars, as for the smaller cases: the FP64 path takes the oracle's iterates
(same iteration count, mu_k within 1e-6 relative; condensing is an exact
elimination) and is within 1e-10 of the oracle's u* when both run to 1e-11;
mixed paths are within 1e-6.  At the metric's 1e-8 stop the degenerate
optimum (zero multipliers at active bounds, u converging like sqrt(mu)) lets
two correct solvers stop ~1e-5 apart, so stop-point comparisons of paths
that do not follow the oracle's iterates exactly use the matched-tolerance
bar only where the iterates match.  Relative error is
||u - u*||_inf / max(1, ||u*||_inf).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2209_13049_b300 import binding, build, inputs

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.load()


def rel(u, ref):
    return float(np.max(np.abs(u - ref)) / max(1.0, np.max(np.abs(ref))))


@pytest.fixture(scope="module")
def c3():
    g = np.load(os.path.join(GOLD, "heat2d_g100_nu20_N50.npz"))
    p, x0 = inputs.config_2d_100(0)
    np.testing.assert_array_equal(x0, g["heat2d_100_s0_x0"])
    return p, x0, g


def test_c3_fp64_takes_the_oracle_iterates(c3):
    p, x0, g = c3
    s = binding.Solver(p, precision="fp64")
    u, st = s.solve(x0)
    tr_ref = g["heat2d_100_s0_trace8"]
    assert st["status"] == 0
    assert st["iters"] == len(tr_ref) - 1
    tr = s.get_trace()
    np.testing.assert_allclose(tr[:, 0], tr_ref[:, 0], rtol=1e-6)
    assert rel(u, g["heat2d_100_s0_u8"]) <= 1e-8
    s.set_options(tol=1e-11)
    u12, st12 = s.solve(x0)
    assert st12["status"] == 0
    assert rel(u12, g["heat2d_100_s0_u12"]) <= 1e-10


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_c3_mixed_matches_oracle(c3, precision):
    """The FP32 tier (the metric's path: split-TF32 formation, queued
    dataflow FP32 Cholesky for n = 1000, two-level tier) and the BF16 tier."""
    p, x0, g = c3
    s = binding.Solver(p, precision=precision)
    u, st = s.solve(x0)
    assert st["status"] == 0
    assert rel(u, g["heat2d_100_s0_u8"]) <= 1e-6
    s.set_options(tol=1e-11)
    u12, st12 = s.solve(x0)
    assert st12["status"] == 0
    if precision == "fp32":
        # follows the oracle's iterates to the same stop
        assert rel(u12, g["heat2d_100_s0_u12"]) <= 1e-6
    else:
        # The BF16 tier's inexact Newton steps leave the dual residual a
        # little above the oracle's near the end, so it stops two iterations
        # later at a smaller mu.  This optimum is degenerate (state bounds
        # active with vanishing multipliers): u converges like sqrt(mu), and
        # the oracle's own 1e-11 stop lies ~2.4e-6 from its 1e-12 stop.  Two
        # valid stops at tol 1e-11 are compared within sqrt(tol), and the
        # result must satisfy the optimality conditions on its own.
        assert rel(u12, g["heat2d_100_s0_u12"]) <= np.sqrt(1e-11)
        k = oracle.kkt_check(p, x0, u12, s.get_duals())
        assert k["primal_violation"] <= 1e-9
        assert k["dual_min"] >= 0.0
        assert k["stationarity"] <= 1e-8
        assert k["complementarity"] <= 1e-8


def test_c3_kkt_conditions_with_the_oracle_checker(c3):
    """Independent of the stored solution: primal feasibility, dual sign,
    stationarity and complementarity of the FP32 tier's result (Eq. 5)."""
    p, x0, _ = c3
    s = binding.Solver(p, precision="fp32", tol=1e-10)
    u, st = s.solve(x0)
    assert st["status"] == 0
    k = oracle.kkt_check(p, x0, u, s.get_duals())
    assert k["primal_violation"] <= 1e-9
    assert k["dual_min"] >= 0.0
    assert k["stationarity"] <= 1e-8
    assert k["complementarity"] <= 1e-8


@pytest.fixture(scope="module")
def batch256():
    g = np.load(os.path.join(GOLD, "batch256_sample.npz"))
    inst = inputs.batch_instances(256, 0)
    sample = [int(k) for k in g["sample"]]
    for k in sample:
        np.testing.assert_array_equal(inst[k][1], g[f"i{k}_x0"])
    return inst, sample, g


def test_batch256_fp32_matches_oracle_on_sampled_instances(batch256):
    """The whole uneven 256-instance batch in the FP32 tier, autotuned, as
    bench.py runs it; the sampled instances against the oracle at the same
    1e-8 stop, and at 1e-11 within the degenerate band plus the optimality
    conditions."""
    inst, sample, g = batch256
    solvers = [binding.Solver(p, precision="fp32") for p, _ in inst]
    x0s = [x for _, x in inst]
    binding.autotune(solvers)
    us, stats, code = binding.solve_batch(solvers, x0s)
    assert code == 0
    assert all(st["status"] == 0 for st in stats)
    for k in sample:
        assert rel(us[k], g[f"i{k}_u8"]) <= 1e-6, k
    for s in solvers:
        s.set_options(tol=1e-11)
    us12, stats12, code = binding.solve_batch(solvers, x0s, check=False)
    for k in sample:
        assert stats12[k]["status"] == 0
        # At 1e-11 the batch's instances need not follow the oracle's iterates
        # (rounding in the batched kernels can change where a refinement
        # escalates), and on degenerate instances two valid stops differ by
        # O(sqrt(tol)): instance 0 (20 x 20 plate) converges, in every tier
        # pushed further, to a point 4.4e-6 from the oracle's own 1e-11
        # stop.  So the stop is compared within 3 sqrt(tol), and the result
        # must satisfy the optimality conditions on its own: the stop test
        # bounds the mean complementarity product (mu <= tol), one product
        # can be up to m times that.
        assert rel(us12[k], g[f"i{k}_u12"]) <= 3.0 * np.sqrt(1e-11), k
        p, x0 = inst[k]
        kc = oracle.kkt_check(p, x0, us12[k], solvers[k].get_duals())
        assert kc["primal_violation"] <= 1e-9, k
        assert kc["dual_min"] >= 0.0, k
        assert kc["stationarity"] <= 1e-8, k
        assert kc["complementarity_mean"] <= 1.01e-11, k


def test_batch256_sampled_instances_fp64_single_solves(batch256):
    """The baseline bench.py times (one FP64 solve per instance) takes the
    oracle's iterates on the sampled instances."""
    inst, sample, g = batch256
    for k in sample:
        s = binding.Solver(inst[k][0], precision="fp64")
        u, st = s.solve(inst[k][1])
        assert st["status"] == 0
        assert st["iters"] == len(g[f"i{k}_trace8"]) - 1, k
        assert rel(u, g[f"i{k}_u8"]) <= 1e-8, k
        s.set_options(tol=1e-11)
        u12, _ = s.solve(inst[k][1])
        assert rel(u12, g[f"i{k}_u12"]) <= 1e-10, k
        s.close()


@pytest.fixture(scope="module")
def warm_gold():
    g = np.load(os.path.join(GOLD, "warm_heldout_g32.npz"))
    seed0 = int(g["seed0"])
    nw = sum(1 for key in g.files if key.startswith("w") and key.endswith("_u12"))
    xt = [g[f"w{j}_x0"] for j in range(nw)]
    for j in range(nw):
        np.testing.assert_array_equal(xt[j], inputs.x0_gaussians(32, seed0 + j))
    return g, xt


def test_warm_start_from_stored_guess_takes_the_oracle_warm_iterates(warm_gold):
    """The warm start itself (clip into the box with a margin, slacks floored
    at 1e-2, duals mu0 / s) against the oracle started from the same stored
    guess: the FP64 path takes the oracle's warm iterates (same count, mu_k);
    the FP32 tier, single and batched, stops within 1e-6 of the oracle's warm
    stop point; at 1e-11 the FP64 path stops within the degenerate optimum's
    band of the oracle's and meets the KKT conditions."""
    g, xt = warm_gold
    p = inputs.heat2d(32, 10, 50)
    s = binding.Solver(p, precision="fp64")
    for j in range(len(xt)):
        u, st = s.solve_warm(xt[j], g[f"v{j}_guess"])
        assert st["status"] == 0
        assert st["iters"] == len(g[f"v{j}_trace8"]) - 1, j
        np.testing.assert_allclose(s.get_trace()[:, 0], g[f"v{j}_trace8"][:, 0], rtol=1e-6)
        assert rel(u, g[f"v{j}_u8"]) <= 1e-8, j
    # Both run on to 1e-11: the same iterates in exact arithmetic, but at
    # mu ~ 1e-11 the rounding of each Newton step is amplified by
    # cond(M) ~ 1/mu, and the warm start of held-out x0 3 meets a degenerate
    # optimum (a pair of inputs moves by +-2.6e-6 along a direction the cost
    # does not see to first order): the oracle's own 1e-11 stop lies 2.45e-6
    # from where it stalls at 1e-12 and 1e-13.  So the stop is compared
    # within sqrt(tol), and the result must satisfy the optimality
    # conditions on its own (the stop test bounds the mean complementarity).
    s.set_options(tol=1e-11)
    for j in range(len(xt)):
        u, _ = s.solve_warm(xt[j], g[f"v{j}_guess"])
        assert rel(u, g[f"v{j}_u12"]) <= np.sqrt(1e-11), j
        kc = oracle.kkt_check(p, xt[j], u, s.get_duals())
        assert kc["primal_violation"] <= 1e-9, j
        assert kc["dual_min"] >= 0.0, j
        assert kc["stationarity"] <= 1e-8, j
        assert kc["complementarity_mean"] <= 1.01e-11, j
    m = binding.Solver(p, precision="fp32")
    for j in range(len(xt)):
        u, st = m.solve_warm(xt[j], g[f"v{j}_guess"])
        assert st["status"] == 0
        assert rel(u, g[f"v{j}_u8"]) <= 1e-6, j
    solvers = [binding.Solver(p, precision="fp32") for _ in xt]
    us, stats, code = binding.solve_batch(solvers, xt, u_inits=[g[f"v{j}_guess"] for j in range(len(xt))])
    assert code == 0
    for j in range(len(xt)):
        assert rel(us[j], g[f"v{j}_u8"]) <= 1e-6, j


def test_warm_start_c5_network_saves_iterations_and_meets_kkt(warm_gold):
    """The 1024-512-512-500 network trained on (x0, u*) pairs from the FP64
    GPU solver (lockstep batches, as bench.py makes them; fewer pairs here),
    then warm-started solves of the held-out x0: fewer iterations than cold
    starts at the metric's 1e-8 stop; at 1e-11 the KKT conditions of Eq. 5
    hold, single and batched, and u is within the degenerate optimum's band
    of the oracle's (zero multipliers at active bounds: a stop at tolerance
    tol sits O(sqrt(tol)) from u*; bar 30 sqrt(tol))."""
    g, xt = warm_gold
    p = inputs.heat2d(32, 10, 50)
    gen = [binding.Solver(p, precision="fp64") for _ in range(256)]
    X, U = [], []
    for k0 in range(0, 1024, 256):
        x0s = [inputs.x0_gaussians(32, s) for s in range(k0, k0 + 256)]
        u, st, code = binding.solve_batch(gen, x0s)
        assert code == 0
        X += x0s
        U += u
    for s in gen:
        s.close()
    net = binding.MLP(p.ns, 512, p.n, max_batch=256, seed=1)
    net.set_bounds(np.tile(p.ul, p.N), np.tile(p.uu, p.N))
    losses = net.train(np.array(X), np.array(U), epochs=40, batch=256, lr=1e-3, seed=2)
    assert losses[-1] < 0.2 * losses[0]
    guess = net.infer(np.array(xt))
    s = binding.Solver(p, precision="fp32")
    warm_it, cold_it = [], []
    for j in range(len(xt)):
        _, stw = s.solve_warm(xt[j], guess[j])
        _, stc = s.solve(xt[j])
        warm_it.append(stw["iters"])
        cold_it.append(stc["iters"])
    assert np.mean(warm_it) < np.mean(cold_it)
    s.set_options(tol=1e-11)
    band = 30.0 * np.sqrt(1e-11)
    for j in range(len(xt)):
        u, st = s.solve_warm(xt[j], guess[j])
        assert st["status"] == 0
        k = oracle.kkt_check(p, xt[j], u, s.get_duals())
        assert k["primal_violation"] <= 1e-9 and k["dual_min"] >= 0.0
        assert k["stationarity"] <= 1e-8 and k["complementarity"] <= 1e-9
        assert rel(u, g[f"w{j}_u12"]) <= band, j
    solvers = [binding.Solver(p, precision="fp32", tol=1e-11) for _ in xt]
    us, stats, code = binding.solve_batch(solvers, xt, u_inits=list(guess))
    assert code == 0
    for j in range(len(xt)):
        k = oracle.kkt_check(p, xt[j], us[j], solvers[j].get_duals())
        assert k["stationarity"] <= 1e-8 and k["complementarity"] <= 1e-9
        assert rel(us[j], g[f"w{j}_u12"]) <= band, j


CUBE = np.load(os.path.join(GOLD, "cube_table1.npz"))
CUBE_CASES = [tuple(int(v) for v in c) for c in CUBE["cases"]]


@pytest.mark.parametrize("g,T", CUBE_CASES, ids=[f"g{g}_T{T}" for g, T in CUBE_CASES])
def test_cube_plant_matches_oracle(g, T):
    """The paper's 3-D cube problem (Table I, nu = 6, n = 6T): the FP64 path
    takes the oracle's iterates; FP64 and the FP32 tier reach the oracle's
    optimum when both run to 1e-11.  T = 250 and 500 (n = 1500 and 3000, the
    paper's longest horizon) are past the queued dataflow Cholesky's n <= 1024:
    the grid-cooperative kernel factors them."""
    p, x0 = inputs.heat3d_cube(g, T), inputs.x0_cube(g)
    tag = f"g{g}_T{T}"
    s = binding.Solver(p, precision="fp64")
    u, st = s.solve(x0)
    assert st["status"] == 0
    assert st["iters"] == len(CUBE[f"{tag}_trace8"]) - 1
    np.testing.assert_allclose(s.get_trace()[:, 0], CUBE[f"{tag}_trace8"][:, 0], rtol=1e-6)
    assert rel(u, CUBE[f"{tag}_u8"]) <= 1e-8
    for precision, bar in (("fp64", 1e-10), ("fp32", 1e-6)):
        s = binding.Solver(p, precision=precision, tol=1e-11)
        u, st = s.solve(x0)
        assert st["status"] == 0, precision
        assert rel(u, CUBE[f"{tag}_u12"]) <= bar, precision


@pytest.mark.parametrize("g,T", [(4, 250), (4, 500)], ids=["g4_T250", "g4_T500"])
def test_cube_two_level_tier_past_n1024_matches_oracle(g, T):
    """Solves started in the two-level FP32 tier at n = 1500 and 3000, where
    the grid-cooperative Cholesky factors (both of the tier's factorisations):
    no escalation to FP64 and the oracle's optimum at the 1e-8 stop."""
    p, x0 = inputs.heat3d_cube(g, T), inputs.x0_cube(g)
    tag = f"g{g}_T{T}"
    s = binding.Solver(p, precision="fp32x2")
    u, st = s.solve(x0)
    assert st["status"] == 0
    assert st["fallbacks"] == 0, st["fallbacks"]
    assert rel(u, CUBE[f"{tag}_u8"]) <= 1e-6
