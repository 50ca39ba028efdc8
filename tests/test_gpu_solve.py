"""End-to-end parity of the GPU interior-point solve (through the C ABI)
against the oracle and against properties that hold at any size.

Bars: FP64 GPU path within 1e-10 relative of the oracle's u* (both run to a
tight tolerance), and, at the 1e-8 stop tolerance, the same iteration count
and per-iteration mu as the oracle (condensing is an exact elimination, so
the two methods take the same iterates in exact arithmetic).  Mixed paths
within 1e-6 relative of the oracle's u*.  Relative error is
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
def heat1d_gold():
    return np.load(os.path.join(GOLD, "heat1d_ns50_nu5_N10.npz"))


@pytest.fixture(scope="module")
def heat2d_gold():
    return np.load(os.path.join(GOLD, "heat2d_g32_nu10_N50.npz"))


@pytest.mark.parametrize("seed", range(4))
def test_fp64_heat1d_matches_oracle(seed, heat1d_gold):
    p, x0 = inputs.config_1d_small(seed)
    np.testing.assert_array_equal(x0, heat1d_gold[f"heat1d_50_s{seed}_x0"])
    s = binding.Solver(p, tol=1e-11)
    u, st = s.solve(x0)
    assert st["status"] == 0
    assert rel(u, heat1d_gold[f"heat1d_50_s{seed}_u12"]) <= 1e-10
    s.set_options(tol=1e-8)
    u8, st8 = s.solve(x0)
    tr_ref = heat1d_gold[f"heat1d_50_s{seed}_trace8"]
    assert st8["iters"] == len(tr_ref) - 1
    tr = s.get_trace()
    np.testing.assert_allclose(tr[:, 0], tr_ref[:, 0], rtol=1e-8)
    np.testing.assert_allclose(tr[:-1, 3:6], tr_ref[:-1, 3:6], rtol=1e-7, atol=1e-12)
    assert rel(u8, heat1d_gold[f"heat1d_50_s{seed}_u8"]) <= 1e-9


def test_fp64_heat2d_matches_oracle(heat2d_gold):
    p, x0 = inputs.config_2d_32(0)
    s = binding.Solver(p)
    u, st = s.solve(x0)
    tr_ref = heat2d_gold["heat2d_32_s0_trace8"]
    assert st["status"] == 0
    assert st["iters"] == len(tr_ref) - 1
    tr = s.get_trace()
    np.testing.assert_allclose(tr[:, 0], tr_ref[:, 0], rtol=1e-6)
    assert rel(u, heat2d_gold["heat2d_32_s0_u8"]) <= 1e-8
    # Degenerate active constraints (zero multiplier at a bound) make u converge
    # like sqrt(mu): the 1e-8 stop point sits about 5e-5 from the optimum.
    assert rel(u, heat2d_gold["heat2d_32_s0_u12"]) <= 2e-4
    s.set_options(tol=1e-11)
    u12, _ = s.solve(x0)
    assert rel(u12, heat2d_gold["heat2d_32_s0_u12"]) <= 1e-10


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
def test_mixed_heat2d_matches_oracle(precision, heat2d_gold):
    """Mixed path against the oracle at the same stop tolerance (1e-8, the
    metric's) and near the optimum (1e-11)."""
    p, x0 = inputs.config_2d_32(0)
    s = binding.Solver(p, precision=precision)
    u, st = s.solve(x0)
    assert st["status"] == 0
    assert rel(u, heat2d_gold["heat2d_32_s0_u8"]) <= 1e-6
    s.set_options(tol=1e-11)
    u, st = s.solve(x0)
    assert st["status"] == 0
    assert rel(u, heat2d_gold["heat2d_32_s0_u12"]) <= 1e-6


@pytest.mark.parametrize("precision", ["fp64", "bf16", "fp32x2"])
def test_mixed_heat1d_matches_oracle(precision, heat1d_gold):
    p, x0 = inputs.config_1d_small(1)
    s = binding.Solver(p, precision=precision, tol=1e-11)
    u, st = s.solve(x0)
    assert st["status"] == 0
    assert rel(u, heat1d_gold["heat1d_50_s1_u12"]) <= (1e-10 if precision == "fp64" else 1e-6)


def test_batch_uneven_matches_oracle():
    g = np.load(os.path.join(GOLD, "batch_small.npz"))
    solvers, x0s, refs = [], [], []
    for k in range(6):
        ns, nu, N, gside = (int(v) for v in g[f"b{k}_dims"])
        p = inputs.heat1d(ns, nu, N) if gside == 0 else inputs.heat2d(gside, nu, N)
        solvers.append(binding.Solver(p, tol=1e-11))
        x0s.append(g[f"b{k}_x0"])
        refs.append(g[f"b{k}_u12"])
    us, stats, code = binding.solve_batch(solvers, x0s)
    assert code == 0
    for k in range(6):
        assert stats[k]["status"] == 0
        assert rel(us[k], refs[k]) <= 1e-10, k
        # the batched lockstep result equals the single-instance result
        u1, _ = solvers[k].solve(x0s[k])
        assert rel(us[k], u1) <= 1e-12


def test_kkt_properties_at_full_size_100x100():
    """ns = 10000, nu = 20, N = 50 (n = 1000): too large for the oracle's IPM;
    check the KKT conditions of the GPU solution with the oracle's checker."""
    p, x0 = inputs.config_2d_100(0)
    s = binding.Solver(p, precision="bf16")
    u, st = s.solve(x0)
    assert st["status"] == 0
    z = s.get_duals()
    k = oracle.kkt_check(p, x0, u, z)
    assert k["primal_violation"] <= 1e-7
    assert k["dual_min"] >= 0.0
    assert k["stationarity"] <= 1e-6
    assert k["complementarity"] <= 1e-6


def test_unbounded_is_one_newton_step():
    """Every bound infinite: m = 0, the first Newton step is exact."""
    p = inputs.heat1d(30, 3, 7)
    p.xl[:], p.xu[:], p.ul[:], p.uu[:] = -np.inf, np.inf, -np.inf, np.inf
    x0 = inputs.x0_uniform(30, 0)
    u, st = binding.Solver(p).solve(x0)
    Gam, y, H, h = oracle.condensed(p, x0)
    assert st["iters"] <= 2
    assert rel(u, -np.linalg.solve(H, h)) <= 1e-11


@pytest.mark.parametrize("dims", [(1, 1, 1), (3, 1, 1), (1, 2, 5), (65, 1, 2), (33, 33, 2)])
def test_edge_sizes_match_oracle(dims):
    ns, nu, N = dims
    p = inputs.random_small(ns, nu, N, 11, xb=2.0, ub=1.0)
    x0 = np.random.default_rng(3).uniform(-0.5, 0.5, ns)
    ref = oracle.ipm_solve(p, x0, tol=1e-11)
    assert ref["status"] == 0
    u, st = binding.Solver(p, tol=1e-11).solve(x0)
    assert st["status"] == 0
    assert rel(u, ref["u"]) <= 1e-9


def test_invalid_arguments_rejected():
    p = inputs.heat1d(10, 2, 3)
    p.xl[0] = 2.0                      # crossed bound
    with pytest.raises(binding.LqmpcError) as e:
        binding.Solver(p)
    assert e.value.code == 1
    p = inputs.heat1d(10, 2, 3)
    s = binding.Solver(p)
    x0 = np.zeros(10)
    x0[3] = np.nan
    with pytest.raises(binding.LqmpcError):
        s.solve(x0)


def test_maxiter_reported():
    p, x0 = inputs.config_1d_small(0)
    s = binding.Solver(p, max_iter=2)
    u, st = s.solve(x0, check=False)
    assert st["status"] == 4 and st["iters"] == 2


def test_solve_device_equals_host():
    import torch
    p, x0 = inputs.config_1d_small(3)
    s = binding.Solver(p)
    u_host, _ = s.solve(x0)
    xd = torch.tensor(x0, dtype=torch.float64, device="cuda")
    ud = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    s.solve_device(xd, ud)
    np.testing.assert_array_equal(ud.cpu().numpy(), u_host)


def test_large_batch_cluster_factor_matches_single():
    """A batch large enough to give every instance its own 8-CTA cluster for
    the Cholesky factorisation (the single-instance solves use the
    grid-cooperative kernel): same iterates up to rounding, so the same u*."""
    sizes = [(20 + 3 * k, 2 + k % 4, 4 + k % 7) for k in range(20)]
    solvers, x0s = [], []
    for k, (ns, nu, N) in enumerate(sizes):
        solvers.append(binding.Solver(inputs.heat1d(ns, nu, N), tol=1e-11))
        x0s.append(inputs.x0_uniform(ns, 100 + k))
    us, stats, code = binding.solve_batch(solvers, x0s)
    assert code == 0
    for k in range(len(sizes)):
        assert stats[k]["status"] == 0
        u1, _ = solvers[k].solve(x0s[k])
        assert rel(us[k], u1) <= 1e-9, k
    ref = oracle.ipm_solve(inputs.heat1d(*sizes[7]), x0s[7], tol=1e-11)
    assert rel(us[7], ref["u"]) <= 1e-9


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
def test_batch_uneven_tensor_core_matches_oracle(precision):
    """Batches run the tensor-core SYRK with every instance's own tensor maps
    and split plan (grid.y = instance)."""
    g = np.load(os.path.join(GOLD, "batch_small.npz"))
    solvers, x0s, refs = [], [], []
    for k in range(6):
        ns, nu, N, gside = (int(v) for v in g[f"b{k}_dims"])
        p = inputs.heat1d(ns, nu, N) if gside == 0 else inputs.heat2d(gside, nu, N)
        solvers.append(binding.Solver(p, tol=1e-11, precision=precision))
        x0s.append(g[f"b{k}_x0"])
        refs.append(g[f"b{k}_u12"])
    us, stats, code = binding.solve_batch(solvers, x0s)
    assert code == 0
    for k in range(6):
        assert stats[k]["status"] == 0
        assert rel(us[k], refs[k]) <= 1e-6, k
    assert stats[0]["syrk_tc_launches"] > 0


def test_uneven_batch_cooperative_factor_matches_single():
    """First 24 instances of the uneven 256-instance batch (n up to 800, too
    large for the cluster factorisation): the grid-cooperative Cholesky then
    interleaves the panels of many instances, and each instance must still
    take the iterates it takes alone."""
    inst = inputs.batch_instances(256, 0)[:24]
    solvers = [binding.Solver(p) for p, _ in inst]
    x0s = [x for _, x in inst]
    singles = [s.solve(x)[0] for s, x in zip(solvers, x0s)]
    us, stats, code = binding.solve_batch(solvers, x0s)
    assert code == 0
    for k in range(len(inst)):
        assert stats[k]["status"] == 0
        assert rel(us[k], singles[k]) <= 1e-8, k


@pytest.mark.parametrize("variant", ["rule", "queued", "coop"])
def test_uneven_batch_fp32_factor_variants_match_single(variant):
    """The 24 first instances of the uneven batch in the FP32 tier (n up to
    800): by the rule the queued dataflow Cholesky factors every instance
    (too few instances for one cluster each), and the forced variants must
    agree too; each instance within the FP32 tier's own solve-to-solve spread
    of its single solve (both stop at the 1e-8 test)."""
    inst = inputs.batch_instances(256, 0)[:24]
    if variant != "rule":
        os.environ["LQMPC_POTRF"] = variant
    try:
        solvers = [binding.Solver(p, precision="fp32") for p, _ in inst]
        x0s = [x for _, x in inst]
        us, stats, code = binding.solve_batch(solvers, x0s)
    finally:
        os.environ.pop("LQMPC_POTRF", None)
    assert code == 0
    for k in range(len(inst)):
        assert stats[k]["status"] == 0
        ref = binding.Solver(inst[k][0], precision="fp64").solve(x0s[k])[0]
        assert rel(us[k], ref) <= 1e-6, k


def test_two_level_tier_batch_matches_fp64():
    """A batch started in the two-level FP32 tier (FP64 formation, FP32
    factor of M, FP32 factor of L1^-1 M L1^-T, combined inverse): every
    instance within the mixed tiers' spread of its FP64 single solve."""
    inst = inputs.batch_instances(256, 0)[:12]
    solvers = [binding.Solver(p, precision="fp32x2") for p, _ in inst]
    x0s = [x for _, x in inst]
    us, stats, code = binding.solve_batch(solvers, x0s)
    assert code == 0
    for k in range(len(inst)):
        assert stats[k]["status"] == 0
        ref = binding.Solver(inst[k][0], precision="fp64").solve(x0s[k])[0]
        assert rel(us[k], ref) <= 1e-6, k
