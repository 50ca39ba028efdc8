"""The warm-start network on the GPU (tcgen05 BF16 GEMMs, FP32 accumulation)
against the FP64 oracle (oracle/mlp.py), and the warm-started IPM against the
cold-started one and the oracle.

Tolerances.  The GPU rounds inputs, weights, activations and back-propagated
gradients to BF16 (relative rounding 2^-9 = 0.2%) and accumulates in FP32.
The oracle is evaluated on the BF16-rounded inputs and weights, so the
remaining differences come from the two stored activations and three stored
gradients, a handful of 0.2% roundings in sequence: norm-wise 2% per
parameter block is several times that.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_2209_13049_b300 import binding, build, inputs

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.load()


def bf16(a):
    """Round to the nearest BF16 (ties to even) and back to FP64."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def rel_norm(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def _net_and_data(n_in=200, n_h=128, n_out=70, B=100, seed=0):
    rng = np.random.default_rng(seed)
    net = binding.MLP(n_in, n_h, n_out, max_batch=256, seed=seed + 11)
    X = rng.uniform(-1, 1, (B, n_in)).astype(np.float32)
    U = rng.normal(0, 0.5, (B, n_out)).astype(np.float32)
    return net, X, U


def _oracle_params(net, quantize=True):
    p = omlp.unpack(net.get_params().astype(np.float64), net.n_in, net.n_hidden, net.n_out)
    if quantize:
        for k in (0, 2, 4):
            p[k] = bf16(p[k])
    return p


def test_gradients_match_oracle_ragged_sizes():
    net, X, U = _net_and_data()
    g, loss = net.grad(X, U)
    p = _oracle_params(net)
    ref, ref_loss = omlp.grad(p, bf16(X), U.astype(np.float64))
    got = omlp.unpack(g.astype(np.float64), net.n_in, net.n_hidden, net.n_out)
    assert loss == pytest.approx(ref_loss, rel=1e-2)
    for k, (a, b) in enumerate(zip(got, ref)):
        assert rel_norm(a, b) <= 2e-2, (k, rel_norm(a, b))


def test_inference_matches_oracle_with_projection():
    net, X, _ = _net_and_data(B=300, seed=3)
    lo = np.full(net.n_out, -0.05)
    hi = np.full(net.n_out, 0.08)
    net.set_bounds(lo, hi)
    u = net.infer(X.astype(np.float64))
    ref = omlp.infer(_oracle_params(net), bf16(X), lo, hi)
    assert np.all(u >= lo) and np.all(u <= hi)
    assert np.max(np.abs(u - ref)) <= 2e-2 * max(np.max(np.abs(ref)), 1e-3)


def test_first_adam_step_moves_by_lr_sign_g():
    """From zero moments Adam's first step is lr * g / (|g| + eps)."""
    net, X, U = _net_and_data(B=128, seed=4)
    p0 = net.get_params().astype(np.float64)
    ref, _ = omlp.grad(_oracle_params(net), bf16(X), U.astype(np.float64))
    gref = omlp.pack(ref)
    lr = 1e-3
    net.train(X, U, epochs=1, batch=128, lr=lr, seed=0)      # one step over the whole set
    dp = net.get_params().astype(np.float64) - p0
    big = np.abs(gref) > 0.1 * np.sqrt(np.mean(gref ** 2))
    np.testing.assert_allclose(dp[big], -lr * np.sign(gref[big]), rtol=1e-3, atol=1e-7)


def test_training_fits_a_teacher_network():
    rng = np.random.default_rng(7)
    n_in, n_h, n_out, S = 64, 128, 32, 2048
    teacher = binding.MLP(n_in, n_h, n_out, max_batch=256, seed=99)
    X = rng.uniform(0, 1, (S, n_in))
    U = teacher.infer(X)
    net = binding.MLP(n_in, n_h, n_out, max_batch=256, seed=5)
    losses = net.train(X, U, epochs=60, batch=256, lr=2e-3, seed=1)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.05 * losses[0]


@pytest.fixture(scope="module")
def small_plant_pairs():
    """(x0, u*) pairs of a heat2d 8x8 plant (ns = 64, nu = 4, N = 10) from the FP64 GPU solver."""
    p = inputs.heat2d(8, 4, 10)
    s = binding.Solver(p, tol=1e-10)
    xs, us, it = [], [], []
    for seed in range(1600):
        x0 = inputs.x0_gaussians(8, seed)
        u, st = s.solve(x0)
        xs.append(x0)
        us.append(u)
        it.append(st["iters"])
    return p, np.array(xs), np.array(us), np.array(it)


def test_warm_start_from_trained_network_saves_iterations(small_plant_pairs):
    p, xs, us, cold_iters = small_plant_pairs
    train, test = slice(0, 1536), slice(1536, 1600)
    net = binding.MLP(p.ns, 128, p.n, max_batch=256, seed=3)
    net.set_bounds(np.tile(p.ul, p.N), np.tile(p.uu, p.N))
    losses = net.train(xs[train], us[train], epochs=150, batch=128, lr=2e-3, seed=2)
    assert losses[-1] < 0.1 * losses[0]
    guess = net.infer(xs[test])
    s = binding.Solver(p, tol=1e-10)
    warm_iters = []
    for k, x0 in enumerate(xs[test]):
        u, st = s.solve_warm(x0, guess[k])
        assert st["status"] == 0
        warm_iters.append(st["iters"])
        # the same optimum: these problems are degenerate (zero multipliers at
        # active bounds), where iterates stopped at 1e-10 from different starts
        # differ like sqrt(1e-10); the KKT conditions of the warm result decide
        ref = us[test][k]
        assert np.max(np.abs(u - ref)) / max(1.0, np.max(np.abs(ref))) <= 1e-3
        kk = oracle.kkt_check(p, x0, u, s.get_duals())
        assert kk["primal_violation"] <= 1e-8 and kk["dual_min"] >= 0.0
        assert kk["stationarity"] <= 1e-7 and kk["complementarity"] <= 1e-6
    assert np.mean(warm_iters) < np.mean(cold_iters[test]) - 1.0


def test_warm_start_from_any_guess_reaches_the_oracle_optimum():
    g = np.load(os.path.join(GOLD, "heat1d_ns50_nu5_N10.npz"))
    p, x0 = inputs.config_1d_small(2)
    ref = g["heat1d_50_s2_u12"]
    s = binding.Solver(p, tol=1e-11)
    u_cold, st_cold = s.solve(x0)
    rng = np.random.default_rng(0)
    # any start reaches the unique optimum; stopping at 1e-11 from a different
    # start leaves a different last iterate, within 1e-8 of the 1e-12 optimum
    for guess in (ref, np.zeros(p.n), rng.uniform(-10, 10, p.n)):
        u, st = s.solve_warm(x0, guess)
        assert st["status"] == 0
        assert np.max(np.abs(u - ref)) / max(1.0, np.max(np.abs(ref))) <= 1e-8
    u, st = s.solve_warm(x0, ref)
    assert st["iters"] < st_cold["iters"]
