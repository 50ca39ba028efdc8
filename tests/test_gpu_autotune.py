"""The autotuner (lqmpc_autotune): measured launch shapes for a batch
signature, a cache file of decisions, and solves that still match the oracle
with the tuned shapes."""
import os

import numpy as np
import pytest

from paper_2209_13049_b300 import binding, build, inputs

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.load()


def rel(u, ref):
    return float(np.max(np.abs(u - ref)) / max(1.0, np.max(np.abs(ref))))


def test_autotune_cache_and_parity(tmp_path):
    g = np.load(os.path.join(GOLD, "batch_small.npz"))
    solvers, x0s, refs = [], [], []
    for k in range(6):
        ns, nu, N, gside = (int(v) for v in g[f"b{k}_dims"])
        p = inputs.heat1d(ns, nu, N) if gside == 0 else inputs.heat2d(gside, nu, N)
        solvers.append(binding.Solver(p, tol=1e-11))
        x0s.append(g[f"b{k}_x0"])
        refs.append(g[f"b{k}_u12"])
    cache = tmp_path / "tune.txt"
    binding.autotune(solvers, cache)
    lines = cache.read_text().split("\n")
    lines = [l for l in lines if l.strip()]
    assert len(lines) == 1
    key, cc, p32, p64, k64 = lines[0].split()
    assert key.startswith("b6-") and int(cc) >= 1 and int(p32) in (0, 1, 2, 3) and int(p64) in (0, 1)
    assert int(k64) in (-1, 0, 1)
    # a second call finds the signature in the cache and appends nothing
    binding.autotune(solvers, cache)
    assert len([l for l in cache.read_text().split("\n") if l.strip()]) == 1
    us, stats, code = binding.solve_batch(solvers, x0s)
    assert code == 0
    for k in range(6):
        assert rel(us[k], refs[k]) <= 1e-9, k


def test_autotune_single_instance_then_solve():
    p, x0 = inputs.config_2d_32(0, N=20)
    s = binding.Solver(p, precision="bf16")
    u0, st0 = s.solve(x0)
    binding.autotune([s])
    u1, st1 = s.solve(x0)
    assert st1["status"] == 0
    assert rel(u1, u0) <= 1e-6
