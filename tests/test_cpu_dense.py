"""The CPU condensed-dense baseline (baseline/, the analogue of the paper's
"CPU dense" columns) against the oracle: the same method on the condensed
problem takes the oracle's iterates in exact arithmetic (condensing is an
exact elimination), so iteration counts agree and u agrees to FP64 rounding
amplified by the conditioning of the late iterations (bar 1e-9 relative).
CPU only."""
import os

import numpy as np
import pytest

import baseline
import oracle
from paper_2209_13049_b300 import inputs

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rel(u, ref):
    return float(np.max(np.abs(u - ref)) / max(1.0, np.max(np.abs(ref))))


@pytest.mark.parametrize("seed", range(4))
def test_heat1d_matches_oracle(seed):
    g = np.load(os.path.join(GOLD, "heat1d_ns50_nu5_N10.npz"))
    p, x0 = inputs.config_1d_small(seed)
    r = baseline.solve(p, x0, tol=1e-8, threads=2)
    assert r["status"] == 0
    assert r["stats"]["iters"] == len(g[f"heat1d_50_s{seed}_trace8"]) - 1
    assert rel(r["u"], g[f"heat1d_50_s{seed}_u8"]) <= 1e-9
    r = baseline.solve(p, x0, tol=1e-11, threads=2)
    assert rel(r["u"], g[f"heat1d_50_s{seed}_u12"]) <= 1e-9


def test_uneven_small_batch_instances_match_oracle():
    g = np.load(os.path.join(GOLD, "batch_small.npz"))
    for k in range(6):
        ns, nu, N, gside = (int(v) for v in g[f"b{k}_dims"])
        p = inputs.heat1d(ns, nu, N) if gside == 0 else inputs.heat2d(gside, nu, N)
        r = baseline.solve(p, g[f"b{k}_x0"], tol=1e-8)
        assert r["status"] == 0
        assert r["stats"]["iters"] == len(g[f"b{k}_trace8"]) - 1, k
        assert rel(r["u"], g[f"b{k}_u8"]) <= 1e-9, k


def test_cube_plant_matches_oracle():
    g = np.load(os.path.join(GOLD, "cube_table1.npz"))
    p, x0 = inputs.heat3d_cube(5, 50), inputs.x0_cube(5)
    r = baseline.solve(p, x0, tol=1e-8)
    assert r["status"] == 0
    assert r["stats"]["iters"] == len(g["g5_T50_trace8"]) - 1
    assert rel(r["u"], g["g5_T50_u8"]) <= 1e-9


def test_random_dense_plant_matches_oracle():
    """A non-symmetric dense A, dense Q and R (the heat plants have a
    symmetric stencil A and diagonal Q)."""
    p = inputs.random_small(9, 3, 12, 5, xb=1.5, ub=0.6, dense_q=True)
    x0 = np.random.default_rng(2).uniform(-1, 1, 9)
    ref = oracle.ipm_solve(p, x0, tol=1e-11)
    r = baseline.solve(p, x0, tol=1e-11)
    assert ref["status"] == 0 and r["status"] == 0
    assert r["stats"]["iters"] == ref["stats"]["iters"]
    assert rel(r["u"], ref["u"]) <= 1e-9


def test_unbounded_is_the_unconstrained_minimiser():
    """No finite bound: one Newton step gives u = -H^-1 h (Eq. 3)."""
    p = inputs.heat1d(30, 3, 7)
    p.xl[:], p.xu[:], p.ul[:], p.uu[:] = -np.inf, np.inf, -np.inf, np.inf
    x0 = inputs.x0_uniform(30, 0)
    r = baseline.solve(p, x0)
    _, _, H, h = oracle.condensed(p, x0)
    assert r["status"] == 0 and r["stats"]["iters"] <= 2
    assert rel(r["u"], -np.linalg.solve(H, h)) <= 1e-11


def test_threads_do_not_change_the_result_beyond_rounding():
    p, x0 = inputs.config_1d_small(1)
    a = baseline.solve(p, x0, tol=1e-10, threads=1)
    b = baseline.solve(p, x0, tol=1e-10, threads=4)
    assert a["stats"]["iters"] == b["stats"]["iters"]
    assert rel(a["u"], b["u"]) <= 1e-12
