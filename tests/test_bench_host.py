"""Host arithmetic of bench.py's roofline fields, on CPU.

The algorithmic flop count of one formation of M (Eq. 7) is pinned by
counting the block products of the block-Toeplitz Gamma one by one, and the
Cholesky roofline by its definition: the method's n^3/3 flops per
factorisation over the live launch time, against the FP32 pipe's rate from
the unit counts and the clock.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


@pytest.mark.parametrize("ns,nu,N", [(50, 5, 10), (1024, 10, 50), (10000, 20, 50), (7, 3, 1)])
def test_formation_flops_count_the_toeplitz_block_products(ns, nu, N):
    # M[j, k] (j >= k, block columns of Gamma) = sum over stages t >= j of
    # Gamma[t, j]' Sigma_t Gamma[t, k]: N - j products of (nu x ns)(ns x nu)
    products = sum(N - j for j in range(N) for _ in range(j + 1))
    assert bench.syrk_alg_flops(ns, nu, N) == pytest.approx(products * 2.0 * ns * nu * nu, rel=1e-15)


def test_potrf_roofline_is_n_cubed_over_three_per_live_launch():
    st = [{"potrf32_launches": 3, "t_potrf32_ms": 0.30}, {"potrf32_launches": 1, "t_potrf32_ms": 0.10}]
    r = bench._potrf_roofline(st, 500, 2032.0, 765184, "k")
    assert r["avg_launch_us"] == pytest.approx(100.0)
    assert r["flops_per_launch"] == pytest.approx(500 ** 3 / 3)
    assert r["achieved"] == pytest.approx(500 ** 3 / 3 / 100e-6 / 1e12)
    assert r["peak"] == pytest.approx(148 * 128 * 2 * 2032e6 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["traffic"] == 765184


def test_tensor_roofline_counts_algorithmic_not_executed_flops():
    st = [{"syrk_tc3_launches": 2, "t_syrk_tc3_ms": 0.12, "syrk_tc_launches": 2, "t_syrk_tc_ms": 0.12}]
    peaks = {"bf16_tflops_sustained": 1348.1}
    r = bench._tc_roofline(st, 1024, 10, 50, peaks, "measured")
    f = bench.syrk_alg_flops(1024, 10, 50)
    s = r["split_tf32"]
    assert s["avg_launch_us"] == pytest.approx(60.0)
    assert s["achieved"] == pytest.approx(f / 60e-6 / 1e12)
    assert s["peak"] == pytest.approx(1348.1 / 2)
    assert s["frac"] == pytest.approx(s["achieved"] / s["peak"])
    assert s["executed_flops_per_launch"] == pytest.approx(3 * f)
    assert "single_product" not in r
