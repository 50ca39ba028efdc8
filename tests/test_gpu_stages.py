"""Parity of each hot-path step (CUDA via the C ABI) against the oracle.

Tolerances (element-wise, derived from the arithmetic):
  FP64 steps: 1e-12 relative to the sum of absolute terms of each entry.
  FP32 CUDA-core SYRK: 4 * 2^-24 * (sqrt(K) + 2) relative to the absolute sum.
  TF32 tensor-core SYRK: operands rounded to 10 mantissa bits (relative 2^-11
    each) and the scaled operand rounded again: |err| <= 4 * 2^-11 * abs-sum.
  BF16 tensor-core SYRK: 8 mantissa bits: |err| <= 4 * 2^-8 * abs-sum.
"""
import numpy as np
import pytest

import oracle
from paper_2209_13049_b300 import binding, build, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.load()


def _abs_sum(Gam, H, sigx, sigu):
    return np.abs(H) + np.abs(Gam).T @ (np.asarray(sigx)[:, None] * np.abs(Gam)) + np.diag(np.abs(sigu))


CASES = [
    ("heat1d_50", lambda: inputs.heat1d(50, 5, 10)),
    ("heat2d_10_ragged", lambda: inputs.heat2d(10, 7, 23)),      # n = 161: ragged 128/64/32 tiles
    ("heat1d_300_N37", lambda: inputs.heat1d(300, 3, 37)),        # n = 111
    ("dense_q", lambda: inputs.random_small(9, 4, 33, 3, dense_q=True)),  # non-diagonal Q, n = 132
    # more than 16 inputs: the Gamma' product takes its input columns in several passes
    ("heat1d_60_nu20", lambda: inputs.heat1d(60, 20, 6)),         # n = 120, two full passes
    ("heat1d_70_nu17", lambda: inputs.heat1d(70, 17, 5)),         # n = 85, a one-column second pass
]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    p = request.param[1]()
    s = binding.Solver(p)
    Gam, _, H, _ = oracle.condensed(p, np.zeros(p.ns))
    return p, s, Gam, H


def test_gstack_matches_oracle(case):
    p, s, _, _ = case
    G = s.get_gstack()
    np.testing.assert_allclose(G, oracle.gstack(p), rtol=1e-13, atol=1e-15)


def test_hessian_matches_oracle(case):
    p, s, Gam, H = case
    Hg = s.get_hessian()
    ref = np.abs(Gam).T @ np.abs(Gam) * max(1.0, np.abs(p.dense("Q")).max()) + np.abs(H)
    assert np.all(np.abs(Hg - H) <= 1e-12 * ref + 1e-300)


@pytest.mark.parametrize("arith,rel", [("fp64", 1e-14), ("bf16", 2e-12)])
def test_gamma_products_match_oracle(case, arith, rel):
    """FP64 products: ~n eps64 of the absolute sum; float-float products (used
    by the mixed solves): a few 2^-44 per term, bounded here by 2e-12 of the
    largest absolute sum (norm-wise: float-float words have FP32's exponent
    range, so entries below ~1e-38 underflow to zero)."""
    p, s, Gam, _ = case
    s.set_options(precision=arith)
    rng = np.random.default_rng(1)
    v = rng.standard_normal(p.n)
    w = rng.standard_normal(p.ns * p.N)
    gv = s.gamma_mv(v)
    assert np.max(np.abs(gv - Gam @ v)) <= rel * np.max(np.abs(Gam) @ np.abs(v))
    gw = s.gamma_tmv(w)
    assert np.max(np.abs(gw - Gam.T @ w)) <= rel * np.max(np.abs(Gam).T @ np.abs(w))
    s.set_options(precision="fp64")


@pytest.mark.parametrize("arith,rel", [("fp64", 1e-12), ("fp32", 1e-11)])
def test_gamma_products_full_size_heat2d_32(arith, rel):
    """Both products at the bench's plant (ns = 1024, nu = 10, N = 50, n = 500)
    in the launch configuration a solve uses: 16 K-splits and anti-diagonal
    sums of up to 50 terms for the float-float Gamma' w, 10 splits for
    Gamma v.  Bars, normwise against the largest absolute sum:
      fp32 (float-float products, float-float split-K partials and sums):
        a few 2^-44 per term (the float-float words), plus one 2^-47 rounding
        per float-float addition in a CTA's 64-term partial and in the sum of
        up to 16 splits x 50 terms (<= 864 additions): <= 8e-12;
      fp64: blocked FP64 sums, (terms per block + blocks) 2^-53 <= 1.2e-13
      with a margin for the block plan."""
    p = inputs.heat2d(32, 10, 50)
    Gam, _, _, _ = oracle.condensed(p, np.zeros(p.ns))
    s = binding.Solver(p, precision=arith)
    rng = np.random.default_rng(11)
    for _ in range(2):
        v = rng.standard_normal(p.n)
        w = rng.standard_normal(p.ns * p.N)
        gv = s.gamma_mv(v)
        assert np.max(np.abs(gv - Gam @ v)) <= rel * np.max(np.abs(Gam) @ np.abs(v))
        gw = s.gamma_tmv(w)
        assert np.max(np.abs(gw - Gam.T @ w)) <= rel * np.max(np.abs(Gam).T @ np.abs(w))
    s.close()


def _sigmas(p, seed, spread=2.0):
    rng = np.random.default_rng(seed)
    sigx = 10.0 ** rng.uniform(-spread, spread, p.ns * p.N)
    sigu = 10.0 ** rng.uniform(-spread, spread, p.n)
    return sigx, sigu


@pytest.mark.parametrize("precision,rel", [("fp64", 1e-12), ("fp32", None), ("tf32", 4 * 2.0**-11),
                                           ("bf16", 4 * 2.0**-8), ("fp32x2", 1e-10)])
def test_kkt_matrix_matches_oracle(case, precision, rel):
    """fp32x2: the float-float Horner chains of the two-level tier, a few
    2^-44 per operation over the horizon's steps: bounded by 1e-10 of the
    absolute sum, far below FP32 rounding (E = M - L1 L1' needs that)."""
    p, s, Gam, H = case
    sigx, sigu = _sigmas(p, 2)
    M = s.form_kkt(sigx, sigu, precision)
    ref = oracle.kkt_matrix(p, sigx, sigu, Gam, H)
    absm = _abs_sum(Gam, H, sigx, sigu)
    if rel is None:
        rel = 4 * 2.0**-24 * (np.sqrt(p.ns * p.N) + 2)
    err = np.abs(M - ref)
    assert np.all(err <= rel * absm + 1e-300), (precision, float((err / absm).max()))
    np.testing.assert_array_equal(M, M.T)


def test_kkt_factor_and_solve_fp64(case):
    p, s, Gam, H = case
    sigx, sigu = _sigmas(p, 3)
    ref = oracle.kkt_matrix(p, sigx, sigu, Gam, H)
    b = np.random.default_rng(4).standard_normal(p.n)
    r = s.kkt_solve(sigx, sigu, b, "fp64", want_L=True)
    L = r["L"]
    Lref = np.linalg.cholesky(ref)
    np.testing.assert_allclose(L, Lref, rtol=0, atol=1e-10 * np.abs(Lref).max())
    x_ref = np.linalg.solve(ref, b)
    assert np.max(np.abs(r["x"] - x_ref)) <= 1e-9 * np.max(np.abs(x_ref))


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
def test_kkt_solve_mixed_refines_to_fp64_accuracy(case, precision):
    """Low-precision factor + FP64 refinement reaches the refinement tolerance
    (1e-10 relative residual) on a moderately conditioned M."""
    p, s, Gam, H = case
    sigx, sigu = _sigmas(p, 5, spread=1.0)
    ref = oracle.kkt_matrix(p, sigx, sigu, Gam, H)
    b = np.random.default_rng(6).standard_normal(p.n)
    r = s.kkt_solve(sigx, sigu, b, precision)
    res = np.max(np.abs(b - ref @ r["x"])) / np.max(np.abs(b))
    assert res <= 2e-10, res
    x_ref = np.linalg.solve(ref, b)
    # forward error <= cond(M) * backward error
    bound = 10 * np.linalg.cond(ref) * 2e-10 * np.max(np.abs(x_ref))
    assert np.max(np.abs(r["x"] - x_ref)) <= bound


def test_not_positive_definite_is_reported():
    """R = 0 with Sigma = 0 makes M singular (only H's zero rows) -> NOT_PD,
    no fault: the Cholesky records the pivot and the step is skipped."""
    p = inputs.heat1d(8, 2, 3)
    p.R = np.zeros((2, 2))
    p.B = np.zeros((8, 2))             # H = 0
    s = binding.Solver(p)
    r = s.kkt_solve(np.zeros(p.ns * p.N), np.zeros(p.n), np.ones(p.n), "fp64", check=False)
    assert r["status"] == 3
