"""The FP32 Cholesky factor of the condensed KKT matrix (Eq. 7, M = L L') and
its inverse (the preconditioner of the mixed-precision solves) against the
FP64 oracle matrix, over sizes spanning one to thirty-three 32-wide block
columns with ragged ends (a single instance of n <= 544 takes the dataflow
factorisation).

Tolerances.  The factor is checked by its backward error, element-wise:
|L L' - M| <= 8 (n + 2) 2^-24 (|L| |L'|) + the FP32-accurate formation error
of M (4 2^-24 (sqrt(K) + 2) of the absolute sum, K = ns N terms).  The
inverse is checked by the conjugate gradients it preconditions: started from
L^-T L^-1 b, FP64 products with M must reach a 2e-10 relative residual in a
few steps (an FP32-accurate inverse contracts the error by about
cond(M) 2^-24 per step; a wrong block of it would not).

Single instances of 544 < n <= 1024 take the queued dataflow kernel (block
columns as tasks from a ticket counter, factor tasks before inverse tasks);
the `queued` cases force it on the small sizes as well (LQMPC_POTRF).  Past
n = 1024 the grid-cooperative kernel factors (the n = 1056 case).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2209_13049_b300 import binding, build, inputs

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24

SIZES = [
    ("n20_one_ragged_block", lambda: inputs.heat1d(10, 2, 10)),
    ("n161_ragged", lambda: inputs.heat2d(10, 7, 23)),
    ("n500_16_blocks_ragged", lambda: inputs.heat1d(40, 10, 50)),
    ("n517_17_blocks_ragged5", lambda: inputs.heat1d(30, 11, 47)),
    ("n544_17_full_blocks", lambda: inputs.heat1d(30, 16, 34)),
    ("n800_25_full_blocks", lambda: inputs.heat1d(40, 16, 50)),
    ("n1000_32_blocks_ragged8", lambda: inputs.heat1d(30, 20, 50)),
    ("n1024_32_full_blocks", lambda: inputs.heat1d(30, 16, 64)),
    ("n1056_33_blocks_cooperative", lambda: inputs.heat1d(30, 16, 66)),   # past the queued kernel's n <= 1024
    ("n161_ragged_queued", lambda: inputs.heat2d(10, 7, 23), "queued"),
    ("n500_16_blocks_ragged_queued", lambda: inputs.heat1d(40, 10, 50), "queued"),
    ("n517_17_blocks_ragged5_queued", lambda: inputs.heat1d(30, 11, 47), "queued"),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.load()


@pytest.fixture(scope="module", params=SIZES, ids=[c[0] for c in SIZES])
def case(request):
    p = request.param[1]()
    variant = request.param[2] if len(request.param) > 2 else None
    if variant:
        os.environ["LQMPC_POTRF"] = variant
    s = binding.Solver(p)
    Gam, _, H, _ = oracle.condensed(p, np.zeros(p.ns))
    rng = np.random.default_rng(11)
    sigx = 10.0 ** rng.uniform(-1, 1, p.ns * p.N)
    sigu = 10.0 ** rng.uniform(-1, 1, p.n)
    M = oracle.kkt_matrix(p, sigx, sigu, Gam, H)
    absm = np.abs(H) + np.abs(Gam).T @ (sigx[:, None] * np.abs(Gam)) + np.diag(sigu)
    yield p, s, sigx, sigu, M, absm
    os.environ.pop("LQMPC_POTRF", None)


def test_fp32_factor_backward_error(case):
    p, s, sigx, sigu, M, absm = case
    b = np.random.default_rng(12).standard_normal(p.n)
    r = s.kkt_solve(sigx, sigu, b, "fp32", want_L=True)
    L = np.tril(r["L"])
    assert np.all(np.isfinite(L)) and np.all(np.diag(L) > 0)
    err = np.abs(L @ L.T - M)
    bound = 8 * (p.n + 2) * U32 * (np.abs(L) @ np.abs(L).T) + 4 * U32 * (np.sqrt(p.ns * p.N) + 2) * absm
    assert np.all(err <= bound), float((err / bound).max())


U64 = 2.0 ** -53


def test_fp64_factor_backward_error(case):
    """FP64 Cholesky of M (grid-cooperative kernel: four-warp diagonal factor
    with the third-order pivot, unit-triangular inverse of the diagonal block,
    quadrant updates): backward error of L L' within the FP64 rounding bound
    of the factorisation plus the FP64 formation of M."""
    p, s, sigx, sigu, M, absm = case
    b = np.random.default_rng(14).standard_normal(p.n)
    r = s.kkt_solve(sigx, sigu, b, "fp64", want_L=True)
    L = np.tril(r["L"])
    assert np.all(np.isfinite(L)) and np.all(np.diag(L) > 0)
    err = np.abs(L @ L.T - M)
    bound = 8 * (p.n + 2) * U64 * (np.abs(L) @ np.abs(L).T) + 4 * U64 * (np.sqrt(p.ns * p.N) + 2) * absm
    assert np.all(err <= bound), float((err / bound).max())
    x_ref = np.linalg.solve(M, b)
    # forward error <= cond(M) x backward error of the factor and the formation
    fwd = 10 * np.linalg.cond(M) * (p.n + np.sqrt(p.ns * p.N) + 2) * U64 * np.max(np.abs(x_ref))
    assert np.max(np.abs(r["x"] - x_ref)) <= fwd


def test_fp32_inverse_preconditions_in_few_steps(case):
    p, s, sigx, sigu, M, _ = case
    b = np.random.default_rng(13).standard_normal(p.n)
    r = s.kkt_solve(sigx, sigu, b, "fp32")
    res = np.max(np.abs(b - M @ r["x"])) / np.max(np.abs(b))
    assert res <= 2e-10, res
    assert r["refine_steps"] <= 8, r["refine_steps"]


@pytest.mark.parametrize("spread", [1, 6])
def test_two_level_preconditioner_converges_where_fp32_struggles(case, spread):
    """LQMPC_FP32X2: the FP32 factor L1 of M, then the FP32 factor of
    L1^-1 M L1^-T formed from E = M - L1 L1' (float-float), combined into
    one explicit inverse.  With Sigma spread over 2 * spread decades either
    side of one the solve must reach the same 2e-10 residual, in no more
    conjugate-gradient steps than the FP32 factor alone needs (and in few
    steps outright).

    The residual bar: the library stops at ||b - M x||_inf <= 1e-10 ||b||_inf
    as its own FP64-accurate products evaluate it; recomputed here from the
    oracle's M, the two evaluations differ by their rounding, about
    (sqrt(ns N) + sqrt(n) + 2) 2^-53 || |M| |x| ||_inf under the usual
    random-rounding model (ns N terms in each entry of M, n in each row of
    the product).  With Sigma over 12 decades || |M| |x| || is up to 1e5
    ||b||, so that floor reaches the 1e-10 level at n ~ 1000."""
    p, s, _, _, _, _ = case
    rng = np.random.default_rng(21)
    sigx = 10.0 ** rng.uniform(-spread, spread, p.ns * p.N)
    sigu = 10.0 ** rng.uniform(-spread, spread, p.n) + 1e-3
    Gam, _, H, _ = oracle.condensed(p, np.zeros(p.ns))
    M = oracle.kkt_matrix(p, sigx, sigu, Gam, H)
    b = rng.standard_normal(p.n)
    r2 = s.kkt_solve(sigx, sigu, b, "fp32x2", check=False)
    assert r2["status"] == 0, r2["status"]
    absm = np.abs(H) + np.abs(Gam).T @ (sigx[:, None] * np.abs(Gam)) + np.diag(sigu)
    floor = (np.sqrt(p.ns * p.N) + np.sqrt(p.n) + 2) * U64 * np.max(absm @ np.abs(r2["x"]))
    res = np.max(np.abs(b - M @ r2["x"])) / np.max(np.abs(b))
    assert res <= 2e-10 + floor / np.max(np.abs(b)), (res, floor / np.max(np.abs(b)))
    assert r2["refine_steps"] <= 6, r2["refine_steps"]
    r1 = s.kkt_solve(sigx, sigu, b, "fp32", check=False)
    if r1["status"] == 0:
        assert r2["refine_steps"] <= r1["refine_steps"], (r2["refine_steps"], r1["refine_steps"])
