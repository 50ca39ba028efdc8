"""The allocation-free KKT formation entry point (a library facility with no
counterpart in the paper) against the context's own FP64 formation
(lqmpc_form_kkt), on two calls in a row.  Collected last on purpose: it must
pass alone and after every other test has used the library.

Tolerance: both sides sum the same FP64 products over K = ns*N terms in
different orders (split counts differ); Gamma, Sigma and H are entrywise
nonnegative for the heat plants, so every entry is a sum without
cancellation and the difference is bounded by 2 K eps |M| entrywise.
"""
import numpy as np
import pytest

from paper_2209_13049_b300 import binding, build, inputs

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.load()


def _sigmas(p, seed):
    rng = np.random.default_rng(seed)
    sigx = 10.0 ** rng.uniform(-4.0, 4.0, size=p.ns * p.N)
    sigu = 10.0 ** rng.uniform(-4.0, 2.0, size=p.n)
    return sigx, sigu


@pytest.mark.parametrize("plant", ["heat2d_g10_nu7_N23", "heat2d_g32_nu10_N50"])
def test_noalloc_matches_form_kkt_two_calls_in_a_row(plant):
    import torch
    p = inputs.heat2d(10, 7, 23) if plant.startswith("heat2d_g10") else inputs.heat2d(32, 10, 50)
    s = binding.Solver(p)
    K = p.ns * p.N
    sig = [_sigmas(p, 40 + c) for c in range(2)]
    refs = [s.form_kkt(sx, su, "fp64") for sx, su in sig]
    outs = []
    for sx, su in sig:      # two calls back to back; the second finds the first's partials in the scratch
        M = torch.full((p.n * p.n,), float("nan"), dtype=torch.float64, device="cuda")
        s.form_kkt_noalloc(torch.tensor(sx, device="cuda"), torch.tensor(su, device="cuda"), M)
        outs.append(M)
    torch.cuda.synchronize()
    for M, ref in zip(outs, refs):
        got = M.cpu().numpy().reshape(p.n, p.n, order="F")
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - ref) <= 2 * K * EPS * np.abs(ref) + 1e-300)
        assert np.array_equal(got, got.T)


def test_noalloc_rejects_oversize_and_bad_pointers():
    import torch
    s = binding.Solver(inputs.heat1d(4, 40, 50))         # n = 2000 > 1984
    sx = torch.zeros(4 * 50, dtype=torch.float64, device="cuda")
    su = torch.zeros(2000, dtype=torch.float64, device="cuda")
    M = torch.zeros(2000 * 2000, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.LqmpcError) as e:
        s.form_kkt_noalloc(sx, su, M)
    assert e.value.code == 9
    lib = binding.load()
    assert lib.lqmpc_form_kkt_noalloc(s.h, None, su.data_ptr(), M.data_ptr()) == 1
    assert lib.lqmpc_form_kkt_noalloc(s.h, sx.data_ptr() + 4, su.data_ptr(), M.data_ptr()) == 1
