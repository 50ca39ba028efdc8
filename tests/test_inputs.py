"""The seeded input recipe against the workloads it stands for (CPU).

The plants are the explicit-Euler heat equations of the paper's problem class
(Section V-A). On the plates the inputs are boundary temperatures, so a
uniform temperature with every input at the same value is a fixed point and
each row of [A B] sums to one; the rod has point actuators inside it and a
zero boundary at its ends. The sizes, weights, bounds and
initial-state distributions are the ones the five benchmark configurations
name (1-D ns = 50, nu = 5, N = 10; the 32 x 32 and 100 x 100 plates; the
uneven 256-instance batch).
"""
import numpy as np
import pytest

from paper_2209_13049_b300 import inputs


def _rows_of_AB_sum_to_one(p):
    A = p.dense("A") if p.ns <= 2048 else None
    s = (np.asarray(p.csr("A").sum(axis=1)).ravel() if A is None else A.sum(axis=1)) + p.B.sum(axis=1)
    return np.allclose(s, 1.0, rtol=0, atol=1e-14)


def test_heat1d_small_plant():
    p = inputs.heat1d(50, 5, 10)
    A = p.dense("A")
    assert (p.ns, p.nu, p.N, p.n) == (50, 5, 10, 50)
    assert np.allclose(np.diag(A), 0.8) and np.allclose(np.diag(A, 1), 0.1) and np.allclose(np.diag(A, -1), 0.1)
    assert np.count_nonzero(A) == 50 + 2 * 49
    rows, cols = np.nonzero(p.B)
    assert list(cols) == [0, 1, 2, 3, 4] and list(rows) == [5, 15, 25, 35, 45]
    assert np.allclose(p.B[rows, cols], 0.1)
    assert np.array_equal(p.dense("Q"), np.eye(50)) and np.array_equal(p.R, 0.1 * np.eye(5))
    assert np.all(p.xl == -1) and np.all(p.xu == 1) and np.all(p.ul == -2) and np.all(p.uu == 2)
    # the rod's ends lose heat to a zero boundary; the actuators are point sources inside it
    s = A.sum(axis=1)
    assert np.allclose(s[1:-1], 1.0) and np.isclose(s[0], 0.9) and np.isclose(s[-1], 0.9)


@pytest.mark.parametrize("g,nu", [(32, 10), (100, 20)])
def test_heat2d_plates(g, nu):
    p = inputs.heat2d(g, nu, 50)
    assert (p.ns, p.nu, p.N, p.n) == (g * g, nu, 50, 50 * nu)
    A = p.csr("A")
    assert np.allclose(A.diagonal(), 0.6)
    assert A.nnz == 5 * g * g - 4 * g                       # 5-point stencil, cut at the edges
    assert _rows_of_AB_sum_to_one(p)                        # boundary arcs carry the missing neighbours
    arcs = p.B.sum(axis=0) / 0.1                            # ghost nodes per arc
    assert arcs.sum() == pytest.approx(4 * g) and arcs.max() - arcs.min() <= 1 + 1e-9
    assert np.all(p.xl == 0) and np.all(p.xu == 1) and np.all(p.ul == -5) and np.all(p.uu == 5)


def test_initial_states():
    a, b = inputs.x0_uniform(50, 0), inputs.x0_uniform(50, 0)
    assert np.array_equal(a, b) and np.all(np.abs(a) <= 0.8) and not np.array_equal(a, inputs.x0_uniform(50, 1))
    f = inputs.x0_gaussians(32, 0)
    assert f.shape == (1024,) and np.all(f >= 0) and f.max() == pytest.approx(0.9, abs=1e-15)
    assert np.array_equal(f, inputs.x0_gaussians(32, 0)) and not np.array_equal(f, inputs.x0_gaussians(32, 1))
    grid = f.reshape(32, 32)                                # smooth: neighbours differ little
    assert np.max(np.abs(np.diff(grid, axis=0))) < 0.25 and np.max(np.abs(np.diff(grid, axis=1))) < 0.25


def test_uneven_batch_recipe():
    inst = inputs.batch_instances(256, 0)
    assert len(inst) == 256
    kinds = {p.kind for p, _ in inst}
    assert kinds == {"heat1d", "heat2d"}
    for p, x0 in inst:
        assert 2 <= p.nu <= 16 and 10 <= p.N <= 50 and 20 <= p.n <= 800 and x0.shape == (p.ns,)
        if p.kind == "heat1d":
            assert 200 <= p.ns <= 2000 and np.all(np.abs(x0) <= 0.8)
        else:
            assert 15 <= p.meta["g"] <= 44 and p.ns == p.meta["g"] ** 2 and np.all(x0 >= 0)
    again = inputs.batch_instances(256, 0)
    assert all(p.ns == q.ns and p.nu == q.nu and p.N == q.N and np.array_equal(x, y)
               for (p, x), (q, y) in zip(inst, again))
