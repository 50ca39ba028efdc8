"""Write the stored expected values used by the GPU parity tests.

Every value here comes from the oracle (oracle/) on the seeded inputs of
paper_2209_13049_b300.inputs; nothing comes from the CUDA path.  Run from the
repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2209_13049_b300 import inputs  # noqa: E402

OUT = os.path.dirname(os.path.abspath(__file__))


def solve_pair(p, x0, tag, store):
    r8 = oracle.ipm_solve(p, x0, tol=1e-8, want_trace=True)
    r12 = oracle.ipm_solve(p, x0, tol=1e-11)
    assert r8["status"] == 0 and r12["status"] == 0, (tag, r8["status"], r12["status"])
    store[f"{tag}_u8"] = r8["u"]
    store[f"{tag}_trace8"] = r8["trace"]
    store[f"{tag}_u12"] = r12["u"]
    store[f"{tag}_x0"] = x0
    print(tag, "iters", r8["stats"]["iters"], r12["stats"]["iters"], flush=True)


def main():
    store = {}
    for seed in range(4):
        p, x0 = inputs.config_1d_small(seed)
        solve_pair(p, x0, f"heat1d_50_s{seed}", store)
    np.savez_compressed(os.path.join(OUT, "heat1d_ns50_nu5_N10.npz"), **store)

    store = {}
    p, x0 = inputs.config_2d_32(0)
    solve_pair(p, x0, "heat2d_32_s0", store)
    np.savez_compressed(os.path.join(OUT, "heat2d_g32_nu10_N50.npz"), **store)

    # small uneven batch (same recipe as the 256-instance batch, smaller sizes)
    store = {}
    rng = np.random.default_rng(7)
    for k in range(6):
        nu = int(rng.integers(2, 7))
        N = int(rng.integers(4, 12))
        if k % 2 == 0:
            ns = int(rng.integers(40, 160))
            p = inputs.heat1d(ns, nu, N)
            x0 = inputs.x0_uniform(ns, 100 + k)
        else:
            g = int(rng.integers(6, 12))
            p = inputs.heat2d(g, nu, N)
            x0 = inputs.x0_gaussians(g, 100 + k)
        store[f"b{k}_dims"] = np.array([p.ns, p.nu, p.N, 0 if p.kind == "heat1d" else p.meta["g"]])
        solve_pair(p, x0, f"b{k}", store)
    np.savez_compressed(os.path.join(OUT, "batch_small.npz"), **store)


if __name__ == "__main__":
    main()
