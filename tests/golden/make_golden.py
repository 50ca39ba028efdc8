"""Write the stored expected values used by the GPU parity tests.

Every value here comes from the oracle (oracle/) on the seeded inputs of
paper_2209_13049_b300.inputs; nothing comes from the CUDA path.  Run from the
repository root:

    python tests/golden/make_golden.py [group ...]

Groups (all when none is named):
  small   1-D ns=50 plant (four seeds), 2-D 32x32 plant (seed 0), a small uneven batch
  c3      2-D 100x100 plant (ns=10000, nu=20, N=50), seed 0 (about an hour per solve)
  batch   eight instances sampled from the uneven 256-instance batch
  warm    four held-out initial states of the 32x32 warm-start workload
  cube    the paper's 3-D cube plant (Table I) on small grids and horizons
Solves of one group run in parallel worker processes (spawned, one solve each).
"""
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2209_13049_b300 import inputs  # noqa: E402

OUT = os.path.dirname(os.path.abspath(__file__))
# instances of inputs.batch_instances(256, 0) with stored oracle solutions
BATCH_SAMPLE = (0, 37, 74, 111, 148, 185, 222, 255)
# held-out warm-start initial states: x0_gaussians(32, WARM_SEED0 + k)
WARM_SEED0 = 10 ** 6
WARM_SAMPLE = 4


def _solve(job):
    """One oracle solve: job = (tag, plant, x0, tol, want_trace[, u_init])."""
    tag, p, x0, tol, want_trace = job[:5]
    u_init = job[5] if len(job) > 5 else None
    t0 = time.time()
    r = oracle.ipm_solve(p, x0, tol=tol, want_trace=want_trace, max_iter=200, u_init=u_init)
    assert r["status"] == 0, (tag, tol, r["status"])
    print(f"{tag} tol={tol:g} iters={r['stats']['iters']} {time.time() - t0:.1f}s", flush=True)
    return tag, tol, r["u"], r.get("trace")


def _pair_jobs(p, x0, tag, u_init=None):
    return [(tag, p, x0, 1e-8, True, u_init), (tag, p, x0, 1e-11, False, u_init)]


def _run(jobs, store, procs):
    if procs > 1:
        with mp.get_context("spawn").Pool(min(procs, len(jobs))) as pool:
            results = pool.map(_solve, jobs, chunksize=1)
    else:
        results = [_solve(j) for j in jobs]
    x0s = {j[0]: j[2] for j in jobs}
    for tag, tol, u, tr in results:
        if tol == 1e-8:
            store[f"{tag}_u8"] = u
            store[f"{tag}_trace8"] = tr
        else:
            store[f"{tag}_u12"] = u
        store[f"{tag}_x0"] = x0s[tag]


def group_small(procs):
    store = {}
    jobs = []
    for seed in range(4):
        p, x0 = inputs.config_1d_small(seed)
        jobs += _pair_jobs(p, x0, f"heat1d_50_s{seed}")
    _run(jobs, store, procs)
    np.savez_compressed(os.path.join(OUT, "heat1d_ns50_nu5_N10.npz"), **store)

    store = {}
    p, x0 = inputs.config_2d_32(0)
    _run(_pair_jobs(p, x0, "heat2d_32_s0"), store, procs)
    np.savez_compressed(os.path.join(OUT, "heat2d_g32_nu10_N50.npz"), **store)

    # small uneven batch (same recipe as the 256-instance batch, smaller sizes)
    store = {}
    jobs = []
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
        jobs += _pair_jobs(p, x0, f"b{k}")
    _run(jobs, store, procs)
    np.savez_compressed(os.path.join(OUT, "batch_small.npz"), **store)


def group_c3(procs):
    store = {}
    p, x0 = inputs.config_2d_100(0)
    _run(_pair_jobs(p, x0, "heat2d_100_s0"), store, procs)
    np.savez_compressed(os.path.join(OUT, "heat2d_g100_nu20_N50.npz"), **store)


def group_batch(procs):
    inst = inputs.batch_instances(256, 0)
    store = {"sample": np.array(BATCH_SAMPLE)}
    jobs = []
    for k in BATCH_SAMPLE:
        p, x0 = inst[k]
        jobs += _pair_jobs(p, x0, f"i{k}")
    _run(jobs, store, procs)
    np.savez_compressed(os.path.join(OUT, "batch256_sample.npz"), **store)


def group_warm(procs):
    """Cold solves of the held-out x0 (w{k}) and warm-started ones (v{k}) from
    the guess u_init = the oracle's 1e-8 solution for training x0 seed k (an
    imperfect guess, like a learned one, that comes from the oracle)."""
    store = {"seed0": np.array(WARM_SEED0)}
    p = inputs.heat2d(32, 10, 50)
    guesses = []
    for k in range(WARM_SAMPLE):
        guesses.append(oracle.ipm_solve(p, inputs.x0_gaussians(32, k), tol=1e-8)["u"])
        store[f"v{k}_guess"] = guesses[-1]
    jobs = []
    for k in range(WARM_SAMPLE):
        x0 = inputs.x0_gaussians(32, WARM_SEED0 + k)
        jobs += _pair_jobs(p, x0, f"w{k}")
        jobs += _pair_jobs(p, x0, f"v{k}", u_init=guesses[k])
    _run(jobs, store, procs)
    np.savez_compressed(os.path.join(OUT, "warm_heldout_g32.npz"), **store)


# (grid points per dimension, horizon) of the stored cube solutions
CUBE_CASES = ((4, 50), (5, 50), (6, 50), (4, 150), (4, 250), (4, 500))


def group_cube(procs):
    store = {"cases": np.array(CUBE_CASES)}
    jobs = []
    for g, T in CUBE_CASES:
        jobs += _pair_jobs(inputs.heat3d_cube(g, T), inputs.x0_cube(g), f"g{g}_T{T}")
    _run(jobs, store, procs)
    np.savez_compressed(os.path.join(OUT, "cube_table1.npz"), **store)


GROUPS = {"small": group_small, "c3": group_c3, "batch": group_batch, "warm": group_warm, "cube": group_cube}


def main(argv):
    procs = int(os.environ.get("GOLDEN_PROCS", "4"))
    for name in (argv or list(GROUPS)):
        GROUPS[name](procs)


if __name__ == "__main__":
    main(sys.argv[1:])
