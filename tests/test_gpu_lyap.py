"""The FP64 KKT matrix by Horner chains over the horizon against the SYRK
formation (child processes choose each with LQMPC_KKT64): the same matrix up
to rounding order, so the same FP64 interior-point iterates and the oracle's
optimum."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2209_13049_b300 import binding, build

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = os.path.join(ROOT, "tests", "golden")

CHILD = r"""
import json
import numpy as np
from paper_2209_13049_b300 import binding, inputs
p, x0 = inputs.config_2d_32(0)
s = binding.Solver(p)
u, st = s.solve(x0)
tr = s.get_trace()
print(json.dumps({"u": u.tolist(), "mu": tr[:, 0].tolist(), "iters": st["iters"], "status": st["status"],
                  "t_fp64": st["t_syrk_fp64_ms"], "n_fp64": st["syrk_fp64_launches"]}))
"""


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.load()


def _run(mode):
    env = dict(os.environ, LQMPC_KKT64=mode)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_recursion_matches_syrk_formation_and_oracle():
    a, b = _run("syrk"), _run("lyap")
    assert a["status"] == 0 and b["status"] == 0
    assert a["iters"] == b["iters"]
    np.testing.assert_allclose(b["mu"], a["mu"], rtol=1e-6)
    ua, ub = np.array(a["u"]), np.array(b["u"])
    assert np.max(np.abs(ua - ub)) / max(1.0, np.max(np.abs(ua))) <= 1e-8
    ref = np.load(os.path.join(GOLD, "heat2d_g32_nu10_N50.npz"))["heat2d_32_s0_u8"]
    assert np.max(np.abs(ub - ref)) / max(1.0, np.max(np.abs(ref))) <= 1e-8
    # the recursion needs about a third of the SYRK's FP64 operations here
    assert b["t_fp64"] / b["n_fp64"] < a["t_fp64"] / a["n_fp64"]
