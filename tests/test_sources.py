"""Source-level properties of the CUDA path that no GPU run can show.

Programmatic dependent launch: every kernel launched through lq_pdl (with
programmatic stream serialisation) must make griddepcontrol.wait (pdl_wait)
its first statement, before any memory access; otherwise it could read
what the kernel before it has not finished writing, and a kernel that
returned early without the wait would let the one after it run ahead too.
"""
import glob
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", "paper_2209_13049_b300", "csrc")


def _sources():
    return {f: open(f).read() for f in glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))}


def _first_statement(src, name):
    """First statement of each __global__ definition of `name` in src."""
    out = []
    for m in re.finditer(r"__global__[^;{]*?\b" + re.escape(name) + r"\s*\(", src):
        i, depth = m.end() - 1, 0
        while True:
            if src[i] == "(":
                depth += 1
            elif src[i] == ")":
                depth -= 1
                if depth == 0:
                    break
            i += 1
        brace = src.index("{", i)
        out.append(src[brace + 1:].lstrip().split("\n", 1)[0])
    return out


def test_every_programmatic_launch_waits_first():
    srcs = _sources()
    launched = set()
    for s in srcs.values():
        launched.update(re.findall(r"lq_pdl\(\s*([A-Za-z_]\w*)", s))
    launched.discard("void")
    assert len(launched) > 40
    for name in sorted(launched):
        firsts = [f for s in srcs.values() for f in _first_statement(s, name)]
        assert firsts, name
        for f in firsts:
            assert f.startswith("pdl_wait();"), (name, f)


def test_launches_go_through_the_programmatic_launcher():
    """No kernel launch of the solver path bypasses lq_pdl inside LQ_LAUNCH."""
    for path, s in _sources().items():
        for m in re.finditer(r"LQ_LAUNCH\((.*?)\);\n", s, re.S):
            body = m.group(1)
            assert "<<<" not in body, (os.path.basename(path), body[:80])
