"""A C program calling the library directly (no Python between it and the
ABI) gets the oracle's memberships and modularity."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def parse_c_output(text: str):
    """(static membership, DF membership, Q) from the example's printout."""
    lines = [ln for ln in text.splitlines() if ln.strip()]
    static = [int(x) for x in lines[0].split(":")[1].split()]
    after, rest = lines[1].split(":")[1].split("Q =")
    q = float(rest.split()[0])
    return static, [int(x) for x in after.split()], q


def parse_step_output(text: str):
    """(membership, Q) after the example's dfl_step call."""
    line = [ln for ln in text.splitlines() if ln.startswith("after step:")][0]
    memb, rest = line.split(":")[1].split("Q =")
    return [int(x) for x in memb.split()], float(rest.split()[0])


def test_parse_step_output():
    assert parse_step_output("static: 0\nafter DF: 0  Q = 0.1  passes = 1  affected = 0\n"
                             "after step: 0 0 0 1 1 1  Q = 0.250000\n") == ([0, 0, 0, 1, 1, 1], 0.25)


def test_parse_c_output():
    s, d, q = parse_c_output("static: 0 0 0 1 1 1\nafter DF: 0 0 0 1 1 1  Q = 0.468750  passes = 1"
                             "  affected = 0\n")
    assert s == d == [0, 0, 0, 1, 1, 1] and q == 0.46875


@pytest.mark.gpu
def test_c_caller_matches_oracle(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    import oracle
    import paper_2404_19634_gb300 as dfl
    lib = dfl.build()
    oracle.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "c_api_example")
    subprocess.check_call([cc, "-std=c99", "-O2", "-I", os.path.join(ROOT, "include"),
                           os.path.join(HERE, "c_api_example.c"), "-o", exe, "-L", libdir, "-ldfl",
                           "-Wl,-rpath," + libdir])
    run = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stdout + run.stderr
    static, after, q = parse_c_output(run.stdout)
    # the same graph and batch through the oracle
    e = [(0, 1), (0, 2), (1, 2), (3, 4), (3, 5), (4, 5), (2, 3)]
    g = synth.EdgeList(6, np.array([a for a, _ in e], np.uint32), np.array([b for _, b in e], np.uint32),
                       np.ones(len(e), np.uint32))
    off, idx, w = synth.to_csr(g)
    o = oracle.Oracle(6, off, idx, w)
    o.static()
    assert static == list(o.membership())
    assert o.apply_batch([(2, 3, 0)], [(0, 1, 2)]) == 0
    o.update(2)
    assert after == list(o.membership())
    assert abs(q - o.modularity()[0]) <= 5e-7  # printed with six decimals
    # dfl_step = apply + DF update
    stepped, q2 = parse_step_output(run.stdout)
    assert o.apply_batch([(4, 5, 0)], [(2, 3, 1)]) == 0
    o.update(2)
    assert stepped == list(o.membership())
    assert abs(q2 - o.modularity()[0]) <= 1e-11  # printed with twelve decimals
