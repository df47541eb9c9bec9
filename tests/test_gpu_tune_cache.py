"""The autotuner's record file (BMG_TUNE_CACHE): a process that finds its
decisions there makes the same choices as the process that timed them,
without timing (fewer launches during setup), and solves to the same bits;
records with out-of-range values are ignored.  Each setup runs in a fresh
process, so the in-process caches start empty."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import hashlib, json, sys, torch
import workloads as w
import paper_2502_05279_gb300 as bmg
kind, planes, f = w.lognormal_problem(255, 2.0, 8.0, seed_k=4, seed_f=7)
h = bmg.Hierarchy(kind, torch.from_numpy(planes).cuda(), precision="fp32", arith="fused")
setup_launches = h.launch_count
x, it, _, _ = h.solve(torch.from_numpy(f).cuda(), tol=0.0, maxit=3)
coefs = [torch.from_numpy(w.lognormal_problem(n, 1.0, 8.0, seed_k=20 + n, seed_f=21 + n)[1]).cuda() for n in (127, 255)]
B = bmg.Batch(9, coefs, precision="fp32")
batch = []
while True:
    try:
        batch.append(B.tuned_cluster(len(batch)))
    except bmg.BmgError:
        break
print(json.dumps({"clusters": [h.tuned_cluster(l) for l in range(h.num_levels)],
                  "pairs": [h.tuned_pair(l) for l in range(h.num_levels)],
                  "batch": batch,
                  "setup_launches": setup_launches,
                  "x": hashlib.sha256(x.cpu().numpy().tobytes()).hexdigest()}))
"""


def run_child(cache):
    env = dict(os.environ, BMG_TUNE_CACHE=cache)
    out = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_recorded_decisions_are_reused(tmp_path):
    cache = str(tmp_path / "tune.txt")
    first = run_child(cache)
    lines = open(cache).read().splitlines()
    assert any(" rows:" in ln for ln in lines) and any(" tile:" in ln for ln in lines)
    assert any(" group:" in ln for ln in lines)
    second = run_child(cache)
    assert second["clusters"] == first["clusters"] and second["pairs"] == first["pairs"]
    assert second["batch"] == first["batch"]
    assert second["x"] == first["x"]
    assert second["setup_launches"] < first["setup_launches"]     # nothing timed
    assert open(cache).read().splitlines() == lines                # nothing new recorded


def test_out_of_range_records_are_ignored(tmp_path):
    cache = str(tmp_path / "tune.txt")
    first = run_child(cache)
    bad = []
    for ln in open(cache).read().splitlines():
        dev, key, count, *vals = ln.split()
        bad.append(" ".join([dev, key, count] + ["99"] * int(count) + [vals[-1]]))
    with open(cache, "w") as fp:
        fp.write("\n".join(bad) + "\nnot a record\n")
    again = run_child(cache)
    assert again["x"] == first["x"]
    # everything was timed again and recorded afresh, with in-range values
    fresh = open(cache).read().splitlines()[len(bad) + 1:]
    assert any(" rows:" in ln for ln in fresh) and any(" group:" in ln for ln in fresh)
    assert all("99" not in ln.split()[3:-1] for ln in fresh)
