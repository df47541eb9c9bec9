"""The debug library (libbmg_debug.so: the same sources compiled with
-DBMG_DEBUG), whose kernels check the index of each global store and the
source range of each row copy against the extent of the array it addresses.

With exact extents, every path the checks cover (FP64, FP32 and BF16 cycles
with their row, one-pass, two-pass and tail kernels, FCG, line relaxation in
both directions, periodic sides, general sizes, batches) runs without a
recorded failure and computes the oracle's bits, so the checks change nothing.
With the test hook that shrinks every checked extent by two rows, the accesses
there are skipped and recorded instead of leaving any array, bmg_solve
returns BMG_EBOUNDS naming the kernel family, and after the hook is reset the
same library solves exactly again.  Each part runs in a child process that
loads the debug library (BMG_LIB=debug)."""
import importlib.util
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def debug_lib():
    spec = importlib.util.spec_from_file_location("_bmg_build", os.path.join(ROOT, "paper_2502_05279_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build(debug=True)


def run_child(code: str) -> dict:
    env = dict(os.environ, BMG_LIB="debug")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-3000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


EXACT = r"""
import json, numpy as np, torch
import workloads as w
import paper_2502_05279_gb300 as bmg
from oracle import boxmg as bx, mixed as mx, periodic as pr
assert bmg.debug_build() and bmg.library_path.endswith("libbmg_debug.so")
dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
inner = lambda a: np.asarray(a)[..., 1:-1, 1:-1]
out = {}
kind, planes, f = w.lognormal_problem(255, 2.0, 8.0, seed_k=4, seed_f=7)
levels = bx.setup(kind, planes, arith="fused")
want, _ = bx.solve(levels, f, tol=0.0, maxit=3)
for sm in ("auto", "rows", "tile0", "tile2"):
    h = bmg.Hierarchy(kind, dev(planes), arith="fused", smoother=sm)
    x, it, _, _ = h.solve(dev(f), tol=0.0, maxit=3)
    out["fp64_" + sm] = [bool(np.array_equal(inner(x.cpu().numpy()), inner(want))), bmg.debug_take()]
    h.close()
for prec, nbf, sm in (("fp32", 0, "auto"), ("fp32", 0, "pair0"), ("bf16", 2, "tile0")):
    lv = bx.setup(kind, planes, arith="fused")
    want32, _ = mx.solve_ir(lv, mx.lower(lv, nbf), f, tol=0.0, maxit=3)
    h = bmg.Hierarchy(kind, dev(planes), precision=prec, arith="fused", smoother=sm)
    x, it, _, _ = h.solve(dev(f), tol=0.0, maxit=3)
    out[prec + "_" + sm] = [bool(np.array_equal(inner(x.cpu().numpy()), inner(want32))), bmg.debug_take()]
    h.close()
for prec in ("fp64", "fp32"):
    h = bmg.Hierarchy(kind, dev(planes), precision=prec, krylov="fcg")
    x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=100)
    out["fcg_" + prec] = [bool(ok), bmg.debug_take()]
    h.close()
ka, pa, fa = 5, w.anisotropic5(127, 1e-3), w.rhs_uniform(127, 5)
for sm in ("line", "yline", "xyline"):
    lv = bx.setup(ka, pa, smoother=sm)
    wl, _ = bx.solve(lv, fa, tol=0.0, maxit=3)
    h = bmg.Hierarchy(ka, dev(pa[:3]), smoother=sm)
    x, it, _, _ = h.solve(dev(fa), tol=0.0, maxit=3)
    out["lines_" + sm] = [bool(np.array_equal(inner(x.cpu().numpy()), inner(wl))), bmg.debug_take()]
    h.close()
kp, pp, fp, px, py = w.periodic_problem(255, "x", std=2.0, corr_len=8.0, seed_k=52, seed_f=53)
lv = pr.setup(kp, pp, px, py, arith="fused")
wp = np.zeros_like(fp)
for _ in range(2):
    pr.vcycle(lv, 0, wp, fp)
for sm in ("tile", "rows"):
    h = bmg.Hierarchy(kp, dev(pp), periodic="x", arith="fused", smoother=sm)
    x, it, _, _ = h.solve(dev(fp), tol=0.0, maxit=2)
    out["periodic_" + sm] = [bool(np.array_equal(inner(x.cpu().numpy()), inner(wp))), bmg.debug_take()]
    h.close()
kg, pg, fg = w.general_size_problem(100, 70)
h = bmg.Hierarchy(kg, dev(pg))
x, it, rr, ok = h.solve(dev(fg), tol=1e-10, maxit=100)
out["general"] = [bool(ok), bmg.debug_take()]
h.close()
probs = [w.lognormal_problem(n, 1.0, 8.0, seed_k=20 + n, seed_f=21 + n) for n in (63, 127, 255)]
B = bmg.Batch(9, [dev(p) for _, p, _ in probs], precision="fp32")
_, its, _, ok = B.solve([dev(q) for _, _, q in probs], tol=1e-8, maxit=60)
out["batched"] = [bool(ok), bmg.debug_take()]
B.close()
print(json.dumps(out))
"""


def test_exact_extents_record_nothing_and_keep_the_bits(debug_lib):
    got = run_child(EXACT)
    assert len(got) == 16, got
    for name, (exact, record) in got.items():
        assert exact, name
        assert record is None, (name, record)


SHRUNK = r"""
import json, numpy as np, torch
import workloads as w
import paper_2502_05279_gb300 as bmg
from oracle import boxmg as bx
dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
inner = lambda a: np.asarray(a)[..., 1:-1, 1:-1]
n = 127
kind, planes, f = w.lognormal_problem(n, 2.0, 8.0, seed_k=4, seed_f=7)
want, _ = bx.solve(bx.setup(kind, planes), f, tol=0.0, maxit=2)
out = {}
for prec in ("fp64", "fp32"):
    h = bmg.Hierarchy(kind, dev(planes), precision=prec)
    bmg.debug_shrink(2 * (n + 2))                 # the last two rows of every array count as outside
    try:
        h.solve(dev(f), tol=0.0, maxit=2)
        code, msg = 0, ""
    except bmg.BmgError as e:
        code, msg = e.code, str(e)
    rec = bmg.debug_take()
    bmg.debug_shrink(0)
    out[prec] = [code, msg, rec, bmg.debug_take()]
    h.close()
h = bmg.Hierarchy(kind, dev(planes))              # the library and the context are still usable
x, it, _, _ = h.solve(dev(f), tol=0.0, maxit=2)
out["after"] = [bool(np.array_equal(inner(x.cpu().numpy()), inner(want))), bmg.debug_take()]
h.close()
print(json.dumps(out))
"""


def test_shrunk_extents_are_caught_and_skipped(debug_lib):
    got = run_child(SHRUNK)
    n = 127
    for prec in ("fp64", "fp32"):
        code, msg, rec, again = got[prec]
        assert code == -8 and "debug bounds check failed" in msg, (prec, code, msg)
        site, index, extent = rec
        assert site != "none" and site != "unknown"
        assert extent == (n + 2) ** 2 - 2 * (n + 2) or extent < (n + 2) ** 2, rec
        assert index >= extent or index < 0, rec
        assert again is None                      # taken records are cleared
    exact, record = got["after"]
    assert exact and record is None


FULL = r"""
import hashlib, json, sys, numpy as np, torch
import workloads as w
import paper_2502_05279_gb300 as bmg
kind, planes, f = w.lognormal_problem(8191, 2.0, 32.0, seed_k=4, seed_f=7)
coef, rhs = torch.from_numpy(planes).cuda(), torch.from_numpy(f).cuda()
del planes
out = {"debug": bmg.debug_build()}
for prec in ("fp64", "fp32", "bf16"):
    h = bmg.Hierarchy(kind, coef, precision=prec, arith="fused")
    x, it, _, _ = h.solve(rhs, tol=0.0, maxit=2)
    out[prec] = [hashlib.sha256(x.cpu().numpy().tobytes()).hexdigest(), bmg.debug_take()]
    h.close()
    del x
    torch.cuda.empty_cache()
print(json.dumps(out))
"""


def test_full_size_workload_records_nothing_and_matches_release(debug_lib):
    """The 8191^2 log-normal workload (two cycles or refinement steps in each
    precision, the launch configuration of the bench): the debug library
    records no bounds failure and returns the release library's bits (the
    release library is compared with the oracle at this size elsewhere)."""
    dbg = run_child(FULL)
    env = {k: v for k, v in os.environ.items() if k != "BMG_LIB"}
    out = subprocess.run([sys.executable, "-c", FULL], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=900)
    assert out.returncode == 0, out.stderr[-3000:]
    rel = json.loads(out.stdout.strip().splitlines()[-1])
    assert dbg["debug"] and not rel["debug"]
    for prec in ("fp64", "fp32", "bf16"):
        assert dbg[prec][1] is None, (prec, dbg[prec][1])
        assert dbg[prec][0] == rel[prec][0], prec
