"""Out-of-memory paths of the setup calls, injected on the host: with the
environment variable BMG_FAIL_ALLOC = k the library's k-th device or pinned
allocation fails as out of memory without reaching the driver.  For every k
up to the number of allocations a setup makes, the call returns BMG_ENOMEM,
leaves no device memory behind, and the library stays usable; nothing runs on
the GPU that could fault."""
import os

import numpy as np
import pytest
import torch

import workloads as w

pytestmark = pytest.mark.gpu

SLACK = 4 << 20        # bytes of device memory the driver may take for itself meanwhile


def free_bytes() -> int:
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def sweep_failures(bmg, make, limit=600):
    """Fail allocation k = 1, 2, ... of make() until it succeeds; returns the
    number of allocations make() needs."""
    make().close()                                   # modules loaded, tuners warm
    base = free_bytes()
    k = 1
    try:
        while True:
            os.environ["BMG_FAIL_ALLOC"] = str(k)
            try:
                obj = make()
            except bmg.BmgError as e:
                assert e.code == bmg.BMG_ENOMEM, str(e)
                k += 1
                assert k < limit
                continue
            break
    finally:
        os.environ.pop("BMG_FAIL_ALLOC", None)
    obj.close()
    assert free_bytes() >= base - SLACK
    return k - 1


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("precision,nbf", [("fp64", 0), ("fp32", 0), ("bf16", 2)])
def test_hierarchy_setup_out_of_memory(bmg, precision, nbf):
    """After every injected failure, a hierarchy set up without one still runs
    the oracle's iterates bit for bit (three cycles or refinement steps)."""
    from oracle import boxmg as bx
    from oracle import mixed as mx
    kind, planes, f = w.lognormal_problem(255, 2.0, 8.0, seed_k=4, seed_f=7)
    coef = dev(planes)
    count = sweep_failures(bmg, lambda: bmg.Hierarchy(kind, coef, precision=precision))
    assert count > 10
    levels = bx.setup(kind, planes)
    if precision == "fp64":
        want, _ = bx.solve(levels, f, tol=0.0, maxit=3)
    else:
        want, _ = mx.solve_ir(levels, mx.lower(levels, nbf), f, tol=0.0, maxit=3)
    h = bmg.Hierarchy(kind, coef, precision=precision)
    x, it, _, _ = h.solve(dev(f), tol=0.0, maxit=3)
    assert it == 3
    assert np.array_equal(x.cpu().numpy()[1:-1, 1:-1], want[1:-1, 1:-1])
    h.close()


def test_krylov_setup_out_of_memory(bmg):
    kind, planes, f = w.lognormal_problem(127, 2.0, 8.0, seed_k=4, seed_f=7)
    coef = dev(planes)
    assert sweep_failures(bmg, lambda: bmg.Hierarchy(kind, coef, precision="fp32", krylov="fcg")) > 10


def test_general_size_and_periodic_setup_out_of_memory(bmg):
    kind, planes, f = w.general_size_problem(100, 70)
    coef = dev(planes)
    assert sweep_failures(bmg, lambda: bmg.Hierarchy(kind, coef)) > 5
    kind, planes, f, px, py = w.periodic_problem(63, "x", std=1.0, corr_len=8.0)
    coefp = dev(planes)
    assert sweep_failures(bmg, lambda: bmg.Hierarchy(kind, coefp, periodic="x")) > 5


def test_batched_setups_out_of_memory(bmg):
    probs = [w.lognormal_problem(n, 1.0, 8.0, seed_k=20 + n, seed_f=21 + n) for n in (63, 127, 255)]
    coefs = [dev(p) for _, p, _ in probs]
    assert sweep_failures(bmg, lambda: bmg.Batch(9, coefs, precision="fp32")) > 5
    h = bmg.Hierarchy(9, coefs[2], precision="fp32")
    assert sweep_failures(bmg, lambda: bmg.Batch.from_hierarchy(h, 4)) > 3
    B = bmg.Batch.from_hierarchy(h, 2)
    rhs = [dev(w.rhs_uniform(255, 500 + q)) for q in range(2)]
    _, its, _, ok = B.solve(rhs, tol=1e-8, maxit=60)
    assert ok
    B.close()
    h.close()


def test_network_creation_out_of_memory(bmg):
    assert sweep_failures(bmg, lambda: bmg.Mlp()) >= 4
