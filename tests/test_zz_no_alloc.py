"""The allocation-free residual-norm entry point (bmg_residual_noalloc), for
callers that cannot let the library allocate device memory, gives what the
allocating entry point (bmg_residual) gives, bit for bit, and what the oracle
gives (the residual bit for bit, the norm to the stated 1e-14 and bit for bit
in the device's summation order).  Two calls in a row, the second on a
smaller grid, so a partial sum left in the shared static scratch by the first
call would show up in the second.  The property the entry point exists for is
checked too: the device's default memory pool, which bmg_residual allocates
its scratch from, sees no allocation during the call.  This file is collected
last."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as w
from oracle import boxmg as bx
from reduction_order import device_norm

pytestmark = pytest.mark.gpu

CU_MEMPOOL_ATTR_USED_MEM_CURRENT = 7    # cuda.h, CUmemPool_attribute
CU_MEMPOOL_ATTR_USED_MEM_HIGH = 8


class DefaultPool:
    """The current device's default stream-ordered pool through the driver
    API: its high-water mark of memory in use, which can be reset to zero."""

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        assert self.cu.cuInit(0) == 0
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, CU_MEMPOOL_ATTR_USED_MEM_HIGH, ctypes.byref(zero)) == 0

    def _get(self, attr) -> int:
        v = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def high(self) -> int:
        return self._get(CU_MEMPOOL_ATTR_USED_MEM_HIGH)

    def current(self) -> int:
        return self._get(CU_MEMPOOL_ATTR_USED_MEM_CURRENT)


def noalloc_fn(bmg):
    fn = bmg.lib.bmg_residual_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    return fn


def test_noalloc_matches_allocating_entry_point_twice(bmg):
    fn = noalloc_fn(bmg)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    pool = DefaultPool()
    cases = [w.binary_contrast_problem(2047, 16, seed_k=2, seed_f=3), w.lognormal_problem(63, 2.0, 8.0, seed_k=4, seed_f=7)]
    for kind, planes, f in cases:
        n = planes.shape[-1] - 2
        coef = torch.from_numpy(planes).cuda()
        rhs = torch.from_numpy(f).cuda()
        xh = w.rhs_uniform(n, 123)
        x = torch.from_numpy(xh).cuda()
        torch.cuda.synchronize()
        in_use = pool.current()
        pool.reset_high()
        r_ref, norm_ref = bmg.residual(kind, coef, x, rhs)
        torch.cuda.synchronize()
        assert pool.high() > in_use         # the allocating entry point draws from the pool: the check sees it
        r = torch.full_like(rhs, np.nan)
        nrm = ctypes.c_double(-1.0)
        torch.cuda.synchronize()
        in_use = pool.current()
        pool.reset_high()
        rc = fn(n, kind, coef.data_ptr(), x.data_ptr(), rhs.data_ptr(), r.data_ptr(), ctypes.byref(nrm), stream)
        assert rc == 0, bmg.lib.bmg_last_error().decode()
        torch.cuda.synchronize()
        assert pool.high() <= in_use        # nothing was allocated from the pool during the call
        assert torch.equal(r, r_ref)
        assert nrm.value == norm_ref        # same kernels, same summation order: the same bits
        want = bx.residual(bx.drop_ghost_couplings(np.array(planes)), xh, f)
        assert np.array_equal(r.cpu().numpy(), want)
        assert nrm.value == device_norm(want)
        assert nrm.value == pytest.approx(bx.norm(want), rel=1e-14, abs=0)


def test_noalloc_without_residual_or_without_norm(bmg):
    fn = noalloc_fn(bmg)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    kind, planes, f = w.lognormal_problem(255, 2.0, 8.0, seed_k=4, seed_f=7)
    coef = torch.from_numpy(planes).cuda()
    rhs = torch.from_numpy(f).cuda()
    x = torch.from_numpy(w.rhs_uniform(255, 77)).cuda()
    r_ref, norm_ref = bmg.residual(kind, coef, x, rhs)
    nrm = ctypes.c_double(-1.0)
    assert fn(255, kind, coef.data_ptr(), x.data_ptr(), rhs.data_ptr(), None, ctypes.byref(nrm), stream) == 0
    assert nrm.value == norm_ref
    r = torch.full_like(rhs, np.nan)
    assert fn(255, kind, coef.data_ptr(), x.data_ptr(), rhs.data_ptr(), r.data_ptr(), None, stream) == 0
    torch.cuda.synchronize()
    assert torch.equal(r, r_ref)
    assert fn(254, kind, coef.data_ptr(), x.data_ptr(), rhs.data_ptr(), r.data_ptr(), None, stream) != 0
