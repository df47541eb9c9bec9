"""The allocation-free residual-norm entry point (bmg_residual_noalloc), for
callers that cannot let the library allocate device memory, gives what the
allocating entry point (bmg_residual) gives.  Two calls in a row, the second
on a smaller grid, so a partial sum left in the shared static scratch by the
first call would show up in the second."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as w

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point_twice(bmg):
    fn = bmg.lib.bmg_residual_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [w.binary_contrast_problem(2047, 16, seed_k=2, seed_f=3), w.lognormal_problem(63, 2.0, 8.0, seed_k=4, seed_f=7)]
    for kind, planes, f in cases:
        n = planes.shape[-1] - 2
        coef = torch.from_numpy(planes).cuda()
        rhs = torch.from_numpy(f).cuda()
        x = torch.from_numpy(w.rhs_uniform(n, 123)).cuda()
        r_ref, norm_ref = bmg.residual(kind, coef, x, rhs)
        r = torch.full_like(rhs, np.nan)
        nrm = ctypes.c_double(-1.0)
        rc = fn(n, kind, coef.data_ptr(), x.data_ptr(), rhs.data_ptr(), r.data_ptr(), ctypes.byref(nrm), stream)
        assert rc == 0, bmg.lib.bmg_last_error().decode()
        assert torch.equal(r, r_ref)
        assert abs(nrm.value - norm_ref) <= 1e-14 * norm_ref
