"""The rule the refinement residual uses to form fl32(r / s) (s a power of
two) without an FP64 multiply: narrowing r to FP32 first and scaling in FP32
gives the same float whenever fl32(r) and the scaled value both lie in
[2^-125, 2^127].  Checked here on the CPU over random doubles across the whole
exponent range, with round-to-nearest ties forced, against the FP64 product
narrowed once (numpy's float32 conversion rounds to nearest even)."""
import numpy as np


def test_narrow_then_scale_equals_scale_then_narrow():
    rng = np.random.default_rng(7)
    fast = 0
    for trial in range(12):
        n = 400_000
        r = (rng.random(n) + 1.0) * np.exp2(rng.integers(-160, 140, n).astype(float))
        r *= np.where(rng.random(n) < 0.5, -1.0, 1.0)
        if trial % 3 == 0:      # halfway cases of the FP64 -> FP32 rounding
            bits = r.view(np.uint64)
            r = ((bits & ~np.uint64((1 << 29) - 1)) | np.uint64(1 << 28)).view(np.float64)
        inv = np.exp2(rng.integers(-140, 140, n).astype(float))
        with np.errstate(all="ignore"):
            want = (r * inv).astype(np.float32)
            a = r.astype(np.float32)
            inv32 = np.where((inv >= 2.0 ** -125) & (inv <= 2.0 ** 125), inv, 0.0).astype(np.float32)
            b = a * inv32
        ma, mb = np.abs(a), np.abs(b)
        ok = (ma >= 2.0 ** -125) & (ma <= 2.0 ** 127) & (mb >= 2.0 ** -125) & (mb <= 2.0 ** 127)
        fast += int(ok.sum())
        assert np.array_equal(b[ok].view(np.uint32), want[ok].view(np.uint32))
    assert fast > 2_000_000
