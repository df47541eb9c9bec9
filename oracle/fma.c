/* Correctly rounded fused multiply-add over arrays, for the oracle's fused
 * arithmetic mode.  TEST INFRASTRUCTURE ONLY: loaded by oracle/fused.py.
 *
 * out[i] = a[i] * b[i] + c[i] with a single rounding to nearest-even, which
 * is C99's fma / fmaf (ISO C 7.12.13.1, IEEE 754 fusedMultiplyAdd).  Compiled
 * with -ffp-contract=off; nothing else here rounds. */
#include <math.h>
#include <stddef.h>

void oracle_fma_f64(size_t n, const double* a, const double* b, const double* c, double* out) {
  for (size_t i = 0; i < n; ++i) out[i] = fma(a[i], b[i], c[i]);
}

void oracle_fma_f32(size_t n, const float* a, const float* b, const float* c, float* out) {
  for (size_t i = 0; i < n; ++i) out[i] = fmaf(a[i], b[i], c[i]);
}
