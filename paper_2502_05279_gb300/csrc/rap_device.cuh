// Galerkin coarse-operator entries A_c(c, c+t) = sum_p P(p,c) sum_q a(p,q) P(q,c+t)
// by local stencil algebra, in the stated order (p over the 3x3 fine block of
// c, dy outer and dx inner; q over the row of A at p in canonical order;
// structural zeros skipped at compile time), one rounding per operation.  The
// stencil planes and the interpolation weights may live in global or shared
// memory: the same templates serve the setup's k_rap and the per-crop
// two-grid training kernel.
#pragma once

#include "common.cuh"

namespace bmg {
namespace rapdev {

// phi(c', dx, dy): weight of fine point 2c' + (dx, dy) toward coarse point c'
// (column c' of P restricted to its 3x3 footprint); zero for a ghost c'.
template <int DX, int DY>
__device__ __forceinline__ double phi(const double* ci, size_t psc, int ldc, int nc, int ic, int jc) {
  if (ic < 1 || ic > nc || jc < 1 || jc > nc) return 0.0;
  if (DX == 0 && DY == 0) return 1.0;
  if (DX == -1 && DY == 0) return ci[CI_LR * psc + (size_t)jc * ldc + ic];
  if (DX == 1 && DY == 0) return ci[CI_LL * psc + (size_t)jc * ldc + ic + 1];
  if (DX == 0 && DY == -1) return ci[CI_LA * psc + (size_t)jc * ldc + ic];
  if (DX == 0 && DY == 1) return ci[CI_LB * psc + (size_t)(jc + 1) * ldc + ic];
  if (DX == -1 && DY == -1) return ci[CI_LNE * psc + (size_t)jc * ldc + ic];
  if (DX == 1 && DY == -1) return ci[CI_LNW * psc + (size_t)jc * ldc + ic + 1];
  if (DX == -1 && DY == 1) return ci[CI_LSE * psc + (size_t)(jc + 1) * ldc + ic];
  return ci[CI_LSW * psc + (size_t)(jc + 1) * ldc + ic + 1];
}

// Inner sum over the row of A at p = 2c + (UX, UY) in canonical order,
// sum_v a(p, v) phi_{c+t}(o), o = u + v - 2t; structural zeros (|o| > 1) are
// skipped at compile time.  Returns false when no term exists.
template <int TX, int TY, int UX, int UY, int K>
struct InnerSum {
  __device__ __forceinline__ static void run(const Planes<double>& A, int ld, size_t p, const double* ci,
                                             size_t psc, int ldc, int nc, int ic, int jc, double& acc,
                                             bool& any) {
    constexpr int OX = UX + nbr_dx(K) - 2 * TX;
    constexpr int OY = UY + nbr_dy(K) - 2 * TY;
    if constexpr (OX >= -1 && OX <= 1 && OY >= -1 && OY <= 1) {
      double term = rmul(A.template a<K>(p, ld), phi<OX, OY>(ci, psc, ldc, nc, ic + TX, jc + TY));
      acc = any ? radd(acc, term) : term;
      any = true;
    }
    if constexpr (K < 8) InnerSum<TX, TY, UX, UY, K + 1>::run(A, ld, p, ci, psc, ldc, nc, ic, jc, acc, any);
  }
};

// Outer sum over the 3x3 fine block of c (dy outer, dx inner):
// A_c(c, c+t) = sum_u phi_c(u) * inner(u).
template <int TX, int TY, int B>
struct OuterSum {
  __device__ __forceinline__ static void run(const Planes<double>& A, int ld, const double* ci, size_t psc,
                                             int ldc, int nc, int ic, int jc, double& acc, bool& any) {
    constexpr int UX = (B % 3) - 1, UY = (B / 3) - 1;
    size_t p = (size_t)(2 * jc + UY) * ld + (2 * ic + UX);
    double inner = 0.0;
    bool iany = false;
    InnerSum<TX, TY, UX, UY, 0>::run(A, ld, p, ci, psc, ldc, nc, ic, jc, inner, iany);
    if (iany) {
      double term = rmul(phi<UX, UY>(ci, psc, ldc, nc, ic, jc), inner);
      acc = any ? radd(acc, term) : term;
      any = true;
    }
    if constexpr (B < 8) OuterSum<TX, TY, B + 1>::run(A, ld, ci, psc, ldc, nc, ic, jc, acc, any);
  }
};

template <int TX, int TY>
__device__ __forceinline__ double rap_entry(const Planes<double>& A, int ld, const double* ci, size_t psc, int ldc,
                                            int nc, int ic, int jc) {
  double acc = 0.0;
  bool any = false;
  OuterSum<TX, TY, 0>::run(A, ld, ci, psc, ldc, nc, ic, jc, acc, any);
  return acc;
}

}  // namespace rapdev
}  // namespace bmg
