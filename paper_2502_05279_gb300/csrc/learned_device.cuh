// Learned interpolation weights per coarse cell (FP64, one rounding per
// operation): Dendy's edge sums split by the network's logits, and Dendy's
// centre formula (the local row solve) with those edge weights.  delta = 0
// gives Dendy's weights exactly.  Planes and weights may live in global or
// shared memory: the same functions serve bmg_setup's learned level 0, the
// test-vector loss and the per-crop two-grid training kernel.
#pragma once

#include "common.cuh"
#include "learned.h"

namespace bmg {
namespace learned {

// Logit k of interior coarse point (ic, jc); 0 for a ghost coarse point or
// without logits (delta = NULL: Dendy's weights).
__device__ __forceinline__ double delta_at(const float* delta, int nc, int ic, int jc, int k) {
  if (delta == nullptr || ic < 1 || jc < 1 || ic > nc || jc > nc) return 0.0;
  return (double)delta[((size_t)(jc - 1) * nc + (ic - 1)) * MLP_OUT + k];
}

// Edge points of cell (ic, jc), 0 <= ic, jc <= nc+1: x-edge (2ic-1, 2jc) between
// (ic-1, jc) [its E logit] and (ic, jc) [its W logit]; y-edge (2ic, 2jc-1)
// between (ic, jc-1) [N logit] and (ic, jc) [S logit].  An edge point keeps
// Dendy's total weight S_D = -(col_1 + col_2)/D and splits it in the shares
// u_k = -col_k exp(logit).  aux (optional, 4 coarse planes) keeps S_D and the
// first share q for the gradient.
__device__ __forceinline__ void edge_cell(const Planes<double>& A, int ld, int nc, const float* delta, int ic, int jc,
                                          double* ci, double* aux) {
  const int ldc = nc + 2;
  const size_t psc = plane_size(nc), pc = (size_t)jc * ldc + ic;
  double ll = 0, lr = 0, lb = 0, la = 0, sdx = 0, qx = 0, sdy = 0, qy = 0;
  if (ic >= 1 && jc >= 1 && jc <= nc) {
    size_t p = (size_t)(2 * jc) * ld + (2 * ic - 1);
    double colW = radd(radd(A.a<5>(p, ld), A.a<1>(p, ld)), A.a<7>(p, ld));
    double colE = radd(radd(A.a<8>(p, ld), A.a<2>(p, ld)), A.a<6>(p, ld));
    double D = radd(radd(A.a<3>(p, ld), A.a<0>(p, ld)), A.a<4>(p, ld));
    sdx = -rdiv(radd(colW, colE), D);
    double uW = rmul(-colW, exp(delta_at(delta, nc, ic - 1, jc, 1)));
    double uE = rmul(-colE, exp(delta_at(delta, nc, ic, jc, 0)));
    qx = rdiv(uW, radd(uW, uE));
    ll = rmul(sdx, qx);
    lr = rmul(sdx, rsub(1.0, qx));
  }
  if (ic >= 1 && ic <= nc && jc >= 1) {
    size_t p = (size_t)(2 * jc - 1) * ld + 2 * ic;
    double rowS = radd(radd(A.a<5>(p, ld), A.a<3>(p, ld)), A.a<8>(p, ld));
    double rowN = radd(radd(A.a<7>(p, ld), A.a<4>(p, ld)), A.a<6>(p, ld));
    double D = radd(radd(A.a<1>(p, ld), A.a<0>(p, ld)), A.a<2>(p, ld));
    sdy = -rdiv(radd(rowS, rowN), D);
    double uS = rmul(-rowS, exp(delta_at(delta, nc, ic, jc - 1, 3)));
    double uN = rmul(-rowN, exp(delta_at(delta, nc, ic, jc, 2)));
    qy = rdiv(uS, radd(uS, uN));
    lb = rmul(sdy, qy);
    la = rmul(sdy, rsub(1.0, qy));
  }
  ci[CI_LL * psc + pc] = ll;
  ci[CI_LR * psc + pc] = lr;
  ci[CI_LB * psc + pc] = lb;
  ci[CI_LA * psc + pc] = la;
  if (aux) {
    aux[0 * psc + pc] = sdx;
    aux[1 * psc + pc] = qx;
    aux[2 * psc + pc] = sdy;
    aux[3 * psc + pc] = qy;
  }
}

// Dendy's centre formula of cell (ic, jc) with the edge planes of ci (which
// must be complete for the neighbouring cells first).
__device__ __forceinline__ void centre_cell(const Planes<double>& A, int ld, int nc, int ic, int jc, double* ci) {
  const int ldc = nc + 2;
  const size_t psc = plane_size(nc), pc = (size_t)jc * ldc + ic;
  if (ic == 0 || jc == 0) {
    for (int k = 0; k < 4; ++k) ci[k * psc + pc] = 0.0;
    return;
  }
  size_t p = (size_t)(2 * jc - 1) * ld + (2 * ic - 1);
  double aO = A.a<0>(p, ld), aW = A.a<1>(p, ld), aE = A.a<2>(p, ld), aS = A.a<3>(p, ld), aN = A.a<4>(p, ld);
  double aSW = A.a<5>(p, ld), aNE = A.a<6>(p, ld), aNW = A.a<7>(p, ld), aSE = A.a<8>(p, ld);
  double lb_w = ci[CI_LB * psc + pc - 1], la_w = ci[CI_LA * psc + pc - 1];
  double lb_e = ci[CI_LB * psc + pc], la_e = ci[CI_LA * psc + pc];
  double ll_s = ci[CI_LL * psc + pc - ldc], lr_s = ci[CI_LR * psc + pc - ldc];
  double ll_n = ci[CI_LL * psc + pc], lr_n = ci[CI_LR * psc + pc];
  ci[CI_LSW * psc + pc] = -rdiv(radd(radd(aSW, rmul(aW, lb_w)), rmul(aS, ll_s)), aO);
  ci[CI_LSE * psc + pc] = -rdiv(radd(radd(aSE, rmul(aE, lb_e)), rmul(aS, lr_s)), aO);
  ci[CI_LNW * psc + pc] = -rdiv(radd(radd(aNW, rmul(aW, la_w)), rmul(aN, ll_n)), aO);
  ci[CI_LNE * psc + pc] = -rdiv(radd(radd(aNE, rmul(aE, la_e)), rmul(aN, lr_n)), aO);
}

}  // namespace learned
}  // namespace bmg
