// BoxMG with periodic sides: setup (stencil preparation, Dendy interpolation,
// Galerkin coarse operators, coarsest Cholesky) and the FP64 V(nu1, nu2)
// cycle over grids whose periodic axes wrap around.
//
// The formulas, term orders and arithmetic modes are those of the Dirichlet
// kernels (k_setup.cu, cycle_device.cuh, rap_device.cuh): Dendy's collapsed-
// stencil weights in the Fig. 2 layout, the Fig. 2 restriction, A_c = P^T A P
// entry by entry, Gauss-Seidel by colours, residual and interpolation rows
// in the order O, W, E, S, N, SW, NE, NW, SE.  What differs is the index map:
// a neighbour across a periodic side is the point on the opposite side (the
// kernels wrap the index; the ghost lines stay zero), and a coarse grid of a
// periodic axis is periodic again.  Dirichlet axes read their zero ghosts as
// the Dirichlet kernels do.
//
// Layout of a level: six planes O, W, S, SW, NW, D = 1/O of (ny+2) x (nx+2)
// doubles; interpolation weights: eight planes of (ny_c+2) x (nx_c+2), the
// cell (ic, jc) whose north-east corner is coarse point (ic, jc) holding the
// weights of fine points (2ic-1, 2jc-1), (2ic-1, 2jc) and (2ic, 2jc-1); a
// periodic axis has N_c cells (1..N_c), a Dirichlet one N_c + 1.
#include <vector>

#include "common.cuh"
#include "cycle_device.cuh"
#include "kernels.h"
#include "periodic.h"

namespace bmg {

namespace {

constexpr int PBX = 32, PBY = 8;

// Index map of one level.
struct PGeom {
  int nx, ny, px, py;
  __device__ __forceinline__ int wi(int i) const { return px ? (i < 1 ? i + nx : (i > nx ? i - nx : i)) : i; }
  __device__ __forceinline__ int wj(int j) const { return py ? (j < 1 ? j + ny : (j > ny ? j - ny : j)) : j; }
  // linear index of point (i, j), i in 0..nx+1, j in 0..ny+1, wrapped on periodic axes
  __device__ __forceinline__ size_t at(int i, int j) const { return (size_t)wj(j) * (nx + 2) + wi(i); }
  __host__ __device__ __forceinline__ size_t ps() const { return (size_t)(nx + 2) * (ny + 2); }
};

// Coarse cells of an axis: 1..N_c (periodic, cell N_c + 1 is cell 1) or
// 1..N_c + 1 (Dirichlet).
struct CellMap {
  int ncx, ncy, px, py;
  __device__ __forceinline__ int ci(int k) const { return px ? (k < 1 ? k + ncx : (k > ncx ? k - ncx : k)) : k; }
  __device__ __forceinline__ int cj(int k) const { return py ? (k < 1 ? k + ncy : (k > ncy ? k - ncy : k)) : k; }
  __device__ __forceinline__ size_t at(int ic, int jc) const { return (size_t)cj(jc) * (ncx + 2) + ci(ic); }
  __device__ __forceinline__ size_t ps() const { return (size_t)(ncx + 2) * (ncy + 2); }
  __device__ __forceinline__ int kx() const { return px ? ncx : ncx + 1; }
  __device__ __forceinline__ int ky() const { return py ? ncy : ncy + 1; }
};

__host__ __device__ inline int coarse_n(int n, int periodic) { return periodic ? n / 2 : (n - 1) / 2; }

__device__ __forceinline__ PGeom coarse_geom(const PGeom& g) {
  return PGeom{coarse_n(g.nx, g.px), coarse_n(g.ny, g.py), g.px, g.py};
}

__device__ __forceinline__ CellMap cells_of(const PGeom& g) {
  return CellMap{coarse_n(g.nx, g.px), coarse_n(g.ny, g.py), g.px, g.py};
}

// a(p, p + (dx_K, dy_K)) at point (i, j), the K-th neighbour in the canonical
// order, through the symmetric storage: E = W(i+1, j), N = S(i, j+1),
// NE = SW(i+1, j+1), SE = NW(i+1, j-1).
template <int K>
__device__ __forceinline__ double coup(const double* __restrict__ st, const PGeom& g, int i, int j) {
  const size_t ps = g.ps();
  if (K == 0) return st[g.at(i, j)];
  if (K == 1) return st[ps + g.at(i, j)];
  if (K == 2) return st[ps + g.at(i + 1, j)];
  if (K == 3) return st[2 * ps + g.at(i, j)];
  if (K == 4) return st[2 * ps + g.at(i, j + 1)];
  if (K == 5) return st[3 * ps + g.at(i, j)];
  if (K == 6) return st[3 * ps + g.at(i + 1, j + 1)];
  if (K == 7) return st[4 * ps + g.at(i, j)];
  return st[4 * ps + g.at(i + 1, j - 1)];
}

template <int K, bool FU>
__device__ __forceinline__ double sub_term(double s, const double* __restrict__ st, const double* __restrict__ x,
                                          const PGeom& g, int i, int j) {
  return msub<FU>(s, coup<K>(st, g, i, j), x[g.at(i + nbr_dx(K), j + nbr_dy(K))]);
}

// s - sum over the row of A at (i, j) of a x, canonical order (O first when WITH_O).
template <bool NINE, bool WITH_O, bool FU>
__device__ __forceinline__ double prow(const double* __restrict__ st, const double* __restrict__ x, const PGeom& g,
                                       int i, int j, double s) {
  if (WITH_O) s = sub_term<0, FU>(s, st, x, g, i, j);
  s = sub_term<1, FU>(s, st, x, g, i, j);
  s = sub_term<2, FU>(s, st, x, g, i, j);
  s = sub_term<3, FU>(s, st, x, g, i, j);
  s = sub_term<4, FU>(s, st, x, g, i, j);
  if (NINE) {
    s = sub_term<5, FU>(s, st, x, g, i, j);
    s = sub_term<6, FU>(s, st, x, g, i, j);
    s = sub_term<7, FU>(s, st, x, g, i, j);
    s = sub_term<8, FU>(s, st, x, g, i, j);
  }
  return s;
}

// ---- setup -------------------------------------------------------------------------
// The caller's planes into the level-0 layout: ghost lines zero, couplings
// toward a Dirichlet ghost zero, couplings across a periodic side kept.
__global__ void k_p_prepare(PGeom g, int kind, const double* __restrict__ in, double* __restrict__ st) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > g.nx + 1 || j > g.ny + 1) return;
  const size_t ps = g.ps(), p = (size_t)j * (g.nx + 2) + i;
  const bool inside = i >= 1 && i <= g.nx && j >= 1 && j <= g.ny;
  double o = 0, w = 0, s = 0, sw = 0, nw = 0;
  if (inside) {
    o = in[p];
    if (g.px || i > 1) w = in[ps + p];
    if (g.py || j > 1) s = in[2 * ps + p];
    if (kind == 9) {
      if ((g.px || i > 1) && (g.py || j > 1)) sw = in[3 * ps + p];
      if ((g.px || i > 1) && (g.py || j < g.ny)) nw = in[4 * ps + p];
    }
  }
  st[p] = o;
  st[ps + p] = w;
  st[2 * ps + p] = s;
  st[3 * ps + p] = sw;
  st[4 * ps + p] = nw;
  st[5 * ps + p] = 0.0;
}

__global__ void k_p_dinv(PGeom g, double* __restrict__ st, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1, j = blockIdx.y * blockDim.y + threadIdx.y + 1;
  if (i > g.nx || j > g.ny) return;
  const size_t p = (size_t)j * (g.nx + 2) + i;
  const double o = st[p];
  if (!(o > 0.0)) atomicExch(err, 1);
  st[5 * g.ps() + p] = rdiv(1.0, o);
}

struct EdgeW {
  double lo, hi;
};

// x-edge point of cell (ic, jc) = fine (2ic-1, 2jc): LL, LR.  Zero outside the cells.
__device__ __forceinline__ EdgeW p_xedge(const double* __restrict__ st, const PGeom& g, const CellMap& c, int ic,
                                         int jc, int* err) {
  if (ic < 1 || ic > c.kx() || jc < 1 || jc > c.ncy) return EdgeW{0.0, 0.0};
  const int i = 2 * ic - 1, j = 2 * jc;
  double D = radd(radd(coup<3>(st, g, i, j), coup<0>(st, g, i, j)), coup<4>(st, g, i, j));
  if (!(fabs(D) > 0.0) || isinf(D)) atomicExch(err, 2);
  double ll = -rdiv(radd(radd(coup<5>(st, g, i, j), coup<1>(st, g, i, j)), coup<7>(st, g, i, j)), D);
  double lr = -rdiv(radd(radd(coup<8>(st, g, i, j), coup<2>(st, g, i, j)), coup<6>(st, g, i, j)), D);
  return EdgeW{ll, lr};
}

// y-edge point of cell (ic, jc) = fine (2ic, 2jc-1): LB, LA.
__device__ __forceinline__ EdgeW p_yedge(const double* __restrict__ st, const PGeom& g, const CellMap& c, int ic,
                                         int jc, int* err) {
  if (ic < 1 || ic > c.ncx || jc < 1 || jc > c.ky()) return EdgeW{0.0, 0.0};
  const int i = 2 * ic, j = 2 * jc - 1;
  double D = radd(radd(coup<1>(st, g, i, j), coup<0>(st, g, i, j)), coup<2>(st, g, i, j));
  if (!(fabs(D) > 0.0) || isinf(D)) atomicExch(err, 2);
  double lb = -rdiv(radd(radd(coup<5>(st, g, i, j), coup<3>(st, g, i, j)), coup<8>(st, g, i, j)), D);
  double la = -rdiv(radd(radd(coup<7>(st, g, i, j), coup<4>(st, g, i, j)), coup<6>(st, g, i, j)), D);
  return EdgeW{lb, la};
}

// One thread per cell (ic, jc) of the (nx_c+2) x (ny_c+2) weight planes: the
// cell's edge points and its centre point, whose row of A is solved with the
// four edge neighbours interpolated (the west and south neighbours belong to
// cells ic - 1 and jc - 1, wrapped on a periodic axis and recomputed here with
// the same code).  Entries outside the cells are zero.
__global__ void k_p_dendy(PGeom g, const double* __restrict__ st, double* __restrict__ ci, int* err) {
  const int ic = blockIdx.x * blockDim.x + threadIdx.x, jc = blockIdx.y * blockDim.y + threadIdx.y;
  const CellMap c = cells_of(g);
  if (ic > c.ncx + 1 || jc > c.ncy + 1) return;
  const size_t psc = c.ps(), pc = (size_t)jc * (c.ncx + 2) + ic;
  if (ic < 1 || jc < 1 || ic > c.kx() || jc > c.ky()) {
#pragma unroll
    for (int k = 0; k < 8; ++k) ci[k * psc + pc] = 0.0;
    return;
  }
  const EdgeW xe = p_xedge(st, g, c, ic, jc, err);
  const EdgeW ye = p_yedge(st, g, c, ic, jc, err);
  const EdgeW yw = p_yedge(st, g, c, g.px ? c.ci(ic - 1) : ic - 1, jc, err);   // west neighbour of the centre
  const EdgeW xs = p_xedge(st, g, c, ic, g.py ? c.cj(jc - 1) : jc - 1, err);   // south neighbour
  const int i = 2 * ic - 1, j = 2 * jc - 1;
  const double aO = coup<0>(st, g, i, j), aW = coup<1>(st, g, i, j), aE = coup<2>(st, g, i, j);
  const double aS = coup<3>(st, g, i, j), aN = coup<4>(st, g, i, j), aSW = coup<5>(st, g, i, j);
  const double aNE = coup<6>(st, g, i, j), aNW = coup<7>(st, g, i, j), aSE = coup<8>(st, g, i, j);
  if (!(aO > 0.0)) atomicExch(err, 2);
  ci[CI_LSW * psc + pc] = -rdiv(radd(radd(aSW, rmul(aW, yw.lo)), rmul(aS, xs.lo)), aO);
  ci[CI_LSE * psc + pc] = -rdiv(radd(radd(aSE, rmul(aE, ye.lo)), rmul(aS, xs.hi)), aO);
  ci[CI_LNW * psc + pc] = -rdiv(radd(radd(aNW, rmul(aW, yw.hi)), rmul(aN, xe.lo)), aO);
  ci[CI_LNE * psc + pc] = -rdiv(radd(radd(aNE, rmul(aE, ye.hi)), rmul(aN, xe.hi)), aO);
  ci[CI_LL * psc + pc] = xe.lo;
  ci[CI_LR * psc + pc] = xe.hi;
  ci[CI_LB * psc + pc] = ye.lo;
  ci[CI_LA * psc + pc] = ye.hi;
}

// phi(c', dx, dy): weight of fine point 2c' + (dx, dy) toward coarse point c'.
// On a periodic axis c' wraps; on a Dirichlet axis a ghost c' has weight 0.
template <int DX, int DY>
__device__ __forceinline__ double p_phi(const double* __restrict__ ci, const CellMap& c, int ic, int jc) {
  if (c.px) ic = c.ci(ic);
  else if (ic < 1 || ic > c.ncx) return 0.0;
  if (c.py) jc = c.cj(jc);
  else if (jc < 1 || jc > c.ncy) return 0.0;
  const size_t psc = c.ps();
  if (DX == 0 && DY == 0) return 1.0;
  if (DX == -1 && DY == 0) return ci[CI_LR * psc + c.at(ic, jc)];
  if (DX == 1 && DY == 0) return ci[CI_LL * psc + c.at(ic + 1, jc)];
  if (DX == 0 && DY == -1) return ci[CI_LA * psc + c.at(ic, jc)];
  if (DX == 0 && DY == 1) return ci[CI_LB * psc + c.at(ic, jc + 1)];
  if (DX == -1 && DY == -1) return ci[CI_LNE * psc + c.at(ic, jc)];
  if (DX == 1 && DY == -1) return ci[CI_LNW * psc + c.at(ic + 1, jc)];
  if (DX == -1 && DY == 1) return ci[CI_LSE * psc + c.at(ic, jc + 1)];
  return ci[CI_LSW * psc + c.at(ic + 1, jc + 1)];
}

// A_c(c, c+t) = sum_u phi_c(u) sum_v a(2c+u, v) phi_{c+t}(u + v - 2t), u over the
// 3x3 block (dy outer, dx inner), v in the canonical order, structural zeros
// skipped at compile time; one rounding per operation (the order of the
// Dirichlet kernel, indices wrapped).
template <int TX, int TY, int UX, int UY, int K>
struct PInner {
  __device__ __forceinline__ static void run(const double* st, const PGeom& g, const double* ci, const CellMap& c,
                                             int ic, int jc, double& acc, bool& any) {
    constexpr int OX = UX + nbr_dx(K) - 2 * TX;
    constexpr int OY = UY + nbr_dy(K) - 2 * TY;
    if constexpr (OX >= -1 && OX <= 1 && OY >= -1 && OY <= 1) {
      double term = rmul(coup<K>(st, g, 2 * ic + UX, 2 * jc + UY), p_phi<OX, OY>(ci, c, ic + TX, jc + TY));
      acc = any ? radd(acc, term) : term;
      any = true;
    }
    if constexpr (K < 8) PInner<TX, TY, UX, UY, K + 1>::run(st, g, ci, c, ic, jc, acc, any);
  }
};

template <int TX, int TY, int B>
struct POuter {
  __device__ __forceinline__ static void run(const double* st, const PGeom& g, const double* ci, const CellMap& c,
                                             int ic, int jc, double& acc, bool& any) {
    constexpr int UX = (B % 3) - 1, UY = (B / 3) - 1;
    double inner = 0.0;
    bool iany = false;
    PInner<TX, TY, UX, UY, 0>::run(st, g, ci, c, ic, jc, inner, iany);
    if (iany) {
      double term = rmul(p_phi<UX, UY>(ci, c, ic, jc), inner);
      acc = any ? radd(acc, term) : term;
      any = true;
    }
    if constexpr (B < 8) POuter<TX, TY, B + 1>::run(st, g, ci, c, ic, jc, acc, any);
  }
};

template <int TX, int TY>
__device__ __forceinline__ double p_rap_entry(const double* st, const PGeom& g, const double* ci, const CellMap& c,
                                              int ic, int jc) {
  double acc = 0.0;
  bool any = false;
  POuter<TX, TY, 0>::run(st, g, ci, c, ic, jc, acc, any);
  return acc;
}

// One thread per coarse point of the (nx_c+2) x (ny_c+2) planes; couplings
// toward a Dirichlet ghost zero, ghost lines zero, D left for k_p_dinv.
__global__ void k_p_rap(PGeom g, const double* __restrict__ st, const double* __restrict__ ci,
                        double* __restrict__ stc) {
  const int ic = blockIdx.x * blockDim.x + threadIdx.x, jc = blockIdx.y * blockDim.y + threadIdx.y;
  const CellMap c = cells_of(g);
  if (ic > c.ncx + 1 || jc > c.ncy + 1) return;
  const size_t psc = c.ps(), pc = (size_t)jc * (c.ncx + 2) + ic;
  if (ic < 1 || jc < 1 || ic > c.ncx || jc > c.ncy) {
#pragma unroll
    for (int k = 0; k < 6; ++k) stc[k * psc + pc] = 0.0;
    return;
  }
  const bool w_in = g.px || ic > 1, s_in = g.py || jc > 1, n_in = g.py || jc < c.ncy;
  stc[pc] = p_rap_entry<0, 0>(st, g, ci, c, ic, jc);
  stc[psc + pc] = w_in ? p_rap_entry<-1, 0>(st, g, ci, c, ic, jc) : 0.0;
  stc[2 * psc + pc] = s_in ? p_rap_entry<0, -1>(st, g, ci, c, ic, jc) : 0.0;
  stc[3 * psc + pc] = (w_in && s_in) ? p_rap_entry<-1, -1>(st, g, ci, c, ic, jc) : 0.0;
  stc[4 * psc + pc] = (w_in && n_in) ? p_rap_entry<-1, 1>(st, g, ci, c, ic, jc) : 0.0;
  stc[5 * psc + pc] = 0.0;
}

// Coarsest Cholesky (one thread, m = nx ny <= 16): the dense matrix over
// lexicographic unknowns (a coupling across a periodic side lands on the
// wrapped unknown, entries landing on one unknown add), then right-looking
// Cholesky in the Dirichlet kernel's order.
__global__ void k_p_factor(PGeom g, const double* __restrict__ st, double* __restrict__ L, double* __restrict__ a,
                           int* err) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const int m = g.nx * g.ny;
  for (int k = 0; k < m * m; ++k) {
    a[k] = 0.0;
    L[k] = 0.0;
  }
  for (int j = 1; j <= g.ny; ++j)
    for (int i = 1; i <= g.nx; ++i) {
      const int r = (j - 1) * g.nx + (i - 1);
      const double v[9] = {coup<0>(st, g, i, j), coup<1>(st, g, i, j), coup<2>(st, g, i, j),
                           coup<3>(st, g, i, j), coup<4>(st, g, i, j), coup<5>(st, g, i, j),
                           coup<6>(st, g, i, j), coup<7>(st, g, i, j), coup<8>(st, g, i, j)};
      for (int k = 0; k < 9; ++k) {
        const int ii = g.wi(i + nbr_dx(k)), jj = g.wj(j + nbr_dy(k));
        if (ii >= 1 && ii <= g.nx && jj >= 1 && jj <= g.ny) {
          double& e = a[(size_t)r * m + (jj - 1) * g.nx + (ii - 1)];
          e = radd(e, v[k]);
        }
      }
    }
  for (int k = 0; k < m; ++k) {
    const double akk = a[(size_t)k * m + k];
    if (!(akk > 0.0)) {
      atomicExch(err, 3);
      return;
    }
    const double lkk = __dsqrt_rn(akk);
    L[(size_t)k * m + k] = lkk;
    for (int i = k + 1; i < m; ++i) L[(size_t)i * m + k] = rdiv(a[(size_t)i * m + k], lkk);
    for (int j = k + 1; j < m; ++j)
      for (int i = j; i < m; ++i)
        a[(size_t)i * m + j] = rsub(a[(size_t)i * m + j], rmul(L[(size_t)i * m + k], L[(size_t)j * m + k]));
  }
}

// ---- cycle -------------------------------------------------------------------------
// One colour (i % 2 == pi, j % 2 == pj) of a Gauss-Seidel sweep: x_p = (f_p -
// sum_{q != p} a_pq x_q) * D_p.  Points of one colour share no coupling (N is
// even on a periodic axis, so the colouring holds across the seam).
template <bool NINE, bool FU>
__global__ void k_p_gs(PGeom g, const double* __restrict__ st, const double* __restrict__ f, double* x, int pi,
                       int pj, const int* done) {
  if (dev::stopped(done)) return;
  const int i = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x) + (pi ? 1 : 2);
  const int j = 2 * (int)(blockIdx.y * blockDim.y + threadIdx.y) + (pj ? 1 : 2);
  if (i > g.nx || j > g.ny) return;
  const size_t p = (size_t)j * (g.nx + 2) + i;
  const double s = prow<NINE, false, FU>(st, x, g, i, j, f[p]);
  if (BMG_IN(DBG_PERIODIC, p, g.ps())) x[p] = rmul(s, st[5 * g.ps() + p]);
}

// Half of a 9-point sweep: one CTA per row j of parity pj, its odd-i points
// (colour (1, pj)) before its even-i points (colour (0, pj)).  The four-colour
// order (odd,odd), (even,odd), (odd,even), (even,even) is row-parity major, so
// the launch for pj = 1 followed by the one for pj = 0 is one sweep, point for
// point the colour-by-colour one: rows of one parity do not couple (N is even
// on a periodic axis), and a whole row, seam included, belongs to one CTA.
// The row goes in chunks of 2 x 256 columns, the odd points of chunk c + 1
// before the even points of chunk c (an even point reads the new odd values
// beside it, an odd point the old even ones), so a chunk's stencil is read by
// both colours while it is still in the caches.
template <bool FU>
__global__ void __launch_bounds__(256) k_p_gs_rows(PGeom g, const double* __restrict__ st,
                                                   const double* __restrict__ f, double* x, int pj, const int* done) {
  if (dev::stopped(done)) return;
  const int j = 2 * (int)blockIdx.x + (pj ? 1 : 2);
  if (j > g.ny) return;
  const size_t row = (size_t)j * (g.nx + 2), dp = 5 * g.ps();
  constexpr int CW = 512;                                   // chunk width (columns)
  const int chunks = (g.nx + CW - 1) / CW;
  auto point = [&](int i) {
    if (i > g.nx) return;
    const size_t p = row + i;
    const double xn = rmul(prow<true, false, FU>(st, x, g, i, j, f[p]), st[dp + p]);
    if (BMG_IN(DBG_PERIODIC, p, g.ps())) x[p] = xn;
  };
  point(1 + 2 * (int)threadIdx.x);                          // odd points of chunk 0
  for (int c = 0; c < chunks; ++c) {
    if (c + 1 < chunks) point((c + 1) * CW + 1 + 2 * (int)threadIdx.x);
    __syncthreads();
    point(c * CW + 2 + 2 * (int)threadIdx.x);               // even points of chunk c
  }
}

// One-pass 9-point sweep xin -> xout: the FP64 strip walk of the Dirichlet
// levels (56-column warp strips of height ty; lane l holds columns 2l, 2l + 1
// of a 64-column window; the colour regions shrink by one column per colour,
// so lanes 2..29 end with the sweep's values; band rows j0 - 1 .. j1 + 1 pass
// through a per-warp ring of 8-byte cp.async copies) with the window's
// columns and band rows taken modulo N on a periodic axis.  Strips stay
// independent across a periodic seam for the reason they are independent
// inside the grid: a strip's first row is odd and reads only old even rows,
// and its last row (even) needs the new odd row above, which the strip forms
// itself as a halo row; on a periodic y axis that halo row is row ny + 1, i.e.
// row 1, computed from copies of the old values and never stored.  Every point
// takes the operands of the colour-by-colour sweep in the same order, so the
// result is bit-identical to it.
template <int RING, bool FU>
__device__ __forceinline__ void p_strip64_body(const PGeom& g, const double* __restrict__ st,
                                               const double* __restrict__ f, const double* __restrict__ xin,
                                               double* __restrict__ xout, int sx, int sy, int ty,
                                               unsigned char* ring) {
  using Row = dev::StripRowT<double, double>;
  const int nx = g.nx, ny = g.ny, ld = nx + 2;
  const size_t ps = g.ps();
  const int lane = threadIdx.x & 31;
  const int i0 = 1 + 56 * sx, j0 = 1 + ty * sy, j1 = j0 + ty;
  const int ic = i0 - 4 + 2 * lane;
  // source column of window column i (modulo nx on a periodic axis, else
  // inside [0, nx + 1] or zero-filled) and whether it is a point of the level
  auto col = [&](int i, bool& copy, bool& point) {
    if (g.px) {
      copy = point = true;
      return 1 + ((i - 1) % nx + nx) % nx;
    }
    copy = i >= 0 && i <= nx + 1;
    point = i >= 1 && i <= nx;
    return copy ? i : 0;
  };
  bool cpa, cpb, pta, ptb;
  const int ca = col(ic, cpa, pta), cb = col(ic + 1, cpb, ptb);
  const bool c1 = pta && lane >= 1, c2 = ptb && lane >= 1 && lane <= 30;
  const bool c3 = pta && lane >= 2 && lane <= 30, c4 = ptb && lane >= 2 && lane <= 29;
  const bool own = lane >= 2 && lane <= 29;
  const int rlim = g.py ? ny + 1 : ny;            // last row a colour-1/2 update reaches
  // ring slot arrays x, f, D, W, S, SW, NW: the iterate, the right-hand side, stencil planes 5, 1, 2, 3, 4
  constexpr int plane[7] = {-1, -1, 5, 1, 2, 3, 4};
  const int NR = ty + 3;                          // band rows q = 0 .. NR - 1, j = j0 - 1 + q
  auto issue = [&](int q) {
    if (q < NR) {
      const int j = j0 - 1 + q;
      const bool rin = g.py || (j >= 0 && j <= ny + 1);
      const int jr = g.py ? 1 + ((j - 1) % ny + ny) % ny : (rin ? j : 0);
      const size_t pa = (size_t)jr * ld + ca, pb = (size_t)jr * ld + cb;
      // (debug builds: a copy from outside the array is zero-filled instead)
      const bool oka = rin && cpa && BMG_IN(DBG_PERIODIC, pa, ps), okb = rin && cpb && BMG_IN(DBG_PERIODIC, pb, ps);
      double* d = reinterpret_cast<double*>(ring + (q % RING) * dev::STRIP64_SLOT) + 2 * lane;
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        const double* a = k == 0 ? xin : k == 1 ? f : st + (size_t)plane[k] * ps;
        dev::cp_async8(d + 64 * k, a + (oka ? pa : 0), oka);
        dev::cp_async8(d + 64 * k + 1, a + (okb ? pb : 0), okb);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
#pragma unroll
  for (int q = 0; q < RING; ++q) issue(q);
  auto take = [&](int q, Row& R) {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(RING - 1) : "memory");
    dev::row64_read(ring + (q % RING) * dev::STRIP64_SLOT, lane, R);
    issue(q + RING);
  };
  auto store = [&](int j, const Row& R) {
    if (!own || j > ny) return;
    const size_t p = (size_t)j * ld + ic;
    if (ic <= nx && BMG_IN(DBG_PERIODIC, p, ps)) xout[p] = R.xa;
    if (ic + 1 <= nx && BMG_IN(DBG_PERIODIC, p + 1, ps)) xout[p + 1] = R.xb;
  };
  Row P0, P1, Q0, Q1;
  take(0, P1);
  take(1, Q0);
  take(2, Q1);
  if (j0 <= rlim) {
    dev::strip_row<double, double, FU>(P1, Q0, Q1, c1, c2);   // row j0: colours 1, 2
    store(j0, Q0);
  }
  auto step = [&](int m, Row& E0, Row& E1, Row& E2, Row& E3) {
    const int a = j0 + 2 * m;
    take(2 * m + 1, E2);
    take(2 * m + 2, E3);
    if (a <= rlim) {
      dev::strip_row<double, double, FU>(E1, E2, E3, c1, c2); // row a: colours 1, 2
      if (a < j1) store(a, E2);
    }
    if (a - 1 <= ny) {
      dev::strip_row<double, double, FU>(E0, E1, E2, c3, c4); // row a - 1: colours 3, 4
      store(a - 1, E1);
    }
  };
#pragma unroll 1
  for (int m = 1; m <= ty / 2; m += 2) {
    step(m, Q0, Q1, P0, P1);
    if (m + 1 <= ty / 2) step(m + 1, P0, P1, Q0, Q1);
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");   // no copy outlives the warp
}

constexpr int P_STRIP_WARPS = 4, P_STRIP_RING = 4;
constexpr size_t P_STRIP_SMEM = (size_t)P_STRIP_WARPS * P_STRIP_RING * dev::STRIP64_SLOT;

template <bool FU>
__global__ void __launch_bounds__(32 * P_STRIP_WARPS, 4) k_p_gs_strip(PGeom g, const double* __restrict__ st,
                                                                   const double* __restrict__ f,
                                                                   const double* __restrict__ xin,
                                                                   double* __restrict__ xout, int ty,
                                                                   const int* done) {
  extern __shared__ __align__(128) unsigned char p_strip_smem[];
  if (dev::stopped(done)) return;
  const int nbx = (g.nx + 55) / 56, nby = (g.ny + ty - 1) / ty;
  const int w = threadIdx.x >> 5, s = blockIdx.x * P_STRIP_WARPS + w;
  if (s >= nbx * nby) return;                     // whole warps only
  p_strip64_body<P_STRIP_RING, FU>(g, st, f, xin, xout, s % nbx, s / nbx, ty,
                                   p_strip_smem + (size_t)w * P_STRIP_RING * dev::STRIP64_SLOT);
}

// r = f - A x (when r != NULL) and the partial sums of r^2 in the canonical
// reduction order (block b of G = min(ny, 1024): rows 1 + b, 1 + b + G, ...;
// thread t: columns 1 + t, 1 + t + 256, ...; then the halving tree).
template <bool NINE, bool FU>
__global__ void __launch_bounds__(dev::NORM_THREADS) k_p_residual(PGeom g, const double* __restrict__ st,
                                                                  const double* __restrict__ x,
                                                                  const double* __restrict__ f, double* __restrict__ r,
                                                                  double* __restrict__ partials, const int* done) {
  if (dev::stopped(done)) return;
  const int b = blockIdx.x, G = gridDim.x;
  double acc = 0.0;
  for (int j = 1 + b; j <= g.ny; j += G)
    for (int i = 1 + threadIdx.x; i <= g.nx; i += dev::NORM_THREADS) {
      const size_t p = (size_t)j * (g.nx + 2) + i;
      const double s = prow<NINE, true, FU>(st, x, g, i, j, f[p]);
      if (r && BMG_IN(DBG_PERIODIC, p, g.ps())) r[p] = s;
      acc = madd<FU>(acc, s, s);
    }
  if (partials) {
    const double tot = dev::block_sum(acc);
    if (threadIdx.x == 0) partials[b] = tot;
  }
}

// f_c = P^T r at coarse point (ic, jc), term by term in the order of the Fig. 2
// loop (a primed weight read at the neighbouring cell, wrapped on a periodic
// axis); the coincident term has weight 1.  Also zeroes the coarse iterate
// there.
template <bool FU>
__global__ void k_p_restrict(PGeom g, const double* __restrict__ ci, const double* __restrict__ r,
                             double* __restrict__ fc, double* __restrict__ xc, const int* done) {
  if (dev::stopped(done)) return;
  const CellMap c = cells_of(g);
  const int ic = blockIdx.x * blockDim.x + threadIdx.x + 1, jc = blockIdx.y * blockDim.y + threadIdx.y + 1;
  if (ic > c.ncx || jc > c.ncy) return;
  const size_t psc = c.ps();
  const int i = 2 * ic, j = 2 * jc;
  auto q = [&](int di, int dj) { return r[g.at(i + di, j + dj)]; };
  auto w = [&](int k, int dic, int djc) { return ci[k * psc + c.at(ic + dic, jc + djc)]; };
  double t = rmul(w(CI_LNE, 0, 0), q(-1, -1));
  t = madd<FU>(t, w(CI_LA, 0, 0), q(0, -1));
  t = madd<FU>(t, w(CI_LNW, 1, 0), q(1, -1));
  t = madd<FU>(t, w(CI_LR, 0, 0), q(-1, 0));
  t = radd(t, q(0, 0));
  t = madd<FU>(t, w(CI_LL, 1, 0), q(1, 0));
  t = madd<FU>(t, w(CI_LSE, 0, 1), q(-1, 1));
  t = madd<FU>(t, w(CI_LB, 0, 1), q(0, 1));
  t = madd<FU>(t, w(CI_LSW, 1, 1), q(1, 1));
  const size_t pc = (size_t)jc * (c.ncx + 2) + ic;
  if (BMG_IN(DBG_PERIODIC, pc, psc)) {
    fc[pc] = t;
    xc[pc] = 0.0;   // the coarse iterate starts from zero (its ghost lines stay zero)
  }
}

// x_out = x_in + P e_c (x_in and x_out may be the same array), one thread per
// coarse cell (ic, jc): its coincident point (2ic, 2jc), x-edge point (2ic-1,
// 2jc), y-edge point (2ic, 2jc-1) and centre point (2ic-1, 2jc-1); a point
// beyond a Dirichlet side is skipped.  The interpolated value is formed first,
// then added (coincident e_NE; x-edge LL e_NW + LR e_NE; y-edge LB e_SE + LA
// e_NE; centre ((LSW e_SW + LSE e_SE) + LNW e_NW) + LNE e_NE, e_SW .. e_NE the
// cell's coarse corners, wrapped on a periodic axis, a Dirichlet ghost reading
// its zero).  Every load of the cell is issued before its first store.
template <bool FU>
__global__ void k_p_interp(PGeom g, const double* __restrict__ ci, const double* __restrict__ ec,
                           const double* xin, double* xout, const int* done) {
  if (dev::stopped(done)) return;
  const CellMap c = cells_of(g);
  const int ic = blockIdx.x * blockDim.x + threadIdx.x + 1, jc = blockIdx.y * blockDim.y + threadIdx.y + 1;
  if (ic > c.kx() || jc > c.ky()) return;
  const PGeom gc = coarse_geom(g);
  const size_t psc = c.ps(), pc = (size_t)jc * (c.ncx + 2) + ic, ld = g.nx + 2;
  const double e_sw = ec[gc.at(ic - 1, jc - 1)], e_se = ec[gc.at(ic, jc - 1)];
  const double e_nw = ec[gc.at(ic - 1, jc)], e_ne = ec[gc.at(ic, jc)];
  auto w = [&](int k) { return ci[k * psc + pc]; };
  const bool ie = 2 * ic <= g.nx, je = 2 * jc <= g.ny;   // the even column / row exists
  const size_t pf = (size_t)(2 * jc) * ld + 2 * ic;       // coincident point
  double x_co = 0, x_xe = 0, x_ye = 0, x_ce, lsw, lse, lnw, lne, ll = 0, lr = 0, lb = 0, la = 0;
  if (ie && je) x_co = xin[pf];
  if (je) {
    x_xe = xin[pf - 1];
    ll = w(CI_LL);
    lr = w(CI_LR);
  }
  if (ie) {
    x_ye = xin[pf - ld];
    lb = w(CI_LB);
    la = w(CI_LA);
  }
  x_ce = xin[pf - ld - 1];
  lsw = w(CI_LSW);
  lse = w(CI_LSE);
  lnw = w(CI_LNW);
  lne = w(CI_LNE);
  const size_t ps = g.ps();
  if (ie && je && BMG_IN(DBG_PERIODIC, pf, ps)) xout[pf] = radd(x_co, e_ne);
  if (je) {
    double t = rmul(ll, e_nw);
    t = madd<FU>(t, lr, e_ne);
    if (BMG_IN(DBG_PERIODIC, pf - 1, ps)) xout[pf - 1] = radd(x_xe, t);
  }
  if (ie) {
    double t = rmul(lb, e_se);
    t = madd<FU>(t, la, e_ne);
    if (BMG_IN(DBG_PERIODIC, pf - ld, ps)) xout[pf - ld] = radd(x_ye, t);
  }
  {
    double t = rmul(lsw, e_sw);
    t = madd<FU>(t, lse, e_se);
    t = madd<FU>(t, lnw, e_nw);
    t = madd<FU>(t, lne, e_ne);
    if (BMG_IN(DBG_PERIODIC, pf - ld - 1, ps)) xout[pf - ld - 1] = radd(x_ce, t);
  }
}

// L L^T x = f on the coarsest level (one thread, m <= 16): forward then backward
// substitution, inner sums in increasing index order.
__global__ void k_p_coarse_solve(PGeom g, const double* __restrict__ L, const double* __restrict__ f,
                                 double* __restrict__ x, const int* done) {
  if (dev::stopped(done)) return;
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const int m = g.nx * g.ny;
  double y[16], z[16];
  for (int i = 0; i < m; ++i) {
    double s = f[(size_t)(i / g.nx + 1) * (g.nx + 2) + (i % g.nx + 1)];
    for (int k = 0; k < i; ++k) s = rsub(s, rmul(L[(size_t)i * m + k], y[k]));
    y[i] = rdiv(s, L[(size_t)i * m + i]);
  }
  for (int i = m - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < m; ++k) s = rsub(s, rmul(L[(size_t)k * m + i], z[k]));
    z[i] = rdiv(s, L[(size_t)i * m + i]);
  }
  for (int i = 0; i < m; ++i) x[(size_t)(i / g.nx + 1) * (g.nx + 2) + (i % g.nx + 1)] = z[i];
}

// ---- flexible CG (FCG(1)) on level 0, preconditioned by the periodic V-cycle ----
// The recurrence of the Dirichlet FCG kernels (k_cycle.cu) over a grid whose
// products wrap: every inner product in the canonical order of k_p_residual
// (block b of G = min(ny, 1024): rows 1 + b, 1 + b + G, ...; thread t: columns
// 1 + t, 1 + t + 256, ...; then the halving tree), the scalars formed once per
// step by the shared reduction kernel.

// r = f - A x (stored), z = 0, partial r.r; the control block's first step.
template <bool NINE, bool FU>
__global__ void __launch_bounds__(dev::NORM_THREADS) k_p_fcg_init(PGeom g, const double* __restrict__ st,
                                                                  const double* __restrict__ x,
                                                                  const double* __restrict__ f,
                                                                  double* __restrict__ r, double* __restrict__ z,
                                                                  double* __restrict__ partials, Ctl* ctl) {
  double acc = 0.0;
  for (int j = 1 + blockIdx.x; j <= g.ny; j += gridDim.x)
    for (int i = 1 + threadIdx.x; i <= g.nx; i += dev::NORM_THREADS) {
      const size_t p = (size_t)j * (g.nx + 2) + i;
      const double rr = prow<NINE, true, FU>(st, x, g, i, j, f[p]);
      if (BMG_IN(DBG_PERIODIC, p, g.ps())) {
        r[p] = rr;
        z[p] = 0.0;
      }
      acc = madd<FU>(acc, rr, rr);
    }
  const double tot = dev::block_sum(acc);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = tot;
    if (blockIdx.x == 0) ctl->first = 1;
  }
}

// partial z.q
template <bool FU>
__global__ void __launch_bounds__(dev::NORM_THREADS) k_p_fcg_zq(PGeom g, const double* __restrict__ z,
                                                                const double* __restrict__ q,
                                                                double* __restrict__ partials, const Ctl* ctl) {
  if (ctl->done) return;
  double acc = 0.0;
  for (int j = 1 + blockIdx.x; j <= g.ny; j += gridDim.x)
    for (int i = 1 + threadIdx.x; i <= g.nx; i += dev::NORM_THREADS) {
      const size_t p = (size_t)j * (g.nx + 2) + i;
      acc = madd<FU>(acc, z[p], q[p]);
    }
  const double tot = dev::block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// p = z (first step) or z + beta p
template <bool FU>
__global__ void k_p_fcg_direction(PGeom g, const double* __restrict__ z, double* __restrict__ pv, const Ctl* ctl) {
  if (ctl->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1, j = blockIdx.y * blockDim.y + threadIdx.y + 1;
  if (i > g.nx || j > g.ny) return;
  const size_t p = (size_t)j * (g.nx + 2) + i;
  if (!BMG_IN(DBG_PERIODIC, p, g.ps())) return;
  pv[p] = ctl->first ? z[p] : madd<FU>(z[p], ctl->beta, pv[p]);
}

// q = A p (a_O p first, then the neighbours in the canonical order, wrapped),
// partial p.q and p.r
template <bool NINE, bool FU>
__global__ void __launch_bounds__(dev::NORM_THREADS) k_p_fcg_matvec(PGeom g, const double* __restrict__ st,
                                                                    const double* __restrict__ pv,
                                                                    const double* __restrict__ r,
                                                                    double* __restrict__ q,
                                                                    double* __restrict__ partials, const Ctl* ctl) {
  if (ctl->done) return;
  double apq = 0.0, apr = 0.0;
  for (int j = 1 + blockIdx.x; j <= g.ny; j += gridDim.x)
    for (int i = 1 + threadIdx.x; i <= g.nx; i += dev::NORM_THREADS) {
      const size_t p = (size_t)j * (g.nx + 2) + i;
      double acc = rmul(coup<0>(st, g, i, j), pv[p]);
      acc = madd<FU>(acc, coup<1>(st, g, i, j), pv[g.at(i - 1, j)]);
      acc = madd<FU>(acc, coup<2>(st, g, i, j), pv[g.at(i + 1, j)]);
      acc = madd<FU>(acc, coup<3>(st, g, i, j), pv[g.at(i, j - 1)]);
      acc = madd<FU>(acc, coup<4>(st, g, i, j), pv[g.at(i, j + 1)]);
      if (NINE) {
        acc = madd<FU>(acc, coup<5>(st, g, i, j), pv[g.at(i - 1, j - 1)]);
        acc = madd<FU>(acc, coup<6>(st, g, i, j), pv[g.at(i + 1, j + 1)]);
        acc = madd<FU>(acc, coup<7>(st, g, i, j), pv[g.at(i - 1, j + 1)]);
        acc = madd<FU>(acc, coup<8>(st, g, i, j), pv[g.at(i + 1, j - 1)]);
      }
      if (BMG_IN(DBG_PERIODIC, p, g.ps())) q[p] = acc;
      apq = madd<FU>(apq, pv[p], acc);
      apr = madd<FU>(apr, pv[p], r[p]);
    }
  const double t1 = dev::block_sum(apq);
  __syncthreads();
  const double t2 = dev::block_sum(apr);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = t1;
    partials[dev::NORM_BLOCKS_MAX + blockIdx.x] = t2;
  }
}

// x += alpha p, r -= alpha q (alpha = (p.r) / (p.q)), z = 0, partial r.r
template <bool FU>
__global__ void __launch_bounds__(dev::NORM_THREADS) k_p_fcg_update(PGeom g, double* __restrict__ x,
                                                                    double* __restrict__ r,
                                                                    const double* __restrict__ pv,
                                                                    const double* __restrict__ q,
                                                                    double* __restrict__ z,
                                                                    double* __restrict__ partials, Ctl* ctl) {
  if (ctl->done) return;
  const double alpha = rdiv(ctl->pr, ctl->pq);
  double acc = 0.0;
  for (int j = 1 + blockIdx.x; j <= g.ny; j += gridDim.x)
    for (int i = 1 + threadIdx.x; i <= g.nx; i += dev::NORM_THREADS) {
      const size_t p = (size_t)j * (g.nx + 2) + i;
      if (!BMG_IN(DBG_PERIODIC, p, g.ps())) continue;
      x[p] = madd<FU>(x[p], alpha, pv[p]);
      const double rr = msub<FU>(r[p], alpha, q[p]);
      r[p] = rr;
      z[p] = 0.0;
      acc = madd<FU>(acc, rr, rr);
    }
  const double tot = dev::block_sum(acc);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = tot;
    if (blockIdx.x == 0) {
      ctl->pq_prev = ctl->pq;
      ctl->first = 0;
    }
  }
}

dim3 pgrid(int nx, int ny) { return dim3((unsigned)((nx + PBX - 1) / PBX), (unsigned)((ny + PBY - 1) / PBY)); }

int m_of(int n, int periodic) {
  const int v = periodic ? n : n + 1;
  if (v < 4 || (v & (v - 1))) return -1;
  int m = 0;
  while ((1 << m) < v) ++m;
  return m;
}

}  // namespace

struct PerLevel {
  PGeom g{};
  int kind = 9;
  double* st = nullptr;   // O, W, S, SW, NW, D
  double* ci = nullptr;   // weights toward the next level
  double* x = nullptr;    // iterate and right-hand side of a coarse level
  double* f = nullptr;
  double* r = nullptr;    // residual of a level above the coarsest
  double* xb = nullptr;   // second iterate for strip sweeps (9-point levels above the coarsest)
  int ty = 0;             // strip height
  bool strip = false;     // swept by the strip kernel (else by the row-parity pair, in place)
};

struct PerHier {
  int periodic = 0, fused = 0, nu1 = 2, nu2 = 1, krylov = 0;
  std::vector<PerLevel> lv;
  double* kr = nullptr;   // FCG: r, z, p, q on level 0's layout (krylov)
  double* L = nullptr;
  double* work = nullptr;
  int* err = nullptr;
};

// The smallest even strip height whose strips fit into one wave of the strip
// kernel's resident warps (a warp walks its strip serially; a partial second
// wave would leave most FP64 pipes idle).
static int strip_height(const PGeom& g, int fused) {
  auto k = fused ? k_p_gs_strip<true> : k_p_gs_strip<false>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P_STRIP_SMEM);
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * P_STRIP_WARPS, P_STRIP_SMEM);
  const int resident = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1) * P_STRIP_WARPS;
  const int nbx = (g.nx + 55) / 56;
  const int nby_max = resident / nbx > 1 ? resident / nbx : 1;
  const int half = (g.ny + 2 * nby_max - 1) / (2 * nby_max);
  return 2 * (half > 1 ? half : 1);
}

int per_levels_for(int nx, int ny, int periodic) {
  const int mx = m_of(nx, periodic & 1), my = m_of(ny, periodic & 2);
  if (mx < 2 || mx != my) return 0;
  return mx - 1;   // m, m-1, ..., 2
}

static int palloc(double** p, size_t count, cudaStream_t s) {
  *p = nullptr;
  if (dev_malloc((void**)p, count * sizeof(double)) != cudaSuccess) {
    *p = nullptr;
    return set_error(BMG_ENOMEM, "periodic setup: device allocation of %zu doubles failed", count);
  }
  return cuda_check(cudaMemsetAsync(*p, 0, count * sizeof(double), s), "periodic setup: memset");
}

void per_free(PerHier* P) {
  if (!P) return;
  for (PerLevel& L : P->lv) {
    cudaFree(L.st);
    cudaFree(L.ci);
    cudaFree(L.x);
    cudaFree(L.f);
    cudaFree(L.r);
    cudaFree(L.xb);
  }
  cudaFree(P->L);
  cudaFree(P->work);
  cudaFree(P->err);
  cudaFree(P->kr);
  delete P;
}

namespace {
template <bool FU>
double* per_sweep(const PerLevel& L, const double* f, double* x, double* home, const int* done, cudaStream_t s);

// The sweep of each 9-point level: the strip walk or the row-parity pair,
// whichever takes less time here over 3 sweeps (after one untimed), run on
// zero data in the level's scratch arrays (r as iterate and right-hand side,
// xb; both stay zero).
int tune_sweeps(PerHier* P, cudaStream_t s) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = cuda_check(cudaEventCreate(&e0), "periodic setup: event");
  if (!rc) rc = cuda_check(cudaEventCreate(&e1), "periodic setup: event");
  for (PerLevel& L : P->lv) {
    if (rc || !L.xb) continue;
    float t[2] = {0.f, 0.f};
    for (int k = 0; k < 2 && !rc; ++k) {
      L.strip = k == 0;
      auto sweep = [&](double* x) {
        return P->fused ? per_sweep<true>(L, L.r, x, L.r, nullptr, s) : per_sweep<false>(L, L.r, x, L.r, nullptr, s);
      };
      double* x = sweep(L.r);
      cudaEventRecord(e0, s);
      for (int q = 0; q < 3; ++q) x = sweep(x);
      cudaEventRecord(e1, s);
      rc = cuda_check(cudaEventSynchronize(e1), "periodic setup: sweep timing");
      if (!rc) rc = cuda_check(cudaEventElapsedTime(&t[k], e0, e1), "periodic setup: sweep timing");
    }
    L.strip = t[0] <= t[1];
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return rc;
}
}  // namespace

int per_setup(PerHier** out, int kind, const double* coef, int nx, int ny, int periodic, int fused, int nu1,
              int nu2, int sweep, int krylov, cudaStream_t s) {
  *out = nullptr;
  const int nlev = per_levels_for(nx, ny, periodic);
  if (nlev < 1)
    return set_error(BMG_EINVAL,
                     "bmg_setup: %d x %d with periodic flags %d: a periodic axis needs 2^m points, a Dirichlet "
                     "axis 2^m - 1, both axes the same m >= 2",
                     nx, ny, periodic);
  PerHier* P = new PerHier();
  P->periodic = periodic;
  P->fused = fused;
  P->nu1 = nu1;
  P->nu2 = nu2;
  P->krylov = krylov;
  P->lv.resize(nlev);
  const int px = periodic & 1 ? 1 : 0, py = periodic & 2 ? 1 : 0;
  int rc = BMG_OK;
  for (int l = 0; l < nlev && !rc; ++l) {
    PerLevel& L = P->lv[l];
    L.g = l == 0 ? PGeom{nx, ny, px, py} : PGeom{coarse_n(P->lv[l - 1].g.nx, px), coarse_n(P->lv[l - 1].g.ny, py), px, py};
    L.kind = l == 0 ? kind : 9;
    const size_t ps = L.g.ps();
    rc = palloc(&L.st, 6 * ps, s);
    if (!rc && l + 1 < nlev) {
      const size_t psc = (size_t)(coarse_n(L.g.nx, px) + 2) * (coarse_n(L.g.ny, py) + 2);
      rc = palloc(&L.ci, 8 * psc, s);
      if (!rc) rc = palloc(&L.r, ps, s);
    }
    if (!rc && sweep != PER_SWEEP_ROWS && l + 1 < nlev && L.kind == 9) rc = palloc(&L.xb, ps, s);
    if (!rc && l > 0) rc = palloc(&L.x, ps, s);
    if (!rc && l > 0) rc = palloc(&L.f, ps, s);
  }
  const PGeom gc = P->lv[nlev - 1].g;
  const int m = gc.nx * gc.ny;
  if (!rc) rc = palloc(&P->L, (size_t)m * m, s);
  if (!rc) rc = palloc(&P->work, (size_t)m * m, s);
  if (!rc && krylov) rc = palloc(&P->kr, 4 * P->lv[0].g.ps(), s);
  if (!rc && dev_malloc((void**)&P->err, sizeof(int)) != cudaSuccess) rc = set_error(BMG_ENOMEM, "periodic setup");
  if (!rc) rc = cuda_check(cudaMemsetAsync(P->err, 0, sizeof(int), s), "periodic setup: memset");
  if (rc) {
    per_free(P);
    return rc;
  }
  for (PerLevel& L : P->lv)
    if (L.xb) {
      L.ty = strip_height(L.g, fused);
      L.strip = true;
    }
  const PGeom g0 = P->lv[0].g;
  k_p_prepare<<<pgrid(g0.nx + 2, g0.ny + 2), dim3(PBX, PBY), 0, s>>>(g0, kind, coef, P->lv[0].st);
  count_launch();
  k_p_dinv<<<pgrid(g0.nx, g0.ny), dim3(PBX, PBY), 0, s>>>(g0, P->lv[0].st, P->err);
  count_launch();
  for (int l = 0; l + 1 < nlev; ++l) {
    PerLevel &F = P->lv[l], &C = P->lv[l + 1];
    const int ncx = C.g.nx, ncy = C.g.ny;
    k_p_dendy<<<pgrid(ncx + 2, ncy + 2), dim3(PBX, PBY), 0, s>>>(F.g, F.st, F.ci, P->err);
    count_launch();
    k_p_rap<<<pgrid(ncx + 2, ncy + 2), dim3(PBX, PBY), 0, s>>>(F.g, F.st, F.ci, C.st);
    count_launch();
    k_p_dinv<<<pgrid(ncx, ncy), dim3(PBX, PBY), 0, s>>>(C.g, C.st, P->err);
    count_launch();
  }
  k_p_factor<<<1, 1, 0, s>>>(gc, P->lv[nlev - 1].st, P->L, P->work, P->err);
  count_launch();
  int herr = 0;
  rc = cuda_check(cudaGetLastError(), "periodic setup");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(&herr, P->err, sizeof(int), cudaMemcpyDeviceToHost, s), "periodic setup");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "periodic setup");
  if (!rc && herr)
    rc = set_error(BMG_ESINGULAR, "periodic setup: non-positive %s (a grid periodic along both axes needs a "
                                  "non-singular operator)",
                   herr == 1 ? "diagonal" : herr == 2 ? "interpolation denominator" : "Cholesky pivot");
  if (!rc && sweep == PER_SWEEP_AUTO) rc = tune_sweeps(P, s);
  if (rc) {
    per_free(P);
    return rc;
  }
  *out = P;
  return BMG_OK;
}

namespace {

struct Bracket {
  const PerMarks* m;
  Bracket(const PerMarks* mk, int level, int kernel) : m(mk) {
    if (m && m->begin) m->begin(m->ctx, level, kernel);
  }
  ~Bracket() {
    if (m && m->end) m->end(m->ctx);
  }
};

// One sweep starting from x, which is the level's iterate `home` or its
// second iterate L.xb; returns the array holding the result: the other one of
// the two for a level swept by strips (one launch), x itself otherwise.
template <bool FU>
double* per_sweep(const PerLevel& L, const double* f, double* x, double* home, const int* done, cudaStream_t s) {
  if (L.strip) {
    double* out = x == L.xb ? home : L.xb;
    const int warps = ((L.g.nx + 55) / 56) * ((L.g.ny + L.ty - 1) / L.ty);
    k_p_gs_strip<FU><<<(warps + P_STRIP_WARPS - 1) / P_STRIP_WARPS, 32 * P_STRIP_WARPS, P_STRIP_SMEM, s>>>(
        L.g, L.st, f, x, out, L.ty, done);
    count_launch();
    return out;
  }
  // 9-point: the two row-parity halves; 5-point (level 0 only): one launch per
  // colour, red ((odd,odd), (even,even)) then black
  static const int c5[4][2] = {{1, 1}, {0, 0}, {0, 1}, {1, 0}};
  const bool nine = L.kind == 9;
  if (nine) {   // two row-parity halves
    for (int pj = 1; pj >= 0; --pj) {
      const int rows = pj ? (L.g.ny + 1) / 2 : L.g.ny / 2;
      k_p_gs_rows<FU><<<rows, 256, 0, s>>>(L.g, L.st, f, x, pj, done);
      count_launch();
    }
    return x;
  }
  for (int k = 0; k < 4; ++k) {
    const int pi = c5[k][0], pj = c5[k][1];
    const int cx = pi ? (L.g.nx + 1) / 2 : L.g.nx / 2, cy = pj ? (L.g.ny + 1) / 2 : L.g.ny / 2;
    k_p_gs<false, FU><<<pgrid(cx, cy), dim3(PBX, PBY), 0, s>>>(L.g, L.st, f, x, pi, pj, done);
    count_launch();
  }
  return x;
}

template <bool FU>
int per_residual(const PerLevel& L, const double* x, const double* f, double* r, double* partials, const int* done,
                 cudaStream_t s) {
  const int G = L.g.ny < dev::NORM_BLOCKS_MAX ? L.g.ny : dev::NORM_BLOCKS_MAX;
  if (L.kind == 9)
    k_p_residual<true, FU><<<G, dev::NORM_THREADS, 0, s>>>(L.g, L.st, x, f, r, partials, done);
  else
    k_p_residual<false, FU><<<G, dev::NORM_THREADS, 0, s>>>(L.g, L.st, x, f, r, partials, done);
  count_launch();
  return G;
}

template <bool FU>
void per_vcycle(PerHier* P, int l, double* x, const double* f, const int* done, cudaStream_t s,
                const PerMarks* mk) {
  PerLevel& L = P->lv[l];
  if (l + 1 == (int)P->lv.size()) {
    Bracket b(mk, l, BMG_K_COARSE);
    k_p_coarse_solve<<<1, 1, 0, s>>>(L.g, P->L, f, x, done);
    count_launch();
    return;
  }
  PerLevel& C = P->lv[l + 1];
  double* cur = x;                                // where the iterate is
  for (int k = 0; k < P->nu1; ++k) {
    Bracket b(mk, l, BMG_K_RELAX);
    cur = per_sweep<FU>(L, f, cur, x, done, s);
  }
  {
    Bracket b(mk, l, BMG_K_RESID_RESTRICT);
    per_residual<FU>(L, cur, f, L.r, nullptr, done, s);
    k_p_restrict<FU><<<pgrid(C.g.nx, C.g.ny), dim3(PBX, PBY), 0, s>>>(L.g, L.ci, L.r, C.f, C.x, done);
    count_launch();
  }
  per_vcycle<FU>(P, l + 1, C.x, C.f, done, s, mk);
  {
    // corrected iterate into the array from which the nu2 post-sweeps end in x
    Bracket b(mk, l, BMG_K_INTERP);
    double* dst = L.strip && (P->nu2 & 1) ? L.xb : x;
    k_p_interp<FU><<<pgrid(L.g.px ? C.g.nx : C.g.nx + 1, L.g.py ? C.g.ny : C.g.ny + 1), dim3(PBX, PBY), 0, s>>>(
        L.g, L.ci, C.x, cur, dst, done);
    count_launch();
    cur = dst;
  }
  for (int k = 0; k < P->nu2; ++k) {
    Bracket b(mk, l, BMG_K_RELAX);
    cur = per_sweep<FU>(L, f, cur, x, done, s);
  }
}

}  // namespace

void per_enqueue_initial(PerHier* P, const double* rhs, double* x, double* partials, Ctl* ctl, cudaStream_t s) {
  if (P->krylov) {
    const PerLevel& L = P->lv[0];
    const size_t ps = L.g.ps();
    const int G = L.g.ny < dev::NORM_BLOCKS_MAX ? L.g.ny : dev::NORM_BLOCKS_MAX;
    auto k = P->fused ? (L.kind == 9 ? k_p_fcg_init<true, true> : k_p_fcg_init<false, true>)
                      : (L.kind == 9 ? k_p_fcg_init<true, false> : k_p_fcg_init<false, false>);
    k<<<G, dev::NORM_THREADS, 0, s>>>(L.g, L.st, x, rhs, P->kr, P->kr + ps, partials, ctl);
    count_launch();
    launch_norm_finalize(partials, G, ctl, 0, nullptr, s);
    return;
  }
  const int G = P->fused ? per_residual<true>(P->lv[0], x, rhs, nullptr, partials, nullptr, s)
                         : per_residual<false>(P->lv[0], x, rhs, nullptr, partials, nullptr, s);
  launch_norm_finalize(partials, G, ctl, 0, nullptr, s);
}

namespace {
// One FCG step after the preconditioner z = V(r): z.q and beta, p, q = A p with
// p.q and p.r, then the x / r update with the r.r partial sums; returns G.
template <bool FU>
int per_fcg_step(PerHier* P, double* x, double* partials, Ctl* ctl, cudaStream_t s) {
  const PerLevel& L = P->lv[0];
  const size_t ps = L.g.ps();
  double *r = P->kr, *z = P->kr + ps, *pv = P->kr + 2 * ps, *q = P->kr + 3 * ps;
  const int G = L.g.ny < dev::NORM_BLOCKS_MAX ? L.g.ny : dev::NORM_BLOCKS_MAX;
  k_p_fcg_zq<FU><<<G, dev::NORM_THREADS, 0, s>>>(L.g, z, q, partials, ctl);
  count_launch();
  launch_fcg_reduce(partials, G, ctl, 0, s);
  k_p_fcg_direction<FU><<<pgrid(L.g.nx, L.g.ny), dim3(PBX, PBY), 0, s>>>(L.g, z, pv, ctl);
  count_launch();
  if (L.kind == 9)
    k_p_fcg_matvec<true, FU><<<G, dev::NORM_THREADS, 0, s>>>(L.g, L.st, pv, r, q, partials, ctl);
  else
    k_p_fcg_matvec<false, FU><<<G, dev::NORM_THREADS, 0, s>>>(L.g, L.st, pv, r, q, partials, ctl);
  count_launch();
  launch_fcg_reduce(partials, G, ctl, 1, s);
  k_p_fcg_update<FU><<<G, dev::NORM_THREADS, 0, s>>>(L.g, x, r, pv, q, z, partials, ctl);
  count_launch();
  return G;
}
}  // namespace

void per_enqueue_iteration(PerHier* P, const double* rhs, double* x, double* partials, Ctl* ctl, cudaStream_t s,
                           const PerMarks* mk) {
  const int* done = &ctl->done;
  int G;
  if (P->krylov) {
    // z = V(r) from z = 0 (zeroed by the previous update or the initial step), then the FCG step
    const size_t ps = P->lv[0].g.ps();
    double *r = P->kr, *z = P->kr + ps;
    if (P->fused)
      per_vcycle<true>(P, 0, z, r, done, s, mk);
    else
      per_vcycle<false>(P, 0, z, r, done, s, mk);
    Bracket b(mk, 0, BMG_K_FCG);
    G = P->fused ? per_fcg_step<true>(P, x, partials, ctl, s) : per_fcg_step<false>(P, x, partials, ctl, s);
  } else {
    if (P->fused)
      per_vcycle<true>(P, 0, x, rhs, done, s, mk);
    else
      per_vcycle<false>(P, 0, x, rhs, done, s, mk);
    Bracket b(mk, 0, BMG_K_NORM);
    G = P->fused ? per_residual<true>(P->lv[0], x, rhs, nullptr, partials, done, s)
                 : per_residual<false>(P->lv[0], x, rhs, nullptr, partials, done, s);
  }
  Bracket b(mk, 0, BMG_K_FINALIZE);
  launch_norm_finalize(partials, G, ctl, 1, nullptr, s);
}

int per_num_levels(const PerHier* P) { return (int)P->lv.size(); }

int per_level_sweep(const PerHier* P, int l) {
  if (l < 0 || l + 1 >= (int)P->lv.size()) return 0;
  return P->lv[l].strip ? 2 : 1;
}

int per_level_shape(const PerHier* P, int l, int* nx, int* ny) {
  if (l < 0 || l >= (int)P->lv.size()) return set_error(BMG_EINVAL, "bmg_level_shape: bad level %d", l);
  if (nx) *nx = P->lv[l].g.nx;
  if (ny) *ny = P->lv[l].g.ny;
  return BMG_OK;
}

int per_get_stencil(const PerHier* P, int l, double* out, cudaStream_t s) {
  if (l < 0 || l >= (int)P->lv.size()) return set_error(BMG_EINVAL, "bmg_get_stencil: bad level %d", l);
  const PerLevel& L = P->lv[l];
  int rc = cuda_check(cudaMemcpyAsync(out, L.st, 5 * L.g.ps() * sizeof(double), cudaMemcpyDeviceToDevice, s),
                      "bmg_get_stencil");
  return rc ? rc : cuda_check(cudaStreamSynchronize(s), "bmg_get_stencil");
}

int per_get_interp(const PerHier* P, int l, double* out, cudaStream_t s) {
  if (l < 0 || l + 1 >= (int)P->lv.size()) return set_error(BMG_EINVAL, "bmg_get_interp: bad level %d", l);
  const PerLevel& C = P->lv[l + 1];
  int rc = cuda_check(cudaMemcpyAsync(out, P->lv[l].ci, 8 * C.g.ps() * sizeof(double), cudaMemcpyDeviceToDevice, s),
                      "bmg_get_interp");
  return rc ? rc : cuda_check(cudaStreamSynchronize(s), "bmg_get_interp");
}

}  // namespace bmg
