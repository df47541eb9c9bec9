// Device bodies of the V-cycle kernels, shared by the single-problem kernels
// (k_cycle.cu) and the batched kernels (k_batched.cu) so that both run the same
// arithmetic.  A body takes its block coordinates explicitly; a batched kernel
// picks its problem from another grid dimension and passes the rest through.
//
// T is the compute type (double or float); S the storage type of the
// off-diagonal stencil planes (T, or bf16 under float).  Every row sum runs in
// the order O, W, E, S, N, SW, NE, NW, SE with one rounding per operation.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"

namespace bmg {
namespace dev {

namespace cg = cooperative_groups;

constexpr int NORM_THREADS = 256;
constexpr int NORM_BLOCKS_MAX = 1024;
constexpr int TXC = 32, TYC = 8;                      // coarse tile of residual + restriction
constexpr int RFX = 2 * TXC + 1, RFY = 2 * TYC + 1;  // its fine block

__device__ __forceinline__ bool stopped(const int* done) { return done != nullptr && *done != 0; }

// s - sum over the listed neighbours of a(p,q) x_q (canonical order).
template <typename T, typename S, bool NINE, bool WITH_O, bool FU = false>
__device__ __forceinline__ T row_residual(const StencilView<T, S>& v, const T* __restrict__ x, size_t p, T s) {
  const int ld = v.ld;
  if (WITH_O) s = msub<FU>(s, v.O[p], x[p]);
  s = msub<FU>(s, cvt<T>(v.W[p]), x[p - 1]);
  s = msub<FU>(s, cvt<T>(v.W[p + 1]), x[p + 1]);
  s = msub<FU>(s, cvt<T>(v.S_[p]), x[p - ld]);
  s = msub<FU>(s, cvt<T>(v.S_[p + ld]), x[p + ld]);
  if (NINE) {
    s = msub<FU>(s, cvt<T>(v.SW[p]), x[p - ld - 1]);
    s = msub<FU>(s, cvt<T>(v.SW[p + ld + 1]), x[p + ld + 1]);
    s = msub<FU>(s, cvt<T>(v.NW[p]), x[p + ld - 1]);
    s = msub<FU>(s, cvt<T>(v.NW[p + 1 - ld]), x[p + 1 - ld]);
  }
  return s;
}

// ---- Gauss-Seidel ------------------------------------------------------------------
// One update: x_p = (f_p - sum_{q != p} a_pq x_q) * d_p, d_p = 1/a_pp (stored, or
// formed here with the same correctly rounded quotient).
template <typename T, typename S, bool NINE, bool FU = false>
__device__ __forceinline__ void gs_point(const StencilView<T, S>& v, const T* __restrict__ f, T* x, size_t p) {
  T s = row_residual<T, S, NINE, false, FU>(v, x, p, f[p]);
  T d = v.D ? v.D[p] : rdiv(T(1), v.O[p]);
  if (BMG_IN(DBG_GS_STORE, p, (size_t)(v.n + 2) * v.ld)) x[p] = rmul(s, d);
}

template <typename T>
struct PairLoads {
  T f, d, c[8], xs[8];
};

template <typename T, typename S>
__device__ __forceinline__ void load_point(const StencilView<T, S>& v, const T* __restrict__ f, const T* x, size_t p,
                                           PairLoads<T>& L, bool same_row_x) {
  const int ld = v.ld;
  L.f = f[p];
  L.d = v.D ? v.D[p] : rdiv(T(1), v.O[p]);
  L.c[0] = cvt<T>(v.W[p]);
  L.c[1] = cvt<T>(v.W[p + 1]);
  L.c[2] = cvt<T>(v.S_[p]);
  L.c[3] = cvt<T>(v.S_[p + ld]);
  L.c[4] = cvt<T>(v.SW[p]);
  L.c[5] = cvt<T>(v.SW[p + ld + 1]);
  L.c[6] = cvt<T>(v.NW[p]);
  L.c[7] = cvt<T>(v.NW[p + 1 - ld]);
  if (same_row_x) {
    L.xs[0] = x[p - 1];
    L.xs[1] = x[p + 1];
  }
  L.xs[2] = x[p - ld];
  L.xs[3] = x[p + ld];
  L.xs[4] = x[p - ld - 1];
  L.xs[5] = x[p + ld + 1];
  L.xs[6] = x[p + ld - 1];
  L.xs[7] = x[p + 1 - ld];
}

// (f - sum_k c_k xs_k) * d in the canonical neighbour order W, E, S, N, SW, NE, NW, SE.
template <typename T, bool FU = false>
__device__ __forceinline__ T update_from(const PairLoads<T>& L) {
  T s = L.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s = msub<FU>(s, L.c[k], L.xs[k]);
  return rmul(s, L.d);
}

template <typename T>
constexpr int rows_threads_max() { return sizeof(T) == 8 ? 512 : 1024; }

// Four-colour sweep, half of it: the rows j with j % 2 == pj.  Rows j +- 1
// belong to the other parity and are not written by this launch, so a row is
// independent of every other row here.  Thread t owns the pair of points
// (i0, i1) = (2t+1, 2t+2) of the row and issues every load of both updates at
// once; it updates the odd-i point i0 (its same-row neighbours are even-i
// points, still old), publishes the new value in shared memory, and after the
// barrier updates the even-i point i1 with the new values at i1 - 1 (its own)
// and i1 + 1 (the next thread's).  Launching pj = 1 then pj = 0 gives the colour
// order (odd,odd), (even,odd), (odd,even), (even,even).  A row longer than one
// CTA is split over a cluster of CL CTAs along x; the pair at a CTA's last
// thread reads its right neighbour from the next CTA's shared memory after
// cluster.sync().  `bx` is the CTA's x index; the caller has already returned
// from CTAs whose problem is finished (uniformly over the cluster).
template <typename T, typename S, int CL, bool FU = false>
__device__ __forceinline__ void gs_rows_body(const StencilView<T, S>& v, const T* __restrict__ f, T* x, int pj,
                                             int bx) {
  __shared__ T xo[rows_threads_max<T>()];
  const int n = v.n, ld = v.ld;
  const int rowid = bx / CL, seg = bx % CL;
  const int j = 2 * rowid + (pj ? 1 : 2);
  const int t = seg * blockDim.x + threadIdx.x;
  const int i0 = 2 * t + 1, i1 = i0 + 1;
  const bool has0 = i0 <= n && j <= n, has1 = i1 < n && j <= n;
  const size_t p0 = (size_t)j * ld + i0, p1 = p0 + 1;
  PairLoads<T> A, B;
  if (has0) load_point(v, f, x, p0, A, true);
  if (has1) load_point(v, f, x, p1, B, false);
  if (has0) {
    T xn = update_from<T, FU>(A);
    if (BMG_IN(DBG_GS_STORE, p0, (size_t)(n + 2) * ld)) x[p0] = xn;
    xo[threadIdx.x] = xn;
    B.xs[0] = xn;
  }
  T right = T(0);
  if constexpr (CL == 1) {
    __syncthreads();
    if (has1) right = xo[threadIdx.x + 1];
  } else {
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();
    if (has1) {
      if (threadIdx.x + 1 < blockDim.x)
        right = xo[threadIdx.x + 1];
      else
        right = *cluster.map_shared_rank(&xo[0], (int)cluster.block_rank() + 1);
    }
    cluster.sync();   // keep every CTA's shared memory alive until its neighbour has read it
  }
  if (has1) {
    B.xs[1] = right;
    const T xn = update_from<T, FU>(B);
    if (BMG_IN(DBG_GS_STORE, p1, (size_t)(n + 2) * ld)) x[p1] = xn;
  }
}

// ---- zebra x-line Gauss-Seidel ------------------------------------------------------------
// Row j solved exactly along x with the rows j - 1, j + 1 held fixed: right-hand
// side g = f - (S, N, SW, NE, NW, SE couplings) x in that order (5-point
// stencils: S, N only), then the Thomas algorithm: m = a_O - a_W c', c' = a_E / m,
// d' = (g - a_W d') / m forward (c' into cp, d' into x), x_i = d'_i - c'_i x_{i+1}
// backward.  One rounding per operation, correctly rounded quotients.
template <typename T, typename S, bool NINE>
__device__ __forceinline__ void line_row_body(const StencilView<T, S>& v, const T* __restrict__ f, T* x,
                                              T* __restrict__ cp, int j) {
  const int n = v.n, ld = v.ld;
  const size_t r0 = (size_t)j * ld;
  T c = T(0), d = T(0);
  for (int i = 1; i <= n; ++i) {
    const size_t p = r0 + i;
    T g = f[p];
    g = rsub(g, rmul(cvt<T>(v.S_[p]), x[p - ld]));
    g = rsub(g, rmul(cvt<T>(v.S_[p + ld]), x[p + ld]));
    if (NINE) {
      g = rsub(g, rmul(cvt<T>(v.SW[p]), x[p - ld - 1]));
      g = rsub(g, rmul(cvt<T>(v.SW[p + ld + 1]), x[p + ld + 1]));
      g = rsub(g, rmul(cvt<T>(v.NW[p]), x[p + ld - 1]));
      g = rsub(g, rmul(cvt<T>(v.NW[p + 1 - ld]), x[p + 1 - ld]));
    }
    const T aO = v.O[p], aW = cvt<T>(v.W[p]), aE = cvt<T>(v.W[p + 1]);
    if (i == 1) {
      c = rdiv(aE, aO);
      d = rdiv(g, aO);
    } else {
      const T m = rsub(aO, rmul(aW, c));
      c = rdiv(aE, m);
      d = rdiv(rsub(g, rmul(aW, d)), m);
    }
    if (BMG_IN(DBG_LINE_STORE, p, (size_t)(n + 2) * ld)) {
      cp[p] = c;
      x[p] = d;
    }
  }
  for (int i = n - 1; i >= 1; --i) {
    const size_t p = r0 + i;
    if (BMG_IN(DBG_LINE_STORE, p, (size_t)(n + 2) * ld)) x[p] = rsub(x[p], rmul(cp[p], x[p + 1]));
  }
}

// Column i of a zebra y-line sweep: the x-line solve with the axes exchanged.
// Right-hand side f minus the couplings to columns i - 1, i + 1 in the order
// W, E, SW, NE, SE, NW; Thomas elimination from j = 1 upward with sub-diagonal
// a_S and super-diagonal a_N, then back substitution; one rounding per operation.
template <typename T, typename S, bool NINE>
__device__ __forceinline__ void line_col_body(const StencilView<T, S>& v, const T* __restrict__ f, T* x,
                                              T* __restrict__ cp, int i) {
  const int n = v.n, ld = v.ld;
  T c = T(0), d = T(0);
  for (int j = 1; j <= n; ++j) {
    const size_t p = (size_t)j * ld + i;
    T g = f[p];
    g = rsub(g, rmul(cvt<T>(v.W[p]), x[p - 1]));
    g = rsub(g, rmul(cvt<T>(v.W[p + 1]), x[p + 1]));
    if (NINE) {
      g = rsub(g, rmul(cvt<T>(v.SW[p]), x[p - ld - 1]));
      g = rsub(g, rmul(cvt<T>(v.SW[p + ld + 1]), x[p + ld + 1]));
      g = rsub(g, rmul(cvt<T>(v.NW[p + 1 - ld]), x[p + 1 - ld]));
      g = rsub(g, rmul(cvt<T>(v.NW[p]), x[p + ld - 1]));
    }
    const T aO = v.O[p], aS = cvt<T>(v.S_[p]), aN = cvt<T>(v.S_[p + ld]);
    if (j == 1) {
      c = rdiv(aN, aO);
      d = rdiv(g, aO);
    } else {
      const T m = rsub(aO, rmul(aS, c));
      c = rdiv(aN, m);
      d = rdiv(rsub(g, rmul(aS, d)), m);
    }
    if (BMG_IN(DBG_LINE_STORE, p, (size_t)(n + 2) * ld)) {
      cp[p] = c;
      x[p] = d;
    }
  }
  for (int j = n - 1; j >= 1; --j) {
    const size_t p = (size_t)j * ld + i;
    if (BMG_IN(DBG_LINE_STORE, p, (size_t)(n + 2) * ld)) x[p] = rsub(x[p], rmul(cp[p], x[p + ld]));
  }
}

// Red-black half sweep for 5-point stencils: the points with (i + j) % 2 == c
// (c = 0 red, c = 1 black), which share no coupling.  Thread grid: x over the
// points of a row, y over rows.
template <typename T, typename S, bool FU = false>
__device__ __forceinline__ void gs_checker_body(const StencilView<T, S>& v, const T* __restrict__ f, T* x, int c,
                                                int bx, int by) {
  const int n = v.n;
  const int j = by * blockDim.y + threadIdx.y + 1;
  if (j > n) return;
  const int i = 2 * (bx * blockDim.x + threadIdx.x) + 1 + ((j + 1 + c) & 1);
  if (i > n) return;
  gs_point<T, S, false, FU>(v, f, x, (size_t)j * v.ld + i);
}

// ---- four-colour sweep in one pass (FP32 compute): warp strips ------------------------
// A warp owns the strip of 56 x TY points i in [i0, i0 + 56), j in [j0, j1),
// i0 = 1 + 56 sx, j0 = 1 + TY sy, j1 = j0 + TY (i0, j0 odd; TY even), and
// produces the values the colour-by-colour sweep leaves there.  Lane l holds
// the local columns c = 2l (odd i) and 2l + 1 (even i), c = i - (i0 - 4), so
// the warp covers i in [i0 - 4, i0 + 60).  A colour's update at p reads the
// new values of the earlier colours and the old values of the later ones, so
// each colour is computed on the columns its successors read:
//   c1 (odd i, odd j)    on c in [2, 62]     c3 (odd i, even j)   on c in [4, 60]
//   c2 (even i, odd j)   on c in [3, 61]     c4 (even i, even j)  on c in [5, 59]
// and the warp walks down its rows: the odd row a (c1 then c2, reading the old
// even rows a +- 1), then the even row a - 1 (c3 then c4, reading the new odd
// rows a - 2 and a).  The odd rows j0 and j1 border the strips above and below
// and are computed by both.  Every recomputed value takes the same operands in
// the same order as in the colour-by-colour sweep, so it is bit-identical;
// values come from xin and the strip's points go to xout (xout != xin), so no
// warp reads what another wrote in this launch.  Same-row neighbours come from
// the adjacent lane by shuffle; the rows a - 2 .. a + 1 live in registers and
// the rows a + 2, a + 3 are loaded while row a is computed.
template <typename T, typename S>
struct StripRowT {          // one row of the strip: lane values at c = 2l (.a) and 2l + 1 (.b)
  T xa, xb, fa, fb, da, db;
  S wa, wb, sa, sb, swa, swb, nwa, nwb;
};
template <typename S>
using StripRow = StripRowT<float, S>;

template <typename S>
__device__ __forceinline__ void strip_load(const StencilView<float, S>& v, const float* __restrict__ f,
                                           const float* __restrict__ xin, int ic, int j, StripRow<S>& R) {
  // ic: absolute i of this lane's column c = 2l
  const int n = v.n, ld = v.ld;
  const bool rowin = j <= n + 1;
  const bool ina = rowin && ic >= 0 && ic <= n + 1, inb = rowin && ic + 1 >= 0 && ic + 1 <= n + 1;
  const size_t pa = ina ? (size_t)j * ld + ic : 0, pb = inb ? (size_t)j * ld + ic + 1 : 0;
  R.xa = ina ? xin[pa] : 0.f;
  R.xb = inb ? xin[pb] : 0.f;
  R.fa = ina ? f[pa] : 0.f;
  R.fb = inb ? f[pb] : 0.f;
  R.da = ina ? v.D[pa] : 0.f;
  R.db = inb ? v.D[pb] : 0.f;
  R.wa = ina ? v.W[pa] : S(0.f);
  R.wb = inb ? v.W[pb] : S(0.f);
  R.sa = ina ? v.S_[pa] : S(0.f);
  R.sb = inb ? v.S_[pb] : S(0.f);
  R.swa = ina ? v.SW[pa] : S(0.f);
  R.swb = inb ? v.SW[pb] : S(0.f);
  R.nwa = ina ? v.NW[pa] : S(0.f);
  R.nwb = inb ? v.NW[pb] : S(0.f);
}

__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_dn1(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_up1(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_dn1(double v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// The two colours of row M (rows L below, U above): first the odd-i points
// (lane value a), then the even-i points (lane value b), each in the order
// W, E, S, N, SW, NE, NW, SE; oka / okb say whether this lane's points are
// updated.
template <typename T, typename S, bool FU = false>
__device__ __forceinline__ void strip_row(const StripRowT<T, S>& L, StripRowT<T, S>& M, const StripRowT<T, S>& U,
                                          bool oka, bool okb) {
  {   // odd-i point c = 2l: same-row neighbours c - 1 (lane l - 1's b) and c + 1 (own b)
    const T xw = shfl_up1(M.xb), xsw = shfl_up1(L.xb), xnw = shfl_up1(U.xb);
    T s = M.fa;
    s = msub<FU>(s, cvt<T>(M.wa), xw);
    s = msub<FU>(s, cvt<T>(M.wb), M.xb);
    s = msub<FU>(s, cvt<T>(M.sa), L.xa);
    s = msub<FU>(s, cvt<T>(U.sa), U.xa);
    s = msub<FU>(s, cvt<T>(M.swa), xsw);
    s = msub<FU>(s, cvt<T>(U.swb), U.xb);
    s = msub<FU>(s, cvt<T>(M.nwa), xnw);
    s = msub<FU>(s, cvt<T>(L.nwb), L.xb);
    const T xn = rmul(s, M.da);
    M.xa = oka ? xn : M.xa;
  }
  {   // even-i point c = 2l + 1: neighbours c - 1 (own a, new) and c + 1 (lane l + 1's a)
    const T xe = shfl_dn1(M.xa), we = shfl_dn1(cvt<T>(M.wa));
    const T xne = shfl_dn1(U.xa), swne = shfl_dn1(cvt<T>(U.swa));
    const T xse = shfl_dn1(L.xa), nwse = shfl_dn1(cvt<T>(L.nwa));
    T s = M.fb;
    s = msub<FU>(s, cvt<T>(M.wb), M.xa);
    s = msub<FU>(s, we, xe);
    s = msub<FU>(s, cvt<T>(M.sb), L.xb);
    s = msub<FU>(s, cvt<T>(U.sb), U.xb);
    s = msub<FU>(s, cvt<T>(M.swb), L.xa);
    s = msub<FU>(s, swne, xne);
    s = msub<FU>(s, cvt<T>(M.nwb), U.xa);
    s = msub<FU>(s, nwse, xse);
    const T xn = rmul(s, M.db);
    M.xb = okb ? xn : M.xb;
  }
}

template <typename T, typename S>
__device__ __forceinline__ void strip_store(T* __restrict__ xout, int n, int ld, int ic, int j, bool own,
                                            const StripRowT<T, S>& R) {
  if (!own || j > n) return;
  const size_t p = (size_t)j * ld + ic;
  if (ic <= n && BMG_IN(DBG_STRIP_STORE, p, (size_t)(n + 2) * ld)) xout[p] = R.xa;
  if (ic + 1 <= n && BMG_IN(DBG_STRIP_STORE, p + 1, (size_t)(n + 2) * ld)) xout[p + 1] = R.xb;
}

template <typename S, int TY, bool FU = false>
__device__ __forceinline__ void gs_strip_body(const StencilView<float, S>& v, const float* __restrict__ f,
                                              const float* __restrict__ xin, float* __restrict__ xout, int sx,
                                              int sy) {
  static_assert(TY % 2 == 0, "strip height must be even");
  const int n = v.n, ld = v.ld;
  const int lane = threadIdx.x & 31;
  const int i0 = 1 + 56 * sx, j0 = 1 + TY * sy, j1 = j0 + TY;
  const int ic = i0 - 4 + 2 * lane;                // i of this lane's odd column
  // update columns per colour (c = 2l or 2l + 1), clipped to the grid
  const bool in_a = ic >= 1 && ic <= n, in_b = ic + 1 >= 1 && ic + 1 <= n;
  const bool c1 = in_a && lane >= 1, c2 = in_b && lane >= 1 && lane <= 30;
  const bool c3 = in_a && lane >= 2 && lane <= 30, c4 = in_b && lane >= 2 && lane <= 29;
  const bool own = lane >= 2 && lane <= 29;        // c in [4, 59]: the strip's own columns
  StripRow<S> r0, r1, r2, r3, p0, p1;              // rows a - 2 .. a + 1 and a + 2, a + 3
  strip_load(v, f, xin, ic, j0 - 1, r1);
  strip_load(v, f, xin, ic, j0, r2);
  strip_load(v, f, xin, ic, j0 + 1, r3);
#pragma unroll 1
  for (int m = 0; m <= TY / 2; ++m) {
    const int a = j0 + 2 * m;                      // odd row
    if (m < TY / 2) {
      strip_load(v, f, xin, ic, a + 2, p0);
      strip_load(v, f, xin, ic, a + 3, p1);
    }
    if (a <= n) {
      strip_row<float, S, FU>(r1, r2, r3, c1, c2);               // row a: c1, c2
      if (a < j1) strip_store(xout, n, ld, ic, a, own, r2);
    }
    if (m >= 1 && a - 1 <= n) {
      strip_row<float, S, FU>(r0, r1, r2, c3, c4);               // row a - 1: c3, c4
      strip_store(xout, n, ld, ic, a - 1, own, r1);
    }
    r0 = r2;
    r1 = r3;
    r2 = p0;
    r3 = p1;
  }
}

// ---- the strip walk fed by bulk copies -------------------------------------------------
// The same walk, with the strip's rows streamed into a per-warp ring of RING
// row slots in shared memory by bulk asynchronous copies (three copies per
// row: x, f and the level's packed stencil, one point's d, w, s, sw, nw
// together; one mbarrier per slot counts the bytes), so that rows are
// requested RING/2 steps before they are used without holding them in
// registers.  Few large copies matter: the copy unit accepts them at a
// limited rate, and seven copies per row (one per array) kept the warps
// waiting on the copy issue more than on the data.  A copy must start on a
// 16-byte boundary: each row segment is copied from the point at or below its
// first column whose index is a multiple of 4 (at most 3 points earlier) for
// 68 points, which requires every array base to be 16-byte aligned with
// STRIP_GUARD readable points before and after it.  A wait that does not complete within STRIP_WAIT_NS (or
// STRIP_WAIT_LIMIT polls) sets
// strip_timeout, waits (bounded) for the warp's copies in flight and returns.
constexpr long STRIP_WAIT_LIMIT = 1L << 20;                 // polls
constexpr unsigned long long STRIP_WAIT_NS = 500000000ull;   // 0.5 s

template <typename S>
struct StripRing {
  static constexpr int CP = 68;                                     // points copied per row segment
  static constexpr int PK = sizeof(S) == 4 ? PK_WORDS_F32 : PK_WORDS_BF16;   // packed words per point
  static constexpr unsigned BF = CP * 4, BP = CP * PK * 4;          // bytes (multiples of 16)
  static constexpr unsigned SLOT = 2 * BF + BP;                     // one row: x, f, packed stencil
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// true once phase `parity` of bar has completed; the warp may be suspended up
// to about STRIP_SUSPEND_NS while it is pending
constexpr unsigned STRIP_SUSPEND_NS = 1000;
__device__ __forceinline__ bool mbar_try(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "n"(STRIP_SUSPEND_NS)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}

// Warp-uniform bounded wait for phase `parity` of bar: false once
// STRIP_WAIT_NS of wall-clock time or STRIP_WAIT_LIMIT polls have passed.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  if (__all_sync(0xffffffffu, mbar_try(bar, parity))) return true;   // the usual case: the row is there
  const unsigned long long t0 = global_ns();
  for (long it = 0; it < STRIP_WAIT_LIMIT; ++it) {
    if (__all_sync(0xffffffffu, mbar_try(bar, parity))) return true;
    if (__any_sync(0xffffffffu, global_ns() - t0 > STRIP_WAIT_NS)) break;
  }
  return false;
}

struct StripSrc {           // the 3 arrays the walk reads
  const float *x, *f, *pk;
};

// Request row j into `slot`, called by the whole warp: lane 0 arms the slot's
// mbarrier for the row's bytes, then lanes 0, 1, 2 copy the row segments of
// x, f and the packed stencil.  The caller's __syncwarp orders the warp's
// earlier reads of the slot before the fences.
template <typename S>
__device__ __forceinline__ void ring_issue_warp(const StripSrc& A, int ld, int icol, int j, unsigned char* slot,
                                                unsigned long long* bar) {
  using RG = StripRing<S>;
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(bar, RG::SLOT);
  }
  __syncwarp();
  if (lane < 3) {
    const long long e = (long long)j * ld + icol;   // first point of the row segment
    const long long e4 = e - (e & 3);
    // (debug builds: a segment outside the array's guarded extent is read from its start instead)
    const long long s4 =
        BMG_IN_RANGE(DBG_RING_COPY, e4, -STRIP_GUARD, (long long)ld * ld + STRIP_GUARD - RG::CP + 1) ? e4 : 0;
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    if (lane < 2)
      bulk_copy(slot + lane * RG::BF, (lane == 0 ? A.x : A.f) + s4, RG::BF, bar);
    else
      bulk_copy(slot + 2 * RG::BF, A.pk + RG::PK * s4, RG::BP, bar);
  }
}

// every lane: its two columns of row j from a filled slot.  Columns or rows
// outside [0, n+1]^2 hold stale values: they feed only lanes and rows whose
// updates and stores are switched off.
__device__ __forceinline__ void packed_read(const float* q, float& d, float& w, float& s, float& sw, float& nw) {
  d = q[0];
  w = q[1];
  s = q[2];
  sw = q[3];
  nw = q[4];
}

// The BF16 halves widened to FP32 once, when the row is read (exact), so that
// the walk's row sums take FP32 coefficients from registers.
__device__ __forceinline__ void packed_read_wide(const float* q, bool bf16, float& d, float& w, float& s, float& sw,
                                                 float& nw) {
  if (!bf16) {
    packed_read(q, d, w, s, sw, nw);
    return;
  }
  const unsigned* u = reinterpret_cast<const unsigned*>(q);
  d = __uint_as_float(u[0]);
  const unsigned a = u[1], b = u[2];
  w = __uint_as_float(a << 16);
  s = __uint_as_float(a & 0xffff0000u);
  sw = __uint_as_float(b << 16);
  nw = __uint_as_float(b & 0xffff0000u);
}

// A row of the walk with every value in FP32 (BF16 coefficients widened).
using StripRowW = StripRowT<float, float>;

template <typename S>
__device__ __forceinline__ void ring_read(const unsigned char* slot, int ld, int icol, int ic, int j, StripRowW& R) {
  using RG = StripRing<S>;
  const long long e = (long long)j * ld + icol;
  const int o = (int)(e & 3) + (ic - icol);
  const float* xf = reinterpret_cast<const float*>(slot);
  const float* ff = reinterpret_cast<const float*>(slot + RG::BF);
  const float* pq = reinterpret_cast<const float*>(slot + 2 * RG::BF) + RG::PK * o;
  constexpr bool BF = sizeof(S) == 2;
  R.xa = xf[o];
  R.xb = xf[o + 1];
  R.fa = ff[o];
  R.fb = ff[o + 1];
  packed_read_wide(pq, BF, R.da, R.wa, R.sa, R.swa, R.nwa);
  packed_read_wide(pq + RG::PK, BF, R.db, R.wb, R.sb, R.swb, R.nwb);
}


// The strip height ty (even, >= 2) is a launch argument, as in the FP64 sweep.
template <typename S, int RING, bool FU = false>
__device__ __forceinline__ bool gs_strip_ring_body(const StencilView<float, S>& v, const float* __restrict__ f,
                                                   const float* __restrict__ xin, float* __restrict__ xout,
                                                   int sx, int sy, int ty, unsigned char* ring,
                                                   unsigned long long* bars) {
  static_assert(RING % 2 == 0 && RING >= 4, "ring size");
  using RG = StripRing<S>;
  const int n = v.n, ld = v.ld;
  const int lane = threadIdx.x & 31;
  const int i0 = 1 + 56 * sx, j0 = 1 + ty * sy, j1 = j0 + ty;
  const int icol = i0 - 4, ic = icol + 2 * lane;
  const bool in_a = ic >= 1 && ic <= n, in_b = ic + 1 >= 1 && ic + 1 <= n;
  const bool c1 = in_a && lane >= 1, c2 = in_b && lane >= 1 && lane <= 30;
  const bool c3 = in_a && lane >= 2 && lane <= 30, c4 = in_b && lane >= 2 && lane <= 29;
  const bool own = lane >= 2 && lane <= 29;
  const StripSrc A{xin, f, static_cast<const float*>(v.pk)};
  const int NR = ty + 3;                          // band rows q = 0 .. NR - 1, j = j0 - 1 + q
  const int last = (n + 1) - (j0 - 1);            // rows q > last lie outside the grid: never copied
  auto valid = [&](int q) { return q < NR && q <= last; };
  if (lane == 0) {
    for (int k = 0; k < RING; ++k) mbar_init(&bars[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncwarp();
  for (int q = 0; q < RING; ++q)
    if (valid(q)) ring_issue_warp<S>(A, ld, icol, j0 - 1 + q, ring + q * RG::SLOT, &bars[q]);
  bool ok = true;
  int taken = 0;                                  // rows 0 .. taken-1 read; rows < taken + RING requested
  // read band row q into R (waiting for its slot), then hand the slot to row q + RING
  auto take = [&](int q, StripRowW& R) {
    const int slot = q % RING;
    if (valid(q) && ok) ok = mbar_wait(&bars[slot], (unsigned)((q / RING) & 1));
    if (!ok) return;
    ring_read<S>(ring + slot * RG::SLOT, ld, icol, ic, j0 - 1 + q, R);
    taken = q + 1;
    __syncwarp();
    if (valid(q) && valid(q + RING))
      ring_issue_warp<S>(A, ld, icol, j0 - 1 + q + RING, ring + slot * RG::SLOT, &bars[slot]);
  };
  StripRowW P0, P1, Q0, Q1;                     // two row pairs in alternating roles
  take(0, P1);
  take(1, Q0);
  take(2, Q1);
  if (ok && j0 <= n) {
    strip_row<float, float, FU>(P1, Q0, Q1, c1, c2);                // row j0: c1, c2
    strip_store(xout, n, ld, ic, j0, own, Q0);
  }
  // step m: old pair = rows a - 2, a - 1; new pair = rows a, a + 1 (band rows 2m + 1, 2m + 2)
  auto step = [&](int m, StripRowW& E0, StripRowW& E1, StripRowW& E2, StripRowW& E3) {
    const int a = j0 + 2 * m;
    take(2 * m + 1, E2);
    take(2 * m + 2, E3);
    if (!ok) return;
    if (a <= n) {
      strip_row<float, float, FU>(E1, E2, E3, c1, c2);              // row a: c1, c2
      if (a < j1) strip_store(xout, n, ld, ic, a, own, E2);
    }
    if (a - 1 <= n) {
      strip_row<float, float, FU>(E0, E1, E2, c3, c4);              // row a - 1: c3, c4
      strip_store(xout, n, ld, ic, a - 1, own, E1);
    }
  };
#pragma unroll 1
  for (int m = 1; m <= ty / 2 && ok; m += 2) {
    step(m, Q0, Q1, P0, P1);
    if (m + 1 <= ty / 2 && ok) step(m + 1, P0, P1, Q0, Q1);
  }
  if (!ok)                                        // drain the copies still in flight, bounded
    for (int q = taken; q < taken + RING; ++q)
      if (valid(q)) mbar_wait(&bars[q % RING], (unsigned)((q / RING) & 1));
  return ok;
}

// ---- two sweeps in one pass (temporal blocking) -----------------------------------------
// The strip walk with a second sweep one step behind the first: at the first
// sweep's odd row a the warp computes, in this order, sweep 1 on rows a (c1, c2)
// and a - 1 (c3, c4), then sweep 2 on rows a - 2 (c1, c2) and a - 3 (c3, c4).
// Sweep 2 reads only rows that sweep 1 has finished and updates them in place.
// Final values on columns [P, Q] need sweep-1 values on [P - 4, Q + 4] and old
// values on [P - 8, Q + 8], so a 64-column window yields 48 output columns
// (c in [8, 55]); a band of TY output rows reads its rows j0 - 3 .. j1 + 3.
// Both sweeps take the same operands in the same order as two colour-by-colour
// sweeps, so the result is bit-identical to them.  Rows stream through the same
// per-warp ring as the single sweep; a row outside [0, n+1] is not copied, its
// slot's phase is completed by a plain arrive so that every slot's fills stay
// in order.
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

template <typename S, int RING, bool FU = false>
__device__ __forceinline__ bool gs_strip2_ring_body(const StencilView<float, S>& v, const float* __restrict__ f,
                                                    const float* __restrict__ xin, float* __restrict__ xout,
                                                    int sx, int sy, int ty, unsigned char* ring,
                                                    unsigned long long* bars) {
  static_assert(RING % 2 == 0 && RING >= 4, "ring size");
  using RG = StripRing<S>;
  const int n = v.n, ld = v.ld;
  const int lane = threadIdx.x & 31;
  const int i0 = 1 + 48 * sx, j0 = 1 + ty * sy, j1 = j0 + ty;
  const int icol = i0 - 8, ic = icol + 2 * lane;
  const bool in_a = ic >= 1 && ic <= n, in_b = ic + 1 >= 1 && ic + 1 <= n;
  // sweep 1 on c in [1, 62], sweep 2 on c in [5, 58]; the strip's own columns c in [8, 55]
  const bool p1 = in_a && lane >= 1, q1 = in_b && lane >= 1 && lane <= 30;
  const bool r1 = in_a && lane >= 2 && lane <= 30, t1 = in_b && lane >= 2 && lane <= 29;
  const bool p2 = in_a && lane >= 3 && lane <= 29, q2 = in_b && lane >= 3 && lane <= 28;
  const bool r2 = in_a && lane >= 4 && lane <= 28, t2 = in_b && lane >= 4 && lane <= 27;
  const bool own = lane >= 4 && lane <= 27;
  const StripSrc A{xin, f, static_cast<const float*>(v.pk)};
  const int NR = ty + 7;                      // band rows q = 0 .. NR - 1, j = j0 - 3 + q
  auto rowok = [&](int q) { const int j = j0 - 3 + q; return j >= 0 && j <= n + 1; };
  // the warp fills the slot of band row q (copies, or lane 0's plain arrive for
  // a row outside the grid)
  auto issue = [&](int q) {
    if (q >= NR) return;
    if (rowok(q))
      ring_issue_warp<S>(A, ld, icol, j0 - 3 + q, ring + (q % RING) * RG::SLOT, &bars[q % RING]);
    else if (lane == 0)
      mbar_arrive(&bars[q % RING]);
  };
  if (lane == 0) {
    for (int k = 0; k < RING; ++k) mbar_init(&bars[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncwarp();
  for (int q = 0; q < RING; ++q) issue(q);
  bool ok = true;
  int taken = 0;
  auto take = [&](int q, StripRowW& R) {
    const int slot = q % RING;
    if (ok) ok = mbar_wait(&bars[slot], (unsigned)((q / RING) & 1));
    if (!ok) return;
    ring_read<S>(ring + slot * RG::SLOT, ld, icol, ic, j0 - 3 + q, R);
    taken = q + 1;
    __syncwarp();
    issue(q + RING);
  };
  // step m on the rows a - 4 .. a + 1 held in R0 .. R5 (R4, R5 taken here for
  // m >= 1).  The rows move down by two per step, so the six registers sets
  // take their roles in a cycle of three steps instead of being copied.
  auto step = [&](int m, StripRowW& R0, StripRowW& R1, StripRowW& R2, StripRowW& R3, StripRowW& R4,
                  StripRowW& R5) {
    const int a = j0 - 2 + 2 * m, b = a - 2;      // sweep-1 and sweep-2 odd rows
    if (m >= 1) {
      take(2 * m + 1, R4);
      take(2 * m + 2, R5);
      if (!ok) return;
    }
    if (a >= 1 && a <= n) strip_row<float, float, FU>(R3, R4, R5, p1, q1);                 // sweep 1, row a
    if (m >= 1 && a - 1 >= 1 && a - 1 <= n) strip_row<float, float, FU>(R2, R3, R4, r1, t1);   // sweep 1, row a - 1
    if (m >= 2 && b <= n) {                                               // sweep 2, row a - 2
      strip_row<float, float, FU>(R1, R2, R3, p2, q2);
      if (b < j1) strip_store(xout, n, ld, ic, b, own, R2);
    }
    if (m >= 3 && b - 1 <= n) {                                           // sweep 2, row a - 3
      strip_row<float, float, FU>(R0, R1, R2, r2, t2);
      strip_store(xout, n, ld, ic, b - 1, own, R1);
    }
  };
  StripRowW S0, S1, S2, S3, S4, S5;
  take(0, S3);
  take(1, S4);
  take(2, S5);
  const int msteps = ty / 2 + 2;                  // steps m = 0 .. msteps
#pragma unroll 1
  for (int m = 0; m <= msteps && ok; m += 3) {
    step(m, S0, S1, S2, S3, S4, S5);
    if (m + 1 <= msteps && ok) step(m + 1, S2, S3, S4, S5, S0, S1);
    if (m + 2 <= msteps && ok) step(m + 2, S4, S5, S0, S1, S2, S3);
  }
  if (!ok)                                        // drain the copies still in flight, bounded
    for (int q = taken; q < taken + RING && q < NR; ++q) mbar_wait(&bars[q % RING], (unsigned)((q / RING) & 1));
  return ok;
}

// ---- one sweep of K right-hand sides of one operator per warp -------------------------------
// The walk of gs_strip_ring_body for K iterates that share a stencil (the
// members of a batch of right-hand sides): a row slot holds the packed
// stencil row once and the x and f rows of every member, so each stencil value
// is read once for the K right-hand sides; the coefficient shuffles are shared
// and the K members' row sums are independent chains.  Each member's
// operations and their order are those of strip_row, so every member's sweep
// is bit-identical to its own one-pass sweep.
template <int K>
struct StripRowK {
  float xa[K], xb[K], fa[K], fb[K];
  float da, db, wa, wb, sa, sb, swa, swb, nwa, nwb;
};

template <int K, bool FU>
__device__ __forceinline__ void strip_row_k(const StripRowK<K>& L, StripRowK<K>& M, const StripRowK<K>& U, bool oka,
                                            bool okb) {
#pragma unroll
  for (int q = 0; q < K; ++q) {   // odd-i points c = 2l
    const float xw = shfl_up1(M.xb[q]), xsw = shfl_up1(L.xb[q]), xnw = shfl_up1(U.xb[q]);
    float s = M.fa[q];
    s = msub<FU>(s, M.wa, xw);
    s = msub<FU>(s, M.wb, M.xb[q]);
    s = msub<FU>(s, M.sa, L.xa[q]);
    s = msub<FU>(s, U.sa, U.xa[q]);
    s = msub<FU>(s, M.swa, xsw);
    s = msub<FU>(s, U.swb, U.xb[q]);
    s = msub<FU>(s, M.nwa, xnw);
    s = msub<FU>(s, L.nwb, L.xb[q]);
    const float xn = rmul(s, M.da);
    M.xa[q] = oka ? xn : M.xa[q];
  }
  const float we = shfl_dn1(M.wa), swne = shfl_dn1(U.swa), nwse = shfl_dn1(L.nwa);
#pragma unroll
  for (int q = 0; q < K; ++q) {   // even-i points c = 2l + 1
    const float xe = shfl_dn1(M.xa[q]), xne = shfl_dn1(U.xa[q]), xse = shfl_dn1(L.xa[q]);
    float s = M.fb[q];
    s = msub<FU>(s, M.wb, M.xa[q]);
    s = msub<FU>(s, we, xe);
    s = msub<FU>(s, M.sb, L.xb[q]);
    s = msub<FU>(s, U.sb, U.xb[q]);
    s = msub<FU>(s, M.swb, L.xa[q]);
    s = msub<FU>(s, swne, xne);
    s = msub<FU>(s, M.nwb, U.xa[q]);
    s = msub<FU>(s, nwse, xse);
    const float xn = rmul(s, M.db);
    M.xb[q] = okb ? xn : M.xb[q];
  }
}

template <typename S, int K>
struct StripRingK {
  static constexpr unsigned SLOT = StripRing<S>::BP + 2 * K * StripRing<S>::BF;   // packed row, then x_q, f_q
};

// the warp requests row j: lane 0 copies the packed stencil segment, lanes
// 1 + 2q and 2 + 2q member q's x and f segments
template <typename S, int K>
__device__ __forceinline__ void ring_issue_warp_k(const float* pk, const float* const* xs, const float* const* fs,
                                                  int ld, int icol, int j, unsigned char* slot,
                                                  unsigned long long* bar) {
  using RG = StripRing<S>;
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(bar, StripRingK<S, K>::SLOT);
  }
  __syncwarp();
  if (lane <= 2 * K) {
    const long long e = (long long)j * ld + icol;
    const long long e4 = e - (e & 3);
    // (debug builds: a segment outside the array's guarded extent is read from its start instead)
    const long long s4 =
        BMG_IN_RANGE(DBG_RING_COPY, e4, -STRIP_GUARD, (long long)ld * ld + STRIP_GUARD - RG::CP + 1) ? e4 : 0;
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    if (lane == 0) {
      bulk_copy(slot, pk + RG::PK * s4, RG::BP, bar);
    } else {
      const int q = (lane - 1) >> 1;
      const float* src = (lane & 1) ? xs[q] : fs[q];
      bulk_copy(slot + RG::BP + (lane - 1) * RG::BF, src + s4, RG::BF, bar);
    }
  }
}

template <typename S, int K>
__device__ __forceinline__ void ring_read_k(const unsigned char* slot, int ld, int icol, int ic, int j,
                                            StripRowK<K>& R) {
  using RG = StripRing<S>;
  const long long e = (long long)j * ld + icol;
  const int o = (int)(e & 3) + (ic - icol);
  const float* pq = reinterpret_cast<const float*>(slot) + RG::PK * o;
  constexpr bool BF = sizeof(S) == 2;
  packed_read_wide(pq, BF, R.da, R.wa, R.sa, R.swa, R.nwa);
  packed_read_wide(pq + RG::PK, BF, R.db, R.wb, R.sb, R.swb, R.nwb);
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const float* xf = reinterpret_cast<const float*>(slot + RG::BP + 2 * q * RG::BF);
    const float* ff = reinterpret_cast<const float*>(slot + RG::BP + (2 * q + 1) * RG::BF);
    R.xa[q] = xf[o];
    R.xb[q] = xf[o + 1];
    R.fa[q] = ff[o];
    R.fb[q] = ff[o + 1];
  }
}

// xin, f, xout: the K members' arrays; member q's points are stored only if
// bit q of `active` is set (a converged member, or a padding slot of the last
// group, computes but writes nothing).
template <typename S, int K, int RING, bool FU>
__device__ __forceinline__ bool gs_strip_ring_k_body(const StencilView<float, S>& v, const float* const* f,
                                                     const float* const* xin, float* const* xout, unsigned active,
                                                     int sx, int sy, int ty, unsigned char* ring,
                                                     unsigned long long* bars) {
  static_assert(RING % 2 == 0 && RING >= 4, "ring size");
  constexpr unsigned SLOT = StripRingK<S, K>::SLOT;
  const int n = v.n, ld = v.ld;
  const int lane = threadIdx.x & 31;
  const int i0 = 1 + 56 * sx, j0 = 1 + ty * sy, j1 = j0 + ty;
  const int icol = i0 - 4, ic = icol + 2 * lane;
  const bool in_a = ic >= 1 && ic <= n, in_b = ic + 1 >= 1 && ic + 1 <= n;
  const bool c1 = in_a && lane >= 1, c2 = in_b && lane >= 1 && lane <= 30;
  const bool c3 = in_a && lane >= 2 && lane <= 30, c4 = in_b && lane >= 2 && lane <= 29;
  const bool own = lane >= 2 && lane <= 29;
  const float* pk = static_cast<const float*>(v.pk);
  const int NR = ty + 3;
  const int last = (n + 1) - (j0 - 1);
  auto valid = [&](int q) { return q < NR && q <= last; };
  if (lane == 0) {
    for (int k = 0; k < RING; ++k) mbar_init(&bars[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncwarp();
  for (int q = 0; q < RING; ++q)
    if (valid(q)) ring_issue_warp_k<S, K>(pk, xin, f, ld, icol, j0 - 1 + q, ring + q * SLOT, &bars[q]);
  bool ok = true;
  int taken = 0;
  auto take = [&](int q, StripRowK<K>& R) {
    const int slot = q % RING;
    if (valid(q) && ok) ok = mbar_wait(&bars[slot], (unsigned)((q / RING) & 1));
    if (!ok) return;
    ring_read_k<S, K>(ring + slot * SLOT, ld, icol, ic, j0 - 1 + q, R);
    taken = q + 1;
    __syncwarp();
    if (valid(q) && valid(q + RING))
      ring_issue_warp_k<S, K>(pk, xin, f, ld, icol, j0 - 1 + q + RING, ring + slot * SLOT, &bars[slot]);
  };
  auto store = [&](int j, const StripRowK<K>& R) {
    if (!own || j > n) return;
    const size_t p = (size_t)j * ld + ic;
#pragma unroll
    for (int q = 0; q < K; ++q) {
      if (!((active >> q) & 1u)) continue;
      if (ic <= n && BMG_IN(DBG_STRIP_STORE, p, (size_t)(n + 2) * ld)) xout[q][p] = R.xa[q];
      if (ic + 1 <= n && BMG_IN(DBG_STRIP_STORE, p + 1, (size_t)(n + 2) * ld)) xout[q][p + 1] = R.xb[q];
    }
  };
  StripRowK<K> P0, P1, Q0, Q1;
  take(0, P1);
  take(1, Q0);
  take(2, Q1);
  if (ok && j0 <= n) {
    strip_row_k<K, FU>(P1, Q0, Q1, c1, c2);
    store(j0, Q0);
  }
  auto step = [&](int m, StripRowK<K>& E0, StripRowK<K>& E1, StripRowK<K>& E2, StripRowK<K>& E3) {
    const int a = j0 + 2 * m;
    take(2 * m + 1, E2);
    take(2 * m + 2, E3);
    if (!ok) return;
    if (a <= n) {
      strip_row_k<K, FU>(E1, E2, E3, c1, c2);
      if (a < j1) store(a, E2);
    }
    if (a - 1 <= n) {
      strip_row_k<K, FU>(E0, E1, E2, c3, c4);
      store(a - 1, E1);
    }
  };
#pragma unroll 1
  for (int m = 1; m <= ty / 2 && ok; m += 2) {
    step(m, Q0, Q1, P0, P1);
    if (m + 1 <= ty / 2 && ok) step(m + 1, P0, P1, Q0, Q1);
  }
  if (!ok)
    for (int q = taken; q < taken + RING; ++q)
      if (valid(q)) mbar_wait(&bars[q % RING], (unsigned)((q / RING) & 1));
  return ok;
}

// ---- two sweeps, then the residual and its restriction, in one pass ---------------------
// The two-sweep walk, narrowed to 44 owned columns so that every owned coarse
// point's 3x3 fine footprint has final values around it: the window of 64
// columns starts 10 columns left of the strip (c = 0 .. 63), the strip owns
// c in [10, 53] and the coarse points at its even fine columns (c = 11, 13,
// .., 53), whose restriction reads residuals on [10, 54], which need final x
// on [9, 55] -- exactly where the two sweeps leave final values.  The walk
// starts one step earlier and runs three steps longer than the two-sweep
// pass, so that the final rows j0 - 1 .. j1 + 1 around the band exist; it
// reads the band's rows j0 - 5 .. j1 + 5.  At step m, after the sweeps, the
// residuals of rows b - 2 (odd) and b - 1 (even) are formed from final rows
// (b = a - 2, a the first sweep's odd row; the x and NW values of row b - 3
// are kept from the previous step), and the coarse row whose fine row is
// b - 3 is restricted from the residual rows b - 4, b - 3 (kept) and b - 2.
// Residual and restriction take the operands and the order of the separate
// residual + restriction kernel (r = f - a_O x - a_W x_W - ..., the nine terms
// of Fig. 2 left to right), so the coarse right-hand side is bit-identical.
// A slot holds x, f, the packed stencil and the diagonal a_O of one row.
struct StripRowR : StripRowW {
  float oa, ob;               // a_O at the lane's two columns
};

template <typename S>
struct StripRingR {
  static constexpr unsigned SLOT = StripRing<S>::SLOT + StripRing<S>::BF;   // + the a_O row segment
};

// residuals of row M from final values of rows L, M, U (the order of
// row_residual: O, W, E, S, N, SW, NE, NW, SE)
template <bool FU>
__device__ __forceinline__ void strip_resid(const StripRowW& L, const StripRowR& M, const StripRowW& U, float& ra,
                                            float& rb) {
  {   // odd-i point c = 2l
    const float xw = shfl_up1(M.xb), xsw = shfl_up1(L.xb), xnw = shfl_up1(U.xb);
    float s = M.fa;
    s = msub<FU>(s, M.oa, M.xa);
    s = msub<FU>(s, M.wa, xw);
    s = msub<FU>(s, M.wb, M.xb);
    s = msub<FU>(s, M.sa, L.xa);
    s = msub<FU>(s, U.sa, U.xa);
    s = msub<FU>(s, M.swa, xsw);
    s = msub<FU>(s, U.swb, U.xb);
    s = msub<FU>(s, M.nwa, xnw);
    s = msub<FU>(s, L.nwb, L.xb);
    ra = s;
  }
  {   // even-i point c = 2l + 1
    const float xe = shfl_dn1(M.xa), we = shfl_dn1(M.wa);
    const float xne = shfl_dn1(U.xa), swne = shfl_dn1(U.swa);
    const float xse = shfl_dn1(L.xa), nwse = shfl_dn1(L.nwa);
    float s = M.fb;
    s = msub<FU>(s, M.ob, M.xb);
    s = msub<FU>(s, M.wb, M.xa);
    s = msub<FU>(s, we, xe);
    s = msub<FU>(s, M.sb, L.xb);
    s = msub<FU>(s, U.sb, U.xb);
    s = msub<FU>(s, M.swb, L.xa);
    s = msub<FU>(s, swne, xne);
    s = msub<FU>(s, M.nwb, U.xa);
    s = msub<FU>(s, nwse, xse);
    rb = s;
  }
}

template <typename S>
__device__ __forceinline__ void ring_issue_warp_r(const StripSrc& A, const float* O, int ld, int icol, int j,
                                                  unsigned char* slot, unsigned long long* bar) {
  using RG = StripRing<S>;
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(bar, StripRingR<S>::SLOT);
  }
  __syncwarp();
  if (lane < 4) {
    const long long e = (long long)j * ld + icol;
    const long long e4 = e - (e & 3);
    // (debug builds: a segment outside the array's guarded extent is read from its start instead)
    const long long s4 =
        BMG_IN_RANGE(DBG_RING_COPY, e4, -STRIP_GUARD, (long long)ld * ld + STRIP_GUARD - RG::CP + 1) ? e4 : 0;
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    if (lane < 2)
      bulk_copy(slot + lane * RG::BF, (lane == 0 ? A.x : A.f) + s4, RG::BF, bar);
    else if (lane == 2)
      bulk_copy(slot + 2 * RG::BF, A.pk + RG::PK * s4, RG::BP, bar);
    else
      bulk_copy(slot + RG::SLOT, O + s4, RG::BF, bar);
  }
}

template <typename S>
__device__ __forceinline__ void ring_read_r(const unsigned char* slot, int ld, int icol, int ic, int j, StripRowR& R) {
  ring_read<S>(slot, ld, icol, ic, j, R);
  const long long e = (long long)j * ld + icol;
  const int o = (int)(e & 3) + (ic - icol);
  const float* of = reinterpret_cast<const float*>(slot + StripRing<S>::SLOT);
  R.oa = of[o];
  R.ob = of[o + 1];
}

// ci: the level's FP32 interpolation weights (8 planes of the coarse level);
// fc, xc: the coarse right-hand side (written on owned coarse points) and
// iterate (zeroed there).
template <typename S, int RING, bool FU = false>
__device__ __forceinline__ bool gs_strip2r_ring_body(const StencilView<float, S>& v, const float* __restrict__ f,
                                                     const float* __restrict__ xin, float* __restrict__ xout,
                                                     const float* __restrict__ ci, float* __restrict__ fc,
                                                     float* __restrict__ xc, int sx, int sy, int ty,
                                                     unsigned char* ring, unsigned long long* bars) {
  static_assert(RING % 2 == 0 && RING >= 4, "ring size");
  constexpr unsigned SLOT = StripRingR<S>::SLOT;
  const int n = v.n, ld = v.ld, nc = (n - 1) / 2, ldc = nc + 2;
  const size_t psc = plane_size(nc);
  const int lane = threadIdx.x & 31;
  const int i0 = 1 + 44 * sx, j0 = 1 + ty * sy, j1 = j0 + ty;
  const int icol = i0 - 10, ic = icol + 2 * lane;
  const bool in_a = ic >= 1 && ic <= n, in_b = ic + 1 >= 1 && ic + 1 <= n;
  const bool p1 = in_a && lane >= 1, q1 = in_b && lane >= 1 && lane <= 30;
  const bool r1 = in_a && lane >= 2 && lane <= 30, t1 = in_b && lane >= 2 && lane <= 29;
  const bool p2 = in_a && lane >= 3 && lane <= 29, q2 = in_b && lane >= 3 && lane <= 28;
  const bool r2 = in_a && lane >= 4 && lane <= 28, t2 = in_b && lane >= 4 && lane <= 27;
  const bool own = lane >= 5 && lane <= 26;       // c in [10, 53]
  const int icc = (ic + 1) / 2;                   // this lane's coarse column (its even fine column ic + 1)
  const bool own_c = own && icc >= 1 && icc <= nc;
  const StripSrc A{xin, f, static_cast<const float*>(v.pk)};
  const int NR = ty + 11;                         // band rows q = 0 .. NR - 1, j = j0 - 5 + q
  auto rowok = [&](int q) { const int j = j0 - 5 + q; return j >= 0 && j <= n + 1; };
  auto issue = [&](int q) {
    if (q >= NR) return;
    if (rowok(q))
      ring_issue_warp_r<S>(A, v.O, ld, icol, j0 - 5 + q, ring + (q % RING) * SLOT, &bars[q % RING]);
    else if (lane == 0)
      mbar_arrive(&bars[q % RING]);
  };
  if (lane == 0) {
    for (int k = 0; k < RING; ++k) mbar_init(&bars[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncwarp();
  for (int q = 0; q < RING; ++q) issue(q);
  bool ok = true;
  int taken = 0;
  auto take = [&](int q, StripRowR& R) {
    const int slot = q % RING;
    if (ok) ok = mbar_wait(&bars[slot], (unsigned)((q / RING) & 1));
    if (!ok) return;
    ring_read_r<S>(ring + slot * SLOT, ld, icol, ic, j0 - 5 + q, R);
    taken = q + 1;
    __syncwarp();
    issue(q + RING);
  };
  StripRowW K;                                    // final x and NW of row b - 3
  float rpa = 0.f, rpb = 0.f, rea = 0.f, reb = 0.f;   // residual rows b - 4 (odd) and b - 3 (even)
  // step m on the rows a - 4 .. a + 1 held in R0 .. R5, a = j0 - 4 + 2m
  auto step = [&](int m, StripRowR& R0, StripRowR& R1, StripRowR& R2, StripRowR& R3, StripRowR& R4,
                  StripRowR& R5) {
    const int a = j0 - 4 + 2 * m, b = a - 2;
    if (m >= 1) {
      take(2 * m + 1, R4);
      take(2 * m + 2, R5);
      if (!ok) return;
    }
    if (a >= 1 && a <= n) strip_row<float, float, FU>(R3, R4, R5, p1, q1);                   // sweep 1, row a
    if (m >= 1 && a - 1 >= 1 && a - 1 <= n) strip_row<float, float, FU>(R2, R3, R4, r1, t1);   // sweep 1, row a - 1
    if (m >= 2 && b >= 1 && b <= n) {                                                        // sweep 2, row b
      strip_row<float, float, FU>(R1, R2, R3, p2, q2);
      if (b >= j0 && b < j1) strip_store(xout, n, ld, ic, b, own, R2);
    }
    if (m >= 3 && b - 1 >= 1 && b - 1 <= n) {                                                // sweep 2, row b - 1
      strip_row<float, float, FU>(R0, R1, R2, r2, t2);
      if (b - 1 >= j0 && b - 1 < j1) strip_store(xout, n, ld, ic, b - 1, own, R1);
    }
    if (m >= 4) {
      // residuals of rows b - 2 (odd: rows K, R0, R1) and b - 1 (even: rows R0, R1, R2)
      float oa, ob, ea, eb;
      strip_resid<FU>(K, R0, R1, oa, ob);
      strip_resid<FU>(R0, R1, R2, ea, eb);
      if (b - 2 > n) oa = ob = 0.f;
      if (b - 1 > n) ea = eb = 0.f;
      if (ic > n) oa = ea = 0.f;
      if (ic + 1 > n) ob = eb = 0.f;
      // restriction of the coarse row whose fine row is b - 3 (odd rows b - 4, b - 2 around it)
      const int jc = (b - 3) / 2;
      if (m >= 5) {
        const float pa_n = shfl_dn1(rpa), ea_n = shfl_dn1(rea), oa_n = shfl_dn1(oa);   // columns 2 icc + 1
        if (own_c && b - 3 >= j0 + 1 && b - 3 <= j1 - 1 && jc >= 1 && jc <= nc) {
          auto w = [&](int k, int dic, int djc) { return ci[k * psc + (size_t)(jc + djc) * ldc + (icc + dic)]; };
          float t = rmul(w(CI_LNE, 0, 0), rpa);
          t = madd<FU>(t, w(CI_LA, 0, 0), rpb);
          t = madd<FU>(t, w(CI_LNW, 1, 0), pa_n);
          t = madd<FU>(t, w(CI_LR, 0, 0), rea);
          t = radd(t, reb);
          t = madd<FU>(t, w(CI_LL, 1, 0), ea_n);
          t = madd<FU>(t, w(CI_LSE, 0, 1), oa);
          t = madd<FU>(t, w(CI_LB, 0, 1), ob);
          t = madd<FU>(t, w(CI_LSW, 1, 1), oa_n);
          const size_t pc = (size_t)jc * ldc + icc;
          if (BMG_IN(DBG_RESTRICT_STORE, pc, (size_t)ldc * ldc)) {
            fc[pc] = t;
            xc[pc] = 0.f;
          }
        }
      }
      rpa = oa;
      rpb = ob;
      rea = ea;
      reb = eb;
    }
    K.xa = R1.xa;
    K.xb = R1.xb;
    K.nwa = R1.nwa;
    K.nwb = R1.nwb;
  };
  StripRowR S0, S1, S2, S3, S4, S5;
  take(0, S3);
  take(1, S4);
  take(2, S5);
  const int msteps = ty / 2 + 4;                  // steps m = 0 .. msteps
#pragma unroll 1
  for (int m = 0; m <= msteps && ok; m += 3) {
    step(m, S0, S1, S2, S3, S4, S5);
    if (m + 1 <= msteps && ok) step(m + 1, S2, S3, S4, S5, S0, S1);
    if (m + 2 <= msteps && ok) step(m + 2, S4, S5, S0, S1, S2, S3);
  }
  if (!ok)                                        // drain the copies still in flight, bounded
    for (int q = taken; q < taken + RING && q < NR; ++q) mbar_wait(&bars[q % RING], (unsigned)((q / RING) & 1));
  return ok;
}

// ---- four-colour sweep in one pass (FP64): per-lane asynchronous row copies ----------------
// The walk of gs_strip_ring_body (56 x TY strips, lane l holding the columns
// c = 2l, 2l + 1 of a 64-column window, the same colour regions, rows and
// stores) for FP64 levels.  Their arrays carry no guard band and no 16-byte
// alignment (the caller's x and f; every other stencil plane, (n+2)^2 doubles
// apart), so rows are not streamed by bulk copies: each lane copies its own two
// columns of a row's seven arrays with 8-byte cp.async copies into its part of
// the warp's ring slot (zero-filled outside [0, n+1]^2, where nothing is read),
// one commit group per band row, and reads them back after cp.async.wait_group.
// A lane reads only what it copied, so the ring needs no barrier.  The FP64
// pipe, not memory, bounds this kernel: the ring keeps RING - 1 rows of copies
// in flight behind the arithmetic.  The strip height ty is a launch argument
// (even, >= 2), so that the launcher can cut a level into as many strips as
// there are resident warps: a warp walks its strip serially, and a second,
// partial wave of strips would leave most of the FP64 pipes idle.
struct StripSrc64 {         // the 7 arrays the walk reads
  const double *x, *f, *d, *w, *s, *sw, *nw;
};
constexpr unsigned STRIP64_SLOT = 7 * 64 * sizeof(double);   // one row of the 7 arrays, 64 columns

__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool in) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(in ? 8 : 0)
               : "memory");
}

// this lane's columns ic, ic + 1 of row j into its part of `slot`, as one commit group
__device__ __forceinline__ void row64_issue(const StripSrc64& A, int n, int ld, int ic, int j, unsigned char* slot,
                                            int lane) {
  const bool rowin = j >= 0 && j <= n + 1;
  const bool ina = rowin && ic >= 0 && ic <= n + 1, inb = rowin && ic + 1 >= 0 && ic + 1 <= n + 1;
  const size_t pa = ina ? (size_t)j * ld + ic : 0, pb = inb ? (size_t)j * ld + ic + 1 : 0;
  // (debug builds: a copy from outside the array is zero-filled instead)
  const bool oka = ina && BMG_IN(DBG_STRIP64_COPY, pa, (size_t)(n + 2) * ld);
  const bool okb = inb && BMG_IN(DBG_STRIP64_COPY, pb, (size_t)(n + 2) * ld);
  double* d = reinterpret_cast<double*>(slot) + 2 * lane;
  const double* src[7] = {A.x, A.f, A.d, A.w, A.s, A.sw, A.nw};
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    cp_async8(d + 64 * k, src[k] + (oka ? pa : 0), oka);
    cp_async8(d + 64 * k + 1, src[k] + (okb ? pb : 0), okb);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void row64_read(const unsigned char* slot, int lane, StripRowT<double, double>& R) {
  const double2* d = reinterpret_cast<const double2*>(slot) + lane;
  double2 v = d[0];
  R.xa = v.x, R.xb = v.y;
  v = d[32];
  R.fa = v.x, R.fb = v.y;
  v = d[64];
  R.da = v.x, R.db = v.y;
  v = d[96];
  R.wa = v.x, R.wb = v.y;
  v = d[128];
  R.sa = v.x, R.sb = v.y;
  v = d[160];
  R.swa = v.x, R.swb = v.y;
  v = d[192];
  R.nwa = v.x, R.nwb = v.y;
}

template <int RING, bool FU = false>
__device__ __forceinline__ void gs_strip64_body(const StencilView<double, double>& v, const double* __restrict__ f,
                                                const double* __restrict__ xin, double* __restrict__ xout, int sx,
                                                int sy, int ty, unsigned char* ring) {
  static_assert(RING >= 2, "ring size");
  using Row = StripRowT<double, double>;
  const int n = v.n, ld = v.ld;
  const int lane = threadIdx.x & 31;
  const int i0 = 1 + 56 * sx, j0 = 1 + ty * sy, j1 = j0 + ty;
  const int icol = i0 - 4, ic = icol + 2 * lane;
  const bool in_a = ic >= 1 && ic <= n, in_b = ic + 1 >= 1 && ic + 1 <= n;
  const bool c1 = in_a && lane >= 1, c2 = in_b && lane >= 1 && lane <= 30;
  const bool c3 = in_a && lane >= 2 && lane <= 30, c4 = in_b && lane >= 2 && lane <= 29;
  const bool own = lane >= 2 && lane <= 29;
  const StripSrc64 A{xin, f, v.D, v.W, v.S_, v.SW, v.NW};
  const int NR = ty + 3;                          // band rows q = 0 .. NR - 1, j = j0 - 1 + q
  // every lane: request band row q (an empty group past the band keeps one group per row)
  auto issue = [&](int q) {
    if (q < NR)
      row64_issue(A, n, ld, ic, j0 - 1 + q, ring + (q % RING) * STRIP64_SLOT, lane);
    else
      asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
#pragma unroll
  for (int q = 0; q < RING; ++q) issue(q);
  // band row q into R: its group is the oldest of the RING outstanding ones
  auto take = [&](int q, Row& R) {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(RING - 1) : "memory");
    row64_read(ring + (q % RING) * STRIP64_SLOT, lane, R);
    issue(q + RING);
  };
  Row P0, P1, Q0, Q1;                             // two row pairs in alternating roles
  take(0, P1);
  take(1, Q0);
  take(2, Q1);
  if (j0 <= n) {
    strip_row<double, double, FU>(P1, Q0, Q1, c1, c2);     // row j0: c1, c2
    strip_store(xout, n, ld, ic, j0, own, Q0);
  }
  // step m: old pair = rows a - 2, a - 1; new pair = rows a, a + 1 (band rows 2m + 1, 2m + 2)
  auto step = [&](int m, Row& E0, Row& E1, Row& E2, Row& E3) {
    const int a = j0 + 2 * m;
    take(2 * m + 1, E2);
    take(2 * m + 2, E3);
    if (a <= n) {
      strip_row<double, double, FU>(E1, E2, E3, c1, c2);   // row a: c1, c2
      if (a < j1) strip_store(xout, n, ld, ic, a, own, E2);
    }
    if (a - 1 <= n) {
      strip_row<double, double, FU>(E0, E1, E2, c3, c4);   // row a - 1: c3, c4
      strip_store(xout, n, ld, ic, a - 1, own, E1);
    }
  };
#pragma unroll 1
  for (int m = 1; m <= ty / 2; m += 2) {
    step(m, Q0, Q1, P0, P1);
    if (m + 1 <= ty / 2) step(m + 1, P0, P1, Q0, Q1);
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");   // no copy outlives the warp
}

// ---- residual + restriction ------------------------------------------------------------
// A CTA owns a TXC x TYC tile of coarse points; it forms the residual on the
// (2 TXC + 1) x (2 TYC + 1) fine block under the tile in shared memory (each
// fine residual once, shared columns/rows recomputed at tile seams), then each
// thread applies the Fig. 2 restriction to one coarse point and zeroes the
// coarse iterate there.
template <typename T, typename S, bool NINE, bool FU = false>
__device__ __forceinline__ void resid_restrict_body(const StencilView<T, S>& v, const T* __restrict__ ci,
                                                    const T* __restrict__ x, const T* __restrict__ f,
                                                    T* __restrict__ fc, T* __restrict__ xc, int bx, int by) {
  __shared__ T r[RFY][RFX + 1];
  const int n = v.n, ld = v.ld, nc = (n - 1) / 2, ldc = nc + 2;
  const int ic0 = bx * TXC + 1, jc0 = by * TYC + 1;
  const int i0 = 2 * ic0 - 1, j0 = 2 * jc0 - 1;
  const int tid = threadIdx.y * TXC + threadIdx.x;
  auto fine = [&](int k) {
    int li = k % RFX, lj = k / RFX;
    int i = i0 + li, j = j0 + lj;
    T val = T(0);
    if (i <= n && j <= n) {
      size_t p = (size_t)j * ld + i;
      val = row_residual<T, S, NINE, true, FU>(v, x, p, f[p]);
    }
    r[lj][li] = val;
  };
  if constexpr (sizeof(T) == 4) {
    // FP32 levels wait on loads: unrolled, the residuals' loads of all of a
    // thread's points can be in flight together
    constexpr int NQ = (RFX * RFY + TXC * TYC - 1) / (TXC * TYC);
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      if (tid + q * TXC * TYC < RFX * RFY) fine(tid + q * TXC * TYC);
  } else {
    for (int k = tid; k < RFX * RFY; k += TXC * TYC) fine(k);
  }
  __syncthreads();
  int ic = ic0 + threadIdx.x, jc = jc0 + threadIdx.y;
  if (ic > nc || jc > nc) return;
  const size_t psc = plane_size(nc);
  const int li = 2 * threadIdx.x + 1, lj = 2 * threadIdx.y + 1;   // fine (2ic, 2jc) in the tile
  auto w = [&](int k, int dic, int djc) { return ci[k * psc + (size_t)(jc + djc) * ldc + (ic + dic)]; };
  T t = rmul(w(CI_LNE, 0, 0), r[lj - 1][li - 1]);
  t = madd<FU>(t, w(CI_LA, 0, 0), r[lj - 1][li]);
  t = madd<FU>(t, w(CI_LNW, 1, 0), r[lj - 1][li + 1]);
  t = madd<FU>(t, w(CI_LR, 0, 0), r[lj][li - 1]);
  t = radd(t, r[lj][li]);
  t = madd<FU>(t, w(CI_LL, 1, 0), r[lj][li + 1]);
  t = madd<FU>(t, w(CI_LSE, 0, 1), r[lj + 1][li - 1]);
  t = madd<FU>(t, w(CI_LB, 0, 1), r[lj + 1][li]);
  t = madd<FU>(t, w(CI_LSW, 1, 1), r[lj + 1][li + 1]);
  size_t pc = (size_t)jc * ldc + ic;
  if (!BMG_IN(DBG_RESTRICT_STORE, pc, (size_t)ldc * ldc)) return;
  fc[pc] = t;
  if (xc) xc[pc] = T(0);
}

// ---- interpolation + correction ----------------------------------------------------------
// One thread per coarse cell (ic, jc), 1..nc+1: its coincident, x-edge, y-edge
// and centre fine points.  xout = xin + (P e)_p, the interpolated value formed
// first; xin and xout may be the same array (every point is read and written by
// the same thread only).
template <typename T, bool FU = false>
__device__ __forceinline__ void interp_body(int n, const T* __restrict__ ci, const T* __restrict__ ec,
                                            const T* xin, T* xout, int ic, int jc) {
  int nc = (n - 1) / 2, ldc = nc + 2, ld = n + 2;
  if (ic < 1 || jc < 1 || ic > nc + 1 || jc > nc + 1) return;
  size_t psc = plane_size(nc), pc = (size_t)jc * ldc + ic;
  T e_sw = ec[pc - ldc - 1], e_se = ec[pc - ldc], e_nw = ec[pc - 1], e_ne = ec[pc];
  size_t pf = (size_t)(2 * jc) * ld + 2 * ic;   // coincident fine point
  const size_t ext = (size_t)ld * ld;
  // the cell's iterate values first (xin may be xout, so a load after a store
  // would wait for it)
  const bool in_i = ic <= nc, in_j = jc <= nc;
  const T x_co = in_i && in_j ? xin[pf] : T(0), x_xe = in_j ? xin[pf - 1] : T(0);
  const T x_ye = in_i ? xin[pf - ld] : T(0), x_ce = xin[pf - ld - 1];
  if (in_i && in_j && BMG_IN(DBG_INTERP_STORE, pf, ext)) xout[pf] = radd(x_co, e_ne);
  if (in_j) {                                     // x-edge (2ic-1, 2jc)
    T t = rmul(ci[CI_LL * psc + pc], e_nw);
    t = madd<FU>(t, ci[CI_LR * psc + pc], e_ne);
    if (BMG_IN(DBG_INTERP_STORE, pf - 1, ext)) xout[pf - 1] = radd(x_xe, t);
  }
  if (in_i) {                                     // y-edge (2ic, 2jc-1)
    T t = rmul(ci[CI_LB * psc + pc], e_se);
    t = madd<FU>(t, ci[CI_LA * psc + pc], e_ne);
    if (BMG_IN(DBG_INTERP_STORE, pf - ld, ext)) xout[pf - ld] = radd(x_ye, t);
  }
  {                                               // centre (2ic-1, 2jc-1)
    T t = rmul(ci[CI_LSW * psc + pc], e_sw);
    t = madd<FU>(t, ci[CI_LSE * psc + pc], e_se);
    t = madd<FU>(t, ci[CI_LNW * psc + pc], e_nw);
    t = madd<FU>(t, ci[CI_LNE * psc + pc], e_ne);
    if (BMG_IN(DBG_INTERP_STORE, pf - ld - 1, ext)) xout[pf - ld - 1] = radd(x_ce, t);
  }
}

// ---- reductions in the canonical order -------------------------------------------------
// Block b of G = min(n, 1024) handles rows j = 1 + b, 1 + b + G, ...; thread t
// the columns i = 1 + t, 1 + t + 256, ...; each thread sums in that order,
// then a fixed halving tree; the G block sums are reduced the same way.
// The halving tree s[t] += s[t + h], h = 128, 64, ..., 1: the levels h >= 32
// through shared memory with a block barrier each, the levels h < 32 inside
// warp 0 by shuffles (lane t adds lane t + h; lanes >= h hold values no lane
// below h reads), so every sum pairs the same operands as the all-shared tree.
__device__ __forceinline__ double block_sum(double acc) {
  __shared__ double red[NORM_THREADS];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = NORM_THREADS / 2; s >= 32; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 32) {
    double v = red[threadIdx.x];
    for (int s = 16; s > 0; s >>= 1) v = v + __shfl_down_sync(0xffffffffu, v, s);
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  double v = red[0];
  __syncthreads();   // the buffer may be reused by a following block_sum
  return v;
}

__host__ __device__ inline int norm_blocks(int n) { return n < NORM_BLOCKS_MAX ? n : NORM_BLOCKS_MAX; }

template <typename T, typename S, bool NINE, bool FU = false>
__device__ __forceinline__ void residual_body(const StencilView<T, S>& v, const T* __restrict__ x,
                                              const T* __restrict__ f, T* __restrict__ r,
                                              double* __restrict__ partials, int b, int G) {
  const int n = v.n, ld = v.ld;
  double acc = 0.0;
  for (int j = 1 + b; j <= n; j += G)
    for (int i = 1 + threadIdx.x; i <= n; i += NORM_THREADS) {
      size_t p = (size_t)j * ld + i;
      T s = row_residual<T, S, NINE, true, FU>(v, x, p, f[p]);
      if (r && BMG_IN(DBG_RESIDUAL_STORE, p, (size_t)(n + 2) * ld)) r[p] = s;
      double d = (double)s;
      acc = madd<FU>(acc, d, d);
    }
  if (partials) {
    double tot = block_sum(acc);
    if (threadIdx.x == 0) partials[b] = tot;
  }
}

__device__ __forceinline__ double scale_of(double rho) {
  if (!(rho > 0.0) || !isfinite(rho)) return 1.0;
  int e;
  frexp(rho, &e);
  return ldexp(1.0, e);
}

// One block: sum the partials in index order per thread, fixed tree, sqrt;
// record the norm in ctl (phase 0 = initial residual, 1 = after a cycle).
__device__ __forceinline__ void finalize_body(const double* __restrict__ partials, int np, Ctl* ctl, int phase,
                                              double* out) {
  if (phase == 1 && ctl && ctl->done) return;
  double acc = 0.0;
  for (int k = threadIdx.x; k < np; k += NORM_THREADS) acc = __dadd_rn(acc, partials[k]);
  double tot = block_sum(acc);
  if (threadIdx.x != 0) return;
  double rho = __dsqrt_rn(tot);
  if (out) *out = rho;
  if (!ctl) return;
  if (phase == 0) {
    ctl->it = 0;
    ctl->hist[0] = rho;
    ctl->done = !isfinite(rho) ? 3 : (rho == 0.0 ? 1 : 0);
    if (ctl->done == 0 && ctl->maxit <= 0) ctl->done = 2;
  } else {
    int it = ctl->it + 1;
    ctl->it = it;
    ctl->hist[it] = rho;
    if (!isfinite(rho)) ctl->done = 3;
    else if (rho / ctl->hist[0] <= ctl->tol) ctl->done = 1;
    else if (it >= ctl->maxit) ctl->done = 2;
  }
  ctl->scale_next = scale_of(rho);
}

// ---- coarsest solve: forward and back substitution ------------------------------------
// L L^T x = f with every thread of the block taking part.  Forward, right-looking:
// once y_k = s_k / L_kk is known, every row i > k subtracts L_ik y_k; each row still
// receives its terms in increasing k, the order of the row-by-row loop, so the
// result is the same bits.  Backward, thread 0: row i's sum runs over k = i+1 .. m-1
// in increasing order and starts with x_{i+1}, so the rows form one chain.  The
// factor is staged in shared memory when it is small (a chain through L2 would
// pay a round trip per term).  y is unused (kept for the callers' layout).
constexpr int COARSE_M_MAX = 225;   // coarsest level n <= 15
constexpr int COARSE_M_SMEM = 9;    // factors of m <= 9 unknowns (n = 3) go to shared memory
template <typename T>
__device__ __forceinline__ void coarse_solve_body(int n, const double* __restrict__ L, const T* __restrict__ f,
                                                  T* __restrict__ x, double* __restrict__ y) {
  __shared__ double ys[COARSE_M_MAX];
  __shared__ double Ls[COARSE_M_SMEM * COARSE_M_SMEM];
  (void)y;
  const int m = n * n, ld = n + 2;
  const bool staged = m <= COARSE_M_SMEM;
  const double* Lp = staged ? Ls : L;
  for (int k = threadIdx.x; k < m; k += blockDim.x) ys[k] = (double)f[(size_t)(k / n + 1) * ld + (k % n + 1)];
  if (staged)
    for (int k = threadIdx.x; k < m * m; k += blockDim.x) Ls[k] = L[k];
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) ys[k] = rdiv(ys[k], Lp[(size_t)k * m + k]);
    __syncthreads();
    const double yk = ys[k];
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) ys[i] = rsub(ys[i], rmul(Lp[(size_t)i * m + k], yk));
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int i = m - 1; i >= 0; --i) {
      double s = ys[i];
      for (int k = i + 1; k < m; ++k) s = rsub(s, rmul(Lp[(size_t)k * m + i], ys[k]));   // ys[k] = x_k
      ys[i] = rdiv(s, Lp[(size_t)i * m + i]);
    }
  __syncthreads();
  for (int k = threadIdx.x; k < m; k += blockDim.x) x[(size_t)(k / n + 1) * ld + (k % n + 1)] = (T)ys[k];
}

// ---- iterative refinement ------------------------------------------------------------------
// s * fl64(e) for a positive normal power of two s (the refinement scales).
// The product is exact, so it is formed from the bit fields: the float's
// exponent, re-biased and raised by log2(s), and its mantissa widened. Only
// when e is subnormal, infinite or NaN, when the product is not a normal
// double, or when s is not such a power of two, does it take the FP64 multiply.
// Both routes give the same bits; the bit route spares the FP64 pipe two
// operations.
// The general route of pow2_times_widened, kept out of line so that the common
// route compiles to integer operations only (no FP64 work predicated in).
static __device__ __noinline__ double pow2_times_widened_slow(double s, float e) { return rmul(s, (double)e); }

__device__ __forceinline__ double pow2_times_widened(double s, float e) {
  const unsigned long long sb = (unsigned long long)__double_as_longlong(s);
  const int es = (int)((sb >> 52) & 0x7ff);
  if (!(sb >> 63) && es != 0 && es != 0x7ff && (sb & 0xfffffffffffffULL) == 0) {
    const unsigned u = __float_as_uint(e);
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    if ((u & 0x7fffffffu) == 0) return __longlong_as_double((long long)sign);   // s * (+-0) = +-0
    const int ef = (int)((u >> 23) & 0xff);
    const int ed = ef - 127 + es;   // (ef - 127) + (es - 1023) + 1023
    if (ef != 0 && ef != 0xff && ed > 0 && ed < 0x7ff)
      return __longlong_as_double(
          (long long)(sign | ((unsigned long long)ed << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
  }
  return pow2_times_widened_slow(s, e);
}

// fl32(r * inv) for inv a power of two (the scaled FP32 residual of the
// refinement).  Narrowed first and scaled in FP32, it is the same number
// whenever fl32(r) and the scaled value lie in [2^-125, 2^127]: both r and
// r * inv are then in normal binades, where rounding to 24 bits commutes with
// scaling by a power of two, and the FP32 product is exact.  Everything else
// (tiny, huge, non-finite values, or a scale outside the FP32 range, signalled
// by inv32 = 0) takes the FP64 product; this spares the FP64 pipe one multiply
// per point on the FP64-bound outer residual.
static __device__ __noinline__ float narrow_scaled_slow(double r, double inv) {
  return __double2float_rn(rmul(r, inv));
}

__device__ __forceinline__ float narrow_scale32(double inv) {
  return inv >= 0x1p-125 && inv <= 0x1p125 ? (float)inv : 0.0f;
}

__device__ __forceinline__ float narrow_scaled(double r, double inv, float inv32) {
  const float a = __double2float_rn(r);
  const float b = __fmul_rn(a, inv32);
  const float ma = fabsf(a), mb = fabsf(b);
  if (ma >= 0x1p-125f && ma <= 0x1p127f && mb >= 0x1p-125f && mb <= 0x1p127f) return b;
  return narrow_scaled_slow(r, inv);
}

// x += scale_applied * e32 on IRU_COLS points of row j, columns i0, i0 + step,
// ...: every load is issued before the first store, so that a thread keeps
// several in flight (one point per thread left the update at 0.72 of the copy
// bandwidth).
constexpr int IRU_COLS = 4;
__device__ __forceinline__ void ir_update_cols(int n, double* __restrict__ x, const float* __restrict__ e32,
                                               double s, int i0, int j, int step) {
  if (j < 1 || j > n) return;
  double xv[IRU_COLS];
  float ev[IRU_COLS];
#pragma unroll
  for (int q = 0; q < IRU_COLS; ++q) {
    const int i = i0 + q * step;
    if (i >= 1 && i <= n) {
      const size_t p = (size_t)j * (n + 2) + i;
      xv[q] = x[p];
      ev[q] = e32[p];
    }
  }
#pragma unroll
  for (int q = 0; q < IRU_COLS; ++q) {
    const int i = i0 + q * step;
    const size_t p = (size_t)j * (n + 2) + i;
    if (i >= 1 && i <= n && BMG_IN(DBG_REFINE_STORE, p, (size_t)(n + 2) * (n + 2)))
      x[p] = radd(xv[q], pow2_times_widened(s, ev[q]));
  }
}

// r = f - A x (FP64), r32 = fl32(r / scale_next), e32 = 0, partial sums of r^2.
template <bool FU = false>
__device__ __forceinline__ void ir_residual_body(const StencilView<double, double>& v, bool nine,
                                                 const double* __restrict__ x, const double* __restrict__ f,
                                                 float* __restrict__ r32, float* __restrict__ e32,
                                                 double* __restrict__ partials, Ctl* ctl, int b, int G) {
  const int n = v.n, ld = v.ld;
  const double s = ctl->scale_next;
  const double inv = 1.0 / s;   // exact: s is a power of two
  const float inv32 = narrow_scale32(inv);
  double acc = 0.0;
  for (int j = 1 + b; j <= n; j += G)
    for (int i = 1 + threadIdx.x; i <= n; i += NORM_THREADS) {
      size_t p = (size_t)j * ld + i;
      double rr = nine ? row_residual<double, double, true, true, FU>(v, x, p, f[p])
                       : row_residual<double, double, false, true, FU>(v, x, p, f[p]);
      if (BMG_IN(DBG_REFINE_STORE, p, (size_t)(n + 2) * ld)) {
        r32[p] = narrow_scaled(rr, inv, inv32);
        e32[p] = 0.0f;
      }
      acc = madd<FU>(acc, rr, rr);
    }
  double tot = block_sum(acc);
  if (threadIdx.x == 0) {
    partials[b] = tot;
    if (b == 0) ctl->scale_applied = s;
  }
}

}  // namespace dev
}  // namespace bmg

// ==== level-fused tail: the V-cycle below a small level in one CTA ===========================
namespace bmg {

constexpr int TAIL_LEVELS = 6;   // levels held by one tail descriptor (n <= 63 down to 3 is 5)

// The levels of one problem from the tail's top level down to the coarsest.
template <typename T>
struct TailDesc {
  LevelDesc<T, T> lv[TAIL_LEVELS];
  int nlev;     // levels in lv (the last is the coarsest)
  int nu1, nu2;
  int top_kind; // stencil kind of lv[0] (5 or 9); the levels below are 9-point
  const int* done;
};

namespace dev {

// Half of a four-colour sweep over one CTA: the rows of parity pj, their odd-i
// points, a barrier, their even-i points, a barrier (the order of k_gs_rows).
template <typename T, typename S, bool FU = false>
__device__ __forceinline__ void gs_half_block(const StencilView<T, S>& v, const T* f, T* x, int pj) {
  const int n = v.n;
  const int R = pj ? (n + 1) / 2 : (n - 1) / 2;
  const int Po = (n + 1) / 2, Pe = (n - 1) / 2;
  for (int k = threadIdx.x; k < R * Po; k += blockDim.x) {
    int j = 2 * (k / Po) + (pj ? 1 : 2), i = 2 * (k % Po) + 1;
    gs_point<T, S, true, FU>(v, f, x, (size_t)j * v.ld + i);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < R * Pe; k += blockDim.x) {
    int j = 2 * (k / Pe) + (pj ? 1 : 2), i = 2 * (k % Pe) + 2;
    gs_point<T, S, true, FU>(v, f, x, (size_t)j * v.ld + i);
  }
  __syncthreads();
}

// One red-black colour over one CTA (5-point levels).
template <typename T, typename S, bool FU = false>
__device__ __forceinline__ void gs_checker_block(const StencilView<T, S>& v, const T* f, T* x, int c) {
  const int n = v.n;
  const int per_row = (n + 1) / 2;
  for (int k = threadIdx.x; k < n * per_row; k += blockDim.x) {
    int j = k / per_row + 1;
    int i = 2 * (k % per_row) + 1 + ((j + 1 + c) & 1);
    if (i <= n) gs_point<T, S, false, FU>(v, f, x, (size_t)j * v.ld + i);
  }
  __syncthreads();
}

template <typename T, bool FU = false>
__device__ __forceinline__ void relax_block(const LevelDesc<T, T>& q, int kind, int sweeps) {
  for (int s = 0; s < sweeps; ++s) {
    if (kind == 9) {
      gs_half_block<T, T, FU>(q.v, q.f, q.x, 1);
      gs_half_block<T, T, FU>(q.v, q.f, q.x, 0);
    } else {
      gs_checker_block<T, T, FU>(q.v, q.f, q.x, 0);
      gs_checker_block<T, T, FU>(q.v, q.f, q.x, 1);
    }
  }
}

// Residual + Fig. 2 restriction, one coarse point per thread iteration; the
// nine fine residuals are formed where they are needed (same values as the
// tiled kernel: each is the same expression of the same data).
template <typename T, bool NINE, bool FU = false>
__device__ __forceinline__ void resid_restrict_block(const LevelDesc<T, T>& q) {
  const StencilView<T, T>& v = q.v;
  const int n = v.n, ld = v.ld, nc = (n - 1) / 2, ldc = nc + 2;
  const size_t psc = plane_size(nc);
  for (int k = threadIdx.x; k < nc * nc; k += blockDim.x) {
    int ic = k % nc + 1, jc = k / nc + 1;
    size_t pf = (size_t)(2 * jc) * ld + 2 * ic;
    auto r = [&](int dx, int dy) {
      size_t p = pf + (size_t)((long long)dy * ld + dx);
      return row_residual<T, T, NINE, true, FU>(v, q.x, p, q.f[p]);
    };
    auto w = [&](int kk, int dic, int djc) { return q.ci[kk * psc + (size_t)(jc + djc) * ldc + (ic + dic)]; };
    T t = rmul(w(CI_LNE, 0, 0), r(-1, -1));
    t = madd<FU>(t, w(CI_LA, 0, 0), r(0, -1));
    t = madd<FU>(t, w(CI_LNW, 1, 0), r(1, -1));
    t = madd<FU>(t, w(CI_LR, 0, 0), r(-1, 0));
    t = radd(t, r(0, 0));
    t = madd<FU>(t, w(CI_LL, 1, 0), r(1, 0));
    t = madd<FU>(t, w(CI_LSE, 0, 1), r(-1, 1));
    t = madd<FU>(t, w(CI_LB, 0, 1), r(0, 1));
    t = madd<FU>(t, w(CI_LSW, 1, 1), r(1, 1));
    size_t pc = (size_t)jc * ldc + ic;
    if (BMG_IN(DBG_RESTRICT_STORE, pc, (size_t)ldc * ldc)) {
      q.fc[pc] = t;
      q.xc[pc] = T(0);
    }
  }
  __syncthreads();
}

template <typename T, bool FU = false>
__device__ __forceinline__ void tail_body(const TailDesc<T>& d, int top_kind) {
  for (int l = 0; l + 1 < d.nlev; ++l) {
    const int kind = l == 0 ? top_kind : 9;
    relax_block<T, FU>(d.lv[l], kind, d.nu1);
    if (kind == 9)
      resid_restrict_block<T, true, FU>(d.lv[l]);
    else
      resid_restrict_block<T, false, FU>(d.lv[l]);
  }
  const LevelDesc<T, T>& c = d.lv[d.nlev - 1];
  coarse_solve_body<T>(c.v.n, c.L, c.f, c.x, c.y);
  __syncthreads();
  for (int l = d.nlev - 2; l >= 0; --l) {
    const LevelDesc<T, T>& q = d.lv[l];
    const int nc = (q.v.n - 1) / 2;
    for (int k = threadIdx.x; k < (nc + 1) * (nc + 1); k += blockDim.x)
      interp_body<T, FU>(q.v.n, q.ci, q.xc, q.x, q.x, k % (nc + 1) + 1, k / (nc + 1) + 1);
    __syncthreads();
    relax_block<T, FU>(q, l == 0 ? top_kind : 9, d.nu2);
  }
}

}  // namespace dev
}  // namespace bmg
