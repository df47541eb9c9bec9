// Two-grid training loss of the learned interpolation and its gradient, on a
// batch of small crops (n = 7, 15 or 31 interior points), one CTA per crop.
//
// For an error vector e the two-grid error propagation of V(2,1) with exact
// coarse solve is
//     E e = S (I - P A_c^{-1} P^T A) S^2 e,   A_c = P^T A P,
// S one four-colour Gauss-Seidel sweep of A e = 0.  The loss of a crop is
// w/K sum_k ||E e_k||_A^2 / e_ref_k (e_ref: Dendy's energies).  Its gradient
// with respect to the weights of P, with u = A_c^{-1} P^T A e1 (e1 = S^2 e),
// e2 = e1 - P u, g2 = S^T (dL/d e3) and the adjoint coarse solve
// v = A_c^{-1} P^T g2, is  dL/dP = (A P v - g2) u^T - (A e2) v^T  on P's
// sparsity pattern; it is chained through Dendy's centre formula and the
// edge split to the network's logits.  Everything is FP64: the crops have
// coefficient jumps of up to 1e6, far beyond what an FP32 coarse solve
// resolves.  A_c keeps the lexicographic band of half-width n_c + 1 and is
// factored by a banded right-looking Cholesky in shared memory; the fine grid
// operations follow the oracle's expression orders (sweeps, apply, the
// Fig. 2 restriction, the interpolation), the Galerkin entries are the
// setup's (bit for bit the oracle's), and only the coarse solves differ from
// the oracle's dense solve by rounding.
#include "common.cuh"
#include "kernels.h"
#include "learned.h"
#include "learned_device.cuh"
#include "rap_device.cuh"

namespace bmg {
namespace {

constexpr int TG_THREADS = 512;
constexpr int TG_WARPS = TG_THREADS / 32;

template <int N>
struct TG {
  static constexpr int LD = N + 2, PS = LD * LD;
  static constexpr int NC = (N - 1) / 2, LDC = NC + 2, PSC = LDC * LDC;
  static constexpr int M = NC * NC, BW = NC + 1, BL = BW + 1;   // coarse unknowns, half band, band row length
  // shared-memory layout, in doubles
  static constexpr int ST = 0;                   // O, W, S, SW, NW, D = 1/O
  static constexpr int CI = ST + 6 * PS;         // 8 weight planes
  static constexpr int AUX = CI + 8 * PSC;       // S_D and share of the x- and y-edge points
  static constexpr int DW = AUX + 4 * PSC;       // dL/dw, 8 planes
  static constexpr int BAND = DW + 8 * PSC;      // lower band of A_c / its factor, M x BL
  static constexpr int X = BAND + M * BL;        // fine vectors
  static constexpr int E2 = X + PS, G = E2 + PS, T = G + PS;
  static constexpr int FC = T + PS, U = FC + PSC, V = U + PSC;   // coarse vectors
  static constexpr int RED = V + PSC;            // TG_WARPS partial sums
  static constexpr int TOTAL = RED + TG_WARPS;
  static constexpr size_t BYTES = (size_t)TOTAL * sizeof(double);
};

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One four-colour sweep of A x = 0 in place (colours (odd,odd), (even,odd),
// (odd,even), (even,even)); x_p = (0 - sum_{q != p} a_pq x_q) d_p.
template <int N>
__device__ void sweep(const Planes<double>& A, const double* D, double* x) {
  using L = TG<N>;
  constexpr int LD = L::LD;
  const int pis[4] = {1, 0, 1, 0}, pjs[4] = {1, 1, 0, 0};
  for (int c = 0; c < 4; ++c) {
    const int i0 = pis[c] ? 1 : 2, j0 = pjs[c] ? 1 : 2;
    const int ni = (N - i0) / 2 + 1, nj = (N - j0) / 2 + 1;
    for (int idx = threadIdx.x; idx < ni * nj; idx += TG_THREADS) {
      const int i = i0 + 2 * (idx % ni), j = j0 + 2 * (idx / ni);
      const size_t p = (size_t)j * LD + i;
      double s = 0.0;
      s = rsub(s, rmul(A.a<1>(p, LD), x[p - 1]));
      s = rsub(s, rmul(A.a<2>(p, LD), x[p + 1]));
      s = rsub(s, rmul(A.a<3>(p, LD), x[p - LD]));
      s = rsub(s, rmul(A.a<4>(p, LD), x[p + LD]));
      s = rsub(s, rmul(A.a<5>(p, LD), x[p - LD - 1]));
      s = rsub(s, rmul(A.a<6>(p, LD), x[p + LD + 1]));
      s = rsub(s, rmul(A.a<7>(p, LD), x[p + LD - 1]));
      s = rsub(s, rmul(A.a<8>(p, LD), x[p + 1 - LD]));
      x[p] = rmul(s, D[p]);
    }
    __syncthreads();
  }
}

// y <- S^T y: for the colours in reverse order, z = d y on the colour's points
// (zero elsewhere), y = y - A z.  z and Az are scratch vectors (ghosts zero).
template <int N>
__device__ void sweep_adjoint(const Planes<double>& A, const double* D, double* y, double* z, double* az);

// out = A in over the interior: a_O in_p first, then the canonical order.
template <int N>
__device__ void apply(const Planes<double>& A, const double* in, double* out) {
  constexpr int LD = TG<N>::LD;
  for (int idx = threadIdx.x; idx < N * N; idx += TG_THREADS) {
    const int i = 1 + idx % N, j = 1 + idx / N;
    const size_t p = (size_t)j * LD + i;
    double s = rmul(A.a<0>(p, LD), in[p]);
    s = radd(s, rmul(A.a<1>(p, LD), in[p - 1]));
    s = radd(s, rmul(A.a<2>(p, LD), in[p + 1]));
    s = radd(s, rmul(A.a<3>(p, LD), in[p - LD]));
    s = radd(s, rmul(A.a<4>(p, LD), in[p + LD]));
    s = radd(s, rmul(A.a<5>(p, LD), in[p - LD - 1]));
    s = radd(s, rmul(A.a<6>(p, LD), in[p + LD + 1]));
    s = radd(s, rmul(A.a<7>(p, LD), in[p + LD - 1]));
    s = radd(s, rmul(A.a<8>(p, LD), in[p + 1 - LD]));
    out[p] = s;
  }
}

template <int N>
__device__ void sweep_adjoint(const Planes<double>& A, const double* D, double* y, double* z, double* az) {
  using L = TG<N>;
  constexpr int LD = L::LD;
  const int pis[4] = {0, 1, 0, 1}, pjs[4] = {0, 0, 1, 1};   // reverse of the sweep's colour order
  for (int c = 0; c < 4; ++c) {
    for (int idx = threadIdx.x; idx < N * N; idx += TG_THREADS) {
      const int i = 1 + idx % N, j = 1 + idx / N;
      const size_t p = (size_t)j * LD + i;
      z[p] = (i % 2 == pis[c] && j % 2 == pjs[c]) ? rmul(y[p], D[p]) : 0.0;
    }
    __syncthreads();
    apply<N>(A, z, az);
    __syncthreads();
    for (int idx = threadIdx.x; idx < N * N; idx += TG_THREADS) {
      const size_t p = (size_t)(1 + idx / N) * LD + 1 + idx % N;
      y[p] = rsub(y[p], az[p]);
    }
    __syncthreads();
  }
}

// fc = P^T r, the nine terms of Fig. 2 left to right.
template <int N>
__device__ void restrict_fig2(const double* ci, const double* r, double* fc) {
  using L = TG<N>;
  constexpr int LD = L::LD, NC = L::NC, LDC = L::LDC, PSC = L::PSC;
  for (int idx = threadIdx.x; idx < NC * NC; idx += TG_THREADS) {
    const int ic = 1 + idx % NC, jc = 1 + idx / NC;
    const size_t pc = (size_t)jc * LDC + ic, q = (size_t)(2 * jc) * LD + 2 * ic;
    double t = rmul(ci[CI_LNE * PSC + pc], r[q - LD - 1]);
    t = radd(t, rmul(ci[CI_LA * PSC + pc], r[q - LD]));
    t = radd(t, rmul(ci[CI_LNW * PSC + pc + 1], r[q - LD + 1]));
    t = radd(t, rmul(ci[CI_LR * PSC + pc], r[q - 1]));
    t = radd(t, r[q]);
    t = radd(t, rmul(ci[CI_LL * PSC + pc + 1], r[q + 1]));
    t = radd(t, rmul(ci[CI_LSE * PSC + pc + LDC], r[q + LD - 1]));
    t = radd(t, rmul(ci[CI_LB * PSC + pc + LDC], r[q + LD]));
    t = radd(t, rmul(ci[CI_LSW * PSC + pc + LDC + 1], r[q + LD + 1]));
    fc[pc] = t;
  }
}

// out_p = base_p - (P ec)_p (base = nullptr: out = P ec), the interpolated
// value formed first as in the oracle's interpolation.
template <int N>
__device__ void interp(const double* ci, const double* ec, const double* base, double* out) {
  using L = TG<N>;
  constexpr int LD = L::LD, NC = L::NC, LDC = L::LDC, PSC = L::PSC;
  for (int idx = threadIdx.x; idx < (NC + 1) * (NC + 1); idx += TG_THREADS) {
    const int ic = 1 + idx % (NC + 1), jc = 1 + idx / (NC + 1);
    const size_t pc = (size_t)jc * LDC + ic, pf = (size_t)(2 * jc) * LD + 2 * ic;
    auto put = [&](size_t p, double v) { out[p] = base ? rsub(base[p], v) : v; };
    if (ic <= NC && jc <= NC) put(pf, ec[pc]);
    if (jc <= NC) put(pf - 1, radd(rmul(ci[CI_LL * PSC + pc], ec[pc - 1]), rmul(ci[CI_LR * PSC + pc], ec[pc])));
    if (ic <= NC) put(pf - LD, radd(rmul(ci[CI_LB * PSC + pc], ec[pc - LDC]), rmul(ci[CI_LA * PSC + pc], ec[pc])));
    double t = rmul(ci[CI_LSW * PSC + pc], ec[pc - LDC - 1]);
    t = radd(t, rmul(ci[CI_LSE * PSC + pc], ec[pc - LDC]));
    t = radd(t, rmul(ci[CI_LNW * PSC + pc], ec[pc - 1]));
    t = radd(t, rmul(ci[CI_LNE * PSC + pc], ec[pc]));
    put(pf - LD - 1, t);
  }
}

// Banded right-looking Cholesky of the lower band (row i holds A(i, i-d) at
// d = 0..BW), by one warp; returns false on a non-positive pivot.
template <int N>
__device__ bool band_cholesky(double* band) {
  using L = TG<N>;
  constexpr int M = L::M, BW = L::BW, BL = L::BL;
  const int lane = threadIdx.x & 31;
  bool ok = true;
  for (int k = 0; k < M; ++k) {
    double p = band[k * BL];
    if (!(p > 0.0)) ok = false;
    const double lkk = sqrt(p);
    __syncwarp();
    if (lane == 0) band[k * BL] = lkk;
    if (lane >= 1 && lane <= BW && k + lane < M) band[(k + lane) * BL + lane] = rdiv(band[(k + lane) * BL + lane], lkk);
    __syncwarp();
    // trailing update of the pairs k < j <= i <= min(k + BW, M - 1)
    for (int e = lane; e < BW * (BW + 1) / 2; e += 32) {
      int a = 0, rem = e;                       // a = j - k - 1, b = i - j
      while (rem >= BW - a) { rem -= BW - a; ++a; }
      const int j = k + 1 + a, i = j + rem;
      if (i < M) band[i * BL + (i - j)] = rsub(band[i * BL + (i - j)], rmul(band[i * BL + (i - k)], band[j * BL + (j - k)]));
    }
    __syncwarp();
  }
  return ok;
}

// x = (L L^T)^{-1} b for coarse vectors in the (NC+2)^2 layout, by one warp.
template <int N>
__device__ void band_solve(const double* band, const double* b, double* x) {
  using L = TG<N>;
  constexpr int M = L::M, NC = L::NC, LDC = L::LDC, BW = L::BW, BL = L::BL;
  const int lane = threadIdx.x & 31;
  auto pos = [](int i) { return (size_t)(i / NC + 1) * LDC + (i % NC + 1); };
  for (int i = 0; i < M; ++i) {
    double t = (lane >= 1 && lane <= BW && i - lane >= 0) ? rmul(band[i * BL + lane], x[pos(i - lane)]) : 0.0;
    const double s = warp_sum(t);
    if (lane == 0) x[pos(i)] = rdiv(rsub(b[pos(i)], s), band[i * BL]);
    __syncwarp();
  }
  for (int i = M - 1; i >= 0; --i) {
    double t = (lane >= 1 && lane <= BW && i + lane < M) ? rmul(band[(i + lane) * BL + lane], x[pos(i + lane)]) : 0.0;
    const double s = warp_sum(t);
    if (lane == 0) x[pos(i)] = rdiv(rsub(x[pos(i)], s), band[i * BL]);
    __syncwarp();
  }
}

// dW += dL/dw of <g, P ec> for every weight w(p -> c) of P: g(p) ec(c).
template <int N>
__device__ void add_outer(const double* g, double gsign, const double* ec, double* dW) {
  using L = TG<N>;
  constexpr int LD = L::LD, NC = L::NC, LDC = L::LDC, PSC = L::PSC;
  for (int idx = threadIdx.x; idx < (NC + 1) * (NC + 1); idx += TG_THREADS) {
    const int ic = 1 + idx % (NC + 1), jc = 1 + idx / (NC + 1);
    const size_t pc = (size_t)jc * LDC + ic, pf = (size_t)(2 * jc) * LD + 2 * ic;
    const double e_sw = ec[pc - LDC - 1], e_se = ec[pc - LDC], e_nw = ec[pc - 1], e_ne = ec[pc];
    if (jc <= NC) {
      const double gg = gsign * g[pf - 1];
      dW[CI_LL * PSC + pc] += gg * e_nw;
      dW[CI_LR * PSC + pc] += gg * e_ne;
    }
    if (ic <= NC) {
      const double gg = gsign * g[pf - LD];
      dW[CI_LB * PSC + pc] += gg * e_se;
      dW[CI_LA * PSC + pc] += gg * e_ne;
    }
    const double gg = gsign * g[pf - LD - 1];
    dW[CI_LSW * PSC + pc] += gg * e_sw;
    dW[CI_LSE * PSC + pc] += gg * e_se;
    dW[CI_LNW * PSC + pc] += gg * e_nw;
    dW[CI_LNE * PSC + pc] += gg * e_ne;
  }
}

template <int N>
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < TG_WARPS; ++w) s += red[w];
  __syncthreads();
  return s;   // valid on thread 0
}

// grid: one CTA per crop.  coefs: ncrop x 5 planes (n+2)^2 (ghost ring and
// couplings to it are ignored); vecs: ncrop x K error vectors (n+2)^2;
// delta: ncrop x n_c^2 x 4 logits (NULL: Dendy's weights); eref: ncrop x K
// normalisers, or NULL for energies only; energies: ncrop x K out;
// ddelta: ncrop x n_c^2 x 4 out (with eref); err: set on a non-positive pivot.
template <int N>
__global__ void __launch_bounds__(TG_THREADS, 1)
    k_twogrid(int K, const double* __restrict__ coefs, const double* __restrict__ vecs,
              const float* __restrict__ delta, const double* __restrict__ eref, double weight,
              double* __restrict__ energies, float* __restrict__ ddelta, int* __restrict__ err) {
  using L = TG<N>;
  constexpr int LD = L::LD, PS = L::PS, NC = L::NC, LDC = L::LDC, PSC = L::PSC, M = L::M, BL = L::BL;
  extern __shared__ double sm[];
  const int crop = blockIdx.x, tid = threadIdx.x;
  double *st = sm + L::ST, *ci = sm + L::CI, *aux = sm + L::AUX, *dW = sm + L::DW, *band = sm + L::BAND;
  double *X = sm + L::X, *E2 = sm + L::E2, *G = sm + L::G, *T = sm + L::T;
  double *FC = sm + L::FC, *U = sm + L::U, *V = sm + L::V, *red = sm + L::RED;
  __shared__ int bad;
  // stencil, with the ghost ring and every coupling to it zero
  const double* src = coefs + (size_t)crop * 5 * PS;
  for (int e = tid; e < PS; e += TG_THREADS) {
    const int i = e % LD, j = e / LD;
    const bool in = i >= 1 && i <= N && j >= 1 && j <= N;
    const double o = in ? src[e] : 0.0;
    st[e] = o;
    st[PS + e] = (in && i > 1) ? src[PS + e] : 0.0;
    st[2 * PS + e] = (in && j > 1) ? src[2 * PS + e] : 0.0;
    st[3 * PS + e] = (in && i > 1 && j > 1) ? src[3 * PS + e] : 0.0;
    st[4 * PS + e] = (in && i > 1 && j < N) ? src[4 * PS + e] : 0.0;
    st[5 * PS + e] = in ? rdiv(1.0, o) : 0.0;
  }
  for (int e = tid; e < L::TOTAL - L::CI; e += TG_THREADS) sm[L::CI + e] = 0.0;
  if (tid == 0) bad = 0;
  __syncthreads();
  const Planes<double> A = planes_at(st, PS);
  const double* D = st + 5 * PS;
  const float* dl = delta ? delta + (size_t)crop * M * MLP_OUT : nullptr;
  for (int e = tid; e < PSC; e += TG_THREADS) learned::edge_cell(A, LD, NC, dl, e % LDC, e / LDC, ci, aux);
  __syncthreads();
  for (int e = tid; e < PSC; e += TG_THREADS) learned::centre_cell(A, LD, NC, e % LDC, e / LDC, ci);
  __syncthreads();
  // Galerkin operator into the lower band: row c holds O; W (d = 1), S (d = NC),
  // SW (d = NC + 1); the NW coupling of c is the SE coupling of row c + NC - 1
  for (int c = tid; c < M; c += TG_THREADS) {
    const int ic = 1 + c % NC, jc = 1 + c / NC;
    band[c * BL] = rapdev::rap_entry<0, 0>(A, LD, ci, PSC, LDC, NC, ic, jc);
    if (ic > 1) band[c * BL + 1] = rapdev::rap_entry<-1, 0>(A, LD, ci, PSC, LDC, NC, ic, jc);
    if (jc > 1) band[c * BL + NC] = rapdev::rap_entry<0, -1>(A, LD, ci, PSC, LDC, NC, ic, jc);
    if (ic > 1 && jc > 1) band[c * BL + NC + 1] = rapdev::rap_entry<-1, -1>(A, LD, ci, PSC, LDC, NC, ic, jc);
    if (ic > 1 && jc < NC) band[(c + NC - 1) * BL + NC - 1] = rapdev::rap_entry<-1, 1>(A, LD, ci, PSC, LDC, NC, ic, jc);
  }
  __syncthreads();
  if (tid < 32) {
    const bool ok = band_cholesky<N>(band);
    if (tid == 0 && !ok) bad = 1;
  }
  __syncthreads();
  if (bad) {
    if (tid == 0) atomicExch(err, 1);
    return;
  }
  for (int k = 0; k < K; ++k) {
    const double* e = vecs + ((size_t)crop * K + k) * PS;
    for (int q = tid; q < N * N; q += TG_THREADS) {
      const size_t p = (size_t)(1 + q / N) * LD + 1 + q % N;
      X[p] = e[p];
    }
    __syncthreads();
    sweep<N>(A, D, X);
    sweep<N>(A, D, X);                                   // e1 = S^2 e
    apply<N>(A, X, T);
    __syncthreads();
    restrict_fig2<N>(ci, T, FC);                         // P^T A e1
    __syncthreads();
    if (tid < 32) band_solve<N>(band, FC, U);            // u
    __syncthreads();
    interp<N>(ci, U, X, E2);                             // e2 = e1 - P u
    __syncthreads();
    for (int q = tid; q < PS; q += TG_THREADS) X[q] = E2[q];
    __syncthreads();
    sweep<N>(A, D, X);                                   // e3 = S e2
    apply<N>(A, X, T);
    __syncthreads();
    double part = 0.0;
    for (int q = tid; q < N * N; q += TG_THREADS) {
      const size_t p = (size_t)(1 + q / N) * LD + 1 + q % N;
      part = radd(part, rmul(X[p], T[p]));
    }
    const double energy = block_sum<N>(part, red);
    if (tid == 0) energies[(size_t)crop * K + k] = energy;
    if (!eref) continue;
    const double sc = rdiv(2.0 * weight, rmul((double)K, eref[(size_t)crop * K + k]));
    for (int q = tid; q < N * N; q += TG_THREADS) {
      const size_t p = (size_t)(1 + q / N) * LD + 1 + q % N;
      G[p] = rmul(sc, T[p]);                             // dL/d e3
    }
    __syncthreads();
    sweep_adjoint<N>(A, D, G, T, X);                     // g2 = S^T dL/d e3
    restrict_fig2<N>(ci, G, FC);
    __syncthreads();
    if (tid < 32) band_solve<N>(band, FC, V);            // v
    __syncthreads();
    interp<N>(ci, V, nullptr, T);                        // P v
    __syncthreads();
    apply<N>(A, T, X);                                   // A P v
    __syncthreads();
    for (int q = tid; q < N * N; q += TG_THREADS) {
      const size_t p = (size_t)(1 + q / N) * LD + 1 + q % N;
      X[p] = rsub(X[p], G[p]);                           // A P v - g2
    }
    __syncthreads();
    add_outer<N>(X, 1.0, U, dW);
    __syncthreads();
    apply<N>(A, E2, X);                                  // A e2
    __syncthreads();
    add_outer<N>(X, -1.0, V, dW);
    __syncthreads();
  }
  if (!eref) return;
  // dL/dw -> dL/d delta: each edge weight's total derivative (its own term plus
  // the two centre formulas that use it), times S_D q (1 - q); tx in FC, ty in U
  auto cc = [&](int a, int b, int kk) -> double {   // a_kk / a_O at the centre point of cell (a, b)
    if (a < 1 || b < 1 || a > NC + 1 || b > NC + 1) return 0.0;
    const size_t p = (size_t)(2 * b - 1) * LD + (2 * a - 1);
    const double o = A.a<0>(p, LD);
    const double c = kk == 1 ? A.a<1>(p, LD) : kk == 2 ? A.a<2>(p, LD) : kk == 3 ? A.a<3>(p, LD) : A.a<4>(p, LD);
    return c / o;
  };
  auto dw = [&](int kk, int a, int b) -> double {
    if (a < 0 || b < 0 || a > NC + 1 || b > NC + 1) return 0.0;
    return dW[kk * PSC + (size_t)b * LDC + a];
  };
  for (int e = tid; e < PSC; e += TG_THREADS) {
    const int ic = e % LDC, jc = e / LDC;
    double t1 = 0.0, t2 = 0.0;
    if (ic >= 1 && jc >= 1 && jc <= NC) {
      const double dll = dw(CI_LL, ic, jc) - cc(ic, jc + 1, 3) * dw(CI_LSW, ic, jc + 1) - cc(ic, jc, 4) * dw(CI_LNW, ic, jc);
      const double dlr = dw(CI_LR, ic, jc) - cc(ic, jc + 1, 3) * dw(CI_LSE, ic, jc + 1) - cc(ic, jc, 4) * dw(CI_LNE, ic, jc);
      const double sd = aux[0 * PSC + e], q = aux[1 * PSC + e];
      t1 = (dll - dlr) * sd * q * (1.0 - q);
    }
    if (ic >= 1 && ic <= NC && jc >= 1) {
      const double dlb = dw(CI_LB, ic, jc) - cc(ic + 1, jc, 1) * dw(CI_LSW, ic + 1, jc) - cc(ic, jc, 2) * dw(CI_LSE, ic, jc);
      const double dla = dw(CI_LA, ic, jc) - cc(ic + 1, jc, 1) * dw(CI_LNW, ic + 1, jc) - cc(ic, jc, 2) * dw(CI_LNE, ic, jc);
      const double sd = aux[2 * PSC + e], q = aux[3 * PSC + e];
      t2 = (dlb - dla) * sd * q * (1.0 - q);
    }
    FC[e] = t1;
    U[e] = t2;
  }
  __syncthreads();
  float* out = ddelta + (size_t)crop * M * MLP_OUT;
  for (int c = tid; c < M; c += TG_THREADS) {
    const int ic = 1 + c % NC, jc = 1 + c / NC;
    const size_t pc = (size_t)jc * LDC + ic;
    out[c * MLP_OUT + 0] = (float)(-FC[pc]);
    out[c * MLP_OUT + 1] = (float)(FC[pc + 1]);
    out[c * MLP_OUT + 2] = (float)(-U[pc]);
    out[c * MLP_OUT + 3] = (float)(U[pc + LDC]);
  }
}

// Features of every crop: (a_W + a_E)/a_O and (a_S + a_N)/a_O at the 9 fine
// points of each interior coarse point's 3x3 block; rows crop-major.
__global__ void k_features_crops(int n, const double* __restrict__ coefs, float* __restrict__ X) {
  const int nc = (n - 1) / 2, ld = n + 2;
  const int crop = blockIdx.y;
  const size_t ps = plane_size(n);
  const Planes<double> A = planes_at(coefs + (size_t)crop * 5 * ps, ps);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc * nc; c += gridDim.x * blockDim.x) {
    const int ic = 1 + c % nc, jc = 1 + c / nc;
    float* row = X + ((size_t)crop * nc * nc + c) * MLP_IN;
    int k = 0;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const size_t p = (size_t)(2 * jc + dy) * ld + (2 * ic + dx);
        const int i = 2 * ic + dx, j = 2 * jc + dy;
        // couplings to ghost points are not entries of a Dirichlet row
        const double w = i > 1 ? A.a<1>(p, ld) : 0.0, e = i < n ? A.a<2>(p, ld) : 0.0;
        const double s = j > 1 ? A.a<3>(p, ld) : 0.0, nn = j < n ? A.a<4>(p, ld) : 0.0;
        const double o = A.a<0>(p, ld);
        row[k++] = __double2float_rn(rdiv(radd(w, e), o));
        row[k++] = __double2float_rn(rdiv(radd(s, nn), o));
      }
  }
}

template <int N>
int launch_twogrid_n(int ncrop, int K, const double* coefs, const double* vecs, const float* delta, const double* eref,
                     double weight, double* energies, float* ddelta, int* err, cudaStream_t s) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(k_twogrid<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TG<N>::BYTES);
  if (attr != cudaSuccess) return cuda_check(attr, "two-grid kernel shared memory");
  k_twogrid<N><<<ncrop, TG_THREADS, TG<N>::BYTES, s>>>(K, coefs, vecs, delta, eref, weight, energies, ddelta, err);
  count_launch();
  return cuda_check(cudaGetLastError(), "two-grid kernel launch");
}

}  // namespace

bool twogrid_size_ok(int n) { return n == 7 || n == 15 || n == 31; }

int launch_twogrid(int n, int ncrop, int K, const double* coefs, const double* vecs, const float* delta,
                   const double* eref, double weight, double* energies, float* ddelta, int* err, cudaStream_t s) {
  switch (n) {
    case 7: return launch_twogrid_n<7>(ncrop, K, coefs, vecs, delta, eref, weight, energies, ddelta, err, s);
    case 15: return launch_twogrid_n<15>(ncrop, K, coefs, vecs, delta, eref, weight, energies, ddelta, err, s);
    case 31: return launch_twogrid_n<31>(ncrop, K, coefs, vecs, delta, eref, weight, energies, ddelta, err, s);
    default: return set_error(BMG_EINVAL, "two-grid loss: crop size %d is not 7, 15 or 31", n);
  }
}

void launch_features_crops(int n, int ncrop, const double* coefs, float* X, cudaStream_t s) {
  const int nc = (n - 1) / 2;
  k_features_crops<<<dim3((nc * nc + 255) / 256, ncrop), 256, 0, s>>>(n, coefs, X);
  count_launch();
}

}  // namespace bmg
