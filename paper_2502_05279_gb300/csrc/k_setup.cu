// Setup kernels of the BoxMG hierarchy (FP64): input preparation, Dendy
// operator-dependent interpolation, the Galerkin coarse operator
// A_c = P^T A P, reciprocal diagonals, the coarsest Cholesky factor and the
// FP32 / BF16 copies used by the mixed-precision cycle.
//
// Every formula keeps the operation order stated in the interface header so
// that results are reproducible bit for bit (no fused multiply-add).
#include "common.cuh"
#include "kernels.h"
#include "rap_device.cuh"

namespace bmg {

namespace {

constexpr int BX = 32, BY = 8;

// Copy a caller stencil (kind 5: O, W, S; kind 9: O, W, S, SW, NW) on an
// nx x ny grid ((ny+2) x (nx+2) planes) into the six-plane layout of the
// n x n level 0, dropping the ghost ring and ghost couplings.  With nx, ny < n
// the caller's points keep their (i, j) and every other interior point gets
// the identity row O = 1 (general sizes: the embedding reading).
__global__ void k_prepare(int n, int nx, int ny, int kind, const double* __restrict__ in, double* __restrict__ st) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int ld = n + 2;
  if (i > n + 1 || j > n + 1) return;
  size_t ps = plane_size(n), p = (size_t)j * ld + i;
  const size_t psi = (size_t)(nx + 2) * (ny + 2), q = (size_t)j * (nx + 2) + i;
  const bool caller = i >= 1 && i <= nx && j >= 1 && j <= ny;
  const bool extra = !caller && i >= 1 && i <= n && j >= 1 && j <= n;
  double o = extra ? 1.0 : 0.0, w = 0, s = 0, sw = 0, nw = 0;
  if (caller) {
    o = in[q];
    if (i > 1) w = in[psi + q];
    if (j > 1) s = in[2 * psi + q];
    if (kind == 9) {
      if (i > 1 && j > 1) sw = in[3 * psi + q];
      if (i > 1 && j < ny) nw = in[4 * psi + q];
    }
  }
  if (!BMG_IN(DBG_SETUP_STORE, p, ps)) return;
  st[p] = o;
  st[ps + p] = w;
  st[2 * ps + p] = s;
  st[3 * ps + p] = sw;
  st[4 * ps + p] = nw;
  st[5 * ps + p] = 0.0;
}

__global__ void k_dinv(int n, double* __restrict__ st, int* err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
  if (i > n || j > n) return;
  size_t ps = plane_size(n), p = (size_t)j * (n + 2) + i;
  double o = st[p];
  if (!(o > 0.0)) atomicExch(err, 1);
  if (BMG_IN(DBG_SETUP_STORE, p, ps)) st[5 * ps + p] = rdiv(1.0, o);
}

// ---- Dendy interpolation -------------------------------------------------
// x-edge fine point (2ic-1, 2jc), 1 <= ic <= nc+1, 1 <= jc <= nc:
//   D = (a_S + a_O) + a_N, LL = -((a_SW + a_W) + a_NW) / D, LR = -((a_SE + a_E) + a_NE) / D.
// y-edge fine point (2ic, 2jc-1), 1 <= ic <= nc, 1 <= jc <= nc+1:
//   D = (a_W + a_O) + a_E, LB = -((a_SW + a_S) + a_SE) / D, LA = -((a_NW + a_N) + a_NE) / D.
// Outside those ranges the weights are 0 (the point is a ghost point).
// Galerkin operators of coarse levels are not M-matrices in general, so D may
// be negative (the weights then stay a partition of unity); only D = 0 or a
// non-finite D is an error.
struct EdgeW {
  double lo, hi;
};

__device__ __forceinline__ EdgeW xedge(const Planes<double>& A, int ld, int nc, int ic, int jc, int* err) {
  if (ic < 1 || ic > nc + 1 || jc < 1 || jc > nc) return EdgeW{0.0, 0.0};
  size_t p = (size_t)(2 * jc) * ld + (2 * ic - 1);
  double D = radd(radd(A.a<3>(p, ld), A.a<0>(p, ld)), A.a<4>(p, ld));
  if (!(fabs(D) > 0.0) || isinf(D)) atomicExch(err, 2);   // zero or non-finite: no weight exists
  double ll = -rdiv(radd(radd(A.a<5>(p, ld), A.a<1>(p, ld)), A.a<7>(p, ld)), D);
  double lr = -rdiv(radd(radd(A.a<8>(p, ld), A.a<2>(p, ld)), A.a<6>(p, ld)), D);
  return EdgeW{ll, lr};
}

__device__ __forceinline__ EdgeW yedge(const Planes<double>& A, int ld, int nc, int ic, int jc, int* err) {
  if (ic < 1 || ic > nc || jc < 1 || jc > nc + 1) return EdgeW{0.0, 0.0};
  size_t p = (size_t)(2 * jc - 1) * ld + 2 * ic;
  double D = radd(radd(A.a<1>(p, ld), A.a<0>(p, ld)), A.a<2>(p, ld));
  if (!(fabs(D) > 0.0) || isinf(D)) atomicExch(err, 2);   // zero or non-finite: no weight exists
  double lb = -rdiv(radd(radd(A.a<5>(p, ld), A.a<3>(p, ld)), A.a<8>(p, ld)), D);
  double la = -rdiv(radd(radd(A.a<7>(p, ld), A.a<4>(p, ld)), A.a<6>(p, ld)), D);
  return EdgeW{lb, la};
}

// One thread per coarse cell (ic, jc), 1..nc+1 each: its x-edge and y-edge
// points and the centre point (2ic-1, 2jc-1), whose row of A is solved with
// the four edge neighbours already interpolated:
//   LSW = -((a_SW + a_W LB_w) + a_S LL_s) / a_O, LSE = -((a_SE + a_E LB_e) + a_S LR_s) / a_O,
//   LNW = -((a_NW + a_W LA_w) + a_N LL_n) / a_O, LNE = -((a_NE + a_E LA_e) + a_N LR_n) / a_O.
// Neighbour edge weights are recomputed with the same code, hence identical.
__global__ void k_dendy(int n, const double* __restrict__ st, double* __restrict__ ci, int* err) {
  int ic = blockIdx.x * blockDim.x + threadIdx.x;
  int jc = blockIdx.y * blockDim.y + threadIdx.y;
  int nc = (n - 1) / 2, ldc = nc + 2, ld = n + 2;
  if (ic > nc + 1 || jc > nc + 1) return;
  size_t pc = (size_t)jc * ldc + ic, psc = plane_size(nc);
  if (!BMG_IN(DBG_SETUP_STORE, pc, psc)) return;
  if (ic == 0 || jc == 0) {
#pragma unroll
    for (int k = 0; k < 8; ++k) ci[k * psc + pc] = 0.0;
    return;
  }
  Planes<double> A = planes_at(st, plane_size(n));
  EdgeW xe = xedge(A, ld, nc, ic, jc, err);
  EdgeW ye = yedge(A, ld, nc, ic, jc, err);
  EdgeW yw = yedge(A, ld, nc, ic - 1, jc, err);   // west neighbour of the centre
  EdgeW xs = xedge(A, ld, nc, ic, jc - 1, err);   // south neighbour of the centre
  size_t p = (size_t)(2 * jc - 1) * ld + (2 * ic - 1);
  double aO = A.a<0>(p, ld), aW = A.a<1>(p, ld), aE = A.a<2>(p, ld), aS = A.a<3>(p, ld), aN = A.a<4>(p, ld);
  double aSW = A.a<5>(p, ld), aNE = A.a<6>(p, ld), aNW = A.a<7>(p, ld), aSE = A.a<8>(p, ld);
  if (!(aO > 0.0)) atomicExch(err, 2);
  double sw = -rdiv(radd(radd(aSW, rmul(aW, yw.lo)), rmul(aS, xs.lo)), aO);
  double se = -rdiv(radd(radd(aSE, rmul(aE, ye.lo)), rmul(aS, xs.hi)), aO);
  double nw = -rdiv(radd(radd(aNW, rmul(aW, yw.hi)), rmul(aN, xe.lo)), aO);
  double ne = -rdiv(radd(radd(aNE, rmul(aE, ye.hi)), rmul(aN, xe.hi)), aO);
  ci[CI_LSW * psc + pc] = sw;
  ci[CI_LSE * psc + pc] = se;
  ci[CI_LNW * psc + pc] = nw;
  ci[CI_LNE * psc + pc] = ne;
  ci[CI_LL * psc + pc] = xe.lo;
  ci[CI_LR * psc + pc] = xe.hi;
  ci[CI_LB * psc + pc] = ye.lo;
  ci[CI_LA * psc + pc] = ye.hi;
}

__global__ void k_rap(int n, const double* __restrict__ st, const double* __restrict__ ci,
                      double* __restrict__ stc) {
  int ic = blockIdx.x * blockDim.x + threadIdx.x;
  int jc = blockIdx.y * blockDim.y + threadIdx.y;
  int nc = (n - 1) / 2, ldc = nc + 2, ld = n + 2;
  if (ic > nc + 1 || jc > nc + 1) return;
  size_t psc = plane_size(nc), pc = (size_t)jc * ldc + ic;
  if (!BMG_IN(DBG_SETUP_STORE, pc, psc)) return;
  if (ic == 0 || jc == 0 || ic == nc + 1 || jc == nc + 1) {
#pragma unroll
    for (int k = 0; k < 6; ++k) stc[k * psc + pc] = 0.0;
    return;
  }
  Planes<double> A = planes_at(st, plane_size(n));
  double o = rapdev::rap_entry<0, 0>(A, ld, ci, psc, ldc, nc, ic, jc);
  double w = rapdev::rap_entry<-1, 0>(A, ld, ci, psc, ldc, nc, ic, jc);
  double s = rapdev::rap_entry<0, -1>(A, ld, ci, psc, ldc, nc, ic, jc);
  double sw = rapdev::rap_entry<-1, -1>(A, ld, ci, psc, ldc, nc, ic, jc);
  double nw = rapdev::rap_entry<-1, 1>(A, ld, ci, psc, ldc, nc, ic, jc);
  stc[pc] = o;
  stc[psc + pc] = ic > 1 ? w : 0.0;
  stc[2 * psc + pc] = jc > 1 ? s : 0.0;
  stc[3 * psc + pc] = (ic > 1 && jc > 1) ? sw : 0.0;
  stc[4 * psc + pc] = (ic > 1 && jc < nc) ? nw : 0.0;
  stc[5 * psc + pc] = 0.0;
}

// ---- coarsest Cholesky (one thread; m = n^2 <= 225) -----------------------
// Dense A over lexicographic unknowns, then right-looking Cholesky: for each
// pivot k, L_kk = sqrt(a_kk), L_ik = a_ik / L_kk, then a_ij -= L_ik L_jk for
// j = k+1.., i = j.. (lower triangle).
__global__ void k_factor(int n, const double* __restrict__ st, double* __restrict__ L, double* __restrict__ a,
                         int* err) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int m = n * n, ld = n + 2;
  Planes<double> A = planes_at(st, plane_size(n));
  for (int k = 0; k < m * m; ++k) {
    a[k] = 0.0;
    L[k] = 0.0;
  }
  for (int j = 1; j <= n; ++j)
    for (int i = 1; i <= n; ++i) {
      size_t p = (size_t)j * ld + i;
      int r = (j - 1) * n + (i - 1);
      double v[9] = {A.a<0>(p, ld), A.a<1>(p, ld), A.a<2>(p, ld), A.a<3>(p, ld), A.a<4>(p, ld),
                     A.a<5>(p, ld), A.a<6>(p, ld), A.a<7>(p, ld), A.a<8>(p, ld)};
      for (int k = 0; k < 9; ++k) {
        int ii = i + nbr_dx(k), jj = j + nbr_dy(k);
        if (ii >= 1 && ii <= n && jj >= 1 && jj <= n) a[(size_t)r * m + (jj - 1) * n + (ii - 1)] = v[k];
      }
    }
  for (int k = 0; k < m; ++k) {
    double akk = a[(size_t)k * m + k];
    if (!(akk > 0.0)) {
      atomicExch(err, 3);
      return;
    }
    double lkk = __dsqrt_rn(akk);
    L[(size_t)k * m + k] = lkk;
    for (int i = k + 1; i < m; ++i) L[(size_t)i * m + k] = rdiv(a[(size_t)i * m + k], lkk);
    for (int j = k + 1; j < m; ++j)
      for (int i = j; i < m; ++i)
        a[(size_t)i * m + j] = rsub(a[(size_t)i * m + j], rmul(L[(size_t)i * m + k], L[(size_t)j * m + k]));
  }
}

// ---- FP32 / BF16 copies -----------------------------------------------------
__global__ void k_round32(size_t count, const double* __restrict__ in, float* __restrict__ out) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < count; k += (size_t)gridDim.x * blockDim.x)
    out[k] = __double2float_rn(in[k]);
}

__device__ __forceinline__ float bf16_of(double v) { return __bfloat162float(__float2bfloat16_rn(__double2float_rn(v))); }

// off16: W, S, SW, NW as bf16(fl32(a)); od32: O32, D32 with
// O32 = fl32(sum_NBR a) - W_b - E_b - S_b - N_b - SW_b - NE_b - NW_b - SE_b, D32 = 1 / O32.
__global__ void k_lower_bf16(int n, const double* __restrict__ st, __nv_bfloat16* __restrict__ off16,
                             float* __restrict__ od32, size_t pst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int ld = n + 2;
  if (i > n + 1 || j > n + 1) return;
  size_t ps = plane_size(n), p = (size_t)j * ld + i;
#pragma unroll
  for (int k = 0; k < 4; ++k) off16[k * pst + p] = __float2bfloat16_rn(__double2float_rn(st[(k + 1) * ps + p]));
  if (i < 1 || i > n || j < 1 || j > n) {
    od32[p] = 0.0f;
    od32[pst + p] = 0.0f;
    return;
  }
  Planes<double> A = planes_at(st, ps);
  double rs = A.a<0>(p, ld);
  rs = radd(rs, A.a<1>(p, ld));
  rs = radd(rs, A.a<2>(p, ld));
  rs = radd(rs, A.a<3>(p, ld));
  rs = radd(rs, A.a<4>(p, ld));
  rs = radd(rs, A.a<5>(p, ld));
  rs = radd(rs, A.a<6>(p, ld));
  rs = radd(rs, A.a<7>(p, ld));
  rs = radd(rs, A.a<8>(p, ld));
  float o = __double2float_rn(rs);
  o = rsub(o, bf16_of(A.a<1>(p, ld)));
  o = rsub(o, bf16_of(A.a<2>(p, ld)));
  o = rsub(o, bf16_of(A.a<3>(p, ld)));
  o = rsub(o, bf16_of(A.a<4>(p, ld)));
  o = rsub(o, bf16_of(A.a<5>(p, ld)));
  o = rsub(o, bf16_of(A.a<6>(p, ld)));
  o = rsub(o, bf16_of(A.a<7>(p, ld)));
  o = rsub(o, bf16_of(A.a<8>(p, ld)));
  od32[p] = o;
  od32[pst + p] = rdiv(1.0f, o);
}

dim3 grid2(int nx, int ny) { return dim3((nx + BX - 1) / BX, (ny + BY - 1) / BY); }

// The packed stencils read by the bulk-copy sweeps: one point's five FP32
// words d, w, s, sw, nw, or three words d, w | s << 16, sw | nw << 16 of a
// BF16 level (the bf16 bit patterns as stored).  The same values as the
// planes, in another layout.
__global__ void k_pack32(int n, const float* __restrict__ st32, float* __restrict__ pk, size_t pst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > n + 1 || j > n + 1) return;
  const size_t p = (size_t)j * (n + 2) + i;
  float* o = pk + PK_WORDS_F32 * p;
  o[0] = st32[5 * pst + p];
  o[1] = st32[pst + p];
  o[2] = st32[2 * pst + p];
  o[3] = st32[3 * pst + p];
  o[4] = st32[4 * pst + p];
}

__global__ void k_pack_bf16(int n, const __nv_bfloat16* __restrict__ off16, const float* __restrict__ od32,
                            float* __restrict__ pk, size_t pst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > n + 1 || j > n + 1) return;
  const size_t p = (size_t)j * (n + 2) + i;
  auto bits = [](__nv_bfloat16 v) { return (unsigned)__bfloat16_as_ushort(v); };
  unsigned* o = reinterpret_cast<unsigned*>(pk + PK_WORDS_BF16 * p);
  o[0] = __float_as_uint(od32[pst + p]);
  o[1] = bits(off16[p]) | (bits(off16[pst + p]) << 16);
  o[2] = bits(off16[2 * pst + p]) | (bits(off16[3 * pst + p]) << 16);
}

}  // namespace

// Interior of an nx x ny grid array into / out of the n x n layout (the other
// points of the destination are left as they are).
__global__ void k_embed_vec(int nx, int ny, int n, const double* __restrict__ in, double* __restrict__ out, int back) {
  int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
  if (i > nx || j > ny) return;
  const size_t pc = (size_t)j * (nx + 2) + i, pn = (size_t)j * (n + 2) + i;
  if (back)
    out[pc] = in[pn];
  else
    out[pn] = in[pc];
}

void launch_embed_vec(int nx, int ny, int n, const double* in, double* out, bool back, cudaStream_t s) {
  k_embed_vec<<<grid2(nx, ny), dim3(BX, BY), 0, s>>>(nx, ny, n, in, out, back ? 1 : 0);
  count_launch();
}

void launch_prepare(int n, int nx, int ny, int kind, const double* coef_in, double* st, int* err, cudaStream_t s) {
  k_prepare<<<grid2(n + 2, n + 2), dim3(BX, BY), 0, s>>>(n, nx, ny, kind, coef_in, st);
  count_launch();
  k_dinv<<<grid2(n, n), dim3(BX, BY), 0, s>>>(n, st, err);
  count_launch();
}

void launch_dendy(int n, const double* st, double* ci, int* err, cudaStream_t s) {
  int nc = (n - 1) / 2;
  k_dendy<<<grid2(nc + 2, nc + 2), dim3(BX, BY), 0, s>>>(n, st, ci, err);
  count_launch();
}

void launch_rap(int n, const double* st, const double* ci, double* stc, cudaStream_t s) {
  int nc = (n - 1) / 2;
  k_rap<<<grid2(nc + 2, nc + 2), dim3(BX, BY), 0, s>>>(n, st, ci, stc);
  count_launch();
}

void launch_dinv(int n, double* st, int* err, cudaStream_t s) {
  k_dinv<<<grid2(n, n), dim3(BX, BY), 0, s>>>(n, st, err);
  count_launch();
}

void launch_factor(int n, const double* st, double* L, double* work, int* err, cudaStream_t s) {
  k_factor<<<1, 1, 0, s>>>(n, st, L, work, err);
  count_launch();
}

void launch_lower32(int n, const double* st, float* st32, const double* ci, float* ci32, cudaStream_t s) {
  if (st) {   // plane k of st32 starts plane_stride32(n) elements after plane k - 1
    size_t cnt = plane_size(n), pst = plane_stride32(n);
    for (int k = 0; k < 6; ++k) {
      k_round32<<<(unsigned)((cnt + 255) / 256 < 4096 ? (cnt + 255) / 256 : 4096), 256, 0, s>>>(cnt, st + k * cnt,
                                                                                              st32 + k * pst);
      count_launch();
    }
  }
  if (ci) {
    size_t cc = 8 * plane_size((n - 1) / 2);
    k_round32<<<(unsigned)((cc + 255) / 256 < 4096 ? (cc + 255) / 256 : 4096), 256, 0, s>>>(cc, ci, ci32);
    count_launch();
  }
}

void launch_lower_bf16(int n, const double* st, __nv_bfloat16* off16, float* od32, cudaStream_t s) {
  k_lower_bf16<<<grid2(n + 2, n + 2), dim3(BX, BY), 0, s>>>(n, st, off16, od32, plane_stride32(n));
  count_launch();
}

void launch_pack32(int n, const float* st32, float* pk, cudaStream_t s) {
  k_pack32<<<grid2(n + 2, n + 2), dim3(BX, BY), 0, s>>>(n, st32, pk, plane_stride32(n));
  count_launch();
}

void launch_pack_bf16(int n, const __nv_bfloat16* off16, const float* od32, float* pk, cudaStream_t s) {
  k_pack_bf16<<<grid2(n + 2, n + 2), dim3(BX, BY), 0, s>>>(n, off16, od32, pk, plane_stride32(n));
  count_launch();
}

}  // namespace bmg
