// Learned interpolation: features, the 18-64-64-4 GELU network (FP32 training
// forward/backward, BF16 tensor-core inference), the learned weights (Dendy's
// edge sums split by the network's logits, Dendy's centre formula) and the
// test-vector training loss with its gradient, plus Adam.  The paper has no
// learned component; the method is the project's extension of Dendy's
// interpolation, with Dendy's weights exactly at zero network output.
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"
#include "kernels.h"
#include "learned.h"
#include "learned_device.cuh"

namespace bmg {
namespace {

constexpr int NI = MLP_IN, NH = MLP_HID, NO = MLP_OUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NI * NH, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH * NO, NPAR = OFF_B3 + NO;
static_assert(NPAR == MLP_PARAMS, "parameter layout");

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// ---- features: (a_W + a_E)/a_O and (a_S + a_N)/a_O at the 9 fine points of
// the 3x3 block of every interior coarse point (dy outer, dx inner) ------------
__global__ void k_features(int n, const double* __restrict__ st, float* __restrict__ X) {
  int ic = blockIdx.x * blockDim.x + threadIdx.x + 1;
  int jc = blockIdx.y * blockDim.y + threadIdx.y + 1;
  int nc = (n - 1) / 2, ld = n + 2;
  if (ic > nc || jc > nc) return;
  Planes<double> A = planes_at(st, plane_size(n));
  float* row = X + ((size_t)(jc - 1) * nc + (ic - 1)) * NI;
  int k = 0;
  for (int dy = -1; dy <= 1; ++dy)
    for (int dx = -1; dx <= 1; ++dx) {
      size_t p = (size_t)(2 * jc + dy) * ld + (2 * ic + dx);
      double o = A.a<0>(p, ld);
      row[k++] = __double2float_rn(rdiv(radd(A.a<1>(p, ld), A.a<2>(p, ld)), o));
      row[k++] = __double2float_rn(rdiv(radd(A.a<3>(p, ld), A.a<4>(p, ld)), o));
    }
}

// ---- training forward (FP32, one row per thread, weights in shared memory) ----
__global__ void k_mlp_fwd(const float* __restrict__ X, int M, const float* __restrict__ par, float* __restrict__ Z1,
                          float* __restrict__ Z2, float* __restrict__ out) {
  __shared__ float w[NPAR];
  for (int k = threadIdx.x; k < NPAR; k += blockDim.x) w[k] = par[k];
  __syncthreads();
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= M) return;
  float x[NI], h1[NH], h2[NH];
  for (int k = 0; k < NI; ++k) x[k] = X[(size_t)r * NI + k];
  for (int j = 0; j < NH; ++j) {
    float z = w[OFF_B1 + j];
    for (int k = 0; k < NI; ++k) z = fmaf(x[k], w[OFF_W1 + k * NH + j], z);
    Z1[(size_t)r * NH + j] = z;
    h1[j] = gelu(z);
  }
  for (int j = 0; j < NH; ++j) {
    float z = w[OFF_B2 + j];
    for (int k = 0; k < NH; ++k) z = fmaf(h1[k], w[OFF_W2 + k * NH + j], z);
    Z2[(size_t)r * NH + j] = z;
    h2[j] = gelu(z);
  }
  for (int j = 0; j < NO; ++j) {
    float z = w[OFF_B3 + j];
    for (int k = 0; k < NH; ++k) z = fmaf(h2[k], w[OFF_W3 + k * NO + j], z);
    out[(size_t)r * NO + j] = z;
  }
}

// ---- training backward: per-row deltas, then per-block partial weight gradients
// over the block's rows (no atomics); a second kernel sums the block partials in
// a fixed order. ------------------------------------------------------------------
constexpr int BR = 32;   // rows per block of the backward kernel
__global__ void __launch_bounds__(256) k_mlp_bwd(const float* __restrict__ X, int M, const float* __restrict__ par,
                                                 const float* __restrict__ Z1, const float* __restrict__ Z2,
                                                 const float* __restrict__ dout, float* __restrict__ partial) {
  __shared__ float sx[BR][NI], sh1[BR][NH], sd1[BR][NH], sh2[BR][NH], sd2[BR][NH], so[BR][NO];
  const int r0 = blockIdx.x * BR;
  const int t = threadIdx.x;
  if (t < BR) {
    int r = r0 + t;
    bool ok = r < M;
    float d[NO], dh[NH];
    for (int j = 0; j < NO; ++j) {
      d[j] = ok ? dout[(size_t)r * NO + j] : 0.0f;
      so[t][j] = d[j];
    }
    for (int k = 0; k < NI; ++k) sx[t][k] = ok ? X[(size_t)r * NI + k] : 0.0f;
    for (int k = 0; k < NH; ++k) {
      float z2 = ok ? Z2[(size_t)r * NH + k] : 0.0f;
      float s = 0.0f;
      for (int j = 0; j < NO; ++j) s = fmaf(par[OFF_W3 + k * NO + j], d[j], s);
      sh2[t][k] = ok ? gelu(z2) : 0.0f;
      sd2[t][k] = ok ? s * gelu_grad(z2) : 0.0f;
    }
    for (int k = 0; k < NH; ++k) {
      float s = 0.0f;
      for (int j = 0; j < NH; ++j) s = fmaf(par[OFF_W2 + k * NH + j], sd2[t][j], s);
      dh[k] = s;
    }
    for (int k = 0; k < NH; ++k) {
      float z1 = ok ? Z1[(size_t)r * NH + k] : 0.0f;
      sh1[t][k] = ok ? gelu(z1) : 0.0f;
      sd1[t][k] = ok ? dh[k] * gelu_grad(z1) : 0.0f;
    }
  }
  __syncthreads();
  float* out = partial + (size_t)blockIdx.x * NPAR;
  for (int e = t; e < NPAR; e += blockDim.x) {
    float s = 0.0f;
    if (e < OFF_B1) {
      int k = e / NH, j = e % NH;
      for (int r = 0; r < BR; ++r) s = fmaf(sx[r][k], sd1[r][j], s);
    } else if (e < OFF_W2) {
      int j = e - OFF_B1;
      for (int r = 0; r < BR; ++r) s += sd1[r][j];
    } else if (e < OFF_B2) {
      int k = (e - OFF_W2) / NH, j = (e - OFF_W2) % NH;
      for (int r = 0; r < BR; ++r) s = fmaf(sh1[r][k], sd2[r][j], s);
    } else if (e < OFF_W3) {
      int j = e - OFF_B2;
      for (int r = 0; r < BR; ++r) s += sd2[r][j];
    } else if (e < OFF_B3) {
      int k = (e - OFF_W3) / NO, j = (e - OFF_W3) % NO;
      for (int r = 0; r < BR; ++r) s = fmaf(sh2[r][k], so[r][j], s);
    } else {
      int j = e - OFF_B3;
      for (int r = 0; r < BR; ++r) s += so[r][j];
    }
    out[e] = s;
  }
}

__global__ void k_sum_partials(const float* __restrict__ partial, int nb, float* __restrict__ grad) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NPAR) return;
  float s = 0.0f;
  for (int b = 0; b < nb; ++b) s += partial[(size_t)b * NPAR + e];
  grad[e] = s;
}

__global__ void k_adam(float* __restrict__ par, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NPAR) return;
  float g = grad[e];
  float mm = b1 * m[e] + (1.0f - b1) * g;
  float vv = b2 * v[e] + (1.0f - b2) * g * g;
  m[e] = mm;
  v[e] = vv;
  par[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// ---- learned weights (FP64) --------------------------------------------------------------
// delta: (nc*nc, 4) logits (W, E, S, N edge of each interior coarse point);
// the per-cell formulas are in learned_device.cuh.
__global__ void k_learned_edges(int n, const double* __restrict__ st, const float* __restrict__ delta,
                                double* __restrict__ ci, double* __restrict__ aux) {
  int ic = blockIdx.x * blockDim.x + threadIdx.x;
  int jc = blockIdx.y * blockDim.y + threadIdx.y;
  int nc = (n - 1) / 2;
  if (ic > nc + 1 || jc > nc + 1) return;
  learned::edge_cell(planes_at(st, plane_size(n)), n + 2, nc, delta, ic, jc, ci, aux);
}

__global__ void k_learned_centres(int n, const double* __restrict__ st, double* __restrict__ ci) {
  int ic = blockIdx.x * blockDim.x + threadIdx.x;
  int jc = blockIdx.y * blockDim.y + threadIdx.y;
  int nc = (n - 1) / 2;
  if (ic > nc + 1 || jc > nc + 1) return;
  learned::centre_cell(planes_at(st, plane_size(n)), n + 2, nc, ic, jc, ci);
}

// ---- test-vector loss ------------------------------------------------------------------
// err = v - P R v over the interior (R: values at coarse points).
__global__ void k_tv_err(int n, const double* __restrict__ ci, const double* __restrict__ v, double* __restrict__ err) {
  int ic = blockIdx.x * blockDim.x + threadIdx.x + 1;
  int jc = blockIdx.y * blockDim.y + threadIdx.y + 1;
  int nc = (n - 1) / 2, ldc = nc + 2, ld = n + 2;
  if (ic > nc + 1 || jc > nc + 1) return;
  size_t psc = plane_size(nc), pc = (size_t)jc * ldc + ic;
  auto vc = [&](int a, int b) -> double {   // v at coarse point (a, b), 0 on ghosts
    return (a < 1 || b < 1 || a > nc || b > nc) ? 0.0 : v[(size_t)(2 * b) * ld + 2 * a];
  };
  double e_sw = vc(ic - 1, jc - 1), e_se = vc(ic, jc - 1), e_nw = vc(ic - 1, jc), e_ne = vc(ic, jc);
  size_t pf = (size_t)(2 * jc) * ld + 2 * ic;
  if (ic <= nc && jc <= nc) err[pf] = 0.0;
  if (jc <= nc) {
    double t = radd(rmul(ci[CI_LL * psc + pc], e_nw), rmul(ci[CI_LR * psc + pc], e_ne));
    err[pf - 1] = rsub(v[pf - 1], t);
  }
  if (ic <= nc) {
    double t = radd(rmul(ci[CI_LB * psc + pc], e_se), rmul(ci[CI_LA * psc + pc], e_ne));
    err[pf - ld] = rsub(v[pf - ld], t);
  }
  double t = rmul(ci[CI_LSW * psc + pc], e_sw);
  t = radd(t, rmul(ci[CI_LSE * psc + pc], e_se));
  t = radd(t, rmul(ci[CI_LNW * psc + pc], e_nw));
  t = radd(t, rmul(ci[CI_LNE * psc + pc], e_ne));
  err[pf - ld - 1] = rsub(v[pf - ld - 1], t);
}

// Ae = A err and one block partial of err . Ae per 256-thread block (row-strided).
__global__ void __launch_bounds__(256) k_tv_apply(int n, const double* __restrict__ st, const double* __restrict__ err,
                                                  double* __restrict__ Ae, double* __restrict__ partials) {
  __shared__ double red[256];
  int ld = n + 2;
  Planes<double> A = planes_at(st, plane_size(n));
  double acc = 0.0;
  for (int j = 1 + blockIdx.x; j <= n; j += gridDim.x)
    for (int i = 1 + threadIdx.x; i <= n; i += 256) {
      size_t p = (size_t)j * ld + i;
      double s = rmul(A.a<0>(p, ld), err[p]);
      s = radd(s, rmul(A.a<1>(p, ld), err[p - 1]));
      s = radd(s, rmul(A.a<2>(p, ld), err[p + 1]));
      s = radd(s, rmul(A.a<3>(p, ld), err[p - ld]));
      s = radd(s, rmul(A.a<4>(p, ld), err[p + ld]));
      s = radd(s, rmul(A.a<5>(p, ld), err[p - ld - 1]));
      s = radd(s, rmul(A.a<6>(p, ld), err[p + ld + 1]));
      s = radd(s, rmul(A.a<7>(p, ld), err[p + ld - 1]));
      s = radd(s, rmul(A.a<8>(p, ld), err[p + 1 - ld]));
      Ae[p] = s;
      acc = radd(acc, rmul(err[p], s));
    }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void k_tv_energy(const double* __restrict__ partials, int np, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int k = 0; k < np; ++k) s += partials[k];
  *out = s;
}

// dW (8 planes) += g(p) v(c) over the K vectors, g = -2 Ae / (K E_ref).
__global__ void k_tv_dw(int n, int K, const double* __restrict__ vecs, const double* __restrict__ Aes,
                        const double* __restrict__ scale, double* __restrict__ dW) {
  int ic = blockIdx.x * blockDim.x + threadIdx.x + 1;
  int jc = blockIdx.y * blockDim.y + threadIdx.y + 1;
  int nc = (n - 1) / 2, ldc = nc + 2, ld = n + 2;
  if (ic > nc + 1 || jc > nc + 1) return;
  size_t psc = plane_size(nc), pc = (size_t)jc * ldc + ic, ps = plane_size(n);
  double d[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  size_t pf = (size_t)(2 * jc) * ld + 2 * ic;
  for (int k = 0; k < K; ++k) {
    const double* v = vecs + (size_t)k * ps;
    const double* Ae = Aes + (size_t)k * ps;
    double sc = scale[k];
    auto vc = [&](int a, int b) -> double {
      return (a < 1 || b < 1 || a > nc || b > nc) ? 0.0 : v[(size_t)(2 * b) * ld + 2 * a];
    };
    double e_sw = vc(ic - 1, jc - 1), e_se = vc(ic, jc - 1), e_nw = vc(ic - 1, jc), e_ne = vc(ic, jc);
    if (jc <= nc) {
      double g = sc * Ae[pf - 1];
      d[CI_LL] += g * e_nw;
      d[CI_LR] += g * e_ne;
    }
    if (ic <= nc) {
      double g = sc * Ae[pf - ld];
      d[CI_LB] += g * e_se;
      d[CI_LA] += g * e_ne;
    }
    double g = sc * Ae[pf - ld - 1];
    d[CI_LSW] += g * e_sw;
    d[CI_LSE] += g * e_se;
    d[CI_LNW] += g * e_nw;
    d[CI_LNE] += g * e_ne;
  }
  for (int k = 0; k < 8; ++k) dW[k * psc + pc] = d[k];
}

// Per cell: total derivative of its x-edge and y-edge splits (direct term plus
// the two centres that use each edge weight), as t = (dw1 - dw2) S_D q (1-q).
__global__ void k_tv_edge_t(int n, const double* __restrict__ st, const double* __restrict__ dW,
                            const double* __restrict__ aux, double* __restrict__ tx, double* __restrict__ ty) {
  int ic = blockIdx.x * blockDim.x + threadIdx.x;
  int jc = blockIdx.y * blockDim.y + threadIdx.y;
  int nc = (n - 1) / 2, ldc = nc + 2, ld = n + 2;
  if (ic > nc + 1 || jc > nc + 1) return;
  size_t psc = plane_size(nc), pc = (size_t)jc * ldc + ic;
  Planes<double> A = planes_at(st, plane_size(n));
  // a_x / a_O at the centre point of cell (a, b) = fine (2a-1, 2b-1); 0 outside 1..nc+1
  auto cc = [&](int a, int b, int K) -> double {
    if (a < 1 || b < 1 || a > nc + 1 || b > nc + 1) return 0.0;
    size_t p = (size_t)(2 * b - 1) * ld + (2 * a - 1);
    double o = A.a<0>(p, ld);
    double c = K == 1 ? A.a<1>(p, ld) : K == 2 ? A.a<2>(p, ld) : K == 3 ? A.a<3>(p, ld) : A.a<4>(p, ld);
    return c / o;
  };
  auto dw = [&](int k, int a, int b) -> double {
    if (a < 0 || b < 0 || a > nc + 1 || b > nc + 1) return 0.0;
    return dW[k * psc + (size_t)b * ldc + a];
  };
  double t1 = 0.0, t2 = 0.0;
  if (ic >= 1 && jc >= 1 && jc <= nc) {
    double dll = dw(CI_LL, ic, jc) - cc(ic, jc + 1, 3) * dw(CI_LSW, ic, jc + 1) - cc(ic, jc, 4) * dw(CI_LNW, ic, jc);
    double dlr = dw(CI_LR, ic, jc) - cc(ic, jc + 1, 3) * dw(CI_LSE, ic, jc + 1) - cc(ic, jc, 4) * dw(CI_LNE, ic, jc);
    double sd = aux[0 * psc + pc], q = aux[1 * psc + pc];
    t1 = (dll - dlr) * sd * q * (1.0 - q);
  }
  if (ic >= 1 && ic <= nc && jc >= 1) {
    double dlb = dw(CI_LB, ic, jc) - cc(ic + 1, jc, 1) * dw(CI_LSW, ic + 1, jc) - cc(ic, jc, 2) * dw(CI_LSE, ic, jc);
    double dla = dw(CI_LA, ic, jc) - cc(ic + 1, jc, 1) * dw(CI_LNW, ic + 1, jc) - cc(ic, jc, 2) * dw(CI_LNE, ic, jc);
    double sd = aux[2 * psc + pc], q = aux[3 * psc + pc];
    t2 = (dlb - dla) * sd * q * (1.0 - q);
  }
  tx[pc] = t1;
  ty[pc] = t2;
}

// dL/d delta of interior coarse point (ic, jc): W from its own cell's x-edge,
// E from cell (ic+1, jc), S from its own y-edge, N from cell (ic, jc+1).
__global__ void k_tv_ddelta(int n, const double* __restrict__ tx, const double* __restrict__ ty,
                            float* __restrict__ dd) {
  int ic = blockIdx.x * blockDim.x + threadIdx.x + 1;
  int jc = blockIdx.y * blockDim.y + threadIdx.y + 1;
  int nc = (n - 1) / 2, ldc = nc + 2;
  if (ic > nc || jc > nc) return;
  size_t pc = (size_t)jc * ldc + ic;
  float* o = dd + ((size_t)(jc - 1) * nc + (ic - 1)) * NO;
  o[0] = (float)(-tx[pc]);
  o[1] = (float)(tx[pc + 1]);
  o[2] = (float)(-ty[pc]);
  o[3] = (float)(ty[pc + ldc]);
}

// ---- inference on BF16 tensor cores (mma.sync m16n8k16, FP32 accumulate) ---------------
// One warp per 16 rows.  Layer outputs stay in registers: the accumulator
// fragments of two neighbouring 8-column tiles form the A fragment of the next
// layer's 16-column k-tile.  Weights are kept in shared memory as bf16, K x N
// row-major, zero-padded to K = 32 (layer 1) and N = 8 (layer 3).
__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<unsigned*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int K1 = 32;   // layer-1 K padded
__global__ void __launch_bounds__(128) k_mlp_infer(const float* __restrict__ X, int M, const float* __restrict__ par,
                                                   float* __restrict__ out) {
  __shared__ __nv_bfloat16 w1[K1 * NH], w2[NH * NH], w3[NH * 8];
  __shared__ float b1[NH], b2[NH], b3[8];
  for (int e = threadIdx.x; e < K1 * NH; e += blockDim.x) {
    int k = e / NH, j = e % NH;
    w1[e] = __float2bfloat16_rn(k < NI ? par[OFF_W1 + k * NH + j] : 0.0f);
  }
  for (int e = threadIdx.x; e < NH * NH; e += blockDim.x) w2[e] = __float2bfloat16_rn(par[OFF_W2 + e]);
  for (int e = threadIdx.x; e < NH * 8; e += blockDim.x) {
    int k = e / 8, j = e % 8;
    w3[e] = __float2bfloat16_rn(j < NO ? par[OFF_W3 + k * NO + j] : 0.0f);
  }
  for (int e = threadIdx.x; e < NH; e += blockDim.x) {
    b1[e] = par[OFF_B1 + e];
    b2[e] = par[OFF_B2 + e];
  }
  if (threadIdx.x < 8) b3[threadIdx.x] = threadIdx.x < NO ? par[OFF_B3 + threadIdx.x] : 0.0f;
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, tg = lane & 3;
  const int row0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 16;
  if (row0 >= M) return;
  auto xval = [&](int r, int k) -> float {
    return (r < M && k < NI) ? X[(size_t)r * NI + k] : 0.0f;
  };
  auto bfrag = [&](const __nv_bfloat16* w, int ncols, int k0, int n0, unsigned& b0, unsigned& b1r) {
    // B[k][n] for k = k0 + 2 tg + {0,1} (b0) and + 8 (b1r), n = n0 + g
    __nv_bfloat162 lo, hi;
    lo.x = w[(k0 + 2 * tg) * ncols + n0 + g];
    lo.y = w[(k0 + 2 * tg + 1) * ncols + n0 + g];
    hi.x = w[(k0 + 2 * tg + 8) * ncols + n0 + g];
    hi.y = w[(k0 + 2 * tg + 9) * ncols + n0 + g];
    b0 = *reinterpret_cast<unsigned*>(&lo);
    b1r = *reinterpret_cast<unsigned*>(&hi);
  };
  // layer 1
  float acc[8][4];
  for (int nt = 0; nt < 8; ++nt) {
    float c0 = b1[nt * 8 + 2 * tg], c1 = b1[nt * 8 + 2 * tg + 1];
    acc[nt][0] = c0;
    acc[nt][1] = c1;
    acc[nt][2] = c0;
    acc[nt][3] = c1;
  }
  for (int kt = 0; kt < K1 / 16; ++kt) {
    unsigned a[4];
    int k = kt * 16 + 2 * tg;
    a[0] = pack_bf16(xval(row0 + g, k), xval(row0 + g, k + 1));
    a[1] = pack_bf16(xval(row0 + g + 8, k), xval(row0 + g + 8, k + 1));
    a[2] = pack_bf16(xval(row0 + g, k + 8), xval(row0 + g, k + 9));
    a[3] = pack_bf16(xval(row0 + g + 8, k + 8), xval(row0 + g + 8, k + 9));
    for (int nt = 0; nt < 8; ++nt) {
      unsigned bb0, bb1;
      bfrag(w1, NH, kt * 16, nt * 8, bb0, bb1);
      mma_bf16(acc[nt], a, bb0, bb1);
    }
  }
  // layer 2: A fragments from GELU(layer-1 accumulators)
  float acc2[8][4];
  for (int nt = 0; nt < 8; ++nt) {
    float c0 = b2[nt * 8 + 2 * tg], c1 = b2[nt * 8 + 2 * tg + 1];
    acc2[nt][0] = c0;
    acc2[nt][1] = c1;
    acc2[nt][2] = c0;
    acc2[nt][3] = c1;
  }
  for (int kt = 0; kt < NH / 16; ++kt) {
    unsigned a[4];
    a[0] = pack_bf16(gelu(acc[2 * kt][0]), gelu(acc[2 * kt][1]));
    a[1] = pack_bf16(gelu(acc[2 * kt][2]), gelu(acc[2 * kt][3]));
    a[2] = pack_bf16(gelu(acc[2 * kt + 1][0]), gelu(acc[2 * kt + 1][1]));
    a[3] = pack_bf16(gelu(acc[2 * kt + 1][2]), gelu(acc[2 * kt + 1][3]));
    for (int nt = 0; nt < 8; ++nt) {
      unsigned bb0, bb1;
      bfrag(w2, NH, kt * 16, nt * 8, bb0, bb1);
      mma_bf16(acc2[nt], a, bb0, bb1);
    }
  }
  // layer 3
  float acc3[4] = {b3[2 * tg], b3[2 * tg + 1], b3[2 * tg], b3[2 * tg + 1]};
  for (int kt = 0; kt < NH / 16; ++kt) {
    unsigned a[4];
    a[0] = pack_bf16(gelu(acc2[2 * kt][0]), gelu(acc2[2 * kt][1]));
    a[1] = pack_bf16(gelu(acc2[2 * kt][2]), gelu(acc2[2 * kt][3]));
    a[2] = pack_bf16(gelu(acc2[2 * kt + 1][0]), gelu(acc2[2 * kt + 1][1]));
    a[3] = pack_bf16(gelu(acc2[2 * kt + 1][2]), gelu(acc2[2 * kt + 1][3]));
    unsigned bb0, bb1;
    bfrag(w3, 8, kt * 16, 0, bb0, bb1);
    mma_bf16(acc3, a, bb0, bb1);
  }
  int c = 2 * tg;
  if (c < NO) {
    int r = row0 + g;
    if (r < M) {
      out[(size_t)r * NO + c] = acc3[0];
      out[(size_t)r * NO + c + 1] = acc3[1];
    }
    r = row0 + g + 8;
    if (r < M) {
      out[(size_t)r * NO + c] = acc3[2];
      out[(size_t)r * NO + c + 1] = acc3[3];
    }
  }
}

// SplitMix64 (Steele, Lea, Flood 2014) in counter form: interior point number
// k = (j-1) n + (i-1) of stream `seed` gets 2 u - 1, u = (z >> 11) 2^-53.
__global__ void k_uniform_pm1(int n, unsigned long long seed, double* __restrict__ x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
  if (i > n || j > n) return;
  unsigned long long k = (unsigned long long)(j - 1) * n + (i - 1);
  unsigned long long z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  double u = (double)(z >> 11) * 0x1.0p-53;
  x[(size_t)j * (n + 2) + i] = 2.0 * u - 1.0;
}

dim3 grid2(int nx, int ny) { return dim3((nx + 31) / 32, (ny + 7) / 8); }

}  // namespace

void launch_features(int n, const double* st, float* X, cudaStream_t s) {
  int nc = (n - 1) / 2;
  k_features<<<grid2(nc, nc), dim3(32, 8), 0, s>>>(n, st, X);
  count_launch();
}

void launch_mlp_infer(const float* X, int M, const float* par, float* out, cudaStream_t s) {
  int warps = (M + 15) / 16;
  k_mlp_infer<<<(warps + 3) / 4, 128, 0, s>>>(X, M, par, out);
  count_launch();
}

void launch_learned_ci(int n, const double* st, const float* delta, double* ci, double* aux, cudaStream_t s) {
  int nc = (n - 1) / 2;
  k_learned_edges<<<grid2(nc + 2, nc + 2), dim3(32, 8), 0, s>>>(n, st, delta, ci, aux);
  count_launch();
  k_learned_centres<<<grid2(nc + 2, nc + 2), dim3(32, 8), 0, s>>>(n, st, ci);
  count_launch();
}

void launch_uniform_pm1(int n, unsigned long long seed, double* x, cudaStream_t s) {
  k_uniform_pm1<<<grid2(n, n), dim3(32, 8), 0, s>>>(n, seed, x);
  count_launch();
}

// Test-vector energies E_k = ||v_k - P R v_k||_A^2 (and A err_k kept in Aes).
void launch_tv_energies(int n, const double* st, const double* ci, int K, const double* vecs, double* errs,
                        double* Aes, double* partials, double* energies, cudaStream_t s) {
  int nc = (n - 1) / 2;
  size_t ps = plane_size(n);
  int G = n < 1024 ? n : 1024;
  for (int k = 0; k < K; ++k) {
    k_tv_err<<<grid2(nc + 1, nc + 1), dim3(32, 8), 0, s>>>(n, ci, vecs + k * ps, errs + k * ps);
    k_tv_apply<<<G, 256, 0, s>>>(n, st, errs + k * ps, Aes + k * ps, partials);
    k_tv_energy<<<1, 32, 0, s>>>(partials, G, energies + k);
    count_launch();
    count_launch();
    count_launch();
  }
}

void launch_tv_grad(int n, const double* st, int K, const double* vecs, const double* Aes, const double* scale,
                    const double* aux, double* dW, double* tx, double* ty, float* ddelta, cudaStream_t s) {
  int nc = (n - 1) / 2;
  k_tv_dw<<<grid2(nc + 1, nc + 1), dim3(32, 8), 0, s>>>(n, K, vecs, Aes, scale, dW);
  k_tv_edge_t<<<grid2(nc + 2, nc + 2), dim3(32, 8), 0, s>>>(n, st, dW, aux, tx, ty);
  k_tv_ddelta<<<grid2(nc, nc), dim3(32, 8), 0, s>>>(n, tx, ty, ddelta);
  count_launch();
  count_launch();
  count_launch();
}

void launch_mlp_fwd(const float* X, int M, const float* par, float* Z1, float* Z2, float* out, cudaStream_t s) {
  k_mlp_fwd<<<(M + 127) / 128, 128, 0, s>>>(X, M, par, Z1, Z2, out);
  count_launch();
}

void launch_mlp_bwd(const float* X, int M, const float* par, const float* Z1, const float* Z2, const float* dout,
                    float* partial, float* grad, cudaStream_t s) {
  int nb = (M + BR - 1) / BR;
  k_mlp_bwd<<<nb, 256, 0, s>>>(X, M, par, Z1, Z2, dout, partial);
  k_sum_partials<<<(NPAR + 255) / 256, 256, 0, s>>>(partial, nb, grad);
  count_launch();
  count_launch();
}

void launch_adam(float* par, const float* grad, float* m, float* v, float lr, int step, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  k_adam<<<(NPAR + 255) / 256, 256, 0, s>>>(par, grad, m, v, lr, b1, b2, 1e-8f, c1, c2);
  count_launch();
}

int mlp_backward_blocks(int M) { return (M + BR - 1) / BR; }

}  // namespace bmg
