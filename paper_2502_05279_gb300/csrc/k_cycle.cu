// V-cycle kernels of the BoxMG solver (Fig. 1): Gauss-Seidel colour passes,
// fused residual + restriction (Fig. 2), interpolation + correction, residual
// norms with a fixed reduction order, the coarsest Cholesky solve and the
// FP64 iterative-refinement steps around an FP32 cycle.
//
// T is the compute type (double or float); S the storage type of the
// off-diagonal stencil planes (T, or bf16 under float).  Every row sum runs in
// the order O, W, E, S, N, SW, NE, NW, SE with one rounding per operation.
#include "common.cuh"
#include "kernels.h"

namespace bmg {

namespace {

constexpr int BX = 32, BY = 8;
constexpr int NORM_THREADS = 256;
constexpr int NORM_BLOCKS_MAX = 1024;

__device__ __forceinline__ bool stopped(const int* done) { return done != nullptr && *done != 0; }

// f - sum over the listed neighbours of a(p,q) x_q, starting from s.
template <typename T, typename S, bool NINE, bool WITH_O>
__device__ __forceinline__ T row_residual(const StencilView<T, S>& v, const T* __restrict__ x, size_t p, T s) {
  const int ld = v.ld;
  if (WITH_O) s = rsub(s, rmul(v.O[p], x[p]));
  s = rsub(s, rmul(cvt<T>(v.W[p]), x[p - 1]));
  s = rsub(s, rmul(cvt<T>(v.W[p + 1]), x[p + 1]));
  s = rsub(s, rmul(cvt<T>(v.S_[p]), x[p - ld]));
  s = rsub(s, rmul(cvt<T>(v.S_[p + ld]), x[p + ld]));
  if (NINE) {
    s = rsub(s, rmul(cvt<T>(v.SW[p]), x[p - ld - 1]));
    s = rsub(s, rmul(cvt<T>(v.SW[p + ld + 1]), x[p + ld + 1]));
    s = rsub(s, rmul(cvt<T>(v.NW[p]), x[p + ld - 1]));
    s = rsub(s, rmul(cvt<T>(v.NW[p + 1 - ld]), x[p + 1 - ld]));
  }
  return s;
}

// ---- Gauss-Seidel: one colour (i % 2 == pi, j % 2 == pj) per launch ----------
template <typename T, typename S, bool NINE>
__global__ void k_gs_colour(StencilView<T, S> v, const T* __restrict__ f, T* x, int pi, int pj, const int* done) {
  if (stopped(done)) return;
  int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + (pi ? 1 : 2);
  int j = 2 * (blockIdx.y * blockDim.y + threadIdx.y) + (pj ? 1 : 2);
  if (i > v.n || j > v.n) return;
  size_t p = (size_t)j * v.ld + i;
  T s = row_residual<T, S, NINE, false>(v, x, p, f[p]);
  T d = v.D ? v.D[p] : rdiv(T(1), v.O[p]);   // stored 1/a_pp, or the same quotient formed here
  x[p] = rmul(s, d);
}

// ---- residual + restriction ---------------------------------------------------
// A CTA owns a TXC x TYC tile of coarse points; it forms the residual on the
// (2 TXC + 1) x (2 TYC + 1) fine block under the tile in shared memory (each
// fine residual once, shared columns/rows recomputed at tile seams), then each
// thread applies the Fig. 2 restriction to one coarse point and zeroes the
// coarse iterate there.
constexpr int TXC = 32, TYC = 8;
constexpr int RFX = 2 * TXC + 1, RFY = 2 * TYC + 1;

template <typename T, typename S, bool NINE>
__global__ void __launch_bounds__(TXC* TYC) k_resid_restrict(StencilView<T, S> v, const T* __restrict__ ci,
                                                            const T* __restrict__ x, const T* __restrict__ f,
                                                            T* __restrict__ fc, T* __restrict__ xc,
                                                            const int* done) {
  if (stopped(done)) return;
  __shared__ T r[RFY][RFX + 1];
  const int n = v.n, ld = v.ld, nc = (n - 1) / 2, ldc = nc + 2;
  const int ic0 = blockIdx.x * TXC + 1, jc0 = blockIdx.y * TYC + 1;
  const int i0 = 2 * ic0 - 1, j0 = 2 * jc0 - 1;
  const int tid = threadIdx.y * TXC + threadIdx.x;
  for (int k = tid; k < RFX * RFY; k += TXC * TYC) {
    int li = k % RFX, lj = k / RFX;
    int i = i0 + li, j = j0 + lj;
    T val = T(0);
    if (i <= n && j <= n) {
      size_t p = (size_t)j * ld + i;
      val = row_residual<T, S, NINE, true>(v, x, p, f[p]);
    }
    r[lj][li] = val;
  }
  __syncthreads();
  int ic = ic0 + threadIdx.x, jc = jc0 + threadIdx.y;
  if (ic > nc || jc > nc) return;
  const size_t psc = plane_size(nc);
  const int li = 2 * threadIdx.x + 1, lj = 2 * threadIdx.y + 1;   // fine (2ic, 2jc) in the tile
  auto w = [&](int k, int dic, int djc) { return ci[k * psc + (size_t)(jc + djc) * ldc + (ic + dic)]; };
  T t = rmul(w(CI_LNE, 0, 0), r[lj - 1][li - 1]);
  t = radd(t, rmul(w(CI_LA, 0, 0), r[lj - 1][li]));
  t = radd(t, rmul(w(CI_LNW, 1, 0), r[lj - 1][li + 1]));
  t = radd(t, rmul(w(CI_LR, 0, 0), r[lj][li - 1]));
  t = radd(t, r[lj][li]);
  t = radd(t, rmul(w(CI_LL, 1, 0), r[lj][li + 1]));
  t = radd(t, rmul(w(CI_LSE, 0, 1), r[lj + 1][li - 1]));
  t = radd(t, rmul(w(CI_LB, 0, 1), r[lj + 1][li]));
  t = radd(t, rmul(w(CI_LSW, 1, 1), r[lj + 1][li + 1]));
  size_t pc = (size_t)jc * ldc + ic;
  fc[pc] = t;
  if (xc) xc[pc] = T(0);
}

// ---- interpolation + correction -------------------------------------------------
// One thread per coarse cell (ic, jc), 1..nc+1: its coincident, x-edge, y-edge
// and centre fine points.  x + (P e)_p, the interpolated value formed first.
template <typename T>
__global__ void k_interp_correct(int n, const T* __restrict__ ci, const T* __restrict__ ec, T* __restrict__ x,
                                 const int* done) {
  if (stopped(done)) return;
  int ic = blockIdx.x * blockDim.x + threadIdx.x + 1;
  int jc = blockIdx.y * blockDim.y + threadIdx.y + 1;
  int nc = (n - 1) / 2, ldc = nc + 2, ld = n + 2;
  if (ic > nc + 1 || jc > nc + 1) return;
  size_t psc = plane_size(nc), pc = (size_t)jc * ldc + ic;
  T e_sw = ec[pc - ldc - 1], e_se = ec[pc - ldc], e_nw = ec[pc - 1], e_ne = ec[pc];
  size_t pf = (size_t)(2 * jc) * ld + 2 * ic;   // coincident fine point
  if (ic <= nc && jc <= nc) x[pf] = radd(x[pf], e_ne);
  if (jc <= nc) {                                 // x-edge (2ic-1, 2jc)
    T t = rmul(ci[CI_LL * psc + pc], e_nw);
    t = radd(t, rmul(ci[CI_LR * psc + pc], e_ne));
    x[pf - 1] = radd(x[pf - 1], t);
  }
  if (ic <= nc) {                                 // y-edge (2ic, 2jc-1)
    T t = rmul(ci[CI_LB * psc + pc], e_se);
    t = radd(t, rmul(ci[CI_LA * psc + pc], e_ne));
    x[pf - ld] = radd(x[pf - ld], t);
  }
  {                                               // centre (2ic-1, 2jc-1)
    T t = rmul(ci[CI_LSW * psc + pc], e_sw);
    t = radd(t, rmul(ci[CI_LSE * psc + pc], e_se));
    t = radd(t, rmul(ci[CI_LNW * psc + pc], e_nw));
    t = radd(t, rmul(ci[CI_LNE * psc + pc], e_ne));
    x[pf - ld - 1] = radd(x[pf - ld - 1], t);
  }
}

// ---- residual with deterministic partial sums of r^2 -----------------------------
// Block b handles rows j = 1 + b, 1 + b + G, ... (G = gridDim.x); thread t the
// columns i = 1 + t, 1 + t + 256, ...; each thread sums in that order, then a
// fixed shared-memory tree.  The result depends only on n and G.
template <typename T>
__device__ __forceinline__ double block_sum(double acc) {
  __shared__ double red[NORM_THREADS];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = NORM_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + s];
    __syncthreads();
  }
  return red[0];
}

template <typename T, typename S, bool NINE>
__global__ void __launch_bounds__(NORM_THREADS) k_residual(StencilView<T, S> v, const T* __restrict__ x,
                                                           const T* __restrict__ f, T* __restrict__ r,
                                                           double* __restrict__ partials, const int* done) {
  if (stopped(done)) return;
  const int n = v.n, ld = v.ld;
  double acc = 0.0;
  for (int j = 1 + blockIdx.x; j <= n; j += gridDim.x)
    for (int i = 1 + threadIdx.x; i <= n; i += NORM_THREADS) {
      size_t p = (size_t)j * ld + i;
      T s = row_residual<T, S, NINE, true>(v, x, p, f[p]);
      if (r) r[p] = s;
      double d = (double)s;
      acc = __dadd_rn(acc, __dmul_rn(d, d));
    }
  if (partials) {
    double tot = block_sum<T>(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
  }
}

__global__ void k_zero_ring(int n, double* r) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  int ld = n + 2;
  if (k >= ld) return;
  r[k] = 0.0;
  r[(size_t)(n + 1) * ld + k] = 0.0;
  r[(size_t)k * ld] = 0.0;
  r[(size_t)k * ld + n + 1] = 0.0;
}

__device__ __forceinline__ double scale_of(double rho) {
  if (!(rho > 0.0) || !isfinite(rho)) return 1.0;
  int e;
  frexp(rho, &e);
  return ldexp(1.0, e);
}

// One block: sum the partials in index order per thread, fixed tree, sqrt.
__global__ void __launch_bounds__(NORM_THREADS) k_norm_finalize(const double* __restrict__ partials, int np,
                                                                Ctl* ctl, int phase, double* out) {
  if (phase == 1 && ctl && ctl->done) return;
  double acc = 0.0;
  for (int k = threadIdx.x; k < np; k += NORM_THREADS) acc = __dadd_rn(acc, partials[k]);
  double tot = block_sum<double>(acc);
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

// ---- coarsest solve: forward and back substitution (one thread) ---------------
template <typename T>
__global__ void k_coarse_solve(int n, const double* __restrict__ L, const T* __restrict__ f, T* __restrict__ x,
                               double* __restrict__ y, const int* done) {
  if (stopped(done)) return;
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int m = n * n, ld = n + 2;
  for (int i = 0; i < m; ++i) {
    double s = (double)f[(size_t)(i / n + 1) * ld + (i % n + 1)];
    for (int k = 0; k < i; ++k) s = rsub(s, rmul(L[(size_t)i * m + k], y[k]));
    y[i] = rdiv(s, L[(size_t)i * m + i]);
  }
  for (int i = m - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < m; ++k) s = rsub(s, rmul(L[(size_t)k * m + i], y[k]));
    y[i] = rdiv(s, L[(size_t)i * m + i]);
  }
  for (int i = 0; i < m; ++i) x[(size_t)(i / n + 1) * ld + (i % n + 1)] = (T)y[i];
}

// ---- iterative refinement ----------------------------------------------------------
__global__ void k_ir_update(int n, double* __restrict__ x, const float* __restrict__ e32, const Ctl* ctl) {
  if (ctl->done) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
  if (i > n || j > n) return;
  size_t p = (size_t)j * (n + 2) + i;
  x[p] = radd(x[p], rmul(ctl->scale_applied, (double)e32[p]));
}

__global__ void __launch_bounds__(NORM_THREADS) k_ir_residual(StencilView<double, double> v, int nine,
                                                              const double* __restrict__ x,
                                                              const double* __restrict__ f, float* __restrict__ r32,
                                                              float* __restrict__ e32, double* __restrict__ partials,
                                                              Ctl* ctl) {
  if (ctl->done) return;
  const int n = v.n, ld = v.ld;
  const double s = ctl->scale_next;
  const double inv = 1.0 / s;   // exact: s is a power of two
  double acc = 0.0;
  for (int j = 1 + blockIdx.x; j <= n; j += gridDim.x)
    for (int i = 1 + threadIdx.x; i <= n; i += NORM_THREADS) {
      size_t p = (size_t)j * ld + i;
      double rr = nine ? row_residual<double, double, true, true>(v, x, p, f[p])
                       : row_residual<double, double, false, true>(v, x, p, f[p]);
      r32[p] = __double2float_rn(rmul(rr, inv));
      e32[p] = 0.0f;
      acc = __dadd_rn(acc, __dmul_rn(rr, rr));
    }
  double tot = block_sum<double>(acc);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = tot;
    if (blockIdx.x == 0) ctl->scale_applied = s;
  }
}

// ---- FP64 throughput probe ---------------------------------------------------------
__global__ void k_dp_probe(double* out, int iters, double a, double b) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  double x0 = t * 1e-9, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int k = 0; k < iters; ++k) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[t] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

dim3 grid2(int nx, int ny) { return dim3((nx + BX - 1) / BX, (ny + BY - 1) / BY); }

int norm_blocks(int n) { return n < NORM_BLOCKS_MAX ? n : NORM_BLOCKS_MAX; }

}  // namespace

int norm_partials_max() { return NORM_BLOCKS_MAX; }

template <typename T, typename S>
void launch_gs(const StencilView<T, S>& v, int kind, const T* f, T* x, int sweeps, const int* done, cudaStream_t s) {
  const int n = v.n;
  auto pass = [&](int pi, int pj) {
    int ni = pi ? (n + 1) / 2 : (n - 1) / 2, nj = pj ? (n + 1) / 2 : (n - 1) / 2;
    if (kind == 9)
      k_gs_colour<T, S, true><<<grid2(ni, nj), dim3(BX, BY), 0, s>>>(v, f, x, pi, pj, done);
    else
      k_gs_colour<T, S, false><<<grid2(ni, nj), dim3(BX, BY), 0, s>>>(v, f, x, pi, pj, done);
    count_launch();
  };
  for (int k = 0; k < sweeps; ++k) {
    if (kind == 9) {
      pass(1, 1); pass(0, 1); pass(1, 0); pass(0, 0);
    } else {
      pass(1, 1); pass(0, 0); pass(0, 1); pass(1, 0);
    }
  }
}

template <typename T, typename S>
void launch_resid_restrict(const StencilView<T, S>& v, int kind, const T* ci, const T* x, const T* f, T* fc, T* xc,
                           const int* done, cudaStream_t s) {
  int nc = (v.n - 1) / 2;
  dim3 g((nc + TXC - 1) / TXC, (nc + TYC - 1) / TYC);
  if (kind == 9)
    k_resid_restrict<T, S, true><<<g, dim3(TXC, TYC), 0, s>>>(v, ci, x, f, fc, xc, done);
  else
    k_resid_restrict<T, S, false><<<g, dim3(TXC, TYC), 0, s>>>(v, ci, x, f, fc, xc, done);
  count_launch();
}

template <typename T>
void launch_interp_correct(int n, const T* ci, const T* ec, T* x, const int* done, cudaStream_t s) {
  int nc = (n - 1) / 2;
  k_interp_correct<T><<<grid2(nc + 1, nc + 1), dim3(BX, BY), 0, s>>>(n, ci, ec, x, done);
  count_launch();
}

template <typename T, typename S>
int launch_residual(const StencilView<T, S>& v, int kind, const T* x, const T* f, T* r, double* partials,
                    const int* done, cudaStream_t s) {
  int g = norm_blocks(v.n);
  if (kind == 9)
    k_residual<T, S, true><<<g, NORM_THREADS, 0, s>>>(v, x, f, r, partials, done);
  else
    k_residual<T, S, false><<<g, NORM_THREADS, 0, s>>>(v, x, f, r, partials, done);
  count_launch();
  return g;
}

template <typename T>
void launch_coarse_solve(int n, const double* L, const T* f, T* x, double* y, const int* done, cudaStream_t s) {
  k_coarse_solve<T><<<1, 1, 0, s>>>(n, L, f, x, y, done);
  count_launch();
}

void launch_norm_finalize(const double* partials, int np, void* ctl, int phase, double* out, cudaStream_t s) {
  k_norm_finalize<<<1, NORM_THREADS, 0, s>>>(partials, np, (Ctl*)ctl, phase, out);
  count_launch();
}

void launch_ir_update(int n, double* x, const float* e32, void* ctl, cudaStream_t s) {
  k_ir_update<<<grid2(n, n), dim3(BX, BY), 0, s>>>(n, x, e32, (const Ctl*)ctl);
  count_launch();
}

int launch_ir_residual(const StencilView<double, double>& v, int kind, const double* x, const double* f, float* r32,
                       float* e32_zero, double* partials, void* ctl, cudaStream_t s) {
  int g = norm_blocks(v.n);
  k_ir_residual<<<g, NORM_THREADS, 0, s>>>(v, kind == 9, x, f, r32, e32_zero, partials, (Ctl*)ctl);
  count_launch();
  return g;
}

void zero_ring(int n, double* r, cudaStream_t s) {
  k_zero_ring<<<(n + 2 + 255) / 256, 256, 0, s>>>(n, r);
  count_launch();
}

double measure_fp64_rate(cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int blocks = sms * 8, threads = 256, iters = 4000;
  double* out = nullptr;
  if (cudaMallocAsync(&out, sizeof(double) * blocks * threads, s) != cudaSuccess) return -1.0;
  k_dp_probe<<<blocks, threads, 0, s>>>(out, 10, 0.999, 1e-3);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  k_dp_probe<<<blocks, threads, 0, s>>>(out, iters, 0.999, 1e-3);
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, s);
  cudaStreamSynchronize(s);
  return (double)blocks * threads * iters * 8.0 / (ms * 1e-3) / 1e9;
}

// ---- explicit instantiations ---------------------------------------------------------
#define BMG_INST(T, S)                                                                                           \
  template void launch_gs<T, S>(const StencilView<T, S>&, int, const T*, T*, int, const int*, cudaStream_t);    \
  template void launch_resid_restrict<T, S>(const StencilView<T, S>&, int, const T*, const T*, const T*, T*, T*, \
                                            const int*, cudaStream_t);                                          \
  template int launch_residual<T, S>(const StencilView<T, S>&, int, const T*, const T*, T*, double*, const int*, \
                                     cudaStream_t);
BMG_INST(double, double)
BMG_INST(float, float)
BMG_INST(float, __nv_bfloat16)
#undef BMG_INST
template void launch_interp_correct<double>(int, const double*, const double*, double*, const int*, cudaStream_t);
template void launch_interp_correct<float>(int, const float*, const float*, float*, const int*, cudaStream_t);
template void launch_coarse_solve<double>(int, const double*, const double*, double*, double*, const int*,
                                          cudaStream_t);
template void launch_coarse_solve<float>(int, const double*, const float*, float*, double*, const int*,
                                         cudaStream_t);

}  // namespace bmg

// ==== flexible conjugate gradients ======================================================
// Notay's FCG(1) with the V-cycle as preconditioner, FP64 outer loop:
//   z = M r; p = z (first step) or z + beta p with beta = -(z.q)/(p.q)_previous;
//   q = A p; alpha = (p.r)/(p.q); x += alpha p; r -= alpha q.
// Every inner product uses the reduction order of k_residual / k_norm_finalize.
namespace bmg {
namespace {

__device__ __forceinline__ double zval(const double* z, const float* z32, double s, size_t p) {
  return z32 ? rmul(s, (double)z32[p]) : z[p];   // s * fl64(z32) is exact: s is a power of two
}

// p.q over the grid with the canonical order; f(p) gives the product term.
template <class F>
__device__ __forceinline__ void ordered_partial(int n, int ld, double* partials, F term) {
  double acc = 0.0;
  for (int j = 1 + blockIdx.x; j <= n; j += gridDim.x)
    for (int i = 1 + threadIdx.x; i <= n; i += NORM_THREADS) acc = __dadd_rn(acc, term((size_t)j * ld + i));
  double tot = block_sum<double>(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(NORM_THREADS) k_fcg_zq(int n, const double* __restrict__ z,
                                                         const float* __restrict__ z32, const double* __restrict__ q,
                                                         double* __restrict__ partials, const Ctl* ctl) {
  if (ctl->done) return;
  const double s = ctl->scale_applied;
  ordered_partial(n, n + 2, partials, [&](size_t p) { return rmul(zval(z, z32, s, p), q[p]); });
}

__device__ __forceinline__ double reduce_partials(const double* partials, int np) {
  double acc = 0.0;
  for (int k = threadIdx.x; k < np; k += NORM_THREADS) acc = __dadd_rn(acc, partials[k]);
  return block_sum<double>(acc);
}

// slot 0: zq; slot 1: pq and pr (second partial array right after the first)
__global__ void __launch_bounds__(NORM_THREADS) k_fcg_reduce(const double* __restrict__ partials, int np, Ctl* ctl,
                                                             int which) {
  if (ctl->done) return;
  if (which == 0) {
    double v = reduce_partials(partials, np);
    if (threadIdx.x == 0) ctl->zq = v;
  } else {
    double a = reduce_partials(partials, np);
    __syncthreads();
    double b = reduce_partials(partials + NORM_BLOCKS_MAX, np);
    if (threadIdx.x == 0) {
      ctl->pq = a;
      ctl->pr = b;
    }
  }
}

__global__ void k_fcg_direction(int n, const double* __restrict__ z, const float* __restrict__ z32,
                                double* __restrict__ pv, const Ctl* ctl) {
  if (ctl->done) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
  if (i > n || j > n) return;
  size_t p = (size_t)j * (n + 2) + i;
  double zp = zval(z, z32, ctl->scale_applied, p);
  if (ctl->first) {
    pv[p] = zp;
  } else {
    double beta = -rdiv(ctl->zq, ctl->pq_prev);
    pv[p] = radd(zp, rmul(beta, pv[p]));
  }
}

// q = A p (row sum a_O p + a_W p_W + ... in canonical order), partial p.q and p.r
__global__ void __launch_bounds__(NORM_THREADS) k_fcg_matvec(StencilView<double, double> v, int nine,
                                                             const double* __restrict__ pv, const double* __restrict__ r,
                                                             double* __restrict__ q, double* __restrict__ partials,
                                                             const Ctl* ctl) {
  if (ctl->done) return;
  const int n = v.n, ld = v.ld;
  double apq = 0.0, apr = 0.0;
  for (int j = 1 + blockIdx.x; j <= n; j += gridDim.x)
    for (int i = 1 + threadIdx.x; i <= n; i += NORM_THREADS) {
      size_t p = (size_t)j * ld + i;
      double acc = rmul(v.O[p], pv[p]);
      acc = radd(acc, rmul(v.W[p], pv[p - 1]));
      acc = radd(acc, rmul(v.W[p + 1], pv[p + 1]));
      acc = radd(acc, rmul(v.S_[p], pv[p - ld]));
      acc = radd(acc, rmul(v.S_[p + ld], pv[p + ld]));
      if (nine) {
        acc = radd(acc, rmul(v.SW[p], pv[p - ld - 1]));
        acc = radd(acc, rmul(v.SW[p + ld + 1], pv[p + ld + 1]));
        acc = radd(acc, rmul(v.NW[p], pv[p + ld - 1]));
        acc = radd(acc, rmul(v.NW[p + 1 - ld], pv[p + 1 - ld]));
      }
      q[p] = acc;
      apq = __dadd_rn(apq, rmul(pv[p], acc));
      apr = __dadd_rn(apr, rmul(pv[p], r[p]));
    }
  double t1 = block_sum<double>(apq);
  __syncthreads();
  double t2 = block_sum<double>(apr);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = t1;
    partials[NORM_BLOCKS_MAX + blockIdx.x] = t2;
  }
}

// x += alpha p, r -= alpha q, partial r.r; zero the preconditioner output and,
// in mixed precision, write r32 = fl32(r / scale_next).
__global__ void __launch_bounds__(NORM_THREADS) k_fcg_update(int n, double* __restrict__ x, double* __restrict__ r,
                                                             const double* __restrict__ pv,
                                                             const double* __restrict__ q, float* __restrict__ r32,
                                                             float* __restrict__ z32, double* __restrict__ z,
                                                             double* __restrict__ partials, Ctl* ctl) {
  if (ctl->done) return;
  const int ld = n + 2;
  const double alpha = rdiv(ctl->pr, ctl->pq);
  const double s = ctl->scale_next;
  const double inv = 1.0 / s;
  double acc = 0.0;
  for (int j = 1 + blockIdx.x; j <= n; j += gridDim.x)
    for (int i = 1 + threadIdx.x; i <= n; i += NORM_THREADS) {
      size_t p = (size_t)j * ld + i;
      x[p] = radd(x[p], rmul(alpha, pv[p]));
      double rr = rsub(r[p], rmul(alpha, q[p]));
      r[p] = rr;
      if (r32) {
        r32[p] = __double2float_rn(rmul(rr, inv));
        z32[p] = 0.0f;
      } else {
        z[p] = 0.0;
      }
      acc = __dadd_rn(acc, rmul(rr, rr));
    }
  double tot = block_sum<double>(acc);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = tot;
    if (blockIdx.x == 0) {
      ctl->scale_applied = s;
      ctl->pq_prev = ctl->pq;
      ctl->first = 0;
    }
  }
}

// r = f - A x, stored; r32 / zero z as in k_fcg_update; partial r.r.
__global__ void __launch_bounds__(NORM_THREADS) k_fcg_init(StencilView<double, double> v, int nine,
                                                           const double* __restrict__ x, const double* __restrict__ f,
                                                           double* __restrict__ r, double* __restrict__ z,
                                                           float* __restrict__ r32, float* __restrict__ z32,
                                                           double* __restrict__ partials, Ctl* ctl) {
  const int n = v.n, ld = v.ld;
  const double s = ctl->scale_next;
  const double inv = 1.0 / s;
  double acc = 0.0;
  for (int j = 1 + blockIdx.x; j <= n; j += gridDim.x)
    for (int i = 1 + threadIdx.x; i <= n; i += NORM_THREADS) {
      size_t p = (size_t)j * ld + i;
      double rr = nine ? row_residual<double, double, true, true>(v, x, p, f[p])
                       : row_residual<double, double, false, true>(v, x, p, f[p]);
      r[p] = rr;
      if (r32) {
        r32[p] = __double2float_rn(rmul(rr, inv));
        z32[p] = 0.0f;
      } else {
        z[p] = 0.0;
      }
      acc = __dadd_rn(acc, rmul(rr, rr));
    }
  double tot = block_sum<double>(acc);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = tot;
    if (blockIdx.x == 0) {
      ctl->scale_applied = s;
      ctl->first = 1;
    }
  }
}

}  // namespace

int launch_fcg_init(const StencilView<double, double>& v, int kind, const double* x, const double* f, double* r,
                    double* z, float* r32, float* z32, double* partials, void* ctl, cudaStream_t s) {
  int g = norm_blocks(v.n);
  k_fcg_init<<<g, NORM_THREADS, 0, s>>>(v, kind == 9, x, f, r, z, r32, z32, partials, (Ctl*)ctl);
  count_launch();
  return g;
}

// One FCG step after the preconditioner: z.q, beta and p, q = A p with p.q and
// p.r, then the x / r update with r.r partials (finalised by the caller).
// `mark(arg, k)` (may be NULL) brackets the sub-steps for profiling.
void launch_fcg_step(const StencilView<double, double>& v, int kind, double* x, double* r, const double* z,
                     const float* z32, double* pv, double* q, float* r32, float* z32_zero, double* z_zero,
                     double* partials, void* ctl, cudaStream_t s, void (*mark)(void*, int), void* mark_arg) {
  const int n = v.n;
  int g = norm_blocks(n);
  Ctl* c = (Ctl*)ctl;
  if (mark) mark(mark_arg, 0);
  k_fcg_zq<<<g, NORM_THREADS, 0, s>>>(n, z, z32, q, partials, c);
  count_launch();
  k_fcg_reduce<<<1, NORM_THREADS, 0, s>>>(partials, g, c, 0);
  count_launch();
  k_fcg_direction<<<grid2(n, n), dim3(BX, BY), 0, s>>>(n, z, z32, pv, c);
  count_launch();
  if (mark) mark(mark_arg, 1);
  k_fcg_matvec<<<g, NORM_THREADS, 0, s>>>(v, kind == 9, pv, r, q, partials, c);
  count_launch();
  k_fcg_reduce<<<1, NORM_THREADS, 0, s>>>(partials, g, c, 1);
  count_launch();
  if (mark) mark(mark_arg, 2);
  k_fcg_update<<<g, NORM_THREADS, 0, s>>>(n, x, r, pv, q, r32, z32_zero, z_zero, partials, c);
  count_launch();
  if (mark) mark(mark_arg, 3);
}

}  // namespace bmg
