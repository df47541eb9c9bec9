// V-cycle kernels of the BoxMG solver (Fig. 1), single problem: Gauss-Seidel
// half sweeps, fused residual + restriction (Fig. 2), interpolation +
// correction, residual norms with a fixed reduction order, the coarsest
// Cholesky solve, FP64 iterative-refinement steps around an FP32 cycle and the
// flexible-CG outer loop.  The arithmetic lives in cycle_device.cuh, shared with
// the batched kernels.
#include <cstdint>

#include "cycle_device.cuh"

namespace bmg {

using namespace dev;

namespace {

constexpr int BX = 32, BY = 8;

// FU (every kernel of the cycle): fused multiply-adds (the hierarchy's
// arithmetic mode BMG_ARITH_FUSED) instead of rounded products and sums.
template <typename T, typename S, int CL, bool FU>
__global__ void __launch_bounds__(rows_threads_max<T>(), sizeof(T) == 8 ? 2 : 1)
    k_gs_rows(StencilView<T, S> v, const T* __restrict__ f, T* x, int pj, const int* done) {
  pdl_enter();
  if (stopped(done)) return;   // uniform over the grid: every CTA of a cluster leaves together
  gs_rows_body<T, S, CL, FU>(v, f, x, pj, blockIdx.x);
}

template <typename T, typename S, bool FU>
__global__ void k_gs_checker(StencilView<T, S> v, const T* __restrict__ f, T* x, int c, const int* done) {
  pdl_enter();
  if (stopped(done)) return;
  gs_checker_body<T, S, FU>(v, f, x, c, blockIdx.x, blockIdx.y);
}

// One warp per strip of 56 x TY points; warp g of the grid takes strip
// (g % nbx, g / nbx), so the warps of a CTA take neighbouring strips of one band.
constexpr int STRIP_WARPS = 4;
template <typename S, int TY, bool FU>
__global__ void __launch_bounds__(32 * STRIP_WARPS) k_gs_strip(StencilView<float, S> v, const float* __restrict__ f,
                                                               const float* __restrict__ xin,
                                                               float* __restrict__ xout, const int* done) {
  pdl_enter();
  if (stopped(done)) return;
  const int nbx = (v.n + 55) / 56, nby = (v.n + TY - 1) / TY;
  const int g = blockIdx.x * STRIP_WARPS + (threadIdx.x >> 5);
  if (g >= nbx * nby) return;                     // whole warps only
  gs_strip_body<S, TY, FU>(v, f, xin, xout, g % nbx, g / nbx);
}

// Bulk-copy form: warp w of the CTA owns ring slots [w RING, (w + 1) RING) and
// mbarriers [w RING, (w + 1) RING) of the dynamic shared memory.
__device__ int g_strip_timeout = 0;
template <typename S, int RING, bool FU>
__global__ void __launch_bounds__(32 * STRIP_WARPS) k_gs_strip_ring(StencilView<float, S> v,
                                                                    const float* __restrict__ f,
                                                                    const float* __restrict__ xin,
                                                                    float* __restrict__ xout, const int* done,
                                                                    int ty) {
  pdl_enter();
  extern __shared__ __align__(128) unsigned char strip_smem[];
  if (stopped(done)) return;
  const int nbx = (v.n + 55) / 56, nby = (v.n + ty - 1) / ty;
  const int w = threadIdx.x >> 5, g = blockIdx.x * STRIP_WARPS + w;
  if (g >= nbx * nby) return;                     // whole warps only
  unsigned char* ring = strip_smem + (size_t)w * RING * StripRing<S>::SLOT;
  unsigned long long* bars =
      reinterpret_cast<unsigned long long*>(strip_smem + (size_t)STRIP_WARPS * RING * StripRing<S>::SLOT) + w * RING;
  if (!gs_strip_ring_body<S, RING, FU>(v, f, xin, xout, g % nbx, g / nbx, ty, ring, bars) && (threadIdx.x & 31) == 0)
    atomicExch(&g_strip_timeout, 1);
}

// Two sweeps in one pass: warps take 48-column strips, otherwise as above.
template <typename S, int RING, bool FU>
__global__ void __launch_bounds__(32 * STRIP_WARPS) k_gs_strip2_ring(StencilView<float, S> v,
                                                                     const float* __restrict__ f,
                                                                     const float* __restrict__ xin,
                                                                     float* __restrict__ xout, const int* done,
                                                                     int ty) {
  pdl_enter();
  extern __shared__ __align__(128) unsigned char strip_smem[];
  if (stopped(done)) return;
  const int nbx = (v.n + 47) / 48, nby = (v.n + ty - 1) / ty;
  const int w = threadIdx.x >> 5, g = blockIdx.x * STRIP_WARPS + w;
  if (g >= nbx * nby) return;
  unsigned char* ring = strip_smem + (size_t)w * RING * StripRing<S>::SLOT;
  unsigned long long* bars =
      reinterpret_cast<unsigned long long*>(strip_smem + (size_t)STRIP_WARPS * RING * StripRing<S>::SLOT) + w * RING;
  if (!gs_strip2_ring_body<S, RING, FU>(v, f, xin, xout, g % nbx, g / nbx, ty, ring, bars) &&
      (threadIdx.x & 31) == 0)
    atomicExch(&g_strip_timeout, 1);
}

// Two sweeps, residual and restriction in one pass: warps take 44-column
// strips; the coarse right-hand side and iterate of the next level are written
// at the strip's coarse points.
template <typename S, int RING, bool FU>
__global__ void __launch_bounds__(32 * STRIP_WARPS) k_gs_strip2r_ring(StencilView<float, S> v,
                                                                      const float* __restrict__ f,
                                                                      const float* __restrict__ xin,
                                                                      float* __restrict__ xout,
                                                                      const float* __restrict__ ci,
                                                                      float* __restrict__ fc, float* __restrict__ xc,
                                                                      const int* done, int ty) {
  pdl_enter();
  extern __shared__ __align__(128) unsigned char strip_smem[];
  if (stopped(done)) return;
  const int nbx = (v.n + 43) / 44, nby = (v.n + ty - 1) / ty;
  const int w = threadIdx.x >> 5, g = blockIdx.x * STRIP_WARPS + w;
  if (g >= nbx * nby) return;
  unsigned char* ring = strip_smem + (size_t)w * RING * StripRingR<S>::SLOT;
  unsigned long long* bars =
      reinterpret_cast<unsigned long long*>(strip_smem + (size_t)STRIP_WARPS * RING * StripRingR<S>::SLOT) + w * RING;
  if (!gs_strip2r_ring_body<S, RING, FU>(v, f, xin, xout, ci, fc, xc, g % nbx, g / nbx, ty, ring, bars) &&
      (threadIdx.x & 31) == 0)
    atomicExch(&g_strip_timeout, 1);
}

// FP64 one-pass sweep with strips of 56 x ty points: warp w of the CTA owns
// ring slots [w RING, (w + 1) RING).
template <int RING, bool FU>
__global__ void __launch_bounds__(32 * STRIP_WARPS) k_gs_strip64(StencilView<double, double> v,
                                                                 const double* __restrict__ f,
                                                                 const double* __restrict__ xin,
                                                                 double* __restrict__ xout, const int* done, int ty) {
  pdl_enter();
  extern __shared__ __align__(128) unsigned char strip_smem[];
  if (stopped(done)) return;
  const int nbx = (v.n + 55) / 56, nby = (v.n + ty - 1) / ty;
  const int w = threadIdx.x >> 5, g = blockIdx.x * STRIP_WARPS + w;
  if (g >= nbx * nby) return;                     // whole warps only
  gs_strip64_body<RING, FU>(v, f, xin, xout, g % nbx, g / nbx, ty, strip_smem + (size_t)w * RING * STRIP64_SLOT);
}

// Zebra x-lines: one thread per row of the parity (first row 1 or 2).
template <typename T, typename S, bool NINE>
__global__ void k_line_rows(StencilView<T, S> v, const T* __restrict__ f, T* x, T* __restrict__ cp, int first,
                            const int* done) {
  pdl_enter();
  if (stopped(done)) return;
  const int j = first + 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (j > v.n) return;
  line_row_body<T, S, NINE>(v, f, x, cp, j);
}

// Zebra y-lines: one thread per column of the parity (first column 1 or 2).
template <typename T, typename S, bool NINE>
__global__ void k_line_cols(StencilView<T, S> v, const T* __restrict__ f, T* x, T* __restrict__ cp, int first,
                            const int* done) {
  pdl_enter();
  if (stopped(done)) return;
  const int i = first + 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (i > v.n) return;
  line_col_body<T, S, NINE>(v, f, x, cp, i);
}

template <typename T, typename S, bool NINE, bool FU>
__global__ void __launch_bounds__(TXC* TYC) k_resid_restrict(StencilView<T, S> v, const T* __restrict__ ci,
                                                            const T* __restrict__ x, const T* __restrict__ f,
                                                            T* __restrict__ fc, T* __restrict__ xc,
                                                            const int* done) {
  pdl_enter();
  if (stopped(done)) return;
  resid_restrict_body<T, S, NINE, FU>(v, ci, x, f, fc, xc, blockIdx.x, blockIdx.y);
}

template <typename T, bool FU>
__global__ void k_interp_correct(int n, const T* __restrict__ ci, const T* __restrict__ ec, const T* xin, T* xout,
                                 const int* done) {
  pdl_enter();
  if (stopped(done)) return;
  interp_body<T, FU>(n, ci, ec, xin, xout, blockIdx.x * blockDim.x + threadIdx.x + 1,
                 blockIdx.y * blockDim.y + threadIdx.y + 1);
}

template <typename T, typename S, bool NINE, bool FU>
__global__ void __launch_bounds__(NORM_THREADS) k_residual(StencilView<T, S> v, const T* __restrict__ x,
                                                           const T* __restrict__ f, T* __restrict__ r,
                                                           double* __restrict__ partials, const int* done) {
  pdl_enter();
  if (stopped(done)) return;
  residual_body<T, S, NINE, FU>(v, x, f, r, partials, blockIdx.x, gridDim.x);
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

__global__ void __launch_bounds__(NORM_THREADS) k_norm_finalize(const double* __restrict__ partials, int np,
                                                                Ctl* ctl, int phase, double* out) {
  pdl_enter();
  finalize_body(partials, np, ctl, phase, out);
}

template <typename T>
__global__ void k_coarse_solve(int n, const double* __restrict__ L, const T* __restrict__ f, T* __restrict__ x,
                               double* __restrict__ y, const int* done) {
  pdl_enter();
  if (stopped(done)) return;
  if (blockIdx.x != 0) return;
  coarse_solve_body<T>(n, L, f, x, y);
}

// x += scale_applied * e32, IRU_COLS points of a row per thread, BX apart.
__global__ void k_ir_update(int n, double* __restrict__ x, const float* __restrict__ e32, const Ctl* ctl) {
  pdl_enter();
  if (ctl->done) return;
  ir_update_cols(n, x, e32, ctl->scale_applied, blockIdx.x * (BX * IRU_COLS) + threadIdx.x + 1,
                 blockIdx.y * blockDim.y + threadIdx.y + 1, BX);
}

template <bool FU>
__global__ void __launch_bounds__(NORM_THREADS) k_ir_residual(StencilView<double, double> v, int nine,
                                                              const double* __restrict__ x,
                                                              const double* __restrict__ f, float* __restrict__ r32,
                                                              float* __restrict__ e32, double* __restrict__ partials,
                                                              Ctl* ctl) {
  pdl_enter();
  if (ctl->done) return;
  ir_residual_body<FU>(v, nine != 0, x, f, r32, e32, partials, ctl, blockIdx.x, gridDim.x);
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

}  // namespace

int norm_partials_max() { return NORM_BLOCKS_MAX; }

// Cluster launch of k_gs_rows: grid = rows * CL CTAs, clusters of CL along x, so
// cluster rank = blockIdx.x % CL and the CTAs of one row form one cluster.
template <typename T, typename S, int CL, bool FU>
void launch_rows_half(const StencilView<T, S>& v, const T* f, T* x, int pj, int rows, int threads, const int* done,
                      cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(rows * CL));
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = CL;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = CL > 1 ? 2 : 1;
  cudaLaunchKernelEx(&cfg, k_gs_rows<T, S, CL, FU>, v, f, x, pj, done);
  count_launch();
}

// Smallest cluster size (1, 2, 4, 8) whose CTAs cover the (n+1)/2 pairs of a row.
template <typename T>
int rows_cluster(int n) {
  const int pairs = (n + 1) / 2;
  int cl = 1;
  while (cl * rows_threads_max<T>() < pairs) cl *= 2;
  return cl;
}

int rows_threads(int n, int cl) {
  int threads = ((n + 1) / 2 + cl - 1) / cl;
  return (threads + 31) / 32 * 32;
}

template <typename T, typename S, bool FU>
static void gs_sweeps(const StencilView<T, S>& v, int kind, const T* f, T* x, int sweeps, const int* done,
                      cudaStream_t s, int cl_req) {
  const int n = v.n;
  if (kind == 9) {
    const int cl = cl_req >= rows_cluster<T>(n) && cl_req <= 8 ? cl_req : rows_cluster<T>(n);
    const int threads = rows_threads(n, cl);
    for (int k = 0; k < sweeps; ++k)
      for (int pj = 1; pj >= 0; --pj) {
        const int rows = pj ? (n + 1) / 2 : (n - 1) / 2;
        switch (cl) {
          case 1: launch_rows_half<T, S, 1, FU>(v, f, x, pj, rows, threads, done, s); break;
          case 2: launch_rows_half<T, S, 2, FU>(v, f, x, pj, rows, threads, done, s); break;
          case 4: launch_rows_half<T, S, 4, FU>(v, f, x, pj, rows, threads, done, s); break;
          default: launch_rows_half<T, S, 8, FU>(v, f, x, pj, rows, threads, done, s); break;
        }
      }
  } else {
    dim3 g(((n + 1) / 2 + BX - 1) / BX, (n + BY - 1) / BY);
    for (int k = 0; k < sweeps; ++k) {
      pdl_launch(k_gs_checker<T, S, FU>, g, dim3(BX, BY), 0, s, v, f, x, 0, done);
      count_launch();
      pdl_launch(k_gs_checker<T, S, FU>, g, dim3(BX, BY), 0, s, v, f, x, 1, done);
      count_launch();
    }
  }
}

template <typename T, typename S>
void launch_gs(const StencilView<T, S>& v, int kind, const T* f, T* x, int sweeps, const int* done, cudaStream_t s,
               int cl_req) {
  if (v.fused)
    gs_sweeps<T, S, true>(v, kind, f, x, sweeps, done, s, cl_req);
  else
    gs_sweeps<T, S, false>(v, kind, f, x, sweeps, done, s, cl_req);
}

template <typename T, typename S>
void launch_resid_restrict(const StencilView<T, S>& v, int kind, const T* ci, const T* x, const T* f, T* fc, T* xc,
                           const int* done, cudaStream_t s) {
  int nc = (v.n - 1) / 2;
  dim3 g((nc + TXC - 1) / TXC, (nc + TYC - 1) / TYC);
  const dim3 b(TXC, TYC);
  if (kind == 9 && v.fused)
    pdl_launch(k_resid_restrict<T, S, true, true>, g, b, 0, s, v, ci, x, f, fc, xc, done);
  else if (kind == 9)
    pdl_launch(k_resid_restrict<T, S, true, false>, g, b, 0, s, v, ci, x, f, fc, xc, done);
  else if (v.fused)
    pdl_launch(k_resid_restrict<T, S, false, true>, g, b, 0, s, v, ci, x, f, fc, xc, done);
  else
    pdl_launch(k_resid_restrict<T, S, false, false>, g, b, 0, s, v, ci, x, f, fc, xc, done);
  count_launch();
}

template <typename S, int TY, bool FU>
static void strip_launch(const StencilView<float, S>& v, const float* f, const float* xin, float* xout,
                         const int* done, cudaStream_t s) {
  const int warps = ((v.n + 55) / 56) * ((v.n + TY - 1) / TY);
  pdl_launch(k_gs_strip<S, TY, FU>, (warps + STRIP_WARPS - 1) / STRIP_WARPS, 32 * STRIP_WARPS, 0, s, v, f, xin,
             xout, done);
  count_launch();
}

// Raise a kernel's dynamic shared-memory limit to `bytes` and return how many
// warps of it (CTAs of STRIP_WARPS warps) fit on the device at once.  Callers
// keep the result in a function-local static, whose initialisation C++ makes
// thread-safe.
template <typename K>
static int resident_strip_warps(K kernel, size_t bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * STRIP_WARPS, bytes);
  return (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1) * STRIP_WARPS;
}

// ty = 0: the smallest even strip height whose strips fit into one wave of
// the kernel's resident warps.
template <typename S, int RING, bool FU>
static void strip_ring_launch(const StencilView<float, S>& v, const float* f, const float* xin, float* xout,
                              const int* done, cudaStream_t s, int ty) {
  constexpr size_t bytes = (size_t)STRIP_WARPS * RING * (StripRing<S>::SLOT + 8);
  static const int resident_warps = resident_strip_warps(k_gs_strip_ring<S, RING, FU>, bytes);
  const int nbx = (v.n + 55) / 56;
  if (ty <= 0) {
    const int nby_max = resident_warps / nbx > 1 ? resident_warps / nbx : 1;
    const int half = (v.n + 2 * nby_max - 1) / (2 * nby_max);
    ty = 2 * (half > 1 ? half : 1);
  }
  const int warps = nbx * ((v.n + ty - 1) / ty);
  pdl_launch(k_gs_strip_ring<S, RING, FU>, (warps + STRIP_WARPS - 1) / STRIP_WARPS, 32 * STRIP_WARPS, bytes, s,
             v, f, xin, xout, done, ty);
  count_launch();
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

template <typename S, bool FU>
static void gs_tile(const StencilView<float, S>& v, const float* f, const float* xin, float* xout, int shape,
                    const int* done, cudaStream_t s) {
  switch (shape) {
    case 1: strip_ring_launch<S, 6, FU>(v, f, xin, xout, done, s, 0); break;   // one wave, deeper rings
    case 2: strip_ring_launch<S, 8, FU>(v, f, xin, xout, done, s, 0); break;
    case 3: strip_ring_launch<S, 4, FU>(v, f, xin, xout, done, s, 32); break;
    case 4: strip_launch<S, 32, FU>(v, f, xin, xout, done, s); break;
    case 5: strip_launch<S, 16, FU>(v, f, xin, xout, done, s); break;
    default: strip_ring_launch<S, 4, FU>(v, f, xin, xout, done, s, 0); break;   // one wave
  }
}

template <typename S>
void launch_gs_tile(const StencilView<float, S>& v, const float* f, const float* xin, float* xout, int shape,
                    const int* done, cudaStream_t s) {
  const bool ring_ok = aligned16(f) && aligned16(xin) && v.pk && aligned16(v.pk);
  if (shape < 4 && !ring_ok) shape = 4;           // bulk copies need 16-byte aligned arrays and the packed stencil
  if (v.fused)
    gs_tile<S, true>(v, f, xin, xout, shape, done, s);
  else
    gs_tile<S, false>(v, f, xin, xout, shape, done, s);
}

// ty = 0: the smallest even height whose strips fit into one wave of the
// kernel's resident warps (occupancy x SMs x warps per CTA).
template <int RING, bool FU>
static void strip64_launch(const StencilView<double, double>& v, const double* f, const double* xin, double* xout,
                           const int* done, cudaStream_t s, int ty) {
  constexpr size_t bytes = (size_t)STRIP_WARPS * RING * STRIP64_SLOT;
  static const int resident_warps = resident_strip_warps(k_gs_strip64<RING, FU>, bytes);
  const int nbx = (v.n + 55) / 56;
  if (ty <= 0) {
    const int nby_max = resident_warps / nbx > 1 ? resident_warps / nbx : 1;
    const int half = (v.n + 2 * nby_max - 1) / (2 * nby_max);
    ty = 2 * (half > 1 ? half : 1);
  }
  const int warps = nbx * ((v.n + ty - 1) / ty);
  pdl_launch(k_gs_strip64<RING, FU>, (warps + STRIP_WARPS - 1) / STRIP_WARPS, 32 * STRIP_WARPS, bytes, s, v, f,
             xin, xout, done, ty);
  count_launch();
}

template <bool FU>
static void gs_tile64(const StencilView<double, double>& v, const double* f, const double* xin, double* xout,
                      int shape, const int* done, cudaStream_t s) {
  switch (shape) {
    case 1: strip64_launch<4, FU>(v, f, xin, xout, done, s, 16); break;
    case 2: strip64_launch<6, FU>(v, f, xin, xout, done, s, 0); break;
    case 3: strip64_launch<4, FU>(v, f, xin, xout, done, s, 8); break;
    default: strip64_launch<4, FU>(v, f, xin, xout, done, s, 0); break;
  }
}

void launch_gs_tile64(const StencilView<double, double>& v, const double* f, const double* xin, double* xout,
                      int shape, const int* done, cudaStream_t s) {
  if (v.fused)
    gs_tile64<true>(v, f, xin, xout, shape, done, s);
  else
    gs_tile64<false>(v, f, xin, xout, shape, done, s);
}

// One warp waits, through the same bounded wait as the bulk-copy sweep, on an
// mbarrier phase that nothing completes; the wait gives up and flags it.
__global__ void k_wait_selftest() {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncwarp();
  if (!mbar_wait(&bar, 0) && threadIdx.x == 0) atomicExch(&g_strip_timeout, 1);
}

void launch_wait_selftest(cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>();
  count_launch();
}

// ty = 0: the one-wave strip height, as strip_ring_launch.
template <typename S, int RING, bool FU>
static void strip2_launch(const StencilView<float, S>& v, const float* f, const float* xin, float* xout,
                          const int* done, cudaStream_t s, int ty) {
  constexpr size_t bytes = (size_t)STRIP_WARPS * RING * (StripRing<S>::SLOT + 8);
  static const int resident_warps = resident_strip_warps(k_gs_strip2_ring<S, RING, FU>, bytes);
  const int nbx = (v.n + 47) / 48;
  if (ty <= 0) {
    const int nby_max = resident_warps / nbx > 1 ? resident_warps / nbx : 1;
    const int half = (v.n + 2 * nby_max - 1) / (2 * nby_max);
    ty = 2 * (half > 1 ? half : 1);
  }
  const int warps = nbx * ((v.n + ty - 1) / ty);
  pdl_launch(k_gs_strip2_ring<S, RING, FU>, (warps + STRIP_WARPS - 1) / STRIP_WARPS, 32 * STRIP_WARPS, bytes, s,
             v, f, xin, xout, done, ty);
  count_launch();
}

template <typename S, bool FU>
static void gs_pair(const StencilView<float, S>& v, const float* f, const float* xin, float* xout, int shape,
                    const int* done, cudaStream_t s) {
  switch (shape) {
    case 1: strip2_launch<S, 6, FU>(v, f, xin, xout, done, s, 0); break;   // one wave, deeper rings
    case 2: strip2_launch<S, 8, FU>(v, f, xin, xout, done, s, 0); break;
    case 3: strip2_launch<S, 4, FU>(v, f, xin, xout, done, s, 26); break;
    default: strip2_launch<S, 4, FU>(v, f, xin, xout, done, s, 0); break;   // one wave
  }
}

// ty = 0: the one-wave strip height, as strip_ring_launch.
template <typename S, int RING, bool FU>
static void strip2r_launch(const StencilView<float, S>& v, const float* f, const float* xin, float* xout,
                           const float* ci, float* fc, float* xc, const int* done, cudaStream_t s) {
  constexpr size_t bytes = (size_t)STRIP_WARPS * RING * (StripRingR<S>::SLOT + 8);
  static const int resident_warps = resident_strip_warps(k_gs_strip2r_ring<S, RING, FU>, bytes);
  const int nbx = (v.n + 43) / 44;
  const int nby_max = resident_warps / nbx > 1 ? resident_warps / nbx : 1;
  const int half = (v.n + 2 * nby_max - 1) / (2 * nby_max);
  const int ty = 2 * (half > 1 ? half : 1);
  const int warps = nbx * ((v.n + ty - 1) / ty);
  pdl_launch(k_gs_strip2r_ring<S, RING, FU>, (warps + STRIP_WARPS - 1) / STRIP_WARPS, 32 * STRIP_WARPS, bytes, s,
             v, f, xin, xout, ci, fc, xc, done, ty);
  count_launch();
}

template <typename S>
bool launch_gs_pair_restrict(const StencilView<float, S>& v, const float* f, const float* xin, float* xout,
                             const float* ci, float* fc, float* xc, int shape, const int* done, cudaStream_t s) {
  if (!(aligned16(f) && aligned16(xin) && v.pk && aligned16(v.pk) && aligned16(v.O) && ci && fc && xc))
    return false;
  const bool deep = shape == 1;
  if (v.fused) {
    if (deep)
      strip2r_launch<S, 6, true>(v, f, xin, xout, ci, fc, xc, done, s);
    else
      strip2r_launch<S, 4, true>(v, f, xin, xout, ci, fc, xc, done, s);
  } else {
    if (deep)
      strip2r_launch<S, 6, false>(v, f, xin, xout, ci, fc, xc, done, s);
    else
      strip2r_launch<S, 4, false>(v, f, xin, xout, ci, fc, xc, done, s);
  }
  return true;
}
template bool launch_gs_pair_restrict<float>(const StencilView<float, float>&, const float*, const float*, float*,
                                             const float*, float*, float*, int, const int*, cudaStream_t);
template bool launch_gs_pair_restrict<__nv_bfloat16>(const StencilView<float, __nv_bfloat16>&, const float*,
                                                     const float*, float*, const float*, float*, float*, int,
                                                     const int*, cudaStream_t);

template <typename S>
bool launch_gs_pair(const StencilView<float, S>& v, const float* f, const float* xin, float* xout, int shape,
                    const int* done, cudaStream_t s) {
  if (!(aligned16(f) && aligned16(xin) && v.pk && aligned16(v.pk))) return false;
  if (v.fused)
    gs_pair<S, true>(v, f, xin, xout, shape, done, s);
  else
    gs_pair<S, false>(v, f, xin, xout, shape, done, s);
  return true;
}
template bool launch_gs_pair<float>(const StencilView<float, float>&, const float*, const float*, float*, int,
                                    const int*, cudaStream_t);
template bool launch_gs_pair<__nv_bfloat16>(const StencilView<float, __nv_bfloat16>&, const float*, const float*,
                                            float*, int, const int*, cudaStream_t);

int strip_timeouts() {
  int h = 0, zero = 0;
  cudaMemcpyFromSymbol(&h, g_strip_timeout, sizeof(int));
  if (h) cudaMemcpyToSymbol(g_strip_timeout, &zero, sizeof(int));
  return h;
}

template <typename T, typename S>
void launch_line(const StencilView<T, S>& v, int kind, const T* f, T* x, T* cp, int sweeps, int dir,
                 const int* done, cudaStream_t s) {
  constexpr int TPB = 64;
  for (int k = 0; k < sweeps; ++k)
    for (int axis = 0; axis <= 1; ++axis) {               // x-lines (rows), then y-lines (columns)
      if ((axis == 0 && dir == LINE_Y) || (axis == 1 && dir == LINE_X)) continue;
      for (int first = 1; first <= 2; ++first) {          // odd lines, then even lines
        const int lines = first == 1 ? (v.n + 1) / 2 : (v.n - 1) / 2;
        if (lines <= 0) continue;
        const unsigned g = (unsigned)((lines + TPB - 1) / TPB);
        if (axis == 0 && kind == 9)
          pdl_launch(k_line_rows<T, S, true>, g, TPB, 0, s, v, f, x, cp, first, done);
        else if (axis == 0)
          pdl_launch(k_line_rows<T, S, false>, g, TPB, 0, s, v, f, x, cp, first, done);
        else if (kind == 9)
          pdl_launch(k_line_cols<T, S, true>, g, TPB, 0, s, v, f, x, cp, first, done);
        else
          pdl_launch(k_line_cols<T, S, false>, g, TPB, 0, s, v, f, x, cp, first, done);
        count_launch();
      }
    }
}
template void launch_line<double, double>(const StencilView<double, double>&, int, const double*, double*, double*,
                                          int, int, const int*, cudaStream_t);
template void launch_line<float, float>(const StencilView<float, float>&, int, const float*, float*, float*, int,
                                        int, const int*, cudaStream_t);
template void launch_line<float, __nv_bfloat16>(const StencilView<float, __nv_bfloat16>&, int, const float*, float*,
                                                float*, int, int, const int*, cudaStream_t);

template <typename T>
void launch_interp_correct(int n, const T* ci, const T* ec, T* x, const int* done, cudaStream_t s, int fused) {
  launch_interp_to<T>(n, ci, ec, x, x, done, s, fused);
}

template <typename T>
void launch_interp_to(int n, const T* ci, const T* ec, const T* xin, T* xout, const int* done, cudaStream_t s,
                      int fused) {
  int nc = (n - 1) / 2;
  if (fused)
    pdl_launch(k_interp_correct<T, true>, grid2(nc + 1, nc + 1), dim3(BX, BY), 0, s, n, ci, ec, xin, xout, done);
  else
    pdl_launch(k_interp_correct<T, false>, grid2(nc + 1, nc + 1), dim3(BX, BY), 0, s, n, ci, ec, xin, xout, done);
  count_launch();
}

template <typename T, typename S>
int launch_residual(const StencilView<T, S>& v, int kind, const T* x, const T* f, T* r, double* partials,
                    const int* done, cudaStream_t s) {
  int g = norm_blocks(v.n);
  if (kind == 9 && v.fused)
    pdl_launch(k_residual<T, S, true, true>, g, NORM_THREADS, 0, s, v, x, f, r, partials, done);
  else if (kind == 9)
    pdl_launch(k_residual<T, S, true, false>, g, NORM_THREADS, 0, s, v, x, f, r, partials, done);
  else if (v.fused)
    pdl_launch(k_residual<T, S, false, true>, g, NORM_THREADS, 0, s, v, x, f, r, partials, done);
  else
    pdl_launch(k_residual<T, S, false, false>, g, NORM_THREADS, 0, s, v, x, f, r, partials, done);
  count_launch();
  return g;
}

template <typename T>
void launch_coarse_solve(int n, const double* L, const T* f, T* x, double* y, const int* done, cudaStream_t s) {
  pdl_launch(k_coarse_solve<T>, 1, 32, 0, s, n, L, f, x, y, done);
  count_launch();
}

void launch_norm_finalize(const double* partials, int np, void* ctl, int phase, double* out, cudaStream_t s) {
  pdl_launch(k_norm_finalize, 1, NORM_THREADS, 0, s, partials, np, (Ctl*)ctl, phase, out);
  count_launch();
}

void launch_ir_update(int n, double* x, const float* e32, void* ctl, cudaStream_t s) {
  pdl_launch(k_ir_update, grid2((n + IRU_COLS - 1) / IRU_COLS, n), dim3(BX, BY), 0, s, n, x, e32, (const Ctl*)ctl);
  count_launch();
}

int launch_ir_residual(const StencilView<double, double>& v, int kind, const double* x, const double* f, float* r32,
                       float* e32_zero, double* partials, void* ctl, cudaStream_t s) {
  int g = norm_blocks(v.n);
  if (v.fused)
    pdl_launch(k_ir_residual<true>, g, NORM_THREADS, 0, s, v, kind == 9, x, f, r32, e32_zero, partials, (Ctl*)ctl);
  else
    pdl_launch(k_ir_residual<false>, g, NORM_THREADS, 0, s, v, kind == 9, x, f, r32, e32_zero, partials, (Ctl*)ctl);
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
  template void launch_gs<T, S>(const StencilView<T, S>&, int, const T*, T*, int, const int*, cudaStream_t, int);    \
  template void launch_resid_restrict<T, S>(const StencilView<T, S>&, int, const T*, const T*, const T*, T*, T*, \
                                            const int*, cudaStream_t);                                          \
  template int launch_residual<T, S>(const StencilView<T, S>&, int, const T*, const T*, T*, double*, const int*, \
                                     cudaStream_t);
BMG_INST(double, double)
BMG_INST(float, float)
BMG_INST(float, __nv_bfloat16)
#undef BMG_INST
template void launch_interp_correct<double>(int, const double*, const double*, double*, const int*, cudaStream_t,
                                            int);
template void launch_interp_correct<float>(int, const float*, const float*, float*, const int*, cudaStream_t, int);
template void launch_gs_tile<float>(const StencilView<float, float>&, const float*, const float*, float*, int,
                                    const int*, cudaStream_t);
template void launch_gs_tile<__nv_bfloat16>(const StencilView<float, __nv_bfloat16>&, const float*, const float*,
                                            float*, int, const int*, cudaStream_t);
template void launch_interp_to<double>(int, const double*, const double*, const double*, double*, const int*,
                                       cudaStream_t, int);
template void launch_interp_to<float>(int, const float*, const float*, const float*, float*, const int*,
                                      cudaStream_t, int);
template void launch_coarse_solve<double>(int, const double*, const double*, double*, double*, const int*,
                                          cudaStream_t);
template void launch_coarse_solve<float>(int, const double*, const float*, float*, double*, const int*,
                                         cudaStream_t);
template int rows_cluster<double>(int);
template int rows_cluster<float>(int);

}  // namespace bmg

// ==== flexible conjugate gradients ======================================================
// Notay's FCG(1) with the V-cycle as preconditioner, FP64 outer loop:
//   z = M r; p = z (first step) or z + beta p with beta = -(z.q)/(p.q)_previous;
//   q = A p; alpha = (p.r)/(p.q); x += alpha p; r -= alpha q.
// Every inner product uses the reduction order of k_residual / k_norm_finalize.
namespace bmg {
using namespace dev;
namespace {

constexpr int FBX = 32, FBY = 8;

__device__ __forceinline__ double zval(const double* z, const float* z32, double s, size_t p) {
  return z32 ? pow2_times_widened(s, z32[p]) : z[p];   // s * fl64(z32) is exact: s is a power of two
}

// FCG_COLS columns of a row per thread iteration (NORM_THREADS apart): their
// loads are issued together, and the running sum still takes the columns in
// the canonical order.
constexpr int FCG_COLS = 4;

template <bool FU>
__global__ void __launch_bounds__(NORM_THREADS) k_fcg_zq(int n, const double* __restrict__ z,
                                                         const float* __restrict__ z32, const double* __restrict__ q,
                                                         double* __restrict__ partials, const Ctl* ctl) {
  pdl_enter();
  if (ctl->done) return;
  const double s = ctl->scale_applied;
  const int ld = n + 2;
  double acc = 0.0;
  for (int j = 1 + blockIdx.x; j <= n; j += gridDim.x)
    for (int i = 1 + threadIdx.x; i <= n; i += NORM_THREADS * FCG_COLS) {
      double zv[FCG_COLS], qv[FCG_COLS];
#pragma unroll
      for (int c = 0; c < FCG_COLS; ++c) {
        const size_t p = (size_t)j * ld + i + c * NORM_THREADS;
        if (i + c * NORM_THREADS <= n) {
          zv[c] = zval(z, z32, s, p);
          qv[c] = q[p];
        }
      }
#pragma unroll
      for (int c = 0; c < FCG_COLS; ++c)
        if (i + c * NORM_THREADS <= n) acc = madd<FU>(acc, zv[c], qv[c]);
    }
  double tot = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

__device__ __forceinline__ double reduce_partials(const double* partials, int np) {
  double acc = 0.0;
  for (int k = threadIdx.x; k < np; k += NORM_THREADS) acc = __dadd_rn(acc, partials[k]);
  return block_sum(acc);
}

// slot 0: zq; slot 1: pq and pr (second partial array right after the first)
__global__ void __launch_bounds__(NORM_THREADS) k_fcg_reduce(const double* __restrict__ partials, int np, Ctl* ctl,
                                                             int which) {
  pdl_enter();
  if (ctl->done) return;
  if (which == 0) {
    double v = reduce_partials(partials, np);
    if (threadIdx.x == 0) {
      ctl->zq = v;
      if (!ctl->first) ctl->beta = -rdiv(v, ctl->pq_prev);   // one division per step, not per point
    }
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

// FCG_COLS points of a row per thread, FBX apart, every load before the first store
template <bool FU>
__global__ void k_fcg_direction(int n, const double* __restrict__ z, const float* __restrict__ z32,
                                double* __restrict__ pv, const Ctl* ctl) {
  pdl_enter();
  if (ctl->done) return;
  const int i0 = blockIdx.x * (FBX * FCG_COLS) + threadIdx.x + 1, j = blockIdx.y * blockDim.y + threadIdx.y + 1;
  if (j > n) return;
  const double s = ctl->scale_applied, beta = ctl->beta;
  const bool first = ctl->first;
  double zp[FCG_COLS], pp[FCG_COLS];
#pragma unroll
  for (int c = 0; c < FCG_COLS; ++c) {
    const size_t p = (size_t)j * (n + 2) + i0 + c * FBX;
    if (i0 + c * FBX <= n) {
      zp[c] = zval(z, z32, s, p);
      pp[c] = first ? 0.0 : pv[p];
    }
  }
#pragma unroll
  for (int c = 0; c < FCG_COLS; ++c) {
    const size_t p = (size_t)j * (n + 2) + i0 + c * FBX;
    if (i0 + c * FBX <= n && BMG_IN(DBG_REFINE_STORE, p, (size_t)(n + 2) * (n + 2)))
      pv[p] = first ? zp[c] : madd<FU>(zp[c], beta, pp[c]);
  }
}

// q = A p (row sum a_O p + a_W p_W + ... in canonical order), partial p.q and p.r
template <bool FU>
__global__ void __launch_bounds__(NORM_THREADS) k_fcg_matvec(StencilView<double, double> v, int nine,
                                                             const double* __restrict__ pv, const double* __restrict__ r,
                                                             double* __restrict__ q, double* __restrict__ partials,
                                                             const Ctl* ctl) {
  pdl_enter();
  if (ctl->done) return;
  const int n = v.n, ld = v.ld;
  double apq = 0.0, apr = 0.0;
  for (int j = 1 + blockIdx.x; j <= n; j += gridDim.x)
    for (int i = 1 + threadIdx.x; i <= n; i += NORM_THREADS) {
      size_t p = (size_t)j * ld + i;
      double acc = rmul(v.O[p], pv[p]);
      acc = madd<FU>(acc, v.W[p], pv[p - 1]);
      acc = madd<FU>(acc, v.W[p + 1], pv[p + 1]);
      acc = madd<FU>(acc, v.S_[p], pv[p - ld]);
      acc = madd<FU>(acc, v.S_[p + ld], pv[p + ld]);
      if (nine) {
        acc = madd<FU>(acc, v.SW[p], pv[p - ld - 1]);
        acc = madd<FU>(acc, v.SW[p + ld + 1], pv[p + ld + 1]);
        acc = madd<FU>(acc, v.NW[p], pv[p + ld - 1]);
        acc = madd<FU>(acc, v.NW[p + 1 - ld], pv[p + 1 - ld]);
      }
      if (BMG_IN(DBG_REFINE_STORE, p, (size_t)(n + 2) * ld)) q[p] = acc;
      apq = madd<FU>(apq, pv[p], acc);
      apr = madd<FU>(apr, pv[p], r[p]);
    }
  double t1 = block_sum(apq);
  __syncthreads();
  double t2 = block_sum(apr);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = t1;
    partials[NORM_BLOCKS_MAX + blockIdx.x] = t2;
  }
}

// x += alpha p, r -= alpha q, partial r.r; zero the preconditioner output and,
// in mixed precision, write r32 = fl32(r / scale_next).
template <bool FU>
__global__ void __launch_bounds__(NORM_THREADS) k_fcg_update(int n, double* __restrict__ x, double* __restrict__ r,
                                                             const double* __restrict__ pv,
                                                             const double* __restrict__ q, float* __restrict__ r32,
                                                             float* __restrict__ z32, double* __restrict__ z,
                                                             double* __restrict__ partials, Ctl* ctl) {
  pdl_enter();
  if (ctl->done) return;
  const int ld = n + 2;
  const double alpha = rdiv(ctl->pr, ctl->pq);
  const double s = ctl->scale_next;
  const double inv = 1.0 / s;
  double acc = 0.0;
  for (int j = 1 + blockIdx.x; j <= n; j += gridDim.x)
    for (int i = 1 + threadIdx.x; i <= n; i += NORM_THREADS * FCG_COLS) {
      double xv[FCG_COLS], rv[FCG_COLS], pw[FCG_COLS], qv[FCG_COLS];
#pragma unroll
      for (int c = 0; c < FCG_COLS; ++c) {
        const size_t p = (size_t)j * ld + i + c * NORM_THREADS;
        if (i + c * NORM_THREADS <= n) {
          xv[c] = x[p];
          rv[c] = r[p];
          pw[c] = pv[p];
          qv[c] = q[p];
        }
      }
#pragma unroll
      for (int c = 0; c < FCG_COLS; ++c) {
        const size_t p = (size_t)j * ld + i + c * NORM_THREADS;
        if (i + c * NORM_THREADS > n || !BMG_IN(DBG_REFINE_STORE, p, (size_t)(n + 2) * ld)) continue;
        x[p] = madd<FU>(xv[c], alpha, pw[c]);
        const double rr = msub<FU>(rv[c], alpha, qv[c]);
        r[p] = rr;
        if (r32) {
          r32[p] = __double2float_rn(rmul(rr, inv));
          z32[p] = 0.0f;
        } else {
          z[p] = 0.0;
        }
        acc = madd<FU>(acc, rr, rr);
      }
    }
  double tot = block_sum(acc);
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
template <bool FU>
__global__ void __launch_bounds__(NORM_THREADS) k_fcg_init(StencilView<double, double> v, int nine,
                                                           const double* __restrict__ x, const double* __restrict__ f,
                                                           double* __restrict__ r, double* __restrict__ z,
                                                           float* __restrict__ r32, float* __restrict__ z32,
                                                           double* __restrict__ partials, Ctl* ctl) {
  pdl_enter();
  const int n = v.n, ld = v.ld;
  const double s = ctl->scale_next;
  const double inv = 1.0 / s;
  double acc = 0.0;
  for (int j = 1 + blockIdx.x; j <= n; j += gridDim.x)
    for (int i = 1 + threadIdx.x; i <= n; i += NORM_THREADS) {
      size_t p = (size_t)j * ld + i;
      double rr = nine ? row_residual<double, double, true, true, FU>(v, x, p, f[p])
                       : row_residual<double, double, false, true, FU>(v, x, p, f[p]);
      if (!BMG_IN(DBG_REFINE_STORE, p, (size_t)(n + 2) * ld)) continue;
      r[p] = rr;
      if (r32) {
        r32[p] = __double2float_rn(rmul(rr, inv));
        z32[p] = 0.0f;
      } else {
        z[p] = 0.0;
      }
      acc = madd<FU>(acc, rr, rr);
    }
  double tot = block_sum(acc);
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
  if (v.fused)
    pdl_launch(k_fcg_init<true>, g, NORM_THREADS, 0, s, v, kind == 9, x, f, r, z, r32, z32, partials, (Ctl*)ctl);
  else
    pdl_launch(k_fcg_init<false>, g, NORM_THREADS, 0, s, v, kind == 9, x, f, r, z, r32, z32, partials, (Ctl*)ctl);
  count_launch();
  return g;
}

// One FCG step after the preconditioner: z.q, beta and p, q = A p with p.q and
// p.r, then the x / r update with r.r partials (finalised by the caller).
// `mark(arg, k)` (may be NULL) brackets the sub-steps for profiling.
template <bool FU>
static void fcg_step(const StencilView<double, double>& v, int kind, double* x, double* r, const double* z,
                     const float* z32, double* pv, double* q, float* r32, float* z32_zero, double* z_zero,
                     double* partials, void* ctl, cudaStream_t s, void (*mark)(void*, int), void* mark_arg) {
  const int n = v.n;
  int g = norm_blocks(n);
  Ctl* c = (Ctl*)ctl;
  if (mark) mark(mark_arg, 0);
  pdl_launch(k_fcg_zq<FU>, g, NORM_THREADS, 0, s, n, z, z32, q, partials, c);
  count_launch();
  pdl_launch(k_fcg_reduce, 1, NORM_THREADS, 0, s, partials, g, c, 0);
  count_launch();
  pdl_launch(k_fcg_direction<FU>, dim3((n + FBX * FCG_COLS - 1) / (FBX * FCG_COLS), (n + FBY - 1) / FBY),
             dim3(FBX, FBY), 0, s, n, z, z32, pv, c);
  count_launch();
  if (mark) mark(mark_arg, 1);
  pdl_launch(k_fcg_matvec<FU>, g, NORM_THREADS, 0, s, v, kind == 9, pv, r, q, partials, c);
  count_launch();
  pdl_launch(k_fcg_reduce, 1, NORM_THREADS, 0, s, partials, g, c, 1);
  count_launch();
  if (mark) mark(mark_arg, 2);
  pdl_launch(k_fcg_update<FU>, g, NORM_THREADS, 0, s, n, x, r, pv, q, r32, z32_zero, z_zero, partials, c);
  count_launch();
  if (mark) mark(mark_arg, 3);
}

void launch_fcg_reduce(const double* partials, int np, void* ctl, int which, cudaStream_t s) {
  pdl_launch(k_fcg_reduce, 1, NORM_THREADS, 0, s, partials, np, (Ctl*)ctl, which);
  count_launch();
}

void launch_fcg_step(const StencilView<double, double>& v, int kind, double* x, double* r, const double* z,
                     const float* z32, double* pv, double* q, float* r32, float* z32_zero, double* z_zero,
                     double* partials, void* ctl, cudaStream_t s, void (*mark)(void*, int), void* mark_arg) {
  if (v.fused)
    fcg_step<true>(v, kind, x, r, z, z32, pv, q, r32, z32_zero, z_zero, partials, ctl, s, mark, mark_arg);
  else
    fcg_step<false>(v, kind, x, r, z, z32, pv, q, r32, z32_zero, z_zero, partials, ctl, s, mark, mark_arg);
}

}  // namespace bmg
